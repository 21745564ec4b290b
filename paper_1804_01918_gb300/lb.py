"""Python binding of the D2Q37 C ABI (include/lb_d2q37.h): argument marshalling only.

Every step of the time step runs in the CUDA library liblb_d2q37.so; this module only converts
arguments. PyTorch supplies the device memory (the context workspace is a torch CUDA tensor)
and the stream (torch's current stream unless one is given). If the library is missing the
import fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

NPOP = 37
LB_FP64, LB_FP32DEV, LB_FP32SPLIT = 0, 1, 2

_STATUS = {0: "LB_OK", 1: "LB_ERR_ARG", 2: "LB_ERR_ALLOC", 3: "LB_ERR_CUDA",
           4: "LB_ERR_NONFINITE", 5: "LB_ERR_STATE", 6: "LB_ERR_RANGE"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblb_d2q37.so")


class LBError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {_STATUS.get(status, status)}"
        if status == 3:
            msg += f" ({last_error()})"
        super().__init__(msg)


class NonFiniteError(LBError):
    pass


class lb_params(C.Structure):
    _fields_ = [("Lx", C.c_int), ("Ly", C.c_int), ("tau", C.c_double), ("gx", C.c_double),
                ("gy", C.c_double), ("T_top", C.c_double), ("T_bottom", C.c_double),
                ("y_periodic", C.c_int), ("precision", C.c_int), ("wall_mode", C.c_int),
                ("stream", C.c_void_p),
                ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t)]


class lb_ensemble_opts(C.Structure):
    _fields_ = [("tile_x", C.c_int), ("tile_y", C.c_int), ("graph_steps", C.c_int),
                ("precision", C.c_int), ("stream", C.c_void_p), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t), ("per_item", C.c_int)]


_lib = None


def lib() -> C.CDLL:
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.lb_status_str.restype = C.c_char_p
        L.lb_status_str.argtypes = [C.c_int]
        L.lb_last_error.restype = C.c_char_p
        L.lb_velocity_set.argtypes = [ip, ip, dp, dp]
        L.lb_workspace_bytes.argtypes = [C.POINTER(lb_params), C.POINTER(C.c_size_t)]
        L.lb_init.argtypes = [C.POINTER(lb_params), vp, vp, vp, vp, C.POINTER(vp)]
        L.lb_step.argtypes = [vp, C.c_int]
        L.lb_propagate.argtypes = [vp]
        L.lb_collide.argtypes = [vp]
        L.lb_set_staging.argtypes = [vp, C.c_int]
        L.lb_sync.argtypes = [vp]
        L.lb_moments.argtypes = [vp, vp, vp, vp, vp]
        L.lb_moments_half_step.argtypes = [vp, vp, vp, vp, vp]
        L.lb_rt_fields.argtypes = [C.c_int, C.c_int, C.c_double, C.c_uint64, vp, vp, vp, vp, vp, vp, vp]
        L.lb_init_rt.argtypes = [C.POINTER(lb_params), C.c_double, C.c_uint64, C.POINTER(vp)]
        L.lb_ensemble_init_rt.argtypes = [C.c_int, C.POINTER(lb_params), vp, vp, C.POINTER(lb_ensemble_opts),
                                          C.POINTER(vp)]
        L.lb_collide_train.argtypes = [vp, vp, vp, C.c_size_t, C.c_int, C.c_uint64]
        L.lb_collide_save.argtypes = [vp, C.c_char_p]
        L.lb_collide_load.argtypes = [vp, C.c_char_p]
        L.lb_moments_device.argtypes = [vp, vp, vp, vp, vp]
        L.lb_get_populations.argtypes = [vp, vp]
        L.lb_set_populations.argtypes = [vp, vp]
        L.lb_steps_done.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.lb_free.argtypes = [vp]
        L.lb_free.restype = None
        L.lb_probe_fma.argtypes = [C.c_int, vp, C.c_int, C.c_int, C.c_int, vp]
        L.lb_probe_wait.argtypes = [C.c_ulonglong, C.c_int, vp, vp]
        L.lb_moments_noalloc.argtypes = [C.POINTER(lb_params), vp, vp, vp, vp, vp]
        PP = C.POINTER(C.c_void_p)
        L.lb_ensemble_workspace_bytes.argtypes = [C.c_int, C.POINTER(lb_params),
                                                  C.POINTER(lb_ensemble_opts), C.POINTER(C.c_size_t)]
        L.lb_ensemble_init.argtypes = [C.c_int, C.POINTER(lb_params), PP, PP, PP, PP,
                                       C.POINTER(lb_ensemble_opts), C.POINTER(vp)]
        L.lb_ensemble_step.argtypes = [vp, C.c_int]
        L.lb_ensemble_sync.argtypes = [vp]
        L.lb_ensemble_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                           C.POINTER(C.c_double)]
        L.lb_ensemble_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_int), C.POINTER(C.c_longlong)]
        L.lb_ensemble_moments.argtypes = [vp, C.c_int, vp, vp, vp, vp]
        L.lb_ensemble_get_populations.argtypes = [vp, C.c_int, vp]
        L.lb_ensemble_free.argtypes = [vp]
        L.lb_ensemble_free.restype = None
        fp = C.POINTER(C.c_float)
        L.lb_mlp_create.argtypes = [C.c_uint64, C.POINTER(vp)]
        L.lb_mlp_free.argtypes = [vp]
        L.lb_mlp_free.restype = None
        L.lb_mlp_get_params.argtypes = [vp, vp, vp]
        L.lb_mlp_set_params.argtypes = [vp, vp, vp]
        L.lb_mlp_eval.argtypes = [vp, vp, vp, C.c_int, vp]
        L.lb_mlp_loss_grad.argtypes = [vp, vp, vp, C.c_int, C.POINTER(C.c_double), vp, vp]
        L.lb_mlp_loss_grad_fp32.argtypes = [vp, vp, vp, C.c_int, C.POINTER(C.c_double), vp, vp]
        L.lb_mlp_train.argtypes = [vp, vp, vp, C.c_longlong, C.c_int, C.c_int, C.c_float, C.c_uint64,
                                   vp, vp]
        L.lb_collect_pairs.argtypes = [vp, vp, C.c_int, vp, vp]
        L.lb_set_collide_learned.argtypes = [vp, vp, C.c_double, C.c_int]
        L.lb_set_collide_plain.argtypes = [vp]
        L.lb_learned_stats.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                       C.POINTER(C.c_double)]
        L.lb_learned_tiles.argtypes = [vp, vp, C.c_int]
        L.lb_init_slab.argtypes = [C.POINTER(lb_params), C.c_int, vp, vp, vp, vp, C.POINTER(vp)]
        L.lb_slab_step.argtypes = [vp, C.c_int]
        L.lb_slab_pack.argtypes = [vp, C.c_int, vp]
        L.lb_slab_unpack.argtypes = [vp, C.c_int, vp]
        L.lb_slab_exchange.argtypes = [vp, vp]
        _lib = L
    return _lib


def last_error() -> str:
    return lib().lb_last_error().decode()


class RangeError(LBError):
    pass


def check(status: int, where: str) -> None:
    if status == 4:
        raise NonFiniteError(status, where)
    if status == 6:
        raise RangeError(status, where)
    if status != 0:
        raise LBError(status, where)


def velocity_set():
    """(cx[37], cy[37], w[37], r) in the library's population order."""
    cx = np.zeros(NPOP, np.int32)
    cy = np.zeros(NPOP, np.int32)
    w = np.zeros(NPOP, np.float64)
    r = C.c_double()
    check(lib().lb_velocity_set(cx.ctypes.data_as(C.POINTER(C.c_int)),
                                cy.ctypes.data_as(C.POINTER(C.c_int)),
                                w.ctypes.data_as(C.POINTER(C.c_double)), C.byref(r)),
          "lb_velocity_set")
    return cx, cy, w, r.value


def _precision_code(p) -> int:
    if p in (LB_FP64, "fp64", "f64"):
        return LB_FP64
    if p in (LB_FP32DEV, "fp32dev", "fp32"):
        return LB_FP32DEV
    if p in (LB_FP32SPLIT, "fp32split"):
        return LB_FP32SPLIT
    raise ValueError(f"unknown precision {p!r}")


WALL_MODES = {"rest": 0, "mirror": 1}


def _wall_code(m) -> int:
    if isinstance(m, int):
        return m  # validated by the library
    if m in WALL_MODES:
        return WALL_MODES[m]
    raise ValueError(f"unknown wall mode {m!r}")


def make_params(Lx, Ly, tau, gx=0.0, gy=0.0, T_top=1.0, T_bottom=1.0, y_periodic=False,
                precision=LB_FP64, stream=None, workspace=0, workspace_bytes=0,
                wall_mode="rest") -> lb_params:
    return lb_params(int(Lx), int(Ly), float(tau), float(gx), float(gy), float(T_top),
                     float(T_bottom), int(bool(y_periodic)), _precision_code(precision),
                     _wall_code(wall_mode), stream, workspace, workspace_bytes)


def workspace_bytes(Lx, Ly, precision=LB_FP64) -> int:
    p = make_params(Lx, Ly, 1.0, precision=precision)
    n = C.c_size_t()
    check(lib().lb_workspace_bytes(C.byref(p), C.byref(n)), "lb_workspace_bytes")
    return n.value


def _ptr(a) -> int:
    """Address of a C-contiguous numpy array or a torch tensor."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _host_f64(a, shape):
    if hasattr(a, "data_ptr"):
        assert a.dtype.__str__() == "torch.float64" and a.is_contiguous() and tuple(a.shape) == shape
        return a
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if arr.shape != shape:
        arr = np.ascontiguousarray(np.broadcast_to(arr, shape))
    return arr


def rt_fields(Lx: int, Ly: int, R: float = 2.0, seed: int = 0):
    """The library's seeded Rayleigh-Taylor fields (lb_rt_fields, host only) as an
    inputs.RTFields."""
    from .inputs import RTFields
    out = [np.empty((Ly, Lx), np.float64) for _ in range(4)]
    tt, tb, gy = C.c_double(), C.c_double(), C.c_double()
    check(lib().lb_rt_fields(int(Lx), int(Ly), float(R), int(seed) & ((1 << 64) - 1),
                             *[o.ctypes.data for o in out], C.byref(tt), C.byref(tb), C.byref(gy)),
          "lb_rt_fields")
    return RTFields(rho=out[0], ux=out[1], uy=out[2], T=out[3], T_top=tt.value, T_bottom=tb.value,
                    gy=gy.value)


@dataclass
class Lattice:
    """One D2Q37 lattice on the GPU (wraps an lb_ctx).

    fields: host arrays (rho, ux, uy, T), each [Ly][Lx] float64 (numpy or pinned torch tensors).
    The workspace is a torch uint8 CUDA tensor unless ``own_memory`` asks the library to allocate.
    Work runs on ``stream`` (a torch.cuda.Stream; a new one if None); torch work that reads the
    outputs of moments_device must run on, or wait for, that stream.
    """

    Lx: int
    Ly: int
    tau: float
    rho: object
    ux: object
    uy: object
    T: object
    gx: float = 0.0
    gy: float = 0.0
    T_top: float = 1.0
    T_bottom: float = 1.0
    y_periodic: bool = False
    precision: object = LB_FP64
    stream: object = None
    own_memory: bool = False
    wall_mode: object = "rest"
    rt_ratio: object = None  # set (with rt_seed) to initialise through lb_init_rt instead of fields
    rt_seed: int = 0
    cuts: int = 0            # a slab of a larger lattice (include/lb_slab.h): bit 0 cut below, bit 1 above

    def __post_init__(self):
        import torch
        self._ctx = C.c_void_p()
        shape = (self.Ly, self.Lx)
        fields = (None if self.rt_ratio is not None else
                  [_host_f64(v, shape) for v in (self.rho, self.ux, self.uy, self.T)])
        prec = _precision_code(self.precision)
        if self.stream is None:
            # a stream of its own: the legacy default stream cannot be captured into a CUDA graph
            self.stream = torch.cuda.Stream()
        sh = self.stream.cuda_stream if hasattr(self.stream, "cuda_stream") else self.stream
        nbytes = workspace_bytes(self.Lx, self.Ly, prec)
        self._ws = None
        ws_ptr = 0
        if not self.own_memory:
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            ws_ptr = self._ws.data_ptr()
        self._params = make_params(self.Lx, self.Ly, self.tau, self.gx, self.gy, self.T_top,
                                   self.T_bottom, self.y_periodic, prec, sh, ws_ptr,
                                   nbytes if ws_ptr else 0, wall_mode=self.wall_mode)
        if self.cuts:
            check(lib().lb_init_slab(C.byref(self._params), int(self.cuts), *[_ptr(f) for f in fields],
                                     C.byref(self._ctx)), "lb_init_slab")
        elif fields is None:
            check(lib().lb_init_rt(C.byref(self._params), float(self.rt_ratio),
                                   int(self.rt_seed) & ((1 << 64) - 1), C.byref(self._ctx)), "lb_init_rt")
            R = float(self.rt_ratio)
            self.T_top, self.T_bottom = 2.0 / (1.0 + R), 2.0 * R / (1.0 + R)
            self.gy = -0.1 * self.T_top / self.Ly
        else:
            check(lib().lb_init(C.byref(self._params), *[_ptr(f) for f in fields], C.byref(self._ctx)),
                  "lb_init")
        self.rho = self.ux = self.uy = self.T = None  # the context holds its own copy

    @classmethod
    def from_fields(cls, fields, tau, **kw):
        """Build from an inputs.RTFields (walls and gravity taken from it)."""
        kw.setdefault("gy", fields.gy)
        kw.setdefault("T_top", fields.T_top)
        kw.setdefault("T_bottom", fields.T_bottom)
        Ly, Lx = fields.rho.shape
        return cls(Lx, Ly, tau, fields.rho, fields.ux, fields.uy, fields.T, **kw)

    @classmethod
    def rayleigh_taylor(cls, Lx, Ly, tau, R=2.0, seed=0, **kw):
        """A lattice initialised by lb_init_rt (the library's seeded Rayleigh-Taylor fields)."""
        return cls(Lx, Ly, tau, None, None, None, None, rt_ratio=R, rt_seed=seed, **kw)

    def collide_train(self, pre, post, epochs: int = 20, seed: int = 0) -> None:
        """lb_collide_train on device pairs pre/post (torch float32 [n, 37])."""
        check(lib().lb_collide_train(self._ctx, pre.data_ptr(), post.data_ptr(), int(pre.shape[0]),
                                     int(epochs), int(seed) & ((1 << 64) - 1)), "lb_collide_train")

    def collide_save(self, path: str) -> None:
        check(lib().lb_collide_save(self._ctx, os.fsencode(path)), "lb_collide_save")

    def collide_load(self, path: str) -> None:
        check(lib().lb_collide_load(self._ctx, os.fsencode(path)), "lb_collide_load")

    @property
    def sites(self) -> int:
        return self.Lx * self.Ly

    def step(self, n: int = 1) -> None:
        check(lib().lb_step(self._ctx, int(n)), "lb_step")

    def propagate(self) -> None:
        check(lib().lb_propagate(self._ctx), "lb_propagate")

    def set_staging(self, use_tma: bool) -> None:
        """FP32-split steps: TMA-staged pulls (default where available) or plain loads."""
        check(lib().lb_set_staging(self._ctx, int(bool(use_tma))), "lb_set_staging")

    def collide(self) -> None:
        """Collide in place (FP64): lb_propagate + lb_collide = one fused step."""
        check(lib().lb_collide(self._ctx), "lb_collide")

    def sync(self) -> None:
        check(lib().lb_sync(self._ctx), "lb_sync")

    def moments(self, out=None):
        """(rho, ux, uy, T) as host float64 arrays [Ly][Lx] (or into the given host buffers)."""
        if out is None:
            out = tuple(np.empty((self.Ly, self.Lx), np.float64) for _ in range(4))
        check(lib().lb_moments(self._ctx, *[_ptr(o) if o is not None else None for o in out]),
              "lb_moments")
        return out

    def moments_half_step(self, out=None):
        """Half-step fields (rho, u - g/2, T + |g|^2/8) of the current post-collision state as host
        float64 arrays [Ly][Lx] (lb_moments_half_step)."""
        if out is None:
            out = tuple(np.empty((self.Ly, self.Lx), np.float64) for _ in range(4))
        check(lib().lb_moments_half_step(self._ctx, *[_ptr(o) if o is not None else None for o in out]),
              "lb_moments_half_step")
        return out

    def moments_device(self, out):
        """Write (rho, ux, uy, T) into 4 torch float64 CUDA tensors of Lx*Ly elements (async)."""
        check(lib().lb_moments_device(self._ctx, *[o.data_ptr() if o is not None else None for o in out]),
              "lb_moments_device")
        return out

    def get_populations(self) -> np.ndarray:
        f = np.empty((NPOP, self.Ly, self.Lx), np.float64)
        check(lib().lb_get_populations(self._ctx, f.ctypes.data), "lb_get_populations")
        return f

    def set_populations(self, f) -> None:
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (NPOP, self.Ly, self.Lx)
        check(lib().lb_set_populations(self._ctx, f.ctypes.data), "lb_set_populations")

    @property
    def steps_done(self) -> int:
        n = C.c_longlong()
        check(lib().lb_steps_done(self._ctx, C.byref(n)), "lb_steps_done")
        return n.value

    def collect_pairs(self, sites, pre, post) -> None:
        """Training pairs of the current state for the given site indices (torch int32 CUDA tensor
        of y * Lx + x) into torch float32 CUDA tensors pre, post of shape [n, 37] (async)."""
        n = int(sites.numel())
        check(lib().lb_collect_pairs(self._ctx, sites.data_ptr(), n, pre.data_ptr(), post.data_ptr()),
              "lb_collect_pairs")

    def set_collide_learned(self, net, bound: float = 1e-4, check_every: int = 1) -> None:
        self._net = net  # keep the network alive while it is in use
        check(lib().lb_set_collide_learned(self._ctx, net._ptr, float(bound), int(check_every)),
              "lb_set_collide_learned")

    def set_collide_plain(self) -> None:
        check(lib().lb_set_collide_plain(self._ctx), "lb_set_collide_plain")
        self._net = None

    def learned_stats(self):
        a, b, r = C.c_longlong(), C.c_longlong(), C.c_double()
        check(lib().lb_learned_stats(self._ctx, C.byref(a), C.byref(b), C.byref(r)), "lb_learned_stats")
        return {"tiles_checked": a.value, "tiles_fallback": b.value, "max_residual": r.value}

    def slab_step(self, part: int = 0) -> None:
        """One step of a slab (0 whole, 1 the rows next to its cuts, 2 the rest; lb_slab_step)."""
        check(lib().lb_slab_step(self._ctx, int(part)), "lb_slab_step")

    def slab_pack(self, side: int, buf) -> None:
        """The rows sent across side (0 below, 1 above) into a CUDA tensor of 26 x Lx elements."""
        check(lib().lb_slab_pack(self._ctx, int(side), buf.data_ptr()), "lb_slab_pack")

    def slab_unpack(self, side: int, buf) -> None:
        """The neighbour's packed rows into the ghost rows at side (0 below, 1 above)."""
        check(lib().lb_slab_unpack(self._ctx, int(side), buf.data_ptr()), "lb_slab_unpack")

    def learned_tiles(self) -> np.ndarray:
        """Per-tile decisions [Ly/32, Lx/32] (1 = fell back to the plain collide at the last check)."""
        out = np.zeros((self.Ly // 32, self.Lx // 32), np.uint8)
        check(lib().lb_learned_tiles(self._ctx, out.ctypes.data, int(out.size)), "lb_learned_tiles")
        return out

    def close(self) -> None:
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().lb_free(self._ctx)
            self._ctx = C.c_void_p()
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_NPARAM = 26149
MLP_TILE = 128


class MLP:
    """The learned collide's network (include/lb_learned.h), device-resident."""

    def __init__(self, seed: int = 0):
        self._ptr = C.c_void_p()
        check(lib().lb_mlp_create(C.c_uint64(seed), C.byref(self._ptr)), "lb_mlp_create")

    def get_params(self):
        p = np.empty(MLP_NPARAM, np.float32)
        nrm = np.empty((4, 37), np.float32)
        check(lib().lb_mlp_get_params(self._ptr, p.ctypes.data, nrm.ctypes.data), "lb_mlp_get_params")
        return p, nrm

    def set_params(self, params, norm=None) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == MLP_NPARAM
        nrm = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        check(lib().lb_mlp_set_params(self._ptr, p.ctypes.data, None if nrm is None else nrm.ctypes.data),
              "lb_mlp_set_params")

    def eval(self, x, y, stream=None) -> None:
        """y = network(x) for torch float32 CUDA tensors [n, 37], n a multiple of 128."""
        sh = None if stream is None else stream.cuda_stream
        check(lib().lb_mlp_eval(self._ptr, x.data_ptr(), y.data_ptr(), int(x.shape[0]), sh), "lb_mlp_eval")

    def loss_grad(self, x, t, stream=None):
        """(loss, gradient[NPARAM]) of the mean squared error on normalised inputs/targets."""
        sh = None if stream is None else stream.cuda_stream
        loss = C.c_double()
        g = np.empty(MLP_NPARAM, np.float32)
        check(lib().lb_mlp_loss_grad(self._ptr, x.data_ptr(), t.data_ptr(), int(x.shape[0]), C.byref(loss),
                                     g.ctypes.data, sh), "lb_mlp_loss_grad")
        return loss.value, g

    def loss_grad_fp32(self, x, t, stream=None):
        """The same in the library's FP32 debug mode (CUDA cores, no BF16 rounding)."""
        sh = None if stream is None else stream.cuda_stream
        loss = C.c_double()
        g = np.empty(MLP_NPARAM, np.float32)
        check(lib().lb_mlp_loss_grad_fp32(self._ptr, x.data_ptr(), t.data_ptr(), int(x.shape[0]),
                                          C.byref(loss), g.ctypes.data, sh), "lb_mlp_loss_grad_fp32")
        return loss.value, g

    def train(self, pre, post, epochs: int = 20, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
              stream=None):
        """Train on device pairs [n, 37]; returns the per-epoch mean losses."""
        sh = None if stream is None else stream.cuda_stream
        losses = np.zeros(epochs, np.float32)
        check(lib().lb_mlp_train(self._ptr, pre.data_ptr(), post.data_ptr(), int(pre.shape[0]), int(epochs),
                                 int(batch), float(lr), C.c_uint64(seed), losses.ctypes.data, sh),
              "lb_mlp_train")
        return losses

    def close(self) -> None:
        if getattr(self, "_ptr", None) and self._ptr.value:
            lib().lb_mlp_free(self._ptr)
            self._ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_fma(kind: str, blocks: int, threads: int, iters: int, out, stream=None) -> None:
    """Launch the FMA-throughput probe (kind 'fp64', 'fp32', or 'fp64_varying': FP64 chains whose
    operands keep changing) into the torch tensor `out`."""
    k = {"fp64": 0, "fp32": 1, "fp64_varying": 2}[kind]
    sh = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
    check(lib().lb_probe_fma(k, sh, blocks, threads, iters, out.data_ptr()), "lb_probe_fma")


def slab_exchange(lo: "Lattice", hi: "Lattice") -> None:
    """Ghost rows across the cut between slab lo (below) and slab hi (above), device to device."""
    check(lib().lb_slab_exchange(lo._ctx, hi._ctx), "lb_slab_exchange")


def probe_wait(limit_ns: int, arrive: bool, stream=None):
    """(gave_up, waited_ns) of the library's bounded barrier wait run alone (lb_probe_wait)."""
    import torch
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    sh = None if stream is None else stream.cuda_stream
    check(lib().lb_probe_wait(int(limit_ns), int(bool(arrive)), sh, out.data_ptr()), "lb_probe_wait")
    torch.cuda.synchronize()
    gave_up, ns = (int(v) for v in out.cpu())
    return bool(gave_up), ns


def moments_noalloc(Lx: int, Ly: int, f_device_ptr: int, precision=LB_FP64, stream=None):
    """(rho, ux, uy, T) host arrays of one caller-owned device population copy, computed without
    any device allocation (lb_moments_noalloc; at most LB_NOALLOC_MAX_SITES = 65536 sites)."""
    sh = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
    p = make_params(Lx, Ly, 1.0, precision=precision, stream=sh)
    out = tuple(np.empty((Ly, Lx), np.float64) for _ in range(4))
    check(lib().lb_moments_noalloc(C.byref(p), f_device_ptr, *[o.ctypes.data for o in out]),
          "lb_moments_noalloc")
    return out


class Ensemble:
    """Independent D2Q37 lattices advanced together by one launch per step
    (include/lb_ensemble.h). members: list of dicts with Lx, Ly, tau and optional gx, gy, T_top,
    T_bottom, y_periodic, plus host fields rho, ux, uy, T ([Ly][Lx] float64) -- or, for every
    member, a temperature ratio R and a seed instead of fields (lb_ensemble_init_rt)."""

    def __init__(self, members, precision="fp32split", tile=(0, 0), graph_steps=0, stream=None,
                 per_item=False):
        import torch
        self._ctx = C.c_void_p()
        n = len(members)
        self.members = [(int(m["Lx"]), int(m["Ly"])) for m in members]
        params = (lb_params * n)()
        keep = []
        ptrs = [(C.c_void_p * n)() for _ in range(4)]
        rt = all("rho" not in m and "R" in m for m in members)  # lb_ensemble_init_rt members
        for k, m in enumerate(members):
            params[k] = make_params(m["Lx"], m["Ly"], m["tau"], m.get("gx", 0.0), m.get("gy", 0.0),
                                    m.get("T_top", 1.0), m.get("T_bottom", 1.0),
                                    m.get("y_periodic", False), precision,
                                    wall_mode=m.get("wall_mode", "rest"))
            if rt:
                continue
            for j, key in enumerate(("rho", "ux", "uy", "T")):
                a = _host_f64(m[key], (int(m["Ly"]), int(m["Lx"])))
                keep.append(a)
                ptrs[j][k] = _ptr(a)
        self.stream = torch.cuda.Stream() if stream is None else stream
        sh = self.stream.cuda_stream if hasattr(self.stream, "cuda_stream") else self.stream
        opts = lb_ensemble_opts(int(tile[0]), int(tile[1]), int(graph_steps),
                                _precision_code(precision), sh, None, 0, int(bool(per_item)))
        nbytes = C.c_size_t()
        check(lib().lb_ensemble_workspace_bytes(n, params, C.byref(opts), C.byref(nbytes)),
              "lb_ensemble_workspace_bytes")
        self._ws = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
        opts.workspace = self._ws.data_ptr()
        opts.workspace_bytes = nbytes.value
        if rt:
            ratios = np.array([float(m["R"]) for m in members], np.float64)
            seeds = np.array([int(m.get("seed", 0)) & ((1 << 64) - 1) for m in members], np.uint64)
            check(lib().lb_ensemble_init_rt(n, params, ratios.ctypes.data, seeds.ctypes.data, C.byref(opts),
                                            C.byref(self._ctx)), "lb_ensemble_init_rt")
        else:
            check(lib().lb_ensemble_init(n, params, *ptrs, C.byref(opts), C.byref(self._ctx)),
                  "lb_ensemble_init")

    def step(self, n: int = 1) -> None:
        check(lib().lb_ensemble_step(self._ctx, int(n)), "lb_ensemble_step")

    def sync(self) -> None:
        check(lib().lb_ensemble_sync(self._ctx), "lb_ensemble_sync")

    def autotune(self, steps: int = 5):
        tx, ty, m = C.c_int(), C.c_int(), C.c_double()
        check(lib().lb_ensemble_autotune(self._ctx, int(steps), C.byref(tx), C.byref(ty), C.byref(m)),
              "lb_ensemble_autotune")
        return tx.value, ty.value, m.value

    def info(self):
        tx, ty, nt, ns = C.c_int(), C.c_int(), C.c_int(), C.c_longlong()
        check(lib().lb_ensemble_info(self._ctx, C.byref(tx), C.byref(ty), C.byref(nt), C.byref(ns)),
              "lb_ensemble_info")
        return {"tile": (tx.value, ty.value), "items": nt.value, "sites": ns.value}

    def moments(self, k: int):
        Lx, Ly = self.members[k]
        out = tuple(np.empty((Ly, Lx), np.float64) for _ in range(4))
        check(lib().lb_ensemble_moments(self._ctx, k, *[o.ctypes.data for o in out]),
              "lb_ensemble_moments")
        return out

    def get_populations(self, k: int) -> np.ndarray:
        Lx, Ly = self.members[k]
        f = np.empty((NPOP, Ly, Lx), np.float64)
        check(lib().lb_ensemble_get_populations(self._ctx, k, f.ctypes.data),
              "lb_ensemble_get_populations")
        return f

    def close(self) -> None:
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().lb_ensemble_free(self._ctx)
            self._ctx = C.c_void_p()
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
