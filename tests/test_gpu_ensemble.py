"""GPU checks of the batched ensemble (include/lb_ensemble.h).

No site depends on another within a step (Sec. 3), so the schedule -- one persistent launch
walking a tile list over all members -- must not change any result: every member must equal,
bit for bit, the same lattice advanced alone by lb_step with the same precision.
"""
import numpy as np
import pytest

from paper_1804_01918_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01918_gb300 import build, lb
    build.build()
    return lb


def member_specs():
    """Uneven sizes (ragged against every tile shape), different tau, gravity and walls."""
    specs = []
    for k, (Lx, Ly, tau, R) in enumerate([(96, 40, 0.7, 2.0), (64, 256, 0.9, 1.5), (130, 52, 1.1, 3.0),
                                          (33, 17, 0.62, 1.2)]):
        st = inputs.rayleigh_taylor(Lx, Ly, R=R, seed=k)
        specs.append({"Lx": Lx, "Ly": Ly, "tau": tau, "gy": st.gy * 3, "T_top": st.T_top,
                      "T_bottom": st.T_bottom, "rho": st.rho, "ux": st.ux, "uy": st.uy, "T": st.T})
    return specs


def single_runs(L, specs, steps, precision):
    out = []
    for m in specs:
        lat = L.Lattice(m["Lx"], m["Ly"], m["tau"], m["rho"], m["ux"], m["uy"], m["T"], gy=m["gy"],
                        T_top=m["T_top"], T_bottom=m["T_bottom"], precision=precision)
        lat.step(steps)
        out.append(lat.get_populations())
        lat.close()
    return out


@pytest.mark.parametrize("per_item", [False, True])
@pytest.mark.parametrize("precision", ["fp32split", "fp32dev"])
def test_ensemble_members_equal_single_lattice_runs(L, precision, per_item):
    """Both launch shapes (a persistent grid claiming the work items; one block per item) give
    every member the single-lattice result bit for bit."""
    specs = member_specs()
    ens = L.Ensemble(specs, precision=precision, graph_steps=10, per_item=per_item)
    ens.step(25)                      # two 10-step graph replays + 5 single launches
    ens.sync()
    want = single_runs(L, specs, 25, precision)
    for k in range(len(specs)):
        assert np.array_equal(ens.get_populations(k), want[k]), k
    ens.close()


def test_ensemble_autotune_keeps_state_and_results(L):
    specs = member_specs()
    ens = L.Ensemble(specs, precision="fp32split", graph_steps=6)
    ens.step(3)
    before = [ens.get_populations(k) for k in range(len(specs))]
    tx, ty, mlups = ens.autotune(steps=2)
    assert tx * ty >= 128 and mlups > 0
    assert ens.info()["tile"] == (tx, ty)
    for k in range(len(specs)):
        assert np.array_equal(ens.get_populations(k), before[k])
    ens.step(9)
    want = single_runs(L, specs, 12, "fp32split")
    for k in range(len(specs)):
        assert np.array_equal(ens.get_populations(k), want[k])
    ens.close()


@pytest.mark.parametrize("tile", [(32, 4), (256, 1), (64, 16)])
def test_ensemble_any_tile_shape_gives_the_same_result(L, tile):
    specs = member_specs()[:2]
    ens = L.Ensemble(specs, precision="fp32split", tile=tile)
    ens.step(7)
    want = single_runs(L, specs, 7, "fp32split")
    for k in range(len(specs)):
        assert np.array_equal(ens.get_populations(k), want[k])
    ens.close()


def test_ensemble_moments_and_seed_drawn_members(L, orc):
    """Eight seed-drawn members (sizes 32..128 x 4 Lx, Atwood 0.05..0.5, tau 0.6..1.2): the
    ensemble's density and temperature stay within the FP32 error budget of the FP64 oracle."""
    descs = inputs.ensemble_members(8, seed=3, lx_min=32, lx_max=128, lx_multiple=32)
    specs = []
    for d in descs:
        st = inputs.rayleigh_taylor(d["Lx"], d["Ly"], R=d["R"], seed=d["seed"])
        specs.append({"Lx": d["Lx"], "Ly": d["Ly"], "tau": d["tau"], "gy": st.gy,
                      "T_top": st.T_top, "T_bottom": st.T_bottom, "rho": st.rho, "ux": st.ux,
                      "uy": st.uy, "T": st.T, "_st": st})
    ens = L.Ensemble(specs, precision="fp32split", graph_steps=20)
    ens.step(40)
    ens.sync()
    for k, m in enumerate(specs):
        st = m["_st"]
        f = orc.run(orc.init_fields(st), tau=m["tau"], nsteps=40, gy=st.gy, T_top=st.T_top,
                    T_bottom=st.T_bottom)
        orho, _, _, oT = orc.moments(f)
        rho, _, _, T = ens.moments(k)
        assert np.linalg.norm(rho - orho) / np.linalg.norm(orho) < 40 * 37 * 2.0**-24 * 0.35
        assert np.linalg.norm(T - oT) / np.linalg.norm(oT) < 40 * 37 * 2.0**-24 * 0.35
    ens.close()


def test_bench_ensemble_64_members_equal_single_lattice_runs(L):
    """The bench's ensemble (64 seed-drawn members, 96 M sites, FP32 split, autotuned tile,
    100-step graphs) in its launch configuration: sampled members -- the smallest, the largest
    and two others -- equal, bit for bit, the same lattices advanced alone."""
    descs = inputs.ensemble_members(64, seed=0)
    specs = []
    for d in descs:
        st = inputs.rayleigh_taylor(d["Lx"], d["Ly"], R=d["R"], seed=d["seed"])
        specs.append({"Lx": d["Lx"], "Ly": d["Ly"], "tau": d["tau"], "gy": st.gy,
                      "T_top": st.T_top, "T_bottom": st.T_bottom, "rho": st.rho, "ux": st.ux,
                      "uy": st.uy, "T": st.T})
    sizes = [d["Lx"] * d["Ly"] for d in descs]
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 42})
    ens = L.Ensemble(specs, precision="fp32split", graph_steps=100)
    ens.autotune(steps=3)
    ens.step(103)                     # one 100-step graph replay + 3 single launches
    ens.sync()
    assert ens.info()["sites"] == sum(sizes)
    got = {k: ens.get_populations(k) for k in pick}
    ens.close()
    want = single_runs(L, [specs[k] for k in pick], 103, "fp32split")
    for k, w in zip(pick, want):
        assert np.array_equal(got[k], w), k
