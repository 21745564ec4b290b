"""GPU checks of the seeded Rayleigh-Taylor initialisations (lb_init_rt, lb_ensemble_init_rt)
and of the context-owned learned collide (lb_collide_train / save / load)."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32split"])
def test_init_rt_equals_init_with_the_generated_fields(L, precision):
    a = L.Lattice.rayleigh_taylor(64, 96, 0.9, R=2.5, seed=11, precision=precision)
    st = L.rt_fields(64, 96, 2.5, 11)
    b = L.Lattice.from_fields(st, tau=0.9, precision=precision)
    assert np.array_equal(a.get_populations(), b.get_populations())
    a.step(9)
    b.step(9)
    assert np.array_equal(a.get_populations(), b.get_populations())


def test_init_rt_run_matches_the_oracle(L, orc):
    """100 FP64 steps from lb_init_rt against the oracle started from the inputs module's fields of
    the same recipe and generator (equal to the library's up to last-place rounding)."""
    lat = L.Lattice.rayleigh_taylor(64, 256, 0.9, R=2.0, seed=3)
    lat.step(100)
    lat.sync()
    cx, cy, _, _ = L.velocity_set()
    got = orc.from_planes(lat.get_populations(), cx, cy)
    st = inputs.rayleigh_taylor_splitmix(64, 256, 2.0, 3)
    want = orc.run(orc.init_fields(st), tau=0.9, nsteps=100, gy=st.gy, T_top=st.T_top,
                   T_bottom=st.T_bottom)
    assert float(np.max(np.abs(got - want) / np.abs(want))) <= 1e-12


def test_ensemble_init_rt_members_equal_single_lattices(L):
    specs = [{"Lx": 64, "Ly": 128, "tau": 0.8, "R": 1.5, "seed": 1},
             {"Lx": 96, "Ly": 64, "tau": 1.0, "R": 3.0, "seed": 2},
             {"Lx": 33, "Ly": 40, "tau": 0.7, "R": 2.0, "seed": 3}]
    ens = L.Ensemble(specs, precision="fp32split", graph_steps=4)
    ens.step(13)                      # three 4-step graph replays + 1 single launch
    ens.sync()
    for k, m in enumerate(specs):
        lat = L.Lattice.rayleigh_taylor(m["Lx"], m["Ly"], m["tau"], R=m["R"], seed=m["seed"],
                                        precision="fp32split")
        lat.step(13)
        assert np.array_equal(ens.get_populations(k), lat.get_populations()), k
        lat.close()
    ens.close()


def pairs(L, lat, steps=6):
    import torch
    n = lat.Lx * lat.Ly
    sites = torch.arange(n, dtype=torch.int32, device="cuda")
    pre, post = [], []
    for _ in range(steps):
        a = torch.empty((n, 37), dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        with torch.cuda.stream(lat.stream):
            lat.collect_pairs(sites, a, b)
        lat.step(1)
        pre.append(a)
        post.append(b)
    lat.sync()
    return torch.cat(pre), torch.cat(post)


def test_collide_train_save_load_round_trip(L, tmp_path):
    src = L.Lattice.rayleigh_taylor(64, 128, 0.9, R=2.0, seed=5, precision="fp32split")
    pre, post = pairs(L, src)
    src.close()
    a = L.Lattice.rayleigh_taylor(64, 128, 0.9, R=2.0, seed=6, precision="fp32split")
    b = L.Lattice.rayleigh_taylor(64, 128, 0.9, R=2.0, seed=6, precision="fp32split")
    with pytest.raises(L.LBError):
        a.collide_save(str(tmp_path / "none.bin"))   # no learned collide yet
    a.collide_train(pre, post, epochs=2, seed=4)
    path = str(tmp_path / "collide.bin")
    a.collide_save(path)
    b.collide_load(path)
    a.step(6)
    b.step(6)
    assert np.array_equal(a.get_populations(), b.get_populations())
    assert a.learned_stats() == b.learned_stats()
    # foreign or missing files are rejected and leave the context usable
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a network file" * 10)
    with pytest.raises(L.LBError):
        b.collide_load(str(bad))
    with pytest.raises(L.LBError):
        b.collide_load(str(tmp_path / "missing.bin"))
    b.step(1)
    b.sync()
    # FP64 contexts have no learned collide
    c = L.Lattice.rayleigh_taylor(64, 128, 0.9, R=2.0, seed=6)
    with pytest.raises(L.LBError):
        c.collide_train(pre, post, epochs=1)
    for lat in (a, b, c):
        lat.close()
