"""Host logic of bench.py that needs no GPU: the validity of the profiled per-site constants, the
clock record and the energy window."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_code_digest_ignores_comments_but_not_code(tmp_path):
    b = load_bench()
    a = tmp_path / "a.cu"
    a.write_text("// header\n__global__ void k(float* x) { x[0] = 1.0f; /* store */ }\n")
    base = b.code_digest(str(a))
    a.write_text("// another header\n__global__ void k(float* x) {\n  x[0] = 1.0f; // store one\n}\n")
    assert b.code_digest(str(a)) == base
    a.write_text("// header\n__global__ void k(float* x) { x[0] = 2.0f; }\n")
    assert b.code_digest(str(a)) != base



def test_profiled_constants_match_the_kernel_sources():
    """The per-site FP64 instruction count and the DRAM traffic in bench.py were profiled on the
    current kernel code: a code change without a new profile fails here (the bench would report
    those figures as null)."""
    b = load_bench()
    assert b.sources_match({"sources": b.FP64_INST_SOURCES})
    assert b.sources_match(b.TRAFFIC_FP64)
    assert b.sources_match(b.TRAFFIC_FP32SPLIT)


def synthetic_samples():
    """(host time, SM MHz, max MHz, W, reasons): idle before 10.0 s, loaded 10.0-10.2 s, idle after."""
    s = [(9.0 + 0.02 * k, 1000.0, 2070.0, 170.0, []) for k in range(50)]
    s += [(10.0 + 0.02 * k, 2070.0 - k, 2070.0, 450.0 + k, ["sw_power_cap"] if k == 3 else [])
          for k in range(11)]
    s += [(10.3 + 0.02 * k, 990.0, 2070.0, 175.0, []) for k in range(20)]
    return s


def test_clock_record_uses_only_samples_inside_the_timed_region():
    b = load_bench()
    win = b.samples_in_window(synthetic_samples(), 10.0, 10.2)
    assert len(win) == 11 and all(10.0 <= s[0] <= 10.2 for s in win)
    rec = b.summarize_clocks(win, "test")
    assert rec["sm_mhz"] == 2065.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 11
    assert rec["power_w_median"] == 455.0 and rec["reasons"] == ["sw_power_cap"]
    assert b.summarize_clocks([], "test")["sm_mhz"] is None


def test_energy_window_arithmetic():
    b = load_bench()
    # 2 s windows at 7.68 ms per step: 261 steps
    assert b.energy_window_steps(7.68) == 261 and b.energy_window_steps(1e4) == 1
    sites = 2304 * 8192
    e = b.energy_from_counter(5_000_000, 5_900_000, 2.0, 250, sites)   # 900 J over 2 s
    assert e["power_w"] == 450.0 and e["joules_per_step"] == 3.6
    assert abs(e["nJ_per_site_update"] - 3.6 / sites * 1e9) < 1e-3
    assert b.energy_from_counter(None, 5, 1.0, 10, sites) is None
    assert b.energy_from_counter(7, 7, 1.0, 10, sites) is None       # counter did not move
    win = b.samples_in_window(synthetic_samples(), 10.0, 10.2)
    p = b.energy_from_power(win, 0.2, 26, sites)
    assert p["power_w"] == 455.0 and abs(p["joules_per_step"] - round(455.0 * 0.2 / 26, 4)) < 1e-12
