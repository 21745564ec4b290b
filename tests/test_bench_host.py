"""Host logic of bench.py that needs no GPU: the validity check of the stored DRAM traffic."""
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

