"""The algorithmic flop count per site update, re-derived by instrumentation: the oracle's own
collide compiled with an operation-counting scalar type (oracle/count_collide_flops.cpp), compared
with the number frozen in the benchmark."""
import ast
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def frozen_count():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    for node in tree.body:
        if isinstance(node, ast.Assign) and any(getattr(t, "id", None) == "ORACLE_FLOP_PER_SITE"
                                                for t in node.targets):
            return ast.literal_eval(node.value)
    raise AssertionError("ORACLE_FLOP_PER_SITE not found")


def test_instrumented_oracle_collide_flops():
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    from oracle import build
    exe = build.build_counter()
    n = int(subprocess.run([exe], check=True, capture_output=True, text=True).stdout.strip())
    assert n == frozen_count()
    # sanity: per population ~60 flops of equilibrium, ~13 of moments, 3 of relaxation
    assert 37 * 60 < n < 37 * 90
