"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
entry point that include/nmf.h declares, and its cycle schedules agree with the oracle."""
import os
import re

import pytest

from conftest import ROOT
from oracle import nmf_oracle as o
from paper_1009_0881_gb300 import native, synth


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "nmf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?(nmf_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1009_0881_gb300 import build
    build.build()
    return native.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("nmf_create", "nmf_solve", "nmf_error", "nmf_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert names
    for name in names:
        assert hasattr(lib, name), name
    # and the binding knows every one of them
    bound = {s[0] for s in native.SIGNATURES}
    assert set(names) <= bound


def test_exports_via_nm(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", native.library_path()], capture_output=True, text=True).stdout
    for name in _declared_functions():
        assert re.search(rf"\bT {name}$", out, flags=re.M), name


@pytest.mark.parametrize("cycle", ["vcycle", "ni", "fmg", "wcycle"])
@pytest.mark.parametrize("L,K", [(1, 10), (2, 100), (3, 100), (3, 500), (4, 37), (5, 8)])
def test_schedule_matches_oracle(lib, cycle, L, K):
    # the library's cycle schedule is integer host logic: bit-exact with the oracle's recursion
    counts = [0] * L
    trace = []
    orig = dict(o.SWEEPS)
    o.SWEEPS["count"] = lambda M, V, W: (V, W)
    try:
        p = synth.make_problem(32, 32, 2, 1)
        o.solve(p.M, 32, 32, p.V, p.W, "count", levels=L, K=K, cycle=cycle, trace=trace)
    finally:
        o.SWEEPS.clear()
        o.SWEEPS.update(orig)
    for level, _ in trace:
        counts[level - 1] += 1
    assert native.schedule(cycle, L, K) == counts


def test_schedule_rejects_bad_arguments(lib):
    with pytest.raises(native.NMFError):
        native.schedule("vcycle", 0, 10)
    with pytest.raises(native.NMFError):
        native.schedule("vcycle", 3, -1)


def test_create_without_gpu_reports_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes
    h = ctypes.c_void_p()
    rc = lib.nmf_create(ctypes.byref(h), 0, 0, 0)
    assert rc == -4 and not h.value
    assert lib.nmf_last_error(None) == b"invalid handle"
