"""The C-ABI library: exported symbols and argument validation (CPU only:
every call below is rejected before any CUDA work)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hm():
    from paper_1806_11558_gb300 import build
    build.build()
    import paper_1806_11558_gb300 as hm
    return hm


def test_header_symbols_exported(hm):
    hdr = open(os.path.join(ROOT, "include", "hm.h")).read()
    declared = set(re.findall(r"HM_API\s+[\w\s\*]*?\b(hm_\w+)\s*\(", hdr))
    assert declared == set(hm.EXPORTED)
    L = hm.lib()
    for name in declared:
        assert hasattr(L, name), name


def test_invalid_arguments_rejected(hm):
    L = hm.lib()
    out = ctypes.c_void_p(1)
    fake = ctypes.c_void_p(64)
    p = hm.TreeParams(1.5, 64)
    assert L.hm_build_tree(None, 10, fake, 4, ctypes.byref(p), None, ctypes.byref(out)) == hm.HM_EINVAL
    assert out.value is None
    assert L.hm_build_tree(fake, 10, fake, 0, ctypes.byref(p), None, ctypes.byref(out)) == hm.HM_EINVAL
    assert L.hm_build_tree(fake, 2, fake, 4, ctypes.byref(p), None, ctypes.byref(out)) == hm.HM_EINVAL
    for bad in (hm.TreeParams(-1.0, 64), hm.TreeParams(1.5, 0), hm.TreeParams(1.5, 255),
                hm.TreeParams(float("nan"), 64)):
        assert L.hm_build_tree(fake, 10, fake, 4, ctypes.byref(bad), None, ctypes.byref(out)) == hm.HM_EINVAL
    assert "leaf_size" in hm.hm_last_error() or "eta" in hm.hm_last_error()
    # handles that are not handles
    ap = hm.AssembleParams(1e-6, 64, 8, 0, 0)
    junk = (ctypes.c_uint32 * 16)()
    assert L.hm_assemble(ctypes.cast(junk, ctypes.c_void_p), ctypes.byref(ap), None, ctypes.byref(out)) == hm.HM_EINVAL
    assert L.hm_assemble(None, ctypes.byref(ap), None, ctypes.byref(out)) == hm.HM_EINVAL
    assert L.hm_matvec(None, 0, 1, 0, fake, fake, 1.0, 0.0, None) == hm.HM_EINVAL
    sp = hm.SolveParams(30, 100, 1e-10, 0, 1, 1e-4, 1, 0)
    assert L.hm_solve(None, 0, 1, fake, fake, ctypes.byref(sp), None, None) == hm.HM_EINVAL
    hm.hm_free(None)


def test_binding_fails_loudly_without_library(hm, monkeypatch, tmp_path):
    monkeypatch.setattr(hm, "_lib", None)
    monkeypatch.setattr(hm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        hm.lib()


def test_injected_allocation_failure_on_the_host(hm):
    """hm_set_fault_injection(1): the first device allocation of the next call
    fails before any CUDA call is made, so the call returns HM_ENOMEM (here,
    without a GPU, and on one); the injection disarms itself."""
    L = hm.lib()
    out = ctypes.c_void_p(1)
    fake = ctypes.c_void_p(64)
    p = hm.TreeParams(1.5, 64)
    hm.hm_set_fault_injection(1)
    try:
        assert L.hm_build_tree(fake, 10, fake, 4, ctypes.byref(p), None, ctypes.byref(out)) == hm.HM_ENOMEM
        assert out.value is None
        assert "injected allocation failure (allocation 1" in hm.hm_last_error()
    finally:
        hm.hm_set_fault_injection(0)
    # the wait limit is a host-side setting: any value is accepted, < 0 restores the default
    hm.hm_set_wait_limit(0)
    hm.hm_set_wait_limit(-1)


def test_fault_injection_from_the_environment(hm):
    code = ("import ctypes, paper_1806_11558_gb300 as hm; L = hm.lib(); f = ctypes.c_void_p(64); "
            "o = ctypes.c_void_p(); p = hm.TreeParams(1.5, 64); "
            "print(L.hm_build_tree(f, 10, f, 4, ctypes.byref(p), None, ctypes.byref(o)))")
    env = dict(os.environ, HM_FAULT_INJECT="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == str(hm.HM_ENOMEM)
