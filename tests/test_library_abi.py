"""CPU checks of the CUDA library: it loads, exports every entry point that
include/celes.h declares, and its compile-time (a5, b5) term tables (App. A.2)
equal the oracle's.  No GPU call is made."""

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import translation
from paper_1706_02145_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return binding.load()


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "celes.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(celes_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for required in ["celes_create", "celes_set_incident", "celes_coupling_matvec", "celes_master_matvec",
                     "celes_precond_build", "celes_precond_apply", "celes_solve", "celes_farfield",
                     "celes_get_coefficients", "celes_destroy", "celes_last_error"]:
        assert required in syms


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name
    bound = {s[0] for s in binding.SIGNATURES}
    assert set(_declared_symbols()) <= bound | {"celes_zz_unused"}


def test_version_string(lib):
    assert "sm_103a" in binding.celes_version()


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5])
def test_compile_time_terms_match_oracle(lib, L):
    idx, val = binding.celes_coupling_terms(L)
    rows = [(l, m) for l in range(1, L + 1) for m in range(-l, l + 1)]
    seen = set()
    for (ri, ro, p, mu, kind), v in zip(idx, val):
        lp, mp = rows[ri]
        l, m = rows[ro]
        assert mu == abs(mp - m) and abs(l - lp) <= p <= l + lp and p >= mu
        a5, b5 = translation.ab5(lp, mp, l, m, p)
        ref = a5.real if kind == 0 else b5.imag
        assert abs(v - ref) <= 1e-13 * max(1.0, abs(ref)), (L, ri, ro, p, kind)
        seen.add((ri, ro, p, kind))
    # no nonzero oracle term is missing
    for ri, (lp, mp) in enumerate(rows):
        for ro, (l, m) in enumerate(rows):
            for p in range(abs(l - lp), l + lp + 1):
                if p < abs(mp - m):
                    continue
                a5, b5 = translation.ab5(lp, mp, l, m, p)
                if abs(a5) > 1e-14:
                    assert (ri, ro, p, 0) in seen
                if abs(b5) > 1e-14:
                    assert (ri, ro, p, 1) in seen


def test_invalid_lmax_rejected(lib):
    assert lib.celes_coupling_terms(0, None, None, 0) == binding.CELES_EINVAL
    assert lib.celes_coupling_terms(6, None, None, 0) == binding.CELES_EINVAL


def test_create_rejects_bad_arguments_before_touching_a_gpu(lib):
    ctx = ctypes.c_void_p()
    pos = np.zeros((2, 3))
    rad = np.array([1.0, -1.0])
    ni = np.array([1.5, 0.0, 1.5, 0.0])
    dp = ctypes.POINTER(ctypes.c_double)
    code = lib.celes_create(ctypes.byref(ctx), 2, pos.ctypes.data_as(dp), rad.ctypes.data_as(dp),
                            ni.ctypes.data_as(dp), 1.0, 0.01, 3, None)
    assert code == binding.CELES_EINVAL
    rad = np.array([1.0, 1.0])
    code = lib.celes_create(ctypes.byref(ctx), 2, pos.ctypes.data_as(dp), rad.ctypes.data_as(dp),
                            ni.ctypes.data_as(dp), 1.0, 0.01, 9, None)
    assert code == binding.CELES_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built library every call raises."""
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "libceles_gb300.so"))
    with pytest.raises(RuntimeError, match="not built"):
        binding.load()
    with pytest.raises(RuntimeError, match="not built"):
        binding.celes_create(np.zeros((1, 3)), np.ones(1), np.full(1, 1.5 + 0j), 1.0, 0.01, 2)


def test_every_binding_signature_names_an_exported_symbol(lib):
    for name, _, _ in binding.SIGNATURES:
        assert hasattr(lib, name), name


def test_binding_checks_device_buffers_before_the_call():
    # the C ABI cannot see buffer sizes: the binding refuses tensors of the
    # wrong dtype, device, size or layout before any pointer is passed
    torch = pytest.importorskip("torch")
    N, L = 4, 2
    nmax = 2 * L * (L + 2)
    pos4 = torch.zeros((N, 4), dtype=torch.float64)
    x = torch.zeros((N, nmax), dtype=torch.complex128)
    for xx, prec in [(x, binding.CELES_FP64), (x.to(torch.complex64), binding.CELES_FP64),
                     (x, binding.CELES_FP32), (x[:2], binding.CELES_FP64)]:
        with pytest.raises(binding.CelesError) as e:
            binding.celes_coupling_matvec_noalloc(N, L, 0.01, pos4, xx, xx.clone(), precision=prec, check=False)
        assert e.value.code == binding.CELES_EINVAL
    with pytest.raises(binding.CelesError):
        binding._check_vec("x", torch.zeros((3, 8), dtype=torch.complex64).t(), 24, binding.CELES_FP32)
