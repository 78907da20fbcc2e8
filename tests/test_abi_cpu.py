"""CPU-side checks of the C ABI: the library loads without a GPU, exports every
function declared in include/hypersara.h, and its host-only helpers agree with
the oracle's independently derived tables (Daubechies filters by a different
root finder; the Kaiser-Bessel fit against the kernel definition)."""

import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hypersara.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"HS_API\s+(?:hs_status|const char\*)\s+(hs_\w+)\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_1806_04596_gb300 import hypersara as hs
    return hs


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["hs_phi_fwd", "hs_phi_adj", "hs_psi_fwd", "hs_psi_adj", "hs_prox_l21",
                     "hs_prox_nuclear", "hs_proj_l2ball", "hs_pd_step", "hs_pd_solve"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.load()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(_declared()) == set(lib.EXPORTED)
    assert "sm_103a" in lib.version()


def test_library_is_built_for_sm103a_only():
    from paper_1806_04596_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("p", range(1, 9))
def test_library_daubechies_filters_match_oracle(lib, p):
    from oracle import wavelets
    np.testing.assert_allclose(lib.daubechies_lowpass(p), wavelets.daubechies_lowpass(p),
                               rtol=0, atol=5e-15)


def test_library_kb_fit_accuracy(lib):
    beta = np.pi * np.sqrt(35.2)
    # coefficients used by the FP32 (9) and FP64 (14) kernels
    assert lib.kb_poly_fit_error(beta, 9) < 1e-8
    assert lib.kb_poly_fit_error(beta, 14) < 2e-14


def test_host_argument_errors_without_gpu(lib):
    """Argument checks happen on the host before any device call."""
    L = lib.load()
    import ctypes as C
    h = C.c_void_p()
    off = np.array([0, 10], dtype=np.int64)
    st = L.hs_plan_create(C.byref(h), 12, 16, 1, off.ctypes.data_as(C.POINTER(C.c_int64)), None, None,
                          None, 2, 8, 0.0, 2, 0, 0, None)
    assert st == lib.HS_ERR_ARG
    assert b"powers of two" in L.hs_last_error()
    st = L.hs_plan_create(C.byref(h), 16, 16, 1, off.ctypes.data_as(C.POINTER(C.c_int64)), None, None,
                          None, 3, 8, 0.0, 2, 0, 0, None)
    assert st == lib.HS_ERR_ARG
    assert L.hs_phi_fwd(None, None, None, None) == lib.HS_ERR_ARG
    assert L.hs_pd_step(None, None) == lib.HS_ERR_ARG
    assert L.hs_plan_destroy(None) == lib.HS_OK


def test_static_l2ball_rejects_channel_counts_on_the_host(lib):
    """hs_proj_l2ball_static checks L against its fixed scratch before any CUDA call."""
    L = lib.load()
    for bad in (0, -1, lib.L2BALL_STATIC_MAX_L + 1):
        st = L.hs_proj_l2ball_static(bad, None, None, None, None, 0, 0, None, None, None)
        assert st == -1, (bad, st)
        assert "outside" in lib.last_error()
    st = L.hs_proj_l2ball_static(4, None, None, None, None, 0, 0, None, None, None)
    assert st == -1 and "null" in lib.last_error()


@pytest.mark.parametrize("terms,tol", [(9, 1e-8), (14, 2e-14)])
def test_kb_mirrored_pieces_evaluate_the_kernel(lib, terms, tol):
    """The gridding kernel evaluates the taps of a window as 4 mirrored pairs:
    piece 7 - m at s and piece m at s are E(s^2) + s O(s^2) and E(s^2) - s O(s^2)
    of piece 7 - m's even and odd coefficients. That needs the fit's pieces to
    be mirror images (the kernel is even, Sec. 2.1), and the pair form to give
    the kernel at both taps to the fit's accuracy (against the oracle's
    Kaiser-Bessel definition)."""
    from oracle import kaiser_bessel as kbo
    beta = kbo.kb_beta(8, 2.0)
    c = lib.kb_poly_coefs(beta, terms)
    sign = (-1.0) ** np.arange(terms)
    for p in range(8):
        # equal up to the rounding of the conversion to monomials (1e-13 to 1e-11 of the largest)
        np.testing.assert_allclose(c[7 - p], sign * c[p], rtol=0, atol=1e-10 * np.abs(c).max())
    peak = kbo.kb(np.array([0.0]), 8, beta)[0]
    f = np.linspace(0.0, 1.0, 1001, endpoint=False)
    s = 2.0 * f - 1.0
    s2 = s * s
    for m in range(4):
        ce, co = c[7 - m][0::2], c[7 - m][1::2]
        E = np.polynomial.polynomial.polyval(s2, ce)
        O = np.polynomial.polynomial.polyval(s2, co)
        # window tap m of a window whose start cell is 3 below the cell of the
        # sample at fraction f: distance m - 3 - f, i.e. piece 7 - m at s; tap 7 - m at 4 - m - f
        tap_m = kbo.kb(m - 3 - f, 8, beta)
        tap_mirror = kbo.kb(4 - m - f, 8, beta)
        assert np.max(np.abs(E + s * O - tap_m)) <= tol * peak
        assert np.max(np.abs(E - s * O - tap_mirror)) <= tol * peak
