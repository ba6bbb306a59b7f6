"""The interpolation-parameter choice of Sec. 2.5: the oracle against values
the mathematics and the paper fix, then the library's host routine against
the oracle.  No GPU needed."""
import numpy as np
import pytest

from oracle import fmm
from oracle import select as osel


# Classical Lebesgue constants of n equally spaced nodes (degree n - 1):
# 1 (linear), 5/4 (quadratic, attained between the first two nodes), and the
# tabulated 1.6311 (cubic), 2.2078 (quartic).
@pytest.mark.parametrize("n,lam", [(2, 1.0), (3, 1.25), (4, 1.6311), (5, 2.2078)])
def test_lebesgue_constants_classical(n, lam):
    assert abs(osel.lebesgue_equispaced(n) - lam) <= 1e-4 * lam


def test_lebesgue_grows_exponentially():
    # equispaced Lebesgue constants roughly double per added node at large n
    r = osel.lebesgue_equispaced(14) / osel.lebesgue_equispaced(13)
    assert 1.6 < r < 2.2


def test_paper_example_fp64_eps_1p25e_12_gives_n_max_10():
    # Sec. 2.5: a relative tolerance of 1.25e-12 in double precision in 3D
    # requires n_max <= 10
    n_max, lam = osel.step1_n_max(1.25e-12, "fp64")
    assert n_max == 10
    assert lam ** 3 * 2.0 ** -53 < 1.25e-12 <= osel.lebesgue_equispaced(11) ** 3 * 2.0 ** -53


def test_step2_exact_for_polynomials():
    # the interpolation step reproduces polynomials of degree < n_max exactly,
    # so its error on G comes from G's non-polynomial part only: it falls with n_b
    e8 = osel.far_field_interp_error(8, 5)
    e16 = osel.far_field_interp_error(16, 5)
    assert 0 < e16 < e8 < 1e-2
    W = fmm.interp_weights(8, 5)
    F = np.fromfunction(lambda z, y, x: (1 + x) ** 2 * (2 + y) * (3 + z) ** 3, (9, 9, 9))
    v = fmm.interp(W, (1, 0, 1), F)
    xs = 4 + 0.5 * np.arange(9)
    ys = 0.5 * np.arange(9)
    exact = np.fromfunction(lambda k, j, i: (1 + xs[i]) ** 2 * (2 + ys[j]) * (3 + xs[k]) ** 3, (9, 9, 9), dtype=int)
    assert np.abs(v - exact).max() <= 1e-9 * np.abs(exact).max()


@pytest.fixture(scope="module")
def lib():
    import paper_1402_6081_gb300 as lgfm
    from paper_1402_6081_gb300 import build as lgf_build
    lgf_build.build()
    lgfm.library()
    return lgfm


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 10, 11, 14])
def test_library_lebesgue_matches_oracle(lib, n):
    assert abs(lib.lgf_lebesgue_constant(n) - osel.lebesgue_equispaced(n)) <= 1e-6 * osel.lebesgue_equispaced(n)


@pytest.mark.parametrize("eps,prec", [(1e-5, "fp32"), (3e-6, "fp32"), (1e-7, "fp64"), (1.25e-12, "fp64")])
def test_library_selection_matches_oracle(lib, eps, prec):
    got = lib.lgf_select_interp(eps, lib.LGF_FP64 if prec == "fp64" else lib.LGF_FP32)
    ref = osel.select(eps, prec)
    assert got["n_max"] == ref["n_max"] and got["n_b"] == ref["n_b"] and got["reached"] == ref["reached"]
    assert abs(got["lebesgue"] - ref["lebesgue"]) <= 1e-6 * ref["lebesgue"]
    # both sides sum FP64 products in different orders; interpolation with
    # n_max nodes amplifies those roundings by up to Lambda^3 (the very bound
    # of step 1)
    slack = 4.0 * ref["lebesgue"] ** 3 * 2.0 ** -53
    assert abs(got["interp_err"] - ref["interp_err"]) <= 1e-6 * ref["interp_err"] + slack
