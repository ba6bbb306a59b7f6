"""The C-ABI library loads and exports every entry point include/lgf.h
declares; its host-side pieces (FP64 LGF generator, interpolation stencils)
agree with the independently written oracle.  No GPU needed."""
import pathlib
import re

import numpy as np
import pytest

import paper_1402_6081_gb300 as lgfm
from paper_1402_6081_gb300 import build as lgf_build
from oracle import fmm, lgf

ROOT = pathlib.Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    lgf_build.build()
    return lgfm.library()


def declared_symbols():
    text = (ROOT / "include" / "lgf.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lgf_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 13
    for s in syms:
        assert hasattr(lib, s), s
    # and the binding wraps each under the same name
    for s in syms:
        assert callable(getattr(lgfm, s)), s


def test_green_values_match_oracle(lib):
    pts = np.array([[0, 0, 0], [1, 0, 0], [2, 3, 4], [10, 0, 0], [64, 64, 64], [100, 3, 7],
                    [512, 512, 512], [0, 0, 512], [-3, 5, -300], [7, 128, 31], [40, 80, 120]])
    a = lgfm.lgf_green_values(pts)
    b = lgf.lgf(pts)
    assert np.all(np.abs(a - b) <= 5e-15 * np.abs(b))


def test_green_table_box_matches_oracle(lib):
    r = np.arange(0, 33)
    a, b, c = np.meshgrid(r, r, r, indexing="ij")
    pts = np.stack([a, b, c], -1).reshape(-1, 3) * 2
    got = lgfm.lgf_green_values(pts)
    ref = lgf.lgf(pts)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 5e-15


@pytest.mark.parametrize("n_b,n_max", [(4, 5), (4, 3), (8, 7), (8, 9), (16, 9), (16, 10), (16, 1)])
def test_interp_weights_match_oracle(lib, n_b, n_max):
    assert np.array_equal(lgfm.lgf_interp_weights(n_b, n_max), fmm.interp_weights(n_b, n_max))


def test_invalid_arguments_raise(lib):
    with pytest.raises(lgfm.LgfError):
        lgfm.lgf_interp_weights(8, 11)
