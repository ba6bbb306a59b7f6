"""The FFT convolution of isolated blocks in one kernel (lgf_conv_blocks,
the "FFT Conv." special case of Sec. 4.2): against the exact direct sum of
each block alone, and bit for bit against the three-launch form
(lgf_solve_blocks_noalloc), which runs the same arithmetic in the same order
with its spectra in device memory."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
from oracle import direct
from paper_1402_6081_gb300 import build as lgf_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    lgfm.library()


@pytest.mark.parametrize("n_b", [4, 8, 16])
@pytest.mark.parametrize("prec", [lgfm.LGF_FP32, lgfm.LGF_FP64])
def test_conv_blocks(n_b, prec):
    dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
    rng = np.random.default_rng(40 + n_b)
    nblk = 37                                     # several CTAs and a ragged last one
    f = rng.uniform(-1.0, 1.0, size=(nblk, n_b, n_b, n_b))
    ft = torch.from_numpy(f).to(dt).cuda()
    u = torch.empty_like(ft)
    lgfm.lgf_conv_blocks(ft, u, nblk, n_b, prec)
    u3 = torch.empty_like(ft)
    lgfm.lgf_solve_blocks_noalloc(ft, u3, nblk, n_b, prec)
    # in place
    ui = ft.clone()
    lgfm.lgf_conv_blocks(ui, ui, nblk, n_b, prec)
    torch.cuda.synchronize()
    got = u.double().cpu().numpy()
    assert np.array_equal(got, u3.double().cpu().numpy())
    assert torch.equal(ui, u)
    one = np.array([[0, 0, 0]], dtype=np.int32)
    tol = 1e-13 if prec == lgfm.LGF_FP64 else 1e-6
    for b in (0, 17, nblk - 1):
        ud = direct.direct_sum(one, n_b, f[b:b + 1])
        assert np.abs(got[b] - ud[0]).max() <= tol * np.abs(ud).max(), b


def test_conv_blocks_errors():
    f = torch.zeros(4 * 8 ** 3, dtype=torch.float32, device="cuda")
    for args, status in (((f, f[8:], 3, 8, lgfm.LGF_FP32), 1),      # partial overlap
                         ((f, f, 0, 8, lgfm.LGF_FP32), 1),          # no blocks
                         ((f, f, 1, 6, lgfm.LGF_FP32), 2),          # block size without the kernel
                         ((f, f, 1, 8, 7), 1)):                     # precision
        with pytest.raises(lgfm.LgfError) as e:
            lgfm.lgf_conv_blocks(*args)
        assert e.value.status == status, args
