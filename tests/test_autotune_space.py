"""The autotuner's search space per block size and precision (host logic)."""
import paper_1402_6081_gb300 as lgfm
from paper_1402_6081_gb300 import autotune


def test_search_space():
    d16 = dict(autotune.candidates(16, lgfm.LGF_FP32))
    assert d16["fft_size_interval"] == [0, 34, 36] and d16["fft_kernel"] == [0, 2]
    assert d16["symmetric_spectra"] == [0, 1] and d16["mac_groups_per_cta"] == [0, 8, 32, 128]
    d64 = dict(autotune.candidates(10, lgfm.LGF_FP64))
    assert "fft_kernel" not in d64 and "free_sms" not in d64 and d64["interval_kernel"] == [0, 1]
    # the run-time-size block sizes: only the persistent-or-not product choice
    # and the SMs left to the levels >= 2 chain remain
    d20 = dict(autotune.candidates(20, lgfm.LGF_FP32))
    assert d20 == {"interval_kernel": [0, 1], "free_sms": [0, -1, 8, 16, 32]}
    assert dict(autotune.candidates(32, lgfm.LGF_FP64)) == {"interval_kernel": [0, 1]}
