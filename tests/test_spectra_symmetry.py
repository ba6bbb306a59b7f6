"""The reflection identity behind the reduced kernel tables (Sec. 3.2, last
paragraph), checked on the oracle's own kernel vectors and numpy's FFT: the
spectrum of offset d equals its representative's (|dx|, min(|dy|,|dz|),
max(|dy|,|dz|)) at the frequency with the axes of negative d_a reflected and,
when |dy| > |dz|, ky and kz exchanged; a reflected kx is read back through
the conjugate symmetry of a real vector.  No twiddle factor: the kernel
vector is centred on index 0.  No GPU needed."""
import numpy as np
import pytest

from oracle import fmm


@pytest.mark.parametrize("n_b,level", [(4, 0), (4, 2), (6, 1)])
def test_every_offset_maps_to_its_representative(n_b, level):
    n = n_b if level == 0 else n_b + 1
    S = 2 * n
    h = 1 if level == 0 else 2 ** (level - 1)
    spec = {}

    def khat(d):
        if d not in spec:
            spec[d] = np.fft.rfftn(fmm.kernel_vector(h, d, n, n_b, S))   # [kz, ky, kx], kx half
        return spec[d]

    NX = S // 2 + 1
    kz, ky, kx = np.meshgrid(np.arange(S), np.arange(S), np.arange(NX), indexing="ij")
    for dz in range(-3, 4):
        for dy in range(-3, 4):
            for dx in range(-3, 4):
                d = (dx, dy, dz)
                ay, az = abs(dy), abs(dz)
                swap = ay > az
                rep = (abs(dx), min(ay, az), max(ay, az))
                xneg = dx < 0
                fy = (dy < 0) != xneg
                fz = (dz < 0) != xneg
                ky1 = np.where(fy, (S - ky) % S, ky)
                kz1 = np.where(fz, (S - kz) % S, kz)
                if swap:
                    ky1, kz1 = kz1, ky1
                got = khat(rep)[kz1, ky1, kx]
                if xneg:
                    got = np.conj(got)
                ref = khat(d)
                assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), d
