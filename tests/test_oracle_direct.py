"""Pins of the exact O(N^2) sum (oracle/direct.c)."""
import numpy as np


from oracle import direct, lgf


def test_matches_python_double_loop():
    rng = np.random.default_rng(5)
    blocks = np.array([[0, 0, 0], [1, 0, 0], [3, 2, 1]], dtype=np.int32)
    n_b = 2
    f = rng.standard_normal((3, n_b, n_b, n_b))
    u = direct.direct_sum(blocks, n_b, f)
    pts = direct.point_coords(blocks, n_b)
    fv = f.reshape(-1)
    ref = np.empty(len(pts))
    for i, p in enumerate(pts):
        ref[i] = sum(lgf.lgf([p - q])[0] * fv[j] for j, q in enumerate(pts))
    assert np.allclose(u.reshape(-1), ref, rtol=0, atol=1e-15 * np.abs(ref).max() * 10)


def test_discrete_poisson_on_interior():
    # u = G * f solves L u = f at every lattice point: check it on the interior
    # of a 2x2x1-block domain, where all six neighbours are active.
    n_b = 6
    blocks = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], dtype=np.int32)
    rng = np.random.default_rng(1)
    f = rng.uniform(-1, 1, size=(4, n_b, n_b, n_b))
    u = direct.direct_sum(blocks, n_b, f)
    grid_u = np.zeros((n_b, 2 * n_b, 2 * n_b))
    grid_f = np.zeros_like(grid_u)
    for b, (bx, by, bz) in enumerate(blocks):
        grid_u[:, by * n_b:(by + 1) * n_b, bx * n_b:(bx + 1) * n_b] = u[b]
        grid_f[:, by * n_b:(by + 1) * n_b, bx * n_b:(bx + 1) * n_b] = f[b]
    c = grid_u[1:-1, 1:-1, 1:-1]
    lap = (grid_u[2:, 1:-1, 1:-1] + grid_u[:-2, 1:-1, 1:-1] + grid_u[1:-1, 2:, 1:-1]
           + grid_u[1:-1, :-2, 1:-1] + grid_u[1:-1, 1:-1, 2:] + grid_u[1:-1, 1:-1, :-2] - 6 * c)
    assert np.abs(lap - grid_f[1:-1, 1:-1, 1:-1]).max() < 1e-12
