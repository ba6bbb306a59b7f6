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


def test_stencil_residual_helper():
    # the residual helper sees the exact solution's residual at roundoff, and a
    # planted error of 1e-6 at one interior point as 6e-6 (the stencil's centre
    # weight) relative to max|f| = 1
    n_b = 6
    blocks = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], dtype=np.int32)
    rng = np.random.default_rng(1)
    f = rng.uniform(-1, 1, size=(4, n_b, n_b, n_b))
    f.flat[0] = 1.0
    u = direct.direct_sum(blocks, n_b, f)
    assert direct.stencil_residual(blocks, n_b, u, f) < 1e-12
    bad = u.copy()
    bad[0, 3, 3, 3] += 1e-6
    assert abs(direct.stencil_residual(blocks, n_b, bad, f) - 6e-6) < 1e-9
    # a corner of the active grid is neither checked nor a neighbour of an
    # interior point (its neighbours are on the boundary too)
    bad = u.copy()
    bad[0, 0, 0, 0] += 1.0
    assert direct.stencil_residual(blocks, n_b, bad, f) < 1e-12
    # a boundary point next to the interior is seen through its neighbour
    bad = u.copy()
    bad[0, 0, 3, 3] += 1e-6                                      # z = 0 face
    assert abs(direct.stencil_residual(blocks, n_b, bad, f) - 1e-6) < 1e-9
