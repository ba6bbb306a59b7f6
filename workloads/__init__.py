"""Seeded synthetic inputs for the LGF solver: block lists and source fields.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
no arithmetic of the solver itself: it only draws block sets and source values.
Every generator is deterministic in its seed (numpy PCG64) and returns

    blocks : int32 array (n_blocks, 3) of block indices (x, y, z)
    f      : float64 array (n_blocks, n_b, n_b, n_b), per block indexed [k][j][i]
             with i (x) fastest, so block b's point (i, j, k) sits at grid point
             blocks[b] * n_b + (i, j, k)

The workloads follow the paper's experiments (Sec. 4): smooth or random sources
on cubes and irregular block-structured domains; no dataset is involved.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem", "full_box_blocks", "gaussian_box", "torus_box", "tori_irregular",
    "manufactured", "batch_problems", "arrival_stream", "config", "CONFIGS", "block_subset", "dipole_box",
]


@dataclasses.dataclass
class Problem:
    blocks: np.ndarray          # (n_blocks, 3) int32
    f: np.ndarray               # (n_blocks, n_b, n_b, n_b) float64
    n_b: int
    n_levels: int
    order: int
    name: str = ""
    u_exact: np.ndarray | None = None   # known exact solution, if any

    @property
    def n_points(self) -> int:
        return int(self.blocks.shape[0]) * self.n_b ** 3


def full_box_blocks(nbx: int, nby: int | None = None, nbz: int | None = None) -> np.ndarray:
    """All blocks of an nbx x nby x nbz block grid, x fastest."""
    nby = nbx if nby is None else nby
    nbz = nbx if nbz is None else nbz
    z, y, x = np.meshgrid(np.arange(nbz), np.arange(nby), np.arange(nbx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.int32)


def levels_for(nb_axis: int) -> int:
    """Tree depth whose top level holds at most two intervals per axis."""
    return max(1, int(math.ceil(math.log2(max(nb_axis, 1)))))


def _block_points(blocks: np.ndarray, n_b: int):
    """Grid coordinates (x, y, z) of every point, shaped (n_blocks, n_b, n_b, n_b)."""
    r = np.arange(n_b)
    kk, jj, ii = np.meshgrid(r, r, r, indexing="ij")
    bx = blocks[:, 0, None, None, None] * n_b
    by = blocks[:, 1, None, None, None] * n_b
    bz = blocks[:, 2, None, None, None] * n_b
    return bx + ii, by + jj, bz + kk


def _grid_noise(rng: np.random.Generator, shape_xyz, blocks, n_b):
    """U(-1,1) drawn over a whole box in x-fastest point order, gathered per block."""
    nx, ny, nz = shape_xyz
    u = rng.uniform(-1.0, 1.0, size=nx * ny * nz).reshape(nz, ny, nx)
    x, y, z = _block_points(blocks, n_b)
    return u[z, y, x]


def gaussian_box(seed: int = 0) -> Problem:
    """32^3 grid, 4^3 blocks of 8^3: Gaussian of width 4 at the grid centre with
    10% multiplicative noise (two-level plain method, interpolation order 6)."""
    n_b, nb = 8, 4
    blocks = full_box_blocks(nb)
    x, y, z = _block_points(blocks, n_b)
    c = 15.5
    r2 = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = _grid_noise(rng, (32, 32, 32), blocks, n_b)
    f = np.exp(-r2 / (2.0 * 4.0 ** 2)) * (1.0 + 0.1 * noise)
    return Problem(blocks, f, n_b, 2, 6, "gaussian_box_32")


def _torus_distance2(x, y, z, centre, normal, radius):
    vx, vy, vz = x - centre[0], y - centre[1], z - centre[2]
    axial = vx * normal[0] + vy * normal[1] + vz * normal[2]
    rx, ry, rz = vx - axial * normal[0], vy - axial * normal[1], vz - axial * normal[2]
    rho = np.sqrt(rx * rx + ry * ry + rz * rz)
    return (rho - radius) ** 2 + axial ** 2


def torus_box(seed: int = 0, nb: int = 8, n_b: int = 16, radius: float = 40.0,
              sigma: float = 6.0, noise: float = 0.05, order: int = 8,
              n_levels: int | None = None) -> Problem:
    """Full box of nb^3 blocks with a Gaussian-cored torus (vortex-ring-like)
    source about the box centre, normal +z, with seeded multiplicative noise.
    The default is the 128^3 single-solve workload (8^3 blocks of 16^3)."""
    side = nb * n_b
    blocks = full_box_blocks(nb)
    x, y, z = _block_points(blocks, n_b)
    c = (side - 1) / 2.0
    d2 = _torus_distance2(x, y, z, (c, c, c), (0.0, 0.0, 1.0), radius)
    rng = np.random.Generator(np.random.PCG64(seed))
    u = _grid_noise(rng, (side, side, side), blocks, n_b)
    f = np.exp(-d2 / (2.0 * sigma ** 2)) * (1.0 + noise * u)
    L = levels_for(nb) if n_levels is None else n_levels
    return Problem(blocks, f, n_b, L, order, f"torus_box_{side}")


def _random_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def tori_irregular(seed: int = 2, nb: int = 32, n_b: int = 16, n_tori: int = 12,
                   keep_rel: float = 1e-6, r_range=(20.0, 120.0), s_range=(6.0, 16.0),
                   order: int = 8) -> Problem:
    """Irregular block-structured domain: inside a (nb*n_b)^3 bounding box, keep
    the blocks where a seeded sum of random Gaussian tori exceeds keep_rel of its
    maximum.  Default: 512^3 box, 16^3 blocks, 12 tori, 5 levels; the radius and
    core ranges were set once so that about 22% of the box (3.0e7 points) is kept."""
    side = nb * n_b
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = side / 4.0, 3.0 * side / 4.0
    tori = []
    for _ in range(n_tori):
        centre = rng.uniform(lo, hi, size=3)
        radius = float(np.exp(rng.uniform(np.log(r_range[0]), np.log(r_range[1]))))
        sigma = float(rng.uniform(*s_range))
        normal = _random_unit(rng)
        amp = float(rng.uniform(0.5, 1.0))
        tori.append((centre, normal, radius, sigma, amp))
    allb = full_box_blocks(nb)
    # Blocks within reach of a ring (beyond ~6.5 sigma from it the Gaussian is
    # below 1e-9 of its amplitude); the keep rule is applied exactly below.
    centres = (allb + 0.5) * n_b - 0.5
    half_diag = math.sqrt(3.0) * n_b / 2.0
    reach = []
    for centre, normal, radius, sigma, amp in tori:
        d2 = _torus_distance2(centres[:, 0], centres[:, 1], centres[:, 2], centre, normal, radius)
        reach.append(np.sqrt(d2) - half_diag < 6.5 * sigma)
    cand = np.nonzero(np.any(reach, axis=0))[0]
    pos = -np.ones(len(allb), dtype=np.int64)
    pos[cand] = np.arange(len(cand))
    f = np.zeros((len(cand), n_b, n_b, n_b))
    for (centre, normal, radius, sigma, amp), mask in zip(tori, reach):
        sel = np.nonzero(mask)[0]
        x, y, z = _block_points(allb[sel], n_b)
        f[pos[sel]] += amp * np.exp(-_torus_distance2(x, y, z, centre, normal, radius) / (2.0 * sigma ** 2))
    blocks = allb[cand]
    fmax = np.abs(f).max()
    keep = np.abs(f).reshape(len(blocks), -1).max(axis=1) > keep_rel * fmax
    return Problem(blocks[keep].copy(), f[keep].copy(), n_b, levels_for(nb), order,
                   f"tori_irregular_{side}")


def block_subset(p: Problem, frac: float, seed: int, name: str | None = None) -> Problem:
    """A seeded random subset of a problem's blocks (each kept with probability
    frac), with their sources: an irregular, sparser domain spanning the same
    box, so the tree keeps its depth."""
    rng = np.random.Generator(np.random.PCG64(seed))
    keep = rng.uniform(size=len(p.blocks)) < frac
    return Problem(p.blocks[keep].copy(), p.f[keep].copy(), p.n_b, p.n_levels, p.order,
                   name or f"{p.name}_subset{frac:g}")


def dipole_box(nb: int = 8, n_b: int = 8, sigma: float = 4.0, sep: float = 16.0, order: int = 8,
               n_levels: int | None = None) -> Problem:
    """A smooth signed source on a full box of nb^3 blocks: two Gaussians of
    width sigma and opposite sign, sep apart along x about the box centre."""
    side = nb * n_b
    blocks = full_box_blocks(nb)
    x, y, z = _block_points(blocks, n_b)
    c = (side - 1) / 2.0
    g = lambda cx: np.exp(-((x - cx) ** 2 + (y - c) ** 2 + (z - c) ** 2) / (2.0 * sigma ** 2))
    f = g(c - sep / 2.0) - g(c + sep / 2.0)
    L = levels_for(nb) if n_levels is None else n_levels
    return Problem(blocks, f, n_b, L, order, f"dipole_{side}_nb{n_b}")


def shape_blocks(shape: str, diameter: int, n_b: int) -> np.ndarray:
    """Active blocks of a cube, a sphere or a spherical shell of the given
    diameter in grid points (the paper's error and rate experiments, Sec. 4):
    a block is active when its centre lies in the region; the shell keeps
    radii between half and all of the outer radius."""
    nb = max(1, int(math.ceil(diameter / n_b)))
    blocks = full_box_blocks(nb)
    if shape == "box":
        return blocks
    c = (blocks + 0.5) * n_b - nb * n_b / 2.0
    r = np.sqrt((c ** 2).sum(axis=1))
    R = diameter / 2.0
    keep = r <= R if shape == "sphere" else (r <= R) & (r >= 0.5 * R)
    if shape not in ("sphere", "shell"):
        raise ValueError(shape)
    return blocks[keep].copy()


def manufactured(blocks: np.ndarray, n_b: int, n_levels: int, order: int,
                 seed: int = 0) -> Problem:
    """Random manufactured solution of Sec. 4.1: u ~ U(-1,1) on the active grid,
    zero on its boundary points (active points with an inactive 6-neighbour) and
    outside; the source is f = L u with the 7-point Laplacian, so u is the exact
    decaying solution of L u = f."""
    blocks = np.asarray(blocks, dtype=np.int32)
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = blocks.min(axis=0) * n_b - 1
    hi = (blocks.max(axis=0) + 1) * n_b + 1
    shape = tuple((hi - lo)[::-1])        # (z, y, x) with a one-point margin
    active = np.zeros(shape, dtype=bool)
    x, y, z = _block_points(blocks, n_b)
    xs, ys, zs = x - lo[0], y - lo[1], z - lo[2]
    active[zs, ys, xs] = True
    interior = active.copy()
    for ax in range(3):
        for sh in (1, -1):
            interior &= np.roll(active, sh, axis=ax)
    u = np.zeros(shape)
    u[zs, ys, xs] = rng.uniform(-1.0, 1.0, size=xs.shape)
    u[~interior] = 0.0
    lap = -6.0 * u
    for ax in range(3):
        for sh in (1, -1):
            lap += np.roll(u, sh, axis=ax)
    f = lap[zs, ys, xs]
    return Problem(blocks, f, n_b, n_levels, order, "manufactured",
                   u_exact=u[zs, ys, xs])


def _blob_problem(rng: np.random.Generator):
    n_b = 8 if rng.uniform() < 0.5 else 16
    side = float(np.exp(rng.uniform(np.log(32.0), np.log(192.0))))
    side = int(math.ceil(side / n_b)) * n_b
    nb = side // n_b
    n_blobs = int(rng.integers(1, 7))
    blobs = [(rng.uniform(0, side, size=3), float(rng.uniform(3.0, 12.0)),
              float(rng.uniform(0.5, 1.0))) for _ in range(n_blobs)]
    allb = full_box_blocks(nb)
    x, y, z = _block_points(allb, n_b)
    f = np.zeros(x.shape)
    for c, s, a in blobs:
        f += a * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * s * s))
    keep = np.abs(f).reshape(len(allb), -1).max(axis=1) > 1e-6 * np.abs(f).max()
    return Problem(allb[keep].copy(), f[keep].copy(), n_b, levels_for(nb), 8,
                   f"blobs_{side}_nb{n_b}")


def batch_problems(n: int = 64, seed: int = 3) -> list[Problem]:
    """Many independent uneven solves: boxes log-uniform in 32^3..192^3 (8^3 or
    16^3 blocks), each a seeded random sum of 1-6 Gaussian blobs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [_blob_problem(rng) for _ in range(n)]


def arrival_stream(n_requests: int = 2200, rate: float = 200.0, seed: int = 1):
    """Poisson arrivals of single solves with point counts log-uniform in
    2^12..2^24; returns a list of (arrival_time_s, n_b, blocks_per_axis)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    out = []
    for ti in t:
        npts = float(np.exp(rng.uniform(np.log(2.0 ** 12), np.log(2.0 ** 24))))
        n_b = 16 if npts >= 2 ** 15 else 8
        nb = max(2, int(round(npts ** (1.0 / 3.0) / n_b)))
        out.append((float(ti), n_b, nb))
    return out


def request_problem(n_b: int, nb: int, seed: int) -> Problem:
    """One served request: a torus scaled to the box (R = 0.3 s, sigma = 0.06 s)
    with 5% noise on a fully occupied box of nb^3 blocks."""
    side = nb * n_b
    return torus_box(seed=seed, nb=nb, n_b=n_b, radius=0.3 * side, sigma=0.06 * side,
                     noise=0.05, order=8)


def config(i: int) -> Problem:
    """The single-solve workloads by index: 0 = 32^3 Gaussian (2 levels, order 6),
    1 = 128^3 torus (3 levels, order 8), 2 = 512^3 irregular tori (5 levels)."""
    if i == 0:
        return gaussian_box(0)
    if i == 1:
        return torus_box(0)
    if i == 2:
        return tori_irregular(2)
    raise ValueError(i)


CONFIGS = {0: "gaussian_box_32", 1: "torus_box_128", 2: "tori_irregular_512"}
