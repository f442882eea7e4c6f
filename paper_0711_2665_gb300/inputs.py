"""Seeded synthetic inputs: geometry masks, initial chains, initial flows.

This module draws and lays out inputs only; it holds none of the method's
arithmetic (no equilibrium, no forces, no streaming).  It is the one module
that both the CUDA path's callers and the oracle's tests use, so that both
start from the same problem.

Geometry follows the set-up of Sec. IV of Fyta et al.: a box periodic in all
directions, a one-site-thick wall across x at ``wall_x`` with a square pore of
side ``h`` centred in y and z.  Arrays are indexed ``[z, y, x]`` (x fastest in
memory), solid = 1.
"""
from __future__ import annotations

import numpy as np

WCA_CUT = 2.0 ** (1.0 / 6.0)


def pore_range(n: int, h: int) -> tuple[int, int]:
    """First and last lattice index of a pore of side ``h`` centred in an axis of ``n`` sites."""
    lo = n // 2 - h // 2
    return lo, lo + h - 1


def pore_wall_mask(nx: int, ny: int, nz: int, wall_x: int, pore_h: int) -> np.ndarray:
    """Solid plane x = wall_x with an h x h square hole at the centre (Sec. IV)."""
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    if wall_x < 0:
        return m
    m[:, :, wall_x] = 1
    ylo, yhi = pore_range(ny, pore_h)
    zlo, zhi = pore_range(nz, pore_h)
    m[zlo:zhi + 1, ylo:yhi + 1, wall_x] = 0
    return m


def slab_walls_mask(nx: int, ny: int, nz: int, axis: str = "y") -> np.ndarray:
    """One solid plane at index 0 along ``axis``: with periodic wrap this is a
    channel bounded by two walls (used for plane Poiseuille flow)."""
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    if axis == "y":
        m[:, 0, :] = 1
    elif axis == "z":
        m[0, :, :] = 1
    else:
        m[:, :, 0] = 1
    return m


def _near_solid(p: np.ndarray, solid: np.ndarray, dmin: float) -> bool:
    nz, ny, nx = solid.shape
    lo = np.floor(p - dmin).astype(int)
    hi = np.floor(p + dmin).astype(int) + 1
    for z in range(lo[2], hi[2] + 1):
        for y in range(lo[1], hi[1] + 1):
            for x in range(lo[0], hi[0] + 1):
                if solid[z % nz, y % ny, x % nx]:
                    d = p - np.array([x, y, z], dtype=float)
                    if d @ d < dmin * dmin:
                        return True
    return False


def _min_image(d: np.ndarray, box: np.ndarray) -> np.ndarray:
    return d - box * np.floor(d / box + 0.5)


def chain_walk(n_beads: int, dims: tuple[int, int, int], wall_x: int, solid: np.ndarray,
               seed: int, bond: float = 1.0, min_dist: float = WCA_CUT,
               max_tries: int = 200) -> np.ndarray:
    """Seeded self-avoiding random walk on the cis side of the wall (Sec. IV).

    The first bead sits at the pore entrance, (wall_x - 1, ny/2, nz/2).  Each
    next bead is one bond length away in a uniformly random direction; a step
    is rejected if it comes closer than ``min_dist`` to any non-bonded bead
    (minimum image) or to a solid site, or leaves the cis half of the box
    ``[wall_x - nx/2 + 1, wall_x - 1]`` in x.  After ``max_tries`` rejections
    the walk backtracks.  Returns unwrapped positions, shape (n_beads, 3).
    """
    nx, ny, nz = dims
    box = np.array([nx, ny, nz], dtype=float)
    rng = np.random.Generator(np.random.PCG64(seed))
    if wall_x >= 0:
        start = np.array([wall_x - 1.0, ny // 2, nz // 2], dtype=float)
        xmin, xmax = wall_x - nx / 2.0 + 1.0, wall_x - 1.0
    else:
        start = np.array([nx / 2.0, ny / 2.0, nz / 2.0])
        xmin, xmax = -np.inf, np.inf
    r = np.zeros((n_beads, 3))
    if n_beads == 0:
        return r
    r[0] = start
    i = 1
    total = 0
    while i < n_beads:
        placed = False
        for _ in range(max_tries):
            total += 1
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            p = r[i - 1] + bond * d
            if p[0] < xmin or p[0] > xmax:
                continue
            if i >= 2:
                dd = _min_image(r[:i - 1] - p, box)
                if np.min(np.einsum("ij,ij->i", dd, dd)) < min_dist * min_dist:
                    continue
            if _near_solid(p, solid, min_dist):
                continue
            r[i] = p
            i += 1
            placed = True
            break
        if not placed:
            i = max(1, i - 5)
        if total > 1000 * max_tries * max(n_beads, 1):
            raise RuntimeError("chain_walk: could not place the chain")
    return r


def chain_lengths(n_real: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Polymer lengths drawn uniformly from {lo, ..., hi}, one per realization."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=n_real).astype(np.int32)


def shear_wave_velocity(nx: int, ny: int, nz: int, amplitude: float) -> np.ndarray:
    """u_y(x) = A sin(2 pi x / nx), u_x = u_z = 0; shape (3, nz, ny, nx)."""
    u = np.zeros((3, nz, ny, nx))
    x = np.arange(nx)
    u[1] = amplitude * np.sin(2.0 * np.pi * x / nx)[None, None, :]
    return u


def smooth_random_velocity(nx: int, ny: int, nz: int, amplitude: float, seed: int, modes: int = 3) -> np.ndarray:
    """A seeded smooth periodic flow: a sum of ``modes`` plane waves per
    component with random integer wave vectors (|k_a| <= 2 per axis), phases
    and weights, scaled so that the largest |u_a| is ``amplitude``; shape
    (3, nz, ny, nx).  Every site moves, so every population deviates."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    for a in range(3):
        for _ in range(modes):
            k = rng.integers(-2, 3, size=3)
            if not k.any():
                k[0] = 1
            ph = 2.0 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz) + rng.uniform(0, 2 * np.pi)
            u[a] += rng.uniform(0.5, 1.0) * np.sin(ph)
        u[a] *= amplitude / max(np.abs(u[a]).max(), 1e-300)
    return u
