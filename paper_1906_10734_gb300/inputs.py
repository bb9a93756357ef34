"""Seeded synthetic particle sets for the HPM solver and its CPU oracle.

This module holds the input generators only. It contains none of the
method's arithmetic, so the GPU path and the FP64 oracle can both draw their
inputs from it without sharing any solver code.

Random numbers come from one counter-based generator, splitmix64: draw ``k``
of a stream seeded with ``s`` is ``mix(s + (k + 1) * 0x9E3779B97F4A7C15)``
(mod 2**64), where ``mix`` is the published splitmix64 finaliser. A draw is
turned into a double in [0, 1) from its top 53 bits.

The paper measures on a point source inside a patch-based grid code
(Sec. 3.2). Its data are not available, so these particle sets stand in for
them: a uniform cube and a truncated Plummer sphere, with the sizes of the
workloads the solver is quoted on.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the splitmix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the splitmix64 draws."""
    z = splitmix64(seed, start, count)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_cube(n: int, seed: int) -> np.ndarray:
    """``n`` positions uniform in [0, 1)^3, shape (n, 3), FP64."""
    return uniform01(seed, 0, 3 * n).reshape(n, 3)


def plummer_sphere(n: int, seed: int, a: float = 0.05, rmax: float = 0.5,
                   center=(0.5, 0.5, 0.5)) -> np.ndarray:
    """``n`` positions from a Plummer sphere of scale radius ``a`` truncated at ``rmax``.

    Textbook inverse-CDF sampling: the enclosed mass fraction is
    m(r) = r^3 / (r^2 + a^2)^{3/2}; X is uniform in (0, m(rmax)] and
    r = a (X^{-2/3} - 1)^{-1/2}. Directions are isotropic.
    """
    u = uniform01(seed, 0, 3 * n).reshape(n, 3)
    mmax = rmax ** 3 / (rmax * rmax + a * a) ** 1.5
    x = mmax * (1.0 - u[:, 0])                      # (0, m(rmax)]
    r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    r = np.minimum(r, rmax)
    cth = 2.0 * u[:, 1] - 1.0
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    ph = 2.0 * math.pi * u[:, 2]
    pos = np.empty((n, 3), dtype=np.float64)
    pos[:, 0] = center[0] + r * sth * np.cos(ph)
    pos[:, 1] = center[1] + r * sth * np.sin(ph)
    pos[:, 2] = center[2] + r * cth
    return np.clip(pos, 0.0, 1.0)


def equal_masses(n: int, total: float = 1.0) -> np.ndarray:
    return np.full(n, total / max(n, 1), dtype=np.float64)


def log_uniform_masses(n: int, seed: int, decades: float = 6.0, total: float = 1.0) -> np.ndarray:
    """Masses log-uniform over ``decades`` decades (10^(decades u), u uniform in [0, 1)),
    scaled to sum to ``total``: boxes of one level then differ in mass by up to that span."""
    m = 10.0 ** (decades * uniform01(seed, 0, n))
    return m * (total / m.sum()) if n else m


def heavy_body_masses(n: int, seed: int, ratio: float = 1e4, total_light: float = 1.0):
    """Equal masses total_light / n, except one particle (index drawn from stream
    ``seed``) of mass ``ratio`` times the total of all the others. Returns (masses, index)."""
    m = equal_masses(n, total_light)
    k = int(uniform01(seed, 0, 1)[0] * n) if n else 0
    if n:
        m[k] = ratio * (m.sum() - m[k])
    return m, k


@dataclass
class Workload:
    """One gravity problem: particles, masses, tree and gridlet parameters."""
    name: str
    pos: np.ndarray
    mass: np.ndarray
    max_depth: int
    leaf_max: int          # 0 = uniform tree refined to max_depth everywhere
    ng: int                # gridlet points per dimension
    eps: float             # Plummer softening of g(r) = 1/sqrt(r^2 + eps^2)
    origin: tuple = (0.0, 0.0, 0.0)
    side: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def uniform_4096_depth3(ng: int = 4) -> Workload:
    """4096 uniform particles, masses 1/N, uniform tree of depth 3, eps = 1e-3 (seed 1)."""
    n = 4096
    return Workload("uniform4096_depth3", uniform_cube(n, 1), equal_masses(n),
                    max_depth=3, leaf_max=0, ng=ng, eps=1e-3)


def plummer_2m_adaptive(ng: int = 4, n: int = 1 << 21) -> Workload:
    """2^21 Plummer particles (a = 0.05, r <= 0.5), adaptive tree (> 32 splits, depth <= 12), eps = 1e-4 (seed 2)."""
    return Workload(f"plummer{n}_adaptive32_depth12", plummer_sphere(n, 2), equal_masses(n),
                    max_depth=12, leaf_max=32, ng=ng, eps=1e-4)


def uniform_16m_depth7(ng: int = 4, n: int = 1 << 24) -> Workload:
    """2^24 uniform particles, uniform tree of depth 7 (128^3 leaves), eps = 1e-4 (seed 3)."""
    return Workload(f"uniform{n}_depth7", uniform_cube(n, 3), equal_masses(n),
                    max_depth=7, leaf_max=0, ng=ng, eps=1e-4)


def batch_problem(k: int, nmin: float = 1e3, nmax: float = 1e6, seed: int = 4,
                  ng: int = 4) -> Workload:
    """Problem ``k`` of the mixed batch: N log-uniform in [nmin, nmax], Plummer or uniform by coin flip.

    Stream ``seed * 2^32 + k`` draws the size and the coin; the positions
    come from the stream ``(seed * 2^32 + k) * 2 + 1``.
    """
    s = (seed << 32) + k
    u = uniform01(s, 0, 2)
    n = int(round(math.exp(math.log(nmin) + u[0] * (math.log(nmax) - math.log(nmin)))))
    pseed = (s * 2 + 1) & 0xFFFFFFFFFFFFFFFF
    if u[1] < 0.5:
        pos, kind = plummer_sphere(n, pseed), "plummer"
    else:
        pos, kind = uniform_cube(n, pseed), "uniform"
    return Workload(f"batch{k}_{kind}{n}", pos, equal_masses(n), max_depth=12, leaf_max=32,
                    ng=ng, eps=1e-4, meta={"kind": kind})


def patch_grid_cells(geometry: str, k: int = 8) -> np.ndarray:
    """Cell centres of a patch-based grid (the grid of the paper's accuracy test, Sec. 3.2):
    the domain [0, 1)^3 is an oct-tree of patches of k^3 cells each.

    ``uniform4`` / ``uniform5``: every patch at level 4 / 5 ((2^l k)^3 cells: 128^3, 256^3).
    ``mixed``: level 3 everywhere, the first octant [0, 1/2)^3 refined to level 4 and the region
    [1/8, 3/8)^3 refined to level 5 (720,896 cells). Cells are ordered patch by patch."""
    levels = {"uniform4": [(4, (0.0, 1.0))], "uniform5": [(5, (0.0, 1.0))],
              "mixed": [(3, (0.0, 1.0)), (4, (0.0, 0.5)), (5, (0.125, 0.375))]}[geometry]
    # later entries refine earlier ones: a patch is kept where no finer one covers it
    out = []
    for idx, (lev, (lo, hi)) in enumerate(levels):
        n = 1 << lev
        c = (np.arange(n) + 0.5) / n
        inside = (c > lo) & (c < hi)
        pc = np.stack(np.meshgrid(c[inside], c[inside], c[inside], indexing="ij"), axis=-1).reshape(-1, 3)
        keep = np.ones(pc.shape[0], dtype=bool)
        for lev2, (lo2, hi2) in levels[idx + 1:]:
            keep &= ~np.all((pc > lo2) & (pc < hi2), axis=1)
        pc = pc[keep]
        h = 1.0 / (n * k)
        off = (np.arange(k) + 0.5) * h - 0.5 / n
        cells = (pc[:, None, None, None, :] + np.stack(np.meshgrid(off, off, off, indexing="ij"), axis=-1)[None])
        out.append(cells.reshape(-1, 3))
    return np.concatenate(out)


def point_source_patch_grid(geometry: str, ng: int = 4, k: int = 8) -> Workload:
    """The accuracy test of Sec. 3.2 as particles: zero-mass particles at the cell centres of the
    patch grid ``geometry`` (patch_grid_cells) and one unit mass at the corner (1, 1, 1) of the
    domain, Newtonian kernel (eps = 0). A cell splits iff it holds more than k^3 + 1 particles,
    so the tree's leaves are exactly the patches (the source adds one particle to the last
    one). The source is particle 0."""
    cells = patch_grid_cells(geometry, k)
    pos = np.concatenate([np.ones((1, 3)), cells])
    mass = np.zeros(pos.shape[0])
    mass[0] = 1.0
    depth = {"uniform4": 4, "uniform5": 5, "mixed": 5}[geometry]
    return Workload(f"pointsource_{geometry}", pos, mass, max_depth=depth, leaf_max=k ** 3 + 1, ng=ng, eps=0.0,
                    meta={"geometry": geometry, "source": 0})


def small_plummer(n: int, seed: int, leaf_max: int = 32, max_depth: int = 12, ng: int = 4,
                  eps: float = 1e-4) -> Workload:
    """Reduced Plummer problem with the same recipe as the 2^21 workload."""
    return Workload(f"plummer{n}_adaptive{leaf_max}", plummer_sphere(n, seed), equal_masses(n),
                    max_depth=max_depth, leaf_max=leaf_max, ng=ng, eps=eps)
