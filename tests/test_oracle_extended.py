"""Oracle pins for the extended target gridlet (Sec. 2.5): the potential is taken at the
cell's Ng^3 nodes widened by one node on each side ((Ng + 2)^3 values) and interpolated
with degree Ng + 1.

The paper's claim that keeps the (8 Ng)^3 FFT valid: every node of the widened gridlet
lies within 4 Ng = P/2 grid points (per axis) of every interaction-zone source, and
wavenumbers up to P/2 are free of the periodic images. Pinned here:
- the FFT convolution read at the widened nodes equals the direct interaction-zone sum
  for all 8 child parities, and widening by two nodes (distance 4 Ng + 1) breaks it;
- the widened interpolant reproduces tensor polynomials of degree Ng + 1;
- the method's error against all-pairs summation falls (modestly, as the paper found)
  when the gridlet is widened.
"""
import numpy as np
import pytest

import oracle as O
from paper_1906_10734_gb300 import inputs as I


def _level_case(ng, depth=3, n=3000, seed=7):
    pos = I.uniform_cube(n, seed)
    mass = I.equal_masses(n)
    tr = O.Tree(pos, max_depth=depth, leaf_max=0)
    lv = tr.levels[depth]
    allb = np.arange(lv.keys.shape[0])
    grid = O.p2g(ng, lv.begin, lv.end, tr.centers(depth, allb), np.full(allb.size, tr.box_side(depth)),
                 tr.spos, mass[tr.perm])
    return tr, lv, allb, grid


def _fft_and_direct(ng, ext, eps=1e-3, depth=3):
    tr, lv, allb, grid = _level_case(ng, depth)
    real = np.flatnonzero(lv.real)
    octs = (lv.keys[real] & np.uint64(7)).astype(int)
    pick = np.concatenate([real[octs == c][:3] for c in range(8)])
    assert len(set((lv.keys[pick] & np.uint64(7)).tolist())) == 8
    rows, tpos = tr.iz_rows(depth, pick)
    h = tr.box_side(depth) / ng
    out = O.m2l_fft(ng, rows, tpos, grid, O.green_hat(ng, eps, h), ext=ext)
    soff = np.concatenate([[0], np.cumsum((rows >= 0).sum(1))])
    ref = O.m2l_direct(ng, eps, tr.centers(depth, pick), np.full(pick.size, tr.box_side(depth)), soff,
                       rows[rows >= 0], tr.centers(depth, allb), grid, ext=ext)
    return out, ref


@pytest.mark.parametrize("ng", [1, 2, 3, 4])
def test_fft_at_widened_nodes_equals_direct_sum(ng):
    out, ref = _fft_and_direct(ng, 1)
    assert out.shape[1] == (ng + 2) ** 3
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("ng", [2, 3])
def test_widening_by_two_nodes_meets_the_periodic_images(ng):
    """Nodes 4 Ng + 1 grid points from a zone source see its periodic image: the FFT
    readout no longer equals the direct sum (the bound of Sec. 2.5 is tight)."""
    out, ref = _fft_and_direct(ng, 2)
    assert np.max(np.abs(out - ref)) > 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("ng", [2, 3, 4])
def test_widened_interpolant_reproduces_degree_ng_plus_1(ng):
    rng = np.random.default_rng(ng)
    deg = ng + 1
    coef = rng.normal(size=(deg + 1, deg + 1, deg + 1))
    x = O.nodes_ext(ng, 1)
    ne = ng + 2

    def poly(u):
        px = np.array([u[0] ** k for k in range(deg + 1)])
        py = np.array([u[1] ** k for k in range(deg + 1)])
        pz = np.array([u[2] ** k for k in range(deg + 1)])
        dpx = np.array([k * u[0] ** (k - 1) if k else 0.0 for k in range(deg + 1)])
        dpy = np.array([k * u[1] ** (k - 1) if k else 0.0 for k in range(deg + 1)])
        dpz = np.array([k * u[2] ** (k - 1) if k else 0.0 for k in range(deg + 1)])
        v = np.einsum("ijk,i,j,k->", coef, px, py, pz)
        g = np.array([np.einsum("ijk,i,j,k->", coef, dpx, py, pz), np.einsum("ijk,i,j,k->", coef, px, dpy, pz),
                      np.einsum("ijk,i,j,k->", coef, px, py, dpz)])
        return v, g

    c, L = np.array([0.3, 0.6, 0.4]), 0.125
    vals = np.array([poly(np.array([x[p % ne], x[(p // ne) % ne], x[p // (ne * ne)]]))[0] for p in range(ne ** 3)])
    pts = c + L * (rng.random((20, 3)) - 0.5)
    phi, acc = O.far_eval(ng, pts, np.arange(21), np.zeros(20, np.int64), c[None, :], np.array([L]),
                          vals[None, :], ext=1)
    for k in range(20):
        v, g = poly((pts[k] - c) / L)
        assert abs(phi[k] - v) < 1e-10 * max(1.0, abs(v))
        assert np.allclose(acc[k], -g / L, rtol=1e-8, atol=1e-8)


def test_widened_gridlets_reduce_the_method_error():
    w = I.Workload("u", I.uniform_cube(3000, 21), I.equal_masses(3000), max_depth=3, leaf_max=0, ng=2, eps=1e-3)
    tr = O.Tree(w.pos, max_depth=3, leaf_max=0)
    sample = np.arange(0, w.n, 6)
    _, a0 = O.direct_sum(w.pos, w.mass, w.eps, targets=sample)
    for ng in (2, 3, 4):
        e_std = O.rel_rms(O.solve_direct(tr, w.mass, ng, w.eps, sample)[1], a0)
        e_ext = O.rel_rms(O.solve_direct(tr, w.mass, ng, w.eps, sample, ext=1)[1], a0)
        print(f"Ng={ng}: method error {e_std:.3e}, widened {e_ext:.3e}")
        assert e_ext < e_std


@pytest.mark.parametrize("depth", [0, 1])
def test_widened_shallow_tree_is_exact_direct_sum(depth):
    pos, mass = I.uniform_cube(300, 11), I.equal_masses(300)
    tr = O.Tree(pos, max_depth=depth, leaf_max=0)
    phi, acc = O.solve_direct(tr, mass, 4, 1e-3, ext=1)
    p0, a0 = O.direct_sum(pos, mass, 1e-3)
    assert O.rel_rms(acc, a0) < 1e-14 and O.rel_rms(phi, p0) < 1e-14
