"""Oracle pins for Green functions other than Plummer (Sec. 4: the method only convolves
with the Green function, so any radial kernel serves).

Each kernel is pinned to what its physics fixes, not to its own formula:
- Yukawa: its potential solves the screened Poisson equation, lap(phi) = phi / lambda^2
  away from the source, and an infinite screening length is the Plummer kernel;
- erf(r/a)/r (a user kernel in C): the potential of a Gaussian charge, so lap(phi) equals
  4 pi m times the Gaussian density;
- every kernel: the acceleration is minus the gradient of the potential (central
  differences of the oracle's own potential), a user kernel equal to Plummer gives the
  Plummer results, the (8 Ng)^3 FFT convolution equals the direct interaction-zone sum,
  and HPM equals the all-pairs sum when every pair is near (depth <= 1) and approaches
  it as the gridlet order grows.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1906_10734_gb300 import inputs as I
import user_kernels as UK


def erf_kernel(a, with_dg=True):
    g, dg, p = UK.erf_kernel(a)
    k = O.Kernel.user(g, dg if with_dg else None, p.ptr)
    k._param = p
    return k


def plummer_user_kernel(eps, with_dg=True):
    g, dg, p = UK.plummer_kernel(eps)
    k = O.Kernel.user(g, dg if with_dg else None, p.ptr)
    k._param = p
    return k


def potential_at(kernel, src, m, pts):
    """phi at pts of one source of mass m at src (targets carry no mass)."""
    pos = np.vstack([src[None, :], pts])
    mass = np.zeros(pos.shape[0])
    mass[0] = m
    phi, acc = O.direct_sum(pos, mass, kernel, targets=np.arange(1, pos.shape[0]))
    return phi, acc


def laplacian(kernel, src, m, x, h):
    """7-point Laplacian at steps h and h/2, Richardson-combined (fourth order), and phi(x)."""
    def lap(hh):
        offs = np.array([[0, 0, 0]] + [[s * hh if d == k else 0.0 for d in range(3)] for k in range(3)
                                       for s in (1, -1)])
        phi, _ = potential_at(kernel, src, m, x[None, :] + offs)
        return (phi[1:].sum() - 6.0 * phi[0]) / (hh * hh), phi[0]
    l1, phi = lap(h)
    l2, _ = lap(0.5 * h)
    return (4.0 * l2 - l1) / 3.0, phi


def test_yukawa_solves_the_screened_poisson_equation():
    lam, m = 0.2, 1.7
    src = np.array([0.31, 0.42, 0.53])
    k = O.Kernel.yukawa(lam)
    rng = np.random.default_rng(1)
    for _ in range(5):
        d = rng.normal(size=3)
        x = src + (0.05 + 0.3 * rng.random()) * d / np.linalg.norm(d)
        lap, phi = laplacian(k, src, m, x, 2e-3)
        assert abs(lap - phi / lam ** 2) < 1e-6 * abs(phi / lam ** 2)


def test_yukawa_without_screening_is_plummer():
    pos, mass = I.uniform_cube(300, 3), I.equal_masses(300)
    for eps in (0.0, 1e-2):
        p1, a1 = O.direct_sum(pos, mass, O.Kernel.yukawa(1e30, eps))
        p0, a0 = O.direct_sum(pos, mass, eps)
        assert O.rel_rms(p1, p0) < 1e-13 and O.rel_rms(a1, a0) < 1e-13


def test_erf_kernel_is_the_potential_of_a_gaussian_charge():
    a, m = 0.05, 2.0
    src = np.array([0.5, 0.5, 0.5])
    k = erf_kernel(a)
    rng = np.random.default_rng(2)
    for r in (0.3 * a, a, 2.0 * a, 3.0 * a):
        d = rng.normal(size=3)
        x = src + r * d / np.linalg.norm(d)
        lap, _ = laplacian(k, src, m, x, 2e-2 * a)
        rho = math.exp(-(r / a) ** 2) / (math.pi ** 1.5 * a ** 3)
        assert abs(lap - 4.0 * math.pi * m * rho) < 1e-6 * 4.0 * math.pi * m * rho


@pytest.mark.parametrize("kind", ["yukawa", "yukawa_soft", "erf", "erf_numeric_derivative"])
def test_acceleration_is_minus_the_gradient_of_the_potential(kind):
    k = {"yukawa": O.Kernel.yukawa(0.1), "yukawa_soft": O.Kernel.yukawa(0.1, 0.02),
         "erf": erf_kernel(0.03), "erf_numeric_derivative": erf_kernel(0.03, with_dg=False)}[kind]
    src = np.array([0.2, 0.7, 0.4])
    rng = np.random.default_rng(3)
    for r in (0.01, 0.05, 0.2):
        d = rng.normal(size=3)
        x = src + r * d / np.linalg.norm(d)
        h = 1e-4 * r
        pts = np.array([x + s * h * np.eye(3)[c] for c in range(3) for s in (1, -1)] + [x])
        phi, acc = potential_at(k, src, 1.3, pts)
        grad = np.array([(phi[2 * c] - phi[2 * c + 1]) / (2 * h) for c in range(3)])
        assert np.linalg.norm(acc[-1] + grad) < 1e-6 * np.linalg.norm(acc[-1])


def test_user_kernel_equal_to_plummer_gives_plummer_results():
    w = I.small_plummer(3000, 5, leaf_max=16)
    tr = O.Tree(w.pos, max_depth=w.max_depth, leaf_max=w.leaf_max)
    sample = np.arange(0, w.n, 7)
    p0, a0 = O.solve_direct(tr, w.mass, 4, 1e-3, sample)
    for with_dg, tol in ((True, 1e-13), (False, 1e-9)):
        p1, a1 = O.solve_direct(tr, w.mass, 4, plummer_user_kernel(1e-3, with_dg), sample)
        assert O.rel_rms(p1, p0) < tol and O.rel_rms(a1, a0) < tol


def _level_case(ng, depth=3, n=3000, seed=7):
    pos = I.uniform_cube(n, seed)
    mass = I.equal_masses(n)
    tr = O.Tree(pos, max_depth=depth, leaf_max=0)
    lv = tr.levels[depth]
    allb = np.arange(lv.keys.shape[0])
    grid = O.p2g(ng, lv.begin, lv.end, tr.centers(depth, allb), np.full(allb.size, tr.box_side(depth)),
                 tr.spos, mass[tr.perm])
    return tr, lv, allb, grid


@pytest.mark.parametrize("ng,kind", [(2, "yukawa"), (4, "yukawa"), (2, "erf"), (4, "erf")])
def test_fft_convolution_equals_direct_sum_other_kernels(ng, kind):
    k = O.Kernel.yukawa(0.15, 1e-3) if kind == "yukawa" else erf_kernel(0.02)
    depth = 3
    tr, lv, allb, grid = _level_case(ng, depth)
    real = np.flatnonzero(lv.real)
    octs = (lv.keys[real] & np.uint64(7)).astype(int)
    pick = np.concatenate([real[octs == c][:3] for c in range(8)])
    rows, tpos = tr.iz_rows(depth, pick)
    h = tr.box_side(depth) / ng
    out = O.m2l_fft(ng, rows, tpos, grid, O.green_hat(ng, k, h))
    soff = np.concatenate([[0], np.cumsum((rows >= 0).sum(1))])
    ref = O.m2l_direct(ng, k, tr.centers(depth, pick), np.full(pick.size, tr.box_side(depth)), soff,
                       rows[rows >= 0], tr.centers(depth, allb), grid)
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("depth", [0, 1])
def test_shallow_tree_is_exact_direct_sum_other_kernels(depth):
    pos, mass = I.uniform_cube(300, 11), I.equal_masses(300) * np.linspace(0.5, 1.5, 300)
    tr = O.Tree(pos, max_depth=depth, leaf_max=0)
    for k in (O.Kernel.yukawa(0.1, 1e-3), erf_kernel(0.02)):
        phi, acc = O.solve_direct(tr, mass, 4, k)
        p0, a0 = O.direct_sum(pos, mass, k)
        assert O.rel_rms(acc, a0) < 1e-14 and O.rel_rms(phi, p0) < 1e-14


def test_hpm_converges_to_all_pairs_with_order_other_kernels():
    """The truncation error of the far field falls with the gridlet order for these
    kernels too (the same tensor-polynomial argument, Sec. 2.2)."""
    pos, mass = I.uniform_cube(1500, 13), I.equal_masses(1500)
    tr = O.Tree(pos, max_depth=3, leaf_max=0)
    sample = np.arange(0, 1500, 5)
    for k in (O.Kernel.yukawa(0.2, 1e-3), erf_kernel(0.01)):
        _, a0 = O.direct_sum(pos, mass, k, targets=sample)
        errs = [O.rel_rms(O.solve_direct(tr, mass, ng, k, sample)[1], a0) for ng in (2, 4, 6)]
        assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3


def test_user_kernel_cut_off_below_rmin():
    """Pairs closer than side * 2^-32 take the user kernel's values there (a documented
    cut-off of the library's user-kernel interface, mirrored here)."""
    k = erf_kernel(0.02)
    r = np.array([0.0, 2.0 ** -40, 2.0 ** -32, 2.0 ** -20])
    g, f = O.kernel_eval(k, r)
    assert g[0] == g[1] == g[2] and f[0] == f[1] == f[2] and g[3] != g[2]
