"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties an oracle routine to something other than itself: a worked
closed form (tests/golden), an identity the paper states, an invariant, a
special case with a textbook answer, or brute force on a tiny input.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1906_10734_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_box_particles(rng, n, center, side):
    pos = center + (rng.random((n, 3)) - 0.5) * side
    mass = rng.random(n) + 0.1
    return np.ascontiguousarray(pos), mass


# ---------------------------------------------------------------------------
# Sec. 2.2: nodes, Lagrange basis, Vandermonde inverse
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ng", [1, 2, 3, 4, 5, 6, 8])
def test_lagrange_interpolates_monomials(ng):
    x = O.nodes(ng)
    for j in range(ng):
        w, _ = O.lagrange(ng, x[j])
        assert np.allclose(w, np.eye(ng)[j], atol=1e-13)
    for t in np.linspace(-0.5, 0.5, 7):
        w, dw = O.lagrange(ng, t)
        for n in range(ng):                       # sum_j x_j^n ell_j(t) = t^n
            assert abs(np.dot(x ** n, w) - t ** n) < 1e-12
            dref = n * t ** (n - 1) if n > 0 else 0.0
            assert abs(np.dot(x ** n, dw) - dref) < 1e-10


def test_ng2_closed_forms_golden():
    g = json.load(open(os.path.join(GOLDEN, "ng2_closed_forms.json")))
    assert np.allclose(O.nodes(2), g["nodes"], atol=0)
    A, B, T = O.paper_matrices(2)
    b1 = np.array(g["B1d"])
    B3 = np.einsum("ad,be,cf->cbafed", b1, b1, b1).reshape(8, 8)   # p = px + 2 py + 4 pz
    assert np.allclose(B, B3, atol=1e-14)
    tm, tp = np.array(g["T_minus_1d"]), np.array(g["T_plus_1d"])
    for c in range(8):
        f = [tp if (c >> d) & 1 else tm for d in range(3)]
        T3 = np.einsum("ad,be,cf->cbafed", f[0], f[1], f[2]).reshape(8, 8)
        assert np.allclose(T[c], T3, atol=1e-14)
    assert abs(T[0][0, 0] - g["T3d_child0_p0_q0"]) < 1e-14
    assert abs(T[7][7, 7] - g["T3d_child7_p7_q7"]) < 1e-14
    M = O.p2g(2, [0], [1], np.zeros((1, 3)), [1.0], np.zeros((1, 3)), np.ones(1))
    assert np.allclose(M[0], g["unit_mass_at_center_gridlet"], atol=1e-15)


@pytest.mark.parametrize("ng", [1, 2, 3, 4, 5, 6])
def test_effective_masses_reproduce_moments(ng):
    """Eq. qn/Anp: sum_p M_p x_p^n equals sum_i m_i xi_i^n for every n in {0..Ng-1}^3."""
    rng = np.random.default_rng(ng)
    c, L = np.array([0.3, -1.2, 2.0]), 0.37
    pos, mass = rand_box_particles(rng, 50, c, L)
    M = O.p2g(ng, [0], [50], c[None], [L], pos, mass)[0]
    x = O.nodes(ng)
    xi = (pos - c) / L
    worst = 0.0
    for nz in range(ng):
        for ny in range(ng):
            for nx in range(ng):
                lhs = sum(M[i + ng * (j + ng * k)] * x[i] ** nx * x[j] ** ny * x[k] ** nz
                          for k in range(ng) for j in range(ng) for i in range(ng))
                rhs = np.sum(mass * xi[:, 0] ** nx * xi[:, 1] ** ny * xi[:, 2] ** nz)
                worst = max(worst, abs(lhs - rhs) / np.sum(mass))
    assert worst < 1e-13
    assert abs(M.sum() - mass.sum()) < 1e-12 * mass.sum()          # monopole


@pytest.mark.parametrize("ng", [2, 3, 4, 5])
def test_paper_form_p2g_equals_lagrange_form(ng):
    """Eq. mp with the Cartesian multipoles of Eq. cm and B = A^{-1} gives the Lagrange weights."""
    rng = np.random.default_rng(10 + ng)
    c, L = np.array([0.5, 0.5, 0.5]), 0.125
    pos, mass = rand_box_particles(rng, 40, c, L)
    A, B, _ = O.paper_matrices(ng)
    assert np.allclose(B @ A, np.eye(ng ** 3), atol=1e-9)
    m1 = O.p2g(ng, [0], [40], c[None], [L], pos, mass)
    m2 = O.p2g_paper(ng, [0], [40], c[None], [L], pos, mass, B)
    cond = np.linalg.cond(A)
    assert np.max(np.abs(m1 - m2)) < 1e-15 * cond * np.sum(mass) * 10


@pytest.mark.parametrize("ng", [2, 3, 4])
def test_t_matrix_paper_formula_is_lagrange_closed_form(ng):
    """Sec. 2.3: T^C_pq from the double sum equals prod_d ell_{p_d}((a_d + x_{q_d})/2)."""
    _, _, T = O.paper_matrices(ng)
    x = O.nodes(ng)
    for c in range(8):
        a = [0.5 if (c >> d) & 1 else -0.5 for d in range(3)]
        one = [np.array([O.lagrange(ng, (a[d] + x[q]) / 2)[0] for q in range(ng)]).T for d in range(3)]
        T3 = np.einsum("ad,be,cf->cbafed", one[0], one[1], one[2]).reshape(ng ** 3, ng ** 3)
        assert np.max(np.abs(T[c] - T3)) < 1e-10


@pytest.mark.parametrize("ng", [2, 3, 4])
def test_child_to_parent_is_exact(ng):
    """sum_C T^C M^C with the children's P2G equals the parent's P2G from its particles."""
    rng = np.random.default_rng(20 + ng)
    cp, Lp = np.array([0.5, 0.5, 0.5]), 0.5
    pos, mass = rand_box_particles(rng, 200, cp, Lp)
    _, _, T = O.paper_matrices(ng)
    Mp = O.p2g(ng, [0], [200], cp[None], [Lp], pos, mass)[0]
    acc = np.zeros(ng ** 3)
    for c in range(8):
        off = np.array([(c >> d) & 1 for d in range(3)]) - 0.5
        cc = cp + off * Lp / 2
        inside = np.all(np.abs(pos - cc) <= Lp / 4, axis=1)
        sp, sm = np.ascontiguousarray(pos[inside]), mass[inside]
        Mc = O.p2g(ng, [0], [sp.shape[0]], cc[None], [Lp / 2], sp, sm)[0]
        acc += T[c] @ Mc
    assert np.max(np.abs(acc - Mp)) < 1e-12 * mass.sum()


@pytest.mark.parametrize("ng", [2, 4])
def test_every_box_equals_child_to_parent_of_its_children_adaptive(ng):
    """On an adaptive tree, every nonempty box at level >= 2 (real cells and the virtual
    boxes inside coarser leaves alike) has P2G equal to sum_C T^C M^C of its nonempty
    children's P2G (Sec. 2.3): the child-to-parent transform can stand in for P2G on any
    box whose children are all present, which is how the GPU path fills expanded boxes."""
    w = I.small_plummer(4000, 17, leaf_max=16, max_depth=7)
    tr = O.Tree(w.pos, max_depth=w.max_depth, leaf_max=w.leaf_max)
    smass = w.mass[tr.perm]
    _, _, T = O.paper_matrices(ng)
    checked = virtual = 0
    for l in range(2, tr.depth):
        lv, ch = tr.levels[l], tr.levels[l + 1]
        pb, cb = np.arange(lv.keys.shape[0]), np.arange(ch.keys.shape[0])
        Mp = O.p2g(ng, lv.begin, lv.end, tr.centers(l, pb), np.full(pb.size, tr.box_side(l)), tr.spos, smass)
        Mc = O.p2g(ng, ch.begin, ch.end, tr.centers(l + 1, cb), np.full(cb.size, tr.box_side(l + 1)), tr.spos,
                   smass)
        par = lv.find(ch.keys >> np.uint64(3))
        assert np.all(par >= 0)
        octant = (ch.keys & np.uint64(7)).astype(np.int64)
        acc = np.zeros_like(Mp)
        for c in range(8):
            sel = octant == c
            np.add.at(acc, par[sel], Mc[sel] @ T[c].T)
        box_mass = np.add.reduceat(smass, lv.begin) if lv.begin.size else np.zeros(0)
        assert np.max(np.abs(acc - Mp) / box_mass[:, None]) < 1e-12
        checked += pb.size
        virtual += int(np.count_nonzero(~lv.real))
    assert checked > 100 and virtual > 10


@pytest.mark.parametrize("ng", [2, 3, 4])
def test_parent_to_child_is_transpose_of_child_to_parent(ng):
    """Sec. 2.4: evaluating Eq. phix at (a^C + x_p)/2 after Eq. c2pmat is (T^C)^T."""
    _, B, T = O.paper_matrices(ng)
    for c in range(8):
        E = O.child_eval_matrix(ng, c)
        assert np.max(np.abs(E @ B.T - T[c].T)) < 1e-10


# ---------------------------------------------------------------------------
# Sec. 2.1: FFT, Green function, the convolution
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [8, 12, 16, 24, 32, 40, 48, 56, 64])
def test_fft_matches_dft_definition(n):
    rng = np.random.default_rng(n)
    x = rng.random(n) + 1j * rng.random(n)
    k = np.arange(n)
    dft = np.exp(-2j * np.pi * np.outer(k, k) / n) @ x
    assert np.max(np.abs(O.fft1d(x, -1) - dft)) < 1e-12 * n
    assert np.max(np.abs(O.fft1d(dft, +1) / n - x)) < 1e-12 * n


def _level_case(ng, eps, seed=3, n=3000, depth=3):
    pos = I.uniform_cube(n, seed)
    mass = I.equal_masses(n)
    tr = O.Tree(pos, max_depth=depth, leaf_max=0)
    lv = tr.levels[depth]
    allb = np.arange(lv.keys.shape[0])
    grid = O.p2g(ng, lv.begin, lv.end, tr.centers(depth, allb), np.full(allb.size, tr.box_side(depth)),
                 tr.spos, mass[tr.perm])
    return tr, lv, allb, grid


@pytest.mark.parametrize("ng,eps", [(1, 0.0), (2, 0.0), (2, 1e-2), (3, 0.0), (4, 1e-3)])
def test_fft_convolution_equals_direct_sum_all_parities(ng, eps):
    """The (8 Ng)^3 periodic convolution with |i|_p equals the direct IZ double sum (Sec. 2.1)."""
    depth = 3
    tr, lv, allb, grid = _level_case(ng, eps, depth=depth)
    real = np.flatnonzero(lv.real)
    octs = (lv.keys[real] & np.uint64(7)).astype(int)
    pick = np.concatenate([real[octs == c][:3] for c in range(8)])
    assert len(set((lv.keys[pick] & np.uint64(7)).tolist())) == 8
    rows, tpos = tr.iz_rows(depth, pick)
    h = tr.box_side(depth) / ng
    out = O.m2l_fft(ng, rows, tpos, grid, O.green_hat(ng, eps, h))
    soff = np.concatenate([[0], np.cumsum((rows >= 0).sum(1))])
    ref = O.m2l_direct(ng, eps, tr.centers(depth, pick), np.full(pick.size, tr.box_side(depth)), soff,
                       rows[rows >= 0], tr.centers(depth, allb), grid)
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))


def test_green_value_at_zero_offset_does_not_reach_targets():
    """G(0) is only a 'softened' placeholder (Sec. 2.1): changing it leaves target values unchanged."""
    ng, eps, depth = 2, 0.0, 3
    tr, lv, allb, grid = _level_case(ng, eps, depth=depth)
    pick = np.flatnonzero(lv.real)[:40]
    rows, tpos = tr.iz_rows(depth, pick)
    h = tr.box_side(depth) / ng
    P = 8 * ng
    g = np.zeros((P, P, P))
    d = np.minimum(np.arange(P), P - np.arange(P))
    dz, dy, dx = np.meshgrid(d, d, d, indexing="ij")
    r = h * np.sqrt(dx ** 2 + dy ** 2 + dz ** 2)
    outs = []
    for g0 in (1.0 / h, 123.0, 0.0):
        g = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), g0)
        gh = np.fft.fftn(g).reshape(-1)                 # x fastest after the C-order flatten of [z][y][x]
        outs.append(O.m2l_fft(ng, rows, tpos, grid, (gh.real.copy(), gh.imag.copy())))
    scale = np.max(np.abs(outs[0]))
    assert np.max(np.abs(outs[1] - outs[0])) < 1e-12 * scale
    assert np.max(np.abs(outs[2] - outs[0])) < 1e-12 * scale


# ---------------------------------------------------------------------------
# Tree and lists: brute force and the partition property
# ---------------------------------------------------------------------------
def _brute_iz(tr, l, tb):
    """IZ by the definition: scan every nonempty level-l box."""
    lv = tr.levels[l]
    bt = lv.coords[tb]
    out = []
    for b in range(lv.keys.shape[0]):
        cb = lv.coords[b]
        if np.max(np.abs((cb >> 1) - (bt >> 1))) <= 1 and np.max(np.abs(cb - bt)) >= 2:
            out.append(b)
    return sorted(out)


@pytest.mark.parametrize("leaf_max,depth,seed", [(0, 3, 1), (4, 6, 2), (8, 8, 3)])
def test_iz_block_enumeration_equals_definition(leaf_max, depth, seed):
    pos = I.plummer_sphere(600, seed) if leaf_max else I.uniform_cube(600, seed)
    tr = O.Tree(pos, max_depth=depth, leaf_max=leaf_max)
    for l in range(2, depth + 1):
        real = np.flatnonzero(tr.levels[l].real)[:25]
        if real.size == 0:
            continue
        rows, _ = tr.iz_rows(l, real)
        for k, t in enumerate(real):
            assert sorted(rows[k][rows[k] >= 0].tolist()) == _brute_iz(tr, l, t)


@pytest.mark.parametrize("leaf_max,depth,seed,n", [(0, 4, 4, 900), (3, 9, 5, 700), (16, 12, 6, 3000)])
def test_near_and_iz_chain_partition_all_particles(leaf_max, depth, seed, n):
    """For every leaf, near(leaf) and the IZs of the leaf and its ancestors (levels >= 2)
    hold every particle exactly once."""
    pos = I.plummer_sphere(n, seed) if leaf_max else I.uniform_cube(n, seed)
    tr = O.Tree(pos, max_depth=depth, leaf_max=leaf_max)
    nleaf = 0
    for L, lv in enumerate(tr.levels):
        for t in np.flatnonzero(lv.leaf)[:60]:
            cover = np.zeros(n, dtype=int)
            nr = tr.near_rows(L, np.array([t]))[0]
            for b in nr[nr >= 0]:
                cover[lv.begin[b]:lv.end[b]] += 1
            s = lv.begin[t]
            for l in range(2, L + 1):
                tb = tr.box_of(l, np.array([s]))
                rows, _ = tr.iz_rows(l, tb)
                for b in rows[0][rows[0] >= 0]:
                    cover[tr.levels[l].begin[b]:tr.levels[l].end[b]] += 1
            assert np.all(cover == 1)
            nleaf += 1
    assert nleaf > 10


def test_tree_split_rule_and_key_convention():
    pos = np.array([[0.1, 0.1, 0.1], [0.9, 0.1, 0.1], [0.1, 0.9, 0.1], [0.1, 0.1, 0.9], [1.0, 1.0, 1.0]])
    tr = O.Tree(pos, max_depth=1, leaf_max=0)
    lv = tr.levels[1]
    # child index C = bx + 2 by + 4 bz; x = 1.0 falls in the last box
    assert lv.keys.tolist() == [0, 1, 2, 4, 7]
    assert tr.perm.tolist() == [0, 1, 2, 3, 4]
    with pytest.raises(O.OutOfDomain):
        O.Tree(np.array([[1.0 + 1e-12, 0.5, 0.5]]), max_depth=2)
    with pytest.raises(O.OutOfDomain):
        O.Tree(np.array([[-1e-300, 0.5, 0.5]]), max_depth=2)
    with pytest.raises(O.OutOfDomain):
        O.Tree(np.array([[np.nan, 0.5, 0.5]]), max_depth=2)
    # adaptive: a cell with more than leaf_max particles splits
    pos = I.plummer_sphere(500, 9)
    tr = O.Tree(pos, max_depth=10, leaf_max=20)
    for l, lv in enumerate(tr.levels):
        assert np.all(lv.count[lv.internal] > 20)
        assert np.all((lv.count[lv.leaf] <= 20) | (l == 10))
    assert sum(int(lv.count[lv.leaf].sum()) for lv in tr.levels) == 500


# ---------------------------------------------------------------------------
# Whole solve: special cases and invariants
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("depth", [0, 1])
def test_shallow_tree_is_exact_direct_sum(depth):
    """With max_depth <= 1 every pair is near: HPM equals the all-pairs sum."""
    pos, mass = I.uniform_cube(300, 11), I.equal_masses(300) * np.linspace(0.5, 1.5, 300)
    tr = O.Tree(pos, max_depth=depth, leaf_max=0)
    phi, acc = O.solve_direct(tr, mass, 4, 1e-3)
    p0, a0 = O.direct_sum(pos, mass, 1e-3)
    assert O.rel_rms(acc, a0) < 1e-14 and O.rel_rms(phi, p0) < 1e-14


def test_monopole_gridlet_is_textbook_point_mass_sum():
    """Ng = 1: each box is one mass sum(m) at its centre; the far potential of a particle is
    -sum over its chain's IZ boxes of M_b / |c_t - c_b| (constant over the target cell)."""
    pos, mass = I.uniform_cube(800, 12), I.equal_masses(800)
    depth, eps = 3, 0.0
    tr = O.Tree(pos, max_depth=depth, leaf_max=0)
    phi, acc = O.solve_direct(tr, mass, 1, eps)
    smass = mass[tr.perm]
    inv = np.empty(800, dtype=np.int64)
    inv[tr.perm] = np.arange(800)
    for i in [0, 17, 333, 799]:
        s = inv[i]
        far = 0.0
        for l in range(2, depth + 1):
            tb = tr.box_of(l, np.array([s]))[0]
            ct = tr.centers(l, [tb])[0]
            rows, _ = tr.iz_rows(l, np.array([tb]))
            for b in rows[0][rows[0] >= 0]:
                lvl = tr.levels[l]
                Mb = smass[lvl.begin[b]:lvl.end[b]].sum()
                far -= Mb / np.linalg.norm(ct - tr.centers(l, [b])[0])
        lv = tr.levels[depth]
        tb = tr.box_of(depth, np.array([s]))[0]
        nr = tr.near_rows(depth, np.array([tb]))[0]
        near = 0.0
        for b in nr[nr >= 0]:
            for j in range(lv.begin[b], lv.end[b]):
                if j != s:
                    near -= smass[j] / np.linalg.norm(tr.spos[s] - tr.spos[j])
        assert abs(phi[i] - (far + near)) < 1e-12 * abs(far + near)


def test_linearity_in_mass():
    w = I.small_plummer(3000, 13, leaf_max=16)
    tr = O.Tree(w.pos, max_depth=w.max_depth, leaf_max=w.leaf_max)
    rng = np.random.default_rng(0)
    m1, m2 = rng.random(w.n), rng.random(w.n)
    sample = np.arange(0, w.n, 37)
    p1, a1 = O.solve_direct(tr, m1, 3, w.eps, sample)
    p2, a2 = O.solve_direct(tr, m2, 3, w.eps, sample)
    p3, a3 = O.solve_direct(tr, m1 + m2, 3, w.eps, sample)
    assert O.rel_rms(a3, a1 + a2) < 1e-13 and O.rel_rms(p3, p1 + p2) < 1e-13


def test_mirror_symmetry():
    """x -> 1 - x mirrors the tree; the potential is unchanged and a_x flips sign."""
    pos = I.uniform_cube(1500, 14)
    mass = I.equal_masses(1500)
    mir = pos.copy()
    mir[:, 0] = 1.0 - mir[:, 0]
    t1 = O.Tree(pos, max_depth=3, leaf_max=0)
    t2 = O.Tree(mir, max_depth=3, leaf_max=0)
    p1, a1 = O.solve_direct(t1, mass, 4, 1e-3)
    p2, a2 = O.solve_direct(t2, mass, 4, 1e-3)
    a2[:, 0] *= -1
    assert O.rel_rms(a2, a1) < 1e-12 and O.rel_rms(p2, p1) < 1e-12


def test_distant_point_mass_gives_minus_m_over_r():
    """A lone source seen through the interaction zone gives -m/r and -m r/r^3 within the
    truncation error, which falls as Ng grows (Sec. 2.2: Ng^3 moments are reproduced)."""
    rng = np.random.default_rng(15)
    errs = {}
    for ng in (2, 4, 6, 8):
        e = []
        for trial in range(30):
            src = rng.random(3)
            tgt = rng.random(3)
            pos = np.stack([src, tgt])
            tr = O.Tree(pos, max_depth=4, leaf_max=0)
            lv = tr.levels[4]
            if np.max(np.abs(lv.coords[0] - lv.coords[1])) <= 1:
                continue                                # near pair: no far field
            phi, acc = O.solve_direct(tr, np.array([1.0, 1e-300]), ng, 0.0, sample=[1])
            d = tgt - src
            r = np.linalg.norm(d)
            e.append(np.linalg.norm(acc[0] + d / r ** 3) / (1 / r ** 2))
            assert abs(phi[0] + 1 / r) < 0.05 / r
        errs[ng] = float(np.sqrt(np.mean(np.square(e))))
    assert errs[2] > errs[4] > errs[6] > errs[8]
    assert errs[4] < 3e-2 and errs[6] < 3e-3 and errs[8] < 3e-4


def test_far_eval_reproduces_tensor_polynomials():
    """A degree <= Ng-1 tensor polynomial given at the nodes is evaluated exactly, with its
    analytic gradient (Eq. phix)."""
    ng = 4
    rng = np.random.default_rng(16)
    coef = rng.random((ng, ng, ng))
    x = O.nodes(ng)
    c, L = np.array([0.2, 0.3, 0.4]), 0.25

    def poly(xi):
        v = 0.0
        g = np.zeros(3)
        for a in range(ng):
            for b in range(ng):
                for k in range(ng):
                    v += coef[a, b, k] * xi[0] ** a * xi[1] ** b * xi[2] ** k
                    g[0] += coef[a, b, k] * (a * xi[0] ** (a - 1) if a else 0) * xi[1] ** b * xi[2] ** k
                    g[1] += coef[a, b, k] * xi[0] ** a * (b * xi[1] ** (b - 1) if b else 0) * xi[2] ** k
                    g[2] += coef[a, b, k] * xi[0] ** a * xi[1] ** b * (k * xi[2] ** (k - 1) if k else 0)
        return v, g

    vals = np.array([poly((x[p % ng], x[(p // ng) % ng], x[p // (ng * ng)]))[0] for p in range(ng ** 3)])
    pts = c + (rng.random((10, 3)) - 0.5) * L
    phi, acc = O.far_eval(ng, pts, np.arange(11), np.zeros(10), c[None], [L], vals[None])
    for k in range(10):
        v, g = poly((pts[k] - c) / L)
        assert abs(phi[k] - v) < 1e-12
        assert np.allclose(acc[k], -g / L, atol=1e-10)


def test_hpm_error_against_all_pairs_is_method_sized():
    """4096 uniform particles, depth 3, Ng = 4, eps = 1e-3: the FP64 HPM differs from the
    all-pairs sum by the method's truncation error only (well below the single-pair RMS
    bound of a few 1e-3 at Ng = 4, and far above rounding)."""
    w = I.uniform_4096_depth3()
    tr = O.Tree(w.pos, max_depth=3, leaf_max=0)
    phi, acc = O.solve_direct(tr, w.mass, 4, w.eps)
    p0, a0 = O.direct_sum(w.pos, w.mass, w.eps)
    e = O.rel_rms(acc, a0)
    assert 1e-5 < e < 1e-2
    pf, af = O.solve_fft(tr, w.mass, 4, w.eps)
    assert O.rel_rms(af, acc) < 1e-11 and O.rel_rms(pf, phi) < 1e-12


def test_paper_pipeline_equals_plain_definitions_adaptive():
    """M2M by T^C, FFT M2L and L2L by Eqs. c2pmat/phix reproduce the plain definitions on an
    adaptive tree with virtual source boxes."""
    w = I.small_plummer(5000, 17, leaf_max=16)
    tr = O.Tree(w.pos, max_depth=w.max_depth, leaf_max=w.leaf_max)
    pd, ad = O.solve_direct(tr, w.mass, 3, w.eps)
    pf, af = O.solve_fft(tr, w.mass, 3, w.eps)
    assert O.rel_rms(af, ad) < 1e-11 and O.rel_rms(pf, pd) < 1e-12


def test_generators_follow_their_distributions():
    u = I.uniform01(5, 0, 200000)
    assert abs(u.mean() - 0.5) < 5e-3 and u.min() >= 0 and u.max() < 1
    assert np.array_equal(I.uniform01(5, 100, 10), u[100:110])     # counter-based
    p = I.plummer_sphere(200000, 6)
    r = np.linalg.norm(p - 0.5, axis=1)
    a, rmax = 0.05, 0.5
    m = lambda x: x ** 3 / (x * x + a * a) ** 1.5
    for rr in (0.02, 0.05, 0.1, 0.3):
        assert abs(np.mean(r <= rr) - m(rr) / m(rmax)) < 5e-3
    assert p.min() >= 0.0 and p.max() <= 1.0
