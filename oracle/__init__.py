"""FP64 CPU oracle for the Hierarchical Particle-Mesh FMM (Gnedin 2019).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code
with the GPU solver: the tree and lists below are written from their
definitions with numpy, and the numerics live in ``hpm_oracle.c`` (plain C,
FP64).

Definitions (Sec. 1 and Sec. 2 of the paper; the readings where the paper
is silent are listed in the design notes of the repository):

* Domain: cube [o, o+S)^3, level-l boxes of side L_l = S / 2^l, integer box
  coordinates b in [0, 2^l)^3, centre o + (b + 1/2) L_l.
* A particle's unit coordinate is v = (x - o)/S in FP64; it is out of the
  domain unless 0 <= v <= 1, and v = 1 falls in the last box. Its 21-bit cell
  coordinate is min(floor(v 2^21), 2^21 - 1); level-l coordinates are that
  shifted right by 21 - l.
* Morton key of a level-l box: bit k of (bx, by, bz) goes to bits
  (3k, 3k+1, 3k+2); the low three bits are the child index C = bx + 2 by + 4 bz.
* Particles are sorted by their level-D key (D = max_depth), ties by
  original index.
* Tree (Sec. 1): the root is a cell; a cell splits into its nonempty
  children iff it holds more than ``leaf_max`` particles and its level is
  below D (``leaf_max = 0``: every nonempty cell above level D splits, the
  uniform tree). Cells that do not split are leaves.
* Adaptive reading of the zones ("virtual completion"): at level l the
  source boxes are all nonempty level-l dyadic boxes, including boxes that lie
  inside a coarser leaf. For a cell t at level l >= 2,
  IZ(t) = {nonempty level-l boxes b : Cheb(parent b, parent t) <= 1 and
  Cheb(b, t) >= 2}; for a leaf t, near(t) = {nonempty level-l boxes b :
  Cheb(b, t) <= 1}. On a uniform tree this is the paper's rule.
* IZ of t as a 216-bit mask over the 6^3 block of the children of the
  parent's 3^3 neighbourhood: block origin 2 (parent - 1), bit bx + 6 by + 36 bz.
  Near of a leaf as a 27-bit mask, bit (dx+1) + 3 (dy+1) + 9 (dz+1).
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from .build import build as _build_lib

MORTON_BITS = 21

_lib = None


def lib():
    """Loads (building first if needed) the C part of the oracle."""
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build_lib())
        vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "or_num_threads": ([], i32),
            "or_lagrange": ([i32, f64, vp, vp], None),
            "or_p2g": ([i32, i64, vp, vp, vp, vp, vp, vp, vp], None),
            "or_vandermonde": ([i32, vp], None),
            "or_invert": ([i32, vp, vp], i32),
            "or_moments": ([i32, i64, vp, vp, vp, vp, vp, vp], None),
            "or_p2g_paper": ([i32, i64, vp, vp, vp, vp], None),
            "or_t_paper": ([i32, vp, vp, i32, vp], None),
            "or_m2l_direct": ([i32, i32, vp, i64, vp, vp, vp, vp, vp, vp, vp], None),
            "or_lagrange_ext": ([i32, i32, f64, vp, vp], None),
            "or_fft1d": ([vp, vp, i32, i32, vp, vp], None),
            "or_green_hat": ([i32, vp, f64, vp, vp], None),
            "or_m2l_fft": ([i32, i32, i64, vp, vp, vp, vp, vp, vp], None),
            "or_far_eval": ([i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp], None),
            "or_g2p_paper": ([i32, i64, vp, vp, vp, vp, vp, vp, vp], None),
            "or_p2p": ([vp, i64, vp, vp, vp, vp, vp, vp, vp, vp], None),
            "or_direct": ([vp, i64, vp, i64, vp, vp, vp, vp], None),
            "or_p2p_leaves": ([vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp], None),
            "or_kernel_eval": ([vp, i64, vp, vp, vp], None),
            "or_apply": ([i32, i64, vp, i32, vp, vp], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


class _Arg:
    """A numpy array passed by pointer; the call helper keeps it alive."""

    def __init__(self, a: np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
        self.a = a


def _p(a: np.ndarray) -> _Arg:
    return _Arg(a)


def _call(name: str, *args):
    keep = []
    conv = []
    for a in args:
        if isinstance(a, _Arg):
            keep.append(a.a)
            conv.append(ctypes.c_void_p(a.a.ctypes.data))
        else:
            conv.append(a)
    r = getattr(lib(), name)(*conv)
    del keep
    return r


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def num_threads() -> int:
    return int(_call("or_num_threads"))


# ---------------------------------------------------------------------------
# The Green function (Sec. 4: any radial kernel; Sec. 2.1, Eq. gf)
# ---------------------------------------------------------------------------
_KFN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_void_p)


class _or_kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("eps", ctypes.c_double), ("lam", ctypes.c_double),
                ("rmin", ctypes.c_double), ("user_g", _KFN), ("user_dg", _KFN), ("ctx", ctypes.c_void_p)]


class Kernel:
    """Radial Green function g: Plummer 1/sqrt(r^2 + eps^2), Newton 1/r, Yukawa
    exp(-s/lam)/s with s = sqrt(r^2 + eps^2), or a user C function g(r, ctx) with an
    optional derivative dg(r, ctx). A user kernel is evaluated at r >= rmin (pairs
    closer than rmin take its values there): the library's cut-off is side * 2^-32."""
    PLUMMER, NEWTON, YUKAWA, USER = 0, 1, 2, 3

    def __init__(self, kind=0, eps=0.0, lam=0.0, user_g=None, user_dg=None, ctx=None, rmin=0.0):
        self.kind, self.eps, self.lam, self.rmin = kind, float(eps), float(lam), float(rmin)
        self.user_g, self.user_dg, self.ctx = user_g, user_dg, ctx

    @classmethod
    def plummer(cls, eps):
        return cls(cls.PLUMMER, eps)

    @classmethod
    def newton(cls):
        return cls(cls.NEWTON)

    @classmethod
    def yukawa(cls, lam, eps=0.0):
        return cls(cls.YUKAWA, eps, lam)

    @classmethod
    def user(cls, g, dg=None, ctx=None, side=1.0):
        return cls(cls.USER, user_g=g, user_dg=dg, ctx=ctx, rmin=side * 2.0 ** -32)

    def struct(self) -> _or_kernel:
        k = _or_kernel(self.kind, self.eps, self.lam, self.rmin)
        if self.user_g is not None:
            k.user_g = ctypes.cast(self.user_g, _KFN)
        if self.user_dg is not None:
            k.user_dg = ctypes.cast(self.user_dg, _KFN)
        if self.ctx is not None:
            k.ctx = ctypes.cast(self.ctx, ctypes.c_void_p)
        return k


def _kern(eps_or_kernel):
    """A float is the Plummer softening; a Kernel is passed through. Returns a pointer arg."""
    k = eps_or_kernel if isinstance(eps_or_kernel, Kernel) else Kernel.plummer(float(eps_or_kernel))
    return ctypes.pointer(k.struct())


def kernel_eval(kernel, r):
    """g(r) and F(r) = -g'(r)/r of the oracle's kernel at the distances r."""
    r = _f64(np.atleast_1d(r))
    g, f = np.zeros_like(r), np.zeros_like(r)
    _call("or_kernel_eval", _kern(kernel), r.shape[0], _p(r), _p(g), _p(f))
    return g, f


# ---------------------------------------------------------------------------
# Gridlet basics (Sec. 2.2)
# ---------------------------------------------------------------------------
def nodes(ng: int) -> np.ndarray:
    """x_j = (j + 1/2)/Ng - 1/2."""
    return (np.arange(ng) + 0.5) / ng - 0.5


def lagrange(ng: int, t: float):
    w = np.zeros(ng)
    dw = np.zeros(ng)
    _call("or_lagrange", ng, float(t), _p(w), _p(dw))
    return w, dw


def nodes_ext(ng: int, ext: int) -> np.ndarray:
    """Nodes of the extended gridlet (Sec. 2.5): x_j for j = -ext .. Ng - 1 + ext."""
    return (np.arange(-ext, ng + ext) + 0.5) / ng - 0.5


def lagrange_ext(ng: int, ext: int, t: float):
    ne = ng + 2 * ext
    w = np.zeros(ne)
    dw = np.zeros(ne)
    _call("or_lagrange_ext", ng, int(ext), float(t), _p(w), _p(dw))
    return w, dw


def vandermonde(ng: int) -> np.ndarray:
    m3 = ng ** 3
    A = np.zeros((m3, m3))
    _call("or_vandermonde", ng, _p(A))
    return A


def invert(A: np.ndarray) -> np.ndarray:
    A = _f64(A)
    Ai = np.zeros_like(A)
    if _call("or_invert", A.shape[0], _p(A), _p(Ai)) != 0:
        raise np.linalg.LinAlgError("singular matrix")
    return Ai


def paper_matrices(ng: int):
    """A (Eq. Anp), B = A^{-1}, and the eight child-to-parent T^C of Sec. 2.3."""
    A = vandermonde(ng)
    B = invert(A)
    m3 = ng ** 3
    T = np.zeros((8, m3, m3))
    for c in range(8):
        _call("or_t_paper", ng, _p(A), _p(B), c, _p(T[c]))
    return A, B, T


def child_eval_matrix(ng: int, c: int) -> np.ndarray:
    """E^C[p][n] = ((a^C + x_p)/2)^n: the monomials of Eq. phix at the child's nodes (Sec. 2.4)."""
    x = nodes(ng)
    m3 = ng ** 3
    a = [0.5 if (c >> d) & 1 else -0.5 for d in range(3)]
    E = np.zeros((m3, m3))
    for p in range(m3):
        pc = (p % ng, (p // ng) % ng, p // (ng * ng))
        for n in range(m3):
            nc = (n % ng, (n // ng) % ng, n // (ng * ng))
            v = 1.0
            for d in range(3):
                v *= ((a[d] + x[pc[d]]) / 2.0) ** nc[d]
            E[p, n] = v
    return E


def p2g(ng, begin, end, center, side, spos, smass) -> np.ndarray:
    begin, end, center, side = _i64(begin), _i64(end), _f64(center), _f64(side)
    out = np.zeros((begin.shape[0], ng ** 3))
    _call("or_p2g", ng, begin.shape[0], _p(begin), _p(end), _p(center), _p(side), _p(spos), _p(smass),
                 _p(out))
    return out


def p2g_paper(ng, begin, end, center, side, spos, smass, B) -> np.ndarray:
    begin, end, center, side = _i64(begin), _i64(end), _f64(center), _f64(side)
    nb = begin.shape[0]
    Q = np.zeros((nb, ng ** 3))
    _call("or_moments", ng, nb, _p(begin), _p(end), _p(center), _p(spos), _p(smass), _p(Q))
    out = np.zeros((nb, ng ** 3))
    _call("or_p2g_paper", ng, nb, _p(Q), _p(side), _p(_f64(B)), _p(out))
    return out


def moments(ng, begin, end, center, spos, smass) -> np.ndarray:
    begin, end, center = _i64(begin), _i64(end), _f64(center)
    Q = np.zeros((begin.shape[0], ng ** 3))
    _call("or_moments", ng, begin.shape[0], _p(begin), _p(end), _p(center), _p(spos), _p(smass), _p(Q))
    return Q


def fft1d(x: np.ndarray, sign: int = -1) -> np.ndarray:
    re, im = _f64(np.real(x)), _f64(np.imag(x))
    ore, oim = np.zeros_like(re), np.zeros_like(im)
    _call("or_fft1d", _p(re), _p(im), re.shape[0], sign, _p(ore), _p(oim))
    return ore + 1j * oim


def green_hat(ng: int, eps, h: float):
    """Transform of the kernel (eps: Plummer softening or a Kernel) on the (8 Ng)^3 grid."""
    P = 8 * ng
    re = np.zeros(P ** 3)
    im = np.zeros(P ** 3)
    _call("or_green_hat", P, _kern(eps), float(h), _p(re), _p(im))
    return re, im


def m2l_direct(ng, eps, tcenter, tside, soff, sidx, scenter, sgrid, ext=0) -> np.ndarray:
    """Direct interaction-zone sum at the targets' (Ng + 2 ext)^3 nodes (ext = 1: the
    extended gridlet of Sec. 2.5)."""
    tcenter, tside, soff, sidx = _f64(tcenter), _f64(tside), _i64(soff), _i64(sidx)
    out = np.zeros((tcenter.shape[0], (ng + 2 * ext) ** 3))
    _call("or_m2l_direct", ng, int(ext), _kern(eps), tcenter.shape[0], _p(tcenter), _p(tside), _p(soff), _p(sidx),
                        _p(_f64(scenter)), _p(_f64(sgrid)), _p(out))
    return out


def m2l_fft(ng, blk, tpos, grid, ghat, ext=0) -> np.ndarray:
    blk = np.ascontiguousarray(blk, dtype=np.int32)
    tpos = np.ascontiguousarray(tpos, dtype=np.int32)
    out = np.zeros((blk.shape[0], (ng + 2 * ext) ** 3))
    _call("or_m2l_fft", ng, int(ext), blk.shape[0], _p(blk), _p(tpos), _p(_f64(grid)), _p(_f64(ghat[0])),
                     _p(_f64(ghat[1])), _p(out))
    return out


def far_eval(ng, pos, coff, ccell, ccenter, cside, cphi, ext=0):
    pos = _f64(pos)
    n = pos.shape[0]
    phi = np.zeros(n)
    acc = np.zeros((n, 3))
    _call("or_far_eval", ng, int(ext), n, _p(pos), _p(_i64(coff)), _p(_i64(ccell)), _p(_f64(ccenter)),
                      _p(_f64(cside)), _p(_f64(cphi)), _p(phi), _p(acc))
    return phi, acc


def p2p(eps, tidx, roff, rbeg, rend, spos, smass):
    tidx = _i64(tidx)
    phi = np.zeros(tidx.shape[0])
    acc = np.zeros((tidx.shape[0], 3))
    _call("or_p2p", _kern(eps), tidx.shape[0], _p(tidx), _p(_i64(roff)), _p(_i64(rbeg)), _p(_i64(rend)),
                 _p(spos), _p(smass), _p(phi), _p(acc))
    return phi, acc


def p2p_leaves(eps, lbeg, lend, roff, rbeg, rend, spos, smass):
    """Near field of every particle of each leaf; returns arrays in the sorted order."""
    n = spos.shape[0]
    phi = np.zeros(n)
    acc = np.zeros((n, 3))
    lbeg = _i64(lbeg)
    _call("or_p2p_leaves", _kern(eps), lbeg.shape[0], _p(lbeg), _p(_i64(lend)), _p(_i64(roff)),
                        _p(_i64(rbeg)), _p(_i64(rend)), _p(spos), _p(smass), _p(phi), _p(acc))
    return phi, acc


def direct_sum(pos, mass, eps, targets=None):
    """O(N^2) potential and acceleration at ``targets`` (indices into pos; default all)."""
    pos, mass = _f64(pos), _f64(mass)
    n = pos.shape[0]
    t = _i64(np.arange(n) if targets is None else targets)
    phi = np.zeros(t.shape[0])
    acc = np.zeros((t.shape[0], 3))
    _call("or_direct", _kern(eps), t.shape[0], _p(t), n, _p(pos), _p(mass), _p(phi), _p(acc))
    return phi, acc


# ---------------------------------------------------------------------------
# Keys and tree (Sec. 1)
# ---------------------------------------------------------------------------
class OutOfDomain(ValueError):
    pass


def cell_coords21(pos, origin, side) -> np.ndarray:
    v = (np.asarray(pos, dtype=np.float64) - np.asarray(origin, dtype=np.float64)) / float(side)
    if not np.all((v >= 0.0) & (v <= 1.0)):
        raise OutOfDomain("a particle lies outside [o, o+S]^3")
    i = np.floor(v * float(1 << MORTON_BITS)).astype(np.int64)
    return np.minimum(i, (1 << MORTON_BITS) - 1)


def morton(c: np.ndarray, bits: int) -> np.ndarray:
    """Interleave bit k of (x, y, z) into bits (3k, 3k+1, 3k+2)."""
    c = np.asarray(c, dtype=np.int64)
    key = np.zeros(c.shape[:-1], dtype=np.uint64)
    for k in range(bits):
        for d in range(3):
            key |= ((c[..., d] >> k) & 1).astype(np.uint64) << np.uint64(3 * k + d)
    return key


def demorton(key: np.ndarray, bits: int) -> np.ndarray:
    key = np.asarray(key, dtype=np.uint64)
    c = np.zeros(key.shape + (3,), dtype=np.int64)
    for k in range(bits):
        for d in range(3):
            c[..., d] |= ((key >> np.uint64(3 * k + d)) & np.uint64(1)).astype(np.int64) << k
    return c


class Level:
    """All nonempty boxes of one level, in Morton order."""

    def __init__(self, level, keys, begin, end):
        self.level = level
        self.keys = keys
        self.begin = begin
        self.end = end
        self.coords = demorton(keys, level)
        self.real = np.zeros(keys.shape[0], dtype=bool)
        self.internal = np.zeros(keys.shape[0], dtype=bool)
        self.leaf = np.zeros(keys.shape[0], dtype=bool)

    @property
    def count(self):
        return self.end - self.begin

    def find(self, keys) -> np.ndarray:
        """Index of each key among the nonempty boxes, -1 if absent."""
        keys = np.asarray(keys, dtype=np.uint64)
        if self.keys.shape[0] == 0:
            return np.full(keys.shape, -1, dtype=np.int64)
        i = np.searchsorted(self.keys, keys)
        ic = np.minimum(i, self.keys.shape[0] - 1)
        return np.where(self.keys[ic] == keys, ic, -1).astype(np.int64)


_BLOCK = np.array([(j % 6, (j // 6) % 6, j // 36) for j in range(216)], dtype=np.int64)
_NEAR = np.array([(j % 3 - 1, (j // 3) % 3 - 1, j // 9 - 1) for j in range(27)], dtype=np.int64)


class Tree:
    def __init__(self, pos, origin=(0.0, 0.0, 0.0), side=1.0, max_depth=3, leaf_max=0):
        pos = _f64(pos)
        self.n = n = pos.shape[0]
        self.origin = np.asarray(origin, dtype=np.float64)
        self.side = float(side)
        self.depth = D = int(max_depth)
        self.leaf_max = int(leaf_max)
        c21 = cell_coords21(pos, self.origin, self.side) if n else np.zeros((0, 3), np.int64)
        keyD = morton(c21 >> (MORTON_BITS - D), D)
        self.perm = np.argsort(keyD, kind="stable")
        self.skeys = keyD[self.perm]
        self.spos = np.ascontiguousarray(pos[self.perm])
        self.levels = []
        for l in range(D + 1):
            kl = self.skeys >> np.uint64(3 * (D - l))
            head = np.ones(n, dtype=bool)
            head[1:] = kl[1:] != kl[:-1]
            begin = np.flatnonzero(head).astype(np.int64)
            end = np.append(begin[1:], n).astype(np.int64)
            self.levels.append(Level(l, kl[begin], begin, end))
        for l, lv in enumerate(self.levels):
            if l == 0:
                lv.real[:] = True
            else:
                par = self.levels[l - 1].find(lv.keys >> np.uint64(3))
                lv.real[:] = self.levels[l - 1].internal[par]
            lv.internal[:] = lv.real & (l < D) & (lv.count > self.leaf_max)
            lv.leaf[:] = lv.real & ~lv.internal

    # geometry -----------------------------------------------------------
    def box_side(self, l):
        return self.side / float(1 << l)

    def centers(self, l, idx):
        return self.origin + (self.levels[l].coords[idx] + 0.5) * self.box_side(l)

    def box_of(self, l, s):
        """Index of the level-l box holding sorted particle s."""
        return self.levels[l].find(self.skeys[s] >> np.uint64(3 * (self.depth - l)))

    # lists ----------------------------------------------------------------
    def iz_rows(self, l, tb):
        """IZ of the level-l targets tb as (n, 216) box indices (-1: not a source) and the
        target's position in its parent block (n, 3)."""
        lv = self.levels[l]
        bt = lv.coords[np.asarray(tb, dtype=np.int64)]
        org = 2 * ((bt >> 1) - 1)
        cand = org[:, None, :] + _BLOCK[None, :, :]
        inside = np.all((cand >= 0) & (cand < (1 << l)), axis=2)
        far = np.max(np.abs(cand - bt[:, None, :]), axis=2) >= 2
        keys = morton(np.where(inside[..., None], cand, 0), l)
        idx = lv.find(keys)
        rows = np.where(inside & far & (idx >= 0), idx, -1)
        return rows, bt - org

    def near_rows(self, l, tb):
        """Near zone of the level-l leaves tb as (n, 27) box indices (-1: absent)."""
        lv = self.levels[l]
        bt = lv.coords[np.asarray(tb, dtype=np.int64)]
        cand = bt[:, None, :] + _NEAR[None, :, :]
        inside = np.all((cand >= 0) & (cand < (1 << l)), axis=2)
        keys = morton(np.where(inside[..., None], cand, 0), l)
        idx = lv.find(keys)
        return np.where(inside & (idx >= 0), idx, -1)

    def leaf_of(self, s):
        """(level, box index) of the leaf holding each sorted particle s."""
        s = np.asarray(s, dtype=np.int64)
        lev = np.full(s.shape, -1, dtype=np.int64)
        box = np.full(s.shape, -1, dtype=np.int64)
        for l in range(self.depth + 1):
            b = self.box_of(l, s)
            hit = (lev < 0) & self.levels[l].leaf[b]
            lev[hit] = l
            box[hit] = b[hit]
        return lev, box


def masks_from_rows(rows: np.ndarray) -> np.ndarray:
    """216-wide occupancy rows -> 4 uint64 words per target (bit j of word j // 64)."""
    bits = (rows >= 0)
    out = np.zeros((rows.shape[0], 4), dtype=np.uint64)
    for j in range(rows.shape[1]):
        out[:, j // 64] |= bits[:, j].astype(np.uint64) << np.uint64(j % 64)
    return out


def canonical_lists(tree: Tree, iz_levels=None, chunk: int = 20000) -> dict:
    """Real cells in (level, key) order with particle ranges and leaf flags, the IZ
    mask of every cell at level >= 2 and the near mask of every leaf."""
    lev, key, beg, end, leaf = [], [], [], [], []
    iz, near = [], []
    for l, lv in enumerate(tree.levels):
        r = np.flatnonzero(lv.real)
        lev.append(np.full(r.shape[0], l, dtype=np.int32))
        key.append(lv.keys[r])
        beg.append(lv.begin[r])
        end.append(lv.end[r])
        leaf.append(lv.leaf[r])
        if l >= 2 and (iz_levels is None or l in iz_levels):
            for c in range(0, r.shape[0], chunk):
                rows, _ = tree.iz_rows(l, r[c:c + chunk])
                iz.append(masks_from_rows(rows))
        lf = np.flatnonzero(lv.leaf)
        for c in range(0, lf.shape[0], chunk):
            nr = tree.near_rows(l, lf[c:c + chunk])
            near.append(((nr >= 0).astype(np.uint32) << np.arange(27, dtype=np.uint32)).sum(
                axis=1, dtype=np.uint32))
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)
    return {
        "level": cat(lev, np.int32), "key": cat(key, np.uint64), "begin": cat(beg, np.int64),
        "end": cat(end, np.int64), "leaf": cat(leaf, np.uint8),
        "iz": np.concatenate(iz) if iz else np.zeros((0, 4), np.uint64),
        "near": cat(near, np.uint32), "perm": tree.perm.astype(np.int64),
    }


# ---------------------------------------------------------------------------
# Solve, plain definitions (parity oracle)
# ---------------------------------------------------------------------------
def solve_direct(tree: Tree, mass, ng: int, eps: float, sample=None, ext: int = 0):
    """FP64 HPM by plain definitions: effective masses of every source box by P2G from its
    particles, source-to-target as the direct interaction-zone double sum, far field at a
    particle as the sum of the interpolants of its leaf and the leaf's ancestors down to
    level 2, near field by direct summation over near(leaf).

    ``sample``: original indices of the particles to evaluate (default all).
    ``ext`` = 1: extended target gridlets (Sec. 2.5), the potential evaluated at the
    cell's nodes widened by one node on each side and interpolated with degree Ng + 1.
    Returns (phi, acc) for those particles, in the order given.
    """
    n = tree.n
    smass = _f64(np.asarray(mass, dtype=np.float64)[tree.perm])
    inv = np.empty(n, dtype=np.int64)
    inv[tree.perm] = np.arange(n)
    orig = np.arange(n) if sample is None else np.asarray(sample, dtype=np.int64)
    s = inv[orig]                                # sorted index of each evaluated particle
    ns = s.shape[0]
    leaf_l, leaf_b = tree.leaf_of(s)

    # targets: the leaf and its ancestors at levels >= 2
    tgt_of = {}                                  # (l, box) -> target row
    t_level, t_box = [], []
    chain = [[] for _ in range(ns)]
    for l in range(2, tree.depth + 1):
        b = tree.box_of(l, s)
        on = leaf_l >= l
        ub = np.unique(b[on])
        for bb in ub:
            tgt_of[(l, int(bb))] = len(t_level)
            t_level.append(l)
            t_box.append(int(bb))
        for k in np.flatnonzero(on):
            chain[k].append(tgt_of[(l, int(b[k]))])
    t_level = np.asarray(t_level, dtype=np.int64)
    t_box = np.asarray(t_box, dtype=np.int64)
    nt = t_level.shape[0]

    # sources: union of the interaction zones, one gridlet per (level, box)
    src_of = {}
    s_level, s_box = [], []
    soff = [0]
    sidx = []
    for l in range(2, tree.depth + 1):
        sel = np.flatnonzero(t_level == l)
        if sel.size == 0:
            continue
        rows, _ = tree.iz_rows(l, t_box[sel])
        for bb in np.unique(rows[rows >= 0]):
            src_of[(l, int(bb))] = len(s_level)
            s_level.append(l)
            s_box.append(int(bb))
    per_t = [None] * nt
    for l in range(2, tree.depth + 1):
        sel = np.flatnonzero(t_level == l)
        if sel.size == 0:
            continue
        rows, _ = tree.iz_rows(l, t_box[sel])
        for k, t in enumerate(sel):
            per_t[t] = [src_of[(l, int(bb))] for bb in rows[k][rows[k] >= 0]]
    for t in range(nt):
        sidx.extend(per_t[t])
        soff.append(len(sidx))
    s_level = np.asarray(s_level, dtype=np.int64)
    s_box = np.asarray(s_box, dtype=np.int64)

    def geom(levels, boxes):
        cen = np.zeros((levels.shape[0], 3))
        side = np.zeros(levels.shape[0])
        beg = np.zeros(levels.shape[0], dtype=np.int64)
        end = np.zeros(levels.shape[0], dtype=np.int64)
        for l in np.unique(levels):
            m = levels == l
            cen[m] = tree.centers(int(l), boxes[m])
            side[m] = tree.box_side(int(l))
            beg[m] = tree.levels[int(l)].begin[boxes[m]]
            end[m] = tree.levels[int(l)].end[boxes[m]]
        return cen, side, beg, end

    phi_far = np.zeros(ns)
    acc_far = np.zeros((ns, 3))
    if nt:
        scen, sside, sbeg, send = geom(s_level, s_box)
        sgrid = p2g(ng, sbeg, send, scen, sside, tree.spos, smass) if s_level.size else np.zeros((0, ng ** 3))
        tcen, tside, _, _ = geom(t_level, t_box)
        tphi = m2l_direct(ng, eps, tcen, tside, np.asarray(soff), np.asarray(sidx, dtype=np.int64),
                          scen if s_level.size else np.zeros((0, 3)), sgrid, ext=ext)
        coff = np.zeros(ns + 1, dtype=np.int64)
        coff[1:] = np.cumsum([len(c) for c in chain])
        ccell = np.asarray([x for c in chain for x in c], dtype=np.int64)
        phi_far, acc_far = far_eval(ng, tree.spos[s], coff, ccell, tcen, tside, tphi, ext=ext)

    # near field over near(leaf)
    roff = [0]
    rbeg, rend = [], []
    near_cache = {}
    for k in range(ns):
        key = (int(leaf_l[k]), int(leaf_b[k]))
        if key not in near_cache:
            nr = tree.near_rows(key[0], np.array([key[1]]))[0]
            nr = nr[nr >= 0]
            lv = tree.levels[key[0]]
            near_cache[key] = (lv.begin[nr], lv.end[nr])
        b, e = near_cache[key]
        rbeg.extend(b.tolist())
        rend.extend(e.tolist())
        roff.append(len(rbeg))
    phi_near, acc_near = p2p(eps, s, np.asarray(roff), np.asarray(rbeg, dtype=np.int64),
                             np.asarray(rend, dtype=np.int64), tree.spos, smass)
    return phi_far + phi_near, acc_far + acc_near


# ---------------------------------------------------------------------------
# Solve, the paper's algorithm (timed CPU baseline and second path for pins)
# ---------------------------------------------------------------------------
def solve_fft(tree: Tree, mass, ng: int, eps: float, timings: dict | None = None):
    """FP64 HPM following the paper's four steps: effective masses at leaves and at the
    virtual source boxes from Cartesian multipoles (Eq. mp), child-to-parent with T^C
    (Sec. 2.3), source-to-target by one zero-padded (8 Ng)^3 FFT convolution per target
    (Sec. 2.1), parent-to-child through Eqs. c2pmat/phix (Sec. 2.4), evaluation at the
    particles with the same interpolant, near field by direct summation.
    Returns (phi, acc) in the original particle order."""
    tm = timings if timings is not None else {}
    t0 = time.perf_counter()
    n, D = tree.n, tree.depth
    m3 = ng ** 3
    A, B, T = paper_matrices(ng)
    E = [child_eval_matrix(ng, c) for c in range(8)]
    smass = _f64(np.asarray(mass, dtype=np.float64)[tree.perm])
    tm["precompute"] = time.perf_counter() - t0

    t0 = time.perf_counter()
    # interaction-zone rows of every real cell at level >= 2
    iz = {}
    for l in range(2, D + 1):
        r = np.flatnonzero(tree.levels[l].real)
        if r.size:
            iz[l] = (r,) + tree.iz_rows(l, r)
    # gridlet rows per level: real cells first, then virtual boxes some IZ needs
    row_of = {}
    grids = {}
    for l in range(D, 1, -1):
        lv = tree.levels[l]
        need = np.zeros(lv.keys.shape[0], dtype=bool)
        need[lv.real] = True
        if l in iz:
            rr = iz[l][1]
            need[rr[rr >= 0]] = True
        boxes = np.flatnonzero(need)
        rmap = np.full(lv.keys.shape[0], -1, dtype=np.int64)
        rmap[boxes] = np.arange(boxes.shape[0])
        row_of[l] = rmap
        g = np.zeros((boxes.shape[0], m3))
        by_p2g = boxes[~lv.internal[boxes]]
        if by_p2g.size:
            g[rmap[by_p2g]] = p2g_paper(ng, lv.begin[by_p2g], lv.end[by_p2g], tree.centers(l, by_p2g),
                                        np.full(by_p2g.shape[0], tree.box_side(l)), tree.spos, smass, B)
        inner = boxes[lv.internal[boxes]]
        if inner.size:
            ch = tree.levels[l + 1]
            cb = np.flatnonzero(ch.real)
            par = lv.find(ch.keys[cb] >> np.uint64(3))
            oct_ = (ch.keys[cb] & np.uint64(7)).astype(np.int64)
            for c in range(8):
                sel = oct_ == c
                if not sel.any():
                    continue
                contrib = np.zeros((int(sel.sum()), m3))
                _call("or_apply", m3, contrib.shape[0], _p(T[c]), 0,
                               _p(np.ascontiguousarray(grids[l + 1][row_of[l + 1][cb[sel]]])), _p(contrib))
                np.add.at(g, rmap[par[sel]], contrib)
        grids[l] = g
    tm["upward"] = time.perf_counter() - t0

    t0 = time.perf_counter()
    local = {}
    for l in range(2, D + 1):
        if l not in iz:
            continue
        r, rows, tpos = iz[l]
        blk = np.where(rows >= 0, row_of[l][np.maximum(rows, 0)], -1)
        gh = green_hat(ng, eps, tree.box_side(l) / ng)
        local[l] = m2l_fft(ng, blk, tpos, grids[l], gh)
    tm["m2l"] = time.perf_counter() - t0

    t0 = time.perf_counter()
    # parent-to-child: Phi^C += E^C B^T Phi^P
    BT = np.ascontiguousarray(B.T)
    for l in range(3, D + 1):
        if l not in local or (l - 1) not in local:
            continue
        r = iz[l][0]
        rp = iz[l - 1][0]
        lv = tree.levels[l]
        par = tree.levels[l - 1].find(lv.keys[r] >> np.uint64(3))
        prow = np.searchsorted(rp, par)
        oct_ = (lv.keys[r] & np.uint64(7)).astype(np.int64)
        V = np.zeros((r.shape[0], m3))
        _call("or_apply", m3, r.shape[0], _p(BT), 0, _p(np.ascontiguousarray(local[l - 1][prow])), _p(V))
        for c in range(8):
            sel = np.flatnonzero(oct_ == c)
            if sel.size == 0:
                continue
            add = np.zeros((sel.shape[0], m3))
            _call("or_apply", m3, sel.shape[0], _p(np.ascontiguousarray(E[c])), 0,
                           _p(np.ascontiguousarray(V[sel])), _p(add))
            local[l][sel] += add
    # evaluation at the particles of each leaf (level >= 2)
    phi_s = np.zeros(n)
    acc_s = np.zeros((n, 3))
    s_all = np.arange(n)
    leaf_l, leaf_b = tree.leaf_of(s_all) if n else (np.zeros(0, np.int64), np.zeros(0, np.int64))
    for l in range(2, D + 1):
        if l not in local:
            continue
        on = np.flatnonzero(leaf_l == l)
        if on.size == 0:
            continue
        r = iz[l][0]
        lrow = np.searchsorted(r, leaf_b[on])
        V = np.zeros((r.shape[0], m3))
        _call("or_apply", m3, r.shape[0], _p(BT), 0, _p(np.ascontiguousarray(local[l])), _p(V))
        ph = np.zeros(on.shape[0])
        ac = np.zeros((on.shape[0], 3))
        _call("or_g2p_paper", ng, on.shape[0], _p(np.ascontiguousarray(tree.spos[on])), _p(_i64(lrow)),
                           _p(_f64(tree.centers(l, r))), _p(np.full(r.shape[0], tree.box_side(l))),
                           _p(V), _p(ph), _p(ac))
        phi_s[on] += ph
        acc_s[on] += ac
    tm["downward"] = time.perf_counter() - t0

    t0 = time.perf_counter()
    lb, le, roff, rbeg, rend = [], [], [0], [], []
    for l in range(D + 1):
        lv = tree.levels[l]
        lf = np.flatnonzero(lv.leaf)
        if lf.size == 0:
            continue
        nr = tree.near_rows(l, lf)
        ok = nr >= 0
        lb.append(lv.begin[lf])
        le.append(lv.end[lf])
        roff.append(np.cumsum(ok.sum(axis=1)))
        rbeg.append(lv.begin[nr[ok]])
        rend.append(lv.end[nr[ok]])
    if lb:
        lb, le = np.concatenate(lb), np.concatenate(le)
        cnt = np.concatenate([np.diff(np.concatenate([[0], r])) for r in roff[1:]])
        roff = np.concatenate([[0], np.cumsum(cnt)])
        ph, ac = p2p_leaves(eps, lb, le, roff, np.concatenate(rbeg), np.concatenate(rend),
                            tree.spos, smass)
        phi_s += ph
        acc_s += ac
    tm["near"] = time.perf_counter() - t0

    phi = np.empty(n)
    acc = np.empty((n, 3))
    phi[tree.perm] = phi_s
    acc[tree.perm] = acc_s
    return phi, acc


def rel_rms(x, ref) -> float:
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.sum(ref * ref)
    return float(np.sqrt(np.sum((x - ref) ** 2) / den)) if den > 0 else float(np.sqrt(np.sum(x * x)))


def rel_max(acc, ref) -> float:
    num = np.linalg.norm(np.asarray(acc) - np.asarray(ref), axis=-1)
    den = np.linalg.norm(np.asarray(ref), axis=-1)
    return float(np.max(num / np.maximum(den, 1e-300))) if num.size else 0.0


# ---------------------------------------------------------------------------
# Stage-by-stage reference values (plain definitions), for element-wise parity
# ---------------------------------------------------------------------------
def _boxes(tree: Tree, levels, keys):
    levels = np.asarray(levels, dtype=np.int64)
    keys = np.asarray(keys, dtype=np.uint64)
    idx = np.zeros(levels.shape[0], dtype=np.int64)
    for l in np.unique(levels):
        m = levels == l
        idx[m] = tree.levels[int(l)].find(keys[m])
    if np.any(idx < 0):
        raise KeyError("empty box")
    return idx


def box_masses(tree: Tree, mass, ng, levels, keys):
    """Effective masses of the given (level, key) boxes straight from their particles
    (Sec. 2.2, Lagrange form of Eq. mp)."""
    smass = _f64(np.asarray(mass, dtype=np.float64)[tree.perm])
    levels = np.asarray(levels, dtype=np.int64)
    idx = _boxes(tree, levels, keys)
    beg = np.zeros_like(idx)
    end = np.zeros_like(idx)
    cen = np.zeros((idx.shape[0], 3))
    side = np.zeros(idx.shape[0])
    for l in np.unique(levels):
        m = levels == l
        lv = tree.levels[int(l)]
        beg[m], end[m] = lv.begin[idx[m]], lv.end[idx[m]]
        cen[m] = tree.centers(int(l), idx[m])
        side[m] = tree.box_side(int(l))
    return p2g(ng, beg, end, cen, side, tree.spos, smass)


def m2l_values(tree: Tree, mass, ng, eps, levels, keys, ext=0):
    """Source-to-target values Phi_{t,p} of the given target cells, direct IZ sum (Sec. 2.1), at
    the (Ng + 2 ext)^3 nodes of their (extended, Sec. 2.5) gridlets."""
    levels = np.asarray(levels, dtype=np.int64)
    keys = np.asarray(keys, dtype=np.uint64)
    idx = _boxes(tree, levels, keys)
    out = np.zeros((levels.shape[0], (ng + 2 * ext) ** 3))
    for l in np.unique(levels):
        sel = np.flatnonzero(levels == l)
        rows, _ = tree.iz_rows(int(l), idx[sel])
        src = np.unique(rows[rows >= 0])
        lv = tree.levels[int(l)]
        grid = box_masses(tree, mass, ng, np.full(src.shape[0], l), lv.keys[src]) if src.size else np.zeros((0, ng ** 3))
        pos_of = {int(b): k for k, b in enumerate(src)}
        soff = [0]
        sidx = []
        for r in rows:
            sidx.extend(pos_of[int(b)] for b in r[r >= 0])
            soff.append(len(sidx))
        out[sel] = m2l_direct(ng, eps, tree.centers(int(l), idx[sel]), np.full(sel.shape[0], tree.box_side(int(l))),
                              np.asarray(soff), np.asarray(sidx, dtype=np.int64),
                              tree.centers(int(l), src) if src.size else np.zeros((0, 3)), grid, ext=ext)
    return out


def local_values(tree: Tree, mass, ng, eps, levels, keys, ext=0):
    """Local gridlet of each target after the parent-to-child pass: the sum over the target
    and its ancestors down to level 2 of their interpolants (Eqs. c2pmat/phix), evaluated at
    the target's nodes (Sec. 2.4: Phi^C_p = Phi^P((a^C + x_p)/2) plus its own values)."""
    levels = np.asarray(levels, dtype=np.int64)
    keys = np.asarray(keys, dtype=np.uint64)
    chain_l, chain_k = [], []
    for l, k in zip(levels, keys):
        for la in range(2, int(l) + 1):
            chain_l.append(la)
            chain_k.append(int(k) >> (3 * (int(l) - la)))
    cl = np.asarray(chain_l, dtype=np.int64)
    ck = np.asarray(chain_k, dtype=np.uint64)
    uniq = {}
    for a, b in zip(cl, ck):
        uniq.setdefault((int(a), int(b)), len(uniq))
    ul = np.asarray([a for a, _ in uniq], dtype=np.int64)
    uk = np.asarray([b for _, b in uniq], dtype=np.uint64)
    phi_c = m2l_values(tree, mass, ng, eps, ul, uk, ext=ext)
    idx_c = _boxes(tree, ul, uk)
    cen_c = np.zeros((ul.shape[0], 3))
    side_c = np.zeros(ul.shape[0])
    for l in np.unique(ul):
        m = ul == l
        cen_c[m] = tree.centers(int(l), idx_c[m])
        side_c[m] = tree.box_side(int(l))
    x = nodes_ext(ng, ext)
    ne = ng + 2 * ext
    m3 = ne ** 3
    node_off = np.array([[x[p % ne], x[(p // ne) % ne], x[p // (ne * ne)]] for p in range(m3)])
    idx = _boxes(tree, levels, keys)
    pts = np.zeros((levels.shape[0] * m3, 3))
    coff = [0]
    ccell = []
    for t, (l, k) in enumerate(zip(levels, keys)):
        c = tree.centers(int(l), [idx[t]])[0]
        pts[t * m3:(t + 1) * m3] = c + tree.box_side(int(l)) * node_off
        chain = [uniq[(la, int(k) >> (3 * (int(l) - la)))] for la in range(2, int(l) + 1)]
        for _ in range(m3):
            ccell.extend(chain)
            coff.append(len(ccell))
    phi, _ = far_eval(ng, pts, np.asarray(coff), np.asarray(ccell, dtype=np.int64), cen_c, side_c, phi_c, ext=ext)
    return phi.reshape(levels.shape[0], m3)
