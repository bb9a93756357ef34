"""Stage-by-stage parity of the GPU path against the FP64 oracle's plain definitions.

Effective masses (P2G at leaves and virtual boxes, child-to-parent at internal
cells), source-to-target values and the local gridlets after the
parent-to-child pass, element by element on every box / target. FP32 bars:
effective masses within 1e-5 of each box's total mass; source-to-target and
local values within 1e-5 relative RMS of the per-target variation (the part
that carries the force) and 1e-6 of the values themselves.
"""
import numpy as np
import pytest

import oracle as O
from paper_1906_10734_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hpm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_10734_gb300 import hpm as H
    return H


def run(H, w, flags=0, green=None):
    dev = torch.device("cuda:0")
    s = H.Solver(w.max_depth, w.ng, w.eps, w.leaf_max, flags=flags, green=green)
    s(torch.from_numpy(w.pos).to(dev), torch.from_numpy(w.mass).to(dev))
    torch.cuda.synchronize()
    out = {"boxes": s.boxes(), "lists": s.lists(), "masses": s.stage(H.HPM_STAGE_MASSES),
           "m2l": s.stage(H.HPM_STAGE_M2L), "local": s.stage(H.HPM_STAGE_LOCAL)}
    s.close()
    return out


def variation_err(gpu_vals, ref_vals):
    g = gpu_vals - gpu_vals.mean(axis=1, keepdims=True)
    r = ref_vals - ref_vals.mean(axis=1, keepdims=True)
    return float(np.sqrt(np.sum((g - r) ** 2) / np.sum(r * r)))


def check_stages(H, w, flags=0, max_targets=None, seed=0, var_tol=1e-5, green=None, kernel=None):
    """Stage parity; `green` (library) and `kernel` (oracle) name another Green function
    than the workload's Plummer softening. With HPM_FLAG_EXTENDED_GRIDLET the target
    gridlets are compared at their (Ng + 2)^3 widened nodes."""
    g = run(H, w, flags, green)
    kern = kernel if kernel is not None else w.eps
    ext = 1 if flags & H.HPM_FLAG_EXTENDED_GRIDLET else 0
    tr = O.Tree(w.pos, max_depth=w.max_depth, leaf_max=w.leaf_max)
    b = g["boxes"]
    sel = np.flatnonzero(b["level"] >= 2)
    ref_m = O.box_masses(tr, w.mass, w.ng, b["level"][sel], b["key"][sel])
    tot = np.abs(ref_m).sum(axis=1, keepdims=True)
    assert np.max(np.abs(g["masses"] - ref_m) / tot) < 1e-5
    lst = g["lists"]
    tmask = lst["level"] >= 2
    tl, tk = lst["level"][tmask], lst["key"][tmask]
    pick = np.arange(tl.shape[0])
    if max_targets and pick.size > max_targets:
        pick = np.sort(np.random.default_rng(seed).choice(pick.size, max_targets, replace=False))
    m3 = (w.ng + 2 * ext) ** 3
    ref = O.m2l_values(tr, w.mass, w.ng, kern, tl[pick], tk[pick], ext=ext)
    got = g["m2l"][pick, :m3].astype(np.float64) + g["m2l"][pick, m3:].astype(np.float64)
    assert variation_err(got, ref) < var_tol
    assert O.rel_rms(got, ref) < 1e-6
    ref = O.local_values(tr, w.mass, w.ng, kern, tl[pick], tk[pick], ext=ext)
    got = g["local"][pick, :m3].astype(np.float64) + g["local"][pick, m3:].astype(np.float64)
    assert variation_err(got, ref) < var_tol
    assert O.rel_rms(got, ref) < 1e-6


def test_stages_uniform_4096(hpm):
    check_stages(hpm, I.uniform_4096_depth3())


def test_stages_adaptive_plummer(hpm):
    check_stages(hpm, I.small_plummer(12000, 60, leaf_max=16), max_targets=600)


def test_stages_fft_kernel_at_order_4(hpm):
    check_stages(hpm, I.uniform_4096_depth3(), flags=hpm.HPM_FLAG_FFT_M2L)
    check_stages(hpm, I.small_plummer(12000, 62, leaf_max=16), flags=hpm.HPM_FLAG_FFT_M2L, max_targets=400)


def test_stages_generic_kernel_at_order_4(hpm):
    check_stages(hpm, I.uniform_4096_depth3(), flags=hpm.HPM_FLAG_GENERIC_M2L)


def test_stages_xtransform_kernel_at_order_4(hpm):
    check_stages(hpm, I.uniform_4096_depth3(), flags=hpm.HPM_FLAG_XTRANSFORM_M2L)
    check_stages(hpm, I.small_plummer(12000, 61, leaf_max=16), flags=hpm.HPM_FLAG_XTRANSFORM_M2L,
                 max_targets=400)


@pytest.mark.parametrize("ng", [2, 3, 5, 6])
def test_stages_other_orders(hpm, ng):
    w = I.Workload(f"u{ng}", I.uniform_cube(2500, 30 + ng), I.equal_masses(2500), max_depth=3, leaf_max=0,
                   ng=ng, eps=1e-3)
    check_stages(hpm, w, max_targets=200)


def test_stages_order_6_adaptive(hpm):
    check_stages(hpm, I.small_plummer(12000, 63, leaf_max=32, ng=6), max_targets=300)


def test_stages_xtransform_kernel_at_order_6(hpm):
    # full FP32 values on this kernel: the variation bar is a few times their rounding
    w = I.Workload("u6x", I.uniform_cube(2500, 36), I.equal_masses(2500), max_depth=3, leaf_max=0, ng=6, eps=1e-3)
    check_stages(hpm, w, flags=hpm.HPM_FLAG_XTRANSFORM_M2L, max_targets=200, var_tol=3e-5)
