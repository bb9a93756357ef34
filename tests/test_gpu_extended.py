"""Widened target gridlets (HPM_FLAG_EXTENDED_GRIDLET, Sec. 2.5) on the GPU against the
FP64 oracle's widened solve: source-to-target values at the (Ng + 2)^3 nodes, the
degree-(Ng + 1) local expansion, and the fields, held to the 1e-5 bar for every order
the flag accepts (Ng <= 6). The widened nodes enclose the cell, so the local expansion
is evaluated by interpolation only, never by extrapolation beyond its outer nodes: its
amplification of the FP32 values' noise stays small even at 8 nodes per axis."""
import numpy as np
import pytest

import oracle as O
from paper_1906_10734_gb300 import inputs as I
from test_gpu_parity import TOL, gpu_solve
from test_gpu_stages import check_stages

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hpm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_10734_gb300 import hpm as H
    return H


@pytest.mark.parametrize("ng", [1, 2, 3, 4, 5, 6])
def test_widened_fields_uniform(hpm, ng):
    pos, mass = I.uniform_cube(2500, 50 + ng), I.equal_masses(2500)
    phi, acc, _ = gpu_solve(hpm, pos, mass, 3, ng, 1e-3, 0, flags=hpm.HPM_FLAG_EXTENDED_GRIDLET)
    tr = O.Tree(pos, max_depth=3, leaf_max=0)
    sample = np.arange(0, 2500, 5)
    p_ref, a_ref = O.solve_direct(tr, mass, ng, 1e-3, sample, ext=1)
    p_std, a_std = O.solve_direct(tr, mass, ng, 1e-3, sample)
    p_dir, a_dir = O.direct_sum(pos, mass, 1e-3, targets=sample)
    e = O.rel_rms(acc[sample], a_ref)
    print(f"Ng={ng} widened: FP32 vs FP64 {e:.3e}; method error widened {O.rel_rms(a_ref, a_dir):.3e}, "
          f"standard {O.rel_rms(a_std, a_dir):.3e}")
    assert e < TOL and O.rel_rms(phi[sample], p_ref) < TOL
    # the widening reduces the method's truncation error (Sec. 2.5)
    assert ng == 1 or O.rel_rms(a_ref, a_dir) < O.rel_rms(a_std, a_dir)


def test_widened_fields_adaptive_plummer(hpm):
    w = I.small_plummer(12000, 52, leaf_max=16, ng=3)
    phi, acc, _ = gpu_solve(hpm, w.pos, w.mass, w.max_depth, w.ng, w.eps, w.leaf_max,
                            flags=hpm.HPM_FLAG_EXTENDED_GRIDLET)
    tr = O.Tree(w.pos, max_depth=w.max_depth, leaf_max=w.leaf_max)
    sample = np.arange(0, w.n, 11)
    p_ref, a_ref = O.solve_direct(tr, w.mass, w.ng, w.eps, sample, ext=1)
    assert O.rel_rms(acc[sample], a_ref) < TOL and O.rel_rms(phi[sample], p_ref) < TOL


@pytest.mark.parametrize("ng", [2, 3])
def test_widened_stages(hpm, ng):
    w = I.Workload(f"u{ng}e", I.uniform_cube(2500, 54 + ng), I.equal_masses(2500), max_depth=3, leaf_max=0,
                   ng=ng, eps=1e-3)
    check_stages(hpm, w, flags=hpm.HPM_FLAG_EXTENDED_GRIDLET, max_targets=200)
