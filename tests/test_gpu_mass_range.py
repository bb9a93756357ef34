"""Masses that span many decades, on the default Ng = 4 tensor-core path.

The dense source-to-target product splits each level's effective masses into
FP16 pairs at one power-of-two scale per (problem, level): a box far lighter
than the level's heaviest keeps fewer significant bits. These cases check that
the fields still meet the 1e-5 relative RMS bar against the FP64 HPM where
the method accepts such inputs: masses log-uniform over six decades, and a
uniform set with one body 10^4 times heavier than all the others together
(element-wise stage parity on reduced sizes, sampled fields at 2^21).
"""
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


def loguniform_plummer(n, seed):
    w = I.small_plummer(n, seed, leaf_max=32)
    w.mass = I.log_uniform_masses(n, seed + 100, decades=6.0)
    return w


def heavy_uniform(n, seed):
    pos = I.uniform_cube(n, seed)
    mass, k = I.heavy_body_masses(n, seed + 100, ratio=1e4)
    return I.Workload(f"uniform{n}_heavy", pos, mass, max_depth=12, leaf_max=32, ng=4, eps=1e-4,
                      meta={"heavy": k})


def test_stages_log_uniform_masses(hpm):
    check_stages(hpm, loguniform_plummer(20000, 70), max_targets=600)


def test_stages_heavy_body(hpm):
    check_stages(hpm, heavy_uniform(20000, 71), max_targets=600)


def check_fields(hpm, w, nsample=256, seed=0, exclude=None):
    phi, acc, _ = gpu_solve(hpm, w.pos, w.mass, w.max_depth, w.ng, w.eps, w.leaf_max)
    tr = O.Tree(w.pos, max_depth=w.max_depth, leaf_max=w.leaf_max)
    cand = np.arange(w.n) if exclude is None else np.setdiff1d(np.arange(w.n), [exclude])
    sample = np.sort(np.random.default_rng(seed).choice(cand, nsample, replace=False))
    p_ref, a_ref = O.solve_direct(tr, w.mass, w.ng, w.eps, sample)
    ea, ep = O.rel_rms(acc[sample], a_ref), O.rel_rms(phi[sample], p_ref)
    # the same bar per particle class: the lightest tenth of the sample on its own
    light = np.argsort(w.mass[sample])[: max(8, nsample // 10)]
    el = O.rel_rms(acc[sample][light], a_ref[light])
    print(f"{w.name}: acc {ea:.3e} phi {ep:.3e}; lightest tenth acc {el:.3e}")
    assert ea < TOL and ep < TOL and el < TOL


def test_fields_log_uniform_masses_small(hpm):
    check_fields(hpm, loguniform_plummer(30000, 72), nsample=1000)


def test_fields_heavy_body_small(hpm):
    w = heavy_uniform(30000, 73)
    check_fields(hpm, w, nsample=1000, exclude=w.meta["heavy"])


@pytest.mark.slow
def test_fields_log_uniform_masses_plummer_2m(hpm):
    w = I.plummer_2m_adaptive()
    w.mass = I.log_uniform_masses(w.n, 74, decades=6.0)
    w.name = "plummer2m_loguniform6"
    check_fields(hpm, w, seed=2)


@pytest.mark.slow
def test_fields_heavy_body_uniform_2m(hpm):
    w = heavy_uniform(1 << 21, 75)
    check_fields(hpm, w, seed=3, exclude=w.meta["heavy"])
