"""Green functions other than Plummer on the GPU, against the FP64 oracle with the same
kernel (Sec. 4: the method only convolves with the Green function).

Yukawa and Newton are closed forms in both; erf(r/a)/r is a user kernel given as a C
function to both the library (which tabulates it on the lattice and, for the near field,
as piecewise cubics of g and -g'/r) and the oracle (which calls it, with its exact
derivative, at every pair). The bar is the parity bar of the Plummer kernel: 1e-5
relative RMS, fields and stages, on the tensor-core path (Ng = 4), the FFT-form kernel
and the other orders.
"""
import numpy as np
import pytest

import oracle as O
import user_kernels as UK
from paper_1906_10734_gb300 import inputs as I
from test_gpu_parity import TOL, TOL_BY_NG, gpu_solve
from test_gpu_stages import check_stages

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hpm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_10734_gb300 import hpm as H
    return H


def kernels(H, name):
    """(library descriptor, oracle kernel, keep-alive) for a named kernel."""
    if name == "yukawa":
        return H.Green.yukawa(0.1, 1e-3), O.Kernel.yukawa(0.1, 1e-3), None
    if name == "newton":
        return H.Green.newton(), O.Kernel.newton(), None
    if name == "erf":
        g, dg, p = UK.erf_kernel(0.01)
        return H.Green.user(g, p.ptr), O.Kernel.user(g, dg, p.ptr), p
    if name == "plummer_user":
        g, dg, p = UK.plummer_kernel(1e-3)
        return H.Green.user(g, p.ptr), O.Kernel.user(g, dg, p.ptr), p
    raise KeyError(name)


@pytest.mark.parametrize("name", ["yukawa", "newton", "erf", "plummer_user"])
def test_fields_uniform_4096(hpm, name):
    green, kern, keep = kernels(hpm, name)
    w = I.uniform_4096_depth3()
    phi, acc, _ = gpu_solve(hpm, w.pos, w.mass, w.max_depth, w.ng, w.eps, w.leaf_max, green=green)
    tr = O.Tree(w.pos, max_depth=w.max_depth, leaf_max=w.leaf_max)
    p_ref, a_ref = O.solve_direct(tr, w.mass, w.ng, kern)
    ea, ep = O.rel_rms(acc, a_ref), O.rel_rms(phi, p_ref)
    print(f"{name}: acc {ea:.3e} phi {ep:.3e}")
    assert ea < TOL and ep < TOL


@pytest.mark.parametrize("name", ["yukawa", "erf"])
def test_fields_adaptive_plummer(hpm, name):
    green, kern, keep = kernels(hpm, name)
    w = I.small_plummer(20000, 81, leaf_max=16)
    phi, acc, _ = gpu_solve(hpm, w.pos, w.mass, w.max_depth, w.ng, w.eps, w.leaf_max, green=green)
    tr = O.Tree(w.pos, max_depth=w.max_depth, leaf_max=w.leaf_max)
    sample = np.arange(0, w.n, 7)
    p_ref, a_ref = O.solve_direct(tr, w.mass, w.ng, kern, sample)
    assert O.rel_rms(acc[sample], a_ref) < TOL and O.rel_rms(phi[sample], p_ref) < TOL


@pytest.mark.parametrize("name", ["yukawa", "erf"])
def test_stages_tensor_and_fft_paths(hpm, name):
    green, kern, keep = kernels(hpm, name)
    w = I.uniform_4096_depth3()
    check_stages(hpm, w, green=green, kernel=kern)
    check_stages(hpm, w, flags=hpm.HPM_FLAG_FFT_M2L, green=green, kernel=kern)
    check_stages(hpm, I.small_plummer(12000, 82, leaf_max=16), max_targets=400, green=green, kernel=kern)


@pytest.mark.parametrize("ng", [2, 3, 5])
def test_other_orders_yukawa(hpm, ng):
    green, kern, keep = kernels(hpm, "yukawa")
    pos, mass = I.uniform_cube(2500, 90 + ng), I.equal_masses(2500)
    phi, acc, _ = gpu_solve(hpm, pos, mass, 3, ng, 1e-3, 0, green=green)
    tr = O.Tree(pos, max_depth=3, leaf_max=0)
    sample = np.arange(0, 2500, 5)
    p_ref, a_ref = O.solve_direct(tr, mass, ng, kern, sample)
    assert O.rel_rms(acc[sample], a_ref) < TOL_BY_NG[ng] and O.rel_rms(phi[sample], p_ref) < TOL


def test_user_kernel_equal_to_plummer_matches_builtin(hpm):
    """The tabulated user path and the closed form of the same kernel agree to the
    table's interpolation error."""
    green, _, keep = kernels(hpm, "plummer_user")
    w = I.small_plummer(20000, 83, leaf_max=16)
    p1, a1, _ = gpu_solve(hpm, w.pos, w.mass, w.max_depth, w.ng, 1e-3, w.leaf_max, green=green)
    p0, a0, _ = gpu_solve(hpm, w.pos, w.mass, w.max_depth, w.ng, 1e-3, w.leaf_max)
    assert O.rel_rms(a1, a0) < 2e-6 and O.rel_rms(p1, p0) < 2e-6
