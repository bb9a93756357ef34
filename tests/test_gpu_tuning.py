"""Launch shapes and their autotuner: every shape gives the same results bit for
bit (the shapes only spread the same work over the GPU differently), the
tuner returns shapes from the documented ranges, and bad shapes are refused."""
import numpy as np
import pytest

from paper_1906_10734_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hpm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_10734_gb300 import hpm as H
    assert torch.cuda.is_available()
    return H


def solve_with(H, w, shapes, flags=0, ng=None):
    dev = torch.device("cuda:0")
    s = H.Solver(w.max_depth, ng or w.ng, w.eps, w.leaf_max, flags=flags)
    H.hpm_set_tuning(s.plan, **shapes)
    p = torch.from_numpy(np.ascontiguousarray(w.pos)).to(dev)
    m = torch.from_numpy(np.ascontiguousarray(w.mass)).to(dev)
    phi, acc = s(p, m)
    torch.cuda.synchronize()
    out = (phi.cpu().numpy(), acc.cpu().numpy())
    s.close()
    return out


def assert_same(a, b):
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_shapes_keep_results_tensor_path(hpm):
    w = I.small_plummer(20000, 61, leaf_max=16)
    ref = solve_with(hpm, w, {})
    for shapes in (dict(level_blocks_per_sm=1), dict(level_blocks_per_sm=3), dict(level_blocks_per_sm=4),
                   dict(gridlet_warps=2), dict(gridlet_warps=4), dict(m2l_block_order=2),
                   dict(m2l_tile_parents=224), dict(m2l_tile_parents=208), dict(m2l_tile_parents=192),
                   dict(m2l_tile_parents=224, m2l_block_order=2)):
        assert_same(solve_with(hpm, w, shapes), ref)
    # Ng = 6 runs on the dense tensor-core path too
    ref6 = solve_with(hpm, w, {}, ng=6)
    assert_same(solve_with(hpm, w, dict(m2l_block_order=2), ng=6), ref6)


def test_tile_widths_keep_results_over_many_tiles(hpm):
    """Parents per tile of the Ng = 4 tensor-core kernel: with 2^18 Plummer particles the
    deeper levels hold several tiles of every width and a ragged last tile; each parent's
    sums are the same bit for bit."""
    w = I.small_plummer(1 << 18, 65, leaf_max=32)
    ref = solve_with(hpm, w, dict(m2l_tile_parents=256))
    for tn in (224, 208, 192):
        assert_same(solve_with(hpm, w, dict(m2l_tile_parents=tn)), ref)
        assert_same(solve_with(hpm, w, dict(m2l_tile_parents=tn, m2l_block_order=2)), ref)


def test_shapes_keep_results_fft_paths(hpm):
    w = I.small_plummer(12000, 62, leaf_max=16)
    for flags, ng in ((hpm.HPM_FLAG_FFT_M2L, 4), (hpm.HPM_FLAG_XTRANSFORM_M2L, 6), (0, 5)):
        ref = solve_with(hpm, w, {}, flags=flags, ng=ng)
        assert_same(solve_with(hpm, w, dict(m2l_ctas_per_sm=1), flags=flags, ng=ng), ref)


def test_tune_picks_valid_shapes_and_keeps_results(hpm):
    w = I.small_plummer(20000, 63, leaf_max=16)
    ref = solve_with(hpm, w, {})
    dev = torch.device("cuda:0")
    s = hpm.Solver(w.max_depth, w.ng, w.eps, w.leaf_max)
    p = torch.from_numpy(np.ascontiguousarray(w.pos)).to(dev)
    m = torch.from_numpy(np.ascontiguousarray(w.mass)).to(dev)
    t = hpm.hpm_tune(s.plan, p, m)
    assert t["level_blocks_per_sm"] in (1, 2, 3, 4)
    assert t["gridlet_warps"] in (2, 4, 8)
    assert t["m2l_block_order"] in (1, 2)
    assert t["m2l_tile_parents"] in (256, 224, 208, 192)
    assert hpm.hpm_get_tuning(s.plan) == t
    phi, acc = s(p, m)
    torch.cuda.synchronize()
    assert_same((phi.cpu().numpy(), acc.cpu().numpy()), ref)
    s.close()


def test_bad_shapes_are_refused(hpm):
    s = hpm.Solver(3, 4, 0.0, 0)
    for shapes in (dict(level_blocks_per_sm=5), dict(gridlet_warps=3), dict(m2l_ctas_per_sm=3),
                   dict(level_blocks_per_sm=-1), dict(m2l_block_order=3), dict(m2l_tile_parents=200),
                   dict(m2l_tile_parents=512)):
        with pytest.raises(hpm.HpmError) as e:
            hpm.hpm_set_tuning(s.plan, **shapes)
        assert e.value.status == -1
    s.close()


def test_a_wait_that_runs_out_is_reported_and_the_plan_recovers(hpm):
    # failure detection without a GPU fault: the source-to-target kernel waits on a
    # barrier nothing arrives at, gives up after ~2^24 cycles, records a timeout; the
    # next synchronising call reports it once, and the plan then solves as before
    w = I.small_plummer(12000, 64, leaf_max=16)
    ref = solve_with(hpm, w, {})
    dev = torch.device("cuda:0")
    s = hpm.Solver(w.max_depth, w.ng, w.eps, w.leaf_max)
    p = torch.from_numpy(np.ascontiguousarray(w.pos)).to(dev)
    m = torch.from_numpy(np.ascontiguousarray(w.mass)).to(dev)
    phi = torch.empty(w.n, dtype=torch.float32, device=dev)
    acc = torch.empty((w.n, 3), dtype=torch.float32, device=dev)
    hpm.hpm_test_stall(s.plan, True, 1 << 24)
    hpm.hpm_build_tree(s.plan, p, w.n)
    hpm.hpm_solve(s.plan, p, m, phi, acc)
    torch.cuda.synchronize()
    with pytest.raises(hpm.HpmError) as e:
        hpm.hpm_build_tree(s.plan, p, w.n)
    assert e.value.status == -5
    hpm.hpm_test_stall(s.plan, False, 0)
    phi, acc = s(p, m)
    torch.cuda.synchronize()
    assert_same((phi.cpu().numpy(), acc.cpu().numpy()), ref)
    s.close()
