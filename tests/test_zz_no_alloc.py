"""The no-allocation sort entry point against the solver's own tree build.

hpm_sort_particles_static serves callers that cannot allocate device memory
(an application that owns every allocation, or code that must not allocate
after set-up); its scratch is a static device array. Its permutation must
equal the one hpm_build_tree produces (integer work: bit for bit), and its
keys must equal the level-max_depth cell keys the build reports, on two calls
in a row that reuse the shared static scratch.
"""
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
    return H


def reference(H, pos, depth):
    """Permutation and per-particle level-depth keys from the uniform-tree build."""
    dev = torch.device("cuda:0")
    p = torch.from_numpy(pos).to(dev)
    plan = H.hpm_plan((0.0, 0.0, 0.0), 1.0, depth, 4, 0.0, 0)
    H.hpm_build_tree(plan, p, pos.shape[0])
    lst = H.hpm_get_lists(plan)
    H.hpm_destroy(plan)
    keys = np.zeros(pos.shape[0], np.uint64)
    deep = lst["level"] == depth
    for k, b, e in zip(lst["key"][deep], lst["begin"][deep], lst["end"][deep]):
        keys[b:e] = k
    return lst["perm"], keys


@pytest.mark.parametrize("pos,depth", [(I.uniform_cube(1 << 20, 71), 7),
                                       (I.plummer_sphere(300001, 72), 12),
                                       (I.uniform_cube(5000, 73), 0)])
def test_static_sort_matches_tree_build(hpm, pos, depth):
    assert pos.shape[0] <= hpm.HPM_STATIC_SORT_MAX_N
    dev = torch.device("cuda:0")
    n = pos.shape[0]
    perm_ref, keys_ref = reference(hpm, pos, depth)
    p = torch.from_numpy(pos).to(dev)
    for _ in range(2):
        keys = torch.full((n,), -1, dtype=torch.int64, device=dev)
        perm = torch.full((n,), -1, dtype=torch.int32, device=dev)
        hpm.hpm_sort_particles_static(p, n, keys, perm, depth)
        torch.cuda.synchronize()
        assert np.array_equal(perm.cpu().numpy().astype(np.uint32).astype(np.int64), perm_ref)
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), keys_ref)


def test_static_sort_rejects_sizes_beyond_its_scratch(hpm):
    n = hpm.HPM_STATIC_SORT_MAX_N + 1
    with pytest.raises(hpm.HpmError) as e:
        hpm.hpm_sort_particles_static(None, n, None, None, 7)
    assert e.value.status == -1
