"""The patch-grid point-source workload (Sec. 3.2) on the CPU: cell counts of the three grid
geometries and a tree whose leaves are exactly the patches of 8^3 cells."""
import numpy as np
import pytest

import oracle as O
from paper_1906_10734_gb300 import inputs as I


@pytest.mark.parametrize("geometry,cells,leaves", [
    ("uniform4", 128 ** 3, {4: 4096}),
    ("mixed", 720896, {3: 448, 4: 448, 5: 512}),
])
def test_patch_grid_tree_is_the_patches(geometry, cells, leaves):
    w = I.point_source_patch_grid(geometry)
    assert w.n == cells + 1 and w.mass[0] == 1.0 and np.all(w.mass[1:] == 0.0)
    assert np.all(w.pos[0] == 1.0)
    tr = O.Tree(w.pos, max_depth=w.max_depth, leaf_max=w.leaf_max)
    got = {l: int(lv.leaf.sum()) for l, lv in enumerate(tr.levels) if lv.leaf.any()}
    assert got == leaves
    for l, lv in enumerate(tr.levels):
        # every leaf holds one patch (plus the source in the corner patch)
        assert np.all((lv.count[lv.leaf] == 512) | (lv.count[lv.leaf] == 513))
    # cell centres of a level-l patch lie on that level's cell grid, (i + 1/2) / (8 2^l)
    c = w.pos[1:]
    assert np.all((c > 0.0) & (c < 1.0))
