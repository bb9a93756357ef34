"""Batched solves: many independent problems through the same launches.

Each problem's potentials and accelerations must be bit-identical whether it is
solved alone or inside a batch (same lists, same arithmetic in the same
order), and the batched lists must equal the oracle's lists of each problem.
"""
import numpy as np
import pytest

import oracle as O
from paper_1906_10734_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEPTH, NG, EPS, LEAF = 12, 4, 1e-4, 32


@pytest.fixture(scope="module")
def hpm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_10734_gb300 import hpm as H
    return H


def problems(count, nmin=300, nmax=30000, seed=4):
    return [I.batch_problem(k, nmin, nmax, seed) for k in range(count)]


def solve_alone(H, w):
    dev = torch.device("cuda:0")
    s = H.Solver(DEPTH, NG, EPS, LEAF)
    phi, acc = s(torch.from_numpy(w.pos).to(dev), torch.from_numpy(w.mass).to(dev))
    torch.cuda.synchronize()
    out = phi.cpu().numpy(), acc.cpu().numpy()
    s.close()
    return out


def test_batch_equals_each_problem_alone(hpm):
    ws = problems(12)
    dev = torch.device("cuda:0")
    bufs = []
    for w in ws:
        bufs.append((torch.from_numpy(w.pos).to(dev), torch.from_numpy(w.mass).to(dev),
                     torch.zeros(w.n, dtype=torch.float32, device=dev),
                     torch.zeros((w.n, 3), dtype=torch.float32, device=dev)))
    plan = hpm.hpm_plan((0.0, 0.0, 0.0), 1.0, DEPTH, NG, EPS, LEAF)
    for _ in range(2):                       # the second batch reuses the plan's buffers
        hpm.hpm_solve_batch(plan, bufs)
        torch.cuda.synchronize()
        for w, b in zip(ws, bufs):
            phi, acc = solve_alone(hpm, w)
            assert np.array_equal(b[2].cpu().numpy(), phi)
            assert np.array_equal(b[3].cpu().numpy(), acc)
    hpm.hpm_destroy(plan)


def test_packed_batch_lists_match_oracle_per_problem(hpm):
    ws = problems(5, seed=9)
    ws.insert(2, I.Workload("empty", np.zeros((0, 3)), np.zeros(0), DEPTH, LEAF, NG, EPS))
    dev = torch.device("cuda:0")
    pos = np.concatenate([w.pos for w in ws])
    mass = np.concatenate([w.mass for w in ws])
    off = np.concatenate([[0], np.cumsum([w.n for w in ws])]).astype(np.int64)
    plan = hpm.hpm_plan((0.0, 0.0, 0.0), 1.0, DEPTH, NG, EPS, LEAF)
    dpos, dmass = torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev)
    phi = torch.zeros(pos.shape[0], dtype=torch.float32, device=dev)
    acc = torch.zeros((pos.shape[0], 3), dtype=torch.float32, device=dev)
    hpm.hpm_build_tree_batch(plan, dpos, off)
    hpm.hpm_solve(plan, dpos, dmass, phi, acc)
    torch.cuda.synchronize()
    lst = hpm.hpm_get_lists(plan)
    hpm.hpm_destroy(plan)
    prob = (lst["key"] >> (3 * lst["level"].astype(np.uint64))).astype(np.int64)
    iz_cells = np.flatnonzero(lst["level"] >= 2)
    leaf_cells = np.flatnonzero(lst["leaf"] == 1)
    for p, w in enumerate(ws):
        if w.n == 0:
            assert not np.any(prob == p)
            continue
        ref = O.canonical_lists(O.Tree(w.pos, max_depth=DEPTH, leaf_max=LEAF))
        mine = prob == p
        assert np.array_equal(lst["level"][mine], ref["level"])
        strip = lst["key"][mine] & ((np.uint64(1) << (np.uint64(3) * lst["level"][mine].astype(np.uint64))) - np.uint64(1))
        assert np.array_equal(strip, ref["key"])
        assert np.array_equal(lst["begin"][mine] - off[p], ref["begin"])
        assert np.array_equal(lst["end"][mine] - off[p], ref["end"])
        assert np.array_equal(lst["leaf"][mine], ref["leaf"])
        assert np.array_equal(lst["iz"][np.isin(iz_cells, np.flatnonzero(mine))], ref["iz"])
        assert np.array_equal(lst["near"][np.isin(leaf_cells, np.flatnonzero(mine))], ref["near"])
        assert np.array_equal(lst["perm"][off[p]:off[p + 1]] - off[p], ref["perm"])
        a_alone = solve_alone(hpm, w)[1]
        assert np.array_equal(acc[off[p]:off[p + 1]].cpu().numpy(), a_alone)
