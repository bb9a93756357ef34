"""Domains other than the unit cube at the origin: positions x = o + S u in a cube of side S
at origin o solve as the unit-cube positions u with the softening eps / S, the potential
scaled by 1/S and the accelerations by 1/S^2 (the Plummer kernel is homogeneous of degree -1
in (r, eps)). With a power-of-two side and positions on a dyadic grid the map is exact, so the
tree (cells, ranges and the permutation) is the unit cube's bit for bit; a side of 3 takes the
division path of the keys and of the gather, where positions on a cell boundary may round to
either side, so only the fields are compared (parity bar)."""
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


def rel_rms(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def solve(hpm, pos, mass, eps, origin=(0.0, 0.0, 0.0), side=1.0):
    dev = torch.device("cuda:0")
    s = hpm.Solver(12, 4, eps, 32, origin=origin, side=side)
    phi, acc = s(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev))
    torch.cuda.synchronize()
    out = (phi.cpu().numpy().astype(np.float64), acc.cpu().numpy().astype(np.float64), s.lists())
    s.close()
    return out


def test_shifted_and_scaled_domains_match_the_unit_cube(hpm):
    n = 30000
    # unit-cube positions on a dyadic grid (30 fraction bits): o + S u is exact in FP64 for
    # the power-of-two side below
    u = np.clip(np.round(I.plummer_sphere(n, 71) * 2.0 ** 30) / 2.0 ** 30, 0.0, 1.0 - 2.0 ** -30)
    mass = I.equal_masses(n)
    eps = 1e-3
    phi_u, acc_u, lists_u = solve(hpm, u, mass, eps)
    for origin, side, exact in (((-4.0, 2.0, 16.0), 8.0, True), ((1.5, -2.25, 0.125), 3.0, False)):
        x = np.asarray(origin) + side * u
        phi, acc, lists = solve(hpm, x, mass, eps * side, origin, side)
        if exact:
            for k in lists_u:
                assert np.array_equal(np.asarray(lists[k]), np.asarray(lists_u[k])), k
            tol = 1e-6
        else:
            tol = 1e-5
        assert rel_rms(phi * side, phi_u) < tol
        assert rel_rms(acc * side * side, acc_u) < tol
