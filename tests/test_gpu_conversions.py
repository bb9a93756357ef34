"""The float <-> double conversions the library does by IEEE 754 bit manipulation on the
integer units (the gather of the sorted particles) against the hardware's conversions, bit
for bit: random doubles over and beyond the float range, exact ties of round to nearest
even (a float plus half its unit in the last place, both ways), zeros of both signs,
subnormals, the edges of the float normal range, infinities and NaNs; random floats with
the same special values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hpm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_10734_gb300 import hpm as H
    return H


def doubles(rng):
    n = 2_000_000
    x = np.ldexp(rng.random(n) + 1.0, rng.integers(-160, 140, n)) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    f = rng.standard_normal(500_000).astype(np.float32)
    half_ulp = 0.5 * np.spacing(np.abs(f)).astype(np.float64)
    ties = np.concatenate([f.astype(np.float64) + half_ulp, f.astype(np.float64) - half_ulp])
    edges = np.array([0.0, -0.0, 1.0, -1.0, 343.0, np.finfo(np.float32).max, -np.finfo(np.float32).max,
                      float(np.finfo(np.float32).max) * (1 + 2.0 ** -25), float(np.finfo(np.float32).max) * 1.5,
                      float(np.finfo(np.float32).tiny), float(np.finfo(np.float32).tiny) * (1 - 2.0 ** -30),
                      1e-40, -1e-45, 5e-324, np.inf, -np.inf, np.nan, 1e300, -1e-300])
    return np.concatenate([x, ties, edges])


def floats(rng):
    special = np.array([0.0, -0.0, 1e-45, -1e-45, 1.1754942e-38, np.finfo(np.float32).tiny, np.finfo(np.float32).max,
                        np.inf, -np.inf, np.nan], np.float32)
    return np.concatenate([rng.standard_normal(1_000_000).astype(np.float32),
                           (rng.random(1_000_000) * 8 - 4).astype(np.float32),
                           np.ldexp(rng.random(200_000) + 1, rng.integers(-149, 128, 200_000)).astype(np.float32),
                           special])


def test_integer_unit_conversions_match_the_hardware(hpm):
    rng = np.random.default_rng(11)
    dev = torch.device("cuda:0")
    d = torch.from_numpy(doubles(rng)).to(dev)
    f = torch.from_numpy(floats(rng)).to(dev)
    assert hpm.hpm_check_conversions(d, f) == 0
    # and one each way alone
    assert hpm.hpm_check_conversions(d, f[:0]) == 0
    assert hpm.hpm_check_conversions(d[:0], f) == 0
