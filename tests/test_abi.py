"""The C-ABI library loads and exports every entry point include/hpm.h declares.

No compute call is made here (this suite also runs without a GPU); only the
argument checks that return before any CUDA call are exercised.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(hpm_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_10734_gb300 import hpm
    return hpm.load()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("hpm_plan", "hpm_build_tree", "hpm_solve", "hpm_destroy", "hpm_get_lists"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1906_10734_gb300 import hpm
    for name in declared_symbols():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
        assert name in hpm.SIGNATURES, f"{name} has no binding signature"


def test_status_strings(lib):
    from paper_1906_10734_gb300 import hpm
    assert hpm.hpm_status_str(0) == "ok"
    assert hpm.hpm_status_str(-2) == "particle outside the domain"


@pytest.mark.parametrize("kw", [dict(max_depth=-1), dict(max_depth=22), dict(gridlet_order=0),
                                dict(gridlet_order=9), dict(side=0.0), dict(side=float("nan")),
                                dict(eps=-1.0), dict(leaf_max=-3)])
def test_plan_rejects_bad_arguments_before_touching_the_device(lib, kw):
    from paper_1906_10734_gb300 import hpm
    args = dict(origin=(0.0, 0.0, 0.0), side=1.0, max_depth=3, gridlet_order=4, eps=0.0, leaf_max=0)
    args.update(kw)
    with pytest.raises(hpm.HpmError) as e:
        hpm.hpm_plan(**args)
    assert e.value.status == -1


def test_null_plan_is_rejected(lib):
    assert lib.hpm_build_tree(None, None, 0, None) == -1
    assert lib.hpm_solve(None, None, None, None, None, None) == -1
    assert lib.hpm_set_tuning(None, None) == -1
    assert lib.hpm_get_tuning(None, None) == -1
    assert lib.hpm_tune(None, None, None, 0, None, None) == -1
    assert lib.hpm_destroy(None) == 0


def test_plan_refuses_invalid_green_functions(lib):
    """Kernel checks of hpm_plan return before any CUDA call: a Yukawa kernel needs a
    positive screening length and a nonnegative softening, a user kernel a function, and
    an unknown kind is unsupported."""
    from paper_1906_10734_gb300 import hpm
    for g in (hpm.Green(hpm.HPM_GREEN_YUKAWA, 0.0, 0.0), hpm.Green(hpm.HPM_GREEN_YUKAWA, -1.0, 0.1),
              hpm.Green(hpm.HPM_GREEN_USER)):
        with pytest.raises(hpm.HpmError) as e:
            hpm.hpm_plan((0.0, 0.0, 0.0), 1.0, 3, 4, green=g)
        assert e.value.status == -1
    with pytest.raises(hpm.HpmError) as e:
        hpm.hpm_plan((0.0, 0.0, 0.0), 1.0, 3, 4, green=hpm.Green(7))
    assert e.value.status == -8


def test_plan_refuses_widened_gridlets_above_order_6(lib):
    """Widened target gridlets (Sec. 2.5) hold Ng + 2 nodes per axis, at most 8: Ng = 7
    with HPM_FLAG_EXTENDED_GRIDLET is refused before any CUDA call."""
    from paper_1906_10734_gb300 import hpm
    with pytest.raises(hpm.HpmError) as e:
        hpm.hpm_plan((0.0, 0.0, 0.0), 1.0, 3, 7, flags=hpm.HPM_FLAG_EXTENDED_GRIDLET)
    assert e.value.status == -8
