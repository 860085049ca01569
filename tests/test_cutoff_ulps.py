"""CPU checks of the FP64 cutoff workload (tests/cutoff_ulps.py): exact
positions on the fixed-point grid, isolation, and pairs whose exact and
rounded r^2 are decided differently, on both sides of rc."""
from fractions import Fraction

import numpy as np
import pytest

from cutoff_ulps import BOX, Q, RC, classify, exact_r2, rounded_r2, workload


@pytest.fixture(scope="module")
def wl():
    return workload(7)


def test_positions_exact_and_on_grid(wl):
    x, box = wl
    assert np.all((x >= 2.0) & (x < 128.0))
    # multiples of 2^-51 (every double in [2, 128) is) and separations on Q
    d = x[1::2] - x[0::2]
    assert np.all(np.mod(d / Q, 1.0) == 0.0)
    assert np.all(x[0::2] + d == x[1::2])


def test_pairs_isolated(wl):
    """Every atom's only neighbor within rlist = rc + 0.3 is its partner."""
    from scipy.spatial import cKDTree
    x, box = wl
    t = cKDTree(x, boxsize=box)
    dist, idx = t.query(x, k=3)
    assert np.all(idx[:, 1] == (np.arange(len(x)) ^ 1))
    assert np.all(dist[:, 2] > RC + 0.3)


def test_exact_and_rounded_disagree_both_ways(wl):
    x, _ = wl
    ex, ro = classify(x)
    assert ((ex) & (~ro)).sum() >= 400   # inside exactly, outside once rounded
    assert ((~ex) & (ro)).sum() >= 200   # the reverse
    assert (ex == ro).sum() >= 200
    assert ro.sum() >= 200 and (~ro).sum() >= 200


def test_rounded_r2_emulation():
    # pinned against hand-checked cases: a single axis rounds once
    assert rounded_r2((2.5, 0.0, 0.0)) == 6.25
    d = (2.5 - 2.0 ** -51, 0.0, 0.0)
    assert rounded_r2(d) == float(Fraction(d[0]) ** 2)
    assert exact_r2((3.0, 4.0, 0.0)) == 25
    assert rounded_r2((1.5, 2.0, 0.0)) == 6.25
    assert RC * RC == 6.25
