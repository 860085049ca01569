"""The cutoff-decision workload has the properties its GPU test relies on
(no GPU).

test_gpu_mixed_cutoff.py checks that the mixed kernels decide the cutoff as
FP64 does on a lattice of isolated pairs.  Its result means something only
if (a) the pairs are isolated: every pair within the list cutoff is one of
the lattice's own pairs, so each atom's force is that pair's force; (b) an
FP32 cutoff test would decide some of the pairs wrongly; (c) pairs both
inside and outside each cutoff are present; (d) almost no pair lies within
the FP64 band's own accuracy (1e-10) of a cutoff.
"""
import numpy as np
import pytest

from cutoff_lattice import RC, RC_COUL, fp32_flips, pair_lattice, pair_r2

RLIST = RC + 0.3
WORKLOADS = [(101, [RC], [RC]), (103, [RC, RC_COUL], [RC, RC_COUL]), (107, [RC], [RC])]


@pytest.mark.parametrize("seed,radii,cuts", WORKLOADS)
def test_pairs_are_isolated(oracle, seed, radii, cuts):
    x, box = pair_lattice(seed, radii)
    pi, pk = oracle.pairs_cells(x, box, RLIST)
    got = sorted(zip(np.minimum(pi, pk).tolist(), np.maximum(pi, pk).tolist()))
    assert got == [(2 * s, 2 * s + 1) for s in range(len(x) // 2)]


@pytest.mark.parametrize("seed,radii,cuts", WORKLOADS)
def test_fp32_would_decide_some_pairs_wrongly(seed, radii, cuts):
    x, box = pair_lattice(seed, radii)
    for rc in cuts:
        assert fp32_flips(x, box, rc) >= 3


@pytest.mark.parametrize("seed,radii,cuts", WORKLOADS)
def test_both_sides_of_each_cutoff_and_few_ties(seed, radii, cuts):
    x, box = pair_lattice(seed, radii)
    r2 = pair_r2(x, box)
    for k, rc in enumerate(radii):
        mine = (np.arange(len(r2)) // 2) % len(radii) == k  # pairs placed at rc
        rel = r2[mine] / (rc * rc) - 1.0
        assert (rel < 0).sum() > 100 and (rel > 0).sum() > 100
        assert np.abs(rel).max() < 2.1e-5  # within the widest placement band
        assert (np.abs(rel) < 1e-10).sum() <= 2
