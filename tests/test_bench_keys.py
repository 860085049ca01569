"""bench.py's drift and size-sweep summaries (no GPU): the keys the bench line
carries and the arithmetic behind them on synthetic series."""
import math

import numpy as np
import pytest

import bench


def test_lj_u_at_cutoff():
    # Eq. 1 with eps = sigma = 1 at r = 2.5: 4 (2.5^-12 - 2.5^-6)
    assert bench.lj_u(2.5) == pytest.approx(-0.016316891136, rel=1e-10)
    assert bench.lj_u(2 ** (1 / 6)) == pytest.approx(-1.0, rel=1e-12)


def test_drift_summary_keys_and_values():
    n = 1000
    steps = np.arange(0, 10001, 100)
    # E_tot falls by one cutoff jump per 100 steps while the shifted energy
    # (E_tot - n_pairs U(rc)) stays flat: a pair leaving rc raises E by -U(rc)
    npairs = 50000 - steps // 100
    e = -5000.0 + npairs * bench.lj_u(2.5) + 1e-9 * steps
    d = bench.drift_summary(steps, e, npairs, n)
    assert set(d) == {"steps", "samples", "etot", "shifted"}
    assert d["steps"] == 10000 and d["samples"] == steps.size
    for k in ("etot", "shifted"):
        assert set(d[k]) == {"slope_per_atom_step", "max_rel_dev"}
    assert d["shifted"]["slope_per_atom_step"] == pytest.approx(1e-12, rel=1e-6)
    want = (-bench.lj_u(2.5) / 100 + 1e-9) / n
    assert d["etot"]["slope_per_atom_step"] == pytest.approx(want, rel=1e-9)
    e0 = e[0]
    assert d["etot"]["max_rel_dev"] == pytest.approx(np.max(np.abs(e - e0)) / abs(e0))


def test_sweep_row_keys_and_formulas():
    n = 256000
    r = {"ms": 200.0, "pair_ms": 0.15, "rebuild_ms": 0.5, "tpa": 1, "compacted": 2,
         "phase1_entries": 2, "entries": 38 * n, "pairs": 27 * n,
         "clocks": {"sm_mhz": 2070.0}}
    row = bench.sweep_row(40, n, "fp64_half", r, 1000, 6785.5, 629.28)
    for k in ("cells", "n_atoms", "form", "steps", "value", "ms_per_step", "pair_kernel_ms",
              "rebuild_ms", "list_entries_per_atom", "pairs_in_rc_per_atom",
              "pair_kernel_hbm_frac", "step_hbm_frac", "pair_kernel_fp64_frac", "clocks",
              "phase1_entries"):
        assert k in row, k
    assert row["value"] == pytest.approx(n * 1000 / 0.2 / 1e6)
    ops, byts = bench.pair_work("half", "fp64", n, r["entries"], r["pairs"], 2)
    assert ops == 8 * r["pairs"]  # compacted 2: the integer path
    assert bench.pair_work("full", "fp64", n, r["entries"], r["pairs"], 1)[0] == 34 * r["pairs"]
    assert bench.pair_work("half", "fp64", n, 0, r["pairs"], 2, coul=True)[0] == 22 * r["pairs"]
    assert row["pair_kernel_fp64_frac"] == pytest.approx(ops / 0.15e-3 / 1e9 / 629.28)
    assert row["pair_kernel_hbm_frac"] == pytest.approx(byts / 0.15e-3 / 1e9 / 6785.5)
    mixed = bench.sweep_row(40, n, "mixed_full", r, 1000, 6785.5, 629.28)
    assert "pair_kernel_fp64_frac" not in mixed
    assert not math.isnan(mixed["step_hbm_frac"])


def test_kernel_code_keeps_the_filter_depth():
    """md_set_kernel's `compacted` argument for a configuration read back
    from md_get_stats: the fixed-point kernel with two entries per filter
    round is compacted 3, except under the one-launch-per-step schedule,
    which has one entry a round."""
    st = {"compacted": 2, "phase1_entries": 2}
    assert bench.kernel_code(st) == 3
    assert bench.kernel_code(st, 1) == 3
    assert bench.kernel_code(st, 2) == 2
    assert bench.kernel_code({"compacted": 2, "phase1_entries": 1}) == 2
    assert bench.kernel_code({"compacted": 0, "phase1_entries": 2}) == 0  # mixed walk
    assert bench.kernel_code({"compacted": 1, "phase1_entries": 1}) == 1


def test_pair_traffic_keys():
    """The traffic table is keyed by form, compacted mode, threads per atom
    and filter depth, for the current pair sources only."""
    h = bench.pair_source_hash()
    if h not in bench.PAIR_TRAFFIC:
        pytest.skip("pair sources changed since the traffic capture")
    assert bench.pair_traffic("fp64_half", 2, 1, 2, 4_000_000) is not None
    assert bench.pair_traffic("mixed_full", 0, 2, 2, 4_000_000) is not None
    assert bench.pair_traffic("fp64_half", 2, 1, 1, 4_000_000) is None
