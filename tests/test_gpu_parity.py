"""GPU path vs the FP64 CPU oracle, through the C ABI (needs a GB300).

Bars (arXiv 2508.13523 Eq. 1 and Sec. 4/4.1 define the quantities):
  * neighbor sets bit-exact as sets (full: every row; half: every pair once);
  * FP64 forces: max_i |F_i - F_i^ref| / rms(F^ref) <= 1e-12;
  * FP64 energy and virial: relative 1e-12;
  * mixed precision: error against the FP64 oracle reported, sanity bound 1e-4.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_2508_13523_gb300 as md  # noqa: E402
from paper_2508_13523_gb300 import synth as S  # noqa: E402

FORCE_TOL = 1e-12


def rel_err(f, fref):
    rms = np.sqrt(np.mean(np.sum(fref * fref, axis=1)))
    return float(np.max(np.linalg.norm(f - fref, axis=1)) / rms)


def lj_of(p):
    return O.LJ(p.eps, p.sigma, p.rc, ntypes=p.ntypes)


def make(sysm, **kw):
    return md.from_system(sysm, **kw)


def csr_rows(off, idx):
    off = off.cpu().numpy()
    idx = idx.cpu().numpy()
    return [idx[off[i]:off[i + 1]] for i in range(len(off) - 1)]


def check_neighbors(ctx, x, box, rlist, half):
    off, idx = ctx.neighbors()
    rows = csr_rows(off, idx)
    pi, pk = O.pairs_cells(x, box, rlist)
    ref = set(zip(pi.tolist(), pk.tolist()))
    if half:
        got = []
        for i, r in enumerate(rows):
            got += [(min(i, j), max(i, j)) for j in r.tolist()]
        assert len(got) == len(set(got)), "a pair is listed twice"
        assert set(got) == ref
    else:
        n = len(x)
        want = [[] for _ in range(n)]
        for a, b in ref:
            want[a].append(b)
            want[b].append(a)
        for i in range(n):
            assert sorted(rows[i].tolist()) == sorted(want[i]), i


def jittered(n, amp, seed, density=0.8442):
    x, box, _ = S.fcc(n, density)
    return x + amp * (S.uniform(seed, x.size).reshape(x.shape) - 0.5), box


@pytest.fixture(scope="module")
def melt():
    """The 32,000-atom melt after 40 oracle steps (a disordered liquid)."""
    s = S.fcc_liquid(20)
    x, v, _, _ = O.run(s.x, s.v, s.box, O.LJ(), 1.0, nsteps=40)
    s.x, s.v = x, v
    return s


@pytest.fixture(scope="module")
def mixture_small():
    """2-type system on a jittered fcc lattice at density 1.2."""
    x, box = jittered(8, 0.2, seed=31, density=1.2)
    n = len(x)
    t = (S.uniform(32, n) >= 0.8).astype(np.int32)
    p = S.binary_mixture_params()
    v = S.maxwell_boltzmann(p.mass[t], 1.0, 33)
    return S.System(x, v, t, box, p)


CASES = [(k, p) for k in (md.MD_LIST_FULL, md.MD_LIST_HALF) for p in (md.MD_PREC_FP64,)]


KERNELS = {"compacted": (1, -1, 1, 0), "compacted_persistent": (1, -1, 1, 1),
           "fixed": (1, -1, 2, 0), "fixed_persistent": (1, -1, 2, 1),
           "fixed2": (1, -1, 3, 0), "fixed2_persistent": (1, -1, 3, 1),
           "tpa2_persistent_l1": (2, 0, 0, 1)}


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("tpa", [1, 4, 32, "compacted", "compacted_persistent", "fixed",
                                 "fixed_persistent", "fixed2", "fixed2_persistent",
                                 "tpa2_persistent_l1"])
def test_melt_neighbors_and_forces_fp64(melt, kind, tpa):
    """Every pair-kernel configuration: threads per atom, the compacted FP64
    kernel with FP64 or fixed-point force sums, one block per tile (default)
    and persistent per-SM scheduling, the largest-L1 carveout."""
    with make(melt, list_kind=kind, threads_per_atom=tpa if isinstance(tpa, int) else 1) as ctx:
        if tpa in KERNELS:
            ctx.set_kernel(*KERNELS[tpa])
        ctx.compute_forces(0)
        x, v, f = (a.cpu().numpy() for a in ctx.get_state())
        check_neighbors(ctx, x, melt.box, melt.params.rlist, kind == md.MD_LIST_HALF)
        fref, E, W = O.forces(x, melt.box, O.LJ(), skin=0.3)
        assert rel_err(f, fref) <= FORCE_TOL
        th = ctx.energy()
        assert abs(th.pe - E) <= 1e-12 * abs(E)
        np.testing.assert_allclose(th.virial, W, rtol=1e-12, atol=1e-12 * np.abs(W).max())
        ke = O.kinetic(v, 1.0)
        assert abs(th.ke - ke) <= 1e-12 * ke
        # the forces after md_energy are still the same forces
        _, _, f2 = (a.cpu().numpy() for a in ctx.get_state())
        assert rel_err(f2, fref) <= FORCE_TOL


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("tpa", [1, 8, "compacted", "fixed", "fixed2"])
def test_mixture_two_types_fp64(mixture_small, kind, tpa):
    s = mixture_small
    with make(s, list_kind=kind, threads_per_atom=tpa if isinstance(tpa, int) else 1) as ctx:
        if tpa in KERNELS:
            ctx.set_kernel(*KERNELS[tpa])
            ctx.compute_forces(0)
        x, _, f = (a.cpu().numpy() for a in ctx.get_state())
        check_neighbors(ctx, x, s.box, s.params.rlist, kind == md.MD_LIST_HALF)
        fref, E, W = O.forces(x, s.box, lj_of(s.params), type_=s.type, skin=0.3)
        assert rel_err(f, fref) <= FORCE_TOL
        th = ctx.energy()
        assert abs(th.pe - E) <= 1e-12 * abs(E)


@pytest.mark.parametrize("case", ["fcc3_tiny_box", "random_slab", "fcc5", "close_pair", "two_atoms",
                                  "one_atom", "ragged_33"])
@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("kernel", ["tpa2", "fixed"])
def test_edge_cases_fp64(case, kind, kernel):
    """Small and degenerate boxes; random_slab's overlapping atoms give
    contributions far outside the fixed-point range (FP64 path)."""
    if case == "fcc3_tiny_box":      # L = 5.04 < 2 (rc + skin): one cell per axis
        x, box = jittered(3, 0.1, seed=41)
    elif case == "random_slab":
        box = np.array([17.3, 8.5, 12.1])
        x = S.random_positions(900, box, 3)
        x += 0.0  # overlapping atoms give huge forces; parity is still exact
    elif case == "fcc5":
        x, box = jittered(5, 0.3, seed=42)
    elif case == "close_pair":       # pair forces of 300-800: FP64 path of the fixed-point sums
        x, box = jittered(5, 0.05, seed=43)
        x[1] = x[0] + np.array([0.8, 0.0, 0.0])
    elif case == "two_atoms":
        box = np.array([10.0, 10.0, 10.0])
        x = np.array([[0.5, 0.5, 0.5], [0.5 + 2 ** (1 / 6), 0.5, 0.5]])
    elif case == "one_atom":
        box = np.array([10.0, 10.0, 10.0])
        x = np.array([[1.0, 2.0, 3.0]])
    else:                            # 33 atoms: one full tile of 32 plus a ragged tail
        box = np.array([9.0, 9.0, 9.0])
        x = S.random_positions(33, box, 5)
    n = len(x)
    v = np.zeros((n, 3))
    with md.LJMD(x, v, None, box, 1.0, 1.0, 2.5, 1.0, list_kind=kind, threads_per_atom=2) as ctx:
        if kernel == "fixed":
            ctx.set_kernel(*KERNELS["fixed"])
            ctx.compute_forces(0)
        xg, _, f = (a.cpu().numpy() for a in ctx.get_state())
        check_neighbors(ctx, xg, box, 2.8, kind == md.MD_LIST_HALF)
        fref, E, _ = O.forces(xg, box, O.LJ(), skin=0.3)
        th = ctx.energy()
        if n == 1:
            assert not f.any() and th.pe == 0.0
            return
        if kernel == "fixed":
            # the fixed-point sums resolve 2^-44: forces that FP64 gives as
            # rounding noise (two atoms at the minimum) come out as 0
            rms = np.sqrt(np.mean(np.sum(fref * fref, axis=1)))
            tol = max(FORCE_TOL * rms, np.sqrt(3) * (n - 1) * 2.0 ** -45)
            assert np.max(np.linalg.norm(f - fref, axis=1)) <= tol
        else:
            assert rel_err(f, fref) <= FORCE_TOL
        assert abs(th.pe - E) <= 1e-12 * max(1.0, abs(E))
        if case == "two_atoms":
            assert abs(th.pe + 1.0) < 1e-14 and np.abs(f).max() < 1e-12


def test_wrap_matches_oracle():
    box = np.array([9.0, 9.0, 9.0])
    x = S.random_positions(200, box, 9) * 3.0 - 9.0  # spans [-9, 18)
    with md.LJMD(x, np.zeros_like(x), None, box, 1.0, 1.0, 2.5, 1.0) as ctx:
        xg = ctx.get_state()[0].cpu().numpy()
    np.testing.assert_array_equal(xg, O.wrap(x, box))


def test_capacity_growth_keeps_sets_exact(melt):
    with make(melt, max_neigh=8) as ctx:
        st = ctx.stats()
        assert st["max_neigh"] >= st["max_count"] > 8
        x = ctx.get_state()[0].cpu().numpy()
        check_neighbors(ctx, x, melt.box, 2.8, False)


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("compacted,persistent",
                         [(0, 0), (1, 0), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1)])
def test_trajectory_fp64_matches_oracle(melt, kind, compacted, persistent):
    """25 steps with a rebuild every 5 (five rebuilds, each with a sort):
    positions, velocities and forces track the oracle's run.  persistent 2
    runs each step between rebuilds as one cooperative launch."""
    with make(melt, list_kind=kind, rebuild_every=5, threads_per_atom=1) as ctx:
        ctx.set_kernel(1, -1, compacted, persistent)
        ctx.compute_forces(0)
        x0, v0, _ = (a.cpu().numpy() for a in ctx.get_state())
        ctx.step(10)
        ctx.step(15)
        x, v, f = (a.cpu().numpy() for a in ctx.get_state())
        st = ctx.stats()
    xo, vo, fo, _ = O.run(x0, v0, melt.box, O.LJ(), 1.0, nsteps=25, rebuild_every=5)
    assert st["step"] == 25 and st["builds"] == 6
    assert st["persistent"] == persistent
    assert np.abs(x - xo).max() < 1e-11
    assert np.abs(v - vo).max() < 1e-11
    assert rel_err(f, fo) < 1e-11


def test_set_kernel_one_launch_per_step_only_where_it_exists(melt):
    """persistent 2 (one cooperative launch per step) exists for the FP64
    compacted kernel with fixed-point sums only."""
    with make(melt, precision=md.MD_PREC_MIXED, threads_per_atom=1) as ctx:
        with pytest.raises(md.MDError):
            ctx.set_kernel(1, -1, 0, 2)
        assert ctx.stats()["phase1_entries"] == 2  # the mixed walk: two entries a round
    with make(melt, threads_per_atom=1) as ctx:
        with pytest.raises(md.MDError):
            ctx.set_kernel(1, -1, 1, 2)  # FP64 sums
        with pytest.raises(md.MDError):
            ctx.set_kernel(1, -1, 2, 3)
        ctx.set_kernel(1, -1, 2, 2)
        assert ctx.stats()["persistent"] == 2
        with pytest.raises(md.MDError):
            ctx.set_kernel(1, -1, 3, 2)  # the cooperative step has one entry a round
        with pytest.raises(md.MDError):
            ctx.set_kernel(1, -1, 4, 0)
        ctx.set_kernel(1, -1, 3, 1)
        st = ctx.stats()
        assert st["compacted"] == 2 and st["phase1_entries"] == 2 and st["persistent"] == 1
        ctx.set_kernel(1, -1, 2, 0)
        assert ctx.stats()["phase1_entries"] == 1


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
def test_fixed_point_sums_do_not_depend_on_order(melt, kind):
    """Fixed-point force sums (compacted 2) add the contributions, each
    rounded to a multiple of 2^-44, as integers: the forces are bitwise the
    same whatever order the contributions arrive in (repeated launches, one
    block per tile or persistent per-SM scheduling), and they differ from
    the oracle's by at most the rounding of the contributions (count x
    2^-45) plus what FP64 summation itself differs by."""
    with make(melt, list_kind=kind, threads_per_atom=1) as ctx:
        ctx.set_kernel(1, -1, 2, 0)
        ctx.compute_forces(0)
        x, _, f1 = (a.cpu().numpy() for a in ctx.get_state())
        ctx.compute_forces(0)
        f2 = ctx.get_state()[2].cpu().numpy()
        ctx.set_kernel(1, -1, 2, 1)
        ctx.compute_forces(0)
        f3 = ctx.get_state()[2].cpu().numpy()
        ctx.set_kernel(1, -1, 1, 0)  # FP64 atomics
        ctx.compute_forces(0)
        fr = ctx.get_state()[2].cpu().numpy()
    assert np.array_equal(f1, f2) and np.array_equal(f1, f3)
    fref, _, _ = O.forces(x, melt.box, O.LJ(), skin=0.3)
    pi, pk = O.pairs_cells(x, melt.box, 2.5)
    cnt = np.bincount(pi, minlength=len(x)) + np.bincount(pk, minlength=len(x))
    bound = cnt[:, None] * 2.0 ** -45 + np.abs(fr - fref).max() + 2e-16 * np.abs(fref)
    assert np.all(np.abs(f1 - fref) <= bound)
    assert rel_err(f1, fref) <= FORCE_TOL


def test_energy_after_steps(melt):
    with make(melt) as ctx:
        x0, v0, _ = (a.cpu().numpy() for a in ctx.get_state())
        ctx.step(20)
        th = ctx.energy()
        x, v, _ = (a.cpu().numpy() for a in ctx.get_state())
    _, E, W = O.forces(x, melt.box, O.LJ(), skin=0.3)
    assert abs(th.pe - E) <= 1e-12 * abs(E)
    assert abs(th.ke - O.kinetic(v, 1.0)) <= 1e-12 * th.ke
    assert abs(th.temperature - 2 * th.ke / (3 * len(x) - 3)) < 1e-14


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("persistent", [0, 1])
def test_mixed_precision_error_reported(melt, kind, persistent, capsys):
    """Mixed form: FP32 pair arithmetic, compensated accumulation, FP64
    positions.  Its error against the FP64 oracle is a number, not a bar;
    the sanity bound is 1e-4."""
    with make(melt, list_kind=kind, precision=md.MD_PREC_MIXED, threads_per_atom=1) as ctx:
        ctx.set_kernel(2, -1, 0, persistent)
        ctx.compute_forces(0)
        x, _, f = (a.cpu().numpy() for a in ctx.get_state())
        check_neighbors(ctx, x, melt.box, 2.8, kind == md.MD_LIST_HALF)
        th = ctx.energy()
    fref, E, W = O.forces(x, melt.box, O.LJ(), skin=0.3)
    e = rel_err(f, fref)
    print(f"mixed {kind}: force err {e:.3e}, energy rel err {abs(th.pe - E) / abs(E):.3e}")
    assert e < 1e-4
    assert abs(th.pe - E) < 1e-5 * abs(E)


def test_state_roundtrip_host_and_device(melt):
    with make(melt) as ctx:
        xd, vd, fd = ctx.get_state()
        xh, vh, fh = ctx.get_state(host=True)
        np.testing.assert_array_equal(xh, xd.cpu().numpy())
        np.testing.assert_array_equal(vh, vd.cpu().numpy())
        np.testing.assert_array_equal(fh, fd.cpu().numpy())
        ctx.step(3)
        ctx.set_state(xh, vh)  # host path: back to the saved state
        x2, v2, f2 = ctx.get_state(host=True)
        np.testing.assert_array_equal(x2, xh)
        np.testing.assert_array_equal(v2, vh)
        assert rel_err(f2, fh) < 1e-14
        assert ctx.stats()["step"] == 0


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
def test_set_state_keeps_list_while_valid(melt, kind):
    """MD_MEM_KEEP_LIST: a state a few steps from the last build keeps the
    list (no rebuild) and gets exact forces; a state with an atom moved by a
    box length (or beyond skin/2) starts afresh."""
    with make(melt, list_kind=kind, threads_per_atom=1) as ctx:
        ctx.step(4)
        x, v, _ = ctx.get_state(host=True)
        b0 = ctx.stats()["builds"]
        ctx.set_state(x, v, keep_list=True)
        st = ctx.stats()
        assert st["builds"] == b0 and st["step"] == 0
        xg, _, f = (a.cpu().numpy() for a in ctx.get_state())
        np.testing.assert_array_equal(xg, x)
        fref, _, _ = O.forces(x, melt.box, O.LJ(), skin=0.3)
        assert rel_err(f, fref) <= FORCE_TOL
        ctx.step(6)  # continues from the kept list
        x6, v6, f6 = (a.cpu().numpy() for a in ctx.get_state())
        xj = x6.copy()
        xj[7, 0] += melt.box[0]  # the same physical state, one atom in another image
        ctx.set_state(xj, v6, keep_list=True)
        assert ctx.stats()["builds"] == 1  # restarted: one build since the restart
        _, _, fj = (a.cpu().numpy() for a in ctx.get_state())
    xo, _, fo, _ = O.run(x, v, melt.box, O.LJ(), 1.0, nsteps=6, rebuild_every=20, init=False)
    assert np.abs(x6 - xo).max() < 1e-11 and rel_err(f6, fo) < 1e-11
    assert rel_err(fj, f6) <= FORCE_TOL


@pytest.mark.parametrize("prec", [md.MD_PREC_FP64, md.MD_PREC_MIXED])
def test_set_state_keep_list_recomputes_forces_only_when_moved(melt, prec):
    """MD_MEM_KEEP_LIST with positions equal bit for bit to the held ones
    (new velocities only) launches no force kernel and keeps exact forces; a
    small move of one atom recomputes them on the kept list."""
    with make(melt, list_kind=md.MD_LIST_HALF, precision=prec, threads_per_atom=1) as ctx:
        ctx.step(3)
        x, v, _ = ctx.get_state(host=True)
        b0 = ctx.stats()["builds"]
        l0 = ctx.stats()["kernel_launches"]
        ctx.set_state(x, 0.5 * v, keep_list=True)
        l1 = ctx.stats()["kernel_launches"]
        assert l1 - l0 == 2  # the state load, and this stats call's count kernel
        _, vg, f = (a.cpu().numpy() for a in ctx.get_state())
        np.testing.assert_array_equal(vg, 0.5 * v)
        fref, _, _ = O.forces(x, melt.box, O.LJ(), skin=0.3)
        tol = FORCE_TOL if prec == md.MD_PREC_FP64 else 1e-4
        assert rel_err(f, fref) <= tol
        xm = x.copy()
        xm[11, 1] += 0.01
        ctx.set_state(xm, v, keep_list=True)
        st = ctx.stats()
        assert st["builds"] == b0 and st["kernel_launches"] - l1 > 2
        _, _, fm = (a.cpu().numpy() for a in ctx.get_state())
        fmref, _, _ = O.forces(xm, melt.box, O.LJ(), skin=0.3)
        assert rel_err(fm, fmref) <= tol
        assert rel_err(fm, fref) > 10 * tol  # the move changed the forces


def test_check_disp_rebuilds_when_needed(melt):
    """check_disp: from the T* = 1.44 fcc start the 20-step cadence leaves
    most builds dangerous; with the per-step displacement check the list is
    rebuilt before any force evaluation beyond skin/2, no build is
    dangerous, and the trajectory matches the oracle run with a list rebuilt
    every step (the forces then see every pair within rc)."""
    s = S.fcc_liquid(20)
    with md.LJMD(s.x, s.v, None, s.box, 1.0, 1.0, 2.5, 1.0, list_kind=md.MD_LIST_HALF,
                 threads_per_atom=1) as ctx:
        ctx.step(60)
        plain = ctx.stats()
    with md.LJMD(s.x, s.v, None, s.box, 1.0, 1.0, 2.5, 1.0, list_kind=md.MD_LIST_HALF,
                 threads_per_atom=1, check_disp=True) as ctx:
        x0, v0, _ = (a.cpu().numpy() for a in ctx.get_state())
        ctx.step(60)
        st = ctx.stats()
        x, v, f = (a.cpu().numpy() for a in ctx.get_state())
    assert plain["dangerous_builds"] > 0
    assert st["dangerous_builds"] == 0 and st["builds"] > plain["builds"]
    xo, vo, fo, _ = O.run(x0, v0, s.box, O.LJ(), 1.0, nsteps=60, rebuild_every=1)
    # chaotic growth of rounding differences over 60 steps of a melting crystal
    assert np.abs(x - xo).max() < 1e-8
    assert rel_err(f, fo) < 1e-7


def test_launch_counter_and_graph_reuse(melt):
    with make(melt, threads_per_atom=1) as ctx:
        a = ctx.stats()["kernel_launches"]
        ctx.step(40)
        b = ctx.stats()["kernel_launches"]
        ctx.step(40)
        c = ctx.stats()["kernel_launches"]
    assert b > a and c - b == b - a  # same segments, same launches


@pytest.mark.parametrize("prec", [md.MD_PREC_FP64, md.MD_PREC_MIXED])
def test_max_disp_bounds_the_displacement(melt, prec):
    """md_stats.max_disp some steps after the last build: in FP64 contexts an
    upper bound of the largest displacement (from the hi parts of the split,
    within a few grid steps, 2^-18 here, of the exact value); in mixed
    contexts the FP32 displacement of the full split, within ~1e-6 relative."""
    with make(melt, precision=prec, rebuild_every=20, threads_per_atom=1) as ctx:
        xb, _, _ = (a.cpu().numpy() for a in ctx.get_state())
        b0 = ctx.stats()["builds"]
        ctx.step(7)
        st = ctx.stats()
        x, _, _ = (a.cpu().numpy() for a in ctx.get_state())
    assert st["builds"] == b0  # no rebuild in between: x is unwrapped since xb
    true = float(np.max(np.linalg.norm(x - xb, axis=1)))
    assert true > 0.01
    if prec == md.MD_PREC_FP64:
        assert true <= st["max_disp"] <= true + 1e-4
    else:
        assert abs(st["max_disp"] - true) <= 1e-5 * true + 1e-7


@pytest.mark.parametrize("kernel", [(1, -1, 3, 0), (2, -1, 0, 0)])
def test_pair_kernel_timing_keeps_results(melt, kernel):
    """md_time_pair_kernel: the segments run without graphs, with events
    around each pair launch (one per step here); the trajectory is the same,
    bit for bit, as with the graphs."""
    prec = md.MD_PREC_FP64 if kernel[2] else md.MD_PREC_MIXED
    runs = []
    for timing in (False, True):
        with make(melt, precision=prec, rebuild_every=5, threads_per_atom=kernel[0]) as ctx:
            ctx.set_kernel(*kernel)
            ctx.compute_forces(0)
            if timing:
                ctx.time_pair_kernel(True)
            ctx.step(12)
            if timing:
                ms, k = ctx.pair_kernel_time()
                ctx.time_pair_kernel(False)
                assert k == 12 and ms > 0.0
                assert ctx._lib.md_time_pair_kernel(ctx._ctx, 2) == md.MD_EINVAL
            runs.append([a.cpu().numpy() for a in ctx.get_state()])
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)
