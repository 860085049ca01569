"""Pins of the FP64 CPU oracle to facts fixed outside it (no GPU).

Each test checks the oracle against something other than itself: a closed
form of Eq. 1 (arXiv 2508.13523, Sec. 4), a textbook lattice sum, a library
routine, a finite difference, a symmetry or conservation law, or brute force.
The mistakes each one catches are named in its docstring.
"""
import os

import numpy as np
import pytest

from paper_2508_13523_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_table(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def _pair_system(r, box=40.0):
    # atom 0 at the origin so that the separation is exactly r
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    return x, np.array([box, box, box])


# ---- Eq. 1 closed forms -------------------------------------------------------

def test_two_atom_minimum(oracle):
    """At r = 2^(1/6) sigma the pair force vanishes and U = -eps (Eq. 1).
    Catches a wrong exponent, a wrong prefactor in U or fpair."""
    for eps, sigma in ((1.0, 1.0), (1.5, 0.8), (0.5, 0.88)):
        lj = oracle.LJ(eps, sigma, 2.5 * sigma)
        x, box = _pair_system(2.0 ** (1.0 / 6.0) * sigma)
        f, E, _ = oracle.forces(x, box, lj)
        assert abs(E + eps) <= 1e-14 * eps
        assert np.abs(f).max() <= 1e-12 * eps / sigma


def test_two_atom_closed_values(oracle):
    """U(sigma) = 0 with repulsive force 24 eps / sigma; U(2 sigma) =
    4 eps (2^-12 - 2^-6) = -0.0615234375 eps (exact in binary).
    Catches a sign error in the force direction and the 24/48 factors."""
    lj = oracle.LJ(1.0, 1.0, 2.5)
    x, box = _pair_system(1.0)
    f, E, _ = oracle.forces(x, box, lj)
    assert abs(E) < 1e-15
    # atom 0 sits at smaller x: repulsion pushes it towards -x
    np.testing.assert_allclose(f[0], [-24.0, 0, 0], rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(f[1], [24.0, 0, 0], rtol=1e-15, atol=1e-15)
    x, box = _pair_system(2.0)
    _, E, _ = oracle.forces(x, box, lj)
    assert E == -0.0615234375


def test_cutoff_is_strict_and_unshifted(oracle):
    """Eq. 1 sums r < rc only and does not shift U: just inside rc the pair
    contributes the bare U(r); at and beyond rc it contributes nothing."""
    lj = oracle.LJ(1.0, 1.0, 2.5)
    r_in = np.nextafter(2.5, 0.0)
    x, box = _pair_system(r_in)
    _, E, _ = oracle.forces(x, box, lj)
    assert abs(E - 4.0 * (r_in ** -12 - r_in ** -6)) < 1e-16
    for r in (2.5, 2.6):
        x, box = _pair_system(r)
        f, E, _ = oracle.forces(x, box, lj)
        assert E == 0.0 and not f.any()


# ---- forces are minus the gradient of Eq. 1 -----------------------------------

def _jittered_fcc(n, amp, seed, density=0.8442):
    x, box, _ = S.fcc(n, density)
    return x + amp * (S.uniform(seed, x.size).reshape(x.shape) - 0.5), box


@pytest.mark.parametrize("mixture", [False, True])
def test_force_is_minus_energy_gradient(oracle, mixture):
    """F_i = -dE/dx_i by central differences on a periodic, disordered box.
    With two atom types this also pins the type-pair indexing of eps, sigma,
    rc.  Catches sign or index mistakes in the force and in minimum image."""
    x, box = _jittered_fcc(4, 0.25, seed=11)
    if mixture:
        p = S.binary_mixture_params()
        lj = oracle.LJ(p.eps, p.sigma, p.rc, ntypes=2)
        t = (S.uniform(3, len(x)) < 0.3).astype(np.int32)
    else:
        lj = oracle.LJ(1.0, 1.0, 2.5)
        t = None
    f, _, _ = oracle.forces(x, box, lj, type_=t)
    h = 1e-6
    rng = S.splitmix64(5, 12)
    for k in range(12):
        i, a = int(rng[k] % len(x)), int((rng[k] >> np.uint64(40)) % 3)
        xp, xm = x.copy(), x.copy()
        xp[i, a] += h
        xm[i, a] -= h
        Ep = oracle.forces(xp, box, lj, type_=t)[1]
        Em = oracle.forces(xm, box, lj, type_=t)[1]
        fd = -(Ep - Em) / (2 * h)
        assert abs(fd - f[i, a]) <= 1e-6 * max(1.0, abs(f[i, a])), (i, a, fd, f[i, a])


def test_newton_third_law(oracle):
    """Total force vanishes (each pair adds equal and opposite forces)."""
    x, box = _jittered_fcc(5, 0.3, seed=2)
    f, _, _ = oracle.forces(x, box, oracle.LJ())
    assert np.abs(f.sum(axis=0)).max() <= 1e-13 * len(x) * np.abs(f).max()


# ---- fcc lattice sums ---------------------------------------------------------

def _fcc_lattice_energy(a, rc, sigma=1.0, eps=1.0):
    """E/N of a perfect fcc crystal by direct enumeration of lattice vectors
    |R| < rc around one atom (no box, no neighbor list)."""
    m = int(np.ceil(rc / a)) + 1
    g = np.arange(-m, m + 1, dtype=np.float64)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([I.ravel(), J.ravel(), K.ravel()], 1)
    R = ((cells[:, None, :] + S.FCC_BASIS[None]) * a).reshape(-1, 3)
    r = np.sqrt((R * R).sum(1))
    r = np.sort(r[(r > 0) & (r < rc)])
    return 0.5 * np.sum(4 * eps * ((sigma / r) ** 12 - (sigma / r) ** 6))


def test_lattice_enumeration_matches_textbook_sums():
    """The enumeration used below, taken to a large cutoff plus the analytic
    r^-6 tail, reproduces the Lennard-Jones-Ingham fcc sums A12, A6."""
    g = _golden_table("fcc_lattice_sums.txt")
    a = S.fcc_constant(0.8442)
    R = 24 * a
    e = _fcc_lattice_energy(a, R)
    tail = -8.0 * np.pi * 0.8442 / (3.0 * R ** 3)  # (1/2) rho int_R^inf 4 pi r^2 (-4/r^6)
    s = np.sqrt(2.0) / a
    textbook = 2.0 * (g["A12"] * s ** 12 - g["A6"] * s ** 6)
    assert abs(e + tail - textbook) < 2e-5


def test_fcc_crystal_energy_and_zero_forces(oracle):
    """Perfect fcc 20^3 (the 32,000-atom melt start): every force is zero by
    symmetry and E/N equals the lattice sum at rc = 2.5 (-6.77336805325...)."""
    x, box, a = S.fcc(20)
    f, E, W = oracle.forces(x, box, oracle.LJ(), skin=0.3)
    ref = _fcc_lattice_energy(a, 2.5)
    assert abs(ref - (-6.7733680532529545)) < 1e-12
    # sequential summation of ~864,000 pair terms: bound n*u ~ 1e-10 relative
    assert abs(E / len(x) - ref) <= 1e-10 * abs(ref)
    assert np.abs(f).max() < 1e-10
    # cubic symmetry of the virial
    assert abs(W[0] - W[1]) < 1e-9 * abs(W[0]) and abs(W[0] - W[2]) < 1e-9 * abs(W[0])
    assert np.abs(W[3:]).max() < 1e-9 * abs(W[0])


# ---- virial -------------------------------------------------------------------

def test_virial_diagonal_by_box_scaling(oracle):
    """W_aa = -dE/dlambda for x_a -> lambda x_a, L_a -> lambda L_a at lambda=1."""
    x, box = _jittered_fcc(4, 0.2, seed=9)
    lj = oracle.LJ()
    _, _, W = oracle.forces(x, box, lj)
    h = 1e-6
    for a in range(3):
        s = np.ones(3)
        s[a] = 1 + h
        Ep = oracle.forces(x * s, box * s, lj)[1]
        s[a] = 1 - h
        Em = oracle.forces(x * s, box * s, lj)[1]
        assert abs(-(Ep - Em) / (2 * h) - W[a]) <= 1e-6 * abs(W[a])


def test_virial_offdiagonal_by_shear(oracle):
    """W_ab = -dE/dgamma for x_a -> x_a + gamma x_b on an isolated cluster
    (box far larger than the cluster, so no periodic image interacts)."""
    xc, _, _ = S.fcc(3, 0.9)
    xc = xc + 0.15 * (S.uniform(21, xc.size).reshape(xc.shape) - 0.5)
    x = xc + 30.0
    box = np.array([100.0, 100.0, 100.0])
    lj = oracle.LJ()
    _, _, W = oracle.forces(x, box, lj)
    h = 1e-6
    for (a, b), w in (((0, 1), W[3]), ((0, 2), W[4]), ((1, 2), W[5])):
        def E(g):
            y = xc.copy()
            y[:, a] += g * xc[:, b]
            return oracle.forces(y + 30.0, box, lj)[1]
        fd = -(E(h) - E(-h)) / (2 * h)
        assert abs(fd - w) <= 1e-6 * max(1.0, abs(w)), (a, b, fd, w)


# ---- neighbor sets ------------------------------------------------------------

def _pairset(pi, pk):
    return set(zip(np.minimum(pi, pk).tolist(), np.maximum(pi, pk).tolist()))


@pytest.mark.parametrize("case", ["random_cube", "random_slab", "fcc3", "fcc4", "fcc5",
                                  "melt_like"])
def test_pairs_brute_equals_cells_equals_kdtree(oracle, case):
    """Brute-force pairs == the oracle's cell-list pairs == scipy's periodic
    k-d tree (an independent library), as exact sets."""
    spatial = pytest.importorskip("scipy.spatial")
    rlist = 2.8
    if case == "random_cube":
        box = np.array([9.7, 9.7, 9.7])
        x = S.random_positions(900, box, 1)
    elif case == "random_slab":
        box = np.array([17.3, 8.5, 12.1])
        x = S.random_positions(1500, box, 2)
    elif case == "melt_like":
        x, box = _jittered_fcc(6, 0.4, seed=4)
    else:
        x, box, _ = S.fcc(int(case[-1]))
        x = x + 0.05 * (S.uniform(7, x.size).reshape(x.shape) - 0.5)
    xw = oracle.wrap(x, box)
    b = _pairset(*oracle.pairs_brute(xw, box, rlist))
    c = _pairset(*oracle.pairs_cells(xw, box, rlist))
    assert b == c
    if np.all(box > 2 * rlist):  # the k-d tree needs a single image in range
        t = spatial.cKDTree(xw, boxsize=box)
        k = {tuple(p) for p in t.query_pairs(rlist, output_type="ndarray").tolist()}
        assert b == k
    assert len(b) > 0


def test_neighbors_of_matches_pairs(oracle):
    x, box = _jittered_fcc(5, 0.3, seed=6)
    pi, pk = oracle.pairs_brute(x, box, 2.8)
    sample = np.array([0, 7, 133, len(x) - 1])
    lists = oracle.neighbors_of(x, box, 2.8, sample)
    for s, i in enumerate(sample):
        ref = sorted(set(pk[pi == i].tolist()) | set(pi[pk == i].tolist()))
        assert lists[s].tolist() == ref


def test_force_of_matches_forces(oracle):
    x, box = _jittered_fcc(5, 0.3, seed=8)
    lj = oracle.LJ()
    f, _, _ = oracle.forces(x, box, lj)
    sample = np.arange(0, len(x), 37)
    np.testing.assert_allclose(oracle.force_of(x, box, lj, sample), f[sample],
                               rtol=1e-12, atol=1e-12)


def test_min_image_and_wrap(oracle):
    L = 10.0
    assert oracle.min_image(6.0, L) == -4.0
    assert oracle.min_image(-6.0, L) == 4.0
    assert oracle.min_image(5.0, L) == 5.0      # rint(0.5) = 0: half to even
    assert oracle.min_image(15.0, L) == -5.0    # rint(1.5) = 2
    x = np.array([[-0.5, 10.0, 23.0], [9.999, -10.0, -1e-20]])
    w = oracle.wrap(x, np.array([L, L, L]))
    assert np.all(w >= 0) and np.all(w < L)
    k = (x - w) / L
    assert np.allclose(k, np.round(k), atol=1e-12)


# ---- velocity Verlet ----------------------------------------------------------

def test_generator_temperature(oracle):
    """The generator's velocities carry exactly T = 2 KE / (3N - 3) with zero
    momentum (cross-checks the generator against the oracle's KE)."""
    sysm = S.fcc_liquid(5)
    ke = oracle.kinetic(sysm.v, sysm.params.mass, sysm.type)
    assert abs(2 * ke / (3 * sysm.n - 3) - 1.44) < 1e-12
    assert np.abs(sysm.v.sum(axis=0)).max() < 1e-12


def test_free_flight(oracle):
    """Atoms farther apart than rc feel no force: x(t) = x0 + t v exactly up
    to rounding, v constant.  Catches a drift that uses the wrong velocity."""
    g = np.arange(4, dtype=np.float64) * 3.0 + 1.0
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    x = np.stack([I.ravel(), J.ravel(), K.ravel()], 1)
    box = np.array([12.0, 12.0, 12.0])
    v = 0.01 * (S.uniform(3, x.size).reshape(x.shape) - 0.5)
    xt, vt, f, _ = oracle.run(x, v, box, oracle.LJ(), 1.0, nsteps=50, rebuild_every=1000)
    assert not f.any()
    np.testing.assert_array_equal(vt, v)
    np.testing.assert_allclose(xt, x + 50 * 0.005 * v, rtol=0, atol=1e-13)


def _bound_pair_energy_error(oracle, dt):
    x, box = _pair_system(1.3)
    v = np.zeros((2, 3))
    lj = oracle.LJ()
    steps = int(round(4.0 / dt))
    _, _, _, th = oracle.run(x, v, box, lj, 1.0, dt=dt, nsteps=steps, rebuild_every=10 ** 9,
                             thermo_every=1)
    e = th[:, 1] + th[:, 2]
    return np.abs(e - e[0]).max()


def test_verlet_is_second_order(oracle):
    """Energy error of velocity Verlet on a bound pair scales as dt^2: halving
    dt divides it by ~4.  A first-order mistake (e.g. a kick with stale
    forces) gives ~2 instead."""
    e1 = _bound_pair_energy_error(oracle, 0.004)
    e2 = _bound_pair_energy_error(oracle, 0.002)
    assert 3.5 < e1 / e2 < 4.5, (e1, e2)


def test_time_reversibility_and_momentum(oracle):
    """Run 40 steps, negate v, run 40 steps: the start is recovered (Verlet is
    time reversible); total momentum stays zero throughout.  The list is
    rebuilt every step so that the forces are exactly Eq. 1 at every step: a
    list kept for 20 steps from the T*=1.44 fcc start misses pairs that close
    in by more than the skin, and the two runs would then use different lists."""
    sysm = S.fcc_liquid(4, T=1.44)
    lj = oracle.LJ()
    x1, v1, _, _ = oracle.run(sysm.x, sysm.v, sysm.box, lj, 1.0, nsteps=40, rebuild_every=1)
    assert np.abs(v1.sum(axis=0)).max() < 1e-11
    x2, v2, _, _ = oracle.run(x1, -v1, sysm.box, lj, 1.0, nsteps=40, step0=40, init=False,
                              rebuild_every=1)
    d = x2 - oracle.wrap(sysm.x, sysm.box)
    d -= sysm.box * np.round(d / sysm.box)
    assert np.abs(d).max() < 1e-12
    np.testing.assert_allclose(-v2, sysm.v, atol=1e-12)


@pytest.mark.slow
def test_melt_energy_drift(oracle):
    """NVE over the 32,000-atom melt, 100 steps, list rebuilt every 20 steps.
    Eq. 1 is truncated without a shift, so E jumps by U(rc) = -0.0163 eps
    whenever a pair crosses rc; as the crystal melts, pairs enter the cutoff
    sphere and E/N falls by about 0.009 over these 100 steps.  The bound below
    (0.02 per atom) only rules out a blow-up; the conservation pins are the
    dt^2 scaling and the time reversibility above."""
    sysm = S.fcc_liquid(20)
    _, _, _, th = oracle.run(sysm.x, sysm.v, sysm.box, oracle.LJ(), 1.0, nsteps=100,
                             thermo_every=10)
    e = (th[:, 1] + th[:, 2]) / sysm.n
    assert np.abs(e - e[0]).max() < 2e-2
    assert np.isfinite(th).all()


def test_energy_is_virial_trace_over_12_minus_half_lj4_sum_r6():
    """The identity the FP64 GPU kernels use for the energy of one type
    (Eq. 1): lj1 = 12 lj3 and lj2 = 6 lj4, so a pair's energy is
    fpair r^2 / 12 - (lj4 / 2) r^-6 and the total is trace(W) / 12 -
    (lj4 / 2) sum over pairs within rc of r^-6.  Checked on the oracle's own
    E and W for a disordered box, with the r^-6 sum taken here from the
    pair separations."""
    import oracle as O
    from paper_2508_13523_gb300 import synth as S
    s = S.fcc_liquid(6)
    rng = np.random.default_rng(7)
    x = s.x + 0.2 * (rng.random(s.x.shape) - 0.5)
    for eps, sig in ((1.0, 1.0), (1.3, 0.9)):
        lj = O.LJ(eps=eps, sigma=sig, rc=2.5 * sig)
        _, E, W = O.forces(x, s.box, lj)
        pi, pk = O.pairs_brute(x, s.box, lj.rcut)
        d = x[pk] - x[pi]
        d -= s.box * np.rint(d / s.box)
        r2 = np.sum(d * d, axis=1)
        inr = r2 < lj.rcut ** 2
        sum_r6 = np.sum((sig * sig / r2[inr]) ** 3)
        lj4 = 4.0 * eps  # lj4 / sigma^6, with r^-6 taken in units of sigma
        assert abs((W[0] + W[1] + W[2]) / 12.0 - 0.5 * lj4 * sum_r6 - E) <= 1e-12 * abs(E)
