"""Pins of the oracle's second pair style, lj/cut/coul/cut (no GPU).

The paper's pair styles share one two-body base (Sec. 4); the second style
here adds a cut Coulomb term qqrd2e q_a q_b / r for r < rc_coul, with
per-type charges.  Each test checks the oracle against something outside
it: a closed form, a finite difference, a symmetry, the virial theorem of a
1/r potential, an independent lattice enumeration, or brute force.
"""
import numpy as np
import pytest

from paper_2508_13523_gb300 import synth as S


def _pair(r, box=40.0):
    return np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]]), np.array([box, box, box])


def _charged_box(n=4, amp=0.25, seed=21, density=0.8442):
    """Jittered fcc with two types by basis site (sites 0, 1: +q; 2, 3: -q):
    neutral, every pair type present."""
    x, box, _ = S.fcc(n, density)
    x = x + amp * (S.uniform(seed, x.size).reshape(x.shape) - 0.5)
    t = (np.arange(len(x)) % 4 >= 2).astype(np.int32)
    return x, box, t


def test_two_charges_closed_form(oracle):
    """With eps = 0: U = qqrd2e q_a q_b / r, and the force on atom 0 is
    -qq d / r^3 (d = x_1 - x_0): unlike charges attract.  Catches a wrong
    power of r, a sign error and the qqrd2e factor."""
    for qa, qb, k in ((0.7, -1.3, 1.0), (1.0, 1.0, 2.5), (-0.5, 0.25, 1.0)):
        lj = oracle.LJ(0.0, 1.0, 2.5, ntypes=2, q=[qa, qb], rc_coul=3.0, qqrd2e=k)
        x, box = _pair(1.9)
        f, E, W = oracle.forces(x, box, lj, type_=np.array([0, 1], np.int32))
        qq = k * qa * qb
        assert abs(E - qq / 1.9) <= 1e-15 * abs(qq)
        np.testing.assert_allclose(f[0], [-qq / 1.9 ** 2, 0, 0], rtol=1e-14, atol=0)
        np.testing.assert_allclose(f[1], -f[0], rtol=0, atol=0)
        # virial of one pair: fpair d_x^2 = qq / r
        assert abs(W[0] - qq / 1.9) <= 1e-14 * abs(qq)


def test_coulomb_cutoff_is_strict(oracle):
    """No Coulomb term at r = rc_coul exactly; the full term one ulp inside."""
    lj = oracle.LJ(0.0, 1.0, 1.0, ntypes=1, q=[1.0], rc_coul=2.0)
    x, box = _pair(2.0)
    f, E, _ = oracle.forces(x, box, lj)
    assert E == 0.0 and not f.any()
    x, box = _pair(np.nextafter(2.0, 0.0))
    f, E, _ = oracle.forces(x, box, lj)
    assert abs(E - 0.5) < 1e-15


def test_lj_and_coulomb_add(oracle):
    """The two terms add: forces and energy of lj/cut/coul/cut equal those
    of Eq. 1 alone plus those of the Coulomb term alone."""
    x, box, t = _charged_box()
    both = oracle.LJ(1.0, 1.0, 2.5, ntypes=2, q=[0.6, -0.6], rc_coul=2.2)
    lj = oracle.LJ(1.0, 1.0, 2.5, ntypes=2)
    co = oracle.LJ(0.0, 1.0, 2.5, ntypes=2, q=[0.6, -0.6], rc_coul=2.2)
    pairs = oracle.pairs_cells(x, box, 2.8)
    f, E, W = oracle.forces(x, box, both, type_=t, pairs=pairs)
    f1, E1, W1 = oracle.forces(x, box, lj, type_=t, pairs=pairs)
    f2, E2, W2 = oracle.forces(x, box, co, type_=t, pairs=pairs)
    np.testing.assert_allclose(f, f1 + f2, rtol=0, atol=1e-12 * np.abs(f).max())
    assert abs(E - (E1 + E2)) <= 1e-12 * abs(E1)
    np.testing.assert_allclose(W, W1 + W2, rtol=0, atol=1e-12 * np.abs(W).max())


def test_force_is_minus_energy_gradient(oracle):
    """F_i = -dE/dx_i by central differences (LJ + Coulomb, two types,
    periodic, disordered).  Catches sign, power and type-indexing mistakes
    in the Coulomb force."""
    x, box, t = _charged_box(seed=23)
    lj = oracle.LJ(1.0, 1.0, 2.5, ntypes=2, q=[0.8, -0.8], rc_coul=2.5)
    f, _, _ = oracle.forces(x, box, lj, type_=t)
    h = 1e-6
    rng = S.splitmix64(7, 12)
    for k in range(12):
        i, a = int(rng[k] % len(x)), int((rng[k] >> np.uint64(40)) % 3)
        xp, xm = x.copy(), x.copy()
        xp[i, a] += h
        xm[i, a] -= h
        fd = -(oracle.forces(xp, box, lj, type_=t)[1] - oracle.forces(xm, box, lj, type_=t)[1])
        fd /= 2 * h
        assert abs(fd - f[i, a]) <= 1e-6 * max(1.0, abs(f[i, a])), (i, a, fd, f[i, a])


def test_homogeneity_and_virial_theorem(oracle):
    """Pure Coulomb (eps = 0): E(lambda q) = lambda^2 E(q), and for a 1/r
    potential the virial trace sum_pairs fpair r^2 equals E exactly in
    exact arithmetic.  Newton's third law: the forces sum to zero."""
    x, box, t = _charged_box(seed=25)
    co = oracle.LJ(0.0, 1.0, 2.5, ntypes=2, q=[0.6, -0.6], rc_coul=2.5)
    co2 = oracle.LJ(0.0, 1.0, 2.5, ntypes=2, q=[1.2, -1.2], rc_coul=2.5)
    f, E, W = oracle.forces(x, box, co, type_=t)
    f2, E2, _ = oracle.forces(x, box, co2, type_=t)
    assert abs(E2 - 4.0 * E) <= 1e-13 * abs(E2)
    np.testing.assert_allclose(f2, 4.0 * f, rtol=1e-13, atol=1e-13 * np.abs(f2).max())
    assert abs(W[0] + W[1] + W[2] - E) <= 1e-12 * np.abs(W[:3]).sum()
    assert np.abs(f.sum(axis=0)).max() <= 1e-12 * len(x) * np.abs(f).max()


def _charged_lattice_coulomb(a, rc, q):
    """Coulomb E/N of the charged fcc lattice (sites 0, 1: +q; 2, 3: -q) by
    direct enumeration of lattice vectors |R| < rc around each basis site."""
    m = int(np.ceil(rc / a)) + 1
    g = np.arange(-m, m + 1, dtype=np.float64)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([I.ravel(), J.ravel(), K.ravel()], 1)
    qs = np.array([q, q, -q, -q])
    tot = 0.0
    for b0 in range(4):
        R = (cells[:, None, :] + S.FCC_BASIS[None] - S.FCC_BASIS[b0]) * a
        qq = qs[b0] * np.broadcast_to(qs, R.shape[:2])
        r = np.sqrt((R * R).sum(-1))
        keep = (r > 0) & (r < rc)
        tot += 0.5 * np.sum(qq[keep] / r[keep])
    return tot / 4.0


def test_charged_fcc_lattice(oracle):
    """The perfect fcc lattice with +q on sites 0, 1 and -q on 2, 3: every
    atom is a center of inversion of the charges, so all forces vanish, and
    E/N equals the Eq. 1 lattice sum plus an independent enumeration of the
    Coulomb lattice sum."""
    x, box, a = S.fcc(8)
    t = (np.arange(len(x)) % 4 >= 2).astype(np.int32)
    q = 0.5
    both = oracle.LJ(1.0, 1.0, 2.5, ntypes=2, q=[q, -q], rc_coul=2.5)
    co = oracle.LJ(0.0, 1.0, 2.5, ntypes=2, q=[q, -q], rc_coul=2.5)
    f, _, _ = oracle.forces(x, box, both, type_=t, skin=0.3)
    _, Ec, _ = oracle.forces(x, box, co, type_=t, skin=0.3)
    ec = _charged_lattice_coulomb(a, 2.5, q)
    # ~80,000 terms of both signs summed in order: a few 1e-13 relative
    assert abs(Ec / len(x) - ec) <= 1e-11 * abs(ec)
    assert np.abs(f).max() < 1e-11


def test_cells_equal_brute_force_with_longer_coulomb_cutoff(oracle):
    """rc_coul above the LJ cutoff: the cell-list pairs at rc_coul + skin
    and the brute-force pairs give the same forces."""
    x, box, t = _charged_box(n=5, seed=27)
    lj = oracle.LJ(1.0, 1.0, 2.0, ntypes=2, q=[0.5, -0.5], rc_coul=2.6)
    f1, E1, _ = oracle.forces(x, box, lj, type_=t, pairs=oracle.pairs_cells(x, box, 2.9))
    f2, E2, _ = oracle.forces(x, box, lj, type_=t, pairs=oracle.pairs_brute(x, box, 2.9))
    np.testing.assert_allclose(f1, f2, rtol=0, atol=1e-12 * np.abs(f1).max())
    assert abs(E1 - E2) <= 1e-12 * abs(E1)
    fs = oracle.force_of(x, box, lj, np.arange(0, len(x), 7), type_=t)
    np.testing.assert_allclose(fs, f1[::7], rtol=0, atol=1e-12 * np.abs(f1).max())


def test_lj_only_functions_refuse_charges(oracle):
    x, box, t = _charged_box()
    lj = oracle.LJ(1.0, 1.0, 2.5, ntypes=2, q=[0.5, -0.5])
    with pytest.raises(ValueError):
        oracle.force_vjp(x, box, lj, np.zeros_like(x), type_=t)


def test_charged_dynamics_time_reversible(oracle):
    """Velocity Verlet with LJ + cut Coulomb: 40 steps forward, velocities
    negated, 40 steps back recover the start (list rebuilt every step, so
    both directions see the same pairs).  Catches a force that is not a
    function of the positions alone and a wrong Coulomb term in the
    integrator's force calls."""
    x, box, _ = S.fcc(5)
    x = x + 0.1 * (S.uniform(33, x.size).reshape(x.shape) - 0.5)
    t = (np.arange(len(x)) % 4 >= 2).astype(np.int32)
    v = S.maxwell_boltzmann(np.ones(len(x)), 1.0, 31)
    lj = oracle.LJ(1.0, 1.0, 2.5, ntypes=2, q=[0.5, -0.5], rc_coul=2.5)
    x0 = oracle.wrap(x, box)
    x1, v1, _, _ = oracle.run(x0, v, box, lj, np.ones(2), type_=t, nsteps=40, rebuild_every=1)
    x2, v2, _, _ = oracle.run(x1, -v1, box, lj, np.ones(2), type_=t, nsteps=40,
                              rebuild_every=1, init=False)
    d = x2 - x0
    d -= box * np.round(d / box)
    assert np.abs(d).max() < 1e-9
    assert np.abs(v2 + v).max() < 1e-9
