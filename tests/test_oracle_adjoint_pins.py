"""Pins of the oracle's reverse mode (force VJP, trajectory VJP) to finite
differences of the oracle's own forward quantities and to a scaling identity
(no GPU).  The forward quantities are pinned in test_oracle_pins.py."""
import numpy as np
import pytest

from paper_2508_13523_gb300 import synth as S


def _mixture_box(n_cells=4, seed=51, amp=0.2):
    """Jittered fcc at density 1.2 with 20 % B atoms; n_cells >= 4 keeps
    every rc_ab below L/2 (one periodic image in range)."""
    x, box, _ = S.fcc(n_cells, 1.2)
    x = x + amp * (S.uniform(seed, x.size).reshape(x.shape) - 0.5)
    t = (S.uniform(seed + 1, len(x)) >= 0.8).astype(np.int32)
    return x, box, t


def _lj_with(O, eps, sigma):
    p = S.binary_mixture_params()
    return O.LJ(eps, sigma, p.rc, ntypes=2)  # rc fixed at the unperturbed sigma


UNIQUE = [(0, 0), (0, 1), (1, 1)]


def _perturbed(table, a, b, h):
    t = table.copy()
    t[a, b] += h
    if a != b:
        t[b, a] += h
    return t


def test_force_vjp_matches_finite_differences(oracle):
    """L = sum |F(theta, x) - F_ref|^2; dL/dtheta for the six unique pair
    parameters and dL/dx for a sample of coordinates, by central differences."""
    x, box, t = _mixture_box()
    p = S.binary_mixture_params()
    eps, sig = p.eps.copy(), p.sigma.copy()
    fref = 0.3 * (S.uniform(3, x.size).reshape(x.shape) - 0.5)

    def loss(e, s, xx):
        f, _, _ = oracle.forces(xx, box, _lj_with(oracle, e, s), type_=t, skin=0.3)
        return float(np.sum((f - fref) ** 2)), f

    L0, f0 = loss(eps, sig, x)
    xbar, gbar = oracle.force_vjp(x, box, _lj_with(oracle, eps, sig), 2 * (f0 - fref), type_=t,
                                  skin=0.3)
    for which, table in ((0, eps), (1, sig)):
        for a, b in UNIQUE:
            h = 1e-6 * table[a, b]
            args_p = [eps, sig]
            args_m = [eps, sig]
            args_p[which] = _perturbed(table, a, b, h)
            args_m[which] = _perturbed(table, a, b, -h)
            fd = (loss(*args_p, x)[0] - loss(*args_m, x)[0]) / (2 * h)
            assert abs(fd - gbar[which, a, b]) <= 1e-6 * max(1.0, abs(fd)), (which, a, b)
            assert gbar[which, a, b] == gbar[which, b, a]
    rng = S.splitmix64(9, 10)
    for r in rng:
        i, c = int(r % len(x)), int((r >> np.uint64(33)) % 3)
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[i, c] += h
        xm[i, c] -= h
        fd = (loss(eps, sig, xp)[0] - loss(eps, sig, xm)[0]) / (2 * h)
        assert abs(fd - xbar[i, c]) <= 1e-6 * max(1.0, abs(fd)), (i, c)


def test_force_vjp_invariances(oracle):
    """Translation invariance: sum_i dL/dx_i = 0.  Homogeneity in eps: with
    F_ref = 0, L is quadratic in eps, so sum_ab eps_ab dL/deps_ab = 2 L
    (each unordered pair parameter counted once)."""
    x, box, t = _mixture_box(seed=61)
    p = S.binary_mixture_params()
    lj = _lj_with(oracle, p.eps, p.sigma)
    f, _, _ = oracle.forces(x, box, lj, type_=t, skin=0.3)
    xbar, gbar = oracle.force_vjp(x, box, lj, 2 * f, type_=t, skin=0.3)
    assert np.abs(xbar.sum(axis=0)).max() <= 1e-10 * np.abs(xbar).max()
    L = float(np.sum(f * f))
    s = sum(p.eps[a, b] * gbar[0, a, b] for a, b in UNIQUE)
    assert abs(s - 2 * L) <= 1e-10 * L


def _traj_loss(oracle, x0, v0, box, t, eps, sig, fref, K, every):
    lj = _lj_with(oracle, eps, sig)
    _, _, f, _ = oracle.run(x0, v0, box, lj, np.array([1.0, 1.0]), type_=t, nsteps=K,
                            rebuild_every=every)
    return float(np.sum((f - fref) ** 2)), f


@pytest.mark.parametrize("K,every", [(0, 5), (1, 5), (12, 5)])
def test_traj_vjp_matches_finite_differences(oracle, K, every):
    """Backprop through K velocity-Verlet steps (with list rebuilds) against
    central differences of the trajectory loss in theta, x0 and v0.  The
    unshifted cutoff makes the loss jump when a pair crosses rc between the
    two perturbed runs; two step sizes must agree, which rules that out."""
    x, box, t = _mixture_box(n_cells=4, seed=71, amp=0.15)  # L = 5.98 > 2 rc_max
    p = S.binary_mixture_params()
    v0 = S.maxwell_boltzmann(p.mass[t], 1.0, 72)
    eps, sig = p.eps.copy(), p.sigma.copy()
    fref = _traj_loss(oracle, x, v0, box, t, 1.05 * eps, 1.05 * sig, 0.0, K, every)[1]
    L0, fK = _traj_loss(oracle, x, v0, box, t, eps, sig, fref, K, every)
    xb, vb, gb = oracle.traj_vjp(x, v0, box, _lj_with(oracle, eps, sig), np.array([1.0, 1.0]),
                                 2 * (fK - fref), type_=t, nsteps=K, rebuild_every=every)

    def fd(fun, h):
        return (fun(h) - fun(-h)) / (2 * h)

    checks = []
    for which, table in ((0, eps), (1, sig)):
        for a, b in UNIQUE:
            def fun(h, which=which, table=table, a=a, b=b):
                args = [eps, sig]
                args[which] = _perturbed(table, a, b, h)
                return _traj_loss(oracle, x, v0, box, t, *args, fref, K, every)[0]
            checks.append((fun, gb[which, a, b]))
    rng = S.splitmix64(73, 6)
    for r in rng:
        i, c = int(r % len(x)), int((r >> np.uint64(33)) % 3)
        def fx(h, i=i, c=c):
            xx = x.copy()
            xx[i, c] += h
            return _traj_loss(oracle, xx, v0, box, t, eps, sig, fref, K, every)[0]
        def fv(h, i=i, c=c):
            vv = v0.copy()
            vv[i, c] += h
            return _traj_loss(oracle, x, vv, box, t, eps, sig, fref, K, every)[0]
        checks.append((fx, xb[i, c]))
        checks.append((fv, vb[i, c]))
    # step h: truncation (h^2, removed by Richardson) against rounding of L
    # (~ u L / h absolute, with L ~ 1e6 here); h = 1e-4 already moves a pair
    # across rc for sigma_AA in this run
    h = 1e-5
    floor = 50 * np.finfo(float).eps * max(1.0, L0) / h
    for fun, an in checks:
        a1, a2 = fd(fun, h), fd(fun, h / 2)
        assert abs(a1 - a2) <= 1e-4 * max(1.0, abs(a1)) + floor, "a pair crossed rc"
        rich = (4.0 * a2 - a1) / 3.0  # Richardson: removes the h^2 term
        assert abs(rich - an) <= 1e-6 * max(1.0, abs(an)) + floor, (rich, an)


def test_sd_relax_lowers_energy_and_max_force(oracle):
    s = S.binary_mixture(n=500, seed=3)
    lj = _lj_with(oracle, s.params.eps, s.params.sigma)
    _, E0, _ = oracle.forces(s.x, s.box, lj, type_=s.type)
    x = oracle.sd_relax(s.x, s.box, lj, 200, 0.01, type_=s.type)
    f, E1, _ = oracle.forces(x, s.box, lj, type_=s.type)
    assert E1 < E0 and np.isfinite(E1)
    assert np.linalg.norm(f, axis=1).max() < 1e3
