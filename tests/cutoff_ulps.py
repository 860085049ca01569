"""Workload of the FP64 cutoff-decision test: isolated pairs whose squared
separation lies within a few ulps of rc^2, many of them where the exact r^2
and r^2 rounded in the order fma(dz,dz, fma(dy,dy, dx*dx)) fall on
different sides of rc^2.

Shared by the GPU test (test_gpu_fp64_cutoff.py) and the CPU check of the
workload's properties (test_cutoff_ulps.py).  Every coordinate lies in
[2, 128), where doubles are multiples of 2^-51, and each separation
component is a multiple of Q = 2^-46, so every partner position is exactly
site + d.  Holds none of the method's arithmetic beyond exact integer sums
of squares and a rational emulation of the rounded r^2 used to classify the
pairs.
"""
from fractions import Fraction

import numpy as np

RC = 2.5
Q = 2.0 ** -46          # separation grid (partners stay exact below 128)
SPACING = 9.0           # > 2 rc + rlist: the pairs do not see one another
M = 13                  # sites per axis: coordinates 9 .. 117 (+- 2.5)
BOX = 160.0
ULP = 2.0 ** -50        # ulp of doubles in [4, 8), where rc^2 = 6.25 lies


def rounded_r2(d):
    """fma(dz,dz, fma(dy,dy, dx*dx)) with each operation rounded once to
    the nearest double (Python's float() of a Fraction rounds correctly)."""
    dx, dy, dz = (Fraction(float(c)) for c in d)
    t = Fraction(float(dx) * float(dx))          # one rounded product
    t = Fraction(float(dy * dy + t))             # fma: exact, then one rounding
    return float(dz * dz + t)


def exact_r2(d):
    return sum(Fraction(float(c)) ** 2 for c in d)


def pair_offsets(seed, n, span=6):
    """n separation vectors on the Q grid with |r^2 - rc^2| < 3 ulps: for a
    random direction, the integer offsets in [-span, span]^3 of the grid
    point nearest rc u whose exact r^2 lands in that window.  A quarter of
    them lie inside rc exactly but not once rounded, an eighth the reverse
    (rarer), the rest are decided alike (shuffled)."""
    rng = np.random.default_rng(seed)
    c = Fraction(RC) ** 2
    want = {(True, False): n // 4, (False, True): n // 8}
    rest = n - n // 4 - n // 8
    want[(True, True)] = rest // 2
    want[(False, False)] = rest - rest // 2
    got = {key: [] for key in want}
    k = np.arange(-span, span + 1)
    kx, ky, kz = (a.ravel() for a in np.meshgrid(k, k, k, indexing="ij"))
    while any(len(got[key]) < want[key] for key in want):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        base = np.round(RC * u / Q)
        gx, gy, gz = base[0] + kx, base[1] + ky, base[2] + kz
        # float estimate (relative error ~1e-16, i.e. < 1 ulp here) to filter
        r2 = ((gx * Q) ** 2 + (gy * Q) ** 2 + (gz * Q) ** 2)
        for i in np.nonzero(np.abs(r2 - 6.25) < 4 * ULP)[0]:
            d = (gx[i] * Q, gy[i] * Q, gz[i] * Q)
            if abs(exact_r2(d) - c) >= 3 * Fraction(ULP):
                continue
            key = (exact_r2(d) < c, rounded_r2(d) < 6.25)
            if len(got[key]) < want[key]:
                got[key].append(d)
                break
    out = np.array([d for key in want for d in got[key]])
    return out[rng.permutation(n)]


def workload(seed):
    """Positions (2 M^3 atoms: site, partner) and the box."""
    g = SPACING * (1 + np.arange(M))
    site = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    d = pair_offsets(seed, len(site))
    x = np.empty((2 * len(site), 3))
    x[0::2] = site
    x[1::2] = site + d
    return x, np.array([BOX, BOX, BOX])


def classify(x):
    """Per pair: (inside by the exact r^2, inside by the rounded r^2)."""
    c = Fraction(RC) ** 2
    ex, ro = [], []
    for a, b in zip(x[0::2], x[1::2]):
        d = b - a  # exact: both are multiples of 2^-46 below 128
        ex.append(exact_r2(d) < c)
        ro.append(rounded_r2(d) < 6.25)
    return np.array(ex), np.array(ro)
