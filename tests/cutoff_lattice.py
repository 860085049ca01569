"""Workload of the cutoff-decision tests: isolated pairs at separations
within 2e-7 or 1e-5 (relative) of a cutoff, in a 160-wide box.

Shared by the GPU test (test_gpu_mixed_cutoff.py) and the CPU check of
the workload's own properties (test_cutoff_lattice.py).  Holds none of the
method's arithmetic beyond a plain FP32 emulation used to show that the
workload has pairs an FP32 cutoff test would decide wrongly.
"""
import numpy as np

from paper_2508_13523_gb300 import synth as S

RC = 2.5
RC_COUL = 2.2
SPACING = 8.0  # > 2 rc + rlist: the pairs do not see one another
M = 20  # sites per axis: box 160


def pair_lattice(seed, radii):
    """Two atoms per lattice site; partner at distance r * (1 + delta) along a
    random direction, r cycling through radii; |delta| <= 2e-7 on even
    sites (inside the FP64 band), <= 1e-5 on odd ones (mostly decided in
    FP32).  Sites sit at 8k - 1.25 (mod L), so that pairs on the first
    layer cross the boundary."""
    L = SPACING * M
    g = np.arange(M) * SPACING - 1.25
    site = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) % L
    ns = len(site)
    u = S.uniform(seed, 3 * ns).reshape(ns, 3) - 0.5
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    width = np.where(np.arange(ns) % 2 == 0, 4e-7, 2e-5)
    delta = (S.uniform(seed + 1, ns) - 0.5) * width
    r = np.asarray(radii)[(np.arange(ns) // 2) % len(radii)] * (1.0 + delta)
    x = np.empty((2 * ns, 3))
    x[0::2] = site
    x[1::2] = (site + r[:, None] * u) % L
    return x, np.array([L, L, L])


def fp32_flips(x, box, cut):
    """How many pairs an FP32 cutoff test would decide unlike FP64: r^2 from
    the FP32 hi/lo split of the coordinates (the mixed kernels' separation,
    without their fused multiply-adds) against r^2 in FP64."""
    f = np.float32
    a, b = x[0::2], x[1::2]
    ha, hb = a.astype(f), b.astype(f)
    la, lb = (a - ha).astype(f), (b - hb).astype(f)
    h, lo = hb - ha, lb - la
    Lf = box.astype(f)
    Ll = (box - Lf).astype(f)
    up, dn = h > Lf / 2, h < -Lf / 2
    h = np.where(up, (hb - Lf) - ha, np.where(dn, hb - (ha - Lf), h))
    lo = np.where(up, lo - Ll, np.where(dn, lo + Ll, lo))
    d32 = h + lo
    d64 = b - a
    d64 -= box * np.round(d64 / box)
    r64 = (d64 * d64).sum(1) < cut * cut
    r32 = (d32 * d32).sum(1, dtype=f) < f(cut * cut)
    return int((r64 != r32).sum())


def pair_r2(x, box):
    d = x[1::2] - x[0::2]
    d -= box * np.round(d / box)
    return (d * d).sum(1)
