"""FP64 CPU oracle for the Lennard-Jones lj/cut step (arXiv 2508.13523, Sec. 4).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2508_13523_gb300``)
and neither imports the other; both read their inputs from
``paper_2508_13523_gb300.synth``, which holds no arithmetic of the method.

The arithmetic lives in ``ljmd_oracle.c`` (plain C, FP64, one thread,
``-ffp-contract=off``); this module only marshals numpy arrays through ctypes.
Every function names the passage it follows in the C source's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ljmd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_min_image.restype = ctypes.c_double
        lib.orc_min_image.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_wrap.argtypes = [_I64, _d, _d]
        for name in ("orc_pairs_brute", "orc_pairs_cells"):
            fn = getattr(lib, name)
            fn.restype = _I64
            fn.argtypes = [_I64, _d, _d, ctypes.c_double, _I64, _i32, _i32]
        lib.orc_neighbors_of.argtypes = [_I64, _d, _d, ctypes.c_double, _I64, _i64, _I64,
                                         _i32, _i64]
        lib.orc_forces.argtypes = [_I64, _d, _i32, _d, ctypes.c_int32, _d, _d, _d, _d,
                                   ctypes.c_double, _I64, _i32, _i32, _d, _d]
        lib.orc_force_of.argtypes = [_I64, _d, _i32, _d, ctypes.c_int32, _d, _d, _d, _d,
                                     ctypes.c_double, _I64, _i64, _d]
        lib.orc_kinetic.restype = ctypes.c_double
        lib.orc_kinetic.argtypes = [_I64, _d, _i32, _d]
        lib.orc_force_vjp.argtypes = [_I64, _d, _i32, _d, ctypes.c_int32, _d, _d, _d, _I64,
                                      _i32, _i32, _d, _d, _d]
        lib.orc_traj_vjp.restype = ctypes.c_int
        lib.orc_traj_vjp.argtypes = [_I64, _d, _d, _i32, _d, ctypes.c_int32, _d, _d, _d, _d,
                                     ctypes.c_double, ctypes.c_double, _I64, ctypes.c_int32, _d,
                                     _d, _d, _d]
        lib.orc_sd_relax.restype = ctypes.c_int
        lib.orc_sd_relax.argtypes = [_I64, _d, _i32, _d, ctypes.c_int32, _d, _d, _d, _I64,
                                     ctypes.c_double]
        lib.orc_run.restype = _I64
        lib.orc_run.argtypes = [_I64, _d, _d, _d, _i32, _d, ctypes.c_int32, _d, _d, _d, _d,
                                ctypes.c_double, _d, ctypes.c_double, ctypes.c_double, _I64,
                                _I64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _d]
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _types(type_, n):
    if type_ is None:
        return np.zeros(n, dtype=np.int32)
    return np.ascontiguousarray(type_, dtype=np.int32)


def _table(v, nt):
    a = np.asarray(v, dtype=np.float64)
    if a.ndim == 0:
        a = np.full((nt, nt), float(a))
    return np.ascontiguousarray(a.reshape(nt, nt))


class LJ:
    """Per-type-pair Eq. 1 coefficients: eps, sigma, rc as (ntypes, ntypes).

    With per-type charges q (length ntypes) the pair style is
    lj/cut/coul/cut: Eq. 1 plus qqrd2e q_a q_b / r for r < rc_coul (default:
    the largest rc)."""

    def __init__(self, eps=1.0, sigma=1.0, rc=2.5, ntypes=1, q=None, rc_coul=None,
                 qqrd2e=1.0):
        self.ntypes = int(ntypes)
        self.eps = _table(eps, self.ntypes)
        self.sigma = _table(sigma, self.ntypes)
        self.rc = _table(rc, self.ntypes)
        self.qq = None
        self.rc_coul = 0.0
        if q is not None:
            qt = np.asarray(q, dtype=np.float64).reshape(self.ntypes)
            self.qq = np.ascontiguousarray(float(qqrd2e) * np.outer(qt, qt))
            self.rc_coul = float(self.rc.max() if rc_coul is None else rc_coul)

    @property
    def rcut(self):
        """The largest cutoff of any term."""
        return max(float(self.rc.max()), self.rc_coul)

    def _args(self):
        return (ctypes.c_int32(self.ntypes), _p(self.eps, _d), _p(self.sigma, _d),
                _p(self.rc, _d))

    def _cargs(self):
        return (_p(self.qq, _d) if self.qq is not None else None, ctypes.c_double(self.rc_coul))

    def _lj_only(self, what):
        if self.qq is not None:
            raise ValueError(f"{what}: Eq. 1 (lj/cut) only, no Coulomb term")


def min_image(d: float, L: float) -> float:
    return _load().orc_min_image(float(d), float(L))


def wrap(x, box):
    """Return a copy of x (n,3) wrapped into [0, L)."""
    x = _f64(x, (-1, 3)).copy()
    box = _f64(box)
    _load().orc_wrap(len(x), _p(x, _d), _p(box, _d))
    return x


def _pairs(fn, x, box, rlist):
    x = _f64(x, (-1, 3))
    box = _f64(box)
    cap = max(16, 64 * len(x))
    while True:
        pi = np.empty(cap, np.int32)
        pk = np.empty(cap, np.int32)
        m = fn(len(x), _p(x, _d), _p(box, _d), float(rlist), cap, _p(pi, _i32), _p(pk, _i32))
        if m <= cap:
            return pi[:m].copy(), pk[:m].copy()
        cap = int(m)


def pairs_brute(x, box, rlist):
    """All pairs i<k with minimum-image distance < rlist, lexicographic."""
    return _pairs(_load().orc_pairs_brute, x, box, rlist)


def pairs_cells(x, box, rlist):
    """The same pair set found with the oracle's own linked-cell list."""
    return _pairs(_load().orc_pairs_cells, x, box, rlist)


def neighbors_of(x, box, rlist, sample, cap_per=512):
    """Ascending full neighbor list (distance < rlist) of each sampled atom."""
    x = _f64(x, (-1, 3))
    box = _f64(box)
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    out = np.empty((len(sample), cap_per), np.int32)
    counts = np.empty(len(sample), np.int64)
    _load().orc_neighbors_of(len(x), _p(x, _d), _p(box, _d), float(rlist), len(sample),
                             _p(sample, _i64), cap_per, _p(out, _i32), _p(counts, _i64))
    if counts.size and counts.max() > cap_per:
        return neighbors_of(x, box, rlist, sample, int(counts.max()))
    return [out[s, :counts[s]].copy() for s in range(len(sample))]


def forces(x, box, lj: LJ, type_=None, pairs=None, skin=0.0):
    """Forces (n,3), energy and virial (Eq. 1 and its derivative).

    Returns (f, E, W) with W = [xx, yy, zz, xy, xz, yz].  The pair list is
    built with the cell list at max(rc)+skin unless given."""
    x = _f64(x, (-1, 3))
    box = _f64(box)
    n = len(x)
    t = _types(type_, n)
    if pairs is None:
        pairs = pairs_cells(x, box, lj.rcut + skin)
    pi, pk = (np.ascontiguousarray(p, dtype=np.int32) for p in pairs)
    f = np.empty((n, 3))
    ev = np.empty(7)
    _load().orc_forces(n, _p(x, _d), _p(t, _i32), _p(box, _d), *lj._args(), *lj._cargs(),
                       len(pi), _p(pi, _i32), _p(pk, _i32), _p(f, _d), _p(ev, _d))
    return f, ev[0], ev[1:].copy()


def force_of(x, box, lj: LJ, sample, type_=None):
    """Force on each sampled atom by a scan over all atoms (no list)."""
    x = _f64(x, (-1, 3))
    box = _f64(box)
    t = _types(type_, len(x))
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    f = np.empty((len(sample), 3))
    _load().orc_force_of(len(x), _p(x, _d), _p(t, _i32), _p(box, _d), *lj._args(),
                         *lj._cargs(), len(sample), _p(sample, _i64), _p(f, _d))
    return f


def kinetic(v, mass, type_=None):
    v = _f64(v, (-1, 3))
    t = _types(type_, len(v))
    m = _f64(np.atleast_1d(mass))
    return _load().orc_kinetic(len(v), _p(v, _d), _p(t, _i32), _p(m, _d))


def run(x, v, box, lj: LJ, mass, *, type_=None, skin=0.3, dt=0.005, nsteps=1, step0=0,
        rebuild_every=20, init=True, thermo_every=0):
    """Velocity Verlet NVE.  Returns (x, v, f, thermo) with thermo rows
    (step, E_pot, E_kin, W_xx, W_yy, W_zz, W_xy, W_xz, W_yz)."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    n = len(x)
    f = np.zeros((n, 3))
    t = _types(type_, n)
    box = _f64(box)
    m = _f64(np.atleast_1d(mass))
    nrec = 1 + (nsteps // thermo_every if thermo_every > 0 else 0)
    th = np.zeros((nrec, 9))
    r = _load().orc_run(n, _p(x, _d), _p(v, _d), _p(f, _d), _p(t, _i32), _p(box, _d),
                        *lj._args(), *lj._cargs(), _p(m, _d), float(skin), float(dt),
                        int(nsteps), int(step0),
                        int(rebuild_every), int(bool(init)), int(thermo_every), _p(th, _d))
    if r < 0:
        raise MemoryError("oracle run: allocation failed")
    return x, v, f, th[:r]


def force_vjp(x, box, lj: LJ, c, type_=None, pairs=None, skin=0.0):
    """dL/dx (n,3) and dL/d(eps, sigma) (2, nt, nt) for the cotangent
    c = dL/dF of the forces at x (chain rule of Eq. 1's derivative)."""
    lj._lj_only("force_vjp")
    x = _f64(x, (-1, 3))
    box = _f64(box)
    n = len(x)
    t = _types(type_, n)
    if pairs is None:
        pairs = pairs_cells(x, box, float(lj.rc.max()) + skin)
    pi, pk = (np.ascontiguousarray(p, dtype=np.int32) for p in pairs)
    c = _f64(c, (-1, 3))
    xbar = np.empty((n, 3))
    gbar = np.empty(2 * lj.ntypes ** 2)
    _load().orc_force_vjp(n, _p(x, _d), _p(t, _i32), _p(box, _d), *lj._args(), len(pi),
                          _p(pi, _i32), _p(pk, _i32), _p(c, _d), _p(xbar, _d), _p(gbar, _d))
    return xbar, gbar.reshape(2, lj.ntypes, lj.ntypes)


def traj_vjp(x0, v0, box, lj: LJ, mass, cF, *, type_=None, skin=0.3, dt=0.005, nsteps=1,
             rebuild_every=20):
    """Reverse mode through `run(init=True)`: given cF = dL/dF at the final
    positions, returns (dL/dx0, dL/dv0, dL/d(eps, sigma))."""
    lj._lj_only("traj_vjp")
    x0 = _f64(x0, (-1, 3))
    v0 = _f64(v0, (-1, 3))
    n = len(x0)
    t = _types(type_, n)
    box = _f64(box)
    m = _f64(np.atleast_1d(mass))
    cF = _f64(cF, (-1, 3))
    xb = np.empty((n, 3))
    vb = np.empty((n, 3))
    gb = np.empty(2 * lj.ntypes ** 2)
    r = _load().orc_traj_vjp(n, _p(x0, _d), _p(v0, _d), _p(t, _i32), _p(box, _d), *lj._args(),
                             _p(m, _d), float(skin), float(dt), int(nsteps), int(rebuild_every),
                             _p(cF, _d), _p(xb, _d), _p(vb, _d), _p(gb, _d))
    if r != 0:
        raise MemoryError("oracle traj_vjp: allocation failed")
    return xb, vb, gb.reshape(2, lj.ntypes, lj.ntypes)


def sd_relax(x, box, lj: LJ, nsteps, alpha=0.01, type_=None):
    """Steepest descent x <- x + alpha F / max|F| (list rebuilt every step)."""
    lj._lj_only("sd_relax")
    x = _f64(x, (-1, 3)).copy()
    box = _f64(box)
    t = _types(type_, len(x))
    r = _load().orc_sd_relax(len(x), _p(x, _d), _p(t, _i32), _p(box, _d), *lj._args(),
                             int(nsteps), float(alpha))
    if r != 0:
        raise MemoryError("oracle sd_relax: allocation failed")
    return x
