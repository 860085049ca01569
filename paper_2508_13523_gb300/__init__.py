"""GB300-native Lennard-Jones lj/cut short-range step (arXiv 2508.13523).

Python binding of ``libmd.so`` (C ABI in ``include/md.h``).  This module only
marshals arguments: every step of the computation -- cell binning, the
neighbor-list build, the pair force kernel, integration and reductions --
runs in the CUDA kernels of ``libmd.so``.  There is no CPU fallback: if the
library or a CUDA device is missing, the calls raise.

PyTorch is used for device memory and streams only: tensors are passed to
the C ABI by ``data_ptr()`` together with ``torch.cuda.current_stream()``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmd.so")
_lib = None

MD_OK, MD_EINVAL, MD_ENOMEM, MD_ENEIGH, MD_ECUDA, MD_ENONFINITE, MD_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
MD_LIST_FULL, MD_LIST_HALF = 0, 1
MD_PREC_FP64, MD_PREC_MIXED = 0, 1
MD_ENERGY, MD_VIRIAL = 1, 2
MD_MEM_DEVICE, MD_MEM_HOST, MD_MEM_KEEP_LIST = 0, 1, 2
MD_MAX_TYPES = 8
MD_THERMO_N = 10

# every entry point declared in include/md.h
EXPORTS = (
    "md_create", "md_destroy", "md_set_state", "md_get_state", "md_build_neighbors",
    "md_compute_forces", "md_step", "md_energy", "md_neighbor_count", "md_get_neighbors",
    "md_autotune", "md_get_stats", "md_synchronize", "md_strerror", "md_kinetic_noalloc",
    "md_create_batch", "md_energy_replicas", "md_set_lj", "md_force_vjp", "md_traj_forward",
    "md_traj_vjp", "md_minimize", "md_set_kernel", "md_set_coulomb", "md_eval_recip",
    "md_eval_barrier", "md_time_pair_kernel", "md_pair_kernel_time",
)
MD_NOALLOC_MAX_ATOMS = 4194304


class MDError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class md_params(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int64),
        ("n_types", ctypes.c_int32),
        ("list_kind", ctypes.c_int32),
        ("box", ctypes.c_double * 3),
        ("eps", ctypes.POINTER(ctypes.c_double)),
        ("sigma", ctypes.POINTER(ctypes.c_double)),
        ("rc", ctypes.POINTER(ctypes.c_double)),
        ("mass", ctypes.POINTER(ctypes.c_double)),
        ("skin", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("rebuild_every", ctypes.c_int32),
        ("threads_per_atom", ctypes.c_int32),
        ("max_neigh", ctypes.c_int32),
        ("check_disp", ctypes.c_int32),
    ]


class md_stats(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64),
        ("builds", ctypes.c_int64),
        ("dangerous_builds", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("list_entries", ctypes.c_int64),
        ("max_neigh", ctypes.c_int32),
        ("max_count", ctypes.c_int32),
        ("cells", ctypes.c_int32 * 3),
        ("threads_per_atom", ctypes.c_int32),
        ("carveout", ctypes.c_int32),
        ("compacted", ctypes.c_int32),
        ("persistent", ctypes.c_int32),
        ("max_disp", ctypes.c_double),
        ("pairs_in_range", ctypes.c_int64),
        ("n_replicas", ctypes.c_int32),
        ("total_cells", ctypes.c_int64),
        ("coulomb", ctypes.c_int32),
        ("phase1_entries", ctypes.c_int32),
    ]


def library_path() -> str:
    return _LIB_PATH


def load(build_if_missing: bool = True):
    """Load libmd.so (building it with nvcc first if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        if not build_if_missing:
            raise OSError(f"{_LIB_PATH} is missing: run paper_2508_13523_gb300/build.py")
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    I64, I32 = ctypes.c_int64, ctypes.c_int32
    sig = {
        "md_create": ([ctypes.POINTER(md_params), P, P, P, P, ctypes.POINTER(P)], I32),
        "md_destroy": ([P], None),
        "md_set_state": ([P, P, P, I32], I32),
        "md_get_state": ([P, P, P, P, I32], I32),
        "md_build_neighbors": ([P], I32),
        "md_compute_forces": ([P, I32], I32),
        "md_step": ([P, I64], I32),
        "md_energy": ([P, ctypes.POINTER(ctypes.c_double)], I32),
        "md_neighbor_count": ([P, ctypes.POINTER(I64), ctypes.POINTER(I32)], I32),
        "md_get_neighbors": ([P, P, P], I32),
        "md_autotune": ([P], I32),
        "md_get_stats": ([P, ctypes.POINTER(md_stats)], I32),
        "md_synchronize": ([P], I32),
        "md_strerror": ([I32], ctypes.c_char_p),
        "md_kinetic_noalloc": ([I64, P, P, I32, ctypes.POINTER(ctypes.c_double), P, P], I32),
        "md_create_batch": ([ctypes.POINTER(md_params), I32, ctypes.POINTER(I64),
                             ctypes.POINTER(ctypes.c_double), P, P, P, P, ctypes.POINTER(P)], I32),
        "md_energy_replicas": ([P, ctypes.POINTER(ctypes.c_double)], I32),
        "md_set_lj": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], I32),
        "md_force_vjp": ([P, P, P, ctypes.POINTER(ctypes.c_double)], I32),
        "md_traj_forward": ([P, I64, I32, P, P, P, P, P], I32),
        "md_traj_vjp": ([P, I64, I32, P, P, P, P, P, ctypes.POINTER(ctypes.c_double)], I32),
        "md_minimize": ([P, I64, ctypes.c_double], I32),
        "md_set_kernel": ([P, I32, I32, I32, I32], I32),
        "md_set_coulomb": ([P, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                            ctypes.c_double], I32),
        "md_eval_recip": ([I64, P, P, P, P], I32),
        "md_eval_barrier": ([I32, I32, ctypes.c_double, P, P], I32),
        "md_time_pair_kernel": ([P, I32], I32),
        "md_pair_kernel_time": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)], I32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().md_strerror(int(code)).decode()


def _check(code: int, where: str):
    if code != MD_OK:
        raise MDError(code, where)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required: libmd.so has no CPU path")
    return torch


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _host(a):
    """A host numpy copy of a tensor or array-like (argument marshalling)."""
    if hasattr(a, "detach"):
        return a.detach().cpu().numpy()
    return np.asarray(a)


def _table(v, nt):
    a = np.asarray(v, dtype=np.float64)
    if a.ndim == 0:
        a = np.full((nt, nt), float(a))
    return np.ascontiguousarray(a.reshape(nt * nt))


@dataclass
class Thermo:
    pe: float
    ke: float
    etot: float
    temperature: float
    virial: np.ndarray  # xx, yy, zz, xy, xz, yz


class LJMD:
    """One periodic box behind an ``md_ctx`` (C ABI ``md_create`` ...).

    ``x``, ``v``: (n, 3) float64 and ``type_``: (n,) int32, either torch CUDA
    tensors or numpy arrays (copied to the device first).  Parameters follow
    ``md_params``: eps/sigma/rc per type pair, mass per type."""

    def __init__(self, x, v, type_, box, eps, sigma, rc, mass, *, skin=0.3, dt=0.005,
                 list_kind=MD_LIST_FULL, precision=MD_PREC_FP64, rebuild_every=20,
                 threads_per_atom=0, max_neigh=0, stream=None, rep_offset=None,
                 check_disp=False):
        torch = _torch()
        lib = load()
        dev = torch.device("cuda", torch.cuda.current_device())
        self._x = torch.as_tensor(x, dtype=torch.float64, device=dev).contiguous()
        self._v = torch.as_tensor(v, dtype=torch.float64, device=dev).contiguous()
        self.n = int(self._x.shape[0])
        if type_ is None:
            type_ = np.zeros(self.n, dtype=np.int32)
        self._t = torch.as_tensor(type_, dtype=torch.int32, device=dev).contiguous()
        mass = np.atleast_1d(np.asarray(mass, dtype=np.float64))
        nt = len(mass)
        self.ntypes = nt
        self._eps, self._sigma, self._rc = (_table(a, nt) for a in (eps, sigma, rc))
        self._mass = np.ascontiguousarray(mass)
        dp = ctypes.POINTER(ctypes.c_double)
        p = md_params()
        p.n_atoms = self.n
        p.n_types = nt
        p.list_kind = list_kind
        boxes = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(-1, 3))
        if rep_offset is None and len(boxes) != 1:
            raise ValueError("several boxes need rep_offset")
        p.box[:] = [float(b) for b in boxes[0]]
        p.eps = self._eps.ctypes.data_as(dp)
        p.sigma = self._sigma.ctypes.data_as(dp)
        p.rc = self._rc.ctypes.data_as(dp)
        p.mass = self._mass.ctypes.data_as(dp)
        p.skin = skin
        p.dt = dt
        p.precision = precision
        p.rebuild_every = rebuild_every
        p.threads_per_atom = threads_per_atom
        p.max_neigh = max_neigh
        p.check_disp = int(bool(check_disp))
        self.params = p
        # a dedicated stream (graph capture needs a non-default stream), ordered
        # after the work that produced the inputs
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        self._ctx = ctypes.c_void_p()
        if rep_offset is None:
            self.n_replicas = 1
            _check(lib.md_create(ctypes.byref(p), _ptr(self._x), _ptr(self._v), _ptr(self._t),
                                 ctypes.c_void_p(self.stream.cuda_stream),
                                 ctypes.byref(self._ctx)), "md_create")
        else:
            off = np.ascontiguousarray(rep_offset, dtype=np.int64)
            self.n_replicas = len(off) - 1
            self._off, self._boxes = off, boxes
            _check(lib.md_create_batch(ctypes.byref(p), self.n_replicas,
                                       off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       boxes.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       _ptr(self._x), _ptr(self._v), _ptr(self._t),
                                       ctypes.c_void_p(self.stream.cuda_stream),
                                       ctypes.byref(self._ctx)), "md_create_batch")
        self._lib = lib

    # -- lifetime --------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._lib.md_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls -------------------------------------------------------------------
    def step(self, nsteps: int = 1):
        _check(self._lib.md_step(self._ctx, int(nsteps)), "md_step")

    def build_neighbors(self):
        _check(self._lib.md_build_neighbors(self._ctx), "md_build_neighbors")

    def compute_forces(self, flags: int = 0):
        _check(self._lib.md_compute_forces(self._ctx, int(flags)), "md_compute_forces")

    def energy(self) -> Thermo:
        out = (ctypes.c_double * MD_THERMO_N)()
        _check(self._lib.md_energy(self._ctx, out), "md_energy")
        a = np.frombuffer(out, dtype=np.float64).copy()
        return Thermo(a[0], a[1], a[2], a[3], a[4:10])

    def energy_replicas(self) -> np.ndarray:
        """(n_replicas, 10): pe, ke, etot, T, W_xx, W_yy, W_zz, W_xy, W_xz, W_yz."""
        out = np.empty((self.n_replicas, MD_THERMO_N))
        _check(self._lib.md_energy_replicas(
            self._ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "md_energy_replicas")
        return out

    # -- coefficients, gradients, relaxation ----------------------------------------
    def set_lj(self, eps, sigma):
        """md_set_lj: new per-type-pair eps and sigma (rc unchanged)."""
        e = _table(_host(eps), self.ntypes)
        s_ = _table(_host(sigma), self.ntypes)
        dp = ctypes.POINTER(ctypes.c_double)
        _check(self._lib.md_set_lj(self._ctx, e.ctypes.data_as(dp), s_.ctypes.data_as(dp)),
               "md_set_lj")

    def set_coulomb(self, q=None, rc_coul=None, qqrd2e=1.0):
        """md_set_coulomb: the lj/cut/coul/cut style with per-type charges q
        (length n_types; None turns the Coulomb term off), cutoff rc_coul
        (default: the largest rc) and prefactor qqrd2e."""
        dp = ctypes.POINTER(ctypes.c_double)
        if q is None:
            _check(self._lib.md_set_coulomb(self._ctx, None, 0.0, 0.0), "md_set_coulomb")
            return
        qt = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(self.ntypes))
        rcc = float(np.max(self._rc)) if rc_coul is None else float(rc_coul)
        _check(self._lib.md_set_coulomb(self._ctx, qt.ctypes.data_as(dp), rcc, float(qqrd2e)),
               "md_set_coulomb")

    def force_vjp(self, cot):
        """md_force_vjp: (dL/dx as a CUDA tensor (n,3), dL/d(eps, sigma) as a
        numpy array (2, nt, nt), both entries of a pair holding its derivative)."""
        torch = _torch()
        cot = torch.as_tensor(cot, dtype=torch.float64, device=self._x.device).contiguous()
        xbar = torch.empty((self.n, 3), dtype=torch.float64, device=self._x.device)
        g = np.empty(2 * self.ntypes ** 2)
        self.stream.wait_stream(torch.cuda.current_stream())
        _check(self._lib.md_force_vjp(self._ctx, _ptr(cot), _ptr(xbar),
                                      g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "md_force_vjp")
        return xbar, g.reshape(2, self.ntypes, self.ntypes)

    def traj_forward(self, x0, v0, nsteps, every):
        """md_traj_forward: checkpoints (x, v) and the final forces."""
        torch = _torch()
        dev = self._x.device
        x0 = torch.as_tensor(x0, dtype=torch.float64, device=dev).contiguous()
        v0 = torch.as_tensor(v0, dtype=torch.float64, device=dev).contiguous()
        nck = (int(nsteps) + int(every) - 1) // int(every) + 1
        ckx = torch.empty((nck, self.n, 3), dtype=torch.float64, device=dev)
        ckv = torch.empty((nck, self.n, 3), dtype=torch.float64, device=dev)
        fK = torch.empty((self.n, 3), dtype=torch.float64, device=dev)
        self.stream.wait_stream(torch.cuda.current_stream())
        _check(self._lib.md_traj_forward(self._ctx, int(nsteps), int(every), _ptr(x0), _ptr(v0),
                                         _ptr(ckx), _ptr(ckv), _ptr(fK)), "md_traj_forward")
        self.synchronize()
        return ckx, ckv, fK

    def traj_vjp(self, nsteps, every, ckx, ckv, cot_final):
        """md_traj_vjp: (dL/dx0, dL/dv0, dL/d(eps, sigma))."""
        torch = _torch()
        dev = self._x.device
        cot = torch.as_tensor(cot_final, dtype=torch.float64, device=dev).contiguous()
        x0b = torch.empty((self.n, 3), dtype=torch.float64, device=dev)
        v0b = torch.empty((self.n, 3), dtype=torch.float64, device=dev)
        g = np.empty(2 * self.ntypes ** 2)
        self.stream.wait_stream(torch.cuda.current_stream())
        _check(self._lib.md_traj_vjp(self._ctx, int(nsteps), int(every), _ptr(ckx), _ptr(ckv),
                                     _ptr(cot), _ptr(x0b), _ptr(v0b),
                                     g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "md_traj_vjp")
        self.synchronize()
        return x0b, v0b, g.reshape(2, self.ntypes, self.ntypes)

    def minimize(self, nsteps, alpha=0.01):
        """md_minimize: steepest descent x <- x + alpha F / max|F|."""
        _check(self._lib.md_minimize(self._ctx, int(nsteps), float(alpha)), "md_minimize")

    def set_state(self, x, v, keep_list: bool = False):
        """Replace positions and velocities: torch CUDA tensors (device) or
        numpy arrays (host, staged by the library).  keep_list: keep the
        atom order and neighbor list if no atom moved more than skin/2 since
        the last build (MD_MEM_KEEP_LIST)."""
        flag = MD_MEM_KEEP_LIST if keep_list else 0
        if isinstance(x, np.ndarray):
            xh = np.ascontiguousarray(x, dtype=np.float64)
            vh = np.ascontiguousarray(v, dtype=np.float64)
            _check(self._lib.md_set_state(self._ctx, xh.ctypes.data_as(ctypes.c_void_p),
                                          vh.ctypes.data_as(ctypes.c_void_p),
                                          MD_MEM_HOST | flag), "md_set_state")
            return
        self.stream.wait_stream(_torch().cuda.current_stream())
        _check(self._lib.md_set_state(self._ctx, _ptr(x), _ptr(v), MD_MEM_DEVICE | flag),
               "md_set_state")

    def get_state(self, host: bool = False):
        """(x, v, f) in the caller's atom order: torch CUDA tensors, or numpy
        arrays when host=True (the library copies them out)."""
        if host:
            x = np.empty((self.n, 3))
            v = np.empty((self.n, 3))
            f = np.empty((self.n, 3))
            c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
            _check(self._lib.md_get_state(self._ctx, c(x), c(v), c(f), MD_MEM_HOST),
                   "md_get_state")
            return x, v, f
        torch = _torch()
        x, v, f = (torch.empty((self.n, 3), dtype=torch.float64, device=self._x.device)
                   for _ in range(3))
        _check(self._lib.md_get_state(self._ctx, _ptr(x), _ptr(v), _ptr(f), MD_MEM_DEVICE),
               "md_get_state")
        self.synchronize()
        return x, v, f

    def get_state_into(self, x=None, v=None, f=None, mem=MD_MEM_DEVICE):
        """Copy the state into caller buffers (device tensors or host arrays)."""
        def p(a):
            if a is None:
                return None
            return (a.ctypes.data_as(ctypes.c_void_p) if isinstance(a, np.ndarray)
                    else ctypes.c_void_p(a.data_ptr()))
        _check(self._lib.md_get_state(self._ctx, p(x), p(v), p(f), int(mem)), "md_get_state")

    def set_state_from(self, x, v, mem=MD_MEM_DEVICE):
        def p(a):
            return (a.ctypes.data_as(ctypes.c_void_p) if isinstance(a, np.ndarray)
                    else ctypes.c_void_p(a.data_ptr()))
        _check(self._lib.md_set_state(self._ctx, p(x), p(v), int(mem)), "md_set_state")

    def neighbor_count(self):
        total = ctypes.c_int64()
        mx = ctypes.c_int32()
        _check(self._lib.md_neighbor_count(self._ctx, ctypes.byref(total), ctypes.byref(mx)),
               "md_neighbor_count")
        return total.value, mx.value

    def neighbors(self):
        """CSR (offsets int64[n+1], idx int32[total]) in the caller's numbering,
        as torch CUDA tensors."""
        torch = _torch()
        total, _ = self.neighbor_count()
        off = torch.empty(self.n + 1, dtype=torch.int64, device=self._x.device)
        idx = torch.empty(max(total, 1), dtype=torch.int32, device=self._x.device)
        _check(self._lib.md_get_neighbors(self._ctx, _ptr(off), _ptr(idx)), "md_get_neighbors")
        self.synchronize()
        return off, idx[:total]

    def set_kernel(self, threads_per_atom=1, carveout=-1, compacted=0, persistent=1):
        """md_set_kernel: fix the pair kernel's configuration (compacted: 0
        per-atom loop, 1 warp-compacted with FP64 force sums, 2 warp-compacted
        with exact fixed-point force sums, 3 the same with two list entries per
        lane per filter round)."""
        _check(self._lib.md_set_kernel(self._ctx, int(threads_per_atom), int(carveout),
                                       int(compacted), int(persistent)), "md_set_kernel")

    def autotune(self):
        _check(self._lib.md_autotune(self._ctx), "md_autotune")

    def time_pair_kernel(self, enable: bool = True):
        """md_time_pair_kernel: while enabled, md_step runs its segments
        without graphs and records CUDA events around every pair launch."""
        _check(self._lib.md_time_pair_kernel(self._ctx, 1 if enable else 0),
               "md_time_pair_kernel")

    def pair_kernel_time(self):
        """md_pair_kernel_time: (summed milliseconds, launches) of the pair
        launches recorded since time_pair_kernel(True)."""
        ms = ctypes.c_double(0.0)
        k = ctypes.c_int64(0)
        _check(self._lib.md_pair_kernel_time(self._ctx, ctypes.byref(ms), ctypes.byref(k)),
               "md_pair_kernel_time")
        return ms.value, k.value

    def stats(self) -> dict:
        s = md_stats()
        _check(self._lib.md_get_stats(self._ctx, ctypes.byref(s)), "md_get_stats")
        return dict(step=s.step, builds=s.builds, dangerous_builds=s.dangerous_builds,
                    kernel_launches=s.kernel_launches, list_entries=s.list_entries,
                    max_neigh=s.max_neigh, max_count=s.max_count, cells=tuple(s.cells),
                    threads_per_atom=s.threads_per_atom, carveout=s.carveout, compacted=s.compacted, persistent=s.persistent,
                    max_disp=s.max_disp,
                    pairs_in_range=s.pairs_in_range, n_replicas=s.n_replicas,
                    total_cells=s.total_cells, coulomb=s.coulomb,
                    phase1_entries=s.phase1_entries)

    def synchronize(self):
        _check(self._lib.md_synchronize(self._ctx), "md_synchronize")


def kinetic_noalloc(v, type_, mass, out, stream=None):
    """md_kinetic_noalloc: kinetic energy and temperature of device velocities
    v (n, 3) into the device tensor out (2 doubles), without any allocation
    inside the library.  type_ may be None; mass is a host sequence per type."""
    torch = _torch()
    lib = load()
    m = np.ascontiguousarray(np.atleast_1d(np.asarray(mass, dtype=np.float64)))
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib.md_kinetic_noalloc(int(v.shape[0]), _ptr(v),
                                  None if type_ is None else _ptr(type_), len(m),
                                  m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(out),
                                  ctypes.c_void_p(s.cuda_stream)),
           "md_kinetic_noalloc")


def eval_recip(a, rcp=None, rsqrt=None, stream=None):
    """md_eval_recip: the pair kernels' device 1/a and 1/sqrt(a), elementwise,
    for a contiguous float64 device tensor a, into the device tensors rcp and
    rsqrt of the same size (either may be None)."""
    torch = _torch()
    lib = load()
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib.md_eval_recip(int(a.numel()), _ptr(a), None if rcp is None else _ptr(rcp),
                             None if rsqrt is None else _ptr(rsqrt),
                             ctypes.c_void_p(s.cuda_stream)), "md_eval_recip")


def eval_barrier(blocks, missing, limit_ms, word, stream=None) -> int:
    """md_eval_barrier: the fused step's grid barrier alone (word: a device
    tensor of at least 3 int32).  Returns the library's code (MD_OK or
    MD_ETIMEOUT) instead of raising for MD_ETIMEOUT."""
    torch = _torch()
    lib = load()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.md_eval_barrier(int(blocks), int(missing), float(limit_ms), _ptr(word),
                             ctypes.c_void_p(s.cuda_stream))
    if rc not in (MD_OK, MD_ETIMEOUT):
        _check(rc, "md_eval_barrier")
    return rc


def from_systems(systems, **kw) -> LJMD:
    """One batch context for a list of ``synth.System`` boxes that share their
    parameters (md_create_batch)."""
    p = systems[0].params
    kw.setdefault("skin", p.skin)
    kw.setdefault("dt", p.dt)
    kw.setdefault("rebuild_every", p.rebuild_every)
    x = np.concatenate([s.x for s in systems])
    v = np.concatenate([s.v for s in systems])
    t = np.concatenate([s.type for s in systems]).astype(np.int32)
    off = np.concatenate([[0], np.cumsum([s.n for s in systems])]).astype(np.int64)
    boxes = np.stack([s.box for s in systems])
    return LJMD(x, v, t, boxes, p.eps, p.sigma, p.rc, p.mass, rep_offset=off, **kw)


def from_system(sysm, **kw) -> LJMD:
    """An LJMD context for a ``synth.System``."""
    p = sysm.params
    kw.setdefault("skin", p.skin)
    kw.setdefault("dt", p.dt)
    kw.setdefault("rebuild_every", p.rebuild_every)
    return LJMD(sysm.x, sysm.v, sysm.type, sysm.box, p.eps, p.sigma, p.rc, p.mass, **kw)
