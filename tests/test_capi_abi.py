"""The C ABI library loads and exports every entry point include/md.h
declares; argument checks that return before any CUDA call (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2508_13523_gb300 as md

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(md_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    return md.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    assert declared == set(md.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_strerror(lib):
    assert md.strerror(0) == "success"
    assert "invalid" in md.strerror(md.MD_EINVAL)
    assert md.strerror(-99) == "unknown error"


def _params(**over):
    eps = np.ones(1)
    sig = np.ones(1)
    rc = np.full(1, 2.5)
    mass = np.ones(1)
    dp = ctypes.POINTER(ctypes.c_double)
    p = md.md_params()
    p.n_atoms = 100
    p.n_types = 1
    p.list_kind = md.MD_LIST_FULL
    p.box[:] = [10.0, 10.0, 10.0]
    p.eps, p.sigma, p.rc, p.mass = (a.ctypes.data_as(dp) for a in (eps, sig, rc, mass))
    p.skin = 0.3
    p.dt = 0.005
    p.precision = md.MD_PREC_FP64
    p.rebuild_every = 20
    p.threads_per_atom = 1
    p.max_neigh = 0
    for k, v in over.items():
        if k == "box":
            p.box[:] = v
        else:
            setattr(p, k, v)
    return p, (eps, sig, rc, mass)


@pytest.mark.parametrize("bad", [
    dict(n_atoms=0), dict(n_types=0), dict(n_types=9), dict(list_kind=2), dict(precision=7),
    dict(rebuild_every=0), dict(dt=0.0), dict(skin=-1.0), dict(threads_per_atom=3),
    dict(max_neigh=-1), dict(box=[4.9, 10.0, 10.0]),  # rc must be < L/2
])
def test_invalid_params_rejected_before_cuda(lib, bad):
    p, keep = _params(**bad)
    ctx = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)  # never dereferenced: validation comes first
    rc = lib.md_create(ctypes.byref(p), dummy, dummy, dummy, None, ctypes.byref(ctx))
    assert rc == md.MD_EINVAL
    assert not ctx.value


def test_null_arguments(lib):
    p, keep = _params()
    ctx = ctypes.c_void_p()
    assert lib.md_create(ctypes.byref(p), None, None, None, None, ctypes.byref(ctx)) == md.MD_EINVAL
    assert lib.md_create(None, None, None, None, None, ctypes.byref(ctx)) == md.MD_EINVAL
    for fn in ("md_build_neighbors", "md_autotune", "md_synchronize"):
        assert getattr(lib, fn)(None) == md.MD_EINVAL
    assert lib.md_step(None, 1) == md.MD_EINVAL
    assert lib.md_time_pair_kernel(None, 1) == md.MD_EINVAL
    ms, k = ctypes.c_double(), ctypes.c_int64()
    assert lib.md_pair_kernel_time(None, ctypes.byref(ms), ctypes.byref(k)) == md.MD_EINVAL
    lib.md_destroy(None)


def test_asymmetric_table_rejected(lib):
    p, keep = _params(n_types=2)
    eps = np.array([1.0, 1.5, 1.4, 0.5])  # eps_AB != eps_BA
    sig = np.ones(4)
    rc = np.full(4, 2.5)
    mass = np.ones(2)
    dp = ctypes.POINTER(ctypes.c_double)
    p.eps, p.sigma, p.rc, p.mass = (a.ctypes.data_as(dp) for a in (eps, sig, rc, mass))
    ctx = ctypes.c_void_p()
    d = ctypes.c_void_p(16)
    assert lib.md_create(ctypes.byref(p), d, d, d, None, ctypes.byref(ctx)) == md.MD_EINVAL
