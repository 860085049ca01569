"""Mixed precision decides the cutoff as FP64 does (needs a GPU).

lj/cut has a jump of |F(rc)| ~ 0.039 (and of E(rc)) at the cutoff (Eq. 1
truncated at rc).  A pair whose r^2 lies within FP32 rounding of rc^2 can
fall on different sides of it in FP32 and FP64.  Such a pair would add a
force error of the size of F(rc), orders of magnitude above the FP32
arithmetic error.  The mixed kernels take the decision from an FP64 r^2
inside a narrow band around each cutoff.

The workload is a lattice of isolated pairs, each at a separation within
2e-7 or 1e-5 (relative) of a cutoff, in a 160-wide box so that FP32 coordinates
carry only ~2^-16 absolute precision.  One layer of pairs straddles each
periodic boundary.  Every pair the oracle keeps must be kept, with its force
to FP32 accuracy.  Every pair it drops must give exactly zero force.
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

from cutoff_lattice import RC, RC_COUL, fp32_flips, pair_lattice, pair_r2  # noqa: E402


def check(f, fref, x, box, cuts):
    """Dropped pairs give exactly zero force, kept pairs their force to FP32
    accuracy.  The band's FP64 r^2 is accurate to ~3e-12 (relative): pairs
    within 1e-10 of a cutoff may go either way and are left out."""
    r2 = pair_r2(x, box)
    near = np.zeros(len(r2), bool)
    for rc in cuts:
        near |= np.abs(r2 / (rc * rc) - 1.0) < 1e-10
    keep = np.repeat(~near, 2)
    f, fref = f[keep], fref[keep]
    zero = ~fref.any(axis=1)
    assert 0 < zero.sum() < len(f)
    assert not f[zero].any(), "a pair beyond the cutoff contributed"
    err = np.linalg.norm(f[~zero] - fref[~zero], axis=1) / np.linalg.norm(fref[~zero], axis=1)
    assert err.max() < 1e-5, err.max()
    return int(near.sum())


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("tpa", [1, 2, 4])
def test_lj_cutoff_decided_in_fp64(kind, tpa):
    x, box = pair_lattice(101, [RC])
    assert fp32_flips(x, box, RC) >= 3  # the workload has teeth
    n = len(x)
    lj = O.LJ(1.0, 1.0, RC)
    fref, E, _ = O.forces(x, box, lj, skin=0.3)
    with md.LJMD(x, np.zeros((n, 3)), None, box, 1.0, 1.0, RC, 1.0, list_kind=kind,
                 precision=md.MD_PREC_MIXED, threads_per_atom=tpa) as ctx:
        _, _, f = (a.cpu().numpy() for a in ctx.get_state())
        th = ctx.energy()
        npairs = ctx.stats()["pairs_in_range"]
    near = check(f, fref, x, box, [RC])
    assert abs(npairs - int(fref.any(axis=1).sum()) // 2) <= near
    assert abs(th.pe - E) <= 1e-6 * abs(E)


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("tpa", [1, 4])
def test_coulomb_cutoffs_decided_in_fp64(kind, tpa):
    """Two cutoffs (rc_coul = 2.2 < rc = 2.5): pairs near each; the Coulomb
    term's jump qq / rc_coul is the larger one."""
    x, box = pair_lattice(103, [RC, RC_COUL])
    assert fp32_flips(x, box, RC_COUL) >= 3
    n = len(x)
    t = (np.arange(n) % 2).astype(np.int32)  # the two atoms of a pair: +q, -q
    q = [0.5, -0.5]
    lj = O.LJ(1.0, 1.0, RC, ntypes=2, q=q, rc_coul=RC_COUL)
    fref, E, _ = O.forces(x, box, lj, type_=t, skin=0.3)
    with md.LJMD(x, np.zeros((n, 3)), t, box, 1.0, 1.0, RC, [1.0, 1.0], list_kind=kind,
                 precision=md.MD_PREC_MIXED, threads_per_atom=tpa) as ctx:
        ctx.set_coulomb(q, RC_COUL)
        ctx.compute_forces(0)
        _, _, f = (a.cpu().numpy() for a in ctx.get_state())
        th = ctx.energy()
    check(f, fref, x, box, [RC, RC_COUL])
    assert abs(th.pe - E) <= 1e-6 * abs(E)


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
def test_force_vjp_same_pairs(kind):
    """The mixed force VJP (the adjoint's backward pass) takes the same
    cutoff decisions: dropped pairs give exactly zero, kept ones the FP64
    VJP to FP32 accuracy."""
    x, box = pair_lattice(107, [RC])
    n = len(x)
    lj = O.LJ(1.0, 1.0, RC)
    w = S.uniform(108, 3 * n).reshape(n, 3) - 0.5
    xref, _ = O.force_vjp(x, box, lj, w, skin=0.3)
    with md.LJMD(x, np.zeros((n, 3)), None, box, 1.0, 1.0, RC, 1.0, list_kind=kind,
                 precision=md.MD_PREC_MIXED, threads_per_atom=1) as ctx:
        xbar, _ = ctx.force_vjp(w)
    check(xbar.cpu().numpy(), xref, x, box, [RC])
