"""The FP64 pair kernels decide the cutoff exactly as the oracle does (needs
a GPU).

lj/cut jumps by |F(rc)| ~ 0.039 at rc (Eq. 1 truncated).  The oracle keeps
a pair iff fma(dz,dz, fma(dy,dy, dx*dx)) < rc^2.  The compacted kernel's
integer path forms r^2 exactly from fixed-point positions and takes the
decision from it except within 4 ulps of rc^2, where it computes that FP64
expression instead.  The workload (tests/cutoff_ulps.py) puts isolated
pairs within 3 ulps of rc^2, many of them where the exact and the rounded
r^2 lie on different sides: a kernel that decided them on the exact r^2
would miss or add the whole |F(rc)| there.  Every kernel (per-atom,
compacted with FP64 or fixed-point sums), both list kinds, must match the
oracle's forces to 1e-12 of the rms force and its pair count exactly.

eps = 100: with eps = 1 the isolated pairs' forces (~0.039) would be so
small that the fixed-point sums' absolute resolution (a contribution is
rounded to a multiple of 2^-44) alone reaches ~2e-12 of their rms; the
decisions under test do not depend on eps.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_2508_13523_gb300 as md  # noqa: E402

from cutoff_ulps import RC, classify, workload  # noqa: E402

EPS = 100.0


@pytest.fixture(scope="module")
def wl():
    x, box = workload(7)
    ex, ro = classify(x)
    assert (ex != ro).sum() >= 600  # the workload has teeth
    fref, E, _ = O.forces(x, box, O.LJ(EPS, 1.0, RC), skin=0.3)
    return x, box, fref, E, int(ro.sum())


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("compacted", [0, 1, 2, 3])
def test_fp64_cutoff_decisions_match_oracle(wl, kind, compacted):
    x, box, fref, E, npairs_ref = wl
    n = len(x)
    with md.LJMD(x, np.zeros((n, 3)), None, box, EPS, 1.0, RC, 1.0, list_kind=kind,
                 threads_per_atom=1) as ctx:
        ctx.set_kernel(1, -1, compacted, 0)
        ctx.compute_forces(0)
        _, _, f = (a.cpu().numpy() for a in ctx.get_state())
        th = ctx.energy()
        npairs = ctx.stats()["pairs_in_range"]
    rms = np.sqrt(np.mean(np.sum(fref * fref, axis=1)))
    err = np.max(np.linalg.norm(f - fref, axis=1)) / rms
    assert err <= 1e-12, err
    assert npairs == npairs_ref
    assert abs(th.pe - E) <= 1e-12 * abs(E)
