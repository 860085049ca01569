"""Adjoint kernels vs the oracle's reverse mode (needs a GPU).

The oracle's reverse mode is pinned by finite differences in
test_oracle_adjoint_pins.py; here the CUDA VJP and the checkpointed reverse
sweep through velocity Verlet must reproduce it: FP64 within 1e-11 of the
rms (force VJP, one evaluation) and 1e-9 (20 steps, where the two forward
trajectories already differ by rounding), mixed precision reported.
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
from paper_2508_13523_gb300.autograd import lj_forces, lj_trajectory_forces  # noqa: E402

MASS = np.array([1.0, 1.0])


def rel(a, b):
    scale = np.sqrt(np.mean(np.sum(b * b, axis=-1))) if b.ndim > 1 else np.abs(b).max()
    return float(np.abs(a - b).max() / scale)


@pytest.fixture(scope="module")
def mixture():
    """864-atom two-type system (jittered fcc at density 1.2, 20 % B,
    L = 8.96 > 2 rc_max), relaxed 30 steepest-descent steps by the oracle."""
    x, box, _ = S.fcc(6, 1.2)
    x = x + 0.2 * (S.uniform(81, x.size).reshape(x.shape) - 0.5)
    t = (S.uniform(82, len(x)) >= 0.8).astype(np.int32)
    p = S.binary_mixture_params(rebuild_every=10)
    lj = O.LJ(p.eps, p.sigma, p.rc, ntypes=2)
    x = O.sd_relax(x, box, lj, 30, 0.01, type_=t)
    v = S.maxwell_boltzmann(p.mass[t], 1.0, 83)
    return S.System(x, v, t, box, p)


def olj(eps, sig, p):
    return O.LJ(eps, sig, p.rc, ntypes=2)


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("tpa", [1, 4])
def test_force_vjp_fp64(mixture, kind, tpa):
    s = mixture
    cot = S.normal(91, 3 * s.n).reshape(s.n, 3)
    with md.from_system(s, list_kind=kind, threads_per_atom=tpa) as ctx:
        x = ctx.get_state()[0].cpu().numpy()
        xbar, g = ctx.force_vjp(cot)
    xref, gref = O.force_vjp(x, s.box, olj(s.params.eps, s.params.sigma, s.params), cot,
                             type_=s.type, skin=0.3)
    assert rel(xbar.cpu().numpy(), xref) <= 1e-11
    np.testing.assert_allclose(g, gref, rtol=1e-11, atol=1e-11 * np.abs(gref).max())
    assert g[0, 0, 1] == g[0, 1, 0]


def test_force_vjp_mixed_error_reported(mixture, capsys):
    s = mixture
    cot = S.normal(92, 3 * s.n).reshape(s.n, 3)
    with md.from_system(s, precision=md.MD_PREC_MIXED, threads_per_atom=1) as ctx:
        x = ctx.get_state()[0].cpu().numpy()
        xbar, g = ctx.force_vjp(cot)
    xref, gref = O.force_vjp(x, s.box, olj(s.params.eps, s.params.sigma, s.params), cot,
                             type_=s.type, skin=0.3)
    ex, eg = rel(xbar.cpu().numpy(), xref), float(np.abs(g - gref).max() / np.abs(gref).max())
    print(f"mixed force VJP: dL/dx err {ex:.3e}, dL/dtheta err {eg:.3e}")
    assert ex < 1e-3 and eg < 1e-3


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("nsteps", [0, 7, 20, 25])
def test_traj_vjp_fp64(mixture, kind, nsteps):
    """Checkpoints every 10 steps (= the list cadence); nsteps 7 and 25 end
    inside a segment."""
    s = mixture
    cot = S.normal(93, 3 * s.n).reshape(s.n, 3)
    with md.from_system(s, list_kind=kind, threads_per_atom=2) as ctx:
        x0, v0, _ = (a.cpu().numpy() for a in ctx.get_state())
        ckx, ckv, fK = ctx.traj_forward(x0, v0, nsteps, 10)
        x0b, v0b, g = ctx.traj_vjp(nsteps, 10, ckx, ckv, cot)
    _, _, fo, _ = O.run(x0, v0, s.box, olj(s.params.eps, s.params.sigma, s.params), MASS,
                        type_=s.type, nsteps=nsteps, rebuild_every=10)
    ef = rel(fK.cpu().numpy(), fo)
    xr, vr, gr = O.traj_vjp(x0, v0, s.box, olj(s.params.eps, s.params.sigma, s.params), MASS, cot,
                            type_=s.type, nsteps=nsteps, rebuild_every=10)
    ex = rel(x0b.cpu().numpy(), xr)
    ev = rel(v0b.cpu().numpy(), vr) if nsteps > 0 else 0.0
    eg = float(np.abs(g - gr).max() / np.abs(gr).max())
    # the bound is 1e-9, looser than one VJP's 1e-11: the reverse sweep
    # differentiates along the GPU's own forward trajectory, which departs
    # from the oracle's by rounding (forces summed in another order) and
    # grows with the steps; the printed errors show how much of it is used
    print(f"FP64 trajectory VJP ({nsteps} steps, list {kind}): F_K {ef:.2e}, "
          f"dL/dx0 {ex:.2e}, dL/dv0 {ev:.2e}, dL/dtheta {eg:.2e}")
    assert ef <= 1e-10
    assert ex <= 1e-9
    assert ev <= 1e-9
    np.testing.assert_allclose(g, gr, rtol=1e-9, atol=1e-9 * np.abs(gr).max())


def test_traj_vjp_mixed_error_reported(mixture, capsys):
    s = mixture
    cot = S.normal(94, 3 * s.n).reshape(s.n, 3)
    with md.from_system(s, precision=md.MD_PREC_MIXED, threads_per_atom=1) as ctx:
        x0, v0, _ = (a.cpu().numpy() for a in ctx.get_state())
        ckx, ckv, _ = ctx.traj_forward(x0, v0, 20, 10)
        x0b, v0b, g = ctx.traj_vjp(20, 10, ckx, ckv, cot)
    xr, vr, gr = O.traj_vjp(x0, v0, s.box, olj(s.params.eps, s.params.sigma, s.params), MASS, cot,
                            type_=s.type, nsteps=20, rebuild_every=10)
    ex, eg = rel(x0b.cpu().numpy(), xr), float(np.abs(g - gr).max() / np.abs(gr).max())
    print(f"mixed trajectory VJP (20 steps): dL/dx0 err {ex:.3e}, dL/dtheta err {eg:.3e}")
    assert ex < 1e-2 and eg < 1e-2


def test_autograd_functions(mixture):
    """torch.autograd through lj_trajectory_forces equals the C ABI's reverse
    mode, with half of an off-diagonal pair's derivative in each entry."""
    s = mixture
    dev = torch.device("cuda")
    with md.from_system(s, threads_per_atom=1) as ctx:
        x0, v0, _ = ctx.get_state()
        eps = torch.tensor(s.params.eps, device=dev, requires_grad=True)
        sig = torch.tensor(s.params.sigma, device=dev, requires_grad=True)
        x0 = x0.clone().requires_grad_(True)
        v0 = v0.clone().requires_grad_(True)
        fref = torch.as_tensor(S.normal(95, 3 * s.n).reshape(s.n, 3), device=dev)
        fK = lj_trajectory_forces(x0, v0, eps, sig, ctx, 12, 10)
        loss = ((fK - fref) ** 2).sum()
        gx0, gv0, ge, gs = torch.autograd.grad(loss, (x0, v0, eps, sig))
        ckx, ckv, fK2 = ctx.traj_forward(x0.detach(), v0.detach(), 12, 10)
        x0b, v0b, g = ctx.traj_vjp(12, 10, ckx, ckv, 2 * (fK2 - fref))
        assert torch.equal(fK, fK2)
        assert torch.allclose(gx0, x0b, rtol=1e-12, atol=0)
        assert torch.allclose(gv0, v0b, rtol=1e-12, atol=0)
        ge, gs = ge.cpu().numpy(), gs.cpu().numpy()
        assert abs(ge[0, 1] + ge[1, 0] - g[0, 0, 1]) <= 1e-12 * abs(g[0, 0, 1])
        assert abs(gs[1, 1] - g[1, 1, 1]) <= 1e-12 * abs(g[1, 1, 1])
        # one force evaluation
        x = x0.detach().clone().requires_grad_(True)
        f = lj_forces(x, eps, sig, ctx)
        (gx,) = torch.autograd.grad((f * fref).sum(), (x,))
        xb1, _ = ctx.force_vjp(fref)
        assert torch.allclose(gx, xb1, rtol=1e-12, atol=0)


def test_minimize_matches_oracle(mixture):
    """Steepest descent on the GPU (list every 10 steps, 0.1 < skin/2 of
    motion between builds) against the oracle's (list every step)."""
    s = mixture
    x, box, t = s.x, s.box, s.type
    x = x + 0.1 * (S.uniform(96, x.size).reshape(x.shape) - 0.5)
    with md.LJMD(x, np.zeros_like(x), t, box, s.params.eps, s.params.sigma, s.params.rc,
                 s.params.mass, rebuild_every=10, threads_per_atom=1) as ctx:
        x0 = ctx.get_state()[0].cpu().numpy()
        ctx.minimize(20, 0.01)
        x1 = ctx.get_state()[0].cpu().numpy()
    xo = O.sd_relax(x0, box, olj(s.params.eps, s.params.sigma, s.params), 20, 0.01, type_=t)
    d = x1 - xo
    d -= box * np.round(d / box)
    assert np.abs(d).max() < 1e-10
