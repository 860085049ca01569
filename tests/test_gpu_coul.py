"""Second pair style, lj/cut/coul/cut (md_set_coulomb), vs the FP64 oracle
(needs a GPU).

The oracle's Coulomb term is pinned in test_oracle_coul_pins.py.  Here the
warp-compacted FP64 kernel (FP64 and fixed-point force sums, half and full
lists) must match it within 1e-12 of the rms force, with energies and
virials within 1e-12; the mixed-precision kernel's error is reported with a
sanity bound of 1e-4.
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

Q = [0.6, -0.6]


def rel_err(f, fref):
    rms = np.sqrt(np.mean(np.sum(fref * fref, axis=1)))
    return float(np.max(np.linalg.norm(f - fref, axis=1)) / rms)


@pytest.fixture(scope="module")
def salt():
    """864-atom fcc box (6^3 cells) at density 0.8442, jittered, two types by
    basis site (sites 0, 1: +0.6; 2, 3: -0.6), relaxed 20 oracle steps."""
    x, box, _ = S.fcc(6)
    x = x + 0.2 * (S.uniform(61, x.size).reshape(x.shape) - 0.5)
    t = (np.arange(len(x)) % 4 >= 2).astype(np.int32)
    v = S.maxwell_boltzmann(np.ones(len(x)), 1.0, 62)
    lj = O.LJ(1.0, 1.0, 2.5, ntypes=2, q=Q, rc_coul=2.5)
    x, v, _, _ = O.run(x, v, box, lj, np.ones(2), type_=t, nsteps=20, rebuild_every=1)
    return x, v, t, box


def make(x, v, t, box, **kw):
    return md.LJMD(x, v, t, box, 1.0, 1.0, 2.5, [1.0, 1.0], **kw)


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("compacted", [1, 2])
@pytest.mark.parametrize("rc_coul", [2.5, 2.2])
def test_fp64_forces_energy_virial(salt, kind, compacted, rc_coul):
    x, v, t, box = salt
    with make(x, v, t, box, list_kind=kind, threads_per_atom=1) as ctx:
        ctx.set_coulomb(Q, rc_coul)
        ctx.set_kernel(1, -1, compacted, 0)
        ctx.compute_forces(0)
        assert ctx.stats()["coulomb"] == 1
        xg, _, f = (a.cpu().numpy() for a in ctx.get_state())
        th = ctx.energy()
    lj = O.LJ(1.0, 1.0, 2.5, ntypes=2, q=Q, rc_coul=rc_coul)
    fref, E, W = O.forces(xg, box, lj, type_=t, skin=0.3)
    assert rel_err(f, fref) <= 1e-12
    assert abs(th.pe - E) <= 1e-12 * abs(E)
    np.testing.assert_allclose(th.virial, W, rtol=1e-12, atol=1e-12 * np.abs(W).max())


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("tpa", [1, 2, 4])
def test_mixed_error_reported(salt, kind, tpa, capsys):
    x, v, t, box = salt
    with make(x, v, t, box, list_kind=kind, precision=md.MD_PREC_MIXED,
              threads_per_atom=tpa) as ctx:
        ctx.set_coulomb(Q)
        xg, _, f = (a.cpu().numpy() for a in ctx.get_state())
        th = ctx.energy()
    lj = O.LJ(1.0, 1.0, 2.5, ntypes=2, q=Q, rc_coul=2.5)
    fref, E, _ = O.forces(xg, box, lj, type_=t, skin=0.3)
    e = rel_err(f, fref)
    print(f"mixed coul kind={kind} tpa={tpa}: force err {e:.3e}, "
          f"energy rel err {abs(th.pe - E) / abs(E):.3e}")
    assert e < 1e-4 and abs(th.pe - E) < 1e-5 * abs(E)


@pytest.mark.parametrize("compacted", [1, 2])
def test_fp64_trajectory(salt, compacted):
    """25 steps with a rebuild every 5 steps, against the oracle's run."""
    x, v, t, box = salt
    with make(x, v, t, box, list_kind=md.MD_LIST_HALF, rebuild_every=5,
              threads_per_atom=1) as ctx:
        ctx.set_coulomb(Q)
        ctx.set_kernel(1, -1, compacted, 0)
        ctx.compute_forces(0)
        x0, v0, _ = (a.cpu().numpy() for a in ctx.get_state())
        ctx.step(25)
        x1, v1, f1 = (a.cpu().numpy() for a in ctx.get_state())
    lj = O.LJ(1.0, 1.0, 2.5, ntypes=2, q=Q, rc_coul=2.5)
    xo, vo, fo, _ = O.run(x0, v0, box, lj, np.ones(2), type_=t, nsteps=25, rebuild_every=5)
    assert np.abs(x1 - xo).max() < 1e-11
    assert np.abs(v1 - vo).max() < 1e-11
    assert rel_err(f1, fo) < 1e-11


def test_switch_off_and_restrictions(salt):
    """q = None restores Eq. 1 alone; the adjoint and the FP64 per-atom
    kernel refuse the Coulomb style."""
    x, v, t, box = salt
    with make(x, v, t, box, list_kind=md.MD_LIST_HALF, threads_per_atom=1) as ctx:
        ctx.set_coulomb(Q)
        with pytest.raises(md.MDError):
            ctx.set_kernel(1, -1, 0, 0)
        with pytest.raises(md.MDError):
            ctx.force_vjp(np.zeros((len(x), 3)))
        with pytest.raises(md.MDError):
            ctx.set_coulomb(Q, rc_coul=3.0)  # beyond the list's cutoff
        ctx.set_coulomb(None)
        assert ctx.stats()["coulomb"] == 0
        xg, _, f = (a.cpu().numpy() for a in ctx.get_state())
    fref, _, _ = O.forces(xg, box, O.LJ(1.0, 1.0, 2.5, ntypes=2), type_=t, skin=0.3)
    assert rel_err(f, fref) <= 1e-12


def test_batched_replicas_with_coulomb():
    """Four charged boxes of different size in one context: each matches the
    oracle on that box alone."""
    boxes, xs, vs, ts = [], [], [], []
    for k, n in enumerate((4, 5, 6, 4)):
        x, box, _ = S.fcc(n)
        x = x + 0.15 * (S.uniform(70 + k, x.size).reshape(x.shape) - 0.5)
        boxes.append(box)
        xs.append(x)
        vs.append(S.maxwell_boltzmann(np.ones(len(x)), 1.0, 80 + k))
        ts.append((np.arange(len(x)) % 4 >= 2).astype(np.int32))
    off = np.concatenate([[0], np.cumsum([len(x) for x in xs])]).astype(np.int64)
    with md.LJMD(np.concatenate(xs), np.concatenate(vs), np.concatenate(ts), np.stack(boxes),
                 1.0, 1.0, 2.5, [1.0, 1.0], list_kind=md.MD_LIST_HALF, threads_per_atom=1,
                 rep_offset=off) as ctx:
        ctx.set_coulomb(Q)
        ctx.set_kernel(1, -1, 2, 0)
        ctx.compute_forces(0)
        x, _, f = (a.cpu().numpy() for a in ctx.get_state())
        th = ctx.energy_replicas()
    lj = O.LJ(1.0, 1.0, 2.5, ntypes=2, q=Q, rc_coul=2.5)
    for r in range(len(xs)):
        a, b = off[r], off[r + 1]
        fref, E, _ = O.forces(x[a:b], boxes[r], lj, type_=ts[r], skin=0.3)
        assert rel_err(f[a:b], fref) <= 1e-12, r
        assert abs(th[r, 0] - E) <= 1e-12 * abs(E), r

