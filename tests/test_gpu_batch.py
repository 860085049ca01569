"""Batched replicas (md_create_batch) vs the FP64 CPU oracle run on each box
separately (needs a GPU).

Uneven boxes -- fcc n^3 with n from 3 (L = 5.04 < 2 (rc + skin): one cell
per axis) upwards, different temperatures -- share one context and one
launch per kernel per step.  Each box must match the oracle on that box
alone: neighbor sets exact, FP64 forces within 1e-12 of rms, energies and
virials within 1e-12, trajectories with rebuilds.
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


def rel_err(f, fref):
    rms = np.sqrt(np.mean(np.sum(fref * fref, axis=1)))
    return float(np.max(np.linalg.norm(f - fref, axis=1)) / rms)


@pytest.fixture(scope="module")
def boxes():
    """12 boxes, n in 3..8 from the batched workload's generator (seeded),
    each relaxed 10 oracle steps away from the perfect lattice."""
    systems = S.replicas(R=12, seed=7, lo=3, hi=8)
    out = []
    for s in systems:
        x, v, _, _ = O.run(s.x, s.v, s.box, O.LJ(), 1.0, nsteps=10, rebuild_every=1)
        s.x, s.v = x, v
        out.append(s)
    return out


def offsets(systems):
    return np.concatenate([[0], np.cumsum([s.n for s in systems])]).astype(np.int64)


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("tpa", [1, 8, "compacted", "fixed", "fixed2"])
def test_batch_neighbors_forces_energies(boxes, kind, tpa):
    off = offsets(boxes)
    with md.from_systems(boxes, list_kind=kind,
                         threads_per_atom=tpa if isinstance(tpa, int) else 1) as ctx:
        if not isinstance(tpa, int):
            ctx.set_kernel(1, -1, {"compacted": 1, "fixed": 2, "fixed2": 3}[tpa], 0)
            ctx.compute_forces(0)
        assert ctx.stats()["n_replicas"] == len(boxes)
        x, _, f = (a.cpu().numpy() for a in ctx.get_state())
        cso, csi = (a.cpu().numpy() for a in ctx.neighbors())
        th = ctx.energy_replicas()
        tot = ctx.energy()
    for r, s in enumerate(boxes):
        a, b = off[r], off[r + 1]
        xr = x[a:b]
        pi, pk = O.pairs_cells(xr, s.box, s.params.rlist)
        ref = set(zip(pi.tolist(), pk.tolist()))
        got = []
        for i in range(a, b):
            js = csi[cso[i]:cso[i + 1]]
            assert np.all((js >= a) & (js < b)), "a pair crosses boxes"
            got += [(min(i - a, j - a), max(i - a, j - a)) for j in js.tolist()]
        if kind == md.MD_LIST_HALF:
            assert len(got) == len(set(got))
            assert set(got) == ref
        else:
            assert len(got) == 2 * len(ref) and set(got) == ref
        fref, E, W = O.forces(xr, s.box, O.LJ(), skin=0.3)
        assert rel_err(f[a:b], fref) <= 1e-12, r
        assert abs(th[r, 0] - E) <= 1e-12 * abs(E), r
        np.testing.assert_allclose(th[r, 4:10], W, rtol=1e-12, atol=1e-12 * np.abs(W).max())
    assert abs(tot.pe - th[:, 0].sum()) <= 1e-12 * abs(tot.pe)


@pytest.mark.parametrize("kind", [md.MD_LIST_FULL, md.MD_LIST_HALF])
@pytest.mark.parametrize("fused", [False, True])
def test_batch_trajectory_matches_oracle_per_box(boxes, kind, fused):
    """fused: one cooperative launch per step over all boxes (compacted
    fixed-point kernel, persistent 2)."""
    off = offsets(boxes)
    with md.from_systems(boxes, list_kind=kind, rebuild_every=5, threads_per_atom=2) as ctx:
        if fused:
            ctx.set_kernel(1, -1, 2, 2)
            ctx.compute_forces(0)
        x0, v0, _ = (a.cpu().numpy() for a in ctx.get_state())
        ctx.step(25)
        x, v, f = (a.cpu().numpy() for a in ctx.get_state())
        th = ctx.energy_replicas()
    for r, s in enumerate(boxes):
        a, b = off[r], off[r + 1]
        xo, vo, fo, tho = O.run(x0[a:b], v0[a:b], s.box, O.LJ(), 1.0, nsteps=25,
                                rebuild_every=5, thermo_every=25)
        assert np.abs(x[a:b] - xo).max() < 1e-11, r
        assert np.abs(v[a:b] - vo).max() < 1e-11, r
        assert rel_err(f[a:b], fo) < 1e-11, r
        assert abs(th[r, 1] - tho[-1, 2]) <= 1e-11 * tho[-1, 2], r
        assert abs(th[r, 3] - 2 * tho[-1, 2] / (3 * s.n - 3)) <= 1e-11 * th[r, 3]


def test_batch_mixed_error_reported(boxes, capsys):
    off = offsets(boxes)
    with md.from_systems(boxes, precision=md.MD_PREC_MIXED, threads_per_atom=1) as ctx:
        x, _, f = (a.cpu().numpy() for a in ctx.get_state())
    worst = 0.0
    for r, s in enumerate(boxes):
        a, b = off[r], off[r + 1]
        fref, _, _ = O.forces(x[a:b], s.box, O.LJ(), skin=0.3)
        worst = max(worst, rel_err(f[a:b], fref))
    print(f"batched mixed: worst box force err {worst:.3e}")
    assert worst < 1e-4


def test_batch_rejects_bad_offsets():
    s = S.fcc_liquid(4)
    with pytest.raises(md.MDError):
        md.LJMD(s.x, s.v, None, np.stack([s.box, s.box]), 1.0, 1.0, 2.5, 1.0,
                rep_offset=[0, 100, 300])  # last offset != n_atoms
    with pytest.raises(md.MDError):
        md.LJMD(s.x, s.v, None, np.stack([s.box, [4.0, 10.0, 10.0]]), 1.0, 1.0, 2.5, 1.0,
                rep_offset=[0, 100, s.n])  # 4.0 < 2 rc
