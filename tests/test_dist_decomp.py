"""Spatial decomposition (paper_2508_13523_gb300/decomp.py) on 2 and 3 CPU
ranks with the gloo backend: each rank owns a slab of the periodic box,
receives ghost atoms from its neighbors point to point, computes the forces
of its pairs with the oracle, and (newton on) sends the ghosts' forces back.
The owned atoms' forces, and their trajectory over 30 steps with three
reneighborings (atoms migrating between slabs), must match the single-box
oracle.

Inputs are rounded to a 2^-36 grid (box edge included) so that periodic
image shifts and separations are exact on both sides: the two runs then
differ only in the order of the FP64 force sums (and in the host
integrator's unfused multiply-add), well inside 1e-11.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

GRID = 2.0 ** -36
RLIST = 2.8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs():
    """The 4,000-atom fcc liquid (L = 16.8) 40 oracle steps after its fcc
    start (a perfect lattice has zero forces), rounded to the grid."""
    import oracle as O
    from paper_2508_13523_gb300 import synth as S
    s = S.fcc_liquid(10)
    box = np.round(s.box / GRID) * GRID
    x, v, _, _ = O.run(s.x, s.v, box, O.LJ(), 1.0, nsteps=40)
    return np.round(x / GRID) * GRID, v, box


def _engine(O, box_local):
    lj = O.LJ()

    def engine(x_own, xg, ids_own, ids_g, newton):
        xl = np.concatenate([x_own, xg]) if len(xg) else x_own
        n_own = len(x_own)
        pi, pk = O.pairs_cells(xl, box_local, RLIST)
        oi, ok = pi < n_own, pk < n_own
        gid = np.concatenate([ids_own, ids_g])
        if newton:  # each cross pair on the rank that owns its lower global id
            a = np.where(oi, pi, pk)
            b = np.where(oi, pk, pi)
            keep = (oi & ok) | ((oi ^ ok) & (gid[a] < gid[b]))
        else:       # every pair with an owned atom
            keep = oi | ok
        f, E, _ = O.forces(xl, box_local, lj, pairs=(pi[keep], pk[keep]))
        engine.energy = E
        return f[:n_own], f[n_own:]
    return engine


def _worker(rank, world, port, newton, nsteps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle as O
    from paper_2508_13523_gb300 import decomp as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, v, box = _inputs()
        xw = O.wrap(x, box)
        dom = D.SlabDomain(box, world, rank, RLIST)
        # the local frame: x never wraps (4 L), y and z periodic as the box
        box_local = np.array([4.0 * box[0], box[1], box[2]])
        eng = _engine(O, box_local)
        own = np.nonzero(dom.owner_of(xw) == rank)[0]
        ids, xf, vf, f = D.run_slabs(dom, own, xw[own], v[own], eng, nsteps=nsteps, dt=0.005,
                                     mass=1.0, box=box, rebuild_every=10, newton=newton)
        xo, vo, fo, th = O.run(x, v, box, O.LJ(), 1.0, nsteps=nsteps, rebuild_every=10,
                               thermo_every=max(nsteps, 1))
        rms = np.sqrt(np.mean(np.sum(fo * fo, axis=1)))
        e = torch.tensor([eng.energy if newton else 0.0], dtype=torch.float64)
        dist.all_reduce(e)  # the check only (the data path has no collective)
        cnt = torch.tensor([len(ids)], dtype=torch.int64)
        dist.all_reduce(cnt)
        out[rank] = dict(
            n_total=int(cnt.item()), n_ghost=int(len(dom.ghost_ids)),
            dx=float(np.abs(xf - xo[ids]).max()), dv=float(np.abs(vf - vo[ids]).max()),
            df=float(np.max(np.linalg.norm(f - fo[ids], axis=1)) / rms),
            de=abs(float(e.item()) - th[-1, 1]) / abs(th[-1, 1]) if newton else 0.0)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("newton", [False, True])
@pytest.mark.parametrize("nsteps", [0, 30])
def test_slab_decomposition_matches_single_box(world, newton, nsteps):
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(world, port, newton, nsteps, out), nprocs=world,
                       start_method="spawn")
    res = dict(out)
    assert sorted(res) == list(range(world))
    for r, d in res.items():
        assert d["n_total"] == 4000, d       # every atom owned exactly once
        assert d["n_ghost"] > 0, d
        assert d["df"] <= 1e-11, (r, d)
        assert d["dx"] <= 1e-11 and d["dv"] <= 1e-11, (r, d)
        assert d["de"] <= 1e-12, (r, d)


def test_slab_width_limits():
    from paper_2508_13523_gb300 import decomp as D
    box = np.array([16.8, 16.8, 16.8])
    with pytest.raises(ValueError):
        D.SlabDomain(box, 7, 0, RLIST)       # slab 2.4 < rlist
    with pytest.raises(ValueError):
        D.SlabDomain(box, 1, 0, RLIST)       # an atom would be its own ghost
    dom = D.SlabDomain(box, 3, 0, RLIST)
    assert dom.nbrs == [1, 2]
    x = np.array([[0.1, 0, 0], [5.5, 0, 0], [2.0, 0, 0]])
    i, s = dom.ghost_selection(x, 1)          # rank 1's slab [5.6, 11.2)
    assert list(i) == [1] and list(s) == [0]  # 5.5 is within rlist below it
    i, s = dom.ghost_selection(x, 2)          # rank 2's slab [11.2, 16.8)
    assert list(i) == [0, 2] and list(s) == [1, 1]  # 0.1 + L, 2.0 + L just above it
