"""The slab decomposition (decomp.py) with the GPU library as each rank's
force engine (LJMDSlabEngine, newton off), two ranks as two processes on
one GPU exchanging ghosts through gloo on the host (no kernel of one rank
waits on the other's): owned forces and a 30-step trajectory with three
reneighborings match the single-box oracle (needs a GPU)."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

GRID = 2.0 ** -36
RLIST = 2.8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, nsteps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle as O
    import paper_2508_13523_gb300 as md
    from paper_2508_13523_gb300 import decomp as D
    from paper_2508_13523_gb300 import synth as S
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    eng = None
    try:
        s = S.fcc_liquid(10)
        box = np.round(s.box / GRID) * GRID
        x, v, _, _ = O.run(s.x, s.v, box, O.LJ(), 1.0, nsteps=40)
        x = np.round(x / GRID) * GRID
        xw = O.wrap(x, box)
        dom = D.SlabDomain(box, world, rank, RLIST)
        eng = D.LJMDSlabEngine(md, box)
        own = np.nonzero(dom.owner_of(xw) == rank)[0]
        ids, xf, vf, f = D.run_slabs(dom, own, xw[own], v[own], eng, nsteps=nsteps, dt=0.005,
                                     mass=1.0, box=box, rebuild_every=10, newton=False)
        xo, vo, fo, _ = O.run(x, v, box, O.LJ(), 1.0, nsteps=nsteps, rebuild_every=10)
        rms = np.sqrt(np.mean(np.sum(fo * fo, axis=1)))
        out[rank] = dict(n=len(ids), dx=float(np.abs(xf - xo[ids]).max()),
                         dv=float(np.abs(vf - vo[ids]).max()),
                         df=float(np.max(np.linalg.norm(f - fo[ids], axis=1)) / rms))
    finally:
        if eng is not None:
            eng.close()
        dist.destroy_process_group()


@pytest.mark.parametrize("nsteps", [0, 30])
def test_slabs_with_gpu_engine_match_single_box(nsteps):
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(world, port, nsteps, out), nprocs=world,
                       start_method="spawn")
    res = dict(out)
    assert sorted(res) == [0, 1]
    assert sum(d["n"] for d in res.values()) == 4000
    for r, d in res.items():
        assert d["df"] <= 1e-11, (r, d)
        assert d["dx"] <= 1e-11 and d["dv"] <= 1e-11, (r, d)
