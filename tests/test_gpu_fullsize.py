"""Full-size parity on sampled outputs (needs a GB300).

The 4,000,000-atom fcc liquid in the configuration bench.py times (tuned
threads per atom, 20 steps with a rebuild), and the 16,384,000-atom box
(the largest scaling size; list offsets and tiled indices in 64 bits).  The
oracle computes the force and the neighbor set of sampled atoms one by one
by scanning all atoms; properties that hold at any size are checked on
every atom.
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


def sample_ids(n, k, seed):
    return np.unique((S.uniform(seed, k) * n).astype(np.int64))


def check_rows_against_oracle(ctx, x, box, sample, half):
    off, idx = ctx.neighbors()
    off = off.cpu().numpy()
    idx = idx.cpu().numpy()
    ref = O.neighbors_of(x, box, 2.8, sample)
    if not half:
        for s, i in enumerate(sample):
            assert np.array_equal(np.sort(idx[off[i]:off[i + 1]]), ref[s]), i
        return
    # half list: atom i's pairs are its own row plus the rows that list i
    in_sample = np.zeros(len(x), dtype=bool)
    in_sample[sample] = True
    pos = np.nonzero(in_sample[idx])[0]
    owners = np.searchsorted(off, pos, side="right") - 1
    listed_by = {}
    for p, o in zip(pos, owners):
        listed_by.setdefault(int(idx[p]), []).append(int(o))
    for s, i in enumerate(sample):
        got = list(idx[off[i]:off[i + 1]]) + listed_by.get(int(i), [])
        assert len(got) == len(set(got)), i
        assert np.array_equal(np.sort(np.array(got, dtype=np.int64)), ref[s].astype(np.int64)), i


@pytest.fixture(scope="module")
def liquid4m():
    return S.fcc_liquid(100)


@pytest.mark.parametrize("kind,prec", [(md.MD_LIST_HALF, md.MD_PREC_FP64),
                                       (md.MD_LIST_FULL, md.MD_PREC_FP64),
                                       (md.MD_LIST_FULL, md.MD_PREC_MIXED)])
def test_4m_sampled_forces_and_neighbors(liquid4m, kind, prec, capsys):
    s = liquid4m
    with md.from_system(s, list_kind=kind, precision=prec, threads_per_atom=0) as ctx:
        ctx.step(20)  # includes the rebuild after step 19 (wrap + sort)
        x, _, f = (a.cpu().numpy() for a in ctx.get_state())
        st = ctx.stats()
        sample = sample_ids(s.n, 64, 11 + kind + 2 * prec)
        check_rows_against_oracle(ctx, x, s.box, sample, kind == md.MD_LIST_HALF)
    fref = O.force_of(x, s.box, O.LJ(), sample)
    rms = np.sqrt(np.mean(np.sum(f * f, axis=1)))
    err = np.max(np.linalg.norm(f[sample] - fref, axis=1)) / rms
    print(f"4M kind={kind} prec={prec} tpa={st['threads_per_atom']} "
          f"compacted={st['compacted']}: sampled force err {err:.3e}")
    assert err <= (1e-12 if prec == md.MD_PREC_FP64 else 1e-4)
    # Newton's third law over all 4M atoms
    tot = np.abs(f.sum(axis=0)).max()
    assert tot <= (1e-9 if prec == md.MD_PREC_FP64 else 1e-3) * rms * np.sqrt(s.n)


def test_16m_sampled_forces_fp64_half(capsys):
    """Warp-compacted kernel with fixed-point force sums."""
    s = S.fcc_liquid(160)
    with md.from_system(s, list_kind=md.MD_LIST_HALF, threads_per_atom=1) as ctx:
        ctx.set_kernel(1, -1, 2, 0)
        ctx.step(20)  # away from the perfect lattice, whose forces vanish
        x, _, f = (a.cpu().numpy() for a in ctx.get_state())
        st = ctx.stats()
        sample = sample_ids(s.n, 24, 17)
        check_rows_against_oracle(ctx, x, s.box, sample, True)
    assert st["n_replicas"] == 1 and st["total_cells"] == 96 ** 3  # 95 cells, padded to bricks
    fref = O.force_of(x, s.box, O.LJ(), sample)
    rms = np.sqrt(np.mean(np.sum(f * f, axis=1)))
    err = np.max(np.linalg.norm(f[sample] - fref, axis=1)) / rms
    print(f"16.4M half: sampled force err {err:.3e}, list entries {st['list_entries']}")
    assert err <= 1e-12
