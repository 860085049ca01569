"""md_kinetic_noalloc, the entry point for callers that cannot allocate device
memory, against md_energy's kinetic energy and temperature (needs a GPU).

Runs last (file name) so that a failure here, under -x, comes after every
other test; it must pass alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2508_13523_gb300 as md  # noqa: E402
from paper_2508_13523_gb300 import synth as S  # noqa: E402

REL = 1e-12  # the kinetic-energy tolerance of the other GPU tests


def _systems():
    yield S.fcc_liquid(8)                      # 2,048 atoms: two full blocks
    mix = S.binary_mixture(n=3000, seed=5)     # 3,000 atoms: a ragged last block
    yield mix


@pytest.mark.parametrize("which", [0, 1])
def test_noalloc_matches_md_energy_twice(which):
    sysm = list(_systems())[which]
    p = sysm.params
    with md.from_system(sysm, threads_per_atom=1) as ctx:
        th = ctx.energy()
        _, v, _ = ctx.get_state()
    t = torch.as_tensor(sysm.type, dtype=torch.int32, device=v.device)
    for call in range(2):  # two calls in a row share the static scratch
        out = torch.full((2,), float("nan"), dtype=torch.float64, device=v.device)
        md.kinetic_noalloc(v, t, p.mass, out)
        torch.cuda.synchronize()
        ke, temp = out.cpu().tolist()
        assert abs(ke - th.ke) <= REL * th.ke, (call, ke, th.ke)
        assert abs(temp - th.temperature) <= REL * th.temperature, (call, temp)


def test_noalloc_skips_types_out_of_range():
    """Atoms whose type lies outside [0, n_types) add nothing: with two such
    atoms the result is md_energy's kinetic energy less theirs."""
    sysm = S.fcc_liquid(8)
    p = sysm.params
    with md.from_system(sysm, threads_per_atom=1) as ctx:
        th = ctx.energy()
        _, v, _ = ctx.get_state()
    t = torch.zeros(sysm.n, dtype=torch.int32, device=v.device)
    t[5] = 1   # n_types = 1: type 1 is out of range
    t[77] = -3
    vh = v.cpu().numpy()
    drop = 0.5 * p.mass[0] * (np.sum(vh[5] ** 2) + np.sum(vh[77] ** 2))
    expect = th.ke - drop
    for call in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device=v.device)
        md.kinetic_noalloc(v, t, p.mass, out)
        torch.cuda.synchronize()
        ke = out[0].item()
        assert abs(ke - expect) <= REL * th.ke, (call, ke, expect)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    lib = md.load()
    mass = (ctypes.c_double * 1)(1.0)
    d = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    rc = lib.md_kinetic_noalloc(md.MD_NOALLOC_MAX_ATOMS + 1, d, None, 1, mass, d, None)
    assert rc == md.MD_EINVAL
    assert lib.md_kinetic_noalloc(0, d, None, 1, mass, d, None) == md.MD_EINVAL
