"""The bounded grid barrier of the one-launch-per-step schedule (needs a
GPU).  Failure is made without a fault: a cooperative grid whose barrier
waits for one block more than it has can never complete, so every block's
wait runs out after its limit, sets the error word and returns.  The call
must report MD_ETIMEOUT, take about the limit, and leave the context usable;
with every block present the barrier completes at once."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2508_13523_gb300 as md  # noqa: E402


def test_barrier_completes_with_every_block():
    word = torch.zeros(4, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    assert md.eval_barrier(152, 0, 1000.0, word) == md.MD_OK
    assert time.perf_counter() - t0 < 0.5
    assert word[2].item() == 0


def test_barrier_wait_runs_out_and_reports():
    word = torch.zeros(4, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    assert md.eval_barrier(152, 1, 200.0, word) == md.MD_ETIMEOUT
    dt = time.perf_counter() - t0
    assert 0.19 < dt < 5.0, dt
    assert word[2].item() == 1
    # the context still works
    a = torch.linspace(0.5, 7.0, 1000, dtype=torch.float64, device="cuda")
    r = torch.empty_like(a)
    md.eval_recip(a, r, None)
    torch.cuda.synchronize()
    np.testing.assert_allclose(r.cpu().numpy(), 1.0 / a.cpu().numpy(), rtol=1e-15)


def test_barrier_argument_checks():
    lib = md.load()
    assert lib.md_eval_barrier(0, 0, 10.0, None, None) == md.MD_EINVAL
    assert lib.md_eval_barrier(4, 2, 10.0, None, None) == md.MD_EINVAL
