"""Double-float arithmetic (FR_DF) on the GPU.

1. The operations themselves against exact rational arithmetic on the same
   double-float operands (the FP32 pair a Python float rounds to), within the
   error bounds of the double-word algorithms (u = 2^-24): addition
   4u^2 (|a| + |b|) absolute, product 6u^2 relative, fused multiply-add the sum
   of both, division 16u^2 and square root 8u^2 relative; the FP64 value of
   the result adds at most 2^-53 relative.  A lost error term would show as
   an error of order u = 6e-8.
2. The FR residual in double-float arithmetic against the FP64 oracle.  The
   double-float operands carry relative rounding of 2^-48 (32 times FP64's)
   and every operation up to about 5u^2 = 2^-46 (160 times FP64's), so the
   FP64 bound of 1e-12 of max|R| (or of the flux scale) becomes 2e-10 (2e-9 on
   curved meshes, whose FP64 bound is ten times larger).
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

from helpers import gpu_ctx, oracle_fr, parity_ok, small_workloads

pytestmark = pytest.mark.gpu

U2 = Fraction(1, 2 ** 48)
D53 = Fraction(1, 2 ** 53)
WL = small_workloads()
CURVED = ("cylinder", "naca", "box_curved")
TOLDF = 2e-10


def tol_df(name):
    return 2e-9 if name.startswith(CURVED) else TOLDF


@pytest.fixture(scope="module")
def built():
    from paper_1910_03693_gb300 import build as B
    B.build()
    return True


def _df(x):
    """The double-float value a Python float is converted to: nearest FP32,
    plus the nearest FP32 of the remainder."""
    hi = float(np.float32(x))
    lo = float(np.float32(x - hi))
    return Fraction(hi) + Fraction(lo)


def _operands(seed, n):
    rng = np.random.default_rng(seed)
    a = np.sign(rng.standard_normal(n)) * 10.0 ** rng.uniform(-3, 3, n)
    b = np.sign(rng.standard_normal(n)) * 10.0 ** rng.uniform(-3, 3, n)
    c = np.sign(rng.standard_normal(n)) * 10.0 ** rng.uniform(-3, 3, n)
    # cancellation: b close to -a, c close to -a b
    k = n // 4
    b[:k] = -a[:k] * (1.0 + rng.uniform(-1e-6, 1e-6, k))
    c[:k] = -a[:k] * b[:k] * (1.0 + rng.uniform(-1e-9, 1e-9, k))
    return a, b, c


@pytest.mark.parametrize("op", ["add", "sub", "mul", "fma", "div", "sqrt"])
def test_dfloat_operations_within_double_word_bounds(built, op):
    from paper_1910_03693_gb300 import dfloat_eval
    n = 4000
    a, b, c = _operands(11, n)
    if op == "sqrt":
        a = np.abs(a)
    if op == "sub":
        b = -b           # the cancelling pairs of the sum cancel in the difference
    ta, tb, tc = (torch.from_numpy(x).cuda() for x in (a, b, c))
    out = dfloat_eval(op, ta, None if op == "sqrt" else tb, tc if op == "fma" else None).cpu().numpy()
    worst = Fraction(0)
    for i in range(n):
        x, y, z = _df(a[i]), _df(b[i]), _df(c[i])
        r = Fraction(float(out[i]))
        if op == "add":
            exact, bound = x + y, 4 * U2 * (abs(x) + abs(y))
        elif op == "sub":
            exact, bound = x - y, 4 * U2 * (abs(x) + abs(y))
        elif op == "mul":
            exact, bound = x * y, 6 * U2 * abs(x * y)
        elif op == "fma":
            exact, bound = x * y + z, 6 * U2 * abs(x * y) + 4 * U2 * (abs(x * y) + abs(z))
        elif op == "div":
            exact, bound = x / y, 16 * U2 * abs(x / y)
        else:
            # |r - sqrt(x)| = |r^2 - x| / (r + sqrt(x)) ~ |r^2 - x| / (2 r)
            err = abs(r * r - x) / (2 * r)
            bound = 8 * U2 * r + D53 * r
            worst = max(worst, err / bound)
            continue
        err = abs(r - exact)
        bound += D53 * abs(exact)
        worst = max(worst, err / bound if bound > 0 else (0 if err == 0 else Fraction(10 ** 9)))
    assert worst <= 1, (op, float(worst))


def test_dfloat_sqrt_of_zero_and_division_by_one(built):
    from paper_1910_03693_gb300 import dfloat_eval
    x = torch.tensor([0.0, 1.0, 2.0, 0.1], dtype=torch.float64, device="cuda")
    s = dfloat_eval("sqrt", x).cpu().numpy()
    assert s[0] == 0.0 and s[1] == 1.0
    assert abs(s[2] - np.sqrt(2.0)) <= 2e-14
    one = torch.ones_like(x)
    d = dfloat_eval("div", x, one).cpu().numpy()
    assert np.all(np.abs(d - x.cpu().numpy()) <= 4e-15 * np.abs(x.cpu().numpy()))


@pytest.mark.parametrize("name", list(WL))
def test_df_residual_parity(built, name):
    m, q, ph = WL[name]
    fr, ctx = oracle_fr(m, ph), gpu_ctx(m, ph)
    Rref = fr.residual(torch.from_numpy(q)).numpy()
    qs = ctx.pack(torch.from_numpy(q).cuda())
    R = ctx.unpack(ctx.residual(qs, double_float=True)).cpu().numpy()
    assert np.all(np.isfinite(R))
    ok, rel, fs = parity_ok(R, Rref, m, q, tol_df(name))
    assert ok, (name, rel, fs)
    # closer to FP64 than FP32 is by orders of magnitude
    R32 = ctx.unpack(ctx.residual(ctx.pack(torch.from_numpy(q).cuda(), torch.float32))).cpu().numpy()
    assert np.abs(R - Rref).max() <= 1e-3 * np.abs(R32 - Rref).max()


def test_df_residual_takes_fp64_buffers_only(built):
    m, q, ph = WL["vortex2d_16x16_p2"]
    ctx = gpu_ctx(m, ph)
    with pytest.raises(TypeError):
        ctx.residual(ctx.pack(torch.from_numpy(q).cuda(), torch.float32), double_float=True)
