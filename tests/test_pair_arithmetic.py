"""CPU: the pair-of-FP32 arithmetic of the refinement residual, emulated step by
step in IEEE single precision, against exact rational dot products.

Each FP32 operation of the device code (round-to-nearest add, multiply and
fused multiply-add) is emulated by computing in float64 and rounding once to
float32; for operands of similar magnitude (as here) the float64 intermediate is
exact, so the emulation is exactly the device rounding.  The dot product follows
the device kernel: exact product p + e by FMA, two-sum of the leading parts,
low-order terms and rounding errors into the second float, fast two-sum
renormalisation every 4 terms.  The bound checked is the one the design states:
error <= sqrt(K) * 5 * 2^-48 of sum |a_k b_k| (about 4e-14 at K = 512); a
variant with the two-sum error dropped, or the low parts ignored, must fail it.
"""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def add(a, b):
    return f32(float(a) + float(b))


def sub(a, b):
    return f32(float(a) - float(b))


def mul(a, b):
    return f32(float(a) * float(b))


def fma(a, b, c):
    return f32(float(a) * float(b) + float(c))


def split(x):
    hi = f32(x)
    return hi, f32(x - float(hi))


def pair_dot(a, b, drop_twosum_error=False, drop_low=False, renorm_every=4):
    S, C = f32(0), f32(0)
    for k, (x, y) in enumerate(zip(a, b)):
        ah, al = split(x)
        bh, bl = split(y)
        if drop_low:
            al, bl = f32(0), f32(0)
        p = mul(ah, bh)
        e = fma(ah, bh, -p)
        t = fma(ah, bl, fma(al, bh, e))
        s = add(S, p)
        v = sub(s, S)
        err = add(sub(S, sub(s, v)), sub(p, v))
        if drop_twosum_error:
            err = f32(0)
        C = add(C, add(err, t))
        S = s
        if k % renorm_every == renorm_every - 1:
            s = add(S, C)
            C = sub(C, sub(s, S))
            S = s
    return float(S) + float(C)


def exact_dot(a, b):
    return float(sum(Fraction(x) * Fraction(y) for x, y in zip(a, b)))


def bound(a, b):
    K = len(a)
    return np.sqrt(K) * 5 * 2.0 ** -48 * float(np.sum(np.abs(np.asarray(a) * np.asarray(b))))


@pytest.mark.parametrize("K,seed", [(16, 0), (128, 1), (512, 2), (512, 3)])
def test_pair_dot_within_design_bound(K, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(K) * np.exp(rng.uniform(-3, 3, K))
    b = rng.standard_normal(K)
    err = abs(pair_dot(a, b) - exact_dot(a, b))
    assert err <= bound(a, b), (err, bound(a, b))


def test_pair_dot_cancellation():
    """Terms that cancel to a small sum: the error stays relative to sum |a b|."""
    rng = np.random.default_rng(7)
    a = rng.standard_normal(256)
    b = rng.standard_normal(256)
    a = np.concatenate([a, -a * (1 + 1e-9)])
    b = np.concatenate([b, b])
    err = abs(pair_dot(a, b) - exact_dot(a, b))
    assert err <= bound(a, b)


def test_pair_dot_single_precision_inputs_are_exact():
    """Inputs already in FP32 with small integer values: every product and
    partial sum is representable, so the pair result is exact."""
    rng = np.random.default_rng(9)
    a = rng.integers(-1000, 1000, 64).astype(np.float64)
    b = rng.integers(-1000, 1000, 64).astype(np.float64)
    assert pair_dot(a, b) == exact_dot(a, b)


@pytest.mark.parametrize("mutation", ["drop_twosum_error", "drop_low"])
def test_pair_dot_mutations_fail_the_bound(mutation):
    rng = np.random.default_rng(11)
    a = rng.standard_normal(512) * np.exp(rng.uniform(-3, 3, 512))
    b = rng.standard_normal(512)
    err = abs(pair_dot(a, b, **{mutation: True}) - exact_dot(a, b))
    assert err > 100 * bound(a, b)
