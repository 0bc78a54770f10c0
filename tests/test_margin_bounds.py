"""CPU pins for the quantisation part of the scoring margins.

The scoring pass sees rounded rows; the margin m_i bounds |s~ - s| so that
the filter keeps every exact result.  These tests check the bounds against
exact arithmetic, independently of the GPU code:

* BF16: s~ = <bf16(a), bf16(b)>, bound ||a~ - a|| ||b|| + ||a~|| ||b~ - b||;
* BF16 hi/lo split: x = hi + lo + e with hi = bf16(x), lo = bf16(x - hi); the
  tensor cores sum hi.hi + hi.lo + lo.hi, i.e. <a~, b~> - <a_lo, b_lo> with
  a~ = hi + lo, bound ||e_a|| ||b|| + (||a_hi|| + ||a_lo||) ||e_b||
  + ||a_lo|| ||b_lo||.

Products of float32 (or bfloat16) values are exact in float64 and math.fsum
rounds their sum once, so |s - s~| is known to ~1e-16 here, far below the
bounds (~1e-3 for BF16, ~1e-5 for the split).  The accumulation allowance of
the tensor cores is not part of these pins (it is a stated allowance, checked
on the GPU against observed errors).
"""
import math

import numpy as np
import pytest

from paper_2112_07552_gb300 import datagen

torch = pytest.importorskip("torch")


def bf16(x64):
    """Round-to-nearest-even to bfloat16 (as the packing kernel does), in float64."""
    t = torch.from_numpy(np.asarray(x64, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def split(x32):
    hi = bf16(x32)
    r = x32.astype(np.float64) - hi  # exact, and representable in float32
    assert np.array_equal(r, r.astype(np.float32).astype(np.float64))
    lo = bf16(r)
    e = r - lo  # exact
    return hi, lo, e


def dot(u, v):
    return math.fsum((u * v).tolist())


def nrm(u):
    return math.sqrt(math.fsum((u * u).tolist()))


def split_bound(a, b):
    ah, al, ae = split(a)
    bh, bl, be = split(b)
    return (nrm(ae) * nrm(b.astype(np.float64)) + (nrm(ah) + nrm(al)) * nrm(be)
            + nrm(al) * nrm(bl))


def split_product(a, b):
    ah, al, _ = split(a)
    bh, bl, _ = split(b)
    return math.fsum(np.concatenate([ah * bh, ah * bl, al * bh]).tolist())


@pytest.mark.parametrize("d", [64, 256, 768])
def test_split_bound_holds_and_is_near_2_pow_minus_16(d):
    A = datagen.clustered(40, d, 3, 0.1, seed=d, stream=0)
    B = datagen.clustered(60, d, 3, 0.1, seed=d, stream=1)
    worst_ratio, worst_bound = 0.0, 0.0
    for a in A:
        for b in B:
            s = dot(a.astype(np.float64), b.astype(np.float64))
            err = abs(s - split_product(a, b))
            bound = split_bound(a, b)
            assert err <= bound
            worst_ratio = max(worst_ratio, err / bound)
            worst_bound = max(worst_bound, bound)
    # unit rows: the split's quantisation bound is a few times 2^-16, two
    # orders of magnitude below BF16's ~2^-8
    assert worst_bound < 2.0 ** -13
    assert worst_ratio > 0.0


def test_bf16_bound_holds_and_is_much_wider():
    d = 256
    A = datagen.clustered(30, d, 3, 0.1, seed=5, stream=0)
    B = datagen.clustered(40, d, 3, 0.1, seed=5, stream=1)
    widest = 0.0
    for a in A:
        at = bf16(a)
        for b in B:
            bt = bf16(b)
            s = dot(a.astype(np.float64), b.astype(np.float64))
            err = abs(s - dot(at, bt))
            bound = nrm(at - a) * nrm(b.astype(np.float64)) + nrm(at) * nrm(bt - b)
            assert err <= bound
            widest = max(widest, bound)
            assert bound > 30 * split_bound(a, b)
    assert widest > 2.0 ** -10


def test_split_needs_the_lo_lo_term():
    # x = 1 + 2^-8 + 2^-9 rounds to hi = 1 + 2^-7 with lo = -2^-9 exactly
    # (e = 0): the split drops exactly sum lo^2 = d 2^-18, which only the
    # ||a_lo|| ||b_lo|| term of the bound covers
    d = 32
    x = np.full(d, 1.0 + 2.0 ** -8 + 2.0 ** -9, dtype=np.float32)
    hi, lo, e = split(x)
    assert np.all(hi == 1.0 + 2.0 ** -7) and np.all(lo == -(2.0 ** -9)) and np.all(e == 0)
    s = dot(x.astype(np.float64), x.astype(np.float64))
    err = abs(s - split_product(x, x))
    assert err == d * 2.0 ** -18
    assert err <= split_bound(x, x)
    without = nrm(e) * nrm(x.astype(np.float64)) + (nrm(hi) + nrm(lo)) * nrm(e)
    assert err > without
