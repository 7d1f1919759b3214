"""The arithmetic behind the TC_BF16X3 form, checked on the CPU.

Each FP32 operand is split into three BF16 planes, x0 = bf16(x), x1 = bf16(x -
x0), x2 = bf16(x - x0 - x1), and a product accumulates the six terms x_i y_j
with i + j <= 2. Here BF16 rounding (to nearest, ties to even, 8 significant
bits) is emulated exactly on the FP32 bit pattern, and the claims the library
states are checked:
* each difference is exact in FP32;
* the split leaves a residual of at most 2^-24 |x| (measured near 2^-27);
* the six-term dot product is within FP32 rounding of the FP64 one, where a
  single BF16 product is off by about 2^-9.
Nothing here calls the library: it pins the error model the GPU tests rely on."""
import numpy as np


def bf16(x):
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def split3(x):
    x = np.asarray(x, np.float32)
    x0 = bf16(x)
    r1 = (x - x0).astype(np.float32)
    x1 = bf16(r1)
    r2 = (r1 - x1).astype(np.float32)
    x2 = bf16(r2)
    return x0, x1, x2, r1, r2


def test_bf16_rounding_matches_definition():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even one (1)
    v = np.float32(1.0) + np.float32(2.0 ** -8)
    assert bf16(v) == np.float32(1.0)
    # just above the tie rounds up
    v = np.float32(1.0) + np.float32(2.0 ** -8) + np.float32(2.0 ** -20)
    assert bf16(v) == np.float32(1.0 + 2.0 ** -7)
    # BF16 values are fixed points
    x = np.float32([0.5, -3.0, 1.0 + 2.0 ** -7, 2.0 ** -100, 2.0 ** 100])
    assert np.array_equal(bf16(x), x)


def test_split_differences_are_exact_and_residual_is_small():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-30, 30, 200000))).astype(np.float32)
    x0, x1, x2, r1, r2 = split3(x)
    xd = x.astype(np.float64)
    # the FP32 differences equal the exact ones
    assert np.array_equal(r1.astype(np.float64), xd - x0.astype(np.float64))
    assert np.array_equal(r2.astype(np.float64), r1.astype(np.float64) - x1.astype(np.float64))
    rel = np.abs(xd - x0 - x1.astype(np.float64) - x2.astype(np.float64)) / np.abs(xd)
    assert rel.max() <= 2.0 ** -24
    assert np.median(rel) < 2.0 ** -26


def test_six_term_products_reach_fp32_accuracy():
    rng = np.random.default_rng(1)
    K = 512
    a = rng.standard_normal((64, K)).astype(np.float32)
    b = rng.standard_normal((K, 64)).astype(np.float32)
    exact = a.astype(np.float64) @ b.astype(np.float64)
    pa, pb = split3(a)[:3], split3(b)[:3]
    six = sum(pa[i].astype(np.float64) @ pb[j].astype(np.float64)
              for i in range(3) for j in range(3) if i + j <= 2)
    one = pa[0].astype(np.float64) @ pb[0].astype(np.float64)
    scale = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64)
    err6 = np.max(np.abs(six - exact) / scale)
    err1 = np.max(np.abs(one - exact) / scale)
    assert err6 < 2.0 ** -24   # the split terms alone: below FP32 rounding
    assert err1 > 2.0 ** -12   # one BF16 product: about 2^-9
