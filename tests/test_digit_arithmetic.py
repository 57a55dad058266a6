"""The fixed-point digit arithmetic of the mixed path, checked on the CPU in NumPy (float32 where
the kernels use FP32): the four 8-bit signed digits reconstruct an operand to 2^-31 of its scale,
every order accumulator of a 128-deep product stays an integer below 2^24 (so the tensor cores'
FP32 accumulation is exact), and the product assembled from the four orders matches the binary64
product to the FP32 level relative to the row and column scales."""
import numpy as np
import pytest

MAGIC = np.float32(12582912.0)   # 1.5 * 2^23


def _rint(v):
    return (v + MAGIC) - MAGIC   # round to nearest even, in float32, for |v| < 2^22


def pow2_ceil(x):
    x = np.asarray(x, np.float64)
    out = np.ones_like(x)
    pos = x > 0
    out[pos] = 2.0 ** np.ceil(np.log2(x[pos]))
    return out.astype(np.float32)


def digits4(x, inv_scale):
    """d0..d3 with x / scale = (d0 + d1 2^-8 + d2 2^-16 + d3 2^-24) / 2^7, in float32."""
    v = (np.float32(x) * np.float32(inv_scale)) * np.float32(128.0)
    out = []
    for _ in range(4):
        d = _rint(v.astype(np.float32)).astype(np.float32)
        out.append(d)
        v = ((v - d) * np.float32(256.0)).astype(np.float32)
    return out


def test_digits_reconstruct_to_two_to_the_minus_31():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 3, 20000)).astype(np.float32)
    scale = pow2_ceil(np.abs(x).max())
    d = digits4(x, np.float32(1.0) / scale)
    assert all(np.all(np.abs(di) <= 128) for di in d)
    assert all(np.all(di == np.round(di)) for di in d)
    rec = sum(di.astype(np.float64) * 2.0 ** (-7 - 8 * i) for i, di in enumerate(d))
    assert np.max(np.abs(rec - x / scale)) <= 2.0 ** -31


@pytest.mark.parametrize("K", [16, 64, 128])
def test_order_accumulators_are_exact_and_the_product_is_fp32_accurate(K):
    rng = np.random.default_rng(K)
    M, N = 128, 64
    # rows and columns spanning several orders of magnitude, as U and Q do
    A = (rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-3, 1, (M, 1))).astype(np.float32)
    B = (rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-3, 1, (1, N))).astype(np.float32)
    alpha = pow2_ceil(np.abs(A).max(axis=1))
    gamma = pow2_ceil(np.abs(B).max(axis=0))
    da = digits4(A, (np.float32(1.0) / alpha)[:, None])
    db = digits4(B, (np.float32(1.0) / gamma)[None, :])
    D = [np.zeros((M, N)) for _ in range(4)]
    for a in range(4):
        for b in range(4 - a):
            D[a + b] += da[a].astype(np.float64) @ db[b].astype(np.float64)
    for o in range(4):
        assert np.max(np.abs(D[o])) < 2.0 ** 24      # integers the FP32 accumulator holds
        assert np.all(D[o] == np.round(D[o]))
    q = np.float32(2.0 ** -8)
    acc = D[2].astype(np.float32) + D[3].astype(np.float32) * q
    acc = D[0].astype(np.float32) + (D[1].astype(np.float32) + acc * q) * q
    W = acc * gamma[None, :] * (alpha[:, None] * np.float32(2.0 ** -14))
    exact = A.astype(np.float64) @ B.astype(np.float64)
    bound = np.outer(alpha, gamma).astype(np.float64)   # scale of each output's addends
    err = (W - exact) / bound
    assert np.max(np.abs(err)) <= 8 * 2.0 ** -24         # FP32 rounding of the epilogue only
    assert abs(np.mean(err)) <= 0.05 * np.sqrt(np.mean(err ** 2))   # and unbiased
