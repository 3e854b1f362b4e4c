"""tcgen05 BF16 GEMM (the contraction under eqs. 19 and 36 in the mixed path) vs numpy.

The expected value is built independently in numpy: each FP64 row is cut
into fixed-point slices of 8 bits relative to 2^e (e = frexp exponent of the
row's max |x|; balanced base-256 digits of the rounded scaled value), and
the kept slice products are summed in FP64.  Each
product of two slices is an integer times one power of two per (row, row,
slice pair), so the GPU's FP32 chunk sums are exact and its result must
equal the FP64 sum up to the double-float (hi + lo) rounding: <= 2^-40 of
sum |a||b| per entry.
"""
import numpy as np
import pytest

import paper_2303_00689_gb300 as kx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_00689_gb300 import build
    build.build()


def slices(X, k):
    """Fixed-point slices: the balanced base-256 digits of round(x 2^(7 + 8(k-1) - e_r)),
    digit a scaled by 2^(e_r - 7 - 8a), with e_r the frexp exponent of the row's max |x|."""
    amax = np.max(np.abs(X), axis=1)
    _, e = np.frexp(amax)
    e = np.where(amax > 0, e, 0)[:, None]
    Xi = np.rint(np.ldexp(X, 7 + 8 * (k - 1) - e)).astype(np.int64)
    digits = [None] * k
    for a in range(k - 1, 0, -1):
        r = Xi & 0xFF
        r = np.where(r >= 128, r - 256, r)
        digits[a] = r
        Xi = (Xi - r) >> 8
    digits[0] = Xi
    out = []
    for a in range(k):
        assert np.max(np.abs(digits[a])) <= 128
        out.append(np.ldexp(digits[a].astype(np.float64), e - 7 - 8 * a))
    return out


SLICES = {1: 1, 3: 2, 6: 3, 10: 4}


def kept_pairs(k):
    return [(a, d - a) for d in range(k) for a in range(d + 1)]


@pytest.mark.parametrize("n", [64, 128, 200, 333, 700])
@pytest.mark.parametrize("terms", [1, 3, 6, 10])
def test_tc_gemm_is_exact_on_slices(n, terms):
    rng = np.random.default_rng(n * 10 + terms)
    A = rng.normal(size=(n, n)) * np.exp(rng.normal(size=(n, 1)))   # rows of different scale
    B = rng.normal(size=(n, n))
    C = kx.sim_debug_tc_gemm(A, B, terms=terms)
    k = SLICES[terms]
    pa, pb = slices(A, k), slices(B, k)
    ref = sum(pa[i] @ pb[j].T for i, j in kept_pairs(k))
    scale = np.abs(A) @ np.abs(B).T
    assert np.max(np.abs(C - ref) / scale) < 2.0 ** -40
    # and the sliced product approaches the FP64 product as slices are added
    exact = A @ B.T
    bound = {1: 2.0 ** -4, 3: 2.0 ** -12, 6: 2.0 ** -20, 10: 2.0 ** -28}[terms]
    assert np.max(np.abs(C - exact) / scale) < bound


@pytest.mark.parametrize("n", [100, 256, 300])
def test_tc_gemm_symmetric_output(n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n))
    C = kx.sim_debug_tc_gemm(A, A, terms=10, sym=True)
    assert np.array_equal(C, C.T)
    exact = A @ A.T
    scale = np.abs(A) @ np.abs(A).T
    assert np.max(np.abs(C - exact) / scale) < 2.0 ** -26


@pytest.mark.parametrize("n", [64, 128, 200, 333, 700, 1100])
@pytest.mark.parametrize("sym", [False, True])
def test_grouped_product_is_the_three_slice_product(n, sym):
    """The DMPT's slice-grouped kernel: the weight-1 slice product is summed
    exactly per chunk, the lower-weight ones in FP32, so the result is the
    exact 6-term slice product to within 2^-24 of sum |a||b| (the bound the
    kernel's FP32 accumulation of weights 2^-8 and 2^-16 gives, with margin)
    and the FP64 product to within the 3-slice truncation 2^-20."""
    rng = np.random.default_rng(n + 7 * sym)
    A = rng.normal(size=(n, n)) * np.exp(rng.normal(size=(n, 1)))
    B = A if sym else rng.normal(size=(n, n))
    C = kx.sim_debug_tc_gemm_grouped(A, B, sym=sym, slices=3)
    pa, pb = slices(A, 3), slices(B, 3)
    ref = sum(pa[i] @ pb[j].T for i, j in kept_pairs(3))
    scale = np.abs(A) @ np.abs(B).T
    err_slices = np.max(np.abs(C - ref) / scale)
    err_exact = np.max(np.abs(C - A @ B.T) / scale)
    assert err_slices < 2.0 ** -24, err_slices
    assert err_exact < 2.0 ** -20, err_exact
    print(f"\nn {n} sym {sym}: 3-slice grouped vs slice product {np.log2(err_slices):.1f}, "
          f"vs FP64 product {np.log2(err_exact):.1f}")
    if sym:
        assert np.array_equal(C, C.T)


@pytest.mark.parametrize("n", [64, 128, 200, 333, 700, 1100])
@pytest.mark.parametrize("sym", [False, True])
def test_grouped_product_is_the_four_slice_product(n, sym):
    """The 4-slice grouped kernel (density product, back-transformation): the
    exact 10-term slice product to within 2^-24 of sum |a||b| and the FP64
    product likewise.  The bound is set by the tensor core's FP32
    accumulation of the lower-weight group over a 512-K chunk (measured up to
    ~2^-25.6 at n = 333), far above the 4-slice truncation (~2^-32) but far
    below the density bar of the path."""
    rng = np.random.default_rng(3 * n + sym)
    A = rng.normal(size=(n, n)) * np.exp(rng.normal(size=(n, 1)))
    B = A if sym else rng.normal(size=(n, n))
    C = kx.sim_debug_tc_gemm_grouped(A, B, sym=sym, slices=4)
    pa, pb = slices(A, 4), slices(B, 4)
    ref = sum(pa[i] @ pb[j].T for i, j in kept_pairs(4))
    scale = np.abs(A) @ np.abs(B).T
    err_slices = np.max(np.abs(C - ref) / scale)
    err_exact = np.max(np.abs(C - A @ B.T) / scale)
    assert err_slices < 2.0 ** -24, err_slices
    assert err_exact < 2.0 ** -24, err_exact
    print(f"\nn {n} sym {sym}: 4-slice grouped vs slice product {np.log2(err_slices):.1f} (log2 of the max "
          f"relative error), vs FP64 product {np.log2(err_exact):.1f}")
    if sym:
        assert np.array_equal(C, C.T)


def test_grouped_product_rejects_other_slice_counts():
    A = np.eye(64)
    with pytest.raises(kx.SimError) as e:
        kx.sim_debug_tc_gemm_grouped(A, A, slices=2)
    assert e.value.code == kx.SIM_EINVAL
