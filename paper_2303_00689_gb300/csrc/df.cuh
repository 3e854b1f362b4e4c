// Double-float arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| at most
// half an ulp of hi: about 48 significant bits, the FP32 exponent range.  The
// operations are built from two error-free transformations:
//   two_sum(a, b):   s = fl(a + b) and the exact error a + b - s (Knuth),
//   exact product:   p = fl(a * b) and the exact error fma(a, b, -p),
// as in Dekker (1971) and Joldes, Muller and Popescu (ACM TOMS 2017).  GB300
// runs FP32 at 64 times its FP64 rate, so kernels whose work is dominated by
// FP64-accurate multiply-adds run them here.
//
// Device code uses the _rn intrinsics so the compiler cannot contract or
// reassociate the sequences (an fma formed from a * b + c would destroy the
// exactness of the transformations).  The host versions serve host-side
// conversions and checks; compile host code with -ffp-contract=off.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace kx {

struct __align__(8) dfl {
  float hi, lo;
};

#if defined(__CUDA_ARCH__)
#define KX_FADD(a, b) __fadd_rn((a), (b))
#define KX_FSUB(a, b) __fsub_rn((a), (b))
#define KX_FMUL(a, b) __fmul_rn((a), (b))
#define KX_FFMA(a, b, c) __fmaf_rn((a), (b), (c))
#else
#define KX_FADD(a, b) ((a) + (b))
#define KX_FSUB(a, b) ((a) - (b))
#define KX_FMUL(a, b) ((a) * (b))
#define KX_FFMA(a, b, c) fmaf((a), (b), (c))
#endif

__host__ __device__ __forceinline__ dfl df_two_sum(float a, float b) {
  float s = KX_FADD(a, b);
  float bb = KX_FSUB(s, a);
  float e = KX_FADD(KX_FSUB(a, KX_FSUB(s, bb)), KX_FSUB(b, bb));
  return dfl{s, e};
}
// requires |a| >= |b| or a == 0
__host__ __device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
  float s = KX_FADD(a, b);
  float e = KX_FSUB(b, KX_FSUB(s, a));
  return dfl{s, e};
}

__host__ __device__ __forceinline__ dfl df_from_double(double x) {
  float hi = (float)x;
  float lo = (float)(x - (double)hi);
  return dfl{hi, lo};
}
__host__ __device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

// FP32 -> FP64 by integer operations (exact for normal numbers, infinities and
// NaN; subnormal FP32 values, below 2^-126, become zero): keeps the conversion
// off GB300's narrow FP64 pipe.  No branch holds a conversion instruction, so
// none can be evaluated speculatively.
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFFu;
  unsigned long long b = (unsigned long long)(u & 0x80000000u) << 32;
  if (ex != 0) {
    const unsigned long long e64 = (ex == 0xFFu) ? 0x7FFull : (unsigned long long)(ex + 896u);
    b |= (e64 << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  }
  return __longlong_as_double((long long)b);
}
// FP64 -> double-float by integer operations (no FP64 instruction): the top
// 24 significand bits give hi, the remaining 29 bits (rounded to 24 by an
// integer-to-float conversion) give lo, then one renormalisation.  |x| below
// 2^-126 becomes 0, and below 2^-74 only hi is kept; |x| >= 2^128 becomes an
// infinity of its sign and NaN stays NaN (all by integer operations).
__device__ __forceinline__ dfl df_from_double_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const int ex = (int)((hw >> 20) & 0x7FFu);
  if (ex > 1150) {
    const bool nan = ex == 2047 && ((hw & 0xFFFFFu) | lw) != 0;
    return dfl{__uint_as_float(sign | (nan ? 0x7FC00000u : 0x7F800000u)), 0.0f};
  }
  if (ex < 897) return dfl{0.0f, 0.0f};
  const float hi = __uint_as_float(sign | ((unsigned)(ex - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  float lo = 0.0f;
  if (ex >= 949) {
    const float scale = __uint_as_float((unsigned)(ex - 948) << 23);   // 2^(ex - 1075)
    lo = __fmul_rn(__uint2float_rn(lw & 0x1FFFFFFFu), scale);
    lo = __uint_as_float(__float_as_uint(lo) | sign);
  }
  const float s = __fadd_rn(hi, lo);
  return dfl{s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
// hi + lo as a double with one FP64 addition (the two conversions by integer operations)
__device__ __forceinline__ double df_to_double_fast(dfl a) { return f2d_int(a.hi) + f2d_int(a.lo); }
__host__ __device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }

// a + b; absolute error of order 2^-48 (|a| + |b|)
__host__ __device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  dfl s = df_two_sum(a.hi, b.hi);
  float v = KX_FADD(s.lo, KX_FADD(a.lo, b.lo));
  return df_fast_two_sum(s.hi, v);
}
__host__ __device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

// a * b; relative error of order 2^-47 (the lo * lo term is dropped)
__host__ __device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  float p = KX_FMUL(a.hi, b.hi);
  float e = KX_FFMA(a.hi, b.hi, -p);
  e = KX_FFMA(a.hi, b.lo, e);
  e = KX_FFMA(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// Running sum without renormalisation after each term: acc.lo collects the
// rounding errors of acc.hi and the low parts of the products; df_norm once at
// the end.
__host__ __device__ __forceinline__ void df_acc_mul(dfl& acc, dfl a, dfl b) {
  float p = KX_FMUL(a.hi, b.hi);
  float e = KX_FFMA(a.hi, b.hi, -p);
  e = KX_FFMA(a.hi, b.lo, e);
  e = KX_FFMA(a.lo, b.hi, e);
  dfl s = df_two_sum(acc.hi, p);
  acc.hi = s.hi;
  acc.lo = KX_FADD(acc.lo, KX_FADD(s.lo, e));
}
__host__ __device__ __forceinline__ void df_acc(dfl& acc, dfl a) {
  dfl s = df_two_sum(acc.hi, a.hi);
  acc.hi = s.hi;
  acc.lo = KX_FADD(acc.lo, KX_FADD(s.lo, a.lo));
}
__host__ __device__ __forceinline__ dfl df_norm(dfl a) { return df_two_sum(a.hi, a.lo); }

// 1 / a: FP32 estimate and one Newton step in double-float (a.hi != 0)
__host__ __device__ __forceinline__ dfl df_recip(dfl a) {
  const float r0 = 1.0f / a.hi;
  const dfl r = dfl{r0, 0.0f};
  const dfl one_minus = df_sub(dfl{1.0f, 0.0f}, df_mul(a, r));   // 1 - a r0
  return df_add(r, df_mul(r, one_minus));
}
// sqrt(a), a >= 0: FP32 estimate s0 and one Newton correction (a - s0^2) / (2 s0)
__host__ __device__ __forceinline__ dfl df_sqrt(dfl a) {
  if (!(a.hi > 0.0f)) return dfl{0.0f, 0.0f};
  const float s0 = sqrtf(a.hi);
  const dfl e = df_sub(a, df_mul(dfl{s0, 0.0f}, dfl{s0, 0.0f}));
  return df_fast_two_sum(s0, KX_FMUL(e.hi, 0.5f / s0));
}

// x - u1 * w1 - u2 * w2 (the rank-2 update of one matrix element)
__host__ __device__ __forceinline__ dfl df_rank2(dfl x, dfl u1, dfl w1, dfl u2, dfl w2) {
  float p1 = KX_FMUL(u1.hi, w1.hi);
  float e1 = KX_FFMA(u1.hi, w1.hi, -p1);
  e1 = KX_FFMA(u1.hi, w1.lo, e1);
  e1 = KX_FFMA(u1.lo, w1.hi, e1);
  float p2 = KX_FMUL(u2.hi, w2.hi);
  float e2 = KX_FFMA(u2.hi, w2.hi, -p2);
  e2 = KX_FFMA(u2.hi, w2.lo, e2);
  e2 = KX_FFMA(u2.lo, w2.hi, e2);
  dfl s1 = df_two_sum(x.hi, -p1);
  dfl s2 = df_two_sum(s1.hi, -p2);
  float lo = KX_FSUB(KX_FADD(x.lo, KX_FADD(s1.lo, s2.lo)), KX_FADD(e1, e2));
  return df_fast_two_sum(s2.hi, lo);
}

#if defined(__CUDACC__)
__device__ __forceinline__ dfl df_shfl_xor(dfl a, int o) {
  return dfl{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
// sum over the 32 lanes (butterfly; every lane gets the same value)
__device__ __forceinline__ dfl df_warp_sum(dfl v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  return v;
}
#endif

}  // namespace kx
