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

// FP32 -> FP64 by integer operations (exact for normal numbers; subnormal FP32
// values, below 2^-126, become zero; infinities and NaN take the conversion
// instruction): keeps the conversion off GB300's narrow FP64 pipe
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFFu;
  if (ex == 0xFFu) return (double)f;
  unsigned long long b = (unsigned long long)(u & 0x80000000u) << 32;
  if (ex != 0) b |= ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
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

}  // namespace kx
