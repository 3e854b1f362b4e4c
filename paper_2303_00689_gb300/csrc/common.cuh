// Shared device utilities of the KSA-XL-BOMD CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include <mutex>

#ifndef KX_HOST_DEVICE
#define KX_HOST_DEVICE __host__ __device__ __forceinline__
#endif

namespace kx {

// ---------------------------------------------------------------------------
// launch bookkeeping (host)
// ---------------------------------------------------------------------------
void count_launch();            // increments the library-wide launch counter
cudaError_t last_launch_error(); // cudaGetLastError wrapper

// Set-up that belongs to a device (function attributes, __constant__ tables):
// done once per device ordinal, with that device current.  A process-wide
// "once" would leave every device but the first one unconfigured.
constexpr int kMaxDevices = 64;
struct PerDeviceOnce {
  std::mutex mu;
  unsigned long long done = 0;   // bit d: device d is set up
};
template <typename Fn>
bool once_per_device(PerDeviceOnce& flag, Fn&& fn) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
  std::lock_guard<std::mutex> lk(flag.mu);
  const unsigned long long bit = 1ull << dev;
  if (flag.done & bit) return true;
  if (!fn()) return false;
  flag.done |= bit;
  return true;
}

// physical constants (this library's own copy)
constexpr double kE2 = 14.399645;            // e^2/(4 pi eps0), eV*Angstrom
constexpr double kBohr = 0.52917721090;      // Angstrom
constexpr double kBoltz = 8.617333262e-5;    // eV/K
constexpr double kAccel = 9.648533212e-3;    // Angstrom/fs^2 per (eV/Angstrom)/amu

// ---------------------------------------------------------------------------
// per-element parameters as the kernels see them
// ---------------------------------------------------------------------------
struct Elem {
  double zcore, mass;
  double U[2];          // U_ss, U_pp
  double beta[2];       // beta_s, beta_p
  double zeta[2];       // zeta_s, zeta_p (1/bohr)
  double alpha;         // core-core exponent (1/Angstrom)
  double ga[2], gb[2], gc[2];  // AM1 Gaussians
  double G_ss, G_sp, G_pp, G_p2, H_sp, H_pp;
  double D1, D2;        // multipole lengths (Angstrom)
  double rho0, rho1, rho2;  // additive terms (Angstrom)
  double sto_nrm[2];    // Slater normalisation (2 zeta)^(n + 1/2) / sqrt((2n)!) for zeta_s, zeta_p
  int norb, nprin;
};

struct ElemTable {
  Elem e[4];  // H, C, N, O
};

// ---------------------------------------------------------------------------
// FP64 reciprocal and inverse square root: an FP32 estimate refined by two
// Newton-Raphson steps (r <- r + r (1 - x r); y <- y + y (1 - x y^2) / 2),
// each of which squares the relative error (about 2^-22 -> 2^-44 -> below
// FP64 rounding).  GB300 runs FP64 division and square root as long dependent
// sequences on its narrow FP64 pipe; these take 4 and 8 FP64 operations.
// Arguments must be positive and finite in FP32 (x > 2^-126); beyond the FP32
// maximum the results are 0, the limit the callers need.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rcp_nr(double x) {
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y = (double)rsqrtf((float)x);
  double e = fma(-x * y, y, 1.0);
  y = fma(0.5 * y, e, y);
  e = fma(-x * y, y, 1.0);
  return fma(0.5 * y, e, y);
}
KX_HOST_DEVICE double kx_rcp(double x) {
#if defined(__CUDA_ARCH__)
  return rcp_nr(x);
#else
  return 1.0 / x;
#endif
}

// ---------------------------------------------------------------------------
// forward-mode dual number with three derivative directions
// ---------------------------------------------------------------------------
struct D3 {
  double v, d0, d1, d2;
};

KX_HOST_DEVICE D3 mkd(double v) { return D3{v, 0.0, 0.0, 0.0}; }
KX_HOST_DEVICE D3 operator+(D3 a, D3 b) { return D3{a.v + b.v, a.d0 + b.d0, a.d1 + b.d1, a.d2 + b.d2}; }
KX_HOST_DEVICE D3 operator-(D3 a, D3 b) { return D3{a.v - b.v, a.d0 - b.d0, a.d1 - b.d1, a.d2 - b.d2}; }
KX_HOST_DEVICE D3 operator-(D3 a) { return D3{-a.v, -a.d0, -a.d1, -a.d2}; }
KX_HOST_DEVICE D3 operator+(D3 a, double b) { return D3{a.v + b, a.d0, a.d1, a.d2}; }
KX_HOST_DEVICE D3 operator+(double b, D3 a) { return a + b; }
KX_HOST_DEVICE D3 operator-(D3 a, double b) { return D3{a.v - b, a.d0, a.d1, a.d2}; }
KX_HOST_DEVICE D3 operator-(double b, D3 a) { return D3{b - a.v, -a.d0, -a.d1, -a.d2}; }
KX_HOST_DEVICE D3 operator*(D3 a, D3 b) {
  return D3{a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2};
}
KX_HOST_DEVICE D3 operator*(D3 a, double b) { return D3{a.v * b, a.d0 * b, a.d1 * b, a.d2 * b}; }
KX_HOST_DEVICE D3 operator*(double b, D3 a) { return a * b; }
KX_HOST_DEVICE D3 operator/(D3 a, D3 b) {
  double inv = kx_rcp(b.v);
  double q = a.v * inv;
  return D3{q, (a.d0 - q * b.d0) * inv, (a.d1 - q * b.d1) * inv, (a.d2 - q * b.d2) * inv};
}
KX_HOST_DEVICE D3 operator/(D3 a, double b) { return a * kx_rcp(b); }
KX_HOST_DEVICE D3 operator/(double a, D3 b) {
  double inv = kx_rcp(b.v);
  double q = a * inv;
  double s = -q * inv;
  return D3{q, s * b.d0, s * b.d1, s * b.d2};
}
KX_HOST_DEVICE D3& operator+=(D3& a, D3 b) { a = a + b; return a; }
KX_HOST_DEVICE D3& operator-=(D3& a, D3 b) { a = a - b; return a; }

__device__ __forceinline__ D3 sq(D3 a) {
  double r = rsqrt_nr(a.v);
  double s = a.v * r;
  double h = 0.5 * r;
  return D3{s, a.d0 * h, a.d1 * h, a.d2 * h};
}
// 1/sqrt(a) with its derivative -a'/(2 a^{3/2}) = -a' r^3 / 2
__device__ __forceinline__ D3 rsqrt_d(D3 a) {
  double r = rsqrt_nr(a.v);
  double h = -0.5 * r * r * r;
  return D3{r, a.d0 * h, a.d1 * h, a.d2 * h};
}
__device__ __forceinline__ double rsqrt_d(double a) { return rsqrt_nr(a); }
__device__ __forceinline__ D3 ex(D3 a) {
  double e = ::exp(a.v);
  return D3{e, a.d0 * e, a.d1 * e, a.d2 * e};
}
__device__ __forceinline__ double ex(double a) { return ::exp(a); }
__device__ __forceinline__ double sq(double a) { return a * rsqrt_nr(a); }
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(D3 a) { return a.v; }
// forward-mode dual number with one derivative direction (d/dR of the
// quantities that depend on the pair distance R alone)
struct D1 {
  double v, d;
};
KX_HOST_DEVICE D1 operator+(D1 a, D1 b) { return D1{a.v + b.v, a.d + b.d}; }
KX_HOST_DEVICE D1 operator-(D1 a, D1 b) { return D1{a.v - b.v, a.d - b.d}; }
KX_HOST_DEVICE D1 operator-(D1 a) { return D1{-a.v, -a.d}; }
KX_HOST_DEVICE D1 operator+(D1 a, double b) { return D1{a.v + b, a.d}; }
KX_HOST_DEVICE D1 operator+(double b, D1 a) { return D1{a.v + b, a.d}; }
KX_HOST_DEVICE D1 operator-(D1 a, double b) { return D1{a.v - b, a.d}; }
KX_HOST_DEVICE D1 operator-(double b, D1 a) { return D1{b - a.v, -a.d}; }
KX_HOST_DEVICE D1 operator*(D1 a, D1 b) { return D1{a.v * b.v, a.d * b.v + a.v * b.d}; }
KX_HOST_DEVICE D1 operator*(D1 a, double b) { return D1{a.v * b, a.d * b}; }
KX_HOST_DEVICE D1 operator*(double b, D1 a) { return D1{a.v * b, a.d * b}; }
KX_HOST_DEVICE D1 operator/(D1 a, D1 b) {
  double inv = kx_rcp(b.v);
  double q = a.v * inv;
  return D1{q, (a.d - q * b.d) * inv};
}
KX_HOST_DEVICE D1 operator/(double a, D1 b) {
  double inv = kx_rcp(b.v);
  double q = a * inv;
  return D1{q, -q * inv * b.d};
}
KX_HOST_DEVICE D1& operator+=(D1& a, D1 b) { a = a + b; return a; }
__device__ __forceinline__ D1 rsqrt_d(D1 a) {
  double r = rsqrt_nr(a.v);
  return D1{r, -0.5 * r * r * r * a.d};
}
__device__ __forceinline__ D1 ex(D1 a) {
  double e = ::exp(a.v);
  return D1{e, a.d * e};
}
__device__ __forceinline__ double val(D1 a) { return a.v; }

template <typename T> __device__ __forceinline__ T cst(double v);
template <> __device__ __forceinline__ double cst<double>(double v) { return v; }
template <> __device__ __forceinline__ D3 cst<D3>(double v) { return mkd(v); }
template <> __device__ __forceinline__ D1 cst<D1>(double v) { return D1{v, 0.0}; }

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed order (deterministic); every thread gets the total.
// `scratch` holds >= 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  double r = scratch[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// device status word (bitmask), read by the host after a step
// ---------------------------------------------------------------------------
enum DevStatus : int {
  kStatusNumeric = 1,   // NaN/Inf seen
  kStatusTimeout = 2,   // bounded wait expired
  kStatusNoConv = 4,    // mu bisection could not bracket
};

}  // namespace kx
