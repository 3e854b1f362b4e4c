// NDDO two-centre quantities for every atom pair A < B, and their derivatives
// with respect to the pair vector d = R_B - R_A.
//
// Model (MNDO multipole form; the paper names the AM1/MNDO/PM3 Hamiltonians
// in its Introduction and relies on NDDO, S = I, under eq. 6):
//  * each orbital product is a set of point charges in the local frame with
//    z' from A to B; two charges interact as e^2 q_i q_j /
//    sqrt(r_ij^2 + (rho_i + rho_j)^2);
//  * (p_pi p_pi'|p_pi p_pi') = [(p_pi p_pi|p_pi p_pi) - (p_pi p_pi|p_pi' p_pi')]/2
//    keeps the rotated set independent of the choice of x';
//  * the molecular-frame block is C I_loc C^T with C the 10x10 transform
//    of orbital products built from the frame rotation;
//  * resonance uses Slater overlaps from prolate spheroidal integrals;
//  * core-core: Z'_A Z'_B (ss|ss)(1 + e^{-a_A R} + e^{-a_B R}) + AM1 Gaussians.
//
// Derivatives: the whole map d -> (W, S, E) is evaluated once in dual
// numbers carrying d/dd_x, d/dd_y, d/dd_z (forward-mode differentiation), so
// forces (eq. 37) need no second pass over the integrals.
//
// Layout of the outputs (structure of arrays, stride = npair):
//   W[(p*10 + q) * npair + pair]   p: product on A, q: product on B
//   S[(mu*4 + lam) * npair + pair] <A mu | B lam>
//   E[pair]                        core-core energy
//   dW[(k*100 + p*10 + q) * npair + pair], dS[(k*16 + ..)], dE[k*npair + pair]
// Products: 0 ss, 1 sx, 2 sy, 3 sz, 4 xx, 5 yy, 6 zz, 7 xy, 8 xz, 9 yz.
#include <mutex>

#include "common.cuh"
#include "df.cuh"
#include "kernels.h"

namespace kx {

__constant__ double c_ovl_poly[2][2][3][3][5][5];   // [nA-1][nB-1][kindA][kindB][xi^i][eta^j]
__constant__ double c_ovl_phi[3];                    // phi factor per kindA (s, sigma, pi)

__device__ __constant__ int c_prod_mu[10] = {0, 0, 0, 0, 1, 2, 3, 1, 1, 2};
__device__ __constant__ int c_prod_nu[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
// reflection parity class (x -> -x, y -> -y) of each product: integrals
// between products of different classes vanish by symmetry
__device__ __constant__ int c_prod_cls[10] = {0, 1, 2, 0, 0, 0, 0, 3, 1, 2};
__device__ __constant__ int c_grp_lo[10] = {0, 1, 1, 1, 4, 4, 4, 4, 4, 4};
__device__ __constant__ int c_grp_hi[10] = {1, 4, 4, 4, 10, 10, 10, 10, 10, 10};

// point charges of product p on an atom (local frame), returns count
__device__ __forceinline__ int product_charges(int p, const Elem& e, double q[4], double x[4],
                                               double y[4], double z[4], double r[4]) {
  for (int i = 0; i < 4; ++i) { q[i] = 0.0; x[i] = 0.0; y[i] = 0.0; z[i] = 0.0; r[i] = e.rho0; }
  int a = c_prod_mu[p], b = c_prod_nu[p];
  if (a == 0 && b == 0) { q[0] = 1.0; r[0] = e.rho0; return 1; }
  if (a == 0) {
    double* c0 = (b == 1) ? x : (b == 2) ? y : z;
    q[0] = 0.5; c0[0] = e.D1; r[0] = e.rho1;
    q[1] = -0.5; c0[1] = -e.D1; r[1] = e.rho1;
    return 2;
  }
  if (a == b) {
    double* c0 = (a == 1) ? x : (a == 2) ? y : z;
    q[0] = 1.0; r[0] = e.rho0;
    q[1] = 0.25; c0[1] = 2.0 * e.D2; r[1] = e.rho2;
    q[2] = 0.25; c0[2] = -2.0 * e.D2; r[2] = e.rho2;
    q[3] = -0.5; r[3] = e.rho2;
    return 4;
  }
  double* ca = (a == 1) ? x : (a == 2) ? y : z;
  double* cb = (b == 1) ? x : (b == 2) ? y : z;
  const double sa[4] = {1.0, -1.0, 1.0, -1.0};
  const double sb[4] = {1.0, -1.0, -1.0, 1.0};
  for (int i = 0; i < 4; ++i) {
    q[i] = 0.25 * sa[i] * sb[i];
    ca[i] = sa[i] * e.D2;
    cb[i] = sb[i] * e.D2;
    r[i] = e.rho2;
  }
  return 4;
}

template <typename T>
__device__ T local_integral(int p, int qd, const Elem& ea, const Elem& eb, T R) {
  double qa[4], xa[4], ya[4], za[4], ra[4];
  double qb[4], xb[4], yb[4], zb[4], rb[4];
  int na = product_charges(p, ea, qa, xa, ya, za, ra);
  int nb = product_charges(qd, eb, qb, xb, yb, zb, rb);
  T acc = cst<T>(0.0);
  for (int i = 0; i < na; ++i) {
    for (int j = 0; j < nb; ++j) {
      double dx = xa[i] - xb[j], dy = ya[i] - yb[j], rr = ra[i] + rb[j];
      T dz = (za[i] - zb[j]) - R;
      T s2 = dz * dz + (dx * dx + dy * dy + rr * rr);
      acc += (qa[i] * qb[j]) * rsqrt_d(s2);
    }
  }
  return acc * kE2;
}

// A_k(p) = int_1^inf xi^k e^{-p xi}, k = 0..4
template <typename T>
__device__ void aux_A(T p, T* A) {
  T e = ex(-p);
  T ip = 1.0 / p;
  A[0] = e * ip;
#pragma unroll
  for (int k = 1; k < 5; ++k) A[k] = (e + (double)k * A[k - 1]) * ip;
}
// B_k(q) = int_{-1}^{1} eta^k e^{-q eta}, k = 0..4.  For |q| < 1 the series
// sum_m (-q)^m / m! int eta^(k+m) (the loops unroll, so the coefficients are
// compile-time constants); q = 0 (equal exponents) gives int eta^k directly.
template <typename T>
__device__ void aux_B(T q, T* B) {
  if (val(q) == 0.0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) B[k] = (k & 1) ? cst<T>(0.0) : cst<T>(2.0 / (double)(k + 1));
  } else if (fabs(val(q)) < 1.0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) B[k] = cst<T>(0.0);
    T term = cst<T>(1.0);
#pragma unroll
    for (int m = 0; m < 22; ++m) {
#pragma unroll
      for (int k = 0; k < 5; ++k)
        if (((k + m) & 1) == 0) B[k] += term * (2.0 / (double)(k + m + 1));
      term = term * (-q) * (1.0 / (double)(m + 1));
    }
  } else {
    T ep = ex(q), em = ex(-q);
    T iq = 1.0 / q;
    B[0] = (ep - em) * iq;
#pragma unroll
    for (int k = 1; k < 5; ++k) {
      T sgn_ep = (k & 1) ? -ep : ep;
      B[k] = (sgn_ep - em + (double)k * B[k - 1]) * iq;
    }
  }
}

// overlap of normalised Slater orbitals, B at +R z'; kinds 0 s, 1 sigma, 2 pi
template <typename T>
__device__ T sto_overlap(T R, int nA, double zA, double nrmA, int kA, int nB, double zB, double nrmB, int kB) {
  T Rb = R * (1.0 / kBohr);
  T p = Rb * (0.5 * (zA + zB));
  T q = Rb * (0.5 * (zA - zB));
  T A[5], B[5];
  aux_A(p, A);
  aux_B(q, B);
  T acc = cst<T>(0.0);
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      double c = c_ovl_poly[nA - 1][nB - 1][kA][kB][i][j];
      if (c != 0.0) acc += c * (A[i] * B[j]);
    }
  const double cs = 0.28209479177387814;  // 1/sqrt(4 pi)
  const double cp = 0.48860251190291992;  // sqrt(3/(4 pi))
  double pref = nrmA * nrmB * (kA == 0 ? cs : cp) * (kB == 0 ? cs : cp) * c_ovl_phi[kA];
  T half = Rb * 0.5;
  T pw = cst<T>(1.0);
  for (int k = 0; k < nA + nB + 1; ++k) pw = pw * half;
  return acc * pw * pref;
}

// independent variable k of the pair vector (derivative direction k)
template <typename T> __device__ __forceinline__ T seed(double v, int k);
template <> __device__ __forceinline__ double seed<double>(double v, int) { return v; }
template <> __device__ __forceinline__ D3 seed<D3>(double v, int k) {
  return D3{v, k == 0 ? 1.0 : 0.0, k == 1 ? 1.0 : 0.0, k == 2 ? 1.0 : 0.0};
}

// Quantities that depend on the distance R alone (local-frame integrals,
// local overlaps, core-core energy) are evaluated with one derivative,
// d/dR, and promoted to the pair-vector derivatives by the chain rule
// d/dd_k = u_k d/dR (u = d / R): a quarter of the dual-number work.
template <typename T> struct Radial;
template <> struct Radial<double> {
  typedef double type;
  __device__ static double seed(double R) { return R; }
  __device__ static double promote(double a, const double*) { return a; }
};
template <> struct Radial<D3> {
  typedef D1 type;
  __device__ static D1 seed(double R) { return D1{R, 1.0}; }
  __device__ static D3 promote(D1 a, const double* u) { return D3{a.v, a.d * u[0], a.d * u[1], a.d * u[2]}; }
};

// mirror image of an orbital product under x <-> y (a reflection that maps
// the local frame onto itself): sx <-> sy, xx <-> yy, xz <-> yz
__device__ __forceinline__ int mirror_xy(int p) {
  switch (p) {
    case 1: return 2;
    case 2: return 1;
    case 4: return 5;
    case 5: return 4;
    case 8: return 9;
    case 9: return 8;
    default: return p;
  }
}

// Double-float dual number with three derivative directions: the mixed
// path's rotation of the local blocks (C I C^T, eq. 6's two-centre integrals
// in the molecular frame) runs on the FP32 pipe in ~48-bit arithmetic instead
// of GB300's narrow FP64 pipe.
struct G3 {
  dfl v, d[3];
};
__device__ __forceinline__ G3 g3_zero() {
  return G3{{0.0f, 0.0f}, {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}}};
}
__device__ __forceinline__ G3 g3_of(const D3& a) {
  return G3{df_from_double(a.v), {df_from_double(a.d0), df_from_double(a.d1), df_from_double(a.d2)}};
}
__device__ __forceinline__ D3 d3_of(const G3& a) {
  return D3{df_to_double_fast(a.v), df_to_double_fast(a.d[0]), df_to_double_fast(a.d[1]), df_to_double_fast(a.d[2])};
}
__device__ __forceinline__ G3 g3_mul(const G3& a, const G3& b) {
  G3 r;
  r.v = df_mul(a.v, b.v);
#pragma unroll
  for (int k = 0; k < 3; ++k) r.d[k] = df_add(df_mul(a.d[k], b.v), df_mul(a.v, b.d[k]));
  return r;
}
__device__ __forceinline__ G3 g3_add(const G3& a, const G3& b) {
  G3 r;
  r.v = df_add(a.v, b.v);
#pragma unroll
  for (int k = 0; k < 3; ++k) r.d[k] = df_add(a.d[k], b.d[k]);
  return r;
}
// acc += a b, the low parts gathered without renormalisation (g3_norm after
// the last term)
__device__ __forceinline__ void g3_acc_mul(G3& acc, const G3& a, const G3& b) {
  df_acc_mul(acc.v, a.v, b.v);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    df_acc_mul(acc.d[k], a.d[k], b.v);
    df_acc_mul(acc.d[k], a.v, b.d[k]);
  }
}
__device__ __forceinline__ G3 g3_norm(const G3& a) {
  return G3{df_norm(a.v), {df_norm(a.d[0]), df_norm(a.d[1]), df_norm(a.d[2])}};
}

// Double-float radial dual number (value, d/dR) for the local integrals.
struct G1 {
  dfl v, d;
};
__device__ __forceinline__ G1 g1_zero() { return G1{{0.0f, 0.0f}, {0.0f, 0.0f}}; }
__device__ __forceinline__ G1 g1_sub(const G1& a, const G1& b) { return G1{df_sub(a.v, b.v), df_sub(a.d, b.d)}; }
__device__ __forceinline__ G1 g1_half(const G1& a) {
  return G1{{a.v.hi * 0.5f, a.v.lo * 0.5f}, {a.d.hi * 0.5f, a.d.lo * 0.5f}};
}
// a * q for a float q (exact product of the high part, one rounding of the low part)
__device__ __forceinline__ dfl df_mul_f(dfl a, float q) {
  const float p = KX_FMUL(a.hi, q);
  float e = KX_FFMA(a.hi, q, -p);
  e = KX_FFMA(a.lo, q, e);
  return df_fast_two_sum(p, e);
}
// 1/sqrt(s), s > 0: FP32 estimate y0 and one Newton step y0 + y0 (1 - s y0^2) / 2
// with s y0^2 in double-float (relative error ~(3/8) h^2, h = 1 - s y0^2 ~ 1e-7)
__device__ __forceinline__ dfl df_rsqrt(dfl s) {
  const float y0 = rsqrtf(s.hi);
  const float p = KX_FMUL(y0, y0);
  const dfl y2 = dfl{p, KX_FFMA(y0, y0, -p)};
  const dfl t = df_mul(s, y2);
  const float h = KX_FSUB(KX_FSUB(1.0f, t.hi), t.lo);
  return df_fast_two_sum(y0, KX_FMUL(KX_FMUL(y0, h), 0.5f));
}

// point-charge multipole lengths of one element in double-float
struct ChargeDF {
  dfl D1, D2, rho0, rho1, rho2;
};
__device__ __forceinline__ ChargeDF charge_df(const Elem& e) {
  return ChargeDF{df_from_double(e.D1), df_from_double(e.D2), df_from_double(e.rho0), df_from_double(e.rho1),
                  df_from_double(e.rho2)};
}
__device__ __forceinline__ dfl df_twice(dfl a) { return dfl{a.hi * 2.0f, a.lo * 2.0f}; }

// the charge sets of product_charges, positions and radii in double-float
// (the charges themselves, 1, +-1/2 and +-1/4, are exact in FP32)
__device__ __forceinline__ int product_charges_df(int p, const ChargeDF& c, float q[4], dfl x[4], dfl y[4],
                                                  dfl z[4], dfl r[4]) {
  const dfl zero = {0.0f, 0.0f};
  for (int i = 0; i < 4; ++i) { q[i] = 0.0f; x[i] = zero; y[i] = zero; z[i] = zero; r[i] = c.rho0; }
  const int a = c_prod_mu[p], b = c_prod_nu[p];
  if (a == 0 && b == 0) { q[0] = 1.0f; r[0] = c.rho0; return 1; }
  if (a == 0) {
    dfl* c0 = (b == 1) ? x : (b == 2) ? y : z;
    q[0] = 0.5f; c0[0] = c.D1; r[0] = c.rho1;
    q[1] = -0.5f; c0[1] = df_neg(c.D1); r[1] = c.rho1;
    return 2;
  }
  if (a == b) {
    dfl* c0 = (a == 1) ? x : (a == 2) ? y : z;
    q[0] = 1.0f; r[0] = c.rho0;
    q[1] = 0.25f; c0[1] = df_twice(c.D2); r[1] = c.rho2;
    q[2] = 0.25f; c0[2] = df_neg(df_twice(c.D2)); r[2] = c.rho2;
    q[3] = -0.5f; r[3] = c.rho2;
    return 4;
  }
  dfl* ca = (a == 1) ? x : (a == 2) ? y : z;
  dfl* cb = (b == 1) ? x : (b == 2) ? y : z;
  const float sa[4] = {1.0f, -1.0f, 1.0f, -1.0f};
  const float sb[4] = {1.0f, -1.0f, -1.0f, 1.0f};
  for (int i = 0; i < 4; ++i) {
    q[i] = 0.25f * sa[i] * sb[i];
    ca[i] = (sa[i] > 0.0f) ? c.D2 : df_neg(c.D2);
    cb[i] = (sb[i] > 0.0f) ? c.D2 : df_neg(c.D2);
    r[i] = c.rho2;
  }
  return 4;
}

// local_integral in double-float with d/dR: sum of q_i q_j / sqrt(dz^2 + dx^2
// + dy^2 + (rho_i + rho_j)^2), dz = z_i - z_j - R, whose R-derivative is
// q_i q_j dz / s^3; times e^2 (e2 in double-float)
__device__ G1 local_integral_df(int p, int qd, const ChargeDF& ca, const ChargeDF& cb, dfl R, dfl e2) {
  float qa[4], qb[4];
  dfl xa[4], ya[4], za[4], ra[4], xb[4], yb[4], zb[4], rb[4];
  const int na = product_charges_df(p, ca, qa, xa, ya, za, ra);
  const int nb = product_charges_df(qd, cb, qb, xb, yb, zb, rb);
  dfl v = {0.0f, 0.0f}, dv = {0.0f, 0.0f};
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j) {
      const dfl dx = df_sub(xa[i], xb[j]), dy = df_sub(ya[i], yb[j]), rr = df_add(ra[i], rb[j]);
      const dfl dz = df_sub(df_sub(za[i], zb[j]), R);
      dfl s2 = df_mul(dz, dz);
      s2 = df_add(s2, df_mul(dx, dx));
      s2 = df_add(s2, df_mul(dy, dy));
      s2 = df_add(s2, df_mul(rr, rr));
      const dfl r = df_rsqrt(s2);
      const dfl r3dz = df_mul(df_mul(df_mul(r, r), r), dz);
      const float qq = qa[i] * qb[j];
      df_acc(v, df_mul_f(r, qq));
      df_acc(dv, df_mul_f(r3dz, qq));
    }
  return G1{df_mul(df_norm(v), e2), df_mul(df_norm(dv), e2)};
}

// W = C I C^T in double-float from the local integrals as radial duals
// (value, d/dR): promoted by d/dd_k = u_k d/dR, rotated, written as D3
// the products of one group (ss, sp, pp) and the group of product p
__device__ __forceinline__ int grp_of(int p) { return p == 0 ? 0 : (p < 4 ? 1 : 2); }
__device__ __forceinline__ int grp_lo(int g) { return g == 0 ? 0 : (g == 1 ? 1 : 4); }
__device__ __forceinline__ int grp_hi(int g) { return g == 0 ? 1 : (g == 1 ? 4 : 10); }

// W = C I C^T in double-float from the local integrals as radial duals
// (value, d/dR), written straight to the pair's output columns (W[(p*10+q)*np],
// dW[(k*100 + p*10+q)*np]).  The molecular-frame derivatives of I are u_k dI/dR,
// so X = I C^T needs no promoted copy of I:
//   X.v = sum I.v C.v,   X.d_k = sum I.v C.d_k + u_k sum I.d C.v;
// C is kept block by block (at most 6 products per row) and X one product
// group at a time, which keeps the per-thread arrays small.
__device__ void rotate_blocks_df(const G1 (&Ir)[10][10], const D3 (&Tf)[4][4], const double* uv, int pa, int pb,
                                 double* __restrict__ W, double* __restrict__ dW, size_t np, int t) {
  G3 Tg[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) Tg[a][b] = g3_zero();
  Tg[0][0].v = dfl{1.0f, 0.0f};
#pragma unroll
  for (int a = 1; a < 4; ++a)
#pragma unroll
    for (int b = 1; b < 4; ++b) Tg[a][b] = g3_of(Tf[a][b]);
  const dfl ug[3] = {df_from_double(uv[0]), df_from_double(uv[1]), df_from_double(uv[2])};
  // C[p][pp] for pp in the group of p, at Cb[p][pp - grp_lo]
  G3 Cb[10][6];
  for (int p = 0; p < 10; ++p) {
    const int mu = c_prod_mu[p], nu = c_prod_nu[p];
    const int g = grp_of(p), lo = grp_lo(g);
    for (int pp = lo; pp < grp_hi(g); ++pp) {
      const int m2 = c_prod_mu[pp], n2 = c_prod_nu[pp];
      if (m2 == n2)
        Cb[p][pp - lo] = g3_mul(Tg[mu][m2], Tg[nu][m2]);
      else
        Cb[p][pp - lo] = g3_add(g3_mul(Tg[mu][m2], Tg[nu][n2]), g3_mul(Tg[mu][n2], Tg[nu][m2]));
    }
  }
  const int ngrp = (pa == 10) ? 3 : 1;
  for (int g = 0; g < ngrp; ++g) {
    const int lo = grp_lo(g), hi = grp_hi(g);
    G3 Xg[6][10];                       // X[pp][q] for pp in group g
    for (int pp = lo; pp < hi; ++pp)
      for (int q = 0; q < pb; ++q) {
        G3 acc = g3_zero();
        dfl sd = {0.0f, 0.0f};
        const int gq = grp_of(q), qlo = grp_lo(gq);
        for (int qq = qlo; qq < grp_hi(gq); ++qq) {
          if (c_prod_cls[qq] != c_prod_cls[pp]) continue;          // I = 0 between classes
          const G1& iv = Ir[pp][qq];
          const G3& c = Cb[q][qq - qlo];
          df_acc_mul(acc.v, iv.v, c.v);
#pragma unroll
          for (int k = 0; k < 3; ++k) df_acc_mul(acc.d[k], iv.v, c.d[k]);
          df_acc_mul(sd, iv.d, c.v);
        }
        sd = df_norm(sd);
        G3 x = g3_norm(acc);
#pragma unroll
        for (int k = 0; k < 3; ++k) x.d[k] = df_add(x.d[k], df_mul(ug[k], sd));
        Xg[pp - lo][q] = x;
      }
    for (int p = lo; p < hi; ++p)
      for (int q = 0; q < 10; ++q) {
        G3 acc = g3_zero();
        if (q < pb)
          for (int pp = lo; pp < hi; ++pp) g3_acc_mul(acc, Cb[p][pp - lo], Xg[pp - lo][q]);
        const D3 w = d3_of(g3_norm(acc));
        const size_t ix = (size_t)(p * 10 + q) * np + t;
        W[ix] = w.v;
        dW[ix] = w.d0;
        dW[100 * np + ix] = w.d1;
        dW[200 * np + ix] = w.d2;
      }
  }
  // products the partner's group structure leaves out (hydrogen on A: p >= 1)
  for (int p = (ngrp == 1 ? 1 : 10); p < 10; ++p)
    for (int q = 0; q < 10; ++q) {
      const size_t ix = (size_t)(p * 10 + q) * np + t;
      W[ix] = 0.0;
      dW[ix] = 0.0;
      dW[100 * np + ix] = 0.0;
      dW[200 * np + ix] = 0.0;
    }
}

// DFROT (dual numbers only): W and dW go straight to Wg / dWg (column t of
// stride np) and Wout is not used
template <bool DFROT, typename T>
__device__ void pair_block(const double* dvec, const Elem& ea, const Elem& eb, T* Wout /*100*/,
                           T* Sout /*16*/, T* Eout, double* Wg = nullptr, double* dWg = nullptr, size_t np = 0,
                           int t = 0) {
  typedef typename Radial<T>::type Tr;
  T d[3];
  for (int k = 0; k < 3; ++k) d[k] = seed<T>(dvec[k], k);
  T R = sq(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  T iR = 1.0 / R;
  T u[3] = {d[0] * iR, d[1] * iR, d[2] * iR};
  const double uv[3] = {val(u[0]), val(u[1]), val(u[2])};
  const Tr Rr = Radial<T>::seed(val(R));
  // reference axis least aligned with u
  int ref = 0;
  double best = fabs(val(u[0]));
  if (fabs(val(u[1])) < best) { ref = 1; best = fabs(val(u[1])); }
  if (fabs(val(u[2])) < best) { ref = 2; }
  T au = u[ref];
  T nrm = rsqrt_d(1.0 - au * au);
  T fx[3], fy[3];   // local x' and y' axes
  for (int k = 0; k < 3; ++k) fx[k] = ((k == ref ? cst<T>(1.0) : cst<T>(0.0)) - au * u[k]) * nrm;
  fy[0] = u[1] * fx[2] - u[2] * fx[1];
  fy[1] = u[2] * fx[0] - u[0] * fx[2];
  fy[2] = u[0] * fx[1] - u[1] * fx[0];
  // Tf[mu][mu']: molecular orbital slot mu in terms of local slot mu'
  T Tf[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) Tf[a][b] = cst<T>(0.0);
  Tf[0][0] = cst<T>(1.0);
  for (int k = 0; k < 3; ++k) {
    Tf[1 + k][1] = fx[k];
    Tf[1 + k][2] = fy[k];
    Tf[1 + k][3] = u[k];
  }

  const int pa = (ea.norb == 4) ? 10 : 1;
  const int pb = (eb.norb == 4) ? 10 : 1;

  // local integrals: the distinct ones (rows ss, sz, xx, zz of the sigma/
  // delta class, sx and xz of the pi class) from the charge sets, the rest by
  // the x <-> y mirror and the rotational-invariance relation for (xy|xy)
  if constexpr (DFROT) {
    // local integrals and the rotation in double-float (mixed path)
    const ChargeDF ca = charge_df(ea), cb = charge_df(eb);
    const dfl Rd = df_from_double(val(R)), e2 = df_from_double(kE2);
    G1 Ig[10][10];
    for (int p = 0; p < 10; ++p)
      for (int q = 0; q < 10; ++q) Ig[p][q] = g1_zero();
    for (int p = 0; p < pa; ++p) {
      if (p == 2 || p == 5 || p == 7 || p == 9) continue;        // mirrored or derived below
      for (int q = 0; q < pb; ++q) {
        if (c_prod_cls[p] != c_prod_cls[q]) continue;
        if (c_prod_cls[p] == 1 && (q == 2 || q == 9)) continue;
        Ig[p][q] = local_integral_df(p, q, ca, cb, Rd, e2);
      }
    }
    if (pa == 10) {
      for (int q = 0; q < pb; ++q) {
        const int mq = mirror_xy(q);
        if (c_prod_cls[q] == 0) Ig[5][q] = Ig[4][mq];
        if (c_prod_cls[q] == 2) { Ig[2][q] = Ig[1][mq]; Ig[9][q] = Ig[8][mq]; }
      }
      if (pb == 10) Ig[7][7] = g1_half(g1_sub(Ig[4][4], Ig[4][5]));
    }
    rotate_blocks_df(Ig, Tf, uv, pa, pb, Wg, dWg, np, t);
  } else {
  Tr Ir[10][10];
  for (int p = 0; p < 10; ++p)
    for (int q = 0; q < 10; ++q) Ir[p][q] = cst<Tr>(0.0);
  for (int p = 0; p < pa; ++p) {
    if (p == 2 || p == 5 || p == 7 || p == 9) continue;        // mirrored or derived below
    for (int q = 0; q < pb; ++q) {
      if (c_prod_cls[p] != c_prod_cls[q]) continue;
      if (c_prod_cls[p] == 1 && (q == 2 || q == 9)) continue;
      Ir[p][q] = local_integral<Tr>(p, q, ea, eb, Rr);
    }
  }
  if (pa == 10) {
    for (int q = 0; q < pb; ++q) {
      const int mq = mirror_xy(q);
      if (c_prod_cls[q] == 0) Ir[5][q] = Ir[4][mq];
      if (c_prod_cls[q] == 2) { Ir[2][q] = Ir[1][mq]; Ir[9][q] = Ir[8][mq]; }
    }
    if (pb == 10) Ir[7][7] = 0.5 * (Ir[4][4] - Ir[4][5]);
  }

  T I[10][10];
  for (int p = 0; p < 10; ++p)
    for (int q = 0; q < 10; ++q)
      I[p][q] = (c_prod_cls[p] == c_prod_cls[q]) ? Radial<T>::promote(Ir[p][q], uv) : cst<T>(0.0);
  // product transform C[p][p'] (block diagonal over ss / sp / pp groups)
  T C[10][10];
  for (int p = 0; p < 10; ++p) {
    int mu = c_prod_mu[p], nu = c_prod_nu[p];
    for (int pp = c_grp_lo[p]; pp < c_grp_hi[p]; ++pp) {
      int m2 = c_prod_mu[pp], n2 = c_prod_nu[pp];
      if (m2 == n2)
        C[p][pp] = Tf[mu][m2] * Tf[nu][m2];
      else
        C[p][pp] = Tf[mu][m2] * Tf[nu][n2] + Tf[mu][n2] * Tf[nu][m2];
    }
  }
  // X[p'][q] = sum_{q'} I[p'][q'] C[q][q'];  W[p][q] = sum_{p'} C[p][p'] X[p'][q]
  T X[10][10];
  for (int pp = 0; pp < pa; ++pp)
    for (int q = 0; q < pb; ++q) {
      T acc = cst<T>(0.0);
      for (int qq = c_grp_lo[q]; qq < c_grp_hi[q]; ++qq)
        if (c_prod_cls[qq] == c_prod_cls[pp]) acc += I[pp][qq] * C[q][qq];   // other classes: I = 0
      X[pp][q] = acc;
    }
  for (int p = 0; p < 10; ++p)
    for (int q = 0; q < 10; ++q) {
      T acc = cst<T>(0.0);
      if (p < pa && q < pb)
        for (int pp = c_grp_lo[p]; pp < c_grp_hi[p]; ++pp) acc += C[p][pp] * X[pp][q];
      Wout[p * 10 + q] = acc;
    }
  }

  // overlaps in the local frame (functions of R), then in the molecular frame.
  // The local p_x', p_y' overlaps are equal (pi) and the frame (x', y', u) is
  // orthonormal, so x'_a x'_b + y'_a y'_b = delta_ab - u_a u_b and
  //   S_ss = s, S_s,pb = (s|sigma) u_b, S_pa,s = (sigma|s) u_a,
  //   S_pa,pb = pi delta_ab + (sigma - pi) u_a u_b:
  // the molecular-frame overlaps depend on u alone (no x', y').
  const T zero = cst<T>(0.0);
  for (int k = 0; k < 16; ++k) Sout[k] = zero;
  Sout[0] = Radial<T>::promote(
      sto_overlap<Tr>(Rr, ea.nprin, ea.zeta[0], ea.sto_nrm[0], 0, eb.nprin, eb.zeta[0], eb.sto_nrm[0], 0), uv);
  if (ea.norb == 4) {
    const T szs = Radial<T>::promote(
        sto_overlap<Tr>(Rr, ea.nprin, ea.zeta[1], ea.sto_nrm[1], 1, eb.nprin, eb.zeta[0], eb.sto_nrm[0], 0), uv);
    for (int a = 1; a < 4; ++a) Sout[a * 4] = szs * u[a - 1];
  }
  if (eb.norb == 4) {
    const T ssz = Radial<T>::promote(
        sto_overlap<Tr>(Rr, ea.nprin, ea.zeta[0], ea.sto_nrm[0], 0, eb.nprin, eb.zeta[1], eb.sto_nrm[1], 1), uv);
    for (int b = 1; b < 4; ++b) Sout[b] = ssz * u[b - 1];
  }
  if (ea.norb == 4 && eb.norb == 4) {
    const T szz = Radial<T>::promote(
        sto_overlap<Tr>(Rr, ea.nprin, ea.zeta[1], ea.sto_nrm[1], 1, eb.nprin, eb.zeta[1], eb.sto_nrm[1], 1), uv);
    const T spp = Radial<T>::promote(
        sto_overlap<Tr>(Rr, ea.nprin, ea.zeta[1], ea.sto_nrm[1], 2, eb.nprin, eb.zeta[1], eb.sto_nrm[1], 2), uv);
    const T dsp = szz - spp;
    for (int a = 1; a < 4; ++a) {
      const T da = dsp * u[a - 1];
      for (int b = 1; b < 4; ++b) Sout[a * 4 + b] = (a == b) ? da * u[b - 1] + spp : da * u[b - 1];
    }
  }

  // core-core repulsion (a function of R)
  const Tr gss = local_integral<Tr>(0, 0, ea, eb, Rr);
  const double zz = ea.zcore * eb.zcore;
  Tr en = zz * gss * (1.0 + ex(-ea.alpha * Rr) + ex(-eb.alpha * Rr));
  Tr g = cst<Tr>(0.0);
  for (int k = 0; k < 2; ++k) {
    Tr ta = Rr - ea.gc[k];
    Tr tb = Rr - eb.gc[k];
    g += ea.ga[k] * ex(-ea.gb[k] * (ta * ta)) + eb.ga[k] * ex(-eb.gb[k] * (tb * tb));
  }
  *Eout = Radial<T>::promote(en + zz * g / Rr, uv);
}

__global__ void pair_values_kernel(int npair, const int* __restrict__ pA, const int* __restrict__ pB,
                                   const int* __restrict__ elem, const double* __restrict__ R,
                                   ElemTable tab, double* __restrict__ W, double* __restrict__ S,
                                   double* __restrict__ E) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npair) return;
  int A = pA[t], B = pB[t];
  double d[3] = {R[3 * B] - R[3 * A], R[3 * B + 1] - R[3 * A + 1], R[3 * B + 2] - R[3 * A + 2]};
  const Elem& ea = tab.e[elem[A]];
  const Elem& eb = tab.e[elem[B]];
  double w[100], s[16], e;
  pair_block<false, double>(d, ea, eb, w, s, &e);
  for (int k = 0; k < 100; ++k) W[(size_t)k * npair + t] = w[k];
  for (int k = 0; k < 16; ++k) S[(size_t)k * npair + t] = s[k];
  E[t] = e;
}

template <bool DFROT>
__global__ void pair_derivs_kernel(int npair, const int* __restrict__ pA, const int* __restrict__ pB,
                                   const int* __restrict__ elem, const double* __restrict__ R,
                                   ElemTable tab, double* __restrict__ W, double* __restrict__ S,
                                   double* __restrict__ E, double* __restrict__ dW,
                                   double* __restrict__ dS, double* __restrict__ dE) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npair) return;
  int A = pA[t], B = pB[t];
  double d[3] = {R[3 * B] - R[3 * A], R[3 * B + 1] - R[3 * A + 1], R[3 * B + 2] - R[3 * A + 2]};
  const Elem& ea = tab.e[elem[A]];
  const Elem& eb = tab.e[elem[B]];
  size_t np = (size_t)npair;
  D3 s[16], e;
  if constexpr (DFROT) {
    pair_block<true, D3>(d, ea, eb, nullptr, s, &e, W, dW, np, t);
  } else {
    D3 w[100];
    pair_block<false, D3>(d, ea, eb, w, s, &e);
    for (int k = 0; k < 100; ++k) {
      W[k * np + t] = w[k].v;
      dW[(0 * 100 + k) * np + t] = w[k].d0;
      dW[(1 * 100 + k) * np + t] = w[k].d1;
      dW[(2 * 100 + k) * np + t] = w[k].d2;
    }
  }
  for (int k = 0; k < 16; ++k) {
    S[k * np + t] = s[k].v;
    dS[(0 * 16 + k) * np + t] = s[k].d0;
    dS[(1 * 16 + k) * np + t] = s[k].d1;
    dS[(2 * 16 + k) * np + t] = s[k].d2;
  }
  E[t] = e.v;
  dE[0 * np + t] = e.d0;
  dE[1 * np + t] = e.d1;
  dE[2 * np + t] = e.d2;
}

// ---------------------------------------------------------------------------
// host side: overlap polynomial tables (built and uploaded once per device)
// ---------------------------------------------------------------------------
namespace {
struct Poly {
  double c[9][9];
  Poly() { for (auto& r : c) for (auto& x : r) x = 0.0; }
};
Poly pmul(const Poly& a, const Poly& b) {
  Poly o;
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j)
      if (a.c[i][j] != 0.0)
        for (int k = 0; i + k < 9; ++k)
          for (int l = 0; j + l < 9; ++l) o.c[i + k][j + l] += a.c[i][j] * b.c[k][l];
  return o;
}
Poly mono(double c00, double c10, double c01, double c11, double c20, double c02) {
  Poly p;
  p.c[0][0] = c00; p.c[1][0] = c10; p.c[0][1] = c01; p.c[1][1] = c11; p.c[2][0] = c20; p.c[0][2] = c02;
  return p;
}
Poly ppow(const Poly& a, int k) {
  Poly o = mono(1, 0, 0, 0, 0, 0);
  for (int i = 0; i < k; ++i) o = pmul(o, a);
  return o;
}
}  // namespace

static bool upload_overlap_tables_once() {
  double tab[2][2][3][3][5][5] = {};
  const Poly vol = mono(0, 0, 0, 0, 1, -1);          // xi^2 - eta^2
  const Poly rA = mono(0, 1, 1, 0, 0, 0);            // xi + eta
  const Poly rB = mono(0, 1, -1, 0, 0, 0);           // xi - eta
  const Poly zA = mono(1, 0, 0, 1, 0, 0);            // 1 + xi eta
  const Poly zB = mono(-1, 0, 0, 1, 0, 0);           // xi eta - 1
  const Poly perp = pmul(mono(-1, 0, 0, 0, 1, 0), mono(1, 0, 0, 0, 0, -1));  // (xi^2-1)(1-eta^2)
  for (int nA = 1; nA <= 2; ++nA)
    for (int nB = 1; nB <= 2; ++nB)
      for (int kA = 0; kA < 3; ++kA)
        for (int kB = 0; kB < 3; ++kB) {
          if ((kA > 0 && nA < 2) || (kB > 0 && nB < 2)) continue;
          if ((kA == 2) != (kB == 2)) continue;
          Poly p;
          if (kA == 2) {
            p = pmul(pmul(pmul(vol, ppow(rA, nA - 2)), ppow(rB, nB - 2)), perp);
          } else {
            Poly a = (kA == 0) ? ppow(rA, nA - 1) : pmul(ppow(rA, nA - 2), zA);
            Poly b = (kB == 0) ? ppow(rB, nB - 1) : pmul(ppow(rB, nB - 2), zB);
            p = pmul(pmul(vol, a), b);
          }
          for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) {
              if (p.c[i][j] == 0.0) continue;
              if (i >= 5 || j >= 5) return false;  // degree bound violated
              tab[nA - 1][nB - 1][kA][kB][i][j] = p.c[i][j];
            }
        }
  const double phi[3] = {2.0 * M_PI, 2.0 * M_PI, M_PI};
  if (cudaMemcpyToSymbol(c_ovl_poly, tab, sizeof(tab)) != cudaSuccess) return false;
  if (cudaMemcpyToSymbol(c_ovl_phi, phi, sizeof(phi)) != cudaSuccess) return false;
  return true;
}

// __constant__ memory is per device: upload on every device the library runs on
bool upload_overlap_tables() {
  static PerDeviceOnce flag;
  return once_per_device(flag, [] { return upload_overlap_tables_once(); });
}

void launch_pair_values(cudaStream_t s, int npair, const int* pA, const int* pB, const int* elem,
                        const double* R, const ElemTable& tab, double* W, double* S, double* E) {
  if (npair <= 0) return;
  pair_values_kernel<<<(npair + 127) / 128, 128, 0, s>>>(npair, pA, pB, elem, R, tab, W, S, E);
  count_launch();
}

void launch_pair_derivs(cudaStream_t s, int npair, const int* pA, const int* pB, const int* elem,
                        const double* R, const ElemTable& tab, double* W, double* S, double* E,
                        double* dW, double* dS, double* dE, bool df_rotation) {
  if (npair <= 0) return;
  if (df_rotation)
    pair_derivs_kernel<true><<<(npair + 127) / 128, 128, 0, s>>>(npair, pA, pB, elem, R, tab, W, S, E, dW, dS, dE);
  else
    pair_derivs_kernel<false><<<(npair + 127) / 128, 128, 0, s>>>(npair, pA, pB, elem, R, tab, W, S, E, dW, dS, dE);
  count_launch();
}

}  // namespace kx
