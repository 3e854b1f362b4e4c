// Fermi occupations and chemical potential (eqs. 7, 8), entropy (eq. 4),
// the element-wise step of the DMPT response (eq. 36), energies (eq. 13),
// Krylov kernel pieces (eqs. 31-34), the X update (eq. 35) and the nuclear
// velocity Verlet pieces (eqs. 27, 28, 30).
//
// Every reduction runs in a fixed order (per-block tree, then a single block
// over the partials), so results do not depend on scheduling.
#include <cstring>

#include "common.cuh"
#include "df.cuh"
#include "kernels.h"

namespace kx {

constexpr int kRedThreads = 256;
constexpr int kMaxDots = 24;

__device__ __forceinline__ double fermi_occ(double eps, double mu, double beta) {
  return 0.5 * (1.0 - tanh(0.5 * beta * (eps - mu)));
}

// ---- chemical potential and occupations (one block) -------------------------
// block-wide FP32 sum in a fixed order; every thread gets the total
__device__ __forceinline__ float block_sum_f(float v, float* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  float t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0f;
  if (wid == 0)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  const float r = scratch[0];
  __syncthreads();
  return r;
}

// mu (eq. 8): bisection on sum_i f_i = N_occ to 1e-15 relative, as before, but
// (1) a coarse FP32 bisection (eigenvalues staged in shared memory) shrinks the
// bracket first, and (2) the FP64 sums run over the window of eigenvalues within
// 40/beta of the bracket only: outside it every f_i is exactly 0 or 1 in FP64,
// so the window sum plus the count below it is the full sum.  GB300's FP64
// pipe is narrow; the full FP64 bisection took some fifty passes over n.
constexpr int kFermiSmemMax = 11264;     // eigenvalues staged in shared memory (larger n: global)

// number of eigenvalues below x (eps ascending); every thread gets it
__device__ int count_below(int n, const double* __restrict__ eps, double x, double* red) {
  double c = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) c += (eps[i] < x) ? 1.0 : 0.0;
  return (int)block_sum(c, red);
}
// i0 + sum_{i0 <= i < i1} f_i(mu)
__device__ double window_sum(const double* __restrict__ eps, int i0, int i1, double mu, double beta, double* red) {
  double loc = 0.0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) loc += fermi_occ(eps[i], mu, beta);
  return (double)i0 + block_sum(loc, red);
}

__global__ void fermi_kernel(int n, const double* __restrict__ eps, double nocc, double beta,
                             double* __restrict__ f, Scalars* sc) {
  __shared__ double red[32];
  __shared__ float redf[32];
  __shared__ float e32[kFermiSmemMax];
  const bool staged = n <= kFermiSmemMax;
  if (staged)
    for (int i = threadIdx.x; i < n; i += blockDim.x) e32[i] = (float)eps[i];
  __syncthreads();
  const double glo = eps[0] - 40.0 / beta, ghi = eps[n - 1] + 40.0 / beta;
  float lo32 = (float)glo, hi32 = (float)ghi;
  const float b32 = (float)beta, nocc32 = (float)nocc;
  for (int it = 0; it < 80; ++it) {
    const float mid = 0.5f * (lo32 + hi32);
    if (mid <= lo32 || mid >= hi32) break;
    float loc = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float ei = staged ? e32[i] : (float)eps[i];
      loc += 1.0f / (1.0f + __expf(b32 * (ei - mid)));
    }
    const float s = block_sum_f(loc, redf);
    if (s > nocc32) hi32 = mid; else lo32 = mid;
  }
  // FP64 bracket around the FP32 one, widened until it brackets the FP64 root
  double w = 8.0 * ((double)hi32 - (double)lo32) + 1e-12 * fmax(1.0, fabs((double)lo32));
  double lo = fmax(glo, (double)lo32 - w), hi = fmin(ghi, (double)hi32 + w);
  int i0 = 0, i1 = n;
  for (int k = 0; k < 64; ++k) {
    i0 = count_below(n, eps, lo - 40.0 / beta, red);
    i1 = count_below(n, eps, hi + 40.0 / beta, red);
    const bool ok_lo = (lo <= glo) || window_sum(eps, i0, i1, lo, beta, red) <= nocc;
    const bool ok_hi = (hi >= ghi) || window_sum(eps, i0, i1, hi, beta, red) > nocc;
    if (ok_lo && ok_hi) break;
    w *= 4.0;
    if (!ok_lo) lo = fmax(glo, lo - w);
    if (!ok_hi) hi = fmin(ghi, hi + w);
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (window_sum(eps, i0, i1, mid, beta, red) > nocc) hi = mid; else lo = mid;
    if (hi - lo < 1e-15 * fmax(1.0, fabs(mid))) break;
  }
  double mu = 0.5 * (lo + hi);
  for (int it = 0; it < 3; ++it) {
    double l1 = 0.0, l2 = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      double fi = fermi_occ(eps[i], mu, beta);
      l1 += fi;
      l2 += fi * (1.0 - fi);
    }
    double s = (double)i0 + block_sum(l1, red);
    double dn = beta * block_sum(l2, red);
    if (dn < 1e-300) break;
    double step = (nocc - s) / dn;
    if (!isfinite(step) || fabs(step) > 1.0 / beta) break;
    mu += step;
  }
  double ls = 0.0, ll = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double fi = (i < i0) ? 1.0 : (i >= i1) ? 0.0 : fermi_occ(eps[i], mu, beta);
    f[i] = fi;
    if (fi > 0.0 && fi < 1.0) ls += fi * log(fi) + (1.0 - fi) * log(1.0 - fi);
    ll += -beta * fi * (1.0 - fi);
  }
  double S = -kBoltz * block_sum(ls, red);
  double sl = block_sum(ll, red);
  if (threadIdx.x == 0) {
    sc->mu = mu;
    sc->entropy = S;
    sc->sum_lam = sl;
    int no = (int)(nocc + 0.5);
    sc->gap = (no >= 1 && no < n) ? eps[no] - eps[no - 1] : 0.0;
  }
}

void launch_fermi(cudaStream_t s, int n, const double* eps, double nocc, double beta, double* f,
                  Scalars* sc) {
  fermi_kernel<<<1, 1024, 0, s>>>(n, eps, nocc, beta, f, sc);
  count_launch();
}

// Qs = Q diag(f^1/2); each thread owns one column and 64 rows, so the square
// root is taken once per column tile rather than once per element
constexpr int kScaleRows = 64;
__global__ void scale_columns_kernel(int n, const double* __restrict__ Q, const double* __restrict__ f,
                                     double* __restrict__ Qs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double sq = ::sqrt(fmax(f[j], 0.0));
  const int r0 = blockIdx.y * kScaleRows;
  const int r1 = (r0 + kScaleRows < n) ? r0 + kScaleRows : n;
  for (int r = r0; r < r1; ++r) Qs[(size_t)r * n + j] = Q[(size_t)r * n + j] * sq;
}

void launch_scale_columns(cudaStream_t s, int n, const double* Q, const double* f, double* Qs) {
  dim3 grid((n + 255) / 256, (n + kScaleRows - 1) / kScaleRows);
  scale_columns_kernel<<<grid, 256, 0, s>>>(n, Q, f, Qs);
  count_launch();
}

__global__ void transpose_kernel(int n, const double* __restrict__ A, double* __restrict__ At) {
  __shared__ double tile[32][33];
  int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = i0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < n && j < n) ? A[(size_t)i * n + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int j = j0 + r, i = i0 + threadIdx.x;
    if (i < n && j < n) At[(size_t)j * n + i] = tile[threadIdx.x][r];
  }
}

void launch_transpose(cudaStream_t s, int n, const double* A, double* At) {
  int t = (n + 31) / 32;
  transpose_kernel<<<dim3(t, t), dim3(32, 8), 0, s>>>(n, A, At);
  count_launch();
}

// ---- DMPT (eq. 36) -------------------------------------------------------------
__device__ __forceinline__ double lambda_ij(double ei, double ej, double fi, double fj, double mu,
                                            double beta) {
  double de = ei - ej;
  if (beta * fabs(de) < 1e-5) {
    double fm = fermi_occ(0.5 * (ei + ej), mu, beta);
    return -beta * fm * (1.0 - fm);
  }
  return (fi - fj) / de;
}

__global__ void dmu_kernel(int n, const double* __restrict__ F1p, const double* __restrict__ eps,
                           const double* __restrict__ f, double beta, Scalars* sc) {
  __shared__ double red[32];
  if (!sc->active) return;
  double mu = sc->mu;
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double l = lambda_ij(eps[i], eps[i], f[i], f[i], mu, beta);
    num += l * F1p[(size_t)i * n + i];
    den += l;
  }
  num = block_sum(num, red);
  den = block_sum(den, red);
  if (threadIdx.x == 0) sc->dmu = (fabs(den) > 1e-300) ? num / den : 0.0;
}

void launch_dmu(cudaStream_t s, int n, const double* F1p, const double* eps, const double* f, double beta,
                Scalars* sc) {
  dmu_kernel<<<1, 1024, 0, s>>>(n, F1p, eps, f, beta, sc);
  count_launch();
}

// Lambda_ij of eq. 36 for the current eigenpairs (the same for every Krylov
// vector of one evaluation); one row of tiles per blockIdx.y
__global__ void lambda_kernel(int n, const double* __restrict__ eps, const double* __restrict__ f, double beta,
                              const Scalars* sc, double* __restrict__ Lam) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  Lam[(size_t)i * n + j] = lambda_ij(eps[i], eps[j], f[i], f[j], sc->mu, beta);
}

// Mixed path: the divided difference (f_i - f_j) / (e_i - e_j) in double-float
// (an FP64 division is a long FP64 sequence on GB300: 305 -> 87 us per n = 3360
// matrix); pairs within 1e-5 / beta take the derivative of the Fermi function in
// FP64 as above (the test on the FP32 part of e_i - e_j).
__global__ void lambda_df_kernel(int n, const double* __restrict__ eps, const double* __restrict__ f, double beta,
                                 float betaf, const Scalars* sc, double* __restrict__ Lam) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const dfl den = df_sub(df_from_double_bits(eps[i]), df_from_double_bits(eps[j]));
  double l;
  if (betaf * fabsf(den.hi) < 1e-5f) {
    l = lambda_ij(eps[i], eps[j], f[i], f[j], sc->mu, beta);
  } else {
    const dfl num = df_sub(df_from_double_bits(f[i]), df_from_double_bits(f[j]));
    l = df_to_double_fast(df_mul(num, df_recip(den)));
  }
  Lam[(size_t)i * n + j] = l;
}

void launch_lambda(cudaStream_t s, int n, const double* eps, const double* f, double beta, const Scalars* sc,
                   double* Lam, bool df) {
  if (df) lambda_df_kernel<<<dim3((n + 255) / 256, n), 256, 0, s>>>(n, eps, f, beta, (float)beta, sc, Lam);
  else lambda_kernel<<<dim3((n + 255) / 256, n), 256, 0, s>>>(n, eps, f, beta, sc, Lam);
  count_launch();
}

// Y = Lambda o (F1' - dmu I)
__global__ void dmpt_y_kernel(int n, const double* __restrict__ F1p, const double* __restrict__ Lam,
                              const Scalars* sc, double* __restrict__ Y) {
  if (!sc->active) return;
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const size_t t = (size_t)i * n + j;
  double v = F1p[t];
  if (i == j) v -= sc->dmu;
  Y[t] = Lam[t] * v;
}

void launch_dmpt_y(cudaStream_t s, int n, const double* F1p, const double* Lam, const Scalars* sc, double* Y) {
  dmpt_y_kernel<<<dim3((n + 255) / 256, n), 256, 0, s>>>(n, F1p, Lam, sc, Y);
  count_launch();
}

// ---- deterministic multi-dot -------------------------------------------------------
struct DotArgs {
  const double* a[kMaxDots];
  const double* b[kMaxDots];
};

__global__ void dots_partial_kernel(size_t len, int cnt, DotArgs args, double* __restrict__ partial,
                                    const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ double red[32];
  for (int k = 0; k < cnt; ++k) {
    const double* a = args.a[k];
    const double* b = args.b[k];
    double loc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
      loc += a[i] * b[i];
    double s = block_sum(loc, red);
    if (threadIdx.x == 0) partial[k * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void dots_final_kernel(int cnt, int nparts, const double* __restrict__ partial,
                                  double* __restrict__ out, const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ double red[32];
  for (int k = 0; k < cnt; ++k) {
    double loc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) loc += partial[k * nparts + i];
    double s = block_sum(loc, red);
    if (threadIdx.x == 0) out[k] = s;
  }
}

// gate (nullable): both kernels return at once when *gate == 0
static void dots(cudaStream_t s, size_t len, int cnt, const double* const* A, const double* const* B,
                 double* out, double* partial, const int* gate = nullptr) {
  DotArgs args;
  for (int k = 0; k < cnt; ++k) { args.a[k] = A[k]; args.b[k] = B[k]; }
  dots_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(len, cnt, args, partial, gate);
  count_launch();
  dots_final_kernel<<<1, kRedThreads, 0, s>>>(cnt, kRedBlocks, partial, out, gate);
  count_launch();
}

void launch_dots(cudaStream_t s, size_t len, int cnt, const double* const* A, const double* const* B,
                 double* out, double* partial) {
  dots(s, len, cnt, A, B, out, partial);
}

// ---- energies (eq. 13) ---------------------------------------------------------------
__global__ void energy_partial_kernel(size_t len, int npair, const double* __restrict__ h,
                                      const double* __restrict__ D, const double* __restrict__ X,
                                      const double* __restrict__ F, const double* __restrict__ E,
                                      double* __restrict__ partial) {
  __shared__ double red[32];
  double loc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
    loc += 2.0 * h[i] * D[i] + (2.0 * D[i] - X[i]) * (F[i] - h[i]);
  double s = block_sum(loc, red);
  double le = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npair; i += gridDim.x * blockDim.x) le += E[i];
  double se = block_sum(le, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    partial[gridDim.x + blockIdx.x] = se;
  }
}

__global__ void energy_final_kernel(int nparts, const double* __restrict__ partial, Scalars* sc) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) { a += partial[i]; b += partial[nparts + i]; }
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) { sc->e_elec = a; sc->vnn = b; }
}

// Dipole moment (the observable of the paper's IR spectrum, Results): the
// cores Z'_A at R_A and the valence density through the on-site position
// operator of the zero-differential-overlap basis, <mu_A| r |nu_A> = R_A
// delta_mu,nu and D1_A between s_A and p_k,A.  With the total density 2 D:
// mu = sum_A (Z'_A - 2 N_A) R_A - 4 sum_A D1_A (D_s,px, D_s,py, D_s,pz)_A,
// N_A the trace of A's diagonal block of D.  One block, fixed-order sums.
__global__ void dipole_kernel(MolDev m, ElemTable tab, const double* __restrict__ R, const double* __restrict__ Dd,
                              Scalars* sc) {
  __shared__ double red[32];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int A = threadIdx.x; A < m.N; A += blockDim.x) {
    const Elem& e = tab.e[m.elem[A]];
    const double* d = Dd + (size_t)A * 10;
    const double nA = d[0] + d[4] + d[5] + d[6];        // products ss, xx, yy, zz
    const double q = e.zcore - 2.0 * nA;
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] += q * R[3 * A + k] - 4.0 * e.D1 * d[1 + k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double t = block_sum(acc[k], red);
    if (threadIdx.x == 0) sc->dipole[k] = t;
  }
}

void launch_dipole(cudaStream_t s, const MolDev& m, const ElemTable& tab, const double* R, const double* Dd,
                   Scalars* sc) {
  dipole_kernel<<<1, 256, 0, s>>>(m, tab, R, Dd, sc);
  count_launch();
}

void launch_energy(cudaStream_t s, int n, int npair, const double* h, const double* D, const double* X,
                   const double* F, const double* E, Scalars* sc, double* part) {
  energy_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>((size_t)n * n, npair, h, D, X, F, E, part);
  count_launch();
  energy_final_kernel<<<1, kRedThreads, 0, s>>>(kRedBlocks, part, sc);
  count_launch();
}

// ---- fused combination + dot products (one pass over the vectors) -----------------------
// Per element t: y_i = Y_i[t] (i < ny); val = x[t] - sum_i c_i y_i when combo (c_i = 1
// when c is null), else x[t]; out[t] = val when out is set; and dot j sums
// val[t] times its operand: Z_j[t] when Z_j is set, else y_j when dots_on_y (the
// loaded value is reused), else val[t] itself.
// Block partials are added in a fixed order by the last block to finish (a
// counter in Scalars), so each result is deterministic and one launch does it.
constexpr int kFuseY = 16, kFuseDots = 20;
struct FuseArgs {
  const double* x;
  const double* Y[kFuseY];
  const double* c;
  double* out;
  int ny, combo, nd, dots_on_y;
  const double* Z[kFuseDots];
};

// MY, MD: compile-time bounds on ny and nd (registers).  Each thread handles
// pairs of elements (16-byte loads; len is even for the n x n matrices used
// here, an odd tail is handled by the last thread) and issues the loads of U
// pairs, one grid stride apart, before any arithmetic or store, so a thread
// keeps U x (loads per element) 16-byte requests in flight.  Storing out
// after all loads of the batch is safe when out aliases x: each element is
// read and written by the same thread in the same batch.
template <int MY, int MD, int U>
__device__ __forceinline__ void fused_batch(const FuseArgs& f, const double (&cf)[MY], size_t p0, size_t stride,
                                            int cnt, double (&acc)[MD]) {
  double2 yv[U][MY], xv[U], zv[U][MD];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (u < cnt) {
      const size_t p = p0 + (size_t)u * stride;
      xv[u] = ((const double2*)f.x)[p];
#pragma unroll
      for (int i = 0; i < MY; ++i)
        if (i < f.ny) yv[u][i] = ((const double2*)f.Y[i])[p];
#pragma unroll
      for (int j = 0; j < MD; ++j)
        if (j < f.nd && f.Z[j]) zv[u][j] = ((const double2*)f.Z[j])[p];
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (u < cnt) {
      double2 val = xv[u];
      if (f.combo) {
#pragma unroll
        for (int i = 0; i < MY; ++i)
          if (i < f.ny) { val.x -= cf[i] * yv[u][i].x; val.y -= cf[i] * yv[u][i].y; }
      }
      if (f.out) ((double2*)f.out)[p0 + (size_t)u * stride] = val;
#pragma unroll
      for (int j = 0; j < MD; ++j)
        if (j < f.nd) {
          double2 b = val;
          if (f.Z[j]) b = zv[u][j];
          else if (j < MY && f.dots_on_y && j < f.ny) b = yv[u][j];
          acc[j] += val.x * b.x + val.y * b.y;
        }
    }
  }
}

template <int MY, int MD, int U>
__global__ void __launch_bounds__(kRedThreads, (MY <= 2 ? 4 : (MY <= 8 ? 2 : 1))) fused_combo_dots_kernel(
    size_t len, FuseArgs f, double* __restrict__ partial, double* __restrict__ dots_out, Scalars* sc, int gated) {
  if (gated && !sc->active) return;
  __shared__ int s_last;
  __shared__ double sred[MD][kRedThreads / 32];
  double acc[MD];
#pragma unroll
  for (int j = 0; j < MD; ++j) acc[j] = 0.0;
  double cf[MY];
#pragma unroll
  for (int i = 0; i < MY; ++i) cf[i] = (i < f.ny) ? (f.c ? f.c[i] : 1.0) : 0.0;
  const size_t npair = len >> 1;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; p + (size_t)(U - 1) * stride < npair; p += (size_t)U * stride)
    fused_batch<MY, MD, U>(f, cf, p, stride, U, acc);
  if (p < npair) {
    const int rem = (int)((npair - 1 - p) / stride) + 1;     // < U
    fused_batch<MY, MD, U>(f, cf, p, stride, rem, acc);
  }
  if ((len & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) {
    const size_t t = len - 1;
    double val = f.x[t];
    if (f.combo)
#pragma unroll
      for (int i = 0; i < MY; ++i)
        if (i < f.ny) val -= cf[i] * f.Y[i][t];
    if (f.out) f.out[t] = val;
#pragma unroll
    for (int j = 0; j < MD; ++j)
      if (j < f.nd) acc[j] += val * (f.Z[j] ? f.Z[j][t] : ((f.dots_on_y && j < f.ny) ? f.Y[j][t] : val));
  }
  // all dots reduced together: warp shuffles, one CTA barrier, a fixed order
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < MD; ++j) {
    if (j < f.nd) {
      const double v = warp_sum(acc[j]);
      if (lane == 0) sred[j][wid] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < f.nd) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kRedThreads / 32; ++w) t += sred[threadIdx.x][w];
    partial[threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(&sc->red_count, 1u) == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: dot j by warp j mod 8, lanes over the block partials
  for (int j = wid; j < f.nd; j += kRedThreads / 32) {
    double loc = 0.0;
    for (int i = lane; i < (int)gridDim.x; i += 32) loc += __ldcg(partial + j * gridDim.x + i);
    loc = warp_sum(loc);
    if (lane == 0) dots_out[j] = loc;
  }
  if (threadIdx.x == 0) sc->red_count = 0;
}

// the smallest instantiation that holds ny and nd; a fixed grid of kRedBlocks
// (four blocks per SM of a 152-SM GB300) keeps the reduction order, and so
// the results, independent of the instantiation's occupancy
static void fused(cudaStream_t s, size_t len, const FuseArgs& f, double* partial, double* dots_out, Scalars* sc,
                  bool gated) {
  const int g = gated ? 1 : 0;
  if (f.ny <= 1 && f.nd <= 2)
    fused_combo_dots_kernel<1, 2, 2><<<kRedBlocks, kRedThreads, 0, s>>>(len, f, partial, dots_out, sc, g);
  else if (f.ny <= 4 && f.nd <= 4)
    fused_combo_dots_kernel<4, 4, 2><<<kRedBlocks, kRedThreads, 0, s>>>(len, f, partial, dots_out, sc, g);
  else if (f.ny <= 8 && f.nd <= 8)
    fused_combo_dots_kernel<8, 8, 1><<<kRedBlocks, kRedThreads, 0, s>>>(len, f, partial, dots_out, sc, g);
  else
    fused_combo_dots_kernel<kFuseY, kFuseDots, 1><<<kRedBlocks, kRedThreads, 0, s>>>(len, f, partial, dots_out,
                                                                                      sc, g);
  count_launch();
}
static FuseArgs fuse_args() {
  FuseArgs f;
  memset(&f, 0, sizeof(f));
  return f;
}

// ---- Krylov kernel (eqs. 31-34) --------------------------------------------------------
__global__ void krylov_start_kernel(size_t len, const double* __restrict__ D, const double* __restrict__ X,
                                    double* __restrict__ W0) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < len) W0[t] = D[t] - X[t];
}

__global__ void krylov_start_final(const double* n2, Scalars* sc) {
  sc->w0n2 = n2[0];
  sc->res2 = n2[0];
  sc->rank = 0;
  sc->fit = 1.0;
  sc->active = (n2[0] >= 1e-28) ? 1 : 0;   // ||W0|| >= 1e-14
  for (int i = 0; i < 16; ++i) sc->c[i] = 0.0;
}

void launch_krylov_start(cudaStream_t s, size_t len, const double* D, const double* X, double* W0,
                         Scalars* sc, double* partial) {
  // W0 = D - X and ||W0||^2 in one pass
  FuseArgs f = fuse_args();
  f.x = D; f.Y[0] = X; f.ny = 1; f.combo = 1; f.out = W0;
  f.nd = 1;
  double* tmp = partial + kRedBlocks * kMaxDots;  // small result area after the partials
  fused(s, len, f, partial, tmp, sc, false);
  krylov_start_final<<<1, 1, 0, s>>>(tmp, sc);
  count_launch();
}

struct PtrList {
  const double* p[16];
};

// v = src - sum_i coef[i] V_i   (coef on the device)
__global__ void sub_combo_kernel(size_t len, int k, PtrList V, const double* __restrict__ coef,
                                 const double* __restrict__ src, double* __restrict__ v, const Scalars* sc) {
  if (!sc->active) return;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= len) return;
  double x = src[t];
  for (int i = 0; i < k; ++i) x -= coef[i] * V.p[i][t];
  v[t] = x;
}

// scale[0] = 1 / ||v|| from nv2 = ||v||^2, ns2 = ||src||^2; breakdown
// (invariant subspace) when orthogonalisation left < 1e-10 of the norm
__global__ void norm_scale_kernel(const double* __restrict__ nv2, const double* __restrict__ ns2, Scalars* sc,
                                  double* __restrict__ scale) {
  if (!sc->active) return;
  double nv = ::sqrt(nv2[0]), ns = ::sqrt(ns2[0]);
  if (nv < 1e-10 * ns || nv == 0.0) {
    sc->active = 0;
    return;
  }
  scale[0] = 1.0 / nv;
}

__global__ void normalize_kernel(size_t len, double* __restrict__ v, const double* __restrict__ scale,
                                 const Scalars* sc) {
  if (!sc->active) return;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < len) v[t] = v[t] * scale[0];
}

// k = number of existing vectors V_0..V_{k-1}; src -> v orthonormalised (CGS twice).
// Fused passes: c1 = <V_i, src> with ||src||^2; v = src - sum c1_i V_i with
// c2 = <V_i, v>; v -= sum c2_i V_i with ||v||^2; then v *= 1/||v||.
void launch_krylov_orth(cudaStream_t s, size_t len, int k, double* const* Vs, const double* src, double* v,
                        Scalars* sc, double* partial, double* coef) {
  unsigned nb = (unsigned)((len + 255) / 256);
  FuseArgs f = fuse_args();
  const double* ns2 = coef + 16;
  if (k > 0) {
    f.x = src; f.combo = 0; f.out = nullptr; f.ny = 0; f.nd = k + 1;
    for (int j = 0; j < k; ++j) f.Z[j] = Vs[j];                      // dot k: ||src||^2
    fused(s, len, f, partial, coef, sc, true);                       // c1 in coef[0..k-1]
    ns2 = coef + k;
    for (int i = 0; i < k; ++i) { f.Y[i] = Vs[i]; f.Z[i] = nullptr; }
    f.ny = k; f.nd = k; f.dots_on_y = 1;
    f.combo = 1; f.c = coef; f.out = v;
    fused(s, len, f, partial, coef + 20, sc, true);                  // v, c2
    f.x = v; f.c = coef + 20;
  } else {
    f.x = src; f.combo = 0; f.out = v;                               // v = src
  }
  f.nd = 1;
  f.dots_on_y = 0;
  f.Z[0] = nullptr;
  fused(s, len, f, partial, coef + 16, sc, true);                    // v (second pass), ||v||^2
  norm_scale_kernel<<<1, 1, 0, s>>>(coef + 16, ns2, sc, coef + 18);
  count_launch();
  normalize_kernel<<<nb, 256, 0, s>>>(len, v, coef + 18, sc);
  count_launch();
}

__global__ void wk_kernel(size_t len, const double* __restrict__ D1, const double* __restrict__ v,
                          double* __restrict__ Wk, const Scalars* sc) {
  if (!sc->active) return;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < len) Wk[t] = D1[t] - v[t];
}

// dots[0..k]: <W_k, W_j> j = 0..k (W indices 0-based), dots[k+1] = <W_k, W0>
__global__ void gram_solve_kernel(int k, const double* __restrict__ dv, Scalars* sc, double tol, int m_min) {
  if (!sc->active) return;
  int m = k + 1;
  for (int j = 0; j <= k; ++j) {
    sc->O[k * 16 + j] = dv[j];
    sc->O[j * 16 + k] = dv[j];
  }
  sc->b[k] = dv[k + 1];
  // Cholesky of O (m x m); Gaussian elimination with pivoting if it fails
  double L[16][16], y[16], c[16];
  bool spd = true;
  for (int i = 0; i < m && spd; ++i) {
    for (int j = 0; j <= i; ++j) {
      double acc = sc->O[i * 16 + j];
      for (int l = 0; l < j; ++l) acc -= L[i][l] * L[j][l];
      if (i == j) {
        if (acc <= 0.0) { spd = false; break; }
        L[i][i] = ::sqrt(acc);
      } else {
        L[i][j] = acc / L[j][j];
      }
    }
  }
  if (spd) {
    for (int i = 0; i < m; ++i) {
      double acc = sc->b[i];
      for (int l = 0; l < i; ++l) acc -= L[i][l] * y[l];
      y[i] = acc / L[i][i];
    }
    for (int i = m - 1; i >= 0; --i) {
      double acc = y[i];
      for (int l = i + 1; l < m; ++l) acc -= L[l][i] * c[l];
      c[i] = acc / L[i][i];
    }
  } else {
    double M[16][17];
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < m; ++j) M[i][j] = sc->O[i * 16 + j];
      M[i][m] = sc->b[i];
    }
    for (int col = 0; col < m; ++col) {
      int p = col;
      for (int r = col + 1; r < m; ++r)
        if (fabs(M[r][col]) > fabs(M[p][col])) p = r;
      for (int j = 0; j <= m; ++j) { double t = M[col][j]; M[col][j] = M[p][j]; M[p][j] = t; }
      double piv = M[col][col];
      if (fabs(piv) < 1e-300) piv = 1e-300;
      for (int r = col + 1; r < m; ++r) {
        double f = M[r][col] / piv;
        for (int j = col; j <= m; ++j) M[r][j] -= f * M[col][j];
      }
    }
    for (int i = m - 1; i >= 0; --i) {
      double acc = M[i][m];
      for (int j = i + 1; j < m; ++j) acc -= M[i][j] * c[j];
      double piv = fabs(M[i][i]) < 1e-300 ? 1e-300 : M[i][i];
      c[i] = acc / piv;
    }
  }
  double cOc = 0.0, cb = 0.0;
  for (int i = 0; i < m; ++i) {
    cb += c[i] * sc->b[i];
    for (int j = 0; j < m; ++j) cOc += c[i] * sc->O[i * 16 + j] * c[j];
  }
  double r2 = cOc - 2.0 * cb + sc->w0n2;
  double fit = ::sqrt(fmax(r2, 0.0) / sc->w0n2);
  for (int i = 0; i < m; ++i) sc->c[i] = c[i];
  sc->fit = fit;
  sc->rank = m;
  if (m >= m_min && fit < tol) sc->active = 0;
}

// W_k = D1 - v (eq. 31) and its products with W_0..W_k and W0 in one pass
void launch_krylov_w(cudaStream_t s, size_t len, int k, const double* D1, const double* v, double* Wk,
                     double* const* Ws, const double* W0, Scalars* sc, double* partial, double tol,
                     int m_min) {
  FuseArgs f = fuse_args();
  f.x = D1; f.Y[0] = v; f.ny = 1; f.combo = 1; f.out = Wk;
  for (int j = 0; j < k; ++j) f.Z[j] = Ws[j];                       // <W_k, W_j>, <W_k, W_k>, <W_k, W0>
  f.Z[k + 1] = W0;
  f.nd = k + 2;
  double* dv = partial + kRedBlocks * kMaxDots + 32;
  fused(s, len, f, partial, dv, sc, true);
  gram_solve_kernel<<<1, 1, 0, s>>>(k, dv, sc, tol, m_min);
  count_launch();
}

__global__ void combine_kernel(size_t len, int mmax, PtrList V, const Scalars* sc, double* __restrict__ K) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= len) return;
  int r = sc->rank;
  double acc = 0.0;
  for (int i = 0; i < r && i < mmax; ++i) acc += sc->c[i] * V.p[i][t];
  K[t] = acc;
}

void launch_krylov_combine(cudaStream_t s, size_t len, int mmax, double* const* Vs, Scalars* sc, double* K) {
  PtrList V;
  for (int i = 0; i < mmax; ++i) V.p[i] = Vs[i];
  combine_kernel<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, mmax, V, sc, K);
  count_launch();
}

// Original XL-BOMD kernel K = -c I (Results, C240 2+ Langevin run):
// W0 = D0 - X and K (D0 - X) = -c W0; no Krylov vectors, rank 0.
__global__ void scaled_residual_kernel(size_t len, const double* __restrict__ D, const double* __restrict__ X,
                                       double c, double* __restrict__ W0, double* __restrict__ K) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= len) return;
  double w = D[t] - X[t];
  W0[t] = w;
  K[t] = -c * w;
}

__global__ void scaled_residual_final(const double* n2, Scalars* sc) {
  sc->w0n2 = n2[0];
  sc->res2 = n2[0];
  sc->rank = 0;
  sc->fit = 0.0;
  sc->active = 0;
  for (int i = 0; i < 16; ++i) sc->c[i] = 0.0;
}

void launch_scaled_residual(cudaStream_t s, size_t len, const double* D, const double* X, double c, double* W0,
                            double* K, Scalars* sc, double* partial) {
  scaled_residual_kernel<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, D, X, c, W0, K);
  count_launch();
  const double* a[1] = {W0};
  double* tmp = partial + kRedBlocks * kMaxDots;
  dots(s, len, 1, a, a, tmp, partial);
  scaled_residual_final<<<1, 1, 0, s>>>(tmp, sc);
  count_launch();
}

// ---- X update (eq. 35) ------------------------------------------------------------------
struct XHist {
  const double* x[7];
};
__constant__ double c_ck[7] = {-14.0, 36.0, -27.0, -2.0, 12.0, -6.0, 1.0};

__global__ void x_update_kernel(size_t len, XHist h, const double* __restrict__ K, double kappa, double alpha,
                                double* __restrict__ Xn) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= len) return;
  double x = 2.0 * h.x[0][t] - h.x[1][t] - kappa * K[t];
  double damp = 0.0;
  for (int k = 0; k < 7; ++k) damp += c_ck[k] * h.x[k][t];
  Xn[t] = x + alpha * damp;
}

void launch_x_update(cudaStream_t s, size_t len, double* const* Xh, const double* K, double kappa, double alpha,
                     double* Xnew) {
  XHist h;
  for (int k = 0; k < 7; ++k) h.x[k] = Xh[k];
  x_update_kernel<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, h, K, kappa, alpha, Xnew);
  count_launch();
}

// ---- Langevin thermostat ----------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC 2011): ten rounds of 32x32 -> 64-bit products with the
// multipliers 0xD2511F53, 0xCD9E8D57; the key is bumped by 0x9E3779B9, 0xBB67AE85 per round.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

__global__ void langevin_half_kernel(int N, double* __restrict__ V, const double* __restrict__ mass, double c,
                                     double kT, unsigned long long seed, int phase, const Scalars* sc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * N) return;
  const unsigned long long step = sc->step;
  uint32_t ctr[4] = {(uint32_t)t, (uint32_t)phase, (uint32_t)(step & 0xFFFFFFFFull), (uint32_t)(step >> 32)};
  philox4x32_10(ctr, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  const double u1 = ((double)ctr[0] + 0.5) * (1.0 / 4294967296.0);
  const double u2 = ((double)ctr[1] + 0.5) * (1.0 / 4294967296.0);
  const double xi = ::sqrt(-2.0 * ::log(u1)) * ::cos(2.0 * 3.141592653589793 * u2);   // Box-Muller
  const double sigma = ::sqrt((1.0 - c * c) * kT * kAccel / mass[t / 3]);
  V[t] = c * V[t] + sigma * xi;
}

void launch_langevin_half(cudaStream_t s, int N, double* V, const double* mass, double gamma, double dt,
                          double T, unsigned long long seed, int phase, const Scalars* sc) {
  const double c = ::exp(-0.5 * gamma * dt);
  langevin_half_kernel<<<(3 * N + 127) / 128, 128, 0, s>>>(N, V, mass, c, kBoltz * T, seed, phase, sc);
  count_launch();
}

__global__ void step_advance_kernel(Scalars* sc) { sc->step += 1; }

void launch_step_advance(cudaStream_t s, Scalars* sc) {
  step_advance_kernel<<<1, 1, 0, s>>>(sc);
  count_launch();
}

// ---- nuclei (eqs. 27, 28, 30) ---------------------------------------------------------------
__global__ void half_kick_kernel(int N, double* __restrict__ V, const double* __restrict__ F,
                                 const double* __restrict__ mass, double dt) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * N) return;
  V[t] += 0.5 * dt * kAccel * F[t] / mass[t / 3];
}
__global__ void drift_kernel(int N, double* __restrict__ R, const double* __restrict__ V, double dt) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * N) return;
  R[t] += dt * V[t];
}
__global__ void kinetic_kernel(int N, const double* __restrict__ V, const double* __restrict__ mass, Scalars* sc) {
  __shared__ double red[32];
  double loc = 0.0;
  for (int t = threadIdx.x; t < 3 * N; t += blockDim.x) loc += 0.5 * mass[t / 3] * V[t] * V[t] / kAccel;
  double s = block_sum(loc, red);
  if (threadIdx.x == 0) sc->e_kin = s;
}

void launch_half_kick(cudaStream_t s, int N, double* V, const double* F, const double* mass, double dt) {
  half_kick_kernel<<<(3 * N + 255) / 256, 256, 0, s>>>(N, V, F, mass, dt);
  count_launch();
}
void launch_drift(cudaStream_t s, int N, double* R, const double* V, double dt) {
  drift_kernel<<<(3 * N + 255) / 256, 256, 0, s>>>(N, R, V, dt);
  count_launch();
}
void launch_kinetic(cudaStream_t s, int N, const double* V, const double* mass, Scalars* sc) {
  kinetic_kernel<<<1, 256, 0, s>>>(N, V, mass, sc);
  count_launch();
}

__global__ void check_finite_kernel(size_t len, const double* __restrict__ a, Scalars* sc) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  for (; t < len; t += (size_t)gridDim.x * blockDim.x) bad |= !isfinite(a[t]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&sc->status, (int)kStatusNumeric);
}
void launch_check_finite(cudaStream_t s, size_t len, const double* a, Scalars* sc) {
  check_finite_kernel<<<kRedBlocks, 256, 0, s>>>(len, a, sc);
  count_launch();
}

__global__ void fill_kernel(size_t len, double* a, double v) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < len) a[t] = v;
}
void launch_fill(cudaStream_t s, size_t len, double* a, double v) {
  fill_kernel<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, a, v);
  count_launch();
}

__global__ void axpby_kernel(size_t len, double a, const double* __restrict__ x, double b,
                             const double* __restrict__ y, double* __restrict__ out) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < len) out[t] = a * x[t] + b * y[t];
}
void launch_axpby(cudaStream_t s, size_t len, double a, const double* x, double b, const double* y, double* out) {
  axpby_kernel<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, a, x, b, y, out);
  count_launch();
}

__global__ void maxabs_partial_kernel(size_t len, const double* __restrict__ a, const double* __restrict__ b,
                                      double* __restrict__ partial) {
  double m = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[t] - b[t]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, sm[i]);
    partial[blockIdx.x] = fmax(m, sm[0]);
  }
}
__global__ void maxabs_final_kernel(int np, const double* __restrict__ partial, double* out) {
  double m = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) m = fmax(m, partial[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, sm[i]);
    *out = m;
  }
}
void launch_maxabs_diff(cudaStream_t s, size_t len, const double* a, const double* b, double* out, double* partial) {
  maxabs_partial_kernel<<<kRedBlocks, 256, 0, s>>>(len, a, b, partial);
  count_launch();
  maxabs_final_kernel<<<1, 256, 0, s>>>(kRedBlocks, partial, out);
  count_launch();
}

}  // namespace kx
