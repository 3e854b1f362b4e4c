// Core Hamiltonian, Fock matrix and force contractions from the pair blocks.
//
//  h (eq. 6, NDDO): U_mu on the diagonal, electron-core attraction
//     -Z'_B (mu nu|s_B s_B) summed over partners on diagonal blocks, resonance
//     (beta_mu + beta_lam) S_mu,lam / 2 on off-diagonal blocks.
//  G(P) = 2J(P) - K(P) (eq. 3): G_mu,nu = sum P_lam,sig [2(mu nu|lam sig) -
//     (mu lam|nu sig)] with the NDDO-allowed integrals: one-centre terms and
//     two-centre Coulomb on diagonal blocks, two-centre exchange on
//     off-diagonal blocks.  P is the per-spin density; F = h + G(X) (eq. 17).
//  Forces (eq. 37 with S = I): per pair, the derivative of
//     2 Tr[h D] + Tr[(2D - P) G(P)] + V_nn at fixed D, P contracted with the
//     stored dW, dS, dE blocks; F_A += g, F_B -= g with g = dE/dd, d = R_B - R_A.
//
// Diagonal blocks are gathered per atom by one block (deterministic order, no
// atomics); off-diagonal blocks are written by one thread per pair into the
// upper triangle and mirrored by a tiled transpose.
#include "common.cuh"
#include "kernels.h"

namespace kx {

__device__ __constant__ int c_pidx[4][4] = {{0, 1, 2, 3}, {1, 4, 7, 8}, {2, 7, 5, 9}, {3, 8, 9, 6}};
__device__ __constant__ double c_mult[10] = {1, 2, 2, 2, 1, 1, 1, 2, 2, 2};
__device__ __constant__ int c_pmu[10] = {0, 0, 0, 0, 1, 2, 3, 1, 1, 2};
__device__ __constant__ int c_pnu[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};

__device__ __forceinline__ int pair_index(int A, int B, int N) {
  // A < B, pairs enumerated row by row
  return A * (2 * N - A - 1) / 2 + (B - A - 1);
}

// one-centre (ab|cd) on one atom
__device__ __forceinline__ double onec(const Elem& e, int a, int b, int c, int d) {
  if (a == b && c == d) {
    if (a == 0 && c == 0) return e.G_ss;
    if ((a == 0) != (c == 0)) return e.G_sp;
    return (a == c) ? e.G_pp : e.G_p2;
  }
  if (a != b && c != d) {
    bool same = (a == c && b == d) || (a == d && b == c);
    if (!same) return 0.0;
    return (a == 0 || b == 0) ? e.H_sp : e.H_pp;
  }
  return 0.0;
}

__global__ void pack_diag_kernel(int N, int n, const int* __restrict__ off, const double* __restrict__ M,
                                 double* __restrict__ out, const int* gate) {
  if (gate && *gate == 0) return;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * 10) return;
  int A = t / 10, p = t % 10;
  int o = off[A], no = off[A + 1] - o;
  int mu = c_pmu[p], nu = c_pnu[p];
  out[t] = (mu < no && nu < no) ? M[(size_t)(o + mu) * n + o + nu] : 0.0;
}

// Gather over partners of atom A: acc[P] = sum_B sum_q wq(B, q) W_AB[P][q]
// where wq = scale * mult(q) * dens_B[q] (Coulomb) or -Z'_B for q = ss (h).
// mode 0: Coulomb with packed densities; mode 1: electron-core attraction.
// One block of kDiagThreads per atom: threads stride over the partners, then a
// fixed-order reduction (warp shuffles, then warps in order) leaves the sums in
// thread 0.
constexpr int kDiagThreads = 256;

__device__ void gather_diag(int A, const MolDev& m, const PairDev& pd, const ElemTable& tab,
                            const double* __restrict__ dens, int mode, double acc[10]) {
  __shared__ double part[kDiagThreads / 32][10];
  for (int P = 0; P < 10; ++P) acc[P] = 0.0;
  int N = m.N;
  size_t np = (size_t)m.npair;
  for (int B = threadIdx.x; B < N; B += blockDim.x) {
    if (B == A) continue;
    int first = (A < B);
    int pi = first ? pair_index(A, B, N) : pair_index(B, A, N);
    if (mode == 1) {
      double z = -tab.e[m.elem[B]].zcore;
      for (int P = 0; P < 10; ++P) {
        double w = first ? pd.W[(size_t)(P * 10) * np + pi] : pd.W[(size_t)P * np + pi];
        acc[P] += z * w;
      }
    } else {
      const double* db = dens + (size_t)B * 10;
      int nq = (tab.e[m.elem[B]].norb == 4) ? 10 : 1;
      for (int q = 0; q < nq; ++q) {
        double wq = c_mult[q] * db[q];
        if (wq == 0.0) continue;
        for (int P = 0; P < 10; ++P) {
          double w = first ? pd.W[(size_t)(P * 10 + q) * np + pi] : pd.W[(size_t)(q * 10 + P) * np + pi];
          acc[P] += wq * w;
        }
      }
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int P = 0; P < 10; ++P) acc[P] = warp_sum(acc[P]);
  if (lane == 0)
    for (int P = 0; P < 10; ++P) part[warp][P] = acc[P];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int P = 0; P < 10; ++P) {
      double t = part[0][P];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t += part[w][P];
      acc[P] = t;
    }
}

__global__ void __launch_bounds__(kDiagThreads) h_diag_kernel(MolDev m, PairDev pd, ElemTable tab,
                                                              double* __restrict__ h) {
  int A = blockIdx.x;
  if (A >= m.N) return;
  double acc[10];
  gather_diag(A, m, pd, tab, nullptr, 1, acc);
  if (threadIdx.x != 0) return;
  const Elem& e = tab.e[m.elem[A]];
  int o = m.off[A], no = m.off[A + 1] - o;
  for (int mu = 0; mu < no; ++mu)
    for (int nu = 0; nu < no; ++nu) {
      double v = acc[c_pidx[mu][nu]];
      if (mu == nu) v += e.U[mu == 0 ? 0 : 1];
      h[(size_t)(o + mu) * m.n + o + nu] = v;
    }
}

__global__ void h_offdiag_kernel(MolDev m, PairDev pd, ElemTable tab, double* __restrict__ h) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.npair) return;
  int A = m.pA[t], B = m.pB[t];
  const Elem& ea = tab.e[m.elem[A]];
  const Elem& eb = tab.e[m.elem[B]];
  int oa = m.off[A], ob = m.off[B];
  size_t np = (size_t)m.npair;
  for (int mu = 0; mu < ea.norb; ++mu)
    for (int la = 0; la < eb.norb; ++la) {
      double v = 0.5 * (ea.beta[mu ? 1 : 0] + eb.beta[la ? 1 : 0]) * pd.S[(size_t)(mu * 4 + la) * np + t];
      h[(size_t)(oa + mu) * m.n + ob + la] = v;
      h[(size_t)(ob + la) * m.n + oa + mu] = v;
    }
}

__global__ void __launch_bounds__(kDiagThreads)
    fock_diag_kernel(MolDev m, PairDev pd, ElemTable tab, const double* __restrict__ P,
                     const double* __restrict__ Pd, const double* __restrict__ h, double* __restrict__ out,
                     const int* gate) {
  if (gate && *gate == 0) return;
  int A = blockIdx.x;
  if (A >= m.N) return;
  double acc[10];
  gather_diag(A, m, pd, tab, Pd, 0, acc);
  if (threadIdx.x != 0) return;
  const Elem& e = tab.e[m.elem[A]];
  int o = m.off[A], no = m.off[A + 1] - o;
  const double* pa = Pd + (size_t)A * 10;
  for (int mu = 0; mu < no; ++mu)
    for (int nu = 0; nu < no; ++nu) {
      double g = 2.0 * acc[c_pidx[mu][nu]];
      for (int la = 0; la < no; ++la)
        for (int si = 0; si < no; ++si) {
          double p = pa[c_pidx[la][si]];
          g += p * (2.0 * onec(e, mu, nu, la, si) - onec(e, mu, la, nu, si));
        }
      size_t ix = (size_t)(o + mu) * m.n + o + nu;
      out[ix] = (h ? h[ix] : 0.0) + g;
    }
}

__global__ void fock_offdiag_kernel(MolDev m, PairDev pd, ElemTable tab, const double* __restrict__ P,
                                    const double* __restrict__ h, double* __restrict__ out, const int* gate) {
  if (gate && *gate == 0) return;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.npair) return;
  int A = m.pA[t], B = m.pB[t];
  int na = tab.e[m.elem[A]].norb, nb = tab.e[m.elem[B]].norb;
  int oa = m.off[A], ob = m.off[B];
  size_t np = (size_t)m.npair;
  double pab[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      pab[a][b] = (a < na && b < nb) ? P[(size_t)(oa + a) * m.n + ob + b] : 0.0;
  for (int mu = 0; mu < na; ++mu)
    for (int la = 0; la < nb; ++la) {
      double g = 0.0;
      for (int nu = 0; nu < na; ++nu)
        for (int si = 0; si < nb; ++si)
          g -= pab[nu][si] * pd.W[(size_t)(c_pidx[mu][nu] * 10 + c_pidx[la][si]) * np + t];
      size_t ix = (size_t)(oa + mu) * m.n + ob + la;
      out[ix] = (h ? h[ix] : 0.0) + g;
    }
}

// copy the strict upper triangle onto the lower one (32 x 32 tiles)
__global__ void mirror_upper_kernel(int n, double* __restrict__ a, const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ double tile[32][33];
  int bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;
  int i0 = bi * 32, j0 = bj * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = i0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < n && j < n) ? a[(size_t)i * n + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int j = j0 + r, i = i0 + threadIdx.x;  // write a[j][i] = a[i][j] for i < j
    if (i < n && j < n && i < j) a[(size_t)j * n + i] = tile[threadIdx.x][r];
  }
}

__global__ void force_pair_kernel(MolDev m, PairDev pd, ElemTable tab, const double* __restrict__ D,
                                  const double* __restrict__ P, const double* __restrict__ Dd,
                                  const double* __restrict__ Pd, double* __restrict__ g) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.npair) return;
  int A = m.pA[t], B = m.pB[t];
  const Elem& ea = tab.e[m.elem[A]];
  const Elem& eb = tab.e[m.elem[B]];
  int na = ea.norb, nb = eb.norb;
  int oa = m.off[A], ob = m.off[B];
  size_t np = (size_t)m.npair;
  double dab[4][4], pab[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      bool ok = (a < na && b < nb);
      dab[a][b] = ok ? D[(size_t)(oa + a) * m.n + ob + b] : 0.0;
      pab[a][b] = ok ? P[(size_t)(oa + a) * m.n + ob + b] : 0.0;
    }
  const double* DA = Dd + (size_t)A * 10;
  const double* DB = Dd + (size_t)B * 10;
  const double* PA = Pd + (size_t)A * 10;
  const double* PB = Pd + (size_t)B * 10;
  int qa = (na == 4) ? 10 : 1, qb = (nb == 4) ? 10 : 1;
  for (int k = 0; k < 3; ++k) {
    const double* dW = pd.dW + (size_t)k * 100 * np;
    const double* dS = pd.dS + (size_t)k * 16 * np;
    double s = pd.dE[(size_t)k * np + t];
    // electron-core attraction on both diagonal blocks
    double ec = 0.0;
    for (int p = 0; p < qa; ++p) ec -= eb.zcore * c_mult[p] * DA[p] * dW[(size_t)(p * 10) * np + t];
    for (int q = 0; q < qb; ++q) ec -= ea.zcore * c_mult[q] * DB[q] * dW[(size_t)q * np + t];
    s += 2.0 * ec;
    // resonance (off-diagonal blocks appear twice in the trace)
    double rs = 0.0;
    for (int mu = 0; mu < na; ++mu)
      for (int la = 0; la < nb; ++la)
        rs += 0.5 * (ea.beta[mu ? 1 : 0] + eb.beta[la ? 1 : 0]) * dS[(size_t)(mu * 4 + la) * np + t] *
              dab[mu][la];
    s += 4.0 * rs;
    // two-centre Coulomb: Tr[(2D - P) G_R]
    double cb = 0.0;
    for (int p = 0; p < qa; ++p) {
      double aA = c_mult[p] * (2.0 * DA[p] - PA[p]);
      double pA = c_mult[p] * PA[p];
      for (int q = 0; q < qb; ++q) {
        double w = dW[(size_t)(p * 10 + q) * np + t];
        cb += w * (aA * c_mult[q] * PB[q] + pA * c_mult[q] * (2.0 * DB[q] - PB[q]));
      }
    }
    s += 2.0 * cb;
    // two-centre exchange
    double ex = 0.0;
    for (int mu = 0; mu < na; ++mu)
      for (int nu = 0; nu < na; ++nu)
        for (int la = 0; la < nb; ++la)
          for (int si = 0; si < nb; ++si) {
            double w = dW[(size_t)(c_pidx[mu][nu] * 10 + c_pidx[la][si]) * np + t];
            ex += w * (2.0 * dab[mu][la] - pab[mu][la]) * pab[nu][si];
          }
    s -= 2.0 * ex;
    g[(size_t)k * np + t] = s;
  }
}

// forces_I = sum_{B > I} g(I, B) - sum_{A < I} g(A, I); one warp per atom
__global__ void force_atom_kernel(MolDev m, const double* __restrict__ g, double* __restrict__ F) {
  int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (I >= m.N) return;
  size_t np = (size_t)m.npair;
  double f[3] = {0.0, 0.0, 0.0};
  for (int J = lane; J < m.N; J += 32) {
    if (J == I) continue;
    int pi = (I < J) ? pair_index(I, J, m.N) : pair_index(J, I, m.N);
    double sg = (I < J) ? 1.0 : -1.0;
    for (int k = 0; k < 3; ++k) f[k] += sg * g[(size_t)k * np + pi];
  }
  for (int k = 0; k < 3; ++k) f[k] = warp_sum(f[k]);
  if (lane == 0)
    for (int k = 0; k < 3; ++k) F[3 * I + k] = f[k];
}

static inline int blocks_for(long long work, int per) { return (int)((work + per - 1) / per); }

void launch_pack_diag(cudaStream_t s, const MolDev& m, const double* M, double* out, const int* gate) {
  pack_diag_kernel<<<blocks_for((long long)m.N * 10, 256), 256, 0, s>>>(m.N, m.n, m.off, M, out, gate);
  count_launch();
}

static void mirror(cudaStream_t s, int n, double* a, const int* gate) {
  int t = (n + 31) / 32;
  mirror_upper_kernel<<<dim3(t, t), dim3(32, 8), 0, s>>>(n, a, gate);
  count_launch();
}

void launch_build_h(cudaStream_t s, const MolDev& m, const PairDev& pd, const ElemTable& tab,
                    double* h) {
  h_diag_kernel<<<m.N, kDiagThreads, 0, s>>>(m, pd, tab, h);
  count_launch();
  if (m.npair > 0) {
    h_offdiag_kernel<<<blocks_for(m.npair, 128), 128, 0, s>>>(m, pd, tab, h);
    count_launch();
  }
}

void launch_build_fock(cudaStream_t s, const MolDev& m, const PairDev& pd, const ElemTable& tab,
                       const double* P, const double* Pd, const double* h, double* out, const int* gate) {
  fock_diag_kernel<<<m.N, kDiagThreads, 0, s>>>(m, pd, tab, P, Pd, h, out, gate);
  count_launch();
  if (m.npair > 0) {
    fock_offdiag_kernel<<<blocks_for(m.npair, 128), 128, 0, s>>>(m, pd, tab, P, h, out, gate);
    count_launch();
  }
  mirror(s, m.n, out, gate);
}

void launch_forces(cudaStream_t s, const MolDev& m, const PairDev& pd, const ElemTable& tab,
                   const double* D, const double* P, const double* Dd, const double* Pd, double* g,
                   double* forces) {
  if (m.npair > 0) {
    force_pair_kernel<<<blocks_for(m.npair, 128), 128, 0, s>>>(m, pd, tab, D, P, Dd, Pd, g);
    count_launch();
  }
  force_atom_kernel<<<blocks_for((long long)m.N * 32, 128), 128, 0, s>>>(m, g, forces);
  count_launch();
}

}  // namespace kx
