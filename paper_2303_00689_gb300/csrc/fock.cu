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
// h: diagonal blocks are gathered per atom by one block (deterministic order,
// no atomics); off-diagonal blocks by one thread per pair.
// F = h + G(P): one thread per pair reads its 100 integrals once, writes both
// off-diagonal blocks (exchange) and the pair's Coulomb contributions to the
// diagonal blocks of both atoms into cw[X][Y][10] (X the receiving atom);
// one warp per atom then sums its row of cw in a fixed order and adds the
// one-centre terms.  No atomics: the result does not depend on scheduling.
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

// Orbital products on one atom: ss, sx, sy, sz, xx, yy, zz, xy, xz, yz.
// pair_cnt(p) ordered orbital pairs (mu, nu) make up product p; the i-th is
// (pair_mu(p, i), pair_nu(p, i)).  Written as constexpr functions so that in
// the fully unrolled loops below every index is a compile-time constant.
__host__ __device__ constexpr int pair_cnt(int p) { return (p == 0 || (p >= 4 && p <= 6)) ? 1 : 2; }
__host__ __device__ constexpr int pair_mu(int p, int i) {
  return p == 0 ? 0
       : p < 4  ? (i == 0 ? 0 : p)
       : p < 7  ? p - 3
       : p == 7 ? (i == 0 ? 1 : 2)
       : p == 8 ? (i == 0 ? 1 : 3)
                : (i == 0 ? 2 : 3);
}
__host__ __device__ constexpr int pair_nu(int p, int i) {
  return p == 0 ? 0
       : p < 4  ? (i == 0 ? p : 0)
       : p < 7  ? p - 3
       : p == 7 ? (i == 0 ? 2 : 1)
       : p == 8 ? (i == 0 ? 3 : 1)
                : (i == 0 ? 3 : 2);
}
__host__ __device__ constexpr double pair_mult(int p) { return (double)pair_cnt(p); }

// one thread per pair (A < B): exchange blocks F_AB, F_BA = F_AB^T (plus h) and
// the Coulomb contributions cw[A][B][P] = sum_q m_q Pd_B[q] W[P][q],
// cw[B][A][q] = sum_P m_P Pd_A[P] W[P][q] (m = product multiplicity)
__global__ void __launch_bounds__(128) fock_pair_kernel(MolDev m, PairDev pd, ElemTable tab,
                                                       const double* __restrict__ P,
                                                       const double* __restrict__ Pd, const double* __restrict__ h,
                                                       double* __restrict__ out, const int* gate) {
  if (gate && *gate == 0) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.npair) return;
  const int A = m.pA[t], B = m.pB[t];
  const int na = tab.e[m.elem[A]].norb, nb = tab.e[m.elem[B]].norb;
  const int oa = m.off[A], ob = m.off[B];
  const size_t np = (size_t)m.npair;
  const size_t n = (size_t)m.n;
  double pab[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) pab[a][b] = (a < na && b < nb) ? P[(oa + a) * n + ob + b] : 0.0;
  double da[10], db[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    da[k] = pair_mult(k) * Pd[(size_t)A * 10 + k];
    db[k] = pair_mult(k) * Pd[(size_t)B * 10 + k];
  }
  double g[4][4], ca[10], cb[10];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) g[a][b] = 0.0;
#pragma unroll
  for (int k = 0; k < 10; ++k) { ca[k] = 0.0; cb[k] = 0.0; }
  const int qa = (na == 4) ? 10 : 1, qb = (nb == 4) ? 10 : 1;
#pragma unroll
  for (int pp = 0; pp < 10; ++pp) {
#pragma unroll
    for (int qq = 0; qq < 10; ++qq) {
      if (pp < qa && qq < qb) {
        const double w = pd.W[(size_t)(pp * 10 + qq) * np + t];
        ca[pp] += db[qq] * w;
        cb[qq] += da[pp] * w;
        // exchange: g[mu][la] -= P[nu][si] (mu nu | la si) over the orbital pairs of pp, qq
#pragma unroll
        for (int i = 0; i < pair_cnt(pp); ++i)
#pragma unroll
          for (int j = 0; j < pair_cnt(qq); ++j)
            g[pair_mu(pp, i)][pair_mu(qq, j)] -= pab[pair_nu(pp, i)][pair_nu(qq, j)] * w;
      }
    }
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int la = 0; la < 4; ++la) {
      if (mu < na && la < nb) {
        const size_t ix = (oa + mu) * n + ob + la, jx = (ob + la) * n + oa + mu;
        const double v = (h ? h[ix] : 0.0) + g[mu][la];
        out[ix] = v;
        out[jx] = v;
      }
    }
  double* cA = pd.cw + ((size_t)A * m.N + B) * 10;
  double* cB = pd.cw + ((size_t)B * m.N + A) * 10;
#pragma unroll
  for (int k = 0; k < 10; ++k) { cA[k] = ca[k]; cB[k] = cb[k]; }
}

// one warp per atom: Coulomb sums over partners (lanes over partners, fixed
// order), then the diagonal block with the one-centre terms (eq. 3)
__global__ void fock_atom_kernel(MolDev m, PairDev pd, ElemTable tab, const double* __restrict__ Pd,
                                 const double* __restrict__ h, double* __restrict__ out, const int* gate) {
  if (gate && *gate == 0) return;
  const int A = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (A >= m.N) return;
  double acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.0;
  const double* row = pd.cw + (size_t)A * m.N * 10;
  for (int Y = lane; Y < m.N; Y += 32) {
    if (Y == A) continue;
    const double* c = row + (size_t)Y * 10;
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] += c[k];
  }
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = warp_sum(acc[k]);
  if (lane != 0) return;
  const Elem& e = tab.e[m.elem[A]];
  const int o = m.off[A], no = m.off[A + 1] - o;
  const double* pa = Pd + (size_t)A * 10;
  for (int mu = 0; mu < no; ++mu)
    for (int nu = 0; nu < no; ++nu) {
      double g = 2.0 * acc[c_pidx[mu][nu]];
      for (int la = 0; la < no; ++la)
        for (int si = 0; si < no; ++si) {
          const double p = pa[c_pidx[la][si]];
          g += p * (2.0 * onec(e, mu, nu, la, si) - onec(e, mu, la, nu, si));
        }
      const size_t ix = (size_t)(o + mu) * m.n + o + nu;
      out[ix] = (h ? h[ix] : 0.0) + g;
    }
}

// dU/dd for one pair (d = R_B - R_A), d = x, y, z: every term of eq. 37 is a
// stored derivative block contracted with density factors that do not depend
// on the direction, so the factor z[P][Q] of each integral derivative
// dW[P][Q] (Coulomb, exchange and electron-core parts together) is formed
// once and used for all three directions.
__global__ void __launch_bounds__(128) force_pair_kernel(MolDev m, PairDev pd, ElemTable tab,
                                                        const double* __restrict__ D, const double* __restrict__ P,
                                                        const double* __restrict__ Dd, const double* __restrict__ Pd,
                                                        double* __restrict__ g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.npair) return;
  const int A = m.pA[t], B = m.pB[t];
  const Elem& ea = tab.e[m.elem[A]];
  const Elem& eb = tab.e[m.elem[B]];
  const int na = ea.norb, nb = eb.norb;
  const int oa = m.off[A], ob = m.off[B];
  const size_t np = (size_t)m.npair;
  const size_t n = (size_t)m.n;
  double xab[4][4], pab[4][4];                 // xab = 2 D - P on the block
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const bool ok = (a < na && b < nb);
      const double dv = ok ? D[(oa + a) * n + ob + b] : 0.0;
      pab[a][b] = ok ? P[(oa + a) * n + ob + b] : 0.0;
      xab[a][b] = 2.0 * dv - pab[a][b];
    }
  // packed diagonal-block factors with the product multiplicities m_k
  double xa[10], pa[10], xb[10], pb[10];
  const double* DA = Dd + (size_t)A * 10;
  const double* DB = Dd + (size_t)B * 10;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const double mk = pair_mult(k);
    const double PA = Pd[(size_t)A * 10 + k], PB = Pd[(size_t)B * 10 + k];
    xa[k] = mk * (2.0 * DA[k] - PA);
    pa[k] = mk * PA;
    xb[k] = mk * (2.0 * DB[k] - PB);
    pb[k] = mk * PB;
  }
  double s0 = pd.dE[t], s1 = pd.dE[np + t], s2 = pd.dE[2 * np + t];
  const int qa = (na == 4) ? 10 : 1, qb = (nb == 4) ? 10 : 1;
#pragma unroll
  for (int pp = 0; pp < 10; ++pp) {
#pragma unroll
    for (int qq = 0; qq < 10; ++qq) {
      if (pp < qa && qq < qb) {
        // two-centre Coulomb, 2 Tr[(2D - P) G_R] part
        double z = 2.0 * (xa[pp] * pb[qq] + pa[pp] * xb[qq]);
        // two-centre exchange
        double ex = 0.0;
#pragma unroll
        for (int i = 0; i < pair_cnt(pp); ++i)
#pragma unroll
          for (int j = 0; j < pair_cnt(qq); ++j)
            ex += xab[pair_mu(pp, i)][pair_mu(qq, j)] * pab[pair_nu(pp, i)][pair_nu(qq, j)];
        z -= 2.0 * ex;
        // electron-core attraction on both diagonal blocks (2 Tr[h D])
        if (qq == 0) z -= 2.0 * eb.zcore * pair_mult(pp) * DA[pp];
        if (pp == 0) z -= 2.0 * ea.zcore * pair_mult(qq) * DB[qq];
        const size_t ix = (size_t)(pp * 10 + qq) * np + t;
        s0 += z * pd.dW[ix];
        s1 += z * pd.dW[100 * np + ix];
        s2 += z * pd.dW[200 * np + ix];
      }
    }
  }
  // resonance: off-diagonal blocks appear twice in 2 Tr[h D]
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int la = 0; la < 4; ++la) {
      if (mu < na && la < nb) {
        const double r = 2.0 * (ea.beta[mu ? 1 : 0] + eb.beta[la ? 1 : 0]) * D[(oa + mu) * n + ob + la];
        const size_t ix = (size_t)(mu * 4 + la) * np + t;
        s0 += r * pd.dS[ix];
        s1 += r * pd.dS[16 * np + ix];
        s2 += r * pd.dS[32 * np + ix];
      }
    }
  g[t] = s0;
  g[np + t] = s1;
  g[2 * np + t] = s2;
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
  if (m.npair > 0) {
    fock_pair_kernel<<<blocks_for(m.npair, 128), 128, 0, s>>>(m, pd, tab, P, Pd, h, out, gate);
    count_launch();
  }
  fock_atom_kernel<<<blocks_for((long long)m.N * 32, 256), 256, 0, s>>>(m, pd, tab, Pd, h, out, gate);
  count_launch();
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
