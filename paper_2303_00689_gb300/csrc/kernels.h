// Host-side launchers of the library's CUDA kernels (internal header).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace kx {

// ---- pairs.cu ---------------------------------------------------------------
bool upload_overlap_tables();
void launch_pair_values(cudaStream_t s, int npair, const int* pA, const int* pB, const int* elem,
                        const double* R, const ElemTable& tab, double* W, double* S, double* E);
// df_rotation: the molecular-frame rotation of the integral blocks in
// double-float on the FP32 pipe (mixed path) instead of FP64
void launch_pair_derivs(cudaStream_t s, int npair, const int* pA, const int* pB, const int* elem,
                        const double* R, const ElemTable& tab, double* W, double* S, double* E,
                        double* dW, double* dS, double* dE, bool df_rotation);

// ---- fock.cu ----------------------------------------------------------------
struct MolDev {          // read-only molecule description on the device
  int N, n, npair;
  const int* elem;       // element index per atom (0 H, 1 C, 2 N, 3 O)
  const int* off;        // first orbital of each atom (N + 1 entries)
  const int* pA;         // pair -> first atom (A < B)
  const int* pB;         // pair -> second atom
};
struct PairDev {         // pair blocks (SoA, stride npair)
  const double *W, *S, *E, *dW, *dS, *dE;
  double* cw;            // Fock scratch: Coulomb contribution of partner Y to atom X, [X][Y][10]
};

// out[N][10]: diagonal 4x4 block of M per atom, packed by orbital product
// gate (nullable device int): kernels return at once when *gate == 0 (adaptive Krylov rank)
void launch_pack_diag(cudaStream_t s, const MolDev& m, const double* M, double* out, const int* gate = nullptr);
// core Hamiltonian h (dense, symmetric)
void launch_build_h(cudaStream_t s, const MolDev& m, const PairDev& pd, const ElemTable& tab,
                    double* h);
// out = (h ? h : 0) + G(P) (eq. 3 with NDDO integrals); Pd = packed diagonal blocks of P
void launch_build_fock(cudaStream_t s, const MolDev& m, const PairDev& pd, const ElemTable& tab,
                       const double* P, const double* Pd, const double* h, double* out,
                       const int* gate = nullptr);
// per-pair gradient contributions g[3][npair] (eq. 37) and per-atom forces
void launch_forces(cudaStream_t s, const MolDev& m, const PairDev& pd, const ElemTable& tab,
                   const double* D, const double* P, const double* Dd, const double* Pd,
                   double* g, double* forces);

// ---- gemm64.cu --------------------------------------------------------------
// Row-major C = alpha op(A) op(B) + beta C.  ta/tb: 0 = as stored, 1 = transposed.
// sym != 0: C is symmetric; only tiles on or above the diagonal are computed
// and each value is written to (i, j) and (j, i) (bitwise symmetric result).
void dgemm(cudaStream_t s, int ta, int tb, int M, int N, int K, double alpha, const double* A,
           int lda, const double* B, int ldb, double beta, double* C, int ldc, int sym = 0,
           const int* gate = nullptr);

// ---- eig.cu -----------------------------------------------------------------
struct EigWork {
  double *A;            // n x n copy of the input (overwritten)
  double *Vst;          // n x n Householder vectors (row k = v_k)
  double *d, *e, *e2, *tau;
  double *pbuf;         // 4 x n
  double *lu;           // 5 x n x n inverse-iteration workspace
  double *Tm, *Gm, *Wt, *Wt2;  // back-transform panels
  unsigned* bar;        // 2 words grid barrier
  int* clus;            // cluster starts
  double* scal;         // scalars (Gershgorin bounds, norm)
};
size_t eig_work_bytes(int n);
void eig_work_bind(EigWork& w, void* base, int n);
// F (n x n symmetric, row-major) -> eps ascending, Q (eigenvectors as columns),
// in three stages (tridiagonalise; tridiagonal eigenpairs into Q; back-transform Q)
// df: double-float arithmetic on the FP32 pipe (mixed path), else FP64
int eig_tridiagonalize(cudaStream_t s, int n, const double* F, EigWork& w, int* status, int sm_count,
                       bool df);
// Share of the device, in thousandths of an SM, that the cooperative
// tridiagonalisation grid of size n occupies while resident (blocks divided by
// blocks per SM).  Grids that run concurrently must sum to <= 1000 x SMs.
int eig_tridiag_weight(int n, int sm_count);
// wall-time limit of the eigensolver's grid barriers on the current device (default 2 s)
int eig_set_barrier_limit(unsigned long long ns);
// rel_tol: eigenvalues to rel_tol x max(1, ||T||) (1e-12 FP64 path, 1e-9 mixed path)
// eigenvalues to rel_tol x ||T||; df_path: double-float multisection (mixed path), else FP64 bisection
void eig_bisect(cudaStream_t s, int n, double* eps, EigWork& w, double rel_tol, bool df_path);
// tridiagonal eigenvectors by inverse iteration; df_path: double-float arithmetic (mixed path)
void eig_vectors(cudaStream_t s, int n, const double* eps, double* Q, EigWork& w, bool df_path);
struct TcWork;
// tw != nullptr: the large products run on the tensor cores (mixed path)
// returns nonzero when the tensor-core path could not encode its tensor maps
int eig_backtransform(cudaStream_t s, int n, double* Q, EigWork& w, const TcWork* tw);
int symmetric_eig(cudaStream_t s, int n, const double* F, double* eps, double* Q, EigWork& w,
                  int* status, int sm_count);

// ---- electronic.cu ----------------------------------------------------------
struct Scalars {         // device-resident per-evaluation scalars
  double mu, entropy, gap, sum_lam, dmu;
  double e_elec, vnn, e_kin, res2, fit;
  double O[16 * 16], b[16], c[16], w0n2;
  int rank, active, status, pad;
  unsigned long long step;   // MD steps taken (counter of the thermostat's random numbers)
  unsigned red_count;        // blocks done in the current fused reduction (reset by its last block)
  unsigned red_pad;
  double dipole[3];          // dipole moment of the cores and D0, e Angstrom
};
void launch_fermi(cudaStream_t s, int n, const double* eps, double nocc, double beta, double* f,
                  Scalars* sc);
void launch_scale_columns(cudaStream_t s, int n, const double* Q, const double* f, double* Qs);
void launch_transpose(cudaStream_t s, int n, const double* A, double* At);
void launch_dmu(cudaStream_t s, int n, const double* F1p, const double* eps, const double* f,
                double beta, Scalars* sc);
// Lambda_ij of eq. 36 for the current eigenpairs and mu (n x n), then
// Y = Lambda o (F1' - dmu I) per Krylov vector
void launch_lambda(cudaStream_t s, int n, const double* eps, const double* f, double beta, const Scalars* sc,
                   double* Lam, bool df);   // df: double-float divided differences (mixed path)
void launch_dmpt_y(cudaStream_t s, int n, const double* F1p, const double* Lam, const Scalars* sc, double* Y);
// dipole moment of the cores and the per-spin density with packed diagonal
// blocks Dd (10 products per atom): sum_A (Z'_A - 2 N_A) R_A - 4 sum_A D1_A D_s,p
// (the on-site position operator of the NDDO basis), written to sc->dipole
void launch_dipole(cudaStream_t s, const MolDev& m, const ElemTable& tab, const double* R, const double* Dd,
                   Scalars* sc);
// U = 2 Tr[h D] + Tr[(2D - X)(F - h)] and V_nn = sum E_pair
void launch_energy(cudaStream_t s, int n, int npair, const double* h, const double* D,
                   const double* X, const double* F, const double* E, Scalars* sc, double* partial);
// blocks of the grid-wide reductions (partial sums per reduction: four per SM
// of a 152-SM GB300) and the size in doubles of the reduction workspace
// ("partial") the launchers above expect
constexpr int kRedBlocks = 608;
constexpr size_t kReduceWorkDoubles = (size_t)kRedBlocks * 24 + 128;
// out[k] = <A_k, B_k> over n*n elements for k < cnt (deterministic)
void launch_dots(cudaStream_t s, size_t len, int cnt, const double* const* A, const double* const* B,
                 double* out, double* partial);
// Krylov pieces
void launch_krylov_start(cudaStream_t s, size_t len, const double* D, const double* X, double* W0,
                         Scalars* sc, double* partial);
void launch_krylov_orth(cudaStream_t s, size_t len, int k, double* const* Vs, const double* src,
                        double* v, Scalars* sc, double* partial, double* coef);
void launch_krylov_w(cudaStream_t s, size_t len, int k, const double* D1, const double* v, double* Wk,
                     double* const* Ws, const double* W0, Scalars* sc, double* partial, double tol,
                     int m_min);
void launch_krylov_combine(cudaStream_t s, size_t len, int mmax, double* const* Vs, Scalars* sc,
                           double* K);
// original XL-BOMD kernel: W0 = D - X, K = -c W0, rank 0 (sc->active = 0)
void launch_scaled_residual(cudaStream_t s, size_t len, const double* D, const double* X, double c, double* W0,
                            double* K, Scalars* sc, double* partial);
void launch_x_update(cudaStream_t s, size_t len, double* const* Xh /*7 ptrs, k = 0..6*/,
                     const double* K, double kappa, double alpha, double* Xnew);
// nuclei
void launch_half_kick(cudaStream_t s, int N, double* V, const double* F, const double* mass,
                      double dt);
void launch_drift(cudaStream_t s, int N, double* R, const double* V, double dt);
void launch_kinetic(cudaStream_t s, int N, const double* V, const double* mass, Scalars* sc);
// Langevin (OBABO) Ornstein-Uhlenbeck half step V <- c V + sqrt((1 - c^2) k_B T / M) xi with
// c = exp(-gamma dt / 2); xi from Philox4x32-10, counter (3A + k, phase, step), key seed
void launch_langevin_half(cudaStream_t s, int N, double* V, const double* mass, double gamma, double dt,
                          double T, unsigned long long seed, int phase, const Scalars* sc);
void launch_step_advance(cudaStream_t s, Scalars* sc);
void launch_check_finite(cudaStream_t s, size_t len, const double* a, Scalars* sc);
void launch_fill(cudaStream_t s, size_t len, double* a, double v);
void launch_axpby(cudaStream_t s, size_t len, double a, const double* x, double b, const double* y,
                  double* out);
void launch_maxabs_diff(cudaStream_t s, size_t len, const double* a, const double* b, double* out,
                        double* partial);

}  // namespace kx
