// C ABI of the library: handle set-up, the per-step orchestration of the
// kernels, state access and device-side phase timing.  See include/sim.h.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sim.h"
#include "common.cuh"
#include "kernels.h"
#include "tc_gemm.h"

namespace kx {
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
cudaError_t last_launch_error() { return cudaGetLastError(); }
}  // namespace kx

using namespace kx;

static thread_local std::string t_err = "";
static int fail(int code, const std::string& msg) {
  t_err = msg;
  return code;
}
#define CUDA_TRY(x)                                                                  \
  do {                                                                               \
    cudaError_t _e = (x);                                                            \
    if (_e != cudaSuccess)                                                           \
      return fail(SIM_EINTERNAL, std::string(#x) + ": " + cudaGetErrorString(_e));   \
  } while (0)

// Makes a handle's device current for the duration of a call and gives the
// caller back its own current device afterwards.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// damping constants of the modified Verlet scheme, k_max = 6 (eq. 29; the
// paper takes kappa, alpha, c_k from its ref. 24)
static const double kKappa = 1.84;
static const double kAlphaDamp = 0.0055;

// ---------------------------------------------------------------------------
// phases timed with CUDA events
// ---------------------------------------------------------------------------
enum Phase {
  PH_PAIRS = 0, PH_FOCK, PH_TRIDIAG, PH_BISECT, PH_TRIEIG, PH_BACKTR, PH_DENSITY, PH_FORCES,
  PH_KRY_FOCK, PH_KRY_GEMM, PH_KRY_BLAS, PH_UPDATE, PH_COUNT
};
static const char* kPhaseNames[PH_COUNT] = {
    "pair_integrals", "fock_build", "eig_tridiag", "eig_bisection", "eig_tridiag_vectors", "eig_backtransform",
    "density_gemm", "energy_forces", "krylov_fock", "krylov_dmpt_gemm", "krylov_blas", "integrate"};

struct sim_handle {
  int dev = 0, sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // side stream for work that does not feed the next kernels of the step:
  // the Fermi occupations (during inverse iteration and back-transformation)
  // and energy, forces and dipole (during the Krylov kernel); forked from and
  // joined to `stream` by events, so graph capture records both branches
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev[2] = {}, join_ev[2] = {};
  sim_config cfg;
  ElemTable tab;
  int N = 0, n = 0, npair = 0, nocc = 0, mmax = 0;
  double beta = 0.0;
  std::vector<int> elem_h, off_h;
  std::vector<int> Z_h;           // atomic numbers and raw inputs, kept for sim_save
  sim_param_table table_raw{};
  int charge = 0;
  std::vector<double> mass_h;
  // device memory (one arena)
  void* arena = nullptr;
  size_t arena_bytes = 0;
  int *elem = nullptr, *off = nullptr, *pA = nullptr, *pB = nullptr;
  double *R = nullptr, *V = nullptr, *F = nullptr, *mass = nullptr, *g = nullptr;
  double *W = nullptr, *S = nullptr, *E = nullptr, *dW = nullptr, *dS = nullptr, *dE = nullptr;
  double* cw = nullptr;
  double *h = nullptr, *Fock = nullptr, *D = nullptr, *K = nullptr, *Q = nullptr, *Qs = nullptr;
  double *eps = nullptr, *f = nullptr, *Dd = nullptr, *Pd = nullptr, *Vd = nullptr;
  double *T1 = nullptr, *T2 = nullptr, *F1 = nullptr, *Y = nullptr, *D1 = nullptr, *W0 = nullptr;
  double* X[8] = {};
  double* Vk[16] = {};
  double* Wk[16] = {};
  double *red = nullptr, *coef = nullptr;
  double* red2 = nullptr;           // reduction workspace of the side stream (energy)
  Scalars* sc = nullptr;
  sim_step_result* rec = nullptr;   // device per-step records (ring of kRecCap)
  int* rec_idx = nullptr;           // device: index of the next record in rec[]
  long long rec_count = 0;          // host: records written since the last reset
  EigWork ew;
  TcWork tw;
  int xhead = 0;
  int scf_iters = 0;   // SCF iterations used by sim_create (0 when P0 was given)
  double scf_residual = 0.0;
  // host mirror of the last results
  Scalars sc_h;
  // profiling
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double ph_ms[PH_COUNT] = {};
  long long ph_n[PH_COUNT] = {};
  int cur_phase = -1;
  cudaEvent_t cur_start = nullptr;
  // CUDA graphs of one step, one per phase of the 8-slot X ring
  bool graphs = false;
  cudaGraphExec_t gexec[8] = {};
  long long gnodes[8] = {};
};
static const int kRecCap = 4096;

// ---------------------------------------------------------------------------
// parameter derivation (multipole lengths and additive terms)
// ---------------------------------------------------------------------------
static double bisect_root(double (*fn)(double, double), double D, double target) {
  double lo = 1e-8, hi = 1e3;
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (fn(mid, D) > target) lo = mid; else hi = mid;   // fn decreases in rho
  }
  return 0.5 * (lo + hi);
}
static double dipole_limit(double r, double D1) { return 0.25 * kE2 * (1.0 / r - 1.0 / std::sqrt(D1 * D1 + r * r)); }
static double quad_limit(double r, double D2) {
  return 0.125 * kE2 * (1.0 / r - 2.0 / std::sqrt(D2 * D2 + r * r) + 1.0 / std::sqrt(2.0 * D2 * D2 + r * r));
}

static int build_elem(const double* v, Elem& e) {
  e.norb = (int)std::lround(v[SIM_P_NORB]);
  e.nprin = (int)std::lround(v[SIM_P_NPRIN]);
  if (!((e.norb == 1 && e.nprin == 1) || (e.norb == 4 && e.nprin == 2))) return -1;
  e.zcore = v[SIM_P_ZCORE];
  e.mass = v[SIM_P_MASS];
  e.U[0] = v[SIM_P_USS]; e.U[1] = v[SIM_P_UPP];
  e.beta[0] = v[SIM_P_BETA_S]; e.beta[1] = v[SIM_P_BETA_P];
  e.zeta[0] = v[SIM_P_ZETA_S]; e.zeta[1] = v[SIM_P_ZETA_P];
  e.alpha = v[SIM_P_ALPHA];
  e.ga[0] = v[SIM_P_GA0]; e.gb[0] = v[SIM_P_GB0]; e.gc[0] = v[SIM_P_GC0];
  e.ga[1] = v[SIM_P_GA1]; e.gb[1] = v[SIM_P_GB1]; e.gc[1] = v[SIM_P_GC1];
  e.G_ss = v[SIM_P_GSS]; e.G_sp = v[SIM_P_GSP]; e.G_pp = v[SIM_P_GPP]; e.G_p2 = v[SIM_P_GP2];
  e.H_sp = v[SIM_P_HSP];
  e.H_pp = 0.5 * (e.G_pp - e.G_p2);
  for (int k = 0; k < 2; ++k)
    e.sto_nrm[k] = std::pow(2.0 * e.zeta[k], e.nprin + 0.5) / std::sqrt(e.nprin == 1 ? 2.0 : 24.0);
  const double kHuge = 1e30;  // vanishing two-electron parameters -> integrals -> 0
  e.rho0 = (e.G_ss > 0.0) ? kE2 / (2.0 * e.G_ss) : kHuge;
  if (e.norb == 1) {
    e.D1 = e.D2 = 0.0;
    e.rho1 = e.rho2 = e.rho0;
    return 0;
  }
  int n = e.nprin;
  double zs = e.zeta[0], zp = e.zeta[1];
  e.D1 = (2 * n + 1) * std::pow(4.0 * zs * zp, n + 0.5) / (std::pow(zs + zp, 2 * n + 2) * std::sqrt(3.0)) * kBohr;
  e.D2 = std::sqrt((4.0 * n * n + 6.0 * n + 2.0) / 20.0) / zp * kBohr;
  e.rho1 = (e.H_sp > 0.0) ? bisect_root(dipole_limit, e.D1, e.H_sp) : kHuge;
  e.rho2 = (e.H_pp > 0.0) ? bisect_root(quad_limit, e.D2, e.H_pp) : kHuge;
  return 0;
}

static int elem_index(int Z) {
  switch (Z) {
    case 1: return 0;
    case 6: return 1;
    case 7: return 2;
    case 8: return 3;
    default: return -1;
  }
}

// ---------------------------------------------------------------------------
// profiling helpers
// ---------------------------------------------------------------------------
static cudaEvent_t take_event(sim_handle* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
static void phase_begin(sim_handle* h, int ph) {
  if (!h->prof) return;
  h->cur_phase = ph;
  h->cur_start = take_event(h);
  cudaEventRecord(h->cur_start, h->stream);
}
static void phase_end(sim_handle* h) {
  if (!h->prof || h->cur_phase < 0) return;
  cudaEvent_t e = take_event(h);
  cudaEventRecord(e, h->stream);
  h->ev_pending.push_back({h->cur_phase, {h->cur_start, e}});
  h->cur_phase = -1;
}
static void collect_events(sim_handle* h) {
  for (auto& p : h->ev_pending) {
    cudaEventSynchronize(p.second.second);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.second.first, p.second.second);
    h->ph_ms[p.first] += ms;
    h->ph_n[p.first] += 1;
    h->ev_pool.push_back(p.second.first);
    h->ev_pool.push_back(p.second.second);
  }
  h->ev_pending.clear();
}

// ---------------------------------------------------------------------------
// device orchestration
// ---------------------------------------------------------------------------
static MolDev mol(const sim_handle* h) { return MolDev{h->N, h->n, h->npair, h->elem, h->off, h->pA, h->pB}; }
static PairDev pairs(const sim_handle* h) { return PairDev{h->W, h->S, h->E, h->dW, h->dS, h->dE, h->cw}; }
static double* xslot(sim_handle* h, int k) { return h->X[(h->xhead + k) % 8]; }

static bool mixed(const sim_handle* h) { return h->cfg.precision == SIM_PREC_MIXED; }

// D0 = Q diag(f) Q^T = (Q f^1/2)(Q f^1/2)^T, exactly symmetric
static void density(sim_handle* h) {
  cudaStream_t s = h->stream;
  int n = h->n;
  launch_scale_columns(s, n, h->Q, h->f, h->Qs);
  if (mixed(h)) {
    // four fixed-point BF16 slices, ten slice products (32 bits per row scale),
    // all slices of a k-tile staged together (tc_gemm_grouped4)
    tc_split(s, h->tw, kSlotQs, h->Qs, 4, 0);
    tc_gemm_grouped4(s, h->tw, kSlotQs, kSlotQs, 1.0, h->D, 1);
  } else {
    dgemm(s, 0, 1, n, n, n, 1.0, h->Qs, n, h->Qs, n, 0.0, h->D, n, 1);
  }
}

// BF16 pieces of Q and Q^T for the DMPT products (once per evaluation)
static void dmpt_prepare(sim_handle* h) {
  if (!mixed(h)) return;
  tc_split(h->stream, h->tw, kSlotQ, h->Q, 3, 0);
  tc_split(h->stream, h->tw, kSlotQt, h->Q, 3, 1);
}

// D1 = Q [Lambda o (Q^T F1 Q - dmu I)] Q^T (eq. 36).  Every launch reads the
// device flag sc->active and returns at once when the Krylov fit has already
// converged, so unused Krylov vectors cost no work and no host round trip.
static void dmpt(sim_handle* h, const double* F1, double* D1) {
  cudaStream_t s = h->stream;
  int n = h->n;
  const int* g = &h->sc->active;
  if (mixed(h)) {
    // three fixed-point BF16 slices per operand, six slice products (24 bits per row
    // scale), all slices of a k-tile staged together (tc_gemm_grouped)
    tc_split(s, h->tw, kSlotT0, F1, 3, 0, g);
    tc_gemm_grouped(s, h->tw, kSlotQt, kSlotT0, 1.0, h->T1, 0, g);      // T1 = Q^T F1
    tc_split(s, h->tw, kSlotT1, h->T1, 3, 0, g);
    tc_gemm_grouped(s, h->tw, kSlotT1, kSlotQt, 1.0, h->T2, 1, g);      // T2 = (Q^T F1) Q
    launch_dmu(s, n, h->T2, h->eps, h->f, h->beta, h->sc);
    launch_dmpt_y(s, n, h->T2, h->K, h->sc, h->Y);     // h->K holds Lambda until the final combine
    tc_split(s, h->tw, kSlotT0, h->Y, 3, 0, g);
    tc_gemm_grouped(s, h->tw, kSlotQ, kSlotT0, 1.0, h->T1, 0, g);       // T1 = Q Y
    tc_split(s, h->tw, kSlotT1, h->T1, 3, 0, g);
    tc_gemm_grouped(s, h->tw, kSlotT1, kSlotQ, 1.0, D1, 1, g);          // D1 = (Q Y) Q^T
    return;
  }
  dgemm(s, 0, 0, n, n, n, 1.0, F1, n, h->Q, n, 0.0, h->T1, n, 0, g);         // T1 = F1 Q
  dgemm(s, 1, 0, n, n, n, 1.0, h->Q, n, h->T1, n, 0.0, h->T2, n, 1, g);      // T2 = Q^T T1
  launch_dmu(s, n, h->T2, h->eps, h->f, h->beta, h->sc);
  launch_dmpt_y(s, n, h->T2, h->K, h->sc, h->Y);       // h->K holds Lambda until the final combine
  dgemm(s, 0, 0, n, n, n, 1.0, h->Q, n, h->Y, n, 0.0, h->T1, n, 0, g);       // T1 = Q Y
  dgemm(s, 0, 1, n, n, n, 1.0, h->T1, n, h->Q, n, 0.0, D1, n, 1, g);         // D1 = T1 Q^T
}

// fork k: work issued on h->side after this point follows everything issued
// on h->stream so far; join k: h->stream waits for the side work issued since
static void fork_side(sim_handle* h, int k) {
  cudaEventRecord(h->fork_ev[k], h->stream);
  cudaStreamWaitEvent(h->side, h->fork_ev[k], 0);
}
static void join_side(sim_handle* h, int k) {
  cudaEventRecord(h->join_ev[k], h->side);
  cudaStreamWaitEvent(h->stream, h->join_ev[k], 0);
}
// side work only outside phase profiling (whose events time the main stream)
static bool concurrent(const sim_handle* h) { return h->side && !h->prof; }

// eigenpairs of the Fock matrix; with fermi_side, the Fermi occupations and
// mu (eq. 8; they need the eigenvalues only) run on the side stream while the
// eigenvectors are formed, and the caller joins before the density
static int eig(sim_handle* h, bool fermi_side = false) {
  phase_begin(h, PH_TRIDIAG);
  int st = eig_tridiagonalize(h->stream, h->n, h->Fock, h->ew, &h->sc->status, h->sms, mixed(h));
  phase_end(h);
  if (st != 0) return fail(SIM_EINTERNAL, "tridiagonalisation launch failed (code " + std::to_string(st) + ")");
  phase_begin(h, PH_BISECT);
  eig_bisect(h->stream, h->n, h->eps, h->ew, 1e-12, mixed(h));
  phase_end(h);
  if (fermi_side) {
    fork_side(h, 0);
    launch_fermi(h->side, h->n, h->eps, (double)h->nocc, h->beta, h->f, h->sc);
  }
  phase_begin(h, PH_TRIEIG);
  eig_vectors(h->stream, h->n, h->eps, h->Q, h->ew, mixed(h));
  phase_end(h);
  phase_begin(h, PH_BACKTR);
  const int bt = eig_backtransform(h->stream, h->n, h->Q, h->ew, mixed(h) ? &h->tw : nullptr);
  phase_end(h);
  if (bt != 0) return fail(SIM_EINTERNAL, "back-transformation: tensor map encoding failed");
  return SIM_OK;
}

// Krylov kernel of W0 = D - P for the current eigenpairs (eqs. 31-34), result in h->K
static void krylov_kernel(sim_handle* h, const double* P) {
  cudaStream_t s = h->stream;
  size_t nn = (size_t)h->n * h->n;
  MolDev m = mol(h);
  PairDev pd = pairs(h);
  phase_begin(h, PH_KRY_GEMM);
  dmpt_prepare(h);
  phase_end(h);
  phase_begin(h, PH_KRY_BLAS);
  // Lambda of eq. 36 once per evaluation; K is free until launch_krylov_combine writes it
  launch_lambda(s, h->n, h->eps, h->f, h->beta, h->sc, h->K, mixed(h));
  phase_end(h);
  phase_begin(h, PH_KRY_BLAS);
  launch_krylov_start(s, nn, h->D, P, h->W0, h->sc, h->red);
  phase_end(h);
  for (int k = 0; k < h->mmax; ++k) {
    phase_begin(h, PH_KRY_BLAS);
    const double* src = (k == 0) ? h->W0 : h->Wk[k - 1];
    launch_krylov_orth(s, nn, k, h->Vk, src, h->Vk[k], h->sc, h->red, h->coef);
    phase_end(h);
    phase_begin(h, PH_KRY_FOCK);
    launch_pack_diag(s, m, h->Vk[k], h->Vd, &h->sc->active);
    launch_build_fock(s, m, pd, h->tab, h->Vk[k], h->Vd, nullptr, h->F1, &h->sc->active);
    phase_end(h);
    phase_begin(h, PH_KRY_GEMM);
    dmpt(h, h->F1, h->D1);
    phase_end(h);
    phase_begin(h, PH_KRY_BLAS);
    launch_krylov_w(s, nn, k, h->D1, h->Vk[k], h->Wk[k], h->Wk, h->W0, h->sc, h->red, h->cfg.krylov_tol,
                    h->cfg.m_min);
    phase_end(h);
  }
  phase_begin(h, PH_KRY_BLAS);
  launch_krylov_combine(s, nn, h->mmax, h->Vk, h->sc, h->K);
  phase_end(h);
}

// Evaluate everything at (R, X(t)): pair blocks, F, D0, U, forces, Krylov kernel.
static int evaluate(sim_handle* h, bool krylov = true, bool pairs_ready = false) {
  cudaStream_t s = h->stream;
  int n = h->n;
  size_t nn = (size_t)n * n;
  const double* X = xslot(h, 0);
  MolDev m = mol(h);
  PairDev pd = pairs(h);
  if (!pairs_ready) {
    phase_begin(h, PH_PAIRS);
    launch_pair_derivs(s, h->npair, h->pA, h->pB, h->elem, h->R, h->tab, h->W, h->S, h->E, h->dW, h->dS,
                       h->dE, mixed(h));
    phase_end(h);
  }
  phase_begin(h, PH_FOCK);
  if (!pairs_ready) launch_build_h(s, m, pd, h->tab, h->h);
  launch_pack_diag(s, m, X, h->Pd);
  launch_build_fock(s, m, pd, h->tab, X, h->Pd, h->h, h->Fock);
  phase_end(h);
  const bool conc = concurrent(h);
  int rc = eig(h, conc);
  if (rc) {
    if (conc) join_side(h, 0);
    return rc;
  }
  phase_begin(h, PH_DENSITY);
  if (conc)
    join_side(h, 0);
  else
    launch_fermi(s, n, h->eps, (double)h->nocc, h->beta, h->f, h->sc);
  density(h);
  phase_end(h);
  // energy, forces and dipole read D0 and write nothing the Krylov kernel
  // reads: side stream, own reduction workspace
  cudaStream_t fs = conc ? h->side : s;
  if (conc) fork_side(h, 1);
  phase_begin(h, PH_FORCES);
  launch_energy(fs, n, h->npair, h->h, h->D, X, h->Fock, h->E, h->sc, h->red2);
  launch_pack_diag(fs, m, h->D, h->Dd);
  launch_forces(fs, m, pd, h->tab, h->D, X, h->Dd, h->Pd, h->g, h->F);
  launch_dipole(fs, m, h->tab, h->R, h->Dd, h->sc);
  phase_end(h);
  if (!krylov) {
    if (conc) join_side(h, 1);
    return SIM_OK;
  }
  if (h->cfg.kernel == SIM_KERNEL_XL) {
    phase_begin(h, PH_KRY_BLAS);
    launch_scaled_residual(s, nn, h->D, X, h->cfg.xl_c, h->W0, h->K, h->sc, h->red);   // -c (D0 - X)
    phase_end(h);
  } else {
    krylov_kernel(h, X);   // K (D0 - X), eqs. 31-34
  }
  if (conc) join_side(h, 1);
  phase_begin(h, PH_KRY_BLAS);
  launch_check_finite(s, (size_t)3 * h->N, h->F, h->sc);
  launch_check_finite(s, nn, h->K, h->sc);
  phase_end(h);
  return SIM_OK;
}

__global__ void record_kernel(const Scalars* sc, double Te, sim_step_result* base, int* idx, int cap) {
  const int i = *idx;
  *idx = i + 1;
  sim_step_result* out = base + (i % cap);
  sim_step_result r;
  r.E_kin = sc->e_kin;
  r.U = sc->e_elec - 2.0 * Te * sc->entropy + sc->vnn;
  r.E_tot = r.E_kin + r.U;
  r.mu = sc->mu;
  r.gap = sc->gap;
  r.res_norm = ::sqrt(sc->res2);
  r.fit_err = sc->fit;
  r.rank = sc->rank;
  r.pad = sc->status;
  for (int k = 0; k < 3; ++k) r.dipole[k] = sc->dipole[k];
  *out = r;
}

static void record(sim_handle* h) {
  record_kernel<<<1, 1, 0, h->stream>>>(h->sc, h->cfg.Te, h->rec, h->rec_idx, kRecCap);
  count_launch();
  h->rec_count += 1;
}

static void reset_records(sim_handle* h) {
  cudaMemsetAsync(h->rec_idx, 0, sizeof(int), h->stream);
  h->rec_count = 0;
}

extern "C" {
static int scf(sim_handle* h, int* iters, bool from_current);
}

static bool langevin(const sim_handle* h) { return h->cfg.langevin_gamma > 0.0; }

// Langevin Ornstein-Uhlenbeck half step (phase 0 before the first half-kick,
// phase 1 after the second); nothing when the thermostat is off
static void thermostat_half(sim_handle* h, int phase) {
  if (!langevin(h)) return;
  launch_langevin_half(h->stream, h->N, h->V, h->mass, h->cfg.langevin_gamma, h->cfg.dt, h->cfg.langevin_T,
                       h->cfg.langevin_seed, phase, h->sc);
}

// Born-Oppenheimer step (comparison mode, Results: BOMD reusing the previous
// density): Verlet with forces at the SCF ground state of each geometry.
static int bomd_step(sim_handle* h) {
  cudaStream_t s = h->stream;
  double dt = h->cfg.dt;
  phase_begin(h, PH_UPDATE);
  thermostat_half(h, 0);
  launch_half_kick(s, h->N, h->V, h->F, h->mass, dt);     // eq. 27
  launch_drift(s, h->N, h->R, h->V, dt);                  // eq. 28
  phase_end(h);
  phase_begin(h, PH_PAIRS);
  launch_pair_derivs(s, h->npair, h->pA, h->pB, h->elem, h->R, h->tab, h->W, h->S, h->E, h->dW, h->dS, h->dE,
                     mixed(h));
  launch_build_h(s, mol(h), pairs(h), h->tab, h->h);
  phase_end(h);
  int it = 0;
  int rc = scf(h, &it, true);                             // from the previous density
  if (rc) return rc;
  rc = evaluate(h, false, true);                          // forces and energy at X = D_scf
  if (rc) return rc;
  phase_begin(h, PH_KRY_BLAS);
  launch_krylov_start(s, (size_t)h->n * h->n, h->D, xslot(h, 0), h->W0, h->sc, h->red);   // ||D0 - X||
  phase_end(h);
  phase_begin(h, PH_UPDATE);
  launch_half_kick(s, h->N, h->V, h->F, h->mass, dt);     // eq. 30
  thermostat_half(h, 1);
  if (langevin(h)) launch_step_advance(s, h->sc);
  launch_kinetic(s, h->N, h->V, h->mass, h->sc);
  record(h);
  phase_end(h);
  return SIM_OK;
}

static int one_step(sim_handle* h) {
  if (h->cfg.kernel == SIM_KERNEL_BOMD) return bomd_step(h);
  cudaStream_t s = h->stream;
  size_t nn = (size_t)h->n * h->n;
  double dt = h->cfg.dt;
  phase_begin(h, PH_UPDATE);
  thermostat_half(h, 0);
  launch_half_kick(s, h->N, h->V, h->F, h->mass, dt);     // eq. 27
  launch_drift(s, h->N, h->R, h->V, dt);                  // eq. 28
  double* Xh[7];
  for (int k = 0; k < 7; ++k) Xh[k] = xslot(h, k);
  double* Xnew = xslot(h, 7);
  launch_x_update(s, nn, Xh, h->K, kKappa, kAlphaDamp, Xnew);   // eq. 35
  h->xhead = (h->xhead + 7) % 8;
  phase_end(h);
  int rc = evaluate(h);
  if (rc) return rc;
  phase_begin(h, PH_UPDATE);
  launch_half_kick(s, h->N, h->V, h->F, h->mass, dt);     // eq. 30
  thermostat_half(h, 1);
  if (langevin(h)) launch_step_advance(s, h->sc);
  launch_kinetic(s, h->N, h->V, h->mass, h->sc);
  record(h);
  phase_end(h);
  return SIM_OK;
}

// Capture one step per ring phase into CUDA graphs (kernels and copies only:
// the step has no host synchronisation and no allocation).
static int capture_graphs(sim_handle* h) {
  const bool prof = h->prof;
  h->prof = false;
  const int head = h->xhead;
  const long long rc0 = h->rec_count;
  int rc = SIM_OK;
  for (int p = 0; p < 8 && rc == SIM_OK; ++p) {
    h->xhead = p;
    long long c0 = g_launches.load();
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = fail(SIM_EINTERNAL, "cudaStreamBeginCapture failed");
      break;
    }
    int st = one_step(h);
    cudaError_t ee = cudaStreamEndCapture(h->stream, &g);
    if (st != SIM_OK || ee != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      rc = fail(SIM_EINTERNAL, std::string("graph capture of a step failed: ") + cudaGetErrorString(ee));
      break;
    }
    cudaError_t ie = cudaGraphInstantiate(&h->gexec[p], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      h->gexec[p] = nullptr;
      rc = fail(SIM_EINTERNAL, std::string("graph instantiation failed: ") + cudaGetErrorString(ie));
      break;
    }
    long long nodes = g_launches.load() - c0;
    g_launches.fetch_sub(nodes);   // captured, not launched
    h->gnodes[p] = nodes;
  }
  h->xhead = head;
  h->rec_count = rc0;
  h->prof = prof;
  if (rc != SIM_OK)
    for (int p = 0; p < 8; ++p)
      if (h->gexec[p]) { cudaGraphExecDestroy(h->gexec[p]); h->gexec[p] = nullptr; }
  return rc;
}

// one step: graph replay when enabled, else direct launches
static int launch_step(sim_handle* h) {
  if (h->graphs && !h->prof) {
    const int p = h->xhead;
    CUDA_TRY(cudaGraphLaunch(h->gexec[p], h->stream));
    g_launches.fetch_add(h->gnodes[p]);
    h->xhead = (p + 7) % 8;
    h->rec_count += 1;
    return SIM_OK;
  }
  return one_step(h);
}

static int check_status(sim_handle* h) {
  int st = 0, tce = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, &h->sc->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  if (mixed(h)) CUDA_TRY(cudaMemcpyAsync(&tce, tc_error_flag(h->tw), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  CUDA_TRY(cudaGetLastError());
  if (st || tce) {
    // an error is reported once: the device words are cleared for the next call
    CUDA_TRY(cudaMemsetAsync(&h->sc->status, 0, sizeof(int), h->stream));
    if (mixed(h)) CUDA_TRY(cudaMemsetAsync(tc_error_flag(h->tw), 0, sizeof(int), h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
  }
  if (tce) return fail(SIM_ETIMEOUT, "a bounded tensor-core pipeline wait expired");
  if (st & kStatusTimeout) return fail(SIM_ETIMEOUT, "a bounded device-side wait expired");
  if (st & kStatusNumeric) return fail(SIM_ENUMERIC, "NaN or Inf in forces or kernel result");
  return SIM_OK;
}

// ---------------------------------------------------------------------------
// allocation
// ---------------------------------------------------------------------------
struct Arena {
  char* base;
  size_t off, cap;
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    T* p = (T*)(base ? base + off : nullptr);
    off += bytes;
    return p;
  }
};

static void layout(sim_handle* h, Arena& a) {
  size_t nn = (size_t)h->n * h->n;
  size_t np = (size_t)(h->npair > 0 ? h->npair : 1);
  h->elem = a.take<int>(h->N);
  h->off = a.take<int>(h->N + 1);
  h->pA = a.take<int>(np);
  h->pB = a.take<int>(np);
  h->R = a.take<double>(3 * h->N);
  h->V = a.take<double>(3 * h->N);
  h->F = a.take<double>(3 * h->N);
  h->mass = a.take<double>(h->N);
  h->g = a.take<double>(3 * np);
  h->W = a.take<double>(100 * np);
  h->S = a.take<double>(16 * np);
  h->E = a.take<double>(np);
  h->dW = a.take<double>(300 * np);
  h->dS = a.take<double>(48 * np);
  h->dE = a.take<double>(3 * np);
  h->cw = a.take<double>(10 * (size_t)h->N * h->N);
  h->h = a.take<double>(nn);
  h->Fock = a.take<double>(nn);
  h->D = a.take<double>(nn);
  h->K = a.take<double>(nn);
  h->Q = a.take<double>(nn);
  h->Qs = a.take<double>(nn);
  h->T1 = a.take<double>(nn);
  h->T2 = a.take<double>(nn);
  h->F1 = a.take<double>(nn);
  h->Y = a.take<double>(nn);
  h->D1 = a.take<double>(nn);
  h->W0 = a.take<double>(nn);
  for (int k = 0; k < 8; ++k) h->X[k] = a.take<double>(nn);
  for (int k = 0; k < h->mmax; ++k) {
    h->Vk[k] = a.take<double>(nn);
    h->Wk[k] = a.take<double>(nn);
  }
  h->eps = a.take<double>(h->n);
  h->f = a.take<double>(h->n);
  h->Dd = a.take<double>(10 * (size_t)h->N);
  h->Pd = a.take<double>(10 * (size_t)h->N);
  h->Vd = a.take<double>(10 * (size_t)h->N);
  h->red = a.take<double>(kReduceWorkDoubles);
  h->red2 = a.take<double>(kReduceWorkDoubles);
  h->coef = a.take<double>(64);
  h->sc = a.take<Scalars>(1);
  h->rec = a.take<sim_step_result>(kRecCap);
  h->rec_idx = a.take<int>(4);
  void* ewb = a.take<char>(eig_work_bytes(h->n));
  if (a.base) eig_work_bind(h->ew, ewb, h->n);
  if (h->cfg.precision == SIM_PREC_MIXED) {
    void* twb = a.take<char>(tc_work_bytes(h->n));
    if (a.base) tc_work_bind(h->tw, twb, h->n);
  }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void sim_config_default(sim_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->Te = 1000.0;
  c->dt = 0.5;
  c->m_max = 4;
  c->m_min = 4;
  c->krylov_tol = 0.0;
  c->precision = SIM_PREC_FP64;
  c->scf_tol = 1e-10;
  c->scf_max = 5000;
  c->scf_mix = 0.1;
  c->scf_krylov = 0;
  c->kernel = SIM_KERNEL_KRYLOV;
  c->xl_c = 1.0;
  c->langevin_gamma = 0.0;
  c->langevin_T = 300.0;
  c->langevin_seed = 0;
  c->device = 0;
  c->stream = nullptr;
}

const char* sim_last_error(void) { return t_err.c_str(); }
long long sim_launch_count(void) { return g_launches.load(); }
int sim_norb(const sim_handle* h) { return h ? h->n : -1; }
int sim_scf_info(const sim_handle* h, int* iterations, double* residual) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (iterations) *iterations = h->scf_iters;
  if (residual) *residual = h->scf_residual;
  return SIM_OK;
}
int sim_nocc(const sim_handle* h) { return h ? h->nocc : -1; }
void* sim_stream(sim_handle* h) { return h ? (void*)h->stream : nullptr; }

// Ground state at t0 (Results, "SCF Optimization"): linear mixing
// P <- mix P + (1 - mix) D[P], or, with scf_krylov != 0, the low-rank Krylov
// (Newton-like) update P <- P - K (D[P] - P) built from the same DMPT
// responses as the MD kernel.  Stops when max|D[P] - P| < scf_tol.
// from_current: start from X(t) (BOMD reusing the previous density) instead of
// the diagonal guess.
static int scf(sim_handle* h, int* iters, bool from_current = false) {
  cudaStream_t s = h->stream;
  int n = h->n;
  size_t nn = (size_t)n * n;
  MolDev m = mol(h);
  PairDev pd = pairs(h);
  double* P = xslot(h, 0);
  double* Dn = h->D;
  double* err_d = h->coef + 48;
  const bool trace = getenv("KSAXL_SCF_TRACE") != nullptr;
  if (!from_current) {
    // diagonal guess: valence electrons spread over each atom's orbitals, trace N_occ
    std::vector<double> P0(nn, 0.0);
    double tr = 0.0;
    for (int A = 0; A < h->N; ++A) {
      int o = h->off_h[A], no = h->off_h[A + 1] - o;
      double v = 0.5 * h->tab.e[h->elem_h[A]].zcore / no;
      for (int k = 0; k < no; ++k) { P0[(size_t)(o + k) * n + o + k] = v; tr += v; }
    }
    for (int i = 0; i < n; ++i) P0[(size_t)i * n + i] *= h->nocc / tr;
    CUDA_TRY(cudaMemcpyAsync(P, P0.data(), nn * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  double mix = h->cfg.scf_mix;
  double best = 1e300;
  double err = 0.0;
  for (int it = 0; it < h->cfg.scf_max; ++it) {
    launch_pack_diag(s, m, P, h->Pd);
    launch_build_fock(s, m, pd, h->tab, P, h->Pd, h->h, h->Fock);
    int rc = eig(h);
    if (rc) return rc;
    launch_fermi(s, n, h->eps, (double)h->nocc, h->beta, h->f, h->sc);
    density(h);
    launch_maxabs_diff(s, nn, Dn, P, err_d, h->red);
    CUDA_TRY(cudaMemcpyAsync(&err, err_d, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    int st = 0;
    CUDA_TRY(cudaMemcpy(&st, &h->sc->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (trace) fprintf(stderr, "scf %4d  max|D-P| = %.3e\n", it, err);
    if (st & kStatusTimeout) return fail(SIM_ETIMEOUT, "eigensolver barrier timed out during SCF");
    if (!std::isfinite(err)) return fail(SIM_ENUMERIC, "NaN during SCF");
    if (err < h->cfg.scf_tol) {
      CUDA_TRY(cudaMemcpyAsync(P, Dn, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
      *iters = it;
      h->scf_iters = it;
      h->scf_residual = err;
      return SIM_OK;
    }
    if (err < best) {
      best = err;
      CUDA_TRY(cudaMemcpyAsync(xslot(h, 1), P, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));  // best P
    }
    if (h->cfg.scf_krylov && err < 10.0 * best) {
      krylov_kernel(h, P);
      launch_axpby(s, nn, 1.0, P, -1.0, h->K, P);      // P <- P - K (D - P)
    } else {
      launch_axpby(s, nn, mix, P, 1.0 - mix, Dn, P);   // linear mixing
    }
  }
  h->scf_iters = h->cfg.scf_max;
  h->scf_residual = best;
  if (h->cfg.scf_accept) {
    CUDA_TRY(cudaMemcpyAsync(P, xslot(h, 1), nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    *iters = h->cfg.scf_max;
    return SIM_OK;
  }
  char msg[160];
  snprintf(msg, sizeof msg, "SCF did not converge within %d iterations (max|D-P| = %.3e)", h->cfg.scf_max, err);
  return fail(SIM_ENOCONV, msg);
}

int sim_create(const sim_config* cfg, const sim_param_table* table, int natoms, const int* Z,
               const double* R, const double* V, int charge, const double* P0, sim_handle** out) {
  if (!cfg || !table || !Z || !R || !out || natoms < 1) return fail(SIM_EINVAL, "null argument or natoms < 1");
  *out = nullptr;
  if (!(cfg->Te > 0.0) || !(cfg->dt > 0.0) || cfg->m_max < 1 || cfg->m_max > 16 || cfg->m_min < 1 ||
      cfg->m_min > cfg->m_max || cfg->scf_max < 1 || !(cfg->scf_mix >= 0.0 && cfg->scf_mix < 1.0) ||
      (cfg->kernel != SIM_KERNEL_KRYLOV && cfg->kernel != SIM_KERNEL_XL && cfg->kernel != SIM_KERNEL_BOMD) ||
      !std::isfinite(cfg->xl_c) || !(cfg->langevin_gamma >= 0.0) || !std::isfinite(cfg->langevin_gamma) ||
      !(cfg->langevin_T >= 0.0) || !std::isfinite(cfg->langevin_T))
    return fail(SIM_EINVAL, "invalid configuration");
  if (cfg->precision != SIM_PREC_FP64 && cfg->precision != SIM_PREC_MIXED)
    return fail(SIM_EINVAL, "unknown precision mode");
  if (cfg->precision == SIM_PREC_MIXED && !tc_available())
    return fail(SIM_EINVAL, "mixed precision needs the tensor-map driver entry point (tcgen05/TMA path)");
  sim_handle* h = new sim_handle();
  h->cfg = *cfg;
  h->table_raw = *table;
  h->Z_h.assign(Z, Z + natoms);
  h->charge = charge;
  for (int e = 0; e < 4; ++e)
    if (build_elem(table->v[e], h->tab.e[e]) != 0) {
      delete h;
      return fail(SIM_EINVAL, "parameter table: norb/nprin must be (1,1) for H and (4,2) otherwise");
    }
  h->N = natoms;
  h->elem_h.resize(natoms);
  h->off_h.resize(natoms + 1);
  h->mass_h.resize(natoms);
  double zsum = 0.0;
  h->off_h[0] = 0;
  for (int A = 0; A < natoms; ++A) {
    int ei = elem_index(Z[A]);
    if (ei < 0) { delete h; return fail(SIM_EINVAL, "unsupported atomic number " + std::to_string(Z[A])); }
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(R[3 * A + k]) || (V && !std::isfinite(V[3 * A + k]))) {
        delete h;
        return fail(SIM_EINVAL, "non-finite position or velocity");
      }
    h->elem_h[A] = ei;
    h->off_h[A + 1] = h->off_h[A] + h->tab.e[ei].norb;
    h->mass_h[A] = h->tab.e[ei].mass;
    zsum += h->tab.e[ei].zcore;
  }
  h->n = h->off_h[natoms];
  long long nel = std::llround(zsum) - charge;
  if (nel < 0 || nel % 2 != 0 || nel / 2 > h->n) {
    delete h;
    return fail(SIM_EINVAL, "electron count must be even, non-negative and fit the basis (closed shell)");
  }
  h->nocc = (int)(nel / 2);
  h->npair = natoms * (natoms - 1) / 2;
  h->mmax = cfg->m_max;
  h->beta = 1.0 / (kBoltz * cfg->Te);
  h->dev = cfg->device;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || h->dev < 0 || h->dev >= ndev) {
    cudaGetLastError();
    delete h;
    return fail(SIM_EINVAL, "no such CUDA device: " + std::to_string(cfg->device));
  }
  DeviceGuard dg(h->dev);   // the caller's current device is restored on every return
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev);
  if (!upload_overlap_tables()) { delete h; return fail(SIM_EINTERNAL, "overlap table upload failed"); }
  if (cfg->stream) {
    h->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return fail(SIM_EINTERNAL, "stream creation failed");
    }
    h->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    h->side = nullptr;
  }
  for (int k = 0; k < 2 && h->side; ++k)
    if (cudaEventCreateWithFlags(&h->fork_ev[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->join_ev[k], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      sim_destroy(h);
      return fail(SIM_EINTERNAL, "event creation failed");
    }
  Arena sizing{nullptr, 0, 0};
  layout(h, sizing);
  h->arena_bytes = sizing.off + 256;
  // stream-ordered allocation: creating or destroying a handle does not
  // synchronise the device (other handles keep running)
  if (cudaMallocAsync(&h->arena, h->arena_bytes, h->stream) != cudaSuccess) {
    cudaGetLastError();
    size_t need = h->arena_bytes;
    sim_destroy(h);
    return fail(SIM_ENOMEM, "device allocation of " + std::to_string(need) + " bytes failed");
  }
  // the arena is used from other streams below (synchronous copies): wait for it
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    sim_destroy(h);
    return fail(SIM_EINTERNAL, "stream synchronisation after allocation failed");
  }
  Arena a{(char*)h->arena, 0, h->arena_bytes};
  layout(h, a);
  if (mixed(h) && !tc_ready(h->tw)) {
    sim_destroy(h);
    return fail(SIM_EINTERNAL, "tensor map encoding failed for the BF16 operand pieces");
  }
  cudaStream_t s = h->stream;
  std::vector<int> pa, pb;
  pa.reserve(h->npair);
  pb.reserve(h->npair);
  for (int A = 0; A < natoms; ++A)
    for (int B = A + 1; B < natoms; ++B) { pa.push_back(A); pb.push_back(B); }
  std::vector<double> v0(3 * (size_t)natoms, 0.0);
  if (V) std::memcpy(v0.data(), V, v0.size() * sizeof(double));
  int rc = SIM_OK;
  do {
    if (cudaMemsetAsync(h->sc, 0, sizeof(Scalars), s) != cudaSuccess) { rc = fail(SIM_EINTERNAL, "memset"); break; }
    cudaMemcpyAsync(h->elem, h->elem_h.data(), natoms * sizeof(int), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->off, h->off_h.data(), (natoms + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
    if (h->npair) {
      cudaMemcpyAsync(h->pA, pa.data(), h->npair * sizeof(int), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(h->pB, pb.data(), h->npair * sizeof(int), cudaMemcpyHostToDevice, s);
    }
    cudaMemcpyAsync(h->R, R, 3 * (size_t)natoms * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->V, v0.data(), 3 * (size_t)natoms * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->mass, h->mass_h.data(), natoms * sizeof(double), cudaMemcpyHostToDevice, s);
    launch_fill(s, (size_t)h->n * h->n, h->K, 0.0);
    // pair blocks and h at R0
    launch_pair_derivs(s, h->npair, h->pA, h->pB, h->elem, h->R, h->tab, h->W, h->S, h->E, h->dW, h->dS, h->dE,
                     mixed(h));
    launch_build_h(s, mol(h), pairs(h), h->tab, h->h);
    size_t nn = (size_t)h->n * h->n;
    if (P0) {
      for (size_t i = 0; i < nn; ++i)
        if (!std::isfinite(P0[i])) { rc = fail(SIM_EINVAL, "non-finite P0"); break; }
      if (rc) break;
      cudaMemcpyAsync(xslot(h, 0), P0, nn * sizeof(double), cudaMemcpyHostToDevice, s);
    } else {
      int it = 0;
      rc = scf(h, &it);
      if (rc) break;
    }
    for (int k = 1; k < 7; ++k)
      cudaMemcpyAsync(xslot(h, k), xslot(h, 0), nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    rc = evaluate(h, cfg->kernel != SIM_KERNEL_BOMD);
    if (rc) break;
    launch_kinetic(s, h->N, h->V, h->mass, h->sc);
    reset_records(h);
    record(h);
    rc = check_status(h);
  } while (0);
  if (rc != SIM_OK) {
    std::string msg = t_err;
    sim_destroy(h);
    t_err = msg;
    return rc;
  }
  *out = h;
  return SIM_OK;
}

int sim_step_async(sim_handle* h, int nsteps) {
  if (!h || nsteps < 0) return fail(SIM_EINVAL, "bad handle or nsteps");
  DeviceGuard dg(h->dev);
  for (int i = 0; i < nsteps; ++i) {
    int rc = launch_step(h);
    if (rc) return rc;
  }
  return SIM_OK;
}

int sim_step(sim_handle* h, int nsteps, sim_step_result* out) {
  if (!h || nsteps < 0) return fail(SIM_EINVAL, "bad handle or nsteps");
  DeviceGuard dg(h->dev);
  int done = 0;
  while (done < nsteps) {
    int chunk = nsteps - done;
    if (chunk > kRecCap) chunk = kRecCap;
    reset_records(h);
    for (int i = 0; i < chunk; ++i) {
      int rc = launch_step(h);
      if (rc) return rc;
    }
    if (out) {
      CUDA_TRY(cudaMemcpyAsync(out + done, h->rec, chunk * sizeof(sim_step_result), cudaMemcpyDeviceToHost,
                               h->stream));
    }
    int rc = check_status(h);
    if (rc) return rc;
    done += chunk;
  }
  if (h->prof) collect_events(h);
  return SIM_OK;
}

int sim_step_host(sim_handle* h, const double* R_in, const double* V_in, double* R_out, double* V_out,
                  double* F_out, sim_step_result* out) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  DeviceGuard dg(h->dev);
  cudaStream_t s = h->stream;
  size_t b3 = 3 * (size_t)h->N * sizeof(double);
  if (R_in) CUDA_TRY(cudaMemcpyAsync(h->R, R_in, b3, cudaMemcpyHostToDevice, s));
  if (V_in) CUDA_TRY(cudaMemcpyAsync(h->V, V_in, b3, cudaMemcpyHostToDevice, s));
  reset_records(h);
  int rc = launch_step(h);
  if (rc) return rc;
  if (R_out) CUDA_TRY(cudaMemcpyAsync(R_out, h->R, b3, cudaMemcpyDeviceToHost, s));
  if (V_out) CUDA_TRY(cudaMemcpyAsync(V_out, h->V, b3, cudaMemcpyDeviceToHost, s));
  if (F_out) CUDA_TRY(cudaMemcpyAsync(F_out, h->F, b3, cudaMemcpyDeviceToHost, s));
  if (out) CUDA_TRY(cudaMemcpyAsync(out, h->rec, sizeof(sim_step_result), cudaMemcpyDeviceToHost, s));
  if (h->prof) collect_events(h);
  return check_status(h);
}

int sim_last_result(sim_handle* h, sim_step_result* out) {
  if (!h || !out) return fail(SIM_EINVAL, "null argument");
  DeviceGuard dg(h->dev);
  long long i = h->rec_count > 0 ? (h->rec_count - 1) % kRecCap : 0;
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  CUDA_TRY(cudaMemcpy(out, h->rec + i, sizeof(sim_step_result), cudaMemcpyDeviceToHost));
  return SIM_OK;
}

int sim_records(sim_handle* h, sim_step_result* out, int count) {
  if (!h || !out || count < 0) return fail(SIM_EINVAL, "bad arguments");
  DeviceGuard dg(h->dev);
  if (count > kRecCap || count > h->rec_count) return fail(SIM_EINVAL, "fewer records available than requested");
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < count; ++i) {
    long long idx = (h->rec_count - count + i) % kRecCap;
    CUDA_TRY(cudaMemcpy(out + i, h->rec + idx, sizeof(sim_step_result), cudaMemcpyDeviceToHost));
  }
  return SIM_OK;
}

int sim_wait(sim_handle* h) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  DeviceGuard dg(h->dev);
  return check_status(h);
}

size_t sim_estimate_bytes(const sim_config* cfg, int natoms, const int* Z) {
  if (!cfg || !Z || natoms < 1 || cfg->m_max < 1 || cfg->m_max > 16) return 0;
  sim_handle tmp;
  tmp.cfg = *cfg;
  tmp.N = natoms;
  int n = 0;
  for (int A = 0; A < natoms; ++A) n += (Z[A] == 1) ? 1 : 4;
  tmp.n = n;
  tmp.npair = natoms * (natoms - 1) / 2;
  tmp.mmax = cfg->m_max;
  Arena sizing{nullptr, 0, 0};
  layout(&tmp, sizing);
  return sizing.off + 256;
}

int sim_enable_graphs(sim_handle* h, int enable) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  DeviceGuard dg(h->dev);
  if (enable && h->cfg.kernel == SIM_KERNEL_BOMD)
    return fail(SIM_EINVAL, "Born-Oppenheimer steps read the SCF residual on the host and cannot be captured");
  if (enable && !h->graphs) {
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    int rc = capture_graphs(h);
    if (rc) return rc;
    h->graphs = true;
  } else if (!enable && h->graphs) {
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int p = 0; p < 8; ++p)
      if (h->gexec[p]) { cudaGraphExecDestroy(h->gexec[p]); h->gexec[p] = nullptr; }
    h->graphs = false;
  }
  return SIM_OK;
}

// ---- whole-batch graphs -----------------------------------------------------
// One CUDA graph per phase of the X ring holds one MD step of every molecule of
// the batch: each molecule's step is a branch forked from and joined back to a
// master stream, and groups of molecules whose persistent eigensolver grids fit
// on the device together follow one another inside the graph.
struct sim_batch {
  std::vector<sim_handle*> hs;
  std::vector<int> group_end;            // exclusive end index of each group
  cudaStream_t master = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t gexec[8] = {};
  long long gnodes[8] = {};
};

static void batch_release(sim_batch* b) {
  if (!b) return;
  DeviceGuard dg(b->hs.empty() ? 0 : b->hs[0]->dev);
  if (b->master) cudaStreamSynchronize(b->master);
  for (int p = 0; p < 8; ++p)
    if (b->gexec[p]) cudaGraphExecDestroy(b->gexec[p]);
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->master) cudaStreamDestroy(b->master);
  delete b;
}

static int batch_capture(sim_batch* b, int p) {
  const int count = (int)b->hs.size();
  for (auto* h : b->hs) h->xhead = p;
  long long c0 = g_launches.load();
  CUDA_TRY(cudaStreamBeginCapture(b->master, cudaStreamCaptureModeThreadLocal));
  int rc = SIM_OK;
  int g0 = 0;
  for (size_t g = 0; g < b->group_end.size() && rc == SIM_OK; ++g) {
    const int g1 = b->group_end[g];
    if (cudaEventRecord(b->fork, b->master) != cudaSuccess) rc = SIM_EINTERNAL;
    for (int i = g0; i < g1 && rc == SIM_OK; ++i)
      if (cudaStreamWaitEvent(b->hs[i]->stream, b->fork, 0) != cudaSuccess) rc = SIM_EINTERNAL;
    for (int i = g0; i < g1 && rc == SIM_OK; ++i) rc = one_step(b->hs[i]);
    for (int i = g0; i < g1 && rc == SIM_OK; ++i)
      if (cudaEventRecord(b->join[i], b->hs[i]->stream) != cudaSuccess ||
          cudaStreamWaitEvent(b->master, b->join[i], 0) != cudaSuccess)
        rc = SIM_EINTERNAL;
    g0 = g1;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(b->master, &graph);
  long long nodes = g_launches.load() - c0;
  g_launches.fetch_sub(nodes);
  for (auto* h : b->hs) h->rec_count -= 1;   // one_step counted a record per molecule
  if (rc != SIM_OK || ee != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return fail(SIM_EINTERNAL, std::string("capture of the batch step failed: ") + cudaGetErrorString(ee));
  }
  cudaError_t ie = cudaGraphInstantiate(&b->gexec[p], graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    b->gexec[p] = nullptr;
    return fail(SIM_EINTERNAL, std::string("batch graph instantiation failed: ") + cudaGetErrorString(ie));
  }
  b->gnodes[p] = nodes;
  (void)count;
  return SIM_OK;
}

int sim_batch_groups(const sim_batch* b) { return b ? (int)b->group_end.size() : 0; }

int sim_batch_create(sim_handle* const* hs, int count, sim_batch** out) {
  if (!hs || count < 1 || !out) return fail(SIM_EINVAL, "bad batch arguments");
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return fail(SIM_EINVAL, "null handle in batch");
    if (hs[i]->xhead != hs[0]->xhead) return fail(SIM_EINVAL, "batch members must have taken the same number of steps");
    if (hs[i]->cfg.kernel == SIM_KERNEL_BOMD) return fail(SIM_EINVAL, "Born-Oppenheimer steps cannot be captured");
    if (hs[i]->prof) return fail(SIM_EINVAL, "phase profiling is on for a batch member");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i] || hs[j]->stream == hs[i]->stream)
        return fail(SIM_EINVAL, "batch members need distinct handles on distinct streams");
  }
  DeviceGuard dg(hs[0]->dev);
  sim_batch* b = new sim_batch();
  b->hs.assign(hs, hs + count);
  const long long cap = 1000LL * hs[0]->sms;
  long long load = 0;
  for (int i = 0; i < count; ++i) {
    long long w = eig_tridiag_weight(hs[i]->n, hs[i]->sms);
    if (i > 0 && load + w > cap) {
      b->group_end.push_back(i);
      load = 0;
    }
    load += w;
  }
  b->group_end.push_back(count);
  b->join.assign(count, nullptr);
  int rc = SIM_OK;
  if (cudaStreamCreateWithFlags(&b->master, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    rc = fail(SIM_EINTERNAL, "stream or event creation failed");
  for (int i = 0; i < count && rc == SIM_OK; ++i)
    if (cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess)
      rc = fail(SIM_EINTERNAL, "event creation failed");
  for (int i = 0; i < count && rc == SIM_OK; ++i)
    if (cudaStreamSynchronize(hs[i]->stream) != cudaSuccess) rc = fail(SIM_EINTERNAL, "synchronisation failed");
  const int head = hs[0]->xhead;
  for (int p = 0; p < 8 && rc == SIM_OK; ++p) rc = batch_capture(b, p);
  for (auto* h : b->hs) h->xhead = head;
  if (rc != SIM_OK) {
    std::string msg = t_err;
    batch_release(b);
    t_err = msg;
    return rc;
  }
  *out = b;
  return SIM_OK;
}

int sim_batch_run(sim_batch* b, int nsteps) {
  if (!b || nsteps < 0) return fail(SIM_EINVAL, "bad batch run arguments");
  DeviceGuard dg(b->hs[0]->dev);
  for (auto* h : b->hs) {
    if (h->xhead != b->hs[0]->xhead) return fail(SIM_EINVAL, "a batch member was stepped on its own");
    reset_records(h);
    // the members' streams must be idle before the graph writes their buffers
    CUDA_TRY(cudaStreamSynchronize(h->stream));
  }
  for (int k = 0; k < nsteps; ++k) {
    const int p = b->hs[0]->xhead;
    CUDA_TRY(cudaGraphLaunch(b->gexec[p], b->master));
    g_launches.fetch_add(b->gnodes[p]);
    for (auto* h : b->hs) {
      h->xhead = (p + 7) % 8;
      h->rec_count += 1;
    }
  }
  CUDA_TRY(cudaStreamSynchronize(b->master));
  int first = SIM_OK;
  for (auto* h : b->hs) {
    int rc = check_status(h);
    if (rc && first == SIM_OK) first = rc;
  }
  return first;
}

void sim_batch_destroy(sim_batch* b) { batch_release(b); }

int sim_batch_step(sim_handle* const* hs, int count, int nsteps) {
  if (!hs || count < 0 || nsteps < 0) return fail(SIM_EINVAL, "bad batch arguments");
  for (int i = 0; i < count; ++i)
    if (!hs[i]) return fail(SIM_EINVAL, "null handle in batch");
  DeviceGuard dg(count > 0 ? hs[0]->dev : -1);
  int first = SIM_OK;
  // groups of consecutive handles whose persistent eigensolver grids fit on
  // the device at the same time (their grid barriers need every block resident)
  for (int g0 = 0; g0 < count;) {
    const long long cap = 1000LL * hs[g0]->sms;
    long long load = 0;
    int g1 = g0;
    while (g1 < count) {
      long long w = eig_tridiag_weight(hs[g1]->n, hs[g1]->sms);
      if (g1 > g0 && load + w > cap) break;
      load += w;
      ++g1;
    }
    // interleave the group's handles step by step: each runs on its own stream,
    // so the device overlaps the (mostly latency-bound) steps of small systems
    for (int k = 0; k < nsteps; ++k)
      for (int i = g0; i < g1; ++i) {
        if (k == 0) reset_records(hs[i]);
        int rc = launch_step(hs[i]);
        if (rc) return rc;
      }
    for (int i = g0; i < g1; ++i) {
      int rc = check_status(hs[i]);
      if (rc && first == SIM_OK) first = rc;
    }
    g0 = g1;
  }
  return first;
}

int sim_get_state(sim_handle* h, double* R, double* V, double* F, double* D0) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  DeviceGuard dg(h->dev);
  cudaStream_t s = h->stream;
  size_t b3 = 3 * (size_t)h->N * sizeof(double);
  if (R) CUDA_TRY(cudaMemcpyAsync(R, h->R, b3, cudaMemcpyDeviceToHost, s));
  if (V) CUDA_TRY(cudaMemcpyAsync(V, h->V, b3, cudaMemcpyDeviceToHost, s));
  if (F) CUDA_TRY(cudaMemcpyAsync(F, h->F, b3, cudaMemcpyDeviceToHost, s));
  if (D0) CUDA_TRY(cudaMemcpyAsync(D0, h->D, (size_t)h->n * h->n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return SIM_OK;
}

int sim_set_state(sim_handle* h, const double* R, const double* V, const double* Xhist) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  DeviceGuard dg(h->dev);
  cudaStream_t s = h->stream;
  size_t nn = (size_t)h->n * h->n;
  size_t b3 = 3 * (size_t)h->N * sizeof(double);
  if (R) CUDA_TRY(cudaMemcpyAsync(h->R, R, b3, cudaMemcpyHostToDevice, s));
  if (V) CUDA_TRY(cudaMemcpyAsync(h->V, V, b3, cudaMemcpyHostToDevice, s));
  if (Xhist)
    for (int k = 0; k < 7; ++k)
      CUDA_TRY(cudaMemcpyAsync(xslot(h, k), Xhist + k * nn, nn * sizeof(double), cudaMemcpyHostToDevice, s));
  int rc = evaluate(h, h->cfg.kernel != SIM_KERNEL_BOMD);
  if (rc) return rc;
  launch_kinetic(s, h->N, h->V, h->mass, h->sc);
  reset_records(h);
  record(h);
  return check_status(h);
}

// ---- checkpoint / resume ----------------------------------------------------
static const char kCkptMagic[8] = {'K', 'S', 'A', 'X', 'L', 'C', 'K', '1'};

int sim_save(sim_handle* h, const char* path) {
  if (!h || !path) return fail(SIM_EINVAL, "null argument");
  DeviceGuard dg(h->dev);
  size_t nn = (size_t)h->n * h->n;
  std::vector<double> R(3 * (size_t)h->N), V(3 * (size_t)h->N), X(7 * nn);
  cudaStream_t s = h->stream;
  CUDA_TRY(cudaMemcpyAsync(R.data(), h->R, R.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(V.data(), h->V, V.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  for (int k = 0; k < 7; ++k)
    CUDA_TRY(cudaMemcpyAsync(X.data() + k * nn, xslot(h, k), nn * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(SIM_EINVAL, std::string("cannot open ") + path + " for writing");
  sim_config cfg = h->cfg;
  cfg.stream = nullptr;
  unsigned long long step = 0;
  CUDA_TRY(cudaMemcpy(&step, &h->sc->step, sizeof(step), cudaMemcpyDeviceToHost));
  int head[4] = {2 /*version*/, h->N, h->n, h->charge};
  bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(head, sizeof(int), 4, f) == 4 &&
            std::fwrite(&cfg, sizeof(cfg), 1, f) == 1 && std::fwrite(&h->table_raw, sizeof(sim_param_table), 1, f) == 1 &&
            std::fwrite(&step, sizeof(step), 1, f) == 1 &&
            std::fwrite(h->Z_h.data(), sizeof(int), h->N, f) == (size_t)h->N &&
            std::fwrite(R.data(), sizeof(double), R.size(), f) == R.size() &&
            std::fwrite(V.data(), sizeof(double), V.size(), f) == V.size() &&
            std::fwrite(X.data(), sizeof(double), X.size(), f) == X.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? SIM_OK : fail(SIM_EINTERNAL, std::string("short write to ") + path);
}

int sim_load(const char* path, int device, void* stream, sim_handle** out) {
  if (!path || !out) return fail(SIM_EINVAL, "null argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(SIM_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  int head[4];
  sim_config cfg;
  sim_param_table table;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkptMagic, 8) == 0 &&
            std::fread(head, sizeof(int), 4, f) == 4 && head[0] == 2 && head[1] >= 1 && head[1] <= 1000000 &&
            head[2] >= 1 && head[2] <= 4 * head[1] && std::fread(&cfg, sizeof(cfg), 1, f) == 1 &&
            std::fread(&table, sizeof(table), 1, f) == 1;
  std::vector<int> Z;
  std::vector<double> R, V, X;
  unsigned long long step = 0;
  if (ok) ok = std::fread(&step, sizeof(step), 1, f) == 1;
  if (ok) {
    const int N = head[1];
    const size_t nn = (size_t)head[2] * head[2];
    Z.resize(N);
    R.resize(3 * (size_t)N);
    V.resize(3 * (size_t)N);
    X.resize(7 * nn);
    ok = std::fread(Z.data(), sizeof(int), N, f) == (size_t)N && std::fread(R.data(), sizeof(double), R.size(), f) == R.size() &&
         std::fread(V.data(), sizeof(double), V.size(), f) == V.size() &&
         std::fread(X.data(), sizeof(double), X.size(), f) == X.size() && std::fgetc(f) == EOF;
  }
  std::fclose(f);
  if (!ok) return fail(SIM_EINVAL, std::string(path) + " is not a complete checkpoint of this library");
  cfg.device = device;
  cfg.stream = stream;
  sim_handle* h = nullptr;
  int rc = sim_create(&cfg, &table, head[1], Z.data(), R.data(), V.data(), head[3], X.data(), &h);
  if (rc) return rc;
  DeviceGuard dg(h->dev);
  if (h->n != head[2]) {
    sim_destroy(h);
    return fail(SIM_EINVAL, "checkpoint basis size does not match its atoms");
  }
  rc = sim_set_state(h, nullptr, nullptr, X.data());   // full X history, re-evaluated
  if (rc == SIM_OK && cudaMemcpy(&h->sc->step, &step, sizeof(step), cudaMemcpyHostToDevice) != cudaSuccess)
    rc = fail(SIM_EINTERNAL, "restoring the step counter failed");
  if (rc) {
    std::string msg = t_err;
    sim_destroy(h);
    t_err = msg;
    return rc;
  }
  *out = h;
  return SIM_OK;
}

int sim_get_matrix(sim_handle* h, int which, double* out) {
  if (!h || !out) return fail(SIM_EINVAL, "null argument");
  DeviceGuard dg(h->dev);
  const double* src = nullptr;
  switch (which) {
    case SIM_MAT_X: src = xslot(h, 0); break;
    case SIM_MAT_D0: src = h->D; break;
    case SIM_MAT_FOCK: src = h->Fock; break;
    case SIM_MAT_H: src = h->h; break;
    case SIM_MAT_KERNEL: src = h->K; break;
    case SIM_MAT_Q: src = h->Q; break;
    default:
      if (which >= SIM_MAT_XHIST && which <= SIM_MAT_XHIST + 6) {
        src = xslot(h, which - SIM_MAT_XHIST);
        break;
      }
      return fail(SIM_EINVAL, "unknown matrix id");
  }
  CUDA_TRY(cudaMemcpyAsync(out, src, (size_t)h->n * h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

int sim_get_vector(sim_handle* h, int which, double* out) {
  if (!h || !out) return fail(SIM_EINVAL, "null argument");
  DeviceGuard dg(h->dev);
  const double* src = (which == 0) ? h->eps : (which == 1) ? h->f : nullptr;
  if (!src) return fail(SIM_EINVAL, "unknown vector id");
  CUDA_TRY(cudaMemcpyAsync(out, src, (size_t)h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

int sim_profile_enable(sim_handle* h, int enable) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  DeviceGuard dg(h->dev);
  if (h->prof && !enable) collect_events(h);
  h->prof = enable != 0;
  for (int i = 0; i < PH_COUNT; ++i) { h->ph_ms[i] = 0.0; h->ph_n[i] = 0; }
  return SIM_OK;
}

int sim_phase_count(void) { return PH_COUNT; }
const char* sim_phase_name(int p) { return (p >= 0 && p < PH_COUNT) ? kPhaseNames[p] : ""; }

int sim_phase_times(sim_handle* h, double* ms, long long* launches, double* work) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  DeviceGuard dg(h->dev);
  collect_events(h);
  double n = h->n, np = h->npair;
  // algorithmic work of one timed phase instance (bytes for HBM-bound phases,
  // flops for arithmetic-bound ones); see the design notes for the derivation
  double w[PH_COUNT] = {
      np * (117.0 * 4.0) * 8.0,             // pair blocks + derivatives written (bytes)
      (np * 116.0 + 4.0 * n * n) * 8.0,     // h + F: pair blocks read, matrices written (bytes)
      4.0 / 3.0 * n * n * n,                // Householder tridiagonalisation, algorithmic flops
      0.0,                                  // bisection
      0.0,                                  // inverse iteration
      2.0 * n * n * n,                      // back-transformation flops
      n * n * n,                            // D0 = Q f Q^T (symmetric) flops
      np * (468.0) * 8.0,                   // force contraction bytes
      (np * 100.0 + 3.0 * n * n) * 8.0,     // G(V) bytes
      6.0 * n * n * n,                      // DMPT: 3 full + ... (2 general + 2 symmetric GEMMs)
      0.0, 0.0};
  for (int i = 0; i < PH_COUNT; ++i) {
    if (ms) ms[i] = h->ph_ms[i];
    if (launches) launches[i] = h->ph_n[i];
    if (work) work[i] = w[i];
  }
  return SIM_OK;
}

// Test hooks: C = sum of BF16-piece products of A and B^T on the tensor cores
// (terms 1, 3, 6, 10: the exact per-segment kernel; grouped: the DMPT's 3-slice kernel).
static int debug_tc_gemm(int n, const double* A, const double* B, int terms, int sym, bool grouped, double* C) {
  if (grouped && terms != 6 && terms != 10) return fail(SIM_EINVAL, "grouped products take 3 or 4 slices");
  if (n < 1 || !A || !B || !C || (terms != 1 && terms != 3 && terms != 6 && terms != 10))
    return fail(SIM_EINVAL, "bad argument");
  if (!tc_available()) return fail(SIM_EINVAL, "tensor-map entry point unavailable");
  size_t nn = (size_t)n * n;
  size_t bytes = 3 * nn * sizeof(double) + tc_work_bytes(n) + 4096;
  char* arena = nullptr;
  if (cudaMalloc(&arena, bytes) != cudaSuccess) return fail(SIM_ENOMEM, "allocation failed");
  double* dA = (double*)arena;
  double* dB = dA + nn;
  double* dC = dB + nn;
  void* tb = (void*)(((uintptr_t)(dC + nn) + 1023) & ~(uintptr_t)1023);
  TcWork w;
  tc_work_bind(w, tb, n);
  int rc = SIM_OK;
  cudaStream_t s = 0;
  int pieces = (terms == 10) ? 4 : (terms == 6) ? 3 : (terms == 3) ? 2 : 1;
  if (!tc_ready(w)) {
    rc = fail(SIM_EINTERNAL, "tensor map encoding failed");
  } else {
    cudaMemcpy(dA, A, nn * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(dB, B, nn * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemset(dC, 0, nn * sizeof(double));
    tc_split(s, w, kSlotT0, dA, pieces, 0);
    tc_split(s, w, kSlotT1, dB, pieces, 0);
    if (grouped && terms == 6)
      tc_gemm_grouped(s, w, kSlotT0, kSlotT1, 1.0, dC, sym);
    else if (grouped)
      tc_gemm_grouped4(s, w, kSlotT0, kSlotT1, 1.0, dC, sym);
    else
      tc_gemm(s, w, kSlotT0, kSlotT1, terms, 1.0, dC, sym);
    int err = 0;
    cudaError_t ce = cudaDeviceSynchronize();
    cudaMemcpy(&err, tc_error_flag(w), sizeof(int), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) rc = fail(SIM_EINTERNAL, std::string("CUDA error: ") + cudaGetErrorString(ce));
    else if (err) rc = fail(SIM_ETIMEOUT, "tensor-core pipeline wait expired");
    else cudaMemcpy(C, dC, nn * sizeof(double), cudaMemcpyDeviceToHost);
  }
  tc_work_release(w);
  cudaFree(arena);
  return rc;
}

int sim_debug_tc_gemm(int n, const double* A, const double* B, int terms, int sym, double* C) {
  return debug_tc_gemm(n, A, B, terms, sym, false, C);
}

int sim_debug_tc_gemm_grouped(int n, const double* A, const double* B, int slices, int sym, double* C) {
  if (slices != 3 && slices != 4) return fail(SIM_EINVAL, "slices must be 3 or 4");
  return debug_tc_gemm(n, A, B, slices == 3 ? 6 : 10, sym, true, C);
}

void sim_destroy(sim_handle* h) {
  if (!h) return;
  DeviceGuard dg(h->dev);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int p = 0; p < 8; ++p)
    if (h->gexec[p]) cudaGraphExecDestroy(h->gexec[p]);
  for (auto& p : h->ev_pending) { cudaEventDestroy(p.second.first); cudaEventDestroy(p.second.second); }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  if (h->tw.base) tc_work_release(h->tw);
  if (h->arena) {
    cudaFreeAsync(h->arena, h->stream);
    cudaStreamSynchronize(h->stream);
  }
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
  }
  for (int k = 0; k < 2; ++k) {
    if (h->fork_ev[k]) cudaEventDestroy(h->fork_ev[k]);
    if (h->join_ev[k]) cudaEventDestroy(h->join_ev[k]);
  }
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"
