/*
 * sim.h -- C ABI of the GB300 KSA-XL-BOMD library.
 *
 * The library advances semi-empirical (NDDO, sp basis) shadow extended-
 * Lagrangian Born-Oppenheimer molecular dynamics with the Krylov subspace
 * approximation of the kernel (arXiv 2303.00689, "Semi-Empirical Shadow
 * Molecular Dynamics: A PyTorch implementation").  One call of sim_step
 * performs, per MD step and entirely in CUDA kernels on one GPU:
 *   - the modified leap-frog velocity Verlet update with damping
 *     (eqs. 27-30, 35);
 *   - NDDO pair integrals and their derivatives, h and F(X) = h + G(X)
 *     (eqs. 3, 6, 17);
 *   - the eigendecomposition, Fermi occupations and chemical potential,
 *     D0[X] (eqs. 7, 8, 19);
 *   - the shadow energy (eq. 13) and forces (eqs. 22, 37-41);
 *   - the rank-m Krylov approximation of K(D0[X] - X) (eqs. 31-34) with
 *     canonical density-matrix perturbation theory responses (eq. 36).
 *
 * Conventions.  Units: Angstrom, fs, eV, amu, K.  Closed shell, S = I
 * (NDDO), so X = P (the paper's statement under eq. 16).  Densities D, X,
 * P are PER SPIN: Tr D = N_occ = N_electrons / 2.  Matrices are dense,
 * row-major, n x n doubles, orbitals ordered atom by atom (s, px, py, pz for
 * C/N/O; s for H).  Positions/velocities/forces are natoms x 3 row-major.
 *
 * Memory: every pointer argument is HOST memory unless its comment says
 * DEVICE.  The library copies inputs in and owns all device state of a
 * handle; results are copied into caller-owned buffers.  A handle is not
 * thread safe; different handles may be used from different threads.
 *
 * Errors: every int-returning call returns a SIM_* status.  On error the
 * handle's state is unchanged unless stated otherwise, and
 * sim_last_error() returns a message for the calling thread.
 */
#ifndef KSA_XLBOMD_SIM_H
#define KSA_XLBOMD_SIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum sim_status {
  SIM_OK = 0,
  SIM_PENDING = 1,    /* sim_poll: request not finished yet                   */
  SIM_EINVAL = 2,     /* bad argument (open shell, unknown Z, NaN, sizes)      */
  SIM_ENOMEM = 3,     /* device allocation failed or HBM budget exceeded      */
  SIM_ENOCONV = 4,    /* SCF or chemical-potential solve did not converge     */
  SIM_ENUMERIC = 5,   /* NaN/Inf detected on the device                       */
  SIM_ETIMEOUT = 6,   /* a bounded device-side wait gave up                   */
  SIM_EINTERNAL = 7,  /* CUDA error or library bug                            */
};

/* ---- precision modes ---------------------------------------------------- */
enum sim_precision {
  /* every step in FP64 (FP64 SIMT GEMMs for density and DMPT)               */
  SIM_PREC_FP64 = 0,
  /* FP64 eigensolve, mu and Krylov Gram/solve; density D0 = Q f Q^T and the
   * DMPT contractions of eq. 36 on tcgen05 tensor cores: operands cut into
   * fixed-point BF16 slices (4 for the density, 3 for DMPT; 8 bits each
   * relative to the row maximum), exact FP32 chunk sums, double-float
   * accumulation across chunks, FP64 output                                 */
  SIM_PREC_MIXED = 1,
};

/* ---- parameter table ---------------------------------------------------- */
/* One record per element, rows in the order H, C, N, O.  Field order: */
enum sim_param_field {
  SIM_P_Z = 0, SIM_P_NORB, SIM_P_NPRIN, SIM_P_ZCORE, SIM_P_MASS,
  SIM_P_USS, SIM_P_UPP, SIM_P_ZETA_S, SIM_P_ZETA_P, SIM_P_BETA_S, SIM_P_BETA_P,
  SIM_P_GSS, SIM_P_GSP, SIM_P_GPP, SIM_P_GP2, SIM_P_HSP, SIM_P_ALPHA,
  SIM_P_GA0, SIM_P_GB0, SIM_P_GC0, SIM_P_GA1, SIM_P_GB1, SIM_P_GC1,
  SIM_NFIELDS
};
/* Raw MNDO/AM1-form parameters (the paper cites these Hamiltonians in its
 * Introduction; values are supplied by the caller).  Units: eV for U, beta,
 * G, H; 1/bohr for zeta; 1/Angstrom for alpha; AM1 Gaussians a (eV*A),
 * b (1/A^2), c (A); mass in amu.  The library derives the multipole lengths
 * D1, D2 and additive terms rho0..rho2 itself. */
typedef struct sim_param_table {
  double v[4][SIM_NFIELDS];
} sim_param_table;

/* Kernel approximation in the electronic equation of motion (eq. 25). */
enum sim_kernel {
  SIM_KERNEL_KRYLOV = 0,  /* low-rank Krylov subspace approximation, eqs. 31-35 */
  SIM_KERNEL_XL = 1,      /* original XL-BOMD scaled delta function K = -c I
                             (Results, Langevin run of C240 2+); no response
                             calculations, rank reported as 0              */
  SIM_KERNEL_BOMD = 2     /* comparison mode: Born-Oppenheimer MD, an SCF
                             (scf_* settings) from the previous density at
                             every step (Results: BOMD reusing the density);
                             X(t) is the converged density, no X dynamics;
                             host-synchronous (no graph capture)           */
};

/* ---- configuration ------------------------------------------------------ */
typedef struct sim_config {
  double Te;          /* electronic temperature, K (eq. 7); > 0                */
  double dt;          /* time step, fs (eqs. 27-30)                            */
  int m_max;          /* maximum Krylov rank m (eq. 34), 1..16                 */
  int m_min;          /* minimum rank before the adaptive stop (<= m_max)      */
  double krylov_tol;  /* adaptive stop: relative fit error < tol (0 = fixed m) */
  int precision;      /* enum sim_precision                                    */
  double scf_tol;     /* sim_create SCF: stop when max|D[P] - P| < scf_tol     */
  int scf_max;        /* sim_create SCF: maximum iterations                    */
  double scf_mix;     /* linear mixing P <- mix P + (1 - mix) D[P] (paper: 0.1) */
  int device;         /* CUDA device ordinal                                   */
  void* stream;       /* cudaStream_t to launch on, or NULL for a private one  */
  int scf_krylov;     /* 0: linear mixing; 1: low-rank Krylov SCF update
                         P <- P - K (D[P] - P) with K of rank m_max (Results,
                         "SCF Optimization": fixed rank, no preconditioner);
                         a mixing step instead whenever the residual has
                         grown tenfold over the best one                      */
  int scf_accept;     /* 1: if the SCF does not reach scf_tol in scf_max
                         iterations, start from the lowest-residual P seen
                         (reported by sim_scf_info) instead of failing       */
  int kernel;         /* enum sim_kernel: the kernel K of Xddot = -w^2 K (D0 - X)
                         (eq. 25) used by sim_step                           */
  double xl_c;        /* SIM_KERNEL_XL only: K = -xl_c I (Results, C240 2+
                         run: c = 1 originally, 0.9 tuned); any finite value */
  double langevin_gamma; /* Langevin friction, 1/fs (Results: Langevin runs at
                         300 K); 0 = NVE.  Scheme (not printed in the paper):
                         Ornstein-Uhlenbeck half steps around the Verlet step
                         (OBABO), V <- c V + sqrt((1 - c^2) k_B T / M) xi,
                         c = exp(-gamma dt / 2)                              */
  double langevin_T;  /* thermostat temperature, K                           */
  unsigned long long langevin_seed; /* key of the Philox4x32-10 stream; xi of
                         component 3A + k at half step p of MD step s uses
                         counter (3A + k, p, s low, s high)                  */
} sim_config;

/* Fills a config with the defaults used by the paper-shaped workloads:
 * Te 1000 K, dt 0.5 fs, m = 4, fixed rank, FP64, scf_tol 1e-10,
 * scf_max 5000, mix 0.1, linear mixing, device 0, private stream,
 * Krylov kernel (xl_c = 1), no thermostat (langevin_gamma = 0, T 300 K,
 * seed 0).
 * The SCF prints max|D[P] - P| per iteration to stderr when the
 * environment variable KSAXL_SCF_TRACE is set. */
void sim_config_default(sim_config* cfg);

/* ---- per-step diagnostics ------------------------------------------------ */
typedef struct sim_step_result {
  double E_kin;     /* sum M Rdot^2 / 2, eV                                    */
  double U;         /* shadow potential energy, eq. 13 (with -2 T_e S), eV     */
  double E_tot;     /* constant of motion, eq. 26, eV                          */
  double mu;        /* chemical potential, eV (eq. 8)                          */
  double gap;       /* eps_LUMO - eps_HOMO (0 when n == N_occ), eV             */
  double res_norm;  /* ||D0[X] - X||_F                                         */
  double fit_err;   /* relative Krylov fit error of the last rank used         */
  int rank;         /* Krylov rank used                                        */
  int pad;
  double dipole[3]; /* dipole moment of the cores and D0 (the observable of the
                       paper's IR spectrum, Results), e Angstrom:
                       sum_A (Z'_A - 2 N_A) R_A - 4 sum_A D1_A D_{s,p_k}(A),
                       N_A = trace of atom A's block of the per-spin D0; the
                       on-site position operator of the NDDO basis       */
} sim_step_result;

typedef struct sim_handle sim_handle;

/* sim_create -- one molecule, initial state at t0.
 * Follows Methods section 5: X(t0 - k dt) = D_min for k = 0..6.  D_min is
 * P0 when P0 != NULL (caller-supplied per-spin density, n x n, symmetric,
 * trace N_occ), otherwise it comes from an SCF by linear mixing from the
 * diagonal guess (Results, "SCF Optimization").  Then the shadow energy,
 * forces and the first Krylov kernel are evaluated at (R0, X(t0)).
 *   natoms  number of atoms (>= 1)
 *   Z       atomic numbers (1, 6, 7, 8), natoms ints
 *   R       positions, Angstrom, natoms x 3
 *   V       velocities, Angstrom/fs, natoms x 3, or NULL for zero
 *   charge  net charge; (valence electrons - charge) must be even
 *   P0      n x n per-spin density or NULL (SCF)
 *   out     receives the handle
 * Errors: SIM_EINVAL (bad Z, odd electron count, NaN, bad config),
 *         SIM_ENOMEM, SIM_ENOCONV (SCF), SIM_ETIMEOUT, SIM_EINTERNAL. */
int sim_create(const sim_config* cfg, const sim_param_table* table, int natoms,
               const int* Z, const double* R, const double* V, int charge,
               const double* P0, sim_handle** out);

/* SCF iterations used by sim_create and the final max|D[P] - P| (0, 0 when
 * P0 was supplied). */
int sim_scf_info(const sim_handle* h, int* iterations, double* residual);

/* Number of basis functions n and occupied orbitals N_occ of a handle. */
int sim_norb(const sim_handle* h);
int sim_nocc(const sim_handle* h);

/* sim_step -- advance nsteps MD steps (eqs. 27-30 with X from eq. 35).
 * out: NULL or nsteps records (caller-owned) filled with the diagnostics of
 * each step.  Synchronous: returns after the last step finished. */
int sim_step(sim_handle* h, int nsteps, sim_step_result* out);

/* sim_step_host -- one MD step with the state exchanged through host memory:
 * R_in/V_in (natoms x 3, or NULL to keep the device copy) are uploaded,
 * the step of eqs. 27-30/35 runs, and R_out, V_out, F_out (natoms x 3) and
 * the step record are downloaded (any output may be NULL).  Page-locked
 * buffers make the copies asynchronous.  Synchronous on return. */
int sim_step_host(sim_handle* h, const double* R_in, const double* V_in, double* R_out,
                  double* V_out, double* F_out, sim_step_result* out);

/* sim_step_async -- enqueue nsteps steps on the handle's stream without
 * waiting; diagnostics of the last step can be read with sim_last_result
 * after the stream is synchronised.  No host synchronisation inside. */
int sim_step_async(sim_handle* h, int nsteps);
int sim_last_result(sim_handle* h, sim_step_result* out);

/* sim_records -- copy the records of the last `count` steps (oldest first)
 * into `out`; count <= 4096 and <= the steps run since the last sim_step,
 * sim_batch_step, sim_set_state or sim_create (whose initial evaluation is
 * record 0).  Synchronises the handle's stream. */
int sim_records(sim_handle* h, sim_step_result* out, int count);

/* sim_wait -- synchronise the handle's stream and return the first error a
 * kernel reported since the last check (SIM_ETIMEOUT for an expired bounded
 * wait, SIM_ENUMERIC for NaN/Inf), else SIM_OK.  Every device-reported error
 * (here and in the step calls) is reported once and then cleared; after a
 * failed step the handle holds a partial step, so re-establish the state
 * with sim_set_state or sim_load before stepping on. */
int sim_wait(sim_handle* h);

/* sim_enable_graphs -- enable != 0 captures one MD step into CUDA graphs
 * (one per phase of the 8-slot X(t - k dt) ring, eq. 29) and from then on
 * replays them in every step call; 0 releases them.  A replayed step is the
 * same kernel sequence on the same buffers, so results are bitwise those of
 * direct launches.  Steps taken while phase profiling is on launch directly.
 * The configuration and the molecule are fixed by the capture. */
int sim_enable_graphs(sim_handle* h, int enable);

/* sim_batch_step -- advance `count` independent handles by nsteps steps
 * each (molecule batches: one trajectory per molecule).  The steps are
 * issued round-robin, each handle on its own stream, so the device runs the
 * small, latency-bound steps of different molecules concurrently (with
 * graphs enabled each step is one graph launch).  Handles are taken in
 * groups whose persistent eigensolver grids fit on the device at the same
 * time; groups run one after the other.  Synchronous; returns the first
 * error.  Records of the steps are read with sim_records. */
int sim_batch_step(sim_handle* const* handles, int count, int nsteps);

/* sim_batch_create -- capture one MD step of every handle into one CUDA graph
 * (one graph per phase of the X ring): each molecule's step is a branch forked
 * from and joined to a private stream, and groups of molecules whose persistent
 * eigensolver grids fit on the device together run one after the other inside
 * the graph.  The handles must be distinct, on distinct streams, have taken the
 * same number of steps, and not use SIM_KERNEL_BOMD or phase profiling; they
 * stay owned by the caller and must outlive the batch.
 * sim_batch_run -- nsteps steps of the whole batch, one graph launch per step;
 * synchronous; results are bitwise those of stepping each handle alone; the
 * records are read per handle with sim_records.  A run is rejected
 * (SIM_EINVAL) when a member's X-ring phase differs from the batch's, which
 * is what stepping a member on its own a number of times other than a
 * multiple of 8 between runs leads to; members stepped alone by a multiple of
 * 8 steps stay consistent with the captured graphs. */
typedef struct sim_batch sim_batch;
int sim_batch_create(sim_handle* const* handles, int count, sim_batch** out);
int sim_batch_run(sim_batch* b, int nsteps);
/* Number of co-resident groups the batch's graph runs one after the other
 * (1 when every member's eigensolver grid fits on the device together). */
int sim_batch_groups(const sim_batch* b);
void sim_batch_destroy(sim_batch* b);

/* Bytes of device memory sim_create allocates for this molecule/config. */
size_t sim_estimate_bytes(const sim_config* cfg, int natoms, const int* Z);

/* ---- serving: continuous batching of many trajectories ------------------
 * A server owns a device, a memory budget and host threads: admission
 * threads that create trajectories (SCF included) in submission order while
 * their estimated memory fits the budget, fewer than max_active are live and
 * the persistent eigensolver grids of all live trajectories fit on the
 * device at once (their grid barriers need every block resident),
 * and a stepping thread that keeps up to two steps in flight per live trajectory
 * (each on its own stream, through CUDA graphs when use_graphs != 0, except
 * for Born-Oppenheimer trajectories) and retires a trajectory when its steps
 * are done.  Every trajectory computes
 * exactly what sim_create + sim_step compute for it alone: no data is shared
 * between trajectories, so results do not depend on the rest of the mix. */
typedef struct sim_server sim_server;

typedef struct sim_server_config {
  int device;               /* CUDA device ordinal                                 */
  int max_active;           /* live trajectories at most (<= 0: 64)                */
  size_t hbm_budget_bytes;  /* device bytes for trajectories (0: 90% of free)      */
  int use_graphs;           /* step through CUDA graphs                            */
  int admission_threads;    /* concurrent sim_create calls (<= 0: 4)               */
} sim_server_config;

typedef struct sim_request {
  sim_config cfg;           /* copied; cfg.device/stream are set by the server     */
  sim_param_table table;    /* copied                                              */
  int natoms;
  const int* Z;             /* natoms; copied at submission                        */
  const double* R;          /* natoms x 3, Angstrom; copied                        */
  const double* V;          /* natoms x 3 or NULL; copied                          */
  int charge;
  int nsteps;               /* MD steps to run (>= 0, <= 4096)                     */
  double* R_out;            /* caller buffers written at completion (or NULL):     */
  double* V_out;            /*   natoms x 3 final positions, velocities, forces;   */
  double* F_out;            /*   they must stay valid until sim_poll reports done  */
  sim_step_result* records; /* nsteps records or NULL                              */
} sim_request;

typedef struct sim_traj_result {
  int status;               /* SIM_OK or the error of sim_create / a step          */
  int steps_done;
  double queue_ms;          /* submission -> admitted (creation started)           */
  double create_ms;         /* sim_create incl. SCF                                */
  double run_ms;            /* first step launched -> last step finished           */
  char error[160];          /* message when status != SIM_OK                       */
} sim_traj_result;

typedef struct sim_server_stats {
  long long submitted, completed, failed, queued, active, max_active_seen;
  long long atom_steps;     /* sum over finished steps of the molecule's atoms     */
  double step_p50_ms;       /* per-trajectory step latency: time between the       */
  double step_p99_ms;       /*   completions of consecutive steps of one trajectory*/
  double elapsed_s;         /* since sim_server_create                             */
  size_t hbm_in_use, hbm_budget;
  char threads[512];        /* diagnostics: what each server thread is doing and  */
                            /*   ticket:done/launched/nsteps of live trajectories */
} sim_server_stats;

int sim_server_create(const sim_server_config* cfg, sim_server** out);
/* Copies the request; *ticket identifies it.  Thread-safe.  SIM_EINVAL for a
 * request that can never be admitted (bad sizes, larger than the budget). */
int sim_submit(sim_server* s, const sim_request* req, unsigned long long* ticket);
/* SIM_PENDING while the trajectory is queued or running; otherwise fills
 * *out, forgets the ticket and returns SIM_OK (out->status holds the
 * trajectory's own result).  SIM_EINVAL for an unknown ticket.  Thread-safe. */
int sim_poll(sim_server* s, unsigned long long ticket, sim_traj_result* out);
int sim_server_stats_get(sim_server* s, sim_server_stats* out);
/* Wait until no trajectory is queued or live (SIM_ETIMEOUT after timeout_s). */
int sim_server_drain(sim_server* s, double timeout_s);
/* Stops the threads after the live trajectories finish their current step
 * and the creations under way end; unfinished trajectories are dropped. */
void sim_server_destroy(sim_server* s);

/* sim_get_state -- copy the current state out (any pointer may be NULL).
 *   R, V, F: natoms x 3 (F = forces, eV/Angstrom, eq. 37 with the eq. 9 sign)
 *   D0:      n x n per-spin D0[X(t)] of the last evaluation (eq. 19) */
int sim_get_state(sim_handle* h, double* R, double* V, double* F, double* D0);

/* sim_set_state -- overwrite R, V and/or the X history and re-evaluate at
 * (R, X(t)) (any pointer may be NULL to keep the current value).
 *   Xhist: 7 x n x n, Xhist[k] = X(t - k dt), k = 0..6 (eq. 29 history) */
int sim_set_state(sim_handle* h, const double* R, const double* V, const double* Xhist);

/* sim_save -- write the handle's dynamical state to a file: configuration,
 * raw parameter table, atoms, charge, R, V and the X history X(t - k dt),
 * k = 0..6 (everything eq. 29 and eqs. 27-30 carry from step to step).
 * sim_load -- create a handle on `device` (launching on `stream`, or a private
 * one for NULL) from such a file; it re-evaluates F, D0, forces and the kernel
 * at (R, X(t)) with the same kernels, so stepping a loaded handle reproduces
 * the saved trajectory bitwise.  Errors: SIM_EINVAL (unreadable, truncated or
 * foreign file), SIM_EINTERNAL (write failure), and those of sim_create. */
int sim_save(sim_handle* h, const char* path);
int sim_load(const char* path, int device, void* stream, sim_handle** out);

/* Matrices of the last evaluation, copied into an n x n caller buffer. */
enum sim_matrix {
  SIM_MAT_X = 0,       /* X(t)                                              */
  SIM_MAT_D0 = 1,      /* D0[X(t)] (eq. 19)                                 */
  SIM_MAT_FOCK = 2,    /* F(X(t)) = h + G(X(t)) (eq. 17)                    */
  SIM_MAT_H = 3,       /* core Hamiltonian h                                */
  SIM_MAT_KERNEL = 4,  /* sum_i V_i c_i ~ K (D0 - X) (eq. 34)               */
  SIM_MAT_Q = 5,       /* eigenvectors of F as columns                      */
  SIM_MAT_XHIST = 6,   /* SIM_MAT_XHIST + k, k = 0..6: X(t - k dt), the
                          history eq. 29 carries (SIM_MAT_XHIST + 0 = X(t))   */
};
int sim_get_matrix(sim_handle* h, int which, double* out);

/* Vectors of the last evaluation (n doubles): 0 = eigenvalues (ascending),
 * 1 = occupations f_i. */
int sim_get_vector(sim_handle* h, int which, double* out);

/* Device-side per-phase timing (CUDA events on the handle's stream).
 * enable != 0 starts recording; sim_phase_times returns, for each phase
 * id < nphase, the accumulated milliseconds, launch count and the bytes or
 * flops one launch moves/does (algorithmic, see the design notes). */
int sim_profile_enable(sim_handle* h, int enable);
int sim_phase_count(void);
const char* sim_phase_name(int phase);
int sim_phase_times(sim_handle* h, double* ms, long long* launches, double* work_per_launch);

/* Number of CUDA kernel launches the library has issued (all handles). */
long long sim_launch_count(void);

/* Stream (cudaStream_t) the handle launches on. */
void* sim_stream(sim_handle* h);

void sim_destroy(sim_handle* h);

/* sim_tc_gemm_noalloc -- the tensor-core slice product of sim_debug_tc_gemm
 * without any memory allocation.  The paper has no counterpart: it serves
 * callers that cannot allocate device memory, such as a serving process that
 * has divided all of the GPU's memory into fixed slots under a hard budget,
 * or a latency-critical loop where cudaMalloc/cudaFree would synchronise the
 * device.
 *   A, B  DEVICE n x n row-major FP64 inputs; C: DEVICE n x n FP64 output
 *   n     1..256 (larger n returns SIM_EINVAL)
 *   terms 1, 3, 6 or 10 (1-4 fixed-point BF16 slices per operand)
 *   sym   != 0: compute the upper tiles only and mirror (A B^T symmetric)
 *   stream cudaStream_t (NULL = legacy default stream); the call returns
 *          after synchronising it
 * Scratch: one fixed device array of about 1 MB inside the library (held by
 * every device that loads it, until exit), shared by all calls: calls that
 * overlap on the GPU race and must be serialised by the caller.  The error
 * flag in it is cleared on every call.  The first call on a device looks up
 * the array's address (cudaGetSymbolAddress, device current) and should come
 * before any stream capture on that device.  Returns SIM_ETIMEOUT if a
 * bounded pipeline wait expired. */
int sim_tc_gemm_noalloc(int n, const double* A, const double* B, int terms, int sym, double* C,
                        void* stream);

/* sim_debug_tc_gemm -- test hook for the tensor-core contraction used by the
 * mixed-precision path (no counterpart in the paper; it exposes one building
 * block of eq. 19 / eq. 36 so tests can check it in isolation).
 * C = sum over `terms` BF16-piece products A_i B_j^T of the FP64 inputs:
 * terms = 1 (plain BF16), 3 (2 pieces), 6 (3 pieces) or 10 (4 pieces).  A, B, C are host
 * n x n row-major arrays; sym != 0 computes only the upper tiles and mirrors
 * (use only when A B^T is symmetric).  Allocates and frees its own device
 * memory; synchronous. */
int sim_debug_tc_gemm(int n, const double* A, const double* B, int terms, int sym, double* C);

/* sim_debug_tc_gemm_grouped -- the 3-slice (slices = 3, terms 6) or 4-slice
 * (slices = 4, terms 10) product computed the way the mixed path computes the
 * DMPT products of eq. 36 (3 slices) and the density product of eq. 19 and
 * the back-transformation (4 slices): all slices of a k-tile staged together,
 * the weight-1 slice product summed exactly per 512-K chunk and the
 * lower-weight ones in FP32, so C is within ~2^-26 (3 slices) or ~2^-28
 * (4 slices) of sum_k |A_ik||B_jk| of the exact slice product (not bitwise
 * equal).  Other slice counts: SIM_EINVAL.  Arguments, memory and errors as
 * sim_debug_tc_gemm. */
int sim_debug_tc_gemm_grouped(int n, const double* A, const double* B, int slices, int sym, double* C);

/* sim_measure_peak -- kind 0: FP64, kind 1: FP32 FMA throughput of `device`
 * in TFLOP/s (2 flops per FMA; 8 independent chains per thread on 8 blocks of
 * 256 threads per SM; allocates 16 bytes); kind 2: L2 read + write rate in
 * TB/s of a 90 MB L2-resident buffer read and written back 20 times by one
 * block of 512 threads per SM (the double-float tridiagonalisation's launch
 * shape; allocates 90 MB).  Timed with CUDA events after a warm-up launch.
 * The denominators of the roofline fractions (no counterpart in the paper).
 * Other kinds: SIM_EINVAL.  Synchronous. */
int sim_measure_peak(int device, int kind, double* tflops);

/* Failure-path test hooks (no counterpart in the paper).
 * sim_debug_barrier_limit -- wall-time limit, ns, of the eigensolver's grid
 *   barriers on `device` (default 2e9).  A limit of 0 makes the next step's
 *   barrier waits expire: the kernel records the timeout and returns, and the
 *   step reports SIM_ETIMEOUT.  Restore the default afterwards.
 * sim_debug_wait_expiry -- one bounded mbarrier wait (the wait primitive of
 *   the tensor-core pipeline) on a barrier that nothing arrives at, `tries`
 *   polls; returns SIM_ETIMEOUT when the wait expired as it must. */
int sim_debug_barrier_limit(int device, unsigned long long ns);
int sim_debug_wait_expiry(int device, long long tries);

/* Thread-local message of the last error (never NULL). */
const char* sim_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KSA_XLBOMD_SIM_H */
