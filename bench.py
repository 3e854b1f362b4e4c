#!/usr/bin/env python
"""Throughput of the KSA-XL-BOMD MD step on GB300: atom-steps/s and step latency.

Workload (one GPU, N = 1): 840 carbon atoms (3360 sp orbitals) packed at random
at 2.2 g/cc in an open cubic box (seed 2), synthetic NDDO table (seed 1),
T_e = 3000 K, Krylov rank m = 6, dt = 0.5 fs, initial X from the GPU SCF
(linear mixing), mixed precision (FP64 eigensolve; tcgen05 fixed-point-slice
products for D0 and DMPT).  A step is one full pass of the hot path: Verlet
half-kicks and drift, X update, pair integrals and derivatives, h, F(X),
eigendecomposition, occupations, D0, energy, forces and the rank-6 Krylov
kernel.  The working set (~30 dense 3360 x 3360 FP64 matrices, 1.3 GB of
pair blocks) is far larger than L2, so no extra flush is done.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

With torchrun (N > 1) every rank steps its own 840-atom system (independent
replicas: a single system has no natural partition, so there is no data-path
collective) and rank 0 prints the job total.  ``--impl reference`` times the
CPU oracle (tests' FP64 numpy implementation) on one bounded sample step.
"""
import ctypes
import argparse
import json
import os
import statistics
import shutil
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="840-atom random carbon packing, 2.2 g/cc, open box (seed 2)",
                natoms=840, norb=3360, Te_K=3000.0, krylov_rank=6, dt_fs=0.5,
                param_table="synthetic NDDO seed 1", velocities="Maxwell-Boltzmann 300 K seed 2",
                l2="working set > L2 (no flush needed)")
METRIC = "atom-steps/s (KSA-XL-BOMD MD step)"
KERNEL_MODE = [0]      # sim_kernel of the timed runs (--kernel)
# FP32 instructions per FP64-equivalent multiply-add in the double-float
# tridiagonalisation: the rank-2 update costs 27 for two, the product term 12 for
# one (df.cuh), 13 on average over the three multiply-adds of an element
DF_OPS_PER_FMA = 13.0
# DRAM bytes (read + write) of one tridiag_df_kernel launch at n = 3360 from one
# ncu capture of the bench's profile run (dram__bytes_read.sum 1.018e9 +
# dram__bytes_write.sum 3.868e10; a one-pass metric set, kernel unchanged since)
TRIDIAG_TRAFFIC = {"bytes": 1102843648 + 39244797440,
                   "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one tridiag_df_kernel launch "
                             "of bench.py --profile-run at n = 3360"}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device):
    """Largest value of x over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(total_ms, steps, natoms_per_rank, world):
    """(ms per step, whole-job atom-steps/s): every rank steps its own replica."""
    ms_per_step = total_ms / steps
    return ms_per_step, world * natoms_per_rank / (ms_per_step / 1e3)


class EventClock:
    """Step marks as CUDA events on the stream the steps are launched on."""

    def __init__(self, stream):
        import torch
        self.stream, self.torch, self.ev = stream, torch, []

    def mark(self):
        e = self.torch.cuda.Event(enable_timing=True)
        e.record(self.stream)
        self.ev.append(e)

    def laps_ms(self):
        return [self.ev[k].elapsed_time(self.ev[k + 1]) for k in range(len(self.ev) - 1)]


class WallClock:
    """Step marks from the host clock (CPU replicas)."""

    def __init__(self):
        self.t = []

    def mark(self):
        self.t.append(time.perf_counter())

    def laps_ms(self):
        return [1e3 * (self.t[k + 1] - self.t[k]) for k in range(len(self.t) - 1)]


def timed_replica(step, steps, warmup, barrier, clock, world, device):
    """The rank logic of the bench: `warmup` untimed steps, a barrier, `steps`
    steps each bracketed by clock marks, a barrier, then the slowest rank's
    total.  Returns (per-step ms of this rank, max-over-ranks total ms)."""
    for _ in range(warmup):
        step()
    barrier()
    clock.mark()
    for _ in range(steps):
        step()
        clock.mark()
    barrier()
    laps = clock.laps_ms()
    return laps, max_over_ranks(sum(laps), world, device)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        self.proc.wait()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1].split()[0]) for r in rows if r[1].strip()[0].isdigit()]
        mx = [float(r[2].split()[0]) for r in rows if r[2].strip()[0].isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


def _inputs(natoms=None):
    import synth
    mol = synth.carbon_packing(seed=2, natoms=natoms or WORKLOAD["natoms"])
    V = synth.maxwell_boltzmann(mol.Z, 300.0, seed=2)
    table = synth.table_to_array(synth.synthetic_table(1))
    return mol, V, table


def _create(kx, mol, V, table, precision, P0=None):
    """Initial X from the low-rank Krylov SCF, bounded to 30 iterations.

    The random packing is a hard SCF case (linear mixing stalls); the MD step
    cost does not depend on how far X(t0) is from self-consistency, and the
    residual reached is reported in the output line."""
    cfg = kx.sim_config_default(Te=WORKLOAD["Te_K"], dt=WORKLOAD["dt_fs"], m_max=6, m_min=6, precision=precision,
                                scf_tol=1e-8, scf_max=30, scf_krylov=1, scf_accept=1, kernel=KERNEL_MODE[0])
    return kx.sim_create(cfg, kx.param_table(table), mol.Z, mol.R, V=V, P0=P0)


def run_ours(args):
    import torch
    import paper_2303_00689_gb300 as kx
    from paper_2303_00689_gb300 import build

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    peaks = {"fp64_tflops": kx.sim_measure_peak(0, local), "fp32_tflops": kx.sim_measure_peak(1, local),
             "l2_rw_tbs": kx.sim_measure_peak(2, local)}
    mol, V, table = _inputs()
    N = mol.natoms
    prec = kx.SIM_PREC_FP64 if args.precision == "fp64" else kx.SIM_PREC_MIXED
    t0 = time.time()
    h = _create(kx, mol, V, table, prec)
    setup_s = time.time() - t0
    scf_iters, scf_res = kx.sim_scf_info(h)
    X0 = kx.sim_get_matrix(h, kx.SIM_MAT_X)
    stream = torch.cuda.ExternalStream(kx.sim_stream(h))

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-timed steps (state resident in HBM) ---------------------------
    # the production configuration: one CUDA graph launch per step (the step's
    # side-stream branches included); the per-phase breakdown comes from a few
    # further steps with phase profiling (direct launches, side work in line)
    kx.sim_step(h, args.warmup, records=False)
    kx.sim_enable_graphs(h)
    clocks = Clocks(local)
    clocks.start()
    launches0 = kx.sim_launch_count()
    per_step, total_ms = timed_replica(lambda: kx.sim_step_async(h, 1), args.steps, 0, barrier,
                                       EventClock(stream), world, "cuda")
    launches = kx.sim_launch_count() - launches0
    clk = clocks.stop()
    recs = kx.sim_records(h, args.steps)
    prof_steps = min(3, args.steps)
    kx.sim_profile_enable(h, True)
    kx.sim_step(h, prof_steps, records=False)
    phases = kx.sim_phase_times(h)
    kx.sim_profile_enable(h, False)
    ms_per_step, value = job_throughput(total_ms, args.steps, N, world)
    state_dir = None
    if rank == 0 and not args.no_cpu_baseline:
        state_dir = _dump_state(kx, h, N)

    # ---- end to end through the C ABI with pinned host buffers --------------------
    pin = lambda: torch.empty((N, 3), dtype=torch.float64).pin_memory().numpy()
    R_h, V_h, R_o, V_o, F_o = pin(), pin(), pin(), pin(), pin()
    Rc, Vc, _, _ = kx.sim_get_state(h, N)
    R_h[:] = Rc
    V_h[:] = Vc
    rec_h = kx.sim_step_result()
    n_e2e = max(3, min(args.steps, 10))
    w_e2e = 2                                   # untimed: the first calls after the profiled steps

    def host_step():
        kx.sim_step_host(h, R_h, V_h, R_o, V_o, F_o, rec_h)
        R_h[:] = R_o
        V_h[:] = V_o

    for _ in range(w_e2e):
        host_step()
    barrier()
    e2e_ms = []
    te = time.perf_counter()
    for _ in range(n_e2e):
        t1 = time.perf_counter()
        host_step()
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    e2e_s = (time.perf_counter() - te) / n_e2e
    e2e_s = max_over_ranks(e2e_s, world, "cuda")
    kx.sim_destroy(h)

    # ---- dominant phase roofline -----------------------------------------------
    name, ph = max(phases.items(), key=lambda kv: kv[1]["ms"])
    per_launch_s = ph["ms"] / max(1, ph["launches"]) / 1e3
    roof = _roofline(name, ph, per_launch_s, peaks, prec == kx.SIM_PREC_MIXED, int(X0.shape[0]))

    def stats(key):
        v = np.array([r[key] for r in recs], dtype=float)
        return {"min": float(v.min()), "median": float(np.median(v)), "max": float(v.max())}

    out = {
        "metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+bf16-slices" if prec == kx.SIM_PREC_MIXED else "f64",
        "data": "synthetic (seeded generators; synthetic NDDO parameters)",
        "config": dict(WORKLOAD, precision=args.precision, kernel=args.kernel, parallelism=f"replicas x{world}"),
        "latency_ms": {"p50": float(np.percentile(per_step, 50)), "p99": float(np.percentile(per_step, 99)),
                       "per_step": [round(x, 3) for x in per_step]},
        "e2e": {"value": world * N / e2e_s, "unit": "atom-steps/s",
                "h2d_bytes_per_step": 2 * N * 3 * 8,
                "d2h_bytes_per_step": 3 * N * 3 * 8 + ctypes.sizeof(kx.sim_step_result),
                "steps": n_e2e, "warmup": w_e2e, "per_step_ms": [round(x, 3) for x in e2e_ms]},
        "gpu_launches": int(launches),
        "roofline": roof,
        "measured_peaks": peaks,
        "phases_ms_per_step": {k: round(v["ms"] / prof_steps, 3) for k, v in phases.items()},
        "phases_from": f"{prof_steps} further steps with phase profiling (direct launches, side-stream work in line)",
        "timed_steps": {"res_norm": stats("res_norm"), "fit_err": stats("fit_err"), "rank": stats("rank"),
                        "E_tot": stats("E_tot")},
        "setup_s": round(setup_s, 2),
        "scf": {"method": "low-rank Krylov, rank 6", "iterations": scf_iters, "max_abs_residual": scf_res},
        "clocks": clk,
    }
    if rank == 0 and not args.no_fp64_context and prec == kx.SIM_PREC_MIXED:
        out["fp64_path"] = _fp64_context(kx, mol, V, table, X0)
    if rank == 0 and not args.no_extras:
        out["serving"] = _serving_record(kx, args)
        out["batch"] = _batch_record(kx, args)
    if rank == 0 and not args.no_cpu_baseline:
        cb = _cpu_baseline(args, state_dir)
        if "accuracy" in cb:
            out["accuracy"] = cb.pop("accuracy")
        out["cpu_baseline"] = cb
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def _dump_state(kx, h, N):
    """The state after the timed steps, for the oracle's accuracy check."""
    d = tempfile.mkdtemp(prefix="ksaxl_state_")
    R, V, F, D0 = kx.sim_get_state(h, N)
    np.save(os.path.join(d, "R.npy"), R)
    np.save(os.path.join(d, "V.npy"), V)
    np.save(os.path.join(d, "F.npy"), F)
    np.save(os.path.join(d, "D0.npy"), D0)
    np.save(os.path.join(d, "K.npy"), kx.sim_get_matrix(h, kx.SIM_MAT_KERNEL))
    np.save(os.path.join(d, "Xh.npy"), np.stack([kx.sim_get_matrix(h, kx.SIM_MAT_XHIST + k) for k in range(7)]))
    with open(os.path.join(d, "rec.json"), "w") as f:
        json.dump({k: v for k, v in kx.sim_last_result(h).items()}, f)
    return d


def _roofline(name, ph, per_launch_s, peaks, mixed, n):
    """Roofline entry of the dominant phase; peaks measured in this run (n: orbitals)."""
    meas = _peaks()
    work = ph["work"]
    if name == "eig_tridiag" and mixed:
        # FP64-equivalent algorithmic flops (4/3 n^3) run as double-float on the
        # FP32 pipe: the arithmetic peak is the measured FP32 FMA rate divided by
        # the FP32 instructions one FP64-equivalent multiply-add costs
        achieved = work / per_launch_s / 1e12
        peak = peaks["fp32_tflops"] / DF_OPS_PER_FMA
        return {"kernel_phase": name, "kernel": "tridiag_df_kernel", "bound": "alu", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": TRIDIAG_TRAFFIC["bytes"], "traffic_source": TRIDIAG_TRAFFIC["source"],
                "peak_source": f"measured FP32 FMA rate {peaks['fp32_tflops']:.1f} TFLOP/s / {DF_OPS_PER_FMA:g} "
                               "FP32 instructions per double-float multiply-add",
                "fp64_frac": achieved / peaks["fp64_tflops"],
                "fp64_note": "the same algorithmic flops against the measured FP64 FMA rate "
                             f"{peaks['fp64_tflops']:.2f} TFLOP/s",
                "l2": _tridiag_l2(n, per_launch_s, peaks)}
    if name in ("eig_tridiag", "eig_backtransform", "density_gemm"):
        achieved = work / per_launch_s / 1e12
        peak = peaks["fp64_tflops"]
        return {"kernel_phase": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "peak_source": "measured FP64 FMA rate"}
    if name == "krylov_dmpt_gemm":
        achieved = work / per_launch_s / 1e12
        peak = meas.get("bf16_tflops_sustained", 1715.0)
        return {"kernel_phase": name, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "peak_source": "measured bf16 sustained"}
    achieved = work / per_launch_s / 1e9
    peak = meas.get("hbm_gbs", 6792.1)
    return {"kernel_phase": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else 0.0, "traffic": None, "peak_source": "measured HBM copy"}


def _tridiag_l2(n, per_launch_s, peaks):
    """The work items' L2 traffic: every column reads and writes the trailing
    (n-k-1) x (n-k-1) double-float matrix once (16 B per element), against the
    L2 read + write rate measured with the kernel's launch shape."""
    m = np.arange(2, n, dtype=np.float64)
    bytes_ = 16.0 * float(np.sum(m * m))
    achieved = bytes_ / per_launch_s / 1e12
    peak = peaks["l2_rw_tbs"]
    return {"bytes_per_launch": bytes_, "achieved": achieved, "peak": peak, "unit": "TB/s", "frac": achieved / peak,
            "peak_source": "sim_measure_peak kind 2: 90 MB L2-resident buffer read and written back, one block "
                           "of 512 threads per SM"}


def _fp64_context(kx, mol, V, table, X0, steps=2):
    """The plain FP64 GPU path on the same workload and X(t0) (few steps: ~1.8 s each)."""
    import torch
    h = _create(kx, mol, V, table, kx.SIM_PREC_FP64, P0=X0)
    kx.sim_step(h, 1, records=False)
    torch.cuda.synchronize()
    t = time.perf_counter()
    kx.sim_step(h, steps, records=False)
    torch.cuda.synchronize()
    s = (time.perf_counter() - t) / steps
    kx.sim_destroy(h)
    return {"value": mol.natoms / s, "unit": "atom-steps/s", "ms_per_step": 1e3 * s, "steps": steps}


def _cpu_baseline(args, state_dir=None):
    """Times the oracle in a fresh (spawned) interpreter on a bounded sample;
    with a state from the GPU run it also reports the GPU's errors there."""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample"]
    if state_dir:
        cmd += ["--state", state_dir]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=args.cpu_timeout)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # noqa: BLE001
        return {"value": None, "unit": "atom-steps/s", "kind": "oracle", "error": str(e)[:200]}
    finally:
        if state_dir:
            shutil.rmtree(state_dir, ignore_errors=True)


def oracle_sample(state_dir=None):
    """One full oracle MD step of the 840-atom workload (bounded sample).

    Without a state: from the diagonal guess X (no SCF).  With the GPU's state
    after its timed steps (R, V, X(t - k dt)): the oracle's evaluation there
    (untimed) gives the GPU path's errors in D0, forces, U and the Krylov
    kernel K; then one oracle step from that state is timed."""
    import synth
    from oracle import dynamics as dyn, hamiltonian as ham
    mol, V, _ = _inputs()
    sysm = ham.System(mol.Z, synth.synthetic_table(1))
    cfg = dyn.Config(Te=WORKLOAD["Te_K"], dt=WORKLOAD["dt_fs"], m=6)
    acc = None
    if state_dir:
        ld = lambda k: np.load(os.path.join(state_dir, k + ".npy"))
        R, Vg, Xh = ld("R"), ld("V"), ld("Xh")
        t = time.perf_counter()
        st = dyn.State(sysm, R, Vg, cfg, X0=Xh[0])       # evaluation at the GPU's (R, X(t)), not timed
        t_eval = time.perf_counter() - t
        st.X = [x.copy() for x in Xh]                    # the GPU's X history (eq. 29)
        with open(os.path.join(state_dir, "rec.json")) as f:
            rec = json.load(f)
        ev = st.ev
        acc = {"max_abs_dD0": float(np.abs(ld("D0") - ev["D"]).max()),
               "max_abs_dF_eV_per_A": float(np.abs(ld("F") - ev["forces"]).max()),
               "abs_dU_eV": float(abs(rec["U"] - ev["U"])),
               "rel_max_dK": float(np.abs(ld("K") - ev["K"]).max() / np.abs(ev["K"]).max()),
               "where": "state after the timed steps; oracle evaluation at the same R and X(t)",
               "bars": {"D0": 1e-6, "F_eV_per_A": 1e-4}}
        sample = ("one full oracle MD step of the 840-atom workload from the GPU's state after its timed steps "
                  f"(R, V, X history); the evaluation there ({t_eval:.1f} s) untimed")
    else:
        X = dyn.initial_guess(sysm)
        t = time.perf_counter()
        st = dyn.State(sysm, mol.R, V, cfg, X0=X)     # evaluation at t0 (not timed below)
        t_eval = time.perf_counter() - t
        sample = ("one full oracle MD step (teacher-forced from the diagonal guess X, no SCF) of the "
                  f"840-atom workload; first evaluation {t_eval:.1f} s untimed")
    t = time.perf_counter()
    st.step()
    s = time.perf_counter() - t
    cores = len(os.sched_getaffinity(0))
    out = {"value": mol.natoms / s, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
           "sample": sample, "seconds_per_step": s}
    if acc is not None:
        out["accuracy"] = acc
    return out


def profile_run(args):
    """Short fixed run for ncu: the 840-atom workload from the diagonal guess
    (no SCF), `warmup` + `steps` MD steps; prints launch counts to stderr."""
    import paper_2303_00689_gb300 as kx
    from paper_2303_00689_gb300 import build
    build.build()
    mol, V, table = _inputs(args.profile_natoms)
    X0 = 0.5 * np.eye(mol.norb)      # all-carbon: 4 valence electrons over 4 orbitals, per spin
    prec = kx.SIM_PREC_FP64 if args.precision == "fp64" else kx.SIM_PREC_MIXED
    c0 = kx.sim_launch_count()
    h = _create(kx, mol, V, table, prec, P0=X0)
    c1 = kx.sim_launch_count()
    kx.sim_step(h, args.warmup, records=False)
    c2 = kx.sim_launch_count()
    kx.sim_step(h, args.steps, records=False)
    c3 = kx.sim_launch_count()
    kx.sim_destroy(h)
    print(f"launches create={c1 - c0} warmup={c2 - c1} steps={c3 - c2}", file=sys.stderr, flush=True)


BATCH = dict(workload="128 organic molecules, 12-200 atoms (C/N/O/H, seed 3)", molecules=128, Te_K=1000.0,
             krylov_rank=4, dt_fs=0.5, precision="mixed", param_table="synthetic NDDO seed 1")


def _batch_handles(kx, mols, table, graphs):
    cfg = kx.sim_config_default(Te=BATCH["Te_K"], dt=BATCH["dt_fs"], m_max=4, m_min=4,
                                precision=kx.SIM_PREC_MIXED, scf_tol=1e-7, scf_max=40, scf_krylov=1,
                                scf_accept=1)
    hs = []
    for i, m in enumerate(mols):
        import synth
        V = synth.maxwell_boltzmann(m.Z, 300.0, seed=1000 + i)
        hs.append(kx.sim_create(cfg, kx.param_table(table), m.Z, m.R, V=V, charge=m.charge))
        if graphs:
            kx.sim_enable_graphs(hs[-1])
    return hs


def measure_batch(kx, molecules, steps, warmup):
    """Molecule batch: every molecule its own trajectory, all stepped together
    (sim_batch_create/run: one CUDA graph per batch step, one branch per
    molecule).  Returns the measurement as a dict."""
    import torch
    import synth
    mols = synth.molecule_batch(seed=3, count=molecules)
    table = synth.table_to_array(synth.synthetic_table(1))
    atoms = sum(m.natoms for m in mols)
    t = time.time()
    hs = _batch_handles(kx, mols, table, graphs=False)
    batch = kx.sim_batch_create(hs)              # one CUDA graph per batch step
    setup = time.time() - t
    kx.sim_batch_run(batch, warmup)
    l0 = kx.sim_launch_count()
    torch.cuda.synchronize()
    t = time.perf_counter()
    kx.sim_batch_run(batch, steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    launches = kx.sim_launch_count() - l0
    # the same handles stepped one molecule after the other (no overlap)
    k_seq = max(1, min(steps, 3))
    torch.cuda.synchronize()
    t = time.perf_counter()
    for h in hs:
        kx.sim_step(h, k_seq, records=False)
    seq = atoms * k_seq / (time.perf_counter() - t)
    kx.sim_batch_destroy(batch)
    for h in hs:
        kx.sim_destroy(h)
    return {"workload": f"{molecules} organic molecules, 12-200 atoms (C/N/O/H, seed 3)", "atoms": atoms,
            "value": atoms * steps / dt, "unit": "atom-steps/s", "ms_per_batch_step": 1e3 * dt / steps,
            "steps": steps, "sequential_value": seq, "gpu_launches_per_step": launches / steps,
            "graph_launches_per_step": 1, "setup_s": round(setup, 1), "Te_K": BATCH["Te_K"], "krylov_rank": 4,
            "precision": "mixed"}


def _batch_record(kx, args):
    try:
        return measure_batch(kx, args.extra_batch_molecules, 5, 3)
    except Exception as e:  # noqa: BLE001
        return {"error": str(e)[:200]}


def run_batch(args):
    import torch
    import paper_2303_00689_gb300 as kx
    from paper_2303_00689_gb300 import build
    torch.cuda.set_device(0)
    build.build()
    clocks = Clocks(0)
    clocks.start()
    m = measure_batch(kx, BATCH["molecules"], args.steps, args.warmup)
    clk = clocks.stop()
    out = {"metric": "atom-steps/s (128-molecule batch, KSA-XL-BOMD)", "value": m["value"], "unit": "atom-steps/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_batch_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+bf16-slices",
           "data": "synthetic", "config": dict(BATCH, atoms=m["atoms"], l2="per-molecule working sets are small; "
                                                                         "timed region is many consecutive steps"),
           "sequential_value": m["sequential_value"], "gpu_launches": int(m["gpu_launches_per_step"] * args.steps),
           "graph_launches_per_step": 1, "setup_s": m["setup_s"], "clocks": clk}
    print(json.dumps(out), flush=True)


def measure_serving(kx, count, nmax, use_graphs=True, admit=4, timeout_s=900.0):
    """Serving: Poisson arrivals of MD requests (C60 cages, 60..nmax atoms,
    10-100 steps) at 0.8x the measured closed-loop capacity, continuous
    batching under an HBM budget.  Returns the measurement as a dict."""
    import synth
    table = kx.param_table(synth.table_to_array(synth.synthetic_table(1)))
    cfg = kx.sim_config_default(Te=1000.0, dt=0.5, m_max=4, m_min=4, precision=kx.SIM_PREC_MIXED,
                                scf_tol=1e-7, scf_max=40, scf_krylov=1, scf_accept=1)
    # C60 cages: random organic trees heat up and fly apart within a few fs under
    # the synthetic parameter table, which would make long trajectories meaningless
    reqs = synth.serving_requests(seed=4, count=count, rate_per_s=1.0, nmax=nmax, kind="fullerene")
    work = sum(m.natoms * st for _, m, st in reqs)

    def replay(rate_scale):
        """rate_scale None: all requests at t = 0 (closed loop, capacity)."""
        with kx.Server(max_active=64, use_graphs=use_graphs, admission_threads=admit) as srv:
            t0 = time.perf_counter()
            tickets = []
            for (ta, m, st) in reqs:
                if rate_scale is not None:
                    wait = ta * rate_scale - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(wait)
                V = synth.maxwell_boltzmann(m.Z, 300.0, seed=int(ta * 1e3) % 100000)
                tickets.append(srv.submit(cfg, table, m.Z, m.R, V=V, charge=m.charge, nsteps=st, records=False))
            while True:
                st = srv.stats()
                if st["completed"] + st["failed"] == len(reqs):
                    break
                if time.perf_counter() - t0 > timeout_s:
                    raise RuntimeError(f"serving run exceeded {timeout_s} s: {st}")
                time.sleep(0.5)
            wall = time.perf_counter() - t0
            res = [srv.poll(t) for t in tickets]
            st = srv.stats()
        q = [r["queue_ms"] for r in res]
        return dict(wall_s=wall, atom_steps_per_s=st["atom_steps"] / wall, step_p50_ms=st["step_p50_ms"],
                    step_p99_ms=st["step_p99_ms"], queue_p50_ms=float(np.percentile(q, 50)),
                    queue_p99_ms=float(np.percentile(q, 99)), failed=st["failed"],
                    max_active_seen=st["max_active_seen"])

    cap = replay(None)
    # arrival times scaled so the offered load is 0.8 x the closed-loop capacity
    span = reqs[-1][0]
    target_wall = work / (0.8 * cap["atom_steps_per_s"])
    served = replay(target_wall / span)
    return {"workload": f"{count} requests of 1-{nmax // 60} C60 cages (60-{nmax} atoms), 10-100 steps (seed 4)",
            "value": served["atom_steps_per_s"], "unit": "atom-steps/s",
            "latency_ms": {"p50": served["step_p50_ms"], "p99": served["step_p99_ms"]},
            "queue_ms": {"p50": served["queue_p50_ms"], "p99": served["queue_p99_ms"]},
            "offered_load": "0.8 x closed-loop capacity", "Te_K": 1000.0, "krylov_rank": 4, "precision": "mixed",
            "capacity": cap, "served": served}


def _serving_record(kx, args):
    try:
        return measure_serving(kx, args.extra_serve_requests, args.extra_serve_nmax, timeout_s=300.0)
    except Exception as e:  # noqa: BLE001
        return {"error": str(e)[:200]}


def run_serve(args):
    import torch
    import paper_2303_00689_gb300 as kx
    from paper_2303_00689_gb300 import build
    torch.cuda.set_device(0)
    build.build()
    m = measure_serving(kx, args.serve_requests, args.serve_nmax, bool(args.serve_graphs), args.serve_admit,
                        args.serve_timeout)
    out = {"metric": "atom-steps/s served (Poisson arrivals at 0.8x capacity)", "value": m["value"],
           "unit": "atom-steps/s", "n_gpus": 1, "steps": args.serve_requests, "warmup": 0,
           "ms_per_step": m["latency_ms"]["p50"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64+bf16-slices", "data": "synthetic",
           "config": {"workload": m["workload"], "Te_K": 1000.0, "krylov_rank": 4, "precision": "mixed",
                      "offered_load": m["offered_load"]},
           "latency_ms": m["latency_ms"], "queue_ms": m["queue_ms"], "capacity": m["capacity"],
           "served": m["served"]}
    print(json.dumps(out), flush=True)


def _fit_slope(t, y):
    """Least-squares slope of y(t) and its standard error."""
    A = np.vstack([t, np.ones_like(t)]).T
    coef, res, _, _ = np.linalg.lstsq(A, y, rcond=None)
    r = y - A @ coef
    dof = max(len(t) - 2, 1)
    se = np.sqrt((r @ r) / dof / ((t - t.mean()) @ (t - t.mean())))
    return float(coef[0]), float(se)


def run_drift(args):
    """Energy conservation of the shadow dynamics (eq. 26): neutral C60 cages
    (synthetic table, C-C 1.60 A) at T_e = 5000 K, mixed precision, 0.5 fs.
    The cages are first thermalised by Langevin dynamics at 300 K (the
    paper's drifts are for equilibrated systems), then each kernel of eq. 25
    runs `steps` NVE steps (default 2000 = 1 ps) from the same R, V and
    density: adaptive- and fixed-rank Krylov against the XL-BOMD kernel -cI.
    The slope of E_tot(t) per atom is fitted with its standard error."""
    import collections
    import synth
    import paper_2303_00689_gb300 as kx
    from paper_2303_00689_gb300 import build
    build.build()
    mol = synth.fullerene_c60(copies=args.drift_copies, bond=1.60)
    table = kx.param_table(synth.table_to_array(synth.synthetic_table(1)))
    V0 = synth.maxwell_boltzmann(mol.Z, 300.0, seed=5)
    base = dict(Te=5000.0, dt=0.5, precision=kx.SIM_PREC_MIXED, scf_tol=1e-7, scf_max=300, scf_accept=1)
    cfg = kx.sim_config_default(m_max=4, m_min=4, langevin_gamma=0.02, langevin_T=300.0, langevin_seed=11,
                                **base)
    h = kx.sim_create(cfg, table, mol.Z, mol.R, V=V0)
    kx.sim_step(h, args.drift_equil, records=False)
    R, V, _, D = kx.sim_get_state(h, mol.natoms)
    kx.sim_destroy(h)
    modes = [("krylov adaptive m 4-12, tol 1e-3", dict(m_max=12, m_min=4, krylov_tol=1e-3)),
             ("krylov m 4", dict(m_max=4, m_min=4)),
             ("xl -cI, c = 1", dict(kernel=kx.SIM_KERNEL_XL, xl_c=1.0)),
             ("xl -cI, c = 0.9", dict(kernel=kx.SIM_KERNEL_XL, xl_c=0.9))]
    nst = args.steps if args.steps > 10 else 2000
    runs = []
    for name, kw in modes:
        cfg = kx.sim_config_default(**base, **kw)
        h = kx.sim_create(cfg, table, mol.Z, R, V=V, P0=D)
        it, res = kx.sim_scf_info(h)
        t = time.perf_counter()
        recs = kx.sim_step(h, nst)
        dt_s = time.perf_counter() - t
        kx.sim_destroy(h)
        E = np.array([r["E_tot"] for r in recs])
        Ek = np.array([r["E_kin"] for r in recs])
        t_ps = np.arange(len(E)) * 0.5e-3
        slope, se = _fit_slope(t_ps, E)
        runs.append({"kernel": name, "ms_per_step": 1e3 * dt_s / nst,
                     "drift_eV_per_ps_atom": slope / mol.natoms, "stderr_eV_per_ps_atom": se / mol.natoms,
                     "E_tot_std_eV": float(E.std()), "E_tot_ptp_eV": float(np.ptp(E)),
                     "E_kin_ptp_eV": float(np.ptp(Ek)), "finite": bool(np.all(np.isfinite(E))),
                     "max_residual": max(r["res_norm"] for r in recs),
                     "ranks": dict(sorted(collections.Counter(r["rank"] for r in recs).items())),
                     "scf": {"iterations": it, "residual": res}})
    out = {"metric": "energy drift (eV/ps/atom), shadow XL-BOMD", "value": runs[0]["drift_eV_per_ps_atom"],
           "unit": "eV/ps/atom", "n_gpus": 1, "steps": nst, "warmup": 0,
           "ms_per_step": runs[0]["ms_per_step"], "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64+bf16-slices", "data": "synthetic",
           "config": {"workload": f"{args.drift_copies} C60 cages, {mol.natoms} atoms, n = {mol.norb}, C-C 1.60 A",
                      "Te_K": 5000.0, "dt_fs": 0.5,
                      "equilibration": f"{args.drift_equil} Langevin steps at 300 K, gamma 0.02/fs, Krylov m 4"},
           "runs": runs}
    print(json.dumps(out), flush=True)


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    res = oracle_sample()
    out = {"metric": METRIC, "value": res["value"], "unit": "atom-steps/s", "n_gpus": world, "steps": 1,
           "warmup": 0, "ms_per_step": 1e3 * res["seconds_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(WORKLOAD, precision="fp64 (oracle)"), "impl": "reference",
           "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")},
           "e2e": {"value": res["value"], "unit": "atom-steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    p.add_argument("--no-fp64-context", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the short serving and batch records")
    p.add_argument("--extra-serve-requests", type=int, default=12)
    p.add_argument("--extra-serve-nmax", type=int, default=300)
    p.add_argument("--extra-batch-molecules", type=int, default=32)
    p.add_argument("--state", default=None, help=argparse.SUPPRESS)
    p.add_argument("--cpu-timeout", type=float, default=600.0)
    p.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--workload", choices=("md840", "batch", "serve", "drift"), default="md840",
                   help="md840: the headline single-system step; batch: 128-molecule batch; serve: "
                        "Poisson-arrival serving")
    p.add_argument("--kernel", choices=("krylov", "xl", "bomd"), default="krylov",
                   help="kernel of eq. 25: Krylov (the method), XL-BOMD -cI or Born-Oppenheimer (comparison modes)")
    p.add_argument("--serve-requests", type=int, default=48)
    p.add_argument("--serve-nmax", type=int, default=600)
    p.add_argument("--serve-timeout", type=float, default=900.0)
    p.add_argument("--serve-graphs", type=int, default=1)
    p.add_argument("--serve-admit", type=int, default=4, help="server admission threads")
    p.add_argument("--profile-run", action="store_true",
                   help="short run for ncu (no SCF, no baselines); prints launch counts")
    p.add_argument("--drift-copies", type=int, default=2, help="C60 cages in the drift workload")
    p.add_argument("--drift-equil", type=int, default=400, help="Langevin steps before the NVE drift runs")
    p.add_argument("--profile-natoms", type=int, default=None,
                   help="atoms of the carbon packing in --profile-run (default: the headline 840)")
    args = p.parse_args()
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.state)), flush=True)
        return
    if args.profile_run:
        profile_run(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    KERNEL_MODE[0] = {"krylov": 0, "xl": 1, "bomd": 2}[args.kernel]
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "drift":
        run_drift(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
