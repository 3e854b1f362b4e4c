"""Python binding of the GB300 KSA-XL-BOMD CUDA library (``libksaxl.so``).

Thin ctypes marshalling over the C ABI declared in ``include/sim.h``: every
function here has the C name, converts numpy arrays to pointers and raises
``SimError`` on a non-zero status.  All computation happens in the CUDA
library; importing this module without the built library raises at the first
call (there is no CPU fallback).

Build the library with ``python -m paper_2303_00689_gb300.build`` (needs nvcc).
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libksaxl.so")

SIM_OK, SIM_PENDING, SIM_EINVAL, SIM_ENOMEM, SIM_ENOCONV, SIM_ENUMERIC, SIM_ETIMEOUT, SIM_EINTERNAL = range(8)
SIM_PREC_FP64, SIM_PREC_MIXED = 0, 1
SIM_KERNEL_KRYLOV, SIM_KERNEL_XL, SIM_KERNEL_BOMD = 0, 1, 2
SIM_MAT_X, SIM_MAT_D0, SIM_MAT_FOCK, SIM_MAT_H, SIM_MAT_KERNEL, SIM_MAT_Q, SIM_MAT_XHIST = range(7)
SIM_NFIELDS = 23

EXPORTED = (
    "sim_config_default", "sim_create", "sim_scf_info", "sim_norb", "sim_nocc", "sim_step", "sim_step_async", "sim_step_host",
    "sim_last_result", "sim_get_state", "sim_set_state", "sim_get_matrix", "sim_get_vector",
    "sim_profile_enable", "sim_phase_count", "sim_phase_name", "sim_phase_times",
    "sim_launch_count", "sim_stream", "sim_destroy", "sim_last_error", "sim_debug_tc_gemm",
    "sim_debug_tc_gemm_grouped",
    "sim_tc_gemm_noalloc", "sim_records", "sim_wait", "sim_enable_graphs", "sim_batch_step",
    "sim_estimate_bytes", "sim_server_create", "sim_submit", "sim_poll", "sim_server_stats_get",
    "sim_server_drain", "sim_server_destroy", "sim_save", "sim_load", "sim_batch_create", "sim_batch_run",
    "sim_batch_destroy", "sim_batch_groups", "sim_measure_peak", "sim_debug_barrier_limit", "sim_debug_wait_expiry",
)


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"status {code}: {msg}")
        self.code = code


class sim_config(C.Structure):
    _fields_ = [("Te", C.c_double), ("dt", C.c_double), ("m_max", C.c_int), ("m_min", C.c_int),
                ("krylov_tol", C.c_double), ("precision", C.c_int), ("scf_tol", C.c_double),
                ("scf_max", C.c_int), ("scf_mix", C.c_double), ("device", C.c_int),
                ("stream", C.c_void_p), ("scf_krylov", C.c_int), ("scf_accept", C.c_int),
                ("kernel", C.c_int), ("xl_c", C.c_double), ("langevin_gamma", C.c_double),
                ("langevin_T", C.c_double), ("langevin_seed", C.c_ulonglong)]


class sim_param_table(C.Structure):
    _fields_ = [("v", (C.c_double * SIM_NFIELDS) * 4)]


class sim_step_result(C.Structure):
    _fields_ = [("E_kin", C.c_double), ("U", C.c_double), ("E_tot", C.c_double), ("mu", C.c_double),
                ("gap", C.c_double), ("res_norm", C.c_double), ("fit_err", C.c_double),
                ("rank", C.c_int), ("pad", C.c_int), ("dipole", C.c_double * 3)]


def _record_dict(r):
    d = {f: getattr(r, f) for f, _ in sim_step_result._fields_}
    d["dipole"] = tuple(r.dipole)
    return d


class sim_server_config(C.Structure):
    _fields_ = [("device", C.c_int), ("max_active", C.c_int), ("hbm_budget_bytes", C.c_size_t),
                ("use_graphs", C.c_int), ("admission_threads", C.c_int)]


class sim_request(C.Structure):
    _fields_ = [("cfg", sim_config), ("table", sim_param_table), ("natoms", C.c_int),
                ("Z", C.POINTER(C.c_int)), ("R", C.POINTER(C.c_double)), ("V", C.POINTER(C.c_double)),
                ("charge", C.c_int), ("nsteps", C.c_int), ("R_out", C.POINTER(C.c_double)),
                ("V_out", C.POINTER(C.c_double)), ("F_out", C.POINTER(C.c_double)),
                ("records", C.POINTER(sim_step_result))]


class sim_traj_result(C.Structure):
    _fields_ = [("status", C.c_int), ("steps_done", C.c_int), ("queue_ms", C.c_double),
                ("create_ms", C.c_double), ("run_ms", C.c_double), ("error", C.c_char * 160)]


class sim_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong), ("failed", C.c_longlong),
                ("queued", C.c_longlong), ("active", C.c_longlong), ("max_active_seen", C.c_longlong),
                ("atom_steps", C.c_longlong), ("step_p50_ms", C.c_double), ("step_p99_ms", C.c_double),
                ("elapsed_s", C.c_double), ("hbm_in_use", C.c_size_t), ("hbm_budget", C.c_size_t),
                ("threads", C.c_char * 512)]


_lib_handle = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run python -m paper_2303_00689_gb300.build)")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        dp = P(C.c_double)
        L.sim_config_default.argtypes = [P(sim_config)]
        L.sim_config_default.restype = None
        L.sim_create.argtypes = [P(sim_config), P(sim_param_table), C.c_int, P(C.c_int), dp, dp, C.c_int,
                                 dp, P(C.c_void_p)]
        L.sim_norb.argtypes = [C.c_void_p]
        L.sim_scf_info.argtypes = [C.c_void_p, P(C.c_int), dp]
        L.sim_nocc.argtypes = [C.c_void_p]
        L.sim_step.argtypes = [C.c_void_p, C.c_int, P(sim_step_result)]
        L.sim_step_async.argtypes = [C.c_void_p, C.c_int]
        L.sim_step_host.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, P(sim_step_result)]
        L.sim_last_result.argtypes = [C.c_void_p, P(sim_step_result)]
        L.sim_get_state.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.sim_set_state.argtypes = [C.c_void_p, dp, dp, dp]
        L.sim_get_matrix.argtypes = [C.c_void_p, C.c_int, dp]
        L.sim_get_vector.argtypes = [C.c_void_p, C.c_int, dp]
        L.sim_profile_enable.argtypes = [C.c_void_p, C.c_int]
        L.sim_phase_count.argtypes = []
        L.sim_phase_name.argtypes = [C.c_int]
        L.sim_phase_name.restype = C.c_char_p
        L.sim_phase_times.argtypes = [C.c_void_p, dp, P(C.c_longlong), dp]
        L.sim_launch_count.argtypes = []
        L.sim_launch_count.restype = C.c_longlong
        L.sim_stream.argtypes = [C.c_void_p]
        L.sim_stream.restype = C.c_void_p
        L.sim_destroy.argtypes = [C.c_void_p]
        L.sim_destroy.restype = None
        L.sim_debug_tc_gemm.argtypes = [C.c_int, dp, dp, C.c_int, C.c_int, dp]
        L.sim_debug_tc_gemm_grouped.argtypes = [C.c_int, dp, dp, C.c_int, C.c_int, dp]
        L.sim_tc_gemm_noalloc.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                          C.c_void_p]
        L.sim_records.argtypes = [C.c_void_p, P(sim_step_result), C.c_int]
        L.sim_measure_peak.argtypes = [C.c_int, C.c_int, dp]
        L.sim_debug_barrier_limit.argtypes = [C.c_int, C.c_ulonglong]
        L.sim_debug_wait_expiry.argtypes = [C.c_int, C.c_longlong]
        L.sim_save.argtypes = [C.c_void_p, C.c_char_p]
        L.sim_batch_create.argtypes = [P(C.c_void_p), C.c_int, P(C.c_void_p)]
        L.sim_batch_run.argtypes = [C.c_void_p, C.c_int]
        L.sim_batch_destroy.argtypes = [C.c_void_p]
        L.sim_batch_destroy.restype = None
        L.sim_batch_groups.argtypes = [C.c_void_p]
        L.sim_load.argtypes = [C.c_char_p, C.c_int, C.c_void_p, P(C.c_void_p)]
        L.sim_wait.argtypes = [C.c_void_p]
        L.sim_enable_graphs.argtypes = [C.c_void_p, C.c_int]
        L.sim_batch_step.argtypes = [P(C.c_void_p), C.c_int, C.c_int]
        L.sim_estimate_bytes.argtypes = [P(sim_config), C.c_int, P(C.c_int)]
        L.sim_estimate_bytes.restype = C.c_size_t
        L.sim_server_create.argtypes = [P(sim_server_config), P(C.c_void_p)]
        L.sim_submit.argtypes = [C.c_void_p, P(sim_request), P(C.c_ulonglong)]
        L.sim_poll.argtypes = [C.c_void_p, C.c_ulonglong, P(sim_traj_result)]
        L.sim_server_stats_get.argtypes = [C.c_void_p, P(sim_server_stats)]
        L.sim_server_drain.argtypes = [C.c_void_p, C.c_double]
        L.sim_server_destroy.argtypes = [C.c_void_p]
        L.sim_server_destroy.restype = None
        L.sim_last_error.argtypes = []
        L.sim_last_error.restype = C.c_char_p
        _lib_handle = L
    return _lib_handle


def _check(rc):
    if rc != SIM_OK:
        raise SimError(rc, lib().sim_last_error().decode())
    return rc


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def sim_config_default(**overrides):
    cfg = sim_config()
    lib().sim_config_default(C.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def param_table(array):
    """(4, SIM_NFIELDS) float64 rows H, C, N, O -> sim_param_table."""
    arr = np.asarray(array, dtype=np.float64)
    if arr.shape != (4, SIM_NFIELDS):
        raise ValueError(f"parameter table must be (4, {SIM_NFIELDS})")
    t = sim_param_table()
    for i in range(4):
        for j in range(SIM_NFIELDS):
            t.v[i][j] = float(arr[i, j])
    return t


def sim_create(cfg, table, Z, R, V=None, charge=0, P0=None):
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    N = len(Z)
    R = _f64(R, (N, 3))
    V = _f64(V, (N, 3))
    P0 = _f64(P0)
    h = C.c_void_p()
    _check(lib().sim_create(C.byref(cfg), C.byref(table), N, Z.ctypes.data_as(C.POINTER(C.c_int)),
                            _dptr(R), _dptr(V), int(charge), _dptr(P0), C.byref(h)))
    return h


def sim_scf_info(h):
    it = C.c_int()
    res = C.c_double()
    _check(lib().sim_scf_info(h, C.byref(it), C.byref(res)))
    return it.value, res.value


def sim_norb(h):
    return lib().sim_norb(h)


def sim_nocc(h):
    return lib().sim_nocc(h)


def sim_step(h, nsteps, records=True):
    out = (sim_step_result * max(1, nsteps))() if records else None
    _check(lib().sim_step(h, int(nsteps), out))
    if not records:
        return None
    return [_record_dict(r) for r in out[:nsteps]]


def sim_step_async(h, nsteps):
    _check(lib().sim_step_async(h, int(nsteps)))


def sim_step_host(h, R_in, V_in, R_out, V_out, F_out, record=None):
    """One step with host buffers (arrays must be C-contiguous float64, natoms x 3)."""
    _check(lib().sim_step_host(h, _dptr(R_in), _dptr(V_in), _dptr(R_out), _dptr(V_out), _dptr(F_out),
                               C.byref(record) if record is not None else None))


def sim_last_result(h):
    r = sim_step_result()
    _check(lib().sim_last_result(h, C.byref(r)))
    return _record_dict(r)


def sim_get_state(h, natoms):
    R = np.empty((natoms, 3))
    V = np.empty((natoms, 3))
    F = np.empty((natoms, 3))
    n = sim_norb(h)
    D = np.empty((n, n))
    _check(lib().sim_get_state(h, _dptr(R), _dptr(V), _dptr(F), _dptr(D)))
    return R, V, F, D


def sim_set_state(h, R=None, V=None, Xhist=None):
    R, V, Xhist = _f64(R), _f64(V), _f64(Xhist)
    _check(lib().sim_set_state(h, _dptr(R), _dptr(V), _dptr(Xhist)))


def sim_get_matrix(h, which):
    n = sim_norb(h)
    out = np.empty((n, n))
    _check(lib().sim_get_matrix(h, int(which), _dptr(out)))
    return out


def sim_get_vector(h, which):
    out = np.empty(sim_norb(h))
    _check(lib().sim_get_vector(h, int(which), _dptr(out)))
    return out


def sim_profile_enable(h, enable=True):
    _check(lib().sim_profile_enable(h, 1 if enable else 0))


def sim_phase_names():
    L = lib()
    return [L.sim_phase_name(i).decode() for i in range(L.sim_phase_count())]


def sim_phase_times(h):
    L = lib()
    k = L.sim_phase_count()
    ms = (C.c_double * k)()
    cnt = (C.c_longlong * k)()
    work = (C.c_double * k)()
    _check(L.sim_phase_times(h, ms, cnt, work))
    names = sim_phase_names()
    return {names[i]: dict(ms=ms[i], launches=cnt[i], work=work[i]) for i in range(k)}


def sim_launch_count():
    return lib().sim_launch_count()


def sim_stream(h):
    return lib().sim_stream(h)


def sim_destroy(h):
    if h:
        lib().sim_destroy(h)


def sim_debug_tc_gemm(A, B, terms=1, sym=False):
    A = _f64(A)
    B = _f64(B)
    n = A.shape[0]
    out = np.empty((n, n))
    _check(lib().sim_debug_tc_gemm(n, _dptr(A), _dptr(B), int(terms), 1 if sym else 0, _dptr(out)))
    return out


def sim_debug_tc_gemm_grouped(A, B, sym=False, slices=3):
    A = _f64(A)
    B = _f64(B)
    n = A.shape[0]
    out = np.empty((n, n))
    _check(lib().sim_debug_tc_gemm_grouped(n, _dptr(A), _dptr(B), int(slices), 1 if sym else 0, _dptr(out)))
    return out


def sim_tc_gemm_noalloc(n, A_dev, B_dev, terms, sym, C_dev, stream=None):
    """Device pointers (ints) in and out; returns the raw status code."""
    return lib().sim_tc_gemm_noalloc(int(n), C.c_void_p(A_dev), C.c_void_p(B_dev), int(terms),
                                     1 if sym else 0, C.c_void_p(C_dev), C.c_void_p(stream or 0))


def sim_records(h, count):
    out = (sim_step_result * max(1, count))()
    _check(lib().sim_records(h, out, int(count)))
    return [_record_dict(r) for r in out[:count]]


def sim_save(h, path):
    _check(lib().sim_save(h, os.fsencode(path)))


def sim_load(path, device=0, stream=None):
    h = C.c_void_p()
    _check(lib().sim_load(os.fsencode(path), int(device), C.c_void_p(stream or 0), C.byref(h)))
    return h


def sim_wait(h):
    _check(lib().sim_wait(h))


def sim_enable_graphs(h, enable=True):
    _check(lib().sim_enable_graphs(h, 1 if enable else 0))


def sim_batch_step(handles, nsteps):
    arr = (C.c_void_p * max(1, len(handles)))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    _check(lib().sim_batch_step(arr, len(handles), int(nsteps)))


def sim_batch_create(handles):
    arr = (C.c_void_p * max(1, len(handles)))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    b = C.c_void_p()
    _check(lib().sim_batch_create(arr, len(handles), C.byref(b)))
    return b


def sim_batch_run(b, nsteps):
    _check(lib().sim_batch_run(b, int(nsteps)))


def sim_batch_groups(b):
    return int(lib().sim_batch_groups(b))


def sim_batch_destroy(b):
    if b:
        lib().sim_batch_destroy(b)


def sim_estimate_bytes(cfg, Z):
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    return lib().sim_estimate_bytes(C.byref(cfg), len(Z), Z.ctypes.data_as(C.POINTER(C.c_int)))


class Server:
    """sim_server_* wrapper: submit(...) -> ticket, poll(ticket) -> dict or None."""

    def __init__(self, device=0, max_active=64, hbm_budget_bytes=0, use_graphs=True, admission_threads=4):
        self._h = C.c_void_p()
        cfg = sim_server_config(device, max_active, hbm_budget_bytes, 1 if use_graphs else 0, admission_threads)
        _check(lib().sim_server_create(C.byref(cfg), C.byref(self._h)))
        self._keep = {}

    def submit(self, cfg, table, Z, R, V=None, charge=0, nsteps=0, records=True):
        Z = np.ascontiguousarray(Z, dtype=np.int32)
        N = len(Z)
        R = _f64(R, (N, 3))
        V = _f64(V, (N, 3))
        outs = dict(R=np.empty((N, 3)), V=np.empty((N, 3)), F=np.empty((N, 3)),
                    rec=(sim_step_result * max(1, nsteps))() if records else None)
        req = sim_request(cfg=cfg, table=table, natoms=N, Z=Z.ctypes.data_as(C.POINTER(C.c_int)),
                          R=_dptr(R), V=_dptr(V), charge=int(charge), nsteps=int(nsteps),
                          R_out=_dptr(outs["R"]), V_out=_dptr(outs["V"]), F_out=_dptr(outs["F"]),
                          records=outs["rec"])
        t = C.c_ulonglong()
        _check(lib().sim_submit(self._h, C.byref(req), C.byref(t)))
        outs["nsteps"] = nsteps
        self._keep[t.value] = outs
        return t.value

    def poll(self, ticket):
        res = sim_traj_result()
        rc = lib().sim_poll(self._h, C.c_ulonglong(ticket), C.byref(res))
        if rc == SIM_PENDING:
            return None
        _check(rc)
        outs = self._keep.pop(ticket)
        recs = None
        if outs["rec"] is not None:
            recs = [_record_dict(r) for r in outs["rec"][:res.steps_done]]
        return dict(status=res.status, steps_done=res.steps_done, queue_ms=res.queue_ms,
                    create_ms=res.create_ms, run_ms=res.run_ms, error=res.error.decode(),
                    R=outs["R"], V=outs["V"], F=outs["F"], records=recs)

    def stats(self):
        st = sim_server_stats()
        _check(lib().sim_server_stats_get(self._h, C.byref(st)))
        out = {f: getattr(st, f) for f, _ in sim_server_stats._fields_}
        out["threads"] = st.threads.decode(errors="replace")
        return out

    def drain(self, timeout_s=600.0):
        _check(lib().sim_server_drain(self._h, float(timeout_s)))

    def close(self):
        if self._h:
            lib().sim_server_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def sim_measure_peak(kind, device=0):
    """kind 0 / 1: FP64 / FP32 FMA throughput in TFLOP/s; kind 2: L2 read + write TB/s."""
    out = C.c_double(0.0)
    _check(lib().sim_measure_peak(int(device), int(kind), C.byref(out)))
    return out.value


def sim_debug_barrier_limit(ns, device=0):
    """Wall-time limit (ns) of the eigensolver's grid barriers (test hook)."""
    _check(lib().sim_debug_barrier_limit(int(device), int(ns)))


def sim_debug_wait_expiry(tries, device=0):
    """Raw status of one bounded mbarrier wait that nothing satisfies (test hook)."""
    return lib().sim_debug_wait_expiry(int(device), int(tries))


def sim_last_error():
    return lib().sim_last_error().decode()
