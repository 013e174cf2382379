"""Thin ctypes binding of the D-NGD C ABI (include/dngd.h).

Argument marshalling only: every step of the D-NGD path runs in the CUDA
library.  Arrays may be torch tensors (CUDA or CPU, float64, contiguous) or
numpy float64 arrays (host).  Device tensors are passed by pointer; host
arrays are staged by the library itself.  If the library is missing the import
fails loudly; there is no fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdngd.so")

MAX_LAYERS = 12
MAX_DIM = 8
MAX_CLASSES = 4

FP64, MIXED_BF16, MIXED_TF32, MIXED_OZ, MIXED_OZ64 = 0, 1, 2, 3, 4
DENSE, PCG = 0, 1
PCG_OP_TC3, PCG_OP_COMPENSATED = 0, 1
FACTOR_SLICED, FACTOR_DF = 0, 1
SPACE_DUAL, SPACE_PRIMAL, SPACE_AUTO = 0, 1, 2

STATUS = {
    0: "DNGD_OK", -1: "DNGD_ERR_INVALID_ARG", -2: "DNGD_ERR_NOT_SPD", -3: "DNGD_ERR_NO_CONVERGE",
    -4: "DNGD_ERR_NONFINITE", -5: "DNGD_ERR_BUDGET", -6: "DNGD_ERR_TIMEOUT", -7: "DNGD_ERR_CUDA",
    -8: "DNGD_ERR_STATE", -9: "DNGD_ERR_OOM",
}

STAGES = dict(r=0, alpha=1, v=2, fvv=3, beta=4, a=5, gram=6, chol=7, kci=8, gram64=9, linv=10, chol64=11)


class DngdError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"{where}: {STATUS.get(status, status)} ({status})")
        self.status = status


class ClassDesc(C.Structure):
    _fields_ = [("count", C.c_int), ("c_val", C.c_double), ("c_grad", C.c_double * MAX_DIM),
                ("c_lap", C.c_double), ("lap_mask", C.c_int * MAX_DIM)]


class ProblemDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("widths", C.c_int * (MAX_LAYERS + 1)), ("n_classes", C.c_int),
                ("classes", ClassDesc * MAX_CLASSES), ("precision", C.c_int), ("solver", C.c_int),
                ("lam", C.c_double), ("use_ga", C.c_int), ("eps_norm", C.c_double),
                ("ga_ratio_max", C.c_double), ("refine_max_it", C.c_int), ("refine_tol", C.c_double),
                ("shift_mu", C.c_double), ("pcg_rank", C.c_int), ("pcg_tol", C.c_double),
                ("pcg_max_it", C.c_int), ("pcg_seed", C.c_uint64), ("keep_gram", C.c_int),
                ("lambda_cap", C.c_double), ("pcg_operator", C.c_int), ("factor_update", C.c_int),
                ("solve_space", C.c_int)]


class StepInfo(C.Structure):
    _fields_ = [("loss", C.c_double), ("norm_v", C.c_double), ("norm_a", C.c_double), ("ga_ratio", C.c_double),
                ("ga_accepted", C.c_int), ("solve_iters", C.c_int * 2), ("solve_relres", C.c_double * 2),
                ("not_spd_column", C.c_int), ("device_status", C.c_int), ("phase_ms", C.c_float * 8),
                ("shift_used", C.c_double), ("factor_attempts", C.c_int), ("jt_ms", C.c_float),
                ("j_ms", C.c_float), ("lambda_used", C.c_double), ("gram_kernel_ms", C.c_float)]

    def as_dict(self):
        return dict(loss=self.loss, norm_v=self.norm_v, norm_a=self.norm_a, ga_ratio=self.ga_ratio,
                    ga_accepted=bool(self.ga_accepted), solve_iters=list(self.solve_iters),
                    solve_relres=list(self.solve_relres), not_spd_column=self.not_spd_column,
                    device_status=self.device_status, phase_ms=list(self.phase_ms),
                    shift_used=self.shift_used, factor_attempts=self.factor_attempts, jt_ms=self.jt_ms,
                    j_ms=self.j_ms, lambda_used=self.lambda_used, gram_kernel_ms=self.gram_kernel_ms)


class ServerCfg(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_slots", C.c_int), ("line_search_points", C.c_int)]


class JobDesc(C.Structure):
    _fields_ = [("desc", ProblemDesc), ("theta0", C.c_void_p), ("X", C.c_void_p), ("target", C.c_void_p),
                ("n_steps", C.c_int)]


class JobState(C.Structure):
    _fields_ = [("state", C.c_int), ("steps_done", C.c_int), ("status", C.c_int), ("loss", C.c_double),
                ("queue_s", C.c_double), ("run_s", C.c_double)]


class ServingStats(C.Structure):
    _fields_ = [("steps_per_s", C.c_double), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("steps_total", C.c_longlong), ("admitted", C.c_int), ("rejected", C.c_int), ("done", C.c_int),
                ("failed", C.c_int), ("running", C.c_int), ("queued", C.c_int), ("hbm_used_bytes", C.c_size_t),
                ("hbm_budget_bytes", C.c_size_t)]


RESAMPLE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p)


class TrainCfg(C.Structure):
    _fields_ = [("max_iters", C.c_int), ("time_budget_s", C.c_double), ("loss_target", C.c_double),
                ("resample_every", C.c_int), ("resample", RESAMPLE_FN), ("user", C.c_void_p),
                ("etas", C.POINTER(C.c_double)), ("k", C.c_int)]


class TrainResult(C.Structure):
    _fields_ = [("iters", C.c_int), ("stop", C.c_int), ("loss", C.c_double), ("elapsed_s", C.c_double)]


STOP_REASONS = {0: "iters", 1: "budget", 2: "loss"}

JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED, JOB_CANCELLED = range(5)
JOB_STATES = {JOB_QUEUED: "queued", JOB_RUNNING: "running", JOB_DONE: "done", JOB_FAILED: "failed",
              JOB_CANCELLED: "cancelled"}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdngd.so not built at {LIB_PATH}: run __graft_entry__.build() (no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    D = C.POINTER(C.c_double)
    sigs = {
        "dngd_status_string": (C.c_char_p, [C.c_int]),
        "dngd_version": (C.c_char_p, []),
        "dngd_launch_count": (C.c_uint64, []),
        "dngd_num_params": (C.c_int64, [C.POINTER(ProblemDesc)]),
        "dngd_create": (C.c_int, [C.POINTER(P), C.POINTER(ProblemDesc), P]),
        "dngd_workspace_bytes": (C.c_int, [C.POINTER(ProblemDesc), C.POINTER(C.c_size_t)]),
        "dngd_destroy": (C.c_int, [P]),
        "dngd_set_timing": (C.c_int, [P, C.c_int]),
        "dngd_set_lambda": (C.c_int, [P, C.c_double]),
        "dngd_step": (C.c_int, [P, P, P, P, P, C.POINTER(StepInfo)]),
        "dngd_solve": (C.c_int, [P, P, P]),
        "dngd_solve_space_of": (C.c_int, [P]),
        "dngd_loss": (C.c_int, [P, P, P, P, P, D, C.c_int, D]),
        "dngd_line_search": (C.c_int, [P, P, P, P, P, D, C.c_int, P, D]),
        "dngd_residual_jacobian": (C.c_int, [P, P, P, P, P, P]),
        "dngd_fvv": (C.c_int, [P, P, P, P, P, P]),
        "dngd_get_stage": (C.c_int, [P, C.c_int, P]),
        "dngd_gram_bf16_noalloc": (C.c_int, [P, C.c_int, C.c_int, C.c_longlong, P, C.c_longlong, C.c_double, P]),
        "dngd_set_landmarks": (C.c_int, [P, P, C.c_int]),
        "dngd_step_async": (C.c_int, [P, P, P, P, P]),
        "dngd_step_wait": (C.c_int, [P, C.POINTER(StepInfo)]),
        "dngd_batch_create": (C.c_int, [C.POINTER(P), C.POINTER(ProblemDesc), C.c_int, P]),
        "dngd_batch_destroy": (C.c_int, [P]),
        "dngd_batch_size": (C.c_int, [P]),
        "dngd_batch_step": (C.c_int, [P, C.POINTER(P), C.POINTER(P), C.POINTER(P), C.POINTER(P),
                                      C.POINTER(StepInfo)]),
        "dngd_batch_context": (P, [P, C.c_int]),
        "dngd_kvp": (C.c_int, [P, P, P]),
        "dngd_precond_apply": (C.c_int, [P, P, P]),
        "dngd_line_search_async": (C.c_int, [P, P, P, P, P, D, C.c_int]),
        "dngd_check_wait_expiry": (C.c_int, [P, C.c_double]),
        "dngd_server_create": (C.c_int, [C.POINTER(P), C.POINTER(ServerCfg)]),
        "dngd_server_destroy": (C.c_int, [P]),
        "dngd_submit": (C.c_int, [P, C.POINTER(JobDesc), C.POINTER(C.c_uint64)]),
        "dngd_poll": (C.c_int, [P, C.c_uint64, C.POINTER(JobState), P]),
        "dngd_cancel": (C.c_int, [P, C.c_uint64]),
        "dngd_server_stats": (C.c_int, [P, C.POINTER(ServingStats)]),
        "dngd_server_drain": (C.c_int, [P, C.c_double]),
        "dngd_train": (C.c_int, [P, P, P, P, C.POINTER(TrainCfg), D, C.POINTER(TrainResult)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()

EXPORTED = ["dngd_status_string", "dngd_version", "dngd_launch_count", "dngd_num_params", "dngd_create", "dngd_workspace_bytes",
            "dngd_destroy", "dngd_set_timing", "dngd_set_lambda", "dngd_step", "dngd_solve", "dngd_solve_space_of",
            "dngd_loss",
            "dngd_line_search", "dngd_residual_jacobian", "dngd_fvv", "dngd_get_stage",
            "dngd_gram_bf16_noalloc", "dngd_set_landmarks", "dngd_kvp", "dngd_precond_apply",
            "dngd_step_async", "dngd_step_wait", "dngd_batch_create", "dngd_batch_destroy", "dngd_batch_size",
            "dngd_batch_step", "dngd_batch_context", "dngd_line_search_async", "dngd_server_create",
            "dngd_server_destroy", "dngd_submit", "dngd_poll", "dngd_cancel", "dngd_server_stats",
            "dngd_server_drain", "dngd_check_wait_expiry", "dngd_train"]


def _check(status, where):
    if status != 0:
        raise DngdError(status, where)


def _ptr(a):
    """Pointer of a float64 array: torch tensor (CUDA or CPU) or numpy."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensor must be contiguous"
        return C.c_void_p(a.data_ptr())
    assert isinstance(a, np.ndarray) and a.flags.c_contiguous
    return a.ctypes.data_as(C.c_void_p)


def make_desc(spec, precision=FP64, lam=None, use_ga=True, eps_norm=0.0, ga_ratio_max=0.5, refine_max_it=200,
              refine_tol=1e-10, shift_mu=0.0, keep_gram=False, solver=DENSE, pcg_rank=512, pcg_tol=1e-6,
              pcg_max_it=500, lambda_cap=0.0, pcg_operator=PCG_OP_TC3, factor_update=0,
              solve_space=SPACE_DUAL):
    """Problem descriptor from a workload dict (see workloads.py).
    lambda_cap > 0 selects the damping rule lambda_k = min(L(theta_k), cap);
    pcg_operator: the matrix-free operator's GEMMs (PCG_OP_TC3 or
    PCG_OP_COMPENSATED); factor_update: the exact-Gram factor's trailing
    updates (FACTOR_SLICED or FACTOR_DF, what batches use); solve_space: the
    dense FP64 system's space (SPACE_DUAL, SPACE_PRIMAL or SPACE_AUTO)."""
    d = ProblemDesc()
    widths = list(spec["widths"])
    d.n_layers = len(widths) - 1
    for i, w in enumerate(widths):
        d.widths[i] = int(w)
    d.n_classes = len(spec["classes"])
    for c, cl in enumerate(spec["classes"]):
        cd = d.classes[c]
        cd.count = int(cl["count"])
        cd.c_val = float(cl["c_val"])
        for k, g in enumerate(cl["c_grad"]):
            cd.c_grad[k] = float(g)
        cd.c_lap = float(cl["c_lap"])
        for k, b in enumerate(cl["lap_mask"]):
            cd.lap_mask[k] = int(bool(b))
    d.precision = int(precision)
    d.solver = int(solver)
    d.pcg_rank = int(pcg_rank)
    d.pcg_tol = float(pcg_tol)
    d.pcg_max_it = int(pcg_max_it)
    d.lam = float(spec["lam"] if lam is None else lam)
    d.use_ga = int(bool(use_ga))
    d.eps_norm = float(eps_norm)
    d.ga_ratio_max = float(ga_ratio_max)
    d.refine_max_it = int(refine_max_it)
    d.refine_tol = float(refine_tol)
    d.shift_mu = float(shift_mu)
    d.keep_gram = int(bool(keep_gram))
    d.lambda_cap = float(lambda_cap)
    d.pcg_operator = int(pcg_operator)
    d.factor_update = int(factor_update)
    d.solve_space = int(solve_space)
    return d


def dngd_launch_count():
    return int(lib.dngd_launch_count())


def dngd_num_params(desc):
    return int(lib.dngd_num_params(C.byref(desc)))


def dngd_workspace_bytes(desc):
    b = C.c_size_t(0)
    _check(lib.dngd_workspace_bytes(C.byref(desc), C.byref(b)), "dngd_workspace_bytes")
    return int(b.value)


def dngd_gram_bf16_noalloc(J, m, n, ld, K, ldk, shift, stream=None):
    """K = J J^T + shift I from a BF16 device matrix, with no device allocation
    (see include/dngd.h).  Returns the status code."""
    s = C.c_void_p(int(stream)) if stream else None
    return int(lib.dngd_gram_bf16_noalloc(_ptr(J), int(m), int(n), int(ld), _ptr(K), int(ldk), float(shift), s))


class Context:
    """One step context (dngd_create / dngd_destroy)."""

    def __init__(self, desc, stream=None):
        self.desc = desc
        self._h = C.c_void_p()
        s = C.c_void_p(int(stream)) if stream else None
        _check(lib.dngd_create(C.byref(self._h), C.byref(desc), s), "dngd_create")
        self.n = dngd_num_params(desc)
        self.m = sum(desc.classes[c].count for c in range(desc.n_classes))

    def close(self):
        if self._h:
            lib.dngd_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_timing(self, on=True):
        _check(lib.dngd_set_timing(self._h, int(on)), "dngd_set_timing")

    def set_lambda(self, lam):
        _check(lib.dngd_set_lambda(self._h, float(lam)), "dngd_set_lambda")

    def step(self, theta, X, target, delta_out, want_info=True):
        info = StepInfo() if want_info else None
        st = lib.dngd_step(self._h, _ptr(theta), _ptr(X), _ptr(target), _ptr(delta_out),
                           C.byref(info) if info is not None else None)
        _check(st, "dngd_step")
        return info.as_dict() if info is not None else None

    @property
    def solve_space(self):
        """SPACE_PRIMAL or SPACE_DUAL (SPACE_AUTO resolved at creation)."""
        return int(lib.dngd_solve_space_of(self._h))

    def solve(self, rhs, x_out):
        _check(lib.dngd_solve(self._h, _ptr(rhs), _ptr(x_out)), "dngd_solve")

    def loss(self, theta, X, target, delta, etas):
        etas = np.ascontiguousarray(etas, dtype=np.float64)
        out = np.zeros(etas.size)
        dp = C.POINTER(C.c_double)
        _check(lib.dngd_loss(self._h, _ptr(theta), _ptr(X), _ptr(target), _ptr(delta),
                             etas.ctypes.data_as(dp), int(etas.size), out.ctypes.data_as(dp)), "dngd_loss")
        return out

    def line_search(self, theta, X, target, delta, etas, theta_out):
        etas = np.ascontiguousarray(etas, dtype=np.float64)
        eta = C.c_double(0.0)
        _check(lib.dngd_line_search(self._h, _ptr(theta), _ptr(X), _ptr(target), _ptr(delta),
                                    etas.ctypes.data_as(C.POINTER(C.c_double)), int(etas.size), _ptr(theta_out),
                                    C.byref(eta)), "dngd_line_search")
        return eta.value

    def line_search_async(self, theta, X, target, delta, etas):
        """theta += eta* delta on the device (no synchronisation)."""
        etas = np.ascontiguousarray(etas, dtype=np.float64)
        _check(lib.dngd_line_search_async(self._h, _ptr(theta), _ptr(X), _ptr(target), _ptr(delta),
                                          etas.ctypes.data_as(C.POINTER(C.c_double)), int(etas.size)),
               "dngd_line_search_async")

    def check_wait_expiry(self, limit_ms=5.0):
        """Status of one deliberately unsatisfiable bounded device wait."""
        return int(lib.dngd_check_wait_expiry(self._h, float(limit_ms)))

    def residual_jacobian(self, theta, X, target, r_out, J_out=None):
        _check(lib.dngd_residual_jacobian(self._h, _ptr(theta), _ptr(X), _ptr(target), _ptr(r_out),
                                          _ptr(J_out)), "dngd_residual_jacobian")

    def fvv(self, theta, X, target, v, out):
        _check(lib.dngd_fvv(self._h, _ptr(theta), _ptr(X), _ptr(target), _ptr(v), _ptr(out)), "dngd_fvv")

    def set_landmarks(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        _check(lib.dngd_set_landmarks(self._h, idx.ctypes.data_as(C.c_void_p), int(idx.size)), "dngd_set_landmarks")

    def kvp(self, v, out):
        _check(lib.dngd_kvp(self._h, _ptr(v), _ptr(out)), "dngd_kvp")

    def precond_apply(self, x, out):
        _check(lib.dngd_precond_apply(self._h, _ptr(x), _ptr(out)), "dngd_precond_apply")

    def step_async(self, theta, X, target, delta_out):
        _check(lib.dngd_step_async(self._h, _ptr(theta), _ptr(X), _ptr(target), _ptr(delta_out)),
               "dngd_step_async")

    def step_wait(self):
        info = StepInfo()
        _check(lib.dngd_step_wait(self._h, C.byref(info)), "dngd_step_wait")
        return info.as_dict()

    def get_stage(self, name, out):
        _check(lib.dngd_get_stage(self._h, STAGES[name], _ptr(out)), "dngd_get_stage")

    def train(self, theta, X, target, max_iters, time_budget_s=0.0, loss_target=0.0, resample_every=0,
              resample=None, etas=None):
        """dngd_train on device tensors (theta updated in place).  resample(it)
        rewrites X and target in place (device work finished on return).
        Returns (result dict, loss history array of the completed iterations)."""
        cfg = TrainCfg()
        cfg.max_iters = int(max_iters)
        cfg.time_budget_s = float(time_budget_s)
        cfg.loss_target = float(loss_target)
        cfg.resample_every = int(resample_every)
        if resample is not None:
            def cb(user, it, xp, tp):
                try:
                    resample(int(it))
                    return 0
                except Exception:
                    return -1
            cfg.resample = RESAMPLE_FN(cb)
        else:
            cfg.resample = RESAMPLE_FN()
        keep = None
        if etas is not None:
            keep = np.ascontiguousarray(etas, dtype=np.float64)
            cfg.etas = keep.ctypes.data_as(C.POINTER(C.c_double))
            cfg.k = int(keep.size)
        hist = np.full(int(max_iters), np.nan)
        res = TrainResult()
        _check(lib.dngd_train(self._h, _ptr(theta), _ptr(X), _ptr(target), C.byref(cfg),
                              hist.ctypes.data_as(C.POINTER(C.c_double)), C.byref(res)), "dngd_train")
        out = dict(iters=res.iters, stop=STOP_REASONS.get(res.stop, res.stop), loss=res.loss, elapsed_s=res.elapsed_s)
        return out, hist[:res.iters if res.stop != 2 else res.iters + 1]


class _Borrowed(Context):
    """A context owned by a batch (not destroyed by Python)."""

    def __init__(self, handle, desc):
        self.desc = desc
        self._h = C.c_void_p(handle)
        self.n = dngd_num_params(desc)
        self.m = sum(desc.classes[c].count for c in range(desc.n_classes))

    def close(self):
        self._h = C.c_void_p()


class Batch:
    """dngd_batch: independent instances stepped by one CUDA-graph launch."""

    def __init__(self, descs, stream=None):
        self.descs = list(descs)
        arr = (ProblemDesc * len(self.descs))(*self.descs)
        self._h = C.c_void_p()
        s = C.c_void_p(int(stream)) if stream else None
        _check(lib.dngd_batch_create(C.byref(self._h), arr, len(self.descs), s), "dngd_batch_create")

    def __len__(self):
        return int(lib.dngd_batch_size(self._h))

    def close(self):
        if self._h:
            lib.dngd_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def context(self, i):
        return _Borrowed(lib.dngd_batch_context(self._h, int(i)), self.descs[i])

    def step(self, thetas, Xs, targets, deltas):
        n = len(self.descs)
        P = C.c_void_p
        arrs = [(P * n)(*[_ptr(a) for a in lst]) for lst in (thetas, Xs, targets, deltas)]
        infos = (StepInfo * n)()
        _check(lib.dngd_batch_step(self._h, arrs[0], arrs[1], arrs[2], arrs[3], infos), "dngd_batch_step")
        return [i.as_dict() for i in infos]


class Server:
    """dngd_server: PINN solve jobs admitted by HBM budget and slot count,
    each job's iterations (step + line search + update) kept in flight on its
    own stream by a native worker thread."""

    def __init__(self, hbm_budget_bytes=0, max_slots=8, line_search_points=31):
        cfg = ServerCfg(int(hbm_budget_bytes), int(max_slots), int(line_search_points))
        self._h = C.c_void_p()
        _check(lib.dngd_server_create(C.byref(self._h), C.byref(cfg)), "dngd_server_create")
        self._n = {}

    def close(self):
        if self._h:
            lib.dngd_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, desc, theta0, X, target, n_steps):
        """Inputs (numpy or torch float64) are copied before this returns."""
        keep = [np.ascontiguousarray(a, dtype=np.float64) if isinstance(a, np.ndarray) else a
                for a in (theta0, X, target)]
        job = JobDesc(desc, _ptr(keep[0]), _ptr(keep[1]), _ptr(keep[2]), int(n_steps))
        jid = C.c_uint64(0)
        _check(lib.dngd_submit(self._h, C.byref(job), C.byref(jid)), "dngd_submit")
        self._n[jid.value] = dngd_num_params(desc)
        return jid.value

    def poll(self, job_id, theta_out=None):
        st = JobState()
        _check(lib.dngd_poll(self._h, C.c_uint64(job_id), C.byref(st), _ptr(theta_out)), "dngd_poll")
        return dict(state=JOB_STATES[st.state], steps_done=st.steps_done, status=st.status, loss=st.loss,
                    queue_s=st.queue_s, run_s=st.run_s)

    def result(self, job_id):
        theta = np.zeros(self._n[job_id])
        info = self.poll(job_id, theta)
        return info, (theta if info["state"] == "done" else None)

    def cancel(self, job_id):
        _check(lib.dngd_cancel(self._h, C.c_uint64(job_id)), "dngd_cancel")

    def stats(self):
        st = ServingStats()
        _check(lib.dngd_server_stats(self._h, C.byref(st)), "dngd_server_stats")
        return {f: getattr(st, f) for f, _ in ServingStats._fields_}

    def drain(self, timeout_s=600.0):
        _check(lib.dngd_server_drain(self._h, float(timeout_s)), "dngd_server_drain")
