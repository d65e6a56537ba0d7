"""Thin ctypes binding of libgp (include/gp.h), same names as the C ABI.

The binding only marshals arguments: torch tensors become device pointers,
the current torch stream becomes the cudaStream_t, and every step of the
computation runs in libgp's CUDA kernels.  There is no CPU fallback: if
libgp.so is missing or CUDA is unavailable, calls raise.
"""
import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgp.so")

GP_OK, GP_ERR_NOT_PD, GP_ERR_INVALID, GP_ERR_CUDA, GP_ERR_TIMEOUT, GP_ERR_WORKSPACE = range(6)
KERNELS = {"exp": 0, "matern32": 1, "matern52": 2}
PRECISIONS = {"fp64": 0, "mixed_f16": 1, "emu_fp64": 2}

# Exported symbols, in the order include/gp.h declares them.
SYMBOLS = [
    "gp_abi_version",
    "gp_status_string",
    "gp_padded_order",
    "gp_workspace_bytes",
    "gp_chol_workspace_bytes",
    "gp_cov_fill",
    "gp_chol",
    "gp_backsolve",
    "gp_mult_chol",
    "gp_loglik",
    "gp_loglik_grad",
    "gp_loglik_product",
    "gp_batched_workspace_bytes",
    "gp_loglik_grad_batched",
    "gp_predict_workspace_bytes",
    "gp_predict",
    "gp_rng_normal",
    "gp_simulate_workspace_bytes",
    "gp_simulate",
    "gp_simulate_conditional_workspace_bytes",
    "gp_simulate_conditional",
    "gp_loglik_noalloc",
    "gp_syrk_workspace_bytes",
    "gp_syrk_lower",
    "gp_launch_count",
    "gp_prof_enable",
    "gp_prof_read",
    "gp_prof_dropped",
    "gp_batched_profile",
    "gp_batched_task_stats",
    "gp_batched_set_wait_limit",
    "gp_batched_test_unset_tile",
    "gp_batched_set_tile_policy",
    "gp_batched_tile_policy",
    "gp_batched_autotune",
    "gp_batched_plan_check",
]


class GpParams(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("sigma2", ctypes.c_double),
                ("rho", ctypes.c_double), ("tau2", ctypes.c_double)]


class GpProductParams(ctypes.Structure):
    _fields_ = [("sigma2", ctypes.c_double), ("rho_t", ctypes.c_double),
                ("rho_w", ctypes.c_double), ("tau2", ctypes.c_double)]


class GpError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib().gp_status_string(status).decode() if status >= 0 else "?"
        super().__init__(f"{where}: status {status} ({msg})")


class GpDeviceError(RuntimeError):
    """A device-side failure reported through d_info."""

    def __init__(self, info):
        self.info = int(info)
        if self.info > 0:
            msg = f"covariance not positive definite at column {self.info - 1}"
        elif self.info == -1:
            msg = "bounded device wait timed out"
        elif self.info == -2:
            msg = "non-finite input"
        else:
            msg = f"device failure {self.info}"
        super().__init__(msg)


_lock = threading.Lock()
_lib = None


def lib():
    """Load libgp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libgp.so not built ({LIB_PATH}); run "
                                   "`python -m paper_1305_4886_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            p, i64, ci, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
            PP = ctypes.POINTER(GpParams)
            L.gp_abi_version.restype = ci
            L.gp_status_string.argtypes = [ci]
            L.gp_status_string.restype = ctypes.c_char_p
            L.gp_padded_order.argtypes = [i64]
            L.gp_padded_order.restype = i64
            L.gp_workspace_bytes.argtypes = [i64, ci, ci]
            L.gp_workspace_bytes.restype = sz
            L.gp_chol_workspace_bytes.argtypes = [i64, ci]
            L.gp_chol_workspace_bytes.restype = sz
            L.gp_cov_fill.argtypes = [p, i64, PP, ci, p, i64, p]
            L.gp_chol.argtypes = [p, i64, i64, ci, p, sz, p, p]
            L.gp_backsolve.argtypes = [p, i64, i64, ci, p, p, p]
            L.gp_mult_chol.argtypes = [p, i64, i64, p, p, p]
            L.gp_loglik.argtypes = [p, p, p, i64, PP, ci, p, sz, p, p, p, p]
            L.gp_loglik_grad.argtypes = [p, p, p, i64, PP, ci, p, sz, p, p, p, p, p]
            L.gp_loglik_product.argtypes = [p, p, p, p, i64, ctypes.POINTER(GpProductParams), ci,
                                            p, sz, p, p, p, p, p]
            L.gp_loglik_product.restype = ci
            L.gp_batched_workspace_bytes.argtypes = [ci, p, ci]
            L.gp_batched_workspace_bytes.restype = sz
            L.gp_loglik_grad_batched.argtypes = [ci, p, p, p, p, p, ci, p, sz, p, p, p, p]
            L.gp_loglik_grad_batched.restype = ci
            L.gp_predict_workspace_bytes.argtypes = [i64, i64, ci]
            L.gp_predict_workspace_bytes.restype = sz
            L.gp_predict.argtypes = [p, i64, p, i64, PP, p, p, i64, ctypes.c_double, p, p, p, sz,
                                     p, p]
            L.gp_predict.restype = ci
            u64 = ctypes.c_uint64
            L.gp_rng_normal.argtypes = [i64, i64, u64, u64, u64, p, i64, p]
            L.gp_rng_normal.restype = ci
            L.gp_simulate_workspace_bytes.argtypes = [i64, i64]
            L.gp_simulate_workspace_bytes.restype = sz
            L.gp_simulate.argtypes = [p, i64, i64, i64, u64, u64, ctypes.c_double, p, i64, p, sz,
                                      p]
            L.gp_simulate.restype = ci
            L.gp_simulate_conditional_workspace_bytes.argtypes = [i64, i64, i64]
            L.gp_simulate_conditional_workspace_bytes.restype = sz
            L.gp_simulate_conditional.argtypes = [p, i64, p, i64, PP, p, p, i64, ctypes.c_double,
                                                  i64, u64, u64, p, i64, p, sz, p, p]
            L.gp_simulate_conditional.restype = ci
            L.gp_loglik_noalloc.argtypes = [p, p, p, i64, PP, p, p, p, p]
            L.gp_loglik_noalloc.restype = ci
            L.gp_syrk_workspace_bytes.argtypes = [i64, i64, ci]
            L.gp_syrk_workspace_bytes.restype = sz
            L.gp_syrk_lower.argtypes = [p, i64, p, i64, i64, i64, ci, p, sz, p, p]
            L.gp_launch_count.restype = i64
            L.gp_prof_enable.argtypes = [ci]
            L.gp_prof_read.argtypes = [ci, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
            L.gp_prof_dropped.restype = i64
            L.gp_batched_profile.argtypes = [ci]
            L.gp_batched_profile.restype = None
            L.gp_batched_task_stats.argtypes = [p, ctypes.POINTER(ctypes.c_uint64)]
            L.gp_batched_task_stats.restype = ci
            L.gp_batched_set_wait_limit.argtypes = [ctypes.c_double]
            L.gp_batched_set_wait_limit.restype = ci
            L.gp_batched_test_unset_tile.argtypes = [ci, i64, i64]
            L.gp_batched_test_unset_tile.restype = ci
            L.gp_batched_set_tile_policy.argtypes = [i64]
            L.gp_batched_set_tile_policy.restype = ci
            L.gp_batched_tile_policy.restype = i64
            L.gp_batched_autotune.argtypes = [ci, p, p, p, p, p, ci, p, sz, p, p, p, p,
                                              ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_int)]
            L.gp_batched_autotune.restype = ci
            L.gp_batched_plan_check.argtypes = [ci, p, ci, i64, ctypes.POINTER(ctypes.c_int64),
                                                ctypes.POINTER(ctypes.c_int64),
                                                ctypes.POINTER(ctypes.c_int64)]
            L.gp_batched_plan_check.restype = ci
            for name in ["gp_cov_fill", "gp_chol", "gp_backsolve", "gp_mult_chol", "gp_loglik",
                         "gp_loglik_grad", "gp_syrk_lower", "gp_prof_enable", "gp_prof_read"]:
                getattr(L, name).restype = ci
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libgp takes device tensors")
    if not t.is_contiguous():
        raise ValueError("libgp takes contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _f64(t):
    if t is not None and t.dtype != torch.float64:
        raise ValueError("libgp takes float64 tensors")
    return _ptr(t)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def params(kernel, sigma2, rho, tau2):
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    return GpParams(k, float(sigma2), float(rho), float(tau2))


def _prec(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _check(st, where):
    if st != GP_OK:
        raise GpError(st, where)


# ---------------------------------------------------------------------------
# the C ABI, one function per entry point
# ---------------------------------------------------------------------------
def gp_abi_version():
    return lib().gp_abi_version()


def gp_padded_order(n):
    return lib().gp_padded_order(int(n))


def gp_workspace_bytes(n, precision="fp64", want_grad=False):
    return lib().gp_workspace_bytes(int(n), _prec(precision), int(bool(want_grad)))


def gp_chol_workspace_bytes(n, precision="fp64"):
    return lib().gp_chol_workspace_bytes(int(n), _prec(precision))


def gp_cov_fill(x, prm, C, ldc=None, stream=None, precision="fp64"):
    n = x.shape[0]
    ldc = ldc if ldc is not None else C.shape[-1]
    _check(lib().gp_cov_fill(_f64(x), n, ctypes.byref(prm), _prec(precision), _f64(C), int(ldc),
                             _stream(stream)), "gp_cov_fill")


def gp_chol(C, n, ldc, precision, ws, info, stream=None):
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(lib().gp_chol(_f64(C), int(n), int(ldc), _prec(precision), _ptr(ws), wsb, _ptr(info),
                         _stream(stream)), "gp_chol")


def gp_backsolve(L, n, ldc, trans, b, out, stream=None):
    _check(lib().gp_backsolve(_f64(L), int(n), int(ldc), int(trans), _f64(b), _f64(out),
                              _stream(stream)), "gp_backsolve")


def gp_mult_chol(L, n, ldc, z, out, stream=None):
    _check(lib().gp_mult_chol(_f64(L), int(n), int(ldc), _f64(z), _f64(out), _stream(stream)),
           "gp_mult_chol")


def gp_loglik(x, y, mu, n, prm, precision, ws, out, alpha, info, stream=None):
    wsb = ws.numel() * ws.element_size()
    _check(lib().gp_loglik(_f64(x), _f64(y), _f64(mu), int(n), ctypes.byref(prm), _prec(precision),
                           _ptr(ws), wsb, _f64(out), _f64(alpha), _ptr(info), _stream(stream)),
           "gp_loglik")


class Batch:
    """Host-side argument arrays of gp_loglik_grad_batched, kept alive with
    the device tensors they point to."""

    def __init__(self, xs, ys, prms, mus=None):
        self.nprob = len(xs)
        self.xs, self.ys, self.mus = list(xs), list(ys), mus
        self.n = (ctypes.c_int64 * self.nprob)(*[int(x.shape[0]) for x in xs])
        P = ctypes.c_void_p * self.nprob
        self.px = P(*[_f64(x).value for x in xs])
        self.py = P(*[_f64(y).value for y in ys])
        self.pmu = P(*[(_f64(m).value if m is not None else None) for m in mus]) if mus else None
        self.prm = (GpParams * self.nprob)(*prms)


def gp_batched_workspace_bytes(ns, precision="mixed_f16"):
    arr = (ctypes.c_int64 * len(ns))(*[int(v) for v in ns])
    return lib().gp_batched_workspace_bytes(len(ns), ctypes.cast(arr, ctypes.c_void_p),
                                            _prec(precision))


def gp_loglik_grad_batched(batch, precision, ws, out, grad, info, stream=None):
    wsb = ws.numel() * ws.element_size()
    v = ctypes.c_void_p
    _check(lib().gp_loglik_grad_batched(
        batch.nprob, ctypes.cast(batch.n, v), ctypes.cast(batch.px, v), ctypes.cast(batch.py, v),
        ctypes.cast(batch.pmu, v) if batch.pmu is not None else None,
        ctypes.cast(batch.prm, v), _prec(precision), _ptr(ws), wsb, _f64(out), _f64(grad),
        _ptr(info), _stream(stream)), "gp_loglik_grad_batched")


def gp_batched_set_tile_policy(fp64_max_n):
    _check(lib().gp_batched_set_tile_policy(int(fp64_max_n)), "gp_batched_set_tile_policy")


def gp_batched_tile_policy():
    return int(lib().gp_batched_tile_policy())


AUTOTUNE_CANDIDATES = [0, 256, 384, 512, 768, 1024, 1536]


def gp_batched_autotune(batch, precision, ws, out, grad, info, stream=None):
    """Time the batch with each candidate tile threshold and keep the fastest
    as the device's policy (gp.h); returns (choice, {threshold: ms})."""
    wsb = ws.numel() * ws.element_size()
    v = ctypes.c_void_p
    choice = ctypes.c_int64(0)
    ms = (ctypes.c_double * 8)()
    ncand = ctypes.c_int(0)
    _check(lib().gp_batched_autotune(
        batch.nprob, ctypes.cast(batch.n, v), ctypes.cast(batch.px, v), ctypes.cast(batch.py, v),
        ctypes.cast(batch.pmu, v) if batch.pmu is not None else None,
        ctypes.cast(batch.prm, v), _prec(precision), _ptr(ws), wsb, _f64(out), _f64(grad),
        _ptr(info), _stream(stream), ctypes.byref(choice), ms, ctypes.byref(ncand)),
        "gp_batched_autotune")
    nmax = max(batch.n[i] for i in range(batch.nprob))
    cands = [t for t in AUTOTUNE_CANDIDATES if t == 0 or t < nmax][:ncand.value]
    return int(choice.value), {t: ms[q] for q, t in enumerate(cands)}


def gp_batched_plan_check(ns, precision="mixed_f16", fp64_max_n=0):
    """Host check of the batched launch's task order: (tasks, dependencies
    not earlier in the list, list slots not holding exactly one task)."""
    arr = (ctypes.c_int64 * len(ns))(*[int(v) for v in ns])
    nt, bo, bs = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().gp_batched_plan_check(len(ns), ctypes.cast(arr, ctypes.c_void_p), _prec(precision),
                                       int(fp64_max_n), ctypes.byref(nt), ctypes.byref(bo),
                                       ctypes.byref(bs)), "gp_batched_plan_check")
    return nt.value, bo.value, bs.value


def loglik_grad_batched(xs, ys, prms, precision="mixed_f16", mus=None, ws=None):
    """Evaluate a batch on the device; returns dict(out (nprob x 4), grad
    (nprob x 3), info (nprob,), ws, batch).  prms: list of GpParams."""
    batch = Batch(xs, ys, prms, mus)
    dev = xs[0].device
    if ws is None:
        nb = gp_batched_workspace_bytes([x.shape[0] for x in xs], precision)
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    out = torch.empty(batch.nprob, 4, dtype=torch.float64, device=dev)
    grad = torch.empty(batch.nprob, 3, dtype=torch.float64, device=dev)
    info = torch.zeros(batch.nprob, dtype=torch.int64, device=dev)
    gp_loglik_grad_batched(batch, precision, ws, out, grad, info)
    return dict(out=out, grad=grad, info=info, ws=ws, batch=batch)


BATCH_TASK_CLASSES = ["chol_offdiag", "solve", "inverse", "inverse_product_grad", "grad_sum",
                      "refine_residual", "refine_correction", "loglik", "chol_diag",
                      "refine_residual_skipped"]


def gp_batched_profile(on):
    lib().gp_batched_profile(1 if on else 0)


def gp_batched_set_wait_limit(seconds):
    _check(lib().gp_batched_set_wait_limit(float(seconds)), "gp_batched_set_wait_limit")


def gp_batched_test_unset_tile(problem, tile_row=0, tile_col=0):
    """Testing aid: waits for this Cholesky tile of this problem never succeed
    (problem = -1 turns it off); see include/gp.h."""
    _check(lib().gp_batched_test_unset_tile(int(problem), int(tile_row), int(tile_col)),
           "gp_batched_test_unset_tile")


def gp_batched_task_stats(ws):
    """Counters of the last batched call on ws (see gp.h): per task class
    cycles, waiting cycles and task counts, plus tensor-core steps."""
    buf = (ctypes.c_uint64 * 31)()
    _check(lib().gp_batched_task_stats(_ptr(ws), buf), "gp_batched_task_stats")
    v = list(buf)
    out = {name: {"cycles": v[q], "wait_cycles": v[10 + q], "tasks": v[20 + q]}
           for q, name in enumerate(BATCH_TASK_CLASSES)}
    out["steps"] = v[30]
    return out


def gp_predict_workspace_bytes(n, m, want_var=True):
    return lib().gp_predict_workspace_bytes(int(n), int(m), int(bool(want_var)))


def gp_predict(x, n, xnew, m, prm, alpha, L, ldl, mu_new, mean, var, ws, info, stream=None):
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(lib().gp_predict(_f64(x), int(n), _f64(xnew), int(m), ctypes.byref(prm), _f64(alpha),
                            _f64(L), int(ldl), float(mu_new), _f64(mean), _f64(var), _ptr(ws), wsb,
                            _ptr(info), _stream(stream)), "gp_predict")


def predict(x, y, xnew, kernel, sigma2, rho, tau2, mu=None, mu_new=None, precision="fp64",
            want_var=True, check=True):
    """Kriging prediction on the device: one gp_loglik (its factor and alpha),
    then gp_predict.  mu / mu_new: constant means (mu_new defaults to mu).
    Returns dict of device tensors {mean, var (or None), loglik}."""
    n, m = x.shape[0], xnew.shape[0]
    r = loglik(x, y, kernel, sigma2, rho, tau2, mu=mu, precision=precision, check=check)
    dev = x.device
    np_ = gp_padded_order(n)
    mean = torch.empty(m, dtype=torch.float64, device=dev)
    var = torch.empty(m, dtype=torch.float64, device=dev) if want_var else None
    ws = None
    if want_var:
        ws = torch.empty(max(1, gp_predict_workspace_bytes(n, m, True)), dtype=torch.uint8,
                         device=dev)
    info = torch.zeros(1, dtype=torch.int64, device=dev)
    L = r["ws"][: np_ * np_ * 8].view(torch.float64) if want_var else None
    mn = float(mu_new) if mu_new is not None else (0.0 if mu is None else float(mu))
    gp_predict(x, n, xnew, m, params(kernel, sigma2, rho, tau2), r["alpha"], L, np_, mn, mean,
               var, ws, info)
    if check:
        iv = int(info.item())
        if iv != 0:
            raise GpDeviceError(iv)
    return dict(mean=mean, var=var, loglik=r["out"][0])


def gp_rng_normal(n, r, seed, stream_id, first, out, ldo=None, stream=None):
    _check(lib().gp_rng_normal(int(n), int(r), int(seed), int(stream_id), int(first), _f64(out),
                               int(ldo if ldo is not None else n), _stream(stream)),
           "gp_rng_normal")


def gp_simulate_workspace_bytes(n, r):
    return lib().gp_simulate_workspace_bytes(int(n), int(r))


def gp_simulate(L, n, ldl, r, seed, first, mu, out, ldo, ws, stream=None):
    wsb = ws.numel() * ws.element_size()
    _check(lib().gp_simulate(_f64(L), int(n), int(ldl), int(r), int(seed), int(first), float(mu),
                             _f64(out), int(ldo), _ptr(ws), wsb, _stream(stream)), "gp_simulate")


def gp_simulate_conditional_workspace_bytes(n, m, r):
    return lib().gp_simulate_conditional_workspace_bytes(int(n), int(m), int(r))


def gp_simulate_conditional(x, n, xnew, m, prm, alpha, L, ldl, mu_new, r, seed, first, out, ldo,
                            ws, info, stream=None):
    wsb = ws.numel() * ws.element_size()
    _check(lib().gp_simulate_conditional(_f64(x), int(n), _f64(xnew), int(m), ctypes.byref(prm),
                                         _f64(alpha), _f64(L), int(ldl), float(mu_new), int(r),
                                         int(seed), int(first), _f64(out), int(ldo), _ptr(ws), wsb,
                                         _ptr(info), _stream(stream)), "gp_simulate_conditional")


def simulate(x, kernel, sigma2, rho, tau2, r, seed, first=0, mu=0.0, precision="fp64"):
    """Unconditional realisations of N(mu, C(theta)) at the locations x: the
    factor from one gp_loglik (its data vector is irrelevant), then
    gp_simulate.  Returns an (r, n) device tensor (row c = realisation c)."""
    n = x.shape[0]
    zero = torch.zeros(n, dtype=torch.float64, device=x.device)
    lk = loglik(x, zero, kernel, sigma2, rho, tau2, precision=precision)
    np_ = gp_padded_order(n)
    out = torch.empty(r, n, dtype=torch.float64, device=x.device)
    ws = torch.empty(gp_simulate_workspace_bytes(n, r), dtype=torch.uint8, device=x.device)
    gp_simulate(lk["ws"][: np_ * np_ * 8].view(torch.float64), n, np_, r, seed, first, mu, out, n,
                ws)
    return out


def simulate_conditional(x, y, xnew, kernel, sigma2, rho, tau2, r, seed, first=0, mu=None,
                         mu_new=None, precision="fp64", check=True):
    """Posterior realisations of the latent process at xnew given the data:
    one gp_loglik (factor and alpha), then gp_simulate_conditional.  Returns
    an (r, m) device tensor and the status tensor."""
    n, m = x.shape[0], xnew.shape[0]
    lk = loglik(x, y, kernel, sigma2, rho, tau2, mu=mu, precision=precision)
    np_ = gp_padded_order(n)
    out = torch.empty(r, m, dtype=torch.float64, device=x.device)
    ws = torch.empty(gp_simulate_conditional_workspace_bytes(n, m, r), dtype=torch.uint8,
                     device=x.device)
    info = torch.zeros(1, dtype=torch.int64, device=x.device)
    mn = float(mu_new) if mu_new is not None else (0.0 if mu is None else float(mu))
    gp_simulate_conditional(x, n, xnew, m, params(kernel, sigma2, rho, tau2), lk["alpha"],
                            lk["ws"][: np_ * np_ * 8].view(torch.float64), np_, mn, r, seed, first,
                            out, m, ws, info)
    if check:
        iv = int(info.item())
        if iv != 0:
            raise GpDeviceError(iv)
    return out, info


def gp_loglik_noalloc(x, y, mu, n, prm, out, alpha, info, stream=None):
    """FP64 log-likelihood for n <= 512 with the library's static scratch: for
    callers that cannot allocate device memory (see include/gp.h)."""
    _check(lib().gp_loglik_noalloc(_f64(x), _f64(y), _f64(mu), int(n), ctypes.byref(prm),
                                   _f64(out), _f64(alpha), _ptr(info), _stream(stream)),
           "gp_loglik_noalloc")


def gp_loglik_grad(x, y, mu, n, prm, precision, ws, out, alpha, grad, info, stream=None):
    wsb = ws.numel() * ws.element_size()
    _check(lib().gp_loglik_grad(_f64(x), _f64(y), _f64(mu), int(n), ctypes.byref(prm),
                                _prec(precision), _ptr(ws), wsb, _f64(out), _f64(alpha),
                                _f64(grad), _ptr(info), _stream(stream)), "gp_loglik_grad")


def gp_loglik_product(x, y, mu, v, n, prm, precision, ws, out, alpha, grad, info, stream=None):
    wsb = ws.numel() * ws.element_size()
    _check(lib().gp_loglik_product(_f64(x), _f64(y), _f64(mu), _f64(v), int(n), ctypes.byref(prm),
                                   _prec(precision), _ptr(ws), wsb, _f64(out), _f64(alpha),
                                   _f64(grad), _ptr(info), _stream(stream)), "gp_loglik_product")


def loglik_product(x, y, sigma2, rho_t, rho_w, tau2, v=None, mu=None, precision="fp64",
                   want_grad=True, ws=None, check=True):
    """The paper's example model on the device: dict of device tensors {out,
    grad (4: d/d log(sigma2, rho_t, rho_w, tau2)) or None, alpha, info, ws}."""
    n = x.shape[0]
    dev = x.device
    if ws is None:
        ws = workspace(n, precision, want_grad, dev)
    out = torch.empty(4, dtype=torch.float64, device=dev)
    grad = torch.empty(4, dtype=torch.float64, device=dev) if want_grad else None
    alpha = torch.empty(n, dtype=torch.float64, device=dev)
    info = torch.zeros(1, dtype=torch.int64, device=dev)
    mu_t = None
    if mu is not None:
        mu_t = mu if torch.is_tensor(mu) else torch.full((n,), float(mu), dtype=torch.float64,
                                                         device=dev)
    prm = GpProductParams(float(sigma2), float(rho_t), float(rho_w), float(tau2))
    gp_loglik_product(x, y, mu_t, v, n, prm, precision, ws, out, alpha, grad, info)
    if check:
        iv = int(info.item())
        if iv != 0:
            raise GpDeviceError(iv)
    return dict(out=out, grad=grad, alpha=alpha, info=info, ws=ws)


def gp_syrk_workspace_bytes(m, k, precision="mixed_f16"):
    return lib().gp_syrk_workspace_bytes(int(m), int(k), _prec(precision))


def gp_syrk_lower(C, ldc, P, ldp, m, k, precision, ws, info=None, stream=None):
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(lib().gp_syrk_lower(_f64(C), int(ldc), _f64(P), int(ldp), int(m), int(k),
                               _prec(precision), _ptr(ws), wsb, _ptr(info), _stream(stream)),
           "gp_syrk_lower")


PROF_CLASSES = {"contract": 0, "fill": 1, "residual": 2, "grad": 3, "diag_chol": 4,
                "diag_inv": 5, "solve": 6, "pack": 7, "fold": 8}
# roles of the "contract" class (gp_prof_read of "contract" sums them)
PROF_CONTRACT_ROLES = {"contract_chol": 9, "contract_trtri": 10, "contract_lauum": 11}


def gp_launch_count():
    return lib().gp_launch_count()


def gp_prof_enable(on):
    _check(lib().gp_prof_enable(int(bool(on))), "gp_prof_enable")


def gp_prof_read(cls):
    """(total ms, launches, flops, bytes) of one profiled kernel class.
    Raises if any profiled launch went unrecorded: partial sums are not
    returned."""
    c = ({**PROF_CLASSES, **PROF_CONTRACT_ROLES}[cls] if isinstance(cls, str) else int(cls))
    ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    cnt = ctypes.c_int64()
    st = lib().gp_prof_read(c, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(fl),
                            ctypes.byref(by))
    _check(st, f"gp_prof_read ({lib().gp_prof_dropped()} launches unrecorded)"
           if st == GP_ERR_WORKSPACE else "gp_prof_read")
    return ms.value, cnt.value, fl.value, by.value


def gp_prof_dropped():
    return int(lib().gp_prof_dropped())


# ---------------------------------------------------------------------------
# convenience wrappers that allocate with torch (device memory only)
# ---------------------------------------------------------------------------
def workspace(n, precision="fp64", want_grad=False, device="cuda"):
    nbytes = gp_workspace_bytes(n, precision, want_grad)
    if nbytes == 0:
        raise GpError(GP_ERR_INVALID, "gp_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def factor_view(ws, n):
    """The n_p x n_p matrix region at the start of a loglik workspace, as a
    column-major view: element (i, j) is view[j, i]."""
    np_ = gp_padded_order(n)
    return ws[: np_ * np_ * 8].view(torch.float64).view(np_, np_)


def loglik(x, y, kernel, sigma2, rho, tau2, mu=None, precision="fp64", ws=None,
           want_alpha=True, check=True):
    """Evaluate the log-likelihood on the device.  Returns a dict of device
    tensors {out: [loglik, logdet, q, resid], alpha, info} (synchronises and
    raises on a device failure when check=True)."""
    n = x.shape[0]
    dev = x.device
    if ws is None:
        ws = workspace(n, precision, False, dev)
    out = torch.empty(4, dtype=torch.float64, device=dev)
    alpha = torch.empty(n, dtype=torch.float64, device=dev) if want_alpha else None
    info = torch.zeros(1, dtype=torch.int64, device=dev)
    mu_t = None
    if mu is not None:
        mu_t = mu if torch.is_tensor(mu) else torch.full((n,), float(mu), dtype=torch.float64,
                                                         device=dev)
    gp_loglik(x, y, mu_t, n, params(kernel, sigma2, rho, tau2), precision, ws, out, alpha, info)
    if check:
        iv = int(info.item())
        if iv != 0:
            raise GpDeviceError(iv)
    return dict(out=out, alpha=alpha, info=info, ws=ws)


def loglik_grad(x, y, kernel, sigma2, rho, tau2, mu=None, precision="fp64", ws=None,
                want_alpha=True, check=True):
    """Log-likelihood and gradient on the device; returns dict of device tensors
    {out: [loglik, logdet, q, resid], grad: d/d(log s2, log rho, log tau2),
    alpha, info}."""
    n = x.shape[0]
    dev = x.device
    if ws is None:
        ws = workspace(n, precision, True, dev)
    out = torch.empty(4, dtype=torch.float64, device=dev)
    grad = torch.empty(3, dtype=torch.float64, device=dev)
    alpha = torch.empty(n, dtype=torch.float64, device=dev) if want_alpha else None
    info = torch.zeros(1, dtype=torch.int64, device=dev)
    mu_t = None
    if mu is not None:
        mu_t = mu if torch.is_tensor(mu) else torch.full((n,), float(mu), dtype=torch.float64,
                                                         device=dev)
    gp_loglik_grad(x, y, mu_t, n, params(kernel, sigma2, rho, tau2), precision, ws, out, alpha,
                   grad, info)
    if check:
        iv = int(info.item())
        if iv != 0:
            raise GpDeviceError(iv)
    return dict(out=out, grad=grad, alpha=alpha, info=info, ws=ws)
