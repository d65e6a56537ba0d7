"""ctypes wrapper of the plain-C FP64 oracle (``gp_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the product path must never import it.

Every function follows the definitions of Section 1 of Paciorek et al.
(arXiv:1305.4886): covariance C = C_g + C_y with a diagonal nugget, the
Cholesky factor L L^T = C, the forward solve L^{-1}(y - mu), the sum of squares
and log-determinant of Sec. 2.2.2, and the full Gaussian log-density.  The
gradient with respect to (log s2, log rho, log tau2) is the standard identity
1/2 a^T dC a - 1/2 tr(C^{-1} dC) (not in the paper).

Matrices are numpy float64 arrays of shape (n, n) in C order; locations are
(n, 2) float64 arrays.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_LIB = os.path.join(_HERE, "libgp_oracle.so")
_lock = threading.Lock()
_lib = None

KERNELS = {"exp": 0, "matern32": 1, "matern52": 2}


class OracleNotPD(RuntimeError):
    """Raised when the unpivoted Cholesky meets a pivot <= 0 (Sec. 5)."""

    def __init__(self, info):
        super().__init__(f"covariance not positive definite at column {info - 1}")
        self.info = info


def build(force=False):
    """Compile the oracle with gcc (-O2, OpenMP, IEEE: no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d = ctypes.c_double
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            ci = ctypes.c_int
            lib.orc_kernel.argtypes = [ci, d]
            lib.orc_kernel.restype = d
            lib.orc_kernel_dlogrho.argtypes = [ci, d]
            lib.orc_kernel_dlogrho.restype = d
            lib.orc_cov_fill.argtypes = [p, i64, ci, d, d, d, p]
            lib.orc_dcov_dlogrho.argtypes = [p, i64, ci, d, d, p]
            lib.orc_cov_rows.argtypes = [p, i64, p, i64, ci, d, d, d, p]
            lib.orc_cholesky.argtypes = [p, i64]
            lib.orc_cholesky.restype = i64
            lib.orc_forward.argtypes = [p, i64, p, p]
            lib.orc_backward.argtypes = [p, i64, p, p]
            lib.orc_lower_matvec.argtypes = [p, i64, p, p]
            lib.orc_lower_inverse.argtypes = [p, i64, p]
            lib.orc_inverse_from_chol.argtypes = [p, i64, p]
            lib.orc_logdet.argtypes = [p, i64]
            lib.orc_logdet.restype = d
            lib.orc_loglik.argtypes = [p, p, p, i64, ci, d, d, d, p, p, p, p]
            lib.orc_loglik.restype = ci
            lib.orc_loglik_grad.argtypes = [p, p, p, i64, ci, d, d, d, p, p, p, p]
            lib.orc_loglik_grad.restype = ci
            lib.orc_cross_cov.argtypes = [p, i64, p, i64, ci, d, d, p]
            lib.orc_predict.argtypes = [p, i64, p, i64, ci, d, d, p, p, d, p, p]
            u64 = ctypes.c_uint64
            lib.orc_philox4x64.argtypes = [p, p, p]
            lib.orc_normals.argtypes = [i64, i64, u64, u64, u64, p]
            lib.orc_simulate.argtypes = [p, i64, i64, u64, u64, d, p]
            lib.orc_simulate_conditional.argtypes = [p, i64, p, i64, ci, d, d, p, p, d, i64, u64,
                                                     u64, p, p]
            lib.orc_simulate_conditional.restype = ci
            lib.orc_bessel_k.argtypes = [d, d]
            lib.orc_bessel_k.restype = d
            lib.orc_matern2.argtypes = [d]
            lib.orc_matern2.restype = d
            lib.orc_matern2_dlogrho.argtypes = [d]
            lib.orc_matern2_dlogrho.restype = d
            lib.orc_prod_cov_fill.argtypes = [p, i64, p, d, d, d, d, p]
            lib.orc_prod_loglik_grad.argtypes = [p, p, p, p, i64, d, d, d, d, p, p, p, p]
            lib.orc_prod_loglik_grad.restype = ci
            lib.orc_num_threads.restype = ci
            lib.orc_set_threads.argtypes = [ci]
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _kind(kernel):
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def num_threads():
    return _load().orc_num_threads()


def set_threads(t):
    _load().orc_set_threads(int(t))


def kernel(kind, u):
    """Scalar correlation k(u), u = d/rho."""
    return _load().orc_kernel(_kind(kind), float(u))


def kernel_dlogrho(kind, u):
    """Scalar -u k'(u) (derivative of k(d/rho) in log rho)."""
    return _load().orc_kernel_dlogrho(_kind(kind), float(u))


def cov_fill(x, kernel, s2, rho, tau2):
    x = _f64(x)
    n = x.shape[0]
    C = np.empty((n, n))
    _load().orc_cov_fill(_ptr(x), n, _kind(kernel), s2, rho, tau2, _ptr(C))
    return C


def cov_rows(x, rows, kernel, s2, rho, tau2):
    """Rows `rows` of C(theta), shape (len(rows), n)."""
    x = _f64(x)
    n = x.shape[0]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((rows.size, n))
    _load().orc_cov_rows(_ptr(x), n, _ptr(rows), rows.size, _kind(kernel), s2, rho, tau2,
                         _ptr(out))
    return out


def dcov_dlogrho(x, kernel, s2, rho):
    x = _f64(x)
    n = x.shape[0]
    D = np.empty((n, n))
    _load().orc_dcov_dlogrho(_ptr(x), n, _kind(kernel), s2, rho, _ptr(D))
    return D


def cholesky(C):
    """Lower factor L (upper part zero).  Raises OracleNotPD."""
    A = _f64(C).copy()
    info = _load().orc_cholesky(_ptr(A), A.shape[0])
    if info:
        raise OracleNotPD(int(info))
    return A


def forward(L, b):
    L = _f64(L)
    b = _f64(b)
    v = np.empty_like(b)
    _load().orc_forward(_ptr(L), L.shape[0], _ptr(b), _ptr(v))
    return v


def backward(L, v):
    L = _f64(L)
    v = _f64(v)
    a = np.empty_like(v)
    _load().orc_backward(_ptr(L), L.shape[0], _ptr(v), _ptr(a))
    return a


def lower_matvec(L, z):
    L = _f64(L)
    z = _f64(z)
    y = np.empty_like(z)
    _load().orc_lower_matvec(_ptr(L), L.shape[0], _ptr(z), _ptr(y))
    return y


def lower_inverse(L):
    L = _f64(L)
    X = np.empty_like(L)
    _load().orc_lower_inverse(_ptr(L), L.shape[0], _ptr(X))
    return X


def inverse_from_chol(L):
    L = _f64(L)
    W = np.empty_like(L)
    _load().orc_inverse_from_chol(_ptr(L), L.shape[0], _ptr(W))
    return W


def logdet(L):
    L = _f64(L)
    return _load().orc_logdet(_ptr(L), L.shape[0])


def _mu_arg(mu, n):
    if mu is None:
        return None, None
    m = np.asarray(mu, dtype=np.float64)
    if m.ndim == 0:
        m = np.full(n, float(m))
    m = _f64(m)
    return m, _ptr(m)


def loglik(x, y, kernel, s2, rho, tau2, mu=None, want_L=False):
    """Returns dict(loglik, logdet, quad, alpha[, L]).  Raises OracleNotPD."""
    x = _f64(x)
    y = _f64(y)
    n = x.shape[0]
    m, mp = _mu_arg(mu, n)
    out = np.empty(3)
    alpha = np.empty(n)
    L = np.empty((n, n)) if want_L else None
    info = ctypes.c_int64(0)
    st = _load().orc_loglik(_ptr(x), _ptr(y), mp, n, _kind(kernel), s2, rho, tau2,
                            _ptr(out), _ptr(alpha), _ptr(L) if want_L else None,
                            ctypes.byref(info))
    if st == 2:
        raise ValueError("invalid oracle arguments")
    if st == 1:
        raise OracleNotPD(int(info.value))
    res = dict(loglik=out[0], logdet=out[1], quad=out[2], alpha=alpha)
    if want_L:
        res["L"] = L
    return res


def loglik_grad(x, y, kernel, s2, rho, tau2, mu=None):
    """Returns dict(loglik, logdet, quad, alpha, grad) with grad w.r.t.
    (log s2, log rho, log tau2).  Raises OracleNotPD."""
    x = _f64(x)
    y = _f64(y)
    n = x.shape[0]
    m, mp = _mu_arg(mu, n)
    out = np.empty(3)
    alpha = np.empty(n)
    grad = np.empty(3)
    info = ctypes.c_int64(0)
    st = _load().orc_loglik_grad(_ptr(x), _ptr(y), mp, n, _kind(kernel), s2, rho, tau2,
                                 _ptr(out), _ptr(alpha), _ptr(grad), ctypes.byref(info))
    if st == 2:
        raise ValueError("invalid oracle arguments")
    if st == 1:
        raise OracleNotPD(int(info.value))
    return dict(loglik=out[0], logdet=out[1], quad=out[2], alpha=alpha, grad=grad)


def cross_cov(x, xs, kernel, s2, rho):
    """Cross covariance K (n x m): K[i, j] = s2 k(|x_i - xs_j| / rho)."""
    x = _f64(x)
    xs = _f64(xs)
    K = np.empty((x.shape[0], xs.shape[0]))
    _load().orc_cross_cov(_ptr(x), x.shape[0], _ptr(xs), xs.shape[0], _kind(kernel), s2, rho,
                          _ptr(K))
    return K


def predict(x, xs, kernel, s2, rho, L, alpha, mu_new=0.0, want_var=True):
    """Kriging mean (and variance) at new locations xs from the training
    factor L and alpha = C^{-1}(y - mu): dict(mean, var)."""
    x, xs, L, alpha = _f64(x), _f64(xs), _f64(L), _f64(alpha)
    m = xs.shape[0]
    mean = np.empty(m)
    var = np.empty(m) if want_var else None
    _load().orc_predict(_ptr(x), x.shape[0], _ptr(xs), m, _kind(kernel), s2, rho, _ptr(L),
                        _ptr(alpha), float(mu_new), _ptr(mean), _ptr(var) if want_var else None)
    return dict(mean=mean, var=var)


def predict_from_data(x, y, xs, kernel, s2, rho, tau2, mu=None, mu_new=0.0, want_var=True):
    """Factor the training covariance, solve for alpha, then predict."""
    r = loglik(x, y, kernel, s2, rho, tau2, mu=mu, want_L=True)
    return predict(x, xs, kernel, s2, rho, r["L"], r["alpha"], mu_new, want_var)


def philox4x64(counter, key):
    """Philox4x64-10 of one 4-word counter and 2-word key: 4 uint64 words."""
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    _load().orc_philox4x64(_ptr(c), _ptr(k), _ptr(out))
    return out


def normals(n, r, seed, stream=0, first=0):
    """Standard normals of the simulation, shape (r, n): row c is realisation
    first + c of the given stream."""
    out = np.empty((r, n))
    _load().orc_normals(int(n), int(r), int(seed), int(stream), int(first), _ptr(out))
    return out


def simulate(L, r, seed, first=0, mu=0.0):
    """Unconditional realisations mu + L e_c, shape (r, n)."""
    L = _f64(L)
    n = L.shape[0]
    out = np.empty((r, n))
    _load().orc_simulate(_ptr(L), n, int(r), int(seed), int(first), float(mu), _ptr(out))
    return out


def simulate_conditional(x, xs, kernel, s2, rho, L, alpha, r, seed, first=0, mu_new=0.0):
    """Posterior realisations of the latent process at xs, shape (r, m).
    Raises OracleNotPD when the posterior covariance is not numerically
    positive definite."""
    x, xs, L, alpha = _f64(x), _f64(xs), _f64(L), _f64(alpha)
    m = xs.shape[0]
    out = np.empty((r, m))
    info = ctypes.c_int64(0)
    st = _load().orc_simulate_conditional(_ptr(x), x.shape[0], _ptr(xs), m, _kind(kernel), s2, rho,
                                          _ptr(L), _ptr(alpha), float(mu_new), int(r), int(seed),
                                          int(first), _ptr(out), ctypes.byref(info))
    if st == 1:
        raise OracleNotPD(int(info.value))
    return out


def bessel_k(nu, x):
    """K_nu(x) by the trapezoidal rule on its integral representation."""
    return _load().orc_bessel_k(float(nu), float(x))


def matern2(u):
    """Matern nu = 2 correlation k(u) = a^2 K_2(a) / 2, a = 2u."""
    return _load().orc_matern2(float(u))


def matern2_dlogrho(u):
    """-u k'(u) = a^3 K_1(a) / 2 for the Matern nu = 2 correlation."""
    return _load().orc_matern2_dlogrho(float(u))


def prod_cov_fill(x, s2, rho_t, rho_w, tau2, v=None):
    """C of the paper's example model (Sec. 4.2): product Matern nu = 2 in
    (phase, log wavelength), tau2 between equal phases, v_i on the diagonal."""
    x = _f64(x)
    n = x.shape[0]
    vv = _f64(v) if v is not None else None
    C = np.empty((n, n))
    _load().orc_prod_cov_fill(_ptr(x), n, _ptr(vv) if vv is not None else None, s2, rho_t, rho_w,
                              tau2, _ptr(C))
    return C


def prod_loglik_grad(x, y, s2, rho_t, rho_w, tau2, v=None, mu=None, want_grad=True):
    """dict(loglik, logdet, quad, alpha[, grad]) of the product model; grad
    with respect to (log s2, log rho_t, log rho_w, log tau2)."""
    x = _f64(x)
    y = _f64(y)
    n = x.shape[0]
    m, mp = _mu_arg(mu, n)
    vv = _f64(v) if v is not None else None
    out = np.empty(3)
    alpha = np.empty(n)
    grad = np.empty(4) if want_grad else None
    info = ctypes.c_int64(0)
    st = _load().orc_prod_loglik_grad(_ptr(x), _ptr(y), mp, _ptr(vv) if vv is not None else None,
                                      n, s2, rho_t, rho_w, tau2, _ptr(out), _ptr(alpha),
                                      _ptr(grad) if want_grad else None, ctypes.byref(info))
    if st == 2:
        raise ValueError("invalid oracle arguments")
    if st == 1:
        raise OracleNotPD(int(info.value))
    res = dict(loglik=out[0], logdet=out[1], quad=out[2], alpha=alpha)
    if want_grad:
        res["grad"] = grad
    return res
