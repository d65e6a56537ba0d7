"""The C-ABI library: it builds, loads without a GPU, exports every symbol
include/gp.h declares, and its host-side queries and argument checks behave
as documented.  No compute call is made here (no GPU in this suite)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_symbols():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(gp_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libgp():
    from paper_1305_4886_gb300 import build, gp
    build.build()
    return gp


def test_header_declares_the_path(libgp):
    names = declared_symbols()
    # the path's entry points, the workspace query, and the next rows'
    # entry points (prediction, simulation, the paper's example covariance)
    for must in ["gp_cov_fill", "gp_chol", "gp_backsolve", "gp_loglik", "gp_loglik_grad",
                 "gp_loglik_grad_batched", "gp_workspace_bytes", "gp_mult_chol",
                 "gp_predict", "gp_simulate", "gp_simulate_conditional", "gp_rng_normal",
                 "gp_loglik_product"]:
        assert must in names, must


def test_exports_every_declared_symbol(libgp):
    L = ctypes.CDLL(libgp.LIB_PATH)
    missing = [s for s in sorted(declared_symbols()) if not hasattr(L, s)]
    assert not missing, missing
    assert sorted(declared_symbols()) == sorted(libgp.SYMBOLS)


def test_host_queries(libgp):
    L = libgp.lib()
    assert L.gp_abi_version() == 2
    assert libgp.gp_padded_order(1) == 128
    assert libgp.gp_padded_order(128) == 128
    assert libgp.gp_padded_order(129) == 256
    assert libgp.gp_padded_order(67275) == 67328
    assert libgp.gp_padded_order(0) == 0
    for p in ["fp64", "mixed_f16"]:
        b = libgp.gp_workspace_bytes(1024, p)
        assert b >= 1024 * 1024 * 8
        assert libgp.gp_workspace_bytes(0, p) == 0
    assert libgp.gp_workspace_bytes(100, 7) == 0
    for s in range(6):
        assert isinstance(L.gp_status_string(s), bytes)


def test_invalid_arguments_rejected_before_any_device_work(libgp):
    L = libgp.lib()
    P = libgp.params
    dummy = ctypes.c_void_p(16)
    bad = [P("exp", 0.0, 0.1, 0.1), P("exp", 1.0, -1.0, 0.1), P("exp", 1.0, 0.1, -0.1),
           P("exp", float("nan"), 0.1, 0.1), P(7, 1.0, 0.1, 0.1)]
    for prm in bad:
        st = L.gp_loglik(dummy, dummy, None, 10, ctypes.byref(prm), 0, dummy, 1 << 30, dummy,
                         None, dummy, None)
        assert st == libgp.GP_ERR_INVALID
    good = P("exp", 1.0, 0.1, 0.1)
    assert L.gp_loglik(dummy, dummy, None, 0, ctypes.byref(good), 0, dummy, 1 << 30, dummy,
                       None, dummy, None) == libgp.GP_ERR_INVALID
    # workspace too small
    assert L.gp_loglik(dummy, dummy, None, 1000, ctypes.byref(good), 0, dummy, 100, dummy,
                       None, dummy, None) == libgp.GP_ERR_WORKSPACE
    # leading dimension shorter than the padded order
    assert L.gp_cov_fill(dummy, 200, ctypes.byref(good), 0, dummy, 200, None) == libgp.GP_ERR_INVALID
    assert L.gp_cov_fill(dummy, 200, ctypes.byref(good), 7, dummy, 256, None) == libgp.GP_ERR_INVALID
    assert L.gp_backsolve(dummy, 10, 128, 2, dummy, dummy, None) == libgp.GP_ERR_INVALID


def test_wait_limit_and_unset_tile_arguments(libgp):
    """Host-side settings of the batched launch's bounded waits: the limit's
    accepted range and the testing aid's tile coordinates."""
    L = libgp.lib()
    assert L.gp_batched_set_wait_limit(0.0) == libgp.GP_ERR_INVALID
    assert L.gp_batched_set_wait_limit(1e-4) == libgp.GP_ERR_INVALID
    assert L.gp_batched_set_wait_limit(float("nan")) == libgp.GP_ERR_INVALID
    assert L.gp_batched_set_wait_limit(601.0) == libgp.GP_ERR_INVALID
    assert L.gp_batched_set_wait_limit(20.0) == libgp.GP_OK
    assert L.gp_batched_test_unset_tile(0, 1, 2) == libgp.GP_ERR_INVALID  # above the diagonal
    assert L.gp_batched_test_unset_tile(0, 3, -1) == libgp.GP_ERR_INVALID
    assert L.gp_batched_test_unset_tile(2, 3, 1) == libgp.GP_OK
    assert L.gp_batched_test_unset_tile(-1, 0, 0) == libgp.GP_OK


def test_predict_arguments(libgp):
    L = libgp.lib()
    prm = libgp.params("exp", 1.0, 0.1, 0.1)
    d = ctypes.c_void_p(16)
    call = lambda n, m, Lp, ldl, var, ws, wsb: L.gp_predict(  # noqa: E731
        d, n, d, m, ctypes.byref(prm), d, Lp, ldl, 0.0, d, var, ws, wsb, d, None)
    assert call(0, 5, None, 0, None, None, 0) == libgp.GP_ERR_INVALID
    assert call(10, 0, None, 0, None, None, 0) == libgp.GP_ERR_INVALID
    assert call(10, 5, None, 128, d, d, 1 << 30) == libgp.GP_ERR_INVALID  # variance needs L
    assert call(10, 5, d, 64, d, d, 1 << 30) == libgp.GP_ERR_INVALID       # ld below n_p
    assert call(10, 5, d, 128, d, d, 16) == libgp.GP_ERR_WORKSPACE
    assert libgp.gp_predict_workspace_bytes(10, 5, False) == 0
    assert libgp.gp_predict_workspace_bytes(10, 5, True) > 128 * 5 * 8


def test_simulation_arguments(libgp):
    L = libgp.lib()
    d = ctypes.c_void_p(16)
    prm = libgp.params("exp", 1.0, 0.1, 0.1)
    assert L.gp_rng_normal(0, 1, 1, 0, 0, d, 1, None) == libgp.GP_ERR_INVALID
    assert L.gp_rng_normal(10, 1, 1, 0, 0, d, 9, None) == libgp.GP_ERR_INVALID  # ldo < n
    assert L.gp_simulate(d, 10, 10, 2, 1, 0, 0.0, d, 10, d, 8, None) == libgp.GP_ERR_WORKSPACE
    assert L.gp_simulate(d, 10, 9, 2, 1, 0, 0.0, d, 10, d, 1 << 20, None) == libgp.GP_ERR_INVALID
    assert libgp.gp_simulate_workspace_bytes(10, 2) >= 160
    assert L.gp_simulate_conditional(d, 10, d, 3, ctypes.byref(prm), d, d, 64, 0.0, 2, 1, 0, d, 3,
                                     d, 1 << 30, d, None) == libgp.GP_ERR_INVALID  # ldl < n_p
    assert L.gp_simulate_conditional(d, 10, d, 3, ctypes.byref(prm), d, d, 128, 0.0, 2, 1, 0, d, 3,
                                     d, 64, d, None) == libgp.GP_ERR_WORKSPACE
