"""Helpers for the GPU parity tests (device <-> numpy, tolerances)."""
import numpy as np
import torch


def require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test run without a CUDA device")


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def colmajor_to_numpy(buf, np_):
    """(np_ x np_) column-major device matrix -> numpy array indexed [i, j]."""
    return buf[: np_ * np_].reshape(np_, np_).cpu().numpy().T


def rel_err(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def rel_norm(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
