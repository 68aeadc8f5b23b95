"""Shared helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np

TOL_D = 1e-5  # relative tolerance on d_eff, FP32 scan vs FP64 oracle


def deff_err(D_gpu, D_ref, N):
    """|D_gpu - D_ref| / max(|D_ref|, 1e-3 * L^2/2): relative error with a floor for
    random (strongly cancelling) sequences, whose |d_eff| is far below the scale
    L^2/2 of the terms being summed."""
    D_gpu = np.asarray(D_gpu)
    if D_gpu.ndim == 2 and D_gpu.shape[-1] == 2:
        D_gpu = D_gpu[:, 0] + 1j * D_gpu[:, 1]
    floor = 1e-3 * N * N / 2.0
    return np.abs(D_gpu - D_ref) / np.maximum(np.abs(D_ref), floor)


def fit_err(f_gpu, f_ref, N):
    floor = (1e-3 * N * N / 2.0) ** 2
    return np.abs(np.asarray(f_gpu, dtype=np.float64) - f_ref) / np.maximum(np.abs(f_ref), floor)


def lockstep_errors(trace_gpu, trace64, N):
    ok = ~np.isnan(trace_gpu)
    assert np.array_equal(ok, ~np.isnan(trace64)), "NaN pattern of the traces differs"
    return fit_err(trace_gpu[ok], trace64[ok], N)
