"""The allocation-free fitness entry point, qpm_eval_noalloc, against qpm_eval.

qpm_eval_noalloc serves callers that cannot allocate device memory (stream
capture, host callbacks, externally owned device memory); its scratch is a
fixed array inside the library.  This file is collected last on purpose and
must pass both on its own in a fresh process and after the rest of the suite.
"""
import ctypes
import math

import numpy as np
import pytest

from helpers import TOL_D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01255_gb300 as q
    q.lib()
    return q


def _both(q, N, k1, k2, X, comp):
    import torch
    NP = X.shape[0]
    Xd = torch.from_numpy(X).cuda()
    D0 = torch.empty((NP, 2), dtype=torch.float32, device="cuda")
    f0 = torch.empty(NP, dtype=torch.float32, device="cuda")
    D1 = torch.full((NP, 2), float("nan"), dtype=torch.float32, device="cuda")
    f1 = torch.full((NP,), float("nan"), dtype=torch.float32, device="cuda")
    q.qpm_eval(N, k1, k2, Xd, D0, f0, comp)
    # through the C ABI directly
    p = q.Problem(N, k1, k2)
    st = q.lib().qpm_eval_noalloc(ctypes.byref(p), ctypes.c_void_p(Xd.data_ptr()), Xd.stride(0),
                                  NP, ctypes.c_void_p(D1.data_ptr()), ctypes.c_void_p(f1.data_ptr()),
                                  comp, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, q.lib().qpm_last_error()
    torch.cuda.synchronize()
    return D0.cpu().numpy(), f0.cpu().numpy(), D1.cpu().numpy(), f1.cpu().numpy()


def _close(Da, Db, N):
    za = Da[:, 0] + 1j * Da[:, 1]
    zb = Db[:, 0] + 1j * Db[:, 1]
    floor = 1e-3 * N * N / 2.0
    return np.max(np.abs(za - zb) / np.maximum(np.abs(zb), floor))


def test_noalloc_matches_qpm_eval_on_two_calls_in_a_row(q):
    from paper_2511_01255_gb300 import workloads as W
    # different problems back to back: a call must not depend on
    # what the one before left in the shared scratch
    # (rows of 4097 floats take the scalar-load sweep, rows of 4100 the cp.async ring)
    cases = [(4097, 2 * math.pi / 6.9, 2 * math.pi / 1.55, 37, 1, 4097),
             (1000, 2 * math.pi / 7.0, 2 * math.pi / 1.6, 256, 0, 1000),
             (4097, 2 * math.pi / 6.9, 2 * math.pi / 1.55, 37, 1, 4100)]
    for N, k1, k2, NP, comp, ld in cases:
        X = W.random_genes(NP, N, seed=N + NP, ld=ld)
        D0, f0, D1, f1 = _both(q, N, k1, k2, X, comp)
        assert _close(D1, D0, N) < TOL_D
        assert np.all(np.abs(f1 - f0) <= 2 * TOL_D * np.maximum(f0, (1e-3 * N * N / 2) ** 2))


def test_noalloc_rejects_sizes_beyond_its_scratch(q):
    import torch
    N, NP = 600000, 4
    X = torch.zeros((NP, N), dtype=torch.float32, device="cuda")
    D = torch.empty((NP, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(q.QpmError) as e:
        q.qpm_eval_noalloc(N, 1.0, 2.0, X, D)
    assert e.value.status == 1 and "16 MiB" in str(e.value)
