"""The allocation-free fitness entry point, qpm_eval_noalloc.

qpm_eval_noalloc serves callers that cannot allocate device memory: host
callbacks and other code that may not call into the allocator, processes whose
device memory is all owned by an external allocator, and real-time paths that
cannot take the implicit device synchronisation of cudaMalloc/cudaFree.  Its
scratch is a fixed array inside the library.  Its results are checked against
qpm_eval (same tolerance as every fitness test) and against the FP64 oracle.

This file is collected last on purpose and must pass both on its own in a
fresh process and after the rest of the suite.
"""
import ctypes
import math

import numpy as np
import pytest

from helpers import TOL_D, deff_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01255_gb300 as q
    q.lib()
    return q


def _noalloc_abi(q, N, k1, k2, Xd, D, f, comp):
    """qpm_eval_noalloc through the C ABI directly (no binding logic in between)."""
    import torch
    p = q.Problem(N, k1, k2)
    st = q.lib().qpm_eval_noalloc(ctypes.byref(p), ctypes.c_void_p(Xd.data_ptr()), Xd.stride(0),
                                  Xd.shape[0], ctypes.c_void_p(D.data_ptr()),
                                  ctypes.c_void_p(f.data_ptr()), comp,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, q.lib().qpm_last_error()


def _both(q, N, k1, k2, X, comp):
    import torch
    NP = X.shape[0]
    Xd = torch.from_numpy(X).cuda()
    D0 = torch.empty((NP, 2), dtype=torch.float32, device="cuda")
    f0 = torch.empty(NP, dtype=torch.float32, device="cuda")
    D1 = torch.full((NP, 2), float("nan"), dtype=torch.float32, device="cuda")
    f1 = torch.full((NP,), float("nan"), dtype=torch.float32, device="cuda")
    q.qpm_eval(N, k1, k2, Xd, D0, f0, comp)
    _noalloc_abi(q, N, k1, k2, Xd, D1, f1, comp)
    torch.cuda.synchronize()
    return D0.cpu().numpy(), f0.cpu().numpy(), D1.cpu().numpy(), f1.cpu().numpy()


def _close(Da, Db, N):
    za = Da[:, 0] + 1j * Da[:, 1]
    zb = Db[:, 0] + 1j * Db[:, 1]
    floor = 1e-3 * N * N / 2.0
    return np.max(np.abs(za - zb) / np.maximum(np.abs(zb), floor))


CASES = [(4097, 2 * math.pi / 6.9, 2 * math.pi / 1.55, 37, 1, 4097),
         (1000, 2 * math.pi / 7.0, 2 * math.pi / 1.6, 256, 0, 1000),
         (4097, 2 * math.pi / 6.9, 2 * math.pi / 1.55, 37, 1, 4100)]


def test_noalloc_matches_qpm_eval_on_two_calls_in_a_row(q):
    from paper_2511_01255_gb300 import workloads as W
    # different problems back to back: a call must not depend on
    # what the one before left in the shared scratch
    # (rows of 4097 floats take the scalar-load sweep, rows of 4100 the cp.async ring)
    for N, k1, k2, NP, comp, ld in CASES:
        X = W.random_genes(NP, N, seed=N + NP, ld=ld)
        D0, f0, D1, f1 = _both(q, N, k1, k2, X, comp)
        assert _close(D1, D0, N) < TOL_D
        assert np.all(np.abs(f1 - f0) <= 2 * TOL_D * np.maximum(f0, (1e-3 * N * N / 2) ** 2))


def test_noalloc_matches_the_oracle(q, orc):
    """Two calls in a row (different problems) against the FP64 quadrature of the
    Sec. 2.1 integral, plus the closed form L^2/2 of an unpoled row at kappa = 0
    (strictly relative)."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    for N, k1, k2, NP, comp, ld in CASES[:2]:
        X = W.random_genes(NP, N, seed=N + 2 * NP, ld=ld)
        Xd = torch.from_numpy(X).cuda()
        D = torch.empty((NP, 2), dtype=torch.float32, device="cuda")
        f = torch.empty(NP, dtype=torch.float32, device="cuda")
        _noalloc_abi(q, N, k1, k2, Xd, D, f, comp)
        torch.cuda.synchronize()
        rows = [0, NP // 2, NP - 1]
        ref = orc.deff_genes(np.ascontiguousarray(X[rows, :N]), k1, k2)
        assert deff_err(D.cpu().numpy()[rows], ref, N).max() < TOL_D
    N = 20000
    ones = torch.ones((2, N), dtype=torch.float32, device="cuda")
    D = torch.empty((2, 2), dtype=torch.float32, device="cuda")
    f = torch.empty(2, dtype=torch.float32, device="cuda")
    _noalloc_abi(q, N, 0.0, 0.0, ones, D, f, 1)
    torch.cuda.synchronize()
    z = D.cpu().numpy()
    assert np.all(np.abs(z[:, 0] + 1j * z[:, 1] - N * N / 2) <= TOL_D * N * N / 2)


def test_noalloc_leaves_device_memory_unchanged(q):
    """After a first call (which looks up the array's address), further calls
    change neither the device's free memory nor torch's allocation count."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    N, NP = 30000, 64
    Xd = torch.from_numpy(W.random_genes(NP, N, seed=5)).cuda()
    D = torch.empty((NP, 2), dtype=torch.float32, device="cuda")
    f = torch.empty(NP, dtype=torch.float32, device="cuda")
    _noalloc_abi(q, N, 1.0, 2.0, Xd, D, f, 0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for k in range(3):
        _noalloc_abi(q, N - 7 * k, 1.0 + k, 2.0, Xd, D, f, k & 1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == n0


def test_noalloc_rejects_sizes_beyond_its_scratch(q):
    import torch
    N, NP = 600000, 4
    X = torch.zeros((NP, N), dtype=torch.float32, device="cuda")
    D = torch.empty((NP, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(q.QpmError) as e:
        q.qpm_eval_noalloc(N, 1.0, 2.0, X, D)
    assert e.value.status == 1 and "16 MiB" in str(e.value)
