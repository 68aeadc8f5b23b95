"""The C-ABI library builds, loads and exports every entry point declared in
include/qpm.h; argument errors are reported as status codes before any device
work (CPU only: no computing call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(qpm_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def qlib():
    import paper_2511_01255_gb300 as q
    return q.lib()


def test_every_declared_symbol_is_exported(qlib):
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(qlib, n), n


def test_status_strings_and_version(qlib):
    assert qlib.qpm_status_string(0) == b"QPM_OK"
    assert qlib.qpm_status_string(3) == b"QPM_ERR_TIMEOUT"
    assert qlib.qpm_abi_version() >= 1


def test_argument_errors_without_device(qlib):
    import paper_2511_01255_gb300 as q
    # NULL problem
    assert qlib.qpm_eval(None, None, 0, 1, None, None, 0, None) == 1
    p = q.Problem(0, 1.0, 1.0)
    assert qlib.qpm_eval(ctypes.byref(p), ctypes.c_void_p(16), 1, 1, ctypes.c_void_p(16), None, 0, None) == 1
    assert b"N >= 1" in qlib.qpm_last_error()
    st = ctypes.c_void_p()
    p = q.Problem(16, 1.0, 2.0)
    bad = [q.Params(3, 10, 0.5, 0.9, 1, 0, 0), q.Params(8, 0, 0.5, 0.9, 1, 0, 0),
           q.Params(8, 10, 2.5, 0.9, 1, 0, 0), q.Params(8, 10, 0.5, 1.5, 1, 0, 0),
           q.Params(8, 10, 0.5, 0.9, 1, 3, 0), q.Params(8, 10, 0.5, 0.9, 1, 0, 0, 48),
           q.Params(8, 10, 0.5, 0.9, 1, 0, 0, 0, 3)]
    for prm in bad:
        assert qlib.qpm_create(ctypes.byref(p), ctypes.byref(prm), 1, ctypes.byref(st)) == 1
        assert not st.value
    assert qlib.qpm_create(ctypes.byref(p), ctypes.byref(bad[0]), 1, ctypes.byref(st)) == 1
    assert b"NP < 4" in qlib.qpm_last_error()
    assert qlib.qpm_step(None, None) == 1
    assert qlib.qpm_set_batch_cluster(None, 2) == 1
    assert qlib.qpm_destroy(None) == 0


def test_relaxed_saved_block_size_and_errors(qlib):
    import paper_2511_01255_gb300 as q
    # segments of L = min(256, 32 ceil(N / 1024)) domains; 4 + 8 floats per segment
    for N, L in ((1, 32), (5, 32), (1024, 32), (1025, 64), (1000, 32), (4096, 128), (100000, 256)):
        assert qlib.qpm_relaxed_saved_floats(N) == 4 + 8 * ((N + L - 1) // L), N
    assert qlib.qpm_relaxed_saved_floats(0) == 0
    p = q.Problem(64, 1.0, 2.0)
    f16 = ctypes.c_void_p(16)
    # NULL or misaligned saved block, NULL outputs: argument errors before any device work
    assert qlib.qpm_deff_relaxed_fwd(ctypes.byref(p), f16, 64, 2, f16, None, None, None) == 1
    assert b"saved" in qlib.qpm_last_error()
    assert qlib.qpm_deff_relaxed_fwd(ctypes.byref(p), f16, 64, 2, f16, None,
                                     ctypes.c_void_p(20), None) == 1
    assert b"aligned" in qlib.qpm_last_error()
    assert qlib.qpm_deff_relaxed_bwd(ctypes.byref(p), f16, 64, 2, f16, f16, None, None, 64,
                                     None) == 1
    assert qlib.qpm_deff_relaxed_bwd(ctypes.byref(p), f16, 64, 2, f16, f16, None, f16, 63,
                                     None) == 1
    assert qlib.qpm_abi_version() == 2


def test_workload_generators_are_seeded():
    from paper_2511_01255_gb300 import workloads as W
    import numpy as np
    a = W.random_genes(4, 33, seed=5)
    b = W.random_genes(4, 33, seed=5)
    assert np.array_equal(a, b) and a.dtype == np.float32
    words = W.pack_signs(a, 33)
    assert words.shape == (4, 2)
    for i in range(4):
        for j in range(33):
            assert ((int(words[i, j // 32]) >> (j % 32)) & 1) == int(a[i, j] < 0)
    inst = W.batched_instances(512)
    assert len(inst) == 512 and min(x["N"] for x in inst) >= 500 and max(x["N"] for x in inst) <= 8000


def test_binding_rejects_bad_tensors_before_the_library():
    """The binding checks device, dtype, layout and size of every tensor it hands to
    the library; a CPU tensor, a float64 gene array or a short output is a Python
    error, never a device pointer.  (No device is needed: the checks come first.)"""
    import torch

    import paper_2511_01255_gb300 as q
    X = torch.zeros((4, 16), dtype=torch.float32)
    D = torch.zeros((4, 2), dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA"):
        q.qpm_eval(16, 1.0, 2.0, X, D)
    with pytest.raises(ValueError, match="CUDA"):
        q.qpm_eval_noalloc(16, 1.0, 2.0, X.double(), D)
    with pytest.raises(ValueError, match="CUDA"):
        q.qpm_eval_packed(16, 1.0, 2.0, torch.zeros((4, 1), dtype=torch.int32), D)
    with pytest.raises(ValueError, match="CUDA"):
        q.qpm_deff_relaxed_fwd(16, 1.0, 2.0, X, D, None, torch.zeros((4, 8)))
    # host buffers of qpm_solve: dtype and size are checked before the call
    prm = q.Params(8, 10, 0.5, 0.9, 1, 0, 0)
    with pytest.raises(ValueError, match="best_genes_host"):
        q.qpm_solve(16, 1.0, 2.0, prm, q.RUN_PERSISTENT, torch.zeros(15), torch.zeros(2, dtype=torch.float64))
    with pytest.raises(ValueError, match="best_deff64_host"):
        q.qpm_solve(16, 1.0, 2.0, prm, q.RUN_PERSISTENT, torch.zeros(16), torch.zeros(2))

