"""GPU parity of qpm_eval / qpm_eval_packed (Sec. 2.1 d_eff) against the FP64 oracle."""
import math

import numpy as np
import pytest

from helpers import TOL_D, deff_err

pytestmark = pytest.mark.gpu

K1, K2 = 2 * math.pi / 6.9, 2 * math.pi / 1.55


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01255_gb300 as q
    q.lib()
    return q


def run_eval(q, X, N, k1, k2, comp=0, packed=False):
    import torch
    from paper_2511_01255_gb300 import workloads as W
    NP = X.shape[0]
    D = torch.empty((NP, 2), dtype=torch.float32, device="cuda")
    f = torch.empty(NP, dtype=torch.float32, device="cuda")
    if packed:
        words = torch.from_numpy(W.pack_signs(X, N).view(np.int32)).cuda()
        q.qpm_eval_packed(N, k1, k2, words, D, f, comp)
    else:
        q.qpm_eval(N, k1, k2, torch.from_numpy(X).cuda(), D, f, comp)
    torch.cuda.synchronize()
    return D.cpu().numpy(), f.cpu().numpy()


@pytest.mark.parametrize("N", [1, 3, 4, 31, 32, 33, 100, 1000, 4097])
@pytest.mark.parametrize("NP", [1, 5, 33])
@pytest.mark.parametrize("comp", [0, 1])
def test_eval_random_genes(q, orc, N, NP, comp):
    from paper_2511_01255_gb300 import workloads as W
    X = W.random_genes(NP, N, seed=N * 7 + NP)
    D, f = run_eval(q, X, N, K1, K2, comp)
    ref = orc.deff_genes(X, K1, K2)
    assert deff_err(D, ref, N).max() < TOL_D
    assert np.allclose(f, D[:, 0] ** 2 + D[:, 1] ** 2, rtol=1e-6, atol=0)
    # packed signs: the sign-block sweep (4 domains per table lookup)
    Dp, fp = run_eval(q, X, N, K1, K2, comp, packed=True)
    assert deff_err(Dp, ref, N).max() < TOL_D
    assert np.allclose(fp, Dp[:, 0] ** 2 + Dp[:, 1] ** 2, rtol=1e-6, atol=0)


@pytest.mark.parametrize("N", [1, 3, 33, 130, 1001, 4097])
@pytest.mark.parametrize("comp", [0, 1])
def test_eval_aligned_rows_with_ragged_tail(q, orc, N, comp):
    """16-byte aligned rows (leading dimension a multiple of 4) whose length is not:
    the last asynchronous copy of every row is partial and zero-fills the rest; the
    padding columns hold NaN and must never be read."""
    from paper_2511_01255_gb300 import workloads as W
    ld = (N + 3) // 4 * 4 + 4
    X = W.random_genes(37, N, seed=N + 5, ld=ld)
    X[:, N:] = np.nan
    D, f = run_eval(q, X, N, K1, K2, comp)
    ref = orc.deff_genes(np.ascontiguousarray(X[:, :N]), K1, K2)
    assert deff_err(D, ref, N).max() < TOL_D
    assert np.all(np.isfinite(f))


def test_eval_aligned_long_ragged_rows_sampled(q, orc):
    """N = 99997 in 16-byte aligned rows of 100000 floats (NaN padding), 64 rows: many
    segments and 128-domain steps, a ragged last sub-step; 3 rows re-done by the oracle."""
    from paper_2511_01255_gb300 import workloads as W
    N, ld = 99997, 100000
    X = W.random_genes(64, N, seed=17, ld=ld)
    X[:, N:] = np.nan
    D, _ = run_eval(q, X, N, K1, K2, 1)
    rows = [0, 31, 63]
    ref = orc.deff_genes(np.ascontiguousarray(X[rows, :N]), K1, K2)
    assert deff_err(D[rows], ref, N).max() < TOL_D


@pytest.mark.parametrize("N", [1, 5, 30, 33, 1001])
def test_packed_ignores_bits_past_the_row(q, N):
    """Sign bits of the last word beyond domain N - 1 do not change d_eff: the
    sign-block entries of a block that straddles N carry zero phasors there."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    X = W.random_genes(6, N, seed=N + 1)
    words = W.pack_signs(X, N)
    dirty = words.copy()
    if N % 32:
        dirty[:, -1] |= np.uint32((0xFFFFFFFF << (N % 32)) & 0xFFFFFFFF)
    res = []
    for w in (words, dirty):
        D = torch.empty((6, 2), dtype=torch.float32, device="cuda")
        q.qpm_eval_packed(N, K1, K2, torch.from_numpy(w.view(np.int32)).cuda(), D, None, 0)
        torch.cuda.synchronize()
        res.append(D.cpu().numpy())
    assert np.array_equal(res[0], res[1])


def test_eval_strided_rows_and_random_kappa(q, orc):
    import torch
    from paper_2511_01255_gb300 import workloads as W
    rng = np.random.default_rng(3)
    for N, ld in ((77, 81), (500, 503), (1024, 1030)):
        X = W.random_genes(9, N, seed=N, ld=ld)
        k1, k2 = rng.uniform(-4, 4, 2)
        D = torch.empty((9, 2), dtype=torch.float32, device="cuda")
        q.qpm_eval(N, k1, k2, torch.from_numpy(X).cuda(), D, None, 0)
        torch.cuda.synchronize()
        ref = orc.deff_genes(np.ascontiguousarray(X[:, :N]), k1, k2)
        assert deff_err(D.cpu().numpy(), ref, N).max() < TOL_D


@pytest.mark.parametrize("N", [1, 16, 1000, 4096])
def test_closed_forms_on_gpu(q, N):
    ones = np.ones((1, N), dtype=np.float32)
    D, _ = run_eval(q, ones, N, 0.0, 0.0)
    assert abs(complex(*D[0]) - N * N / 2) <= 1e-6 * N * N / 2
    alt = np.where(np.arange(N) % 2 == 0, 1.0, -1.0).astype(np.float32)[None]
    D, _ = run_eval(q, alt, N, math.pi, math.pi)
    exact = -(2 / math.pi) ** 2 * N * N / 2
    assert abs(complex(*D[0]) - exact) <= TOL_D * abs(exact)


def test_sign_flip_exact_on_gpu(q):
    from paper_2511_01255_gb300 import workloads as W
    X = W.random_genes(8, 3001, seed=9)
    X[X == 0] = 0.5
    D1, _ = run_eval(q, X, 3001, K1, K2)
    D2, _ = run_eval(q, -X, 3001, K1, K2)
    assert np.array_equal(D1, D2)


@pytest.mark.parametrize("comp", [0, 1])
def test_eval_full_size_sampled(q, orc, comp):
    """N = 1e5 domains, 1024 sequences: every row on the GPU, 6 rows re-done by the oracle."""
    from paper_2511_01255_gb300 import workloads as W
    N, NP = 100000, 1024
    X = W.random_genes(NP, N, seed=11)
    X[5] = 1.0  # one perfectly unpoled row and one alternating row among the samples
    X[6] = W.alternating(N)
    D, f = run_eval(q, X, N, K1, K2, comp)
    rows = [0, 5, 6, 511, 777, 1023]
    ref = orc.deff_genes(X[rows], K1, K2)
    err = deff_err(D[rows], ref, N)
    assert err.max() < TOL_D, err
    # the same rows as packed sign words (the packed sweep's own segmenting)
    Dp, _ = run_eval(q, X, N, K1, K2, comp, packed=True)
    errp = deff_err(Dp[rows], ref, N)
    assert errp.max() < TOL_D, errp


@pytest.mark.parametrize("N", [1, 7, 1000, 4097, 100000])
def test_shg_field_against_oracle(q, orc, N):
    import torch
    from paper_2511_01255_gb300 import workloads as W
    NP = 19 if N < 100000 else 6
    X = W.random_genes(NP, N, seed=N + 3)
    X[0] = W.alternating(N)
    E = torch.empty((NP, 2), device="cuda")
    f = torch.empty(NP, device="cuda")
    k = 2 * math.pi / 6.9
    q.qpm_eval_shg(N, k, torch.from_numpy(X).cuda(), E, f)
    torch.cuda.synchronize()
    E = E.cpu().numpy()
    ref = orc.shg_genes(X, k)
    z = E[:, 0] + 1j * E[:, 1]
    # random rows cancel: floor at 1e-3 of the all-up magnitude scale N
    err = np.abs(z - ref) / np.maximum(np.abs(ref), 1e-3 * N)
    assert err.max() < TOL_D
    # first-order QPM at kappa = pi: |E| = 2N/pi
    E2 = torch.empty((1, 2), device="cuda")
    q.qpm_eval_shg(N, math.pi, torch.from_numpy(W.alternating(N)[None]).cuda(), E2)
    torch.cuda.synchronize()
    assert abs(np.hypot(*E2.cpu().numpy()[0]) - 2 * N / math.pi) <= TOL_D * 2 * N / math.pi


@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_multi_wavelength_objective_against_oracle(q, orc, K):
    import torch
    from paper_2511_01255_gb300 import workloads as W
    N, NP = 3001, 41
    X = W.random_genes(NP, N, seed=K)
    kap = [(2 * math.pi / (6.5 + 0.4 * k), 2 * math.pi / (1.4 + 0.1 * k)) for k in range(K)]
    G0, beta = 2.0e4, 0.7
    obj = torch.empty(NP, device="cuda")
    D = torch.empty((NP, K, 2), device="cuda")
    q.qpm_eval_multi(N, kap, torch.from_numpy(X).cuda(), G0, beta, obj, D)
    torch.cuda.synchronize()
    Dr, objr = orc.multi_objective(X, kap, G0, beta)
    Dg = D.cpu().numpy()
    for k in range(K):
        assert deff_err(Dg[:, k], Dr[:, k], N).max() < TOL_D
    # each |G0 - G_k| term carries the d_eff error; FP32 rounding of G0-sized sums
    scale = K * G0 + beta * np.abs(Dr).max()
    assert np.max(np.abs(obj.cpu().numpy() - objr)) <= TOL_D * scale
    # one problem through the fused path equals qpm_eval
    if K == 1:
        D1 = torch.empty((NP, 2), device="cuda")
        q.qpm_eval(N, kap[0][0], kap[0][1], torch.from_numpy(X).cuda(), D1)
        torch.cuda.synchronize()
        assert np.array_equal(D1.cpu().numpy(), Dg[:, 0])


@pytest.mark.parametrize("ld_extra", [0, 1])
def test_multi_wavelength_k1_equals_qpm_eval_on_long_rows(q, ld_extra):
    """K = 1 takes qpm_eval's segments and order for long rows too: aligned rows (the
    cp.async ring form, fewer and longer segments) and unaligned rows (ld = N + 1)."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    N, NP = 99996, 70
    X = torch.from_numpy(W.random_genes(NP, N, seed=23, ld=N + ld_extra)).cuda()
    kap = [(2 * math.pi / 6.9, 2 * math.pi / 1.55)]
    obj = torch.empty(NP, device="cuda")
    D = torch.empty((NP, 1, 2), device="cuda")
    q.qpm_eval_multi(N, kap, X, 2.0e4, 0.7, obj, D)
    D1 = torch.empty((NP, 2), device="cuda")
    q.qpm_eval(N, kap[0][0], kap[0][1], X, D1)
    torch.cuda.synchronize()
    assert np.array_equal(D1.cpu().numpy(), D.cpu().numpy()[:, 0])


def test_issue_peak_microbenchmark(q):
    """The measured issue rates are positive and the FFMA rate is within reach of
    the derived peak (SMs x 128 lanes x clock; clocks may run below the maximum)."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    derived = nsm * 128 * 2.07e9
    f = q.qpm_measure_issue_peak(0)
    assert 0.3 * derived < f < 1.1 * derived
    assert q.qpm_measure_issue_peak(1) > 0 and q.qpm_measure_issue_peak(2) > 0
    # whole Philox calls: at most one call per 40 issue slots of the FFMA rate
    assert 0 < q.qpm_measure_issue_peak(3) < f / 40 * 1.1
    with pytest.raises(q.QpmError):
        q.qpm_measure_issue_peak(4)


def test_latency_microbenchmark(q):
    """The barrier and L2 latencies behind the latency floor of the persistent form:
    positive, of the expected order, and the barrier costs more than a load."""
    bar = q.qpm_measure_latency(0, 256)
    l2 = q.qpm_measure_latency(1)
    assert 50.0 < l2 < 5000.0
    assert l2 < bar < 50000.0
    assert q.qpm_measure_latency(0, 1) > 0.0
    # the other ways to synchronise the grid: a relaxed counter is no slower than the
    # ordered one would allow by more than the noise, a lone fence is cheaper than a
    # barrier, and every form finishes (bounded polls) with a positive time
    relaxed = q.qpm_measure_latency(2, 256)
    fence = q.qpm_measure_latency(3, 256)
    tagged = q.qpm_measure_latency(4, 256)
    assert 0.0 < fence < bar and 0.0 < relaxed < 1.5 * bar and tagged > 0.0
    assert q.qpm_measure_latency(4, 1) > 0.0
    with pytest.raises(q.QpmError):
        q.qpm_measure_latency(5)
    with pytest.raises(q.QpmError):
        q.qpm_measure_latency(-1)
    with pytest.raises(q.QpmError):
        q.qpm_measure_latency(0, 10 ** 6)
    with pytest.raises(q.QpmError):
        q.qpm_measure_latency(4, 10 ** 6)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_arithmetic_shortcuts_exact_on_every_pattern(q, kind):
    """The kernels' shortcuts give the oracle's plain operation for all 2^32
    inputs: 0 the GWO mean's division by 3 (Markstein's residual correction)
    against the IEEE quotient; 1 the GWO's 2 r1 - 1 and 2 r2 built in the
    significand against int-to-float conversions; 2 the integer crossover test
    against U <= CR in FP32."""
    bad, first = q.qpm_selfcheck(kind)
    assert bad == 0, f"{bad} mismatches, first pattern 0x{first:08x}"
    assert first == 0xFFFFFFFF


def test_selfcheck_rejects_unknown_kind(q):
    with pytest.raises(q.QpmError):
        q.qpm_selfcheck(3)


def test_multi_wavelength_with_a_full_table_cache(q):
    """63 problems fill the table cache (64 per device); qpm_eval_multi with two new
    problems must make room before its first lookup, never between them, so neither
    of its tables is freed under it (a freed table is reallocated for the next problem
    and the first problem would be scanned with the wrong phasors).  Its d_eff agree
    with qpm_eval's."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    q.qpm_release_caches()
    N, NP = 1001, 40
    X = torch.from_numpy(W.random_genes(NP, N, seed=77)).cuda()
    D = torch.empty((NP, 2), device="cuda")
    for k in range(63):
        q.qpm_eval(N, 0.5 + 0.01 * k, 2.0, X, D)
    kap = [(0.123, 3.21), (0.456, 2.34)]
    obj = torch.empty(NP, device="cuda")
    Dm = torch.empty((NP, 2, 2), device="cuda")
    q.qpm_eval_multi(N, kap, X, 1.0e4, 0.5, obj, Dm)
    torch.cuda.synchronize()
    for k, (k1, k2) in enumerate(kap):
        q.qpm_eval(N, k1, k2, X, D)
        torch.cuda.synchronize()
        a, b = D.cpu().numpy(), Dm.cpu().numpy()[:, k]
        assert deff_err(b, a[:, 0] + 1j * a[:, 1], N).max() < TOL_D
    q.qpm_release_caches()


def test_table_cache_under_concurrent_host_threads(q):
    """Four host threads, each on its own stream, evaluate 40 distinct problems each (160
    in all, more than the 64 the cache holds, so tables are evicted while other threads
    are between their lookups and launches).  The cache's lock is held from a call's
    first lookup to its last launch, so every result equals the single-threaded one,
    bit for bit."""
    import threading

    import torch
    from paper_2511_01255_gb300 import workloads as W
    N, NP = 777, 48
    X = torch.from_numpy(W.random_genes(NP, N, seed=99)).cuda()
    probs = [[(N, 0.3 + 0.013 * (40 * t + k), 2.0 + 0.007 * k) for k in range(40)] for t in range(4)]
    q.qpm_release_caches()
    ref = {}
    for t in range(4):
        for p in probs[t]:
            D = torch.empty((NP, 2), device="cuda")
            q.qpm_eval(p[0], p[1], p[2], X, D)
            torch.cuda.synchronize()
            ref[p] = D.cpu().numpy()
    q.qpm_release_caches()
    out, errors = {}, []

    def work(t):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                res = []
                for p in probs[t]:
                    D = torch.empty((NP, 2), device="cuda")
                    if t % 2:
                        q.qpm_eval_shg(p[0], p[1], X, torch.empty((NP, 2), device="cuda"))
                    q.qpm_eval(p[0], p[1], p[2], X, D)
                    res.append((p, D))
                s.synchronize()
                for p, D in res:
                    out[p] = D.cpu().numpy()
        except Exception as e:  # reported below
            errors.append(repr(e))

    th = [threading.Thread(target=work, args=(t,)) for t in range(4)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    for p, D in ref.items():
        assert np.array_equal(out[p], D), p
    q.qpm_release_caches()
