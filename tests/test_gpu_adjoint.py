"""GPU parity of the relaxed fitness and its hand-written adjoint, and of the
leader polish built on them.

Relaxed rows: d = tanh(theta); f = |d_eff|^2 (Sec. 2.1 integral for real d).
Gradient tolerance (FP32 against FP64): |g - g_ref| <= 1e-4 * max(|g_ref|,
max over the compared coordinates of |g_ref|).
"""
import math

import numpy as np
import pytest

from helpers import TOL_D, deff_err, fit_err

pytestmark = pytest.mark.gpu

K1, K2 = 2 * math.pi / 6.9, 2 * math.pi / 1.55
TOL_G = 1e-4


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01255_gb300 as q
    q.lib()
    return q


def fwd_bwd(q, theta_np, k1, k2, gf=None):
    import torch
    th = torch.from_numpy(theta_np).cuda()
    B, N = th.shape
    D = torch.empty((B, 2), device="cuda")
    f = torch.empty(B, device="cuda")
    A = q.relaxed_saved(B, N)
    q.qpm_deff_relaxed_fwd(N, k1, k2, th, D, f, A)
    g = torch.empty_like(th)
    gft = None if gf is None else torch.from_numpy(gf.astype(np.float32)).cuda()
    q.qpm_deff_relaxed_bwd(N, k1, k2, th, D, A, gft, g)
    torch.cuda.synchronize()
    return D.cpu().numpy(), f.cpu().numpy(), g.cpu().numpy()


def grad_err(g, ref):
    scale = np.maximum(np.abs(ref), np.abs(ref).max())
    return np.max(np.abs(g - ref) / scale)


@pytest.mark.parametrize("N", [1, 5, 255, 256, 257, 1000, 4096])
def test_relaxed_fwd_bwd_against_oracle(q, orc, N):
    from paper_2511_01255_gb300 import workloads as W
    B = 5
    theta = W.relaxed_theta(B, N, seed=N)
    D, f, g = fwd_bwd(q, theta, K1, K2)
    for r in range(B):
        ref_g, ref_D = orc.grad_relaxed(theta[r].astype(np.float64), K1, K2)
        assert deff_err(D[r:r + 1], np.array([ref_D]), N).max() < TOL_D
        assert grad_err(g[r], ref_g) < TOL_G


@pytest.mark.parametrize("N,ld_extra,ldg_extra", [(1000, 0, 0), (1000, 1, 3), (1000, 4, 1),
                                                   (1000, 1, 0), (4097, 3, 3), (100003, 1, 1)])
def test_relaxed_ragged_batch_and_strided_rows(q, orc, N, ld_extra, ldg_extra):
    """B = 130 rows: a warp takes 32 rows (lane = row), so the last warp holds rows
    128-129 and 30 rows past the end; N domains in rows of N + ld_extra floats
    (rows whose pitch is a multiple of 16 bytes arrive as TMA tiles, the others
    through registers) and gradients written into rows of N + ldg_extra floats (TMA
    tile stores for a pitch that is a multiple of 16 bytes, plain stores otherwise).
    N = 4097 in rows of 4100 floats: the last segment (160 domains from 4000) has a
    step with one domain inside the row and one entirely past it.  N = 100003: 391
    segments of 256 domains, more than one warp's 32 lanes, so the combine walks the
    segments in chunks.  The padding holds NaN, which must neither be read into the
    sums nor be overwritten."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    B = 130
    theta = W.relaxed_theta(B, N, seed=7)
    # NaN in the padding: nothing past a row's N floats may enter the sums
    big = torch.full((B, N + ld_extra), float("nan"), dtype=torch.float32, device="cuda")
    big[:, :N] = torch.from_numpy(theta).cuda()
    th = big[:, :N]
    D = torch.empty((B, 2), device="cuda")
    f = torch.empty(B, device="cuda")
    A = q.relaxed_saved(B, N)
    q.qpm_deff_relaxed_fwd(N, K1, K2, th, D, f, A)
    gbig = torch.full((B, N + ldg_extra), 7.0, dtype=torch.float32, device="cuda")
    q.qpm_deff_relaxed_bwd(N, K1, K2, th, D, A, None, gbig[:, :N])
    torch.cuda.synchronize()
    D, gb = D.cpu().numpy(), gbig.cpu().numpy()
    assert np.all(gb[:, N:] == 7.0)  # nothing written past the rows
    assert np.all(np.isfinite(D)) and np.all(np.isfinite(gb[:, :N]))
    for r in (0, 31, 32, 63, 64, 127, 128, 129):
        ref_g, ref_D = orc.grad_relaxed(theta[r].astype(np.float64), K1, K2)
        assert deff_err(D[r:r + 1], np.array([ref_D]), N).max() < TOL_D, r
        assert grad_err(gb[r, :N], ref_g) < TOL_G, r


def test_tanh_and_derivative_accuracy(q):
    """The kernels form d = tanh(theta) and 1 - d^2 from one hardware exponential
    and reciprocal.  A one-domain row exposes both: its sum of a (the first
    float of its saved block) is d itself (p2_0 = 1), and its gradient is 4 |psi|^2 d^3 (1 - d^2).  Checked over a dense
    sweep of theta against FP64: d to 5e-7 absolute, 1 - d^2 to 1e-5 relative
    (where d and the gradient are representable)."""
    import torch
    theta = np.concatenate([np.linspace(-30.0, 30.0, 60001),
                            [0.0, 1e-30, -1e-30, 1e-6, -1e-6, 1e-3, -1e-3]]).astype(np.float32)
    B = theta.size
    _, f, g = fwd_bwd(q, theta[:, None].copy(), K1, K2)
    th = torch.from_numpy(theta[:, None].copy()).cuda()
    Dd = torch.empty((B, 2), device="cuda")
    A = q.relaxed_saved(B, 1)
    q.qpm_deff_relaxed_fwd(1, K1, K2, th, Dd, None, A)
    torch.cuda.synchronize()
    d = A.cpu().numpy()[:, 0].astype(np.float64)
    ref = np.tanh(theta.astype(np.float64))
    assert np.max(np.abs(d - ref)) <= 5e-7
    assert np.all(np.abs(d) <= 1.0) and np.all(np.sign(d) * np.sign(theta) >= 0)
    # f = |psi|^2 d^4 and df/dtheta = 4 |psi|^2 d^3 (1 - d^2), so g d / (4 f) = 1 - d^2
    sech2 = 1.0 / np.cosh(theta.astype(np.float64)) ** 2
    sel = (np.abs(d) > 1e-2) & (sech2 > 1e-30)
    est = g[sel, 0].astype(np.float64) * d[sel] / (4.0 * f[sel].astype(np.float64))
    assert np.max(np.abs(est - sech2[sel]) / sech2[sel]) <= 1e-5


def test_finite_differences_and_euler_full_size(q, orc):
    """B = 4096 rows of N = 4096, theta ~ N(0, 1): all rows on the GPU; FP64 central
    differences (h = 1e-6) on 64 random coordinates of two rows, the oracle's exact
    gradient on four rows, Euler's identity on every row."""
    from paper_2511_01255_gb300 import workloads as W
    c = W.RELAXED
    B, N = c["B"], c["N"]
    theta = W.relaxed_theta(B, N, seed=c["seed"])
    D, f, g = fwd_bwd(q, theta, c["kappa1"], c["kappa2"])
    rng = np.random.default_rng(5)
    for r in (0, B - 1):
        idx = np.sort(rng.choice(N, 64, replace=False))
        fd = orc.fd_grad(theta[r].astype(np.float64), c["kappa1"], c["kappa2"], idx, h=1e-6)
        assert grad_err(g[r, idx], fd) < TOL_G
    for r in (1, 777, 2048, 4000):
        ref_g, ref_D = orc.grad_relaxed(theta[r].astype(np.float64), c["kappa1"], c["kappa2"])
        assert grad_err(g[r], ref_g) < TOL_G
        assert fit_err(f[r:r + 1], np.array([abs(ref_D) ** 2]), N).max() < 2 * TOL_D
    # f is homogeneous of degree 4 in d: sum_k d_k df/dd_k = 4 f (FP64 sum of FP32 terms)
    d = np.tanh(theta.astype(np.float64))
    euler = np.sum(d * g / (1.0 - d * d), axis=1)
    scale = np.abs(d * g / (1.0 - d * d)).sum(axis=1)
    assert np.max(np.abs(euler - 4 * f) / np.maximum(scale, 4 * f)) < 1e-4


def test_autograd_function(q, orc):
    import torch
    from paper_2511_01255_gb300 import workloads as W
    N = 700
    theta = W.relaxed_theta(3, N, seed=2)
    th = torch.from_numpy(theta).cuda().requires_grad_(True)
    w = torch.tensor([0.5, -2.0, 1.0], device="cuda")
    loss = (q.deff_relaxed(th, K1, K2) * w).sum()
    loss.backward()
    g = th.grad.cpu().numpy()
    for r in range(3):
        ref_g, _ = orc.grad_relaxed(theta[r].astype(np.float64), K1, K2)
        assert grad_err(g[r], float(w[r]) * ref_g) < TOL_G


@pytest.mark.parametrize("N,NP", [(1000, 32), (4096, 256)])
def test_polish_leaders(q, orc, N, NP):
    """After polishing, every leader's fitness is at least what it was, its new genes
    evaluate (oracle, FP64) to the stored fitness, and nobody else changed."""
    import torch
    prm = q.Params(NP, 50, 0.5, 0.9, 4, 0, 1)
    with q.State([(N, K1, K2)], [prm]) as st:
        st.init()
        st.run(10, q.RUN_GRAPH)
        X0, f0, _ = st.population()
        acc = torch.zeros(3, dtype=torch.int32, device="cuda")
        q.qpm_polish_leaders(st.h, 0, steps=8, lr=0.5, tau=3.0, accepted_out=acc)
        X1, f1, _ = st.population()
        torch.cuda.synchronize()
        X0, f0, X1, f1 = X0.cpu().numpy(), f0.cpu().numpy(), X1.cpu().numpy(), f1.cpu().numpy()
        lead = orc.top3(f0)
        others = np.setdiff1d(np.arange(NP), lead)
        assert np.array_equal(X0[others], X1[others]) and np.array_equal(f0[others], f1[others])
        assert np.all(f1[lead] >= f0[lead])
        ref = np.abs(orc.deff_genes(X1[lead], K1, K2)) ** 2
        assert fit_err(f1[lead], ref, N).max() < 2 * TOL_D
        a = acc.cpu().numpy()
        assert set(np.unique(a)) <= {0, 1}
        # polish does something: at least one leader is replaced by genes whose FP64
        # fitness is strictly higher than that of the genes they replace
        old64 = np.abs(orc.deff_genes(X0[lead], K1, K2)) ** 2
        assert a.sum() >= 1
        assert np.any((a == 1) & (ref > old64 * (1 + 1e-6)))
        for k in range(3):
            if not a[k]:  # rejected: the leader is untouched
                assert np.array_equal(X0[lead[k]], X1[lead[k]]) and f1[lead[k]] == f0[lead[k]]
        # the run carries on from the polished population
        st.run(5, q.RUN_PERSISTENT)
        X2, f2, _ = st.population()
        torch.cuda.synchronize()
        assert f2.cpu().numpy().max() >= f1.max()
