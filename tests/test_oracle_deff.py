"""Pins for the oracle's d_eff (Sec. 2.1) -- CPU only.

The oracle integrates the d_eff double integral by nested Gauss-Legendre
quadrature.  These tests tie it to things fixed by the mathematics, not to
itself:
  * the Gauss-Legendre rule integrates polynomials of degree <= 2Q-1 exactly;
  * closed forms: all domains +1 at dk1 = dk2 = 0 gives L^2/2; the alternating
    sequence at kappa1 = kappa2 = pi (first-order QPM of both steps) gives
    -(2/pi)^2 L^2/2 for every N; dk1 = 0 with all +1 gives int_0^L z e^{-i k2 z} dz;
  * invariants: a global sign flip leaves d_eff unchanged (bit for bit),
    kappa -> -kappa conjugates it;
  * an independent evaluation written here from exact antiderivatives of the
    piecewise-constant integrand (no quadrature), for arbitrary real d;
  * exhaustive enumeration of all 2^N sign patterns against the same analytic
    evaluation.
"""
import numpy as np
import pytest


def phi(k):
    """int_0^1 e^{-iks} ds, exactly."""
    k = float(k)
    if k == 0.0:
        return 1.0 + 0j
    return (1.0 - np.exp(-1j * k)) / (1j * k)


def psi(k1, k2):
    """int_0^1 e^{-i k2 s} int_0^s e^{-i k1 t} dt ds, exactly."""
    if k1 != 0.0:
        return (phi(k2) - phi(k1 + k2)) / (1j * k1)
    if k2 != 0.0:
        return (np.exp(-1j * k2) * (1 + 1j * k2) - 1) / k2 ** 2
    return 0.5 + 0j


def deff_analytic(d, k1, k2):
    """Exact d_eff of a piecewise-constant d over unit domains (units of w^2)."""
    d = np.asarray(d, dtype=np.float64)
    N = d.shape[-1]
    j = np.arange(N)
    b = d * np.exp(-1j * k1 * j)
    a = d * np.exp(-1j * k2 * j)
    excl = np.cumsum(b, axis=-1) - b
    return phi(k1) * phi(k2) * np.sum(a * excl, axis=-1) + psi(k1, k2) * np.sum(
        d * d * np.exp(-1j * (k1 + k2) * j), axis=-1)


def rel(a, b, floor=0.0):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))


def test_gauss_legendre_exact_on_polynomials(orc):
    for Q in (2, 5, 16):
        t, w = orc.gauss_legendre(Q)
        assert np.all(np.diff(np.sort(t)) > 0) and np.all(w > 0)
        for p in range(2 * Q):
            exact = 0.0 if p % 2 else 2.0 / (p + 1)
            assert abs(np.sum(w * t ** p) - exact) < 1e-13, (Q, p)
        # degree 2Q is not integrated exactly (the rule has exactly degree 2Q-1)
        assert abs(np.sum(w * t ** (2 * Q)) - 2.0 / (2 * Q + 1)) > 1e-15


@pytest.mark.parametrize("N", [1, 2, 3, 16, 1000])
def test_all_up_zero_mismatch_is_L2_over_2(orc, N):
    D = orc.deff(np.ones(N), 0.0, 0.0)
    assert abs(D - N * N / 2) <= 1e-13 * N * N


@pytest.mark.parametrize("N", [1, 2, 7, 64, 1001])
def test_alternating_first_order_qpm(orc, N):
    d = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    D = orc.deff(d, np.pi, np.pi)
    exact = -(2.0 / np.pi) ** 2 * N * N / 2
    assert abs(D - exact) <= 1e-12 * abs(exact)


@pytest.mark.parametrize("k2", [0.3, 1.3, 2 * np.pi / 1.55])
def test_unmatched_shg_all_up(orc, k2):
    L = 50
    D = orc.deff(np.ones(L), 0.0, k2)
    exact = (np.exp(-1j * k2 * L) * (1 + 1j * k2 * L) - 1) / k2 ** 2
    assert abs(D - exact) <= 1e-12 * abs(exact)


def test_sign_flip_and_conjugation(orc):
    rng = np.random.default_rng(11)
    for N in (5, 40, 333):
        d = np.where(rng.random(N) < 0.5, -1.0, 1.0)
        k1, k2 = 2 * np.pi / 6.9, 2 * np.pi / 1.55
        D = orc.deff(d, k1, k2)
        assert orc.deff(-d, k1, k2) == D  # bit for bit
        Dc = orc.deff(d, -k1, -k2)
        assert abs(Dc - np.conj(D)) <= 1e-12 * max(abs(D), 1.0)


@pytest.mark.parametrize("N", [1, 2, 3, 17, 256])
def test_matches_exact_antiderivatives(orc, N):
    rng = np.random.default_rng(100 + N)
    for trial in range(6):
        k1, k2 = rng.uniform(-3.5, 3.5, 2)
        if trial == 0:
            k1 = 0.0
        if trial == 1:
            k1, k2 = 0.0, 0.0
        d = rng.uniform(-1, 1, N) if trial % 2 else np.where(rng.random(N) < 0.5, -1.0, 1.0)
        D = orc.deff(d, k1, k2)
        ref = deff_analytic(d, k1, k2)
        assert abs(D - ref) <= 1e-12 * max(abs(ref), N), (N, trial, D, ref)


@pytest.mark.parametrize("N", [1, 2, 17, 1000])
def test_closed_form_scan_matches_quadrature(orc, N):
    """The FP64 closed-form scan (the CPU throughput reference) against the nested
    quadrature of the same integral, including k1 = 0 and k1 = k2 = 0."""
    rng = np.random.default_rng(7 + N)
    X = rng.uniform(-1, 1, (5, N)).astype(np.float32)
    for k1, k2 in ((0.0, 0.0), (0.0, 2.1), (0.9106, 4.0537), (-3.3, 1.2), (1e-6, 3.0)):
        Dq = orc.deff_genes(X, k1, k2)
        Dc = orc.deff_closed_genes(X, k1, k2)
        assert np.all(np.abs(Dc - Dq) <= 1e-11 * np.maximum(np.abs(Dq), N)), (N, k1, k2)


def test_physical_scaling_with_domain_width(orc):
    # d_eff in physical units is w^2 * D(kappa = dk * w): halving w at fixed L doubles N
    # and, at zero mismatch, leaves the physical L^2/2 unchanged
    for w in (1.0, 0.5, 0.25):
        N = int(round(8 / w))
        assert abs(w * w * orc.deff(np.ones(N), 0.0, 0.0) - 32.0) < 1e-11


def test_bruteforce_enumeration(orc):
    N = 10
    k1, k2 = 2 * np.pi / 7.0, 2 * np.pi / 1.6
    best, mask, fit = orc.bruteforce(N, k1, k2, want_all=True)
    s = np.arange(1 << N)
    d = np.where(((s[:, None] >> np.arange(N)) & 1) == 1, -1.0, 1.0)
    f = np.abs(deff_analytic(d, k1, k2)) ** 2
    assert rel(fit, f, floor=1e-9 * f.max()) < 1e-11
    assert best == fit.max() and mask == int(np.argmax(fit))
    # the sign-flipped twin of the optimum attains the same value
    assert fit[mask ^ ((1 << N) - 1)] == best


def test_shg_integral_closed_forms(orc):
    # all domains up: int_0^N e^{-ikz} dz = (1 - e^{-ikN}) / (ik)
    for N, k in ((1, 0.7), (40, 1.3), (333, 2 * np.pi / 6.9)):
        X = np.ones((1, N), dtype=np.float32)
        E = orc.shg_genes(X, k)[0]
        exact = (1 - np.exp(-1j * k * N)) / (1j * k)
        assert abs(E - exact) <= 1e-12 * max(1.0, abs(exact))
    # first-order QPM of SHG: alternating domains at kappa = pi give |E| = (2/pi) N
    for N in (2, 10, 1001):
        X = np.where(np.arange(N) % 2 == 0, 1.0, -1.0).astype(np.float32)[None]
        E = orc.shg_genes(X, np.pi)[0]
        assert abs(abs(E) - 2 * N / np.pi) <= 1e-12 * N
        # the SHG field is linear in d: a global flip negates it exactly (|E| is kept)
        assert orc.shg_genes(-X, np.pi)[0] == -E


def test_multi_objective_against_single_problems(orc):
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (5, 120)).astype(np.float32)
    kap = [(2 * np.pi / 6.9, 2 * np.pi / 1.55), (2 * np.pi / 7.4, 2 * np.pi / 1.7),
           (0.0, 0.0)]
    D, obj = orc.multi_objective(X, kap, G0=1e4, beta=0.5)
    for k, (k1, k2) in enumerate(kap):
        assert np.allclose(D[:, k], orc.deff_genes(X, k1, k2), rtol=0, atol=0)
    G = np.abs(D)
    ref = np.sum(np.abs(1e4 - G), axis=1) + 0.5 * (G.max(axis=1) - G.min(axis=1))
    assert np.allclose(obj, ref, rtol=1e-15, atol=0)
