"""Pins for the oracle's random numbers, DE/GWO updates, leader choice, HWSDA loop
and relaxed gradient -- CPU only.

  * Philox4x32-10 against curand's host generator (a library implementation of
    the same published generator) on counter words 0-2 and both key words;
  * DE donor indices: distinct, never the target, uniformly spread;
  * DE rand/1 + binomial crossover (Sec. 2.2.1) special cases: CR = 0 leaves only
    the forced dimension from the mutant, CR = 1 takes the whole mutant, F = 0
    copies donor r1; every trial gene is either the target's or the textbook
    rand/1 mutant's; the crossover rate matches CR;
  * GWO (Sec. 2.2.2) distributions: with all leaders at 1/2 and the wolf at 0,
    mean and variance of the candidate follow from A = 2a r1 - a, C = 2 r2;
  * top-3 equals a stable sort (numpy lexsort);
  * the HWSDA loop (Sec. 3.2) never loses its best and reaches the exhaustive
    optimum's neighbourhood on a 16-domain problem;
  * the relaxed gradient equals central finite differences and obeys Euler's
    identity for a quadratic form.
"""
import ctypes
import ctypes.util
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if p and os.path.exists(p) or (p and not p.startswith("/")):
            try:
                return ctypes.CDLL(p)
            except OSError:
                pass
    return None


def test_philox_matches_curand_host_generator(orc):
    cur = _curand()
    if cur is None:
        pytest.skip("libcurand not found")
    seed = 0x0123456789ABCDEF
    key = [seed & 0xFFFFFFFF, seed >> 32]
    # curand's host PHILOX4_32_10 generator emits block b of its stream from
    # counter (word0, word1) = (b + offset/4) // 65536 as a 64-bit value, word2 = b % 65536
    for offset in (0, 2 ** 50 + 4 * 65536 * 3):
        gen = ctypes.c_void_p()
        assert cur.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0
        assert cur.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert cur.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        n = 4 * 65536 * 2
        out = np.zeros(n, dtype=np.uint32)
        assert cur.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
        cur.curandDestroyGenerator(gen)
        blocks = out.reshape(-1, 4)
        base = offset // 4
        for b in (0, 1, 5, 65535, 65536, 65536 + 77, 131071):
            pos = base + b
            hi = pos // 65536
            ctr = [hi & 0xFFFFFFFF, hi >> 32, b % 65536, 0]
            assert np.array_equal(orc.philox(ctr, key), blocks[b]), (offset, b)


def test_uniform_and_index_ranges(orc):
    us = np.array([orc.uniform(7, 0, 2, 3, i, j) for i in range(4) for j in range(64)])
    assert us.min() >= 0.0 and us.max() < 1.0
    assert np.all(us * 2 ** 24 == np.floor(us * 2 ** 24))  # 24-bit grid, exact in FP32
    NP, N = 9, 13
    r1s = []
    for g in range(400):
        for i in range(NP):
            r1, r2, r3, jr = orc.de_indices(5, 1, g, i, NP, N)
            assert len({i, r1, r2, r3}) == 4
            assert 0 <= min(r1, r2, r3) and max(r1, r2, r3) < NP
            assert 0 <= jr < N
            r1s.append((r1 - i) % NP)
    # r1 is spread evenly over the NP-1 other individuals (chi-square, 8 dof)
    cnt = np.bincount(r1s, minlength=NP)[1:]
    exp = len(r1s) / (NP - 1)
    chi2 = np.sum((cnt - exp) ** 2 / exp)
    assert cnt.min() > 0 and chi2 < 30.0


def _cfg(orc, NP=12, N=40, G=10, F=0.5, CR=0.9, seed=3, inst=0, combine=0):
    return orc.make_cfg(NP, N, G, F, CR, seed, inst, combine)


def test_init_population_uniform(orc):
    c = _cfg(orc, NP=64, N=256)
    X = orc.init_population(c)
    assert X.min() >= -1.0 and X.max() < 1.0
    assert abs(X.mean()) < 0.02 and abs(X.var() - 1.0 / 3.0) < 0.02
    # x = 2U - 1 with U on the 24-bit grid
    assert np.all((X + 1) * 2 ** 23 == np.floor((X + 1) * 2 ** 23))
    # the draw of gene j of individual i: word j % 4 of Philox at counter
    # (j / 4, i, 0xFFFFFFFF, tag 0), U = (w >> 8) 2^-24, x = 2U - 1
    key = np.array([c.seed & 0xFFFFFFFF, c.seed >> 32], dtype=np.uint32)
    for i, j in ((0, 0), (3, 7), (63, 255), (17, 130)):
        w = int(orc.philox(np.array([j // 4, i, 0xFFFFFFFF, 0], dtype=np.uint32), key)[j % 4])
        U = np.float32(w >> 8) * np.float32(2.0 ** -24)
        assert X[i, j] == np.float32(2) * U - np.float32(1), (i, j)


def test_de_trial_structure(orc):
    # F = 0.7 (not a power of 2, so F (x_r2 - x_r3) is not exact and a fused
    # multiply-add would show)
    c = _cfg(orc, NP=16, N=64, F=0.7, CR=0.9)
    X = orc.init_population(c)
    U = orc.de_trials(c, 4, X)
    taken = 0
    F = np.float32(c.F)
    for i in range(c.NP):
        r1, r2, r3, jr = orc.de_indices(c.seed, c.inst, 4, i, c.NP, c.N)
        # mutant fl(x_r1 + fl(F fl(x_r2 - x_r3))), every operation rounded to FP32
        v = np.clip(X[r1] + F * (X[r2] - X[r3]), -1, 1).astype(np.float32)
        from_v = U[i] == v
        from_x = U[i] == X[i]
        assert np.all(from_v | from_x)
        assert U[i][jr] == v[jr]
        taken += np.sum(from_v & ~from_x)
    frac = taken / (c.NP * c.N)
    assert 0.8 < frac < 0.97  # about CR


def test_de_trial_special_cases(orc):
    X = orc.init_population(_cfg(orc, NP=10, N=50))
    c0 = _cfg(orc, NP=10, N=50, CR=0.0)
    U = orc.de_trials(c0, 2, X)
    for i in range(10):
        jr = orc.de_indices(c0.seed, 0, 2, i, 10, 50)[3]
        diff = np.nonzero(U[i] != X[i])[0]
        assert set(diff.tolist()) <= {jr}
    c1 = _cfg(orc, NP=10, N=50, CR=1.0, F=0.0)
    U = orc.de_trials(c1, 2, X)
    for i in range(10):
        r1 = orc.de_indices(c1.seed, 0, 2, i, 10, 50)[0]
        assert np.array_equal(U[i], X[r1])  # F = 0: mutant is donor r1


def test_gwo_candidate_moments(orc):
    NP, N, G = 8, 20000, 100
    c = _cfg(orc, NP=NP, N=N, G=G)
    X = np.zeros((NP, N), dtype=np.float32)
    X[:3] = 0.5  # leaders alpha, beta, gamma at 1/2; omega wolves at 0
    g = 90
    a = orc.a_of(g, G)
    assert a == np.float32(0.2)
    Y = orc.gwo_candidates(c, g, X, np.array([0, 1, 2]))
    y = Y[3:].ravel().astype(np.float64)
    assert np.array_equal(Y[:3], X[:3])
    # Y_k = 1/2 - A |C/2| with E[A] = 0, E[A^2] = a^2/3, E[C^2] = 4/3 -> var(y) = a^2/27
    assert abs(y.mean() - 0.5) < 4 * np.sqrt(a * a / 27 / y.size)
    assert abs(y.var() / (a * a / 27) - 1.0) < 0.04
    assert y.min() >= 0.5 - a and y.max() <= 0.5 + a


def test_gwo_pair_from_one_word(orc):
    """The GWO pair (r1, r2) of leader k and gene j are the high and low 16 bits of
    one generator word (tag 3 + k), and the move is evaluated in FP32 in its written
    order: a candidate recomputed here from the words."""
    NP, N, G, seed = 6, 9, 50, 12345
    c = _cfg(orc, NP=NP, N=N, G=G, seed=seed)
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (NP, N)).astype(np.float32)
    lead = np.array([2, 0, 5])
    g, i = 17, 3
    Y = orc.gwo_candidates(c, g, X, lead)
    a = np.float32(orc.a_of(g, G))
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    for j in range(N):
        Xk = []
        for k in range(3):
            w = int(orc.philox(np.array([j // 4, i, g, 3 + k], dtype=np.uint32), key)[j % 4])
            r1 = np.float32(w >> 16) * np.float32(2.0 ** -16)
            r2 = np.float32(w & 0xFFFF) * np.float32(2.0 ** -16)
            A = np.float32(np.float32(2 * a) * r1) - a
            C = np.float32(2) * r2
            Xp = X[lead[k], j]
            d = np.float32(abs(np.float32(C * Xp) - X[i, j]))
            Xk.append(np.float32(Xp - np.float32(A * d)))
        y = np.float32(np.float32(np.float32(Xk[0] + Xk[1]) + Xk[2]) / np.float32(3))
        assert Y[i, j] == np.clip(y, -1, 1), j


def test_gwo_a_schedule(orc):
    G = 2000
    a = np.array([orc.a_of(g, G) for g in range(G)])
    assert a[0] == 2.0 and np.all(np.diff(a) < 0) and abs(a[-1] - 2.0 / G) < 1e-7


@pytest.mark.parametrize("G", [1, 7, 500, 1000, 2000, 4999, 20000])
def test_gwo_a_equals_fp64_form(orc, G):
    """a_g as one rounded FP32 division 2(G - g)/G equals 2(1 - g/G) evaluated in
    FP64 and rounded to FP32, for every generation."""
    g = np.arange(G)
    a = np.array([orc.a_of(int(k), G) for k in g], dtype=np.float32)
    assert np.array_equal(a, (2.0 * (1.0 - g / G)).astype(np.float32))


def test_gwo_weighted_combination_reduces_to_mean(orc):
    # with identical leaders and the wolf on them, A d = A |C-1| |x| for every k, and the
    # |X_k|-weighted combination of equal-sign X_k is (sum X_k^2 / sum |X_k|) / 3
    NP, N = 6, 512
    X = np.full((NP, N), 0.25, dtype=np.float32)
    cm = _cfg(orc, NP=NP, N=N, G=10, combine=0)
    cw = _cfg(orc, NP=NP, N=N, G=10, combine=1)
    Ym = orc.gwo_candidates(cm, 9, X, np.array([0, 1, 2]))
    Yw = orc.gwo_candidates(cw, 9, X, np.array([0, 1, 2]))
    # a = 0.2: every X_k is positive; weighted/3 is about 1/3 of the mean
    assert np.all(Yw[3:] > 0)
    ratio = Yw[3:].mean() / Ym[3:].mean()
    assert abs(ratio - 1.0 / 3.0) < 0.01


def test_top3_matches_stable_sort(orc):
    rng = np.random.default_rng(5)
    for NP in (4, 5, 31, 300):
        f = rng.integers(0, 6, NP).astype(np.float32)  # many ties
        lead = orc.top3(f)
        ref = np.lexsort((np.arange(NP), -f))[:3]
        assert np.array_equal(lead, ref)


def test_hwsda_greedy_selection_never_loses_fitness(orc):
    # one-to-one greedy selection (Sec. 2.2.1 step 4, Sec. 3.2 Step 5): every
    # individual ends at least as fit as it started, and at least as fit as every
    # trial and candidate it was offered in its last generation
    k1, k2 = 2 * np.pi / 7.0, 2 * np.pi / 1.6
    c = _cfg(orc, NP=16, N=16, G=40)
    X, f, tr = orc.hwsda_run(c, k1, k2, want_trace=True)
    NP = c.NP
    assert np.all(f >= tr[:NP])
    last_trial = tr[NP * (1 + 2 * (c.G - 1)):NP * (2 + 2 * (c.G - 1))]
    last_cand = tr[NP * (2 + 2 * (c.G - 1)):NP * (3 + 2 * (c.G - 1))]
    assert np.all(f >= last_trial)
    ok = ~np.isnan(last_cand)
    assert np.all(f[ok] >= last_cand[ok]) and np.sum(~ok) == 3
    # the final fitness is that of the final genes
    assert np.allclose(f, np.abs(orc.deff_genes(X, k1, k2)) ** 2, rtol=1e-13)


def test_hwsda_reaches_bruteforce_optimum_small(orc):
    """N = 16 domains, dk1 w = 2pi/7, dk2 w = 2pi/1.6, NP = 32, 200 generations."""
    with open(os.path.join(GOLDEN, "bruteforce_n16.json")) as fh:
        gold = json.load(fh)
    k1, k2 = gold["kappa1"], gold["kappa2"]
    best, mask, allf = orc.bruteforce(16, k1, k2, want_all=True)
    assert abs(best - gold["best_f"]) <= 1e-12 * best and mask == gold["best_mask"]
    c = _cfg(orc, NP=32, N=16, G=200, F=0.5, CR=0.9, seed=1)
    X, f = orc.hwsda_run(c, k1, k2)
    # reaching the exhaustive optimum is an empirical outcome of the heuristic, not a
    # property of the method: require a design in the top 0.1 % of all 65536 patterns
    # and no value above the optimum (the gap for seed 1 is 1.5 %)
    assert f.max() <= best * (1 + 1e-12)
    assert f.max() >= np.quantile(allf, 0.999), (f.max(), best)


def test_lockstep_replay_equals_free_run_when_decisions_agree(orc):
    k1, k2 = 2 * np.pi / 7.0, 2 * np.pi / 1.6
    c = _cfg(orc, NP=10, N=24, G=15, seed=9)
    X, f, tr = orc.hwsda_run(c, k1, k2, want_trace=True)
    # feed the oracle's own fitness back as FP32 decision values: same trajectory unless
    # rounding to FP32 merges two FP64 values (not the case here)
    ls = tr.astype(np.float32)
    ls[np.isnan(tr)] = np.nan
    X2, f2 = orc.hwsda_run(c, k1, k2, lockstep=ls)
    assert np.array_equal(X, X2)


def test_relaxed_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(21)
    N = 96
    theta = rng.normal(size=N)
    k1, k2 = 2 * np.pi / 6.9, 2 * np.pi / 1.55
    g, D = orc.grad_relaxed(theta, k1, k2)
    fd = orc.fd_grad(theta, k1, k2, np.arange(N), h=1e-6)
    scale = np.abs(fd).max()
    assert np.max(np.abs(g - fd)) <= 1e-6 * scale
    f, D2 = orc.fit_relaxed(theta, k1, k2)
    assert abs(D - D2) <= 1e-12 * abs(D) and abs(f - abs(D) ** 2) <= 1e-12 * f
    # Euler: f is homogeneous of degree 4 in d, so sum_k d_k df/dd_k = 4 f
    d = np.tanh(theta)
    dfdd = g / (1 - d * d)
    assert abs(np.sum(d * dfdd) - 4 * f) <= 1e-9 * f


def test_decaying_F_schedule(orc):
    """Sec. 3.1.1: F follows (cos(pi g / 2G) + 1)/2 times a factor falling from 1.0 to 0.8."""
    c = _cfg(orc, G=1000, F=0.1)
    c.f_schedule = 1
    F = np.array([orc.F_of(c, g) for g in range(c.G)], dtype=np.float64)
    assert F[0] == np.float32(0.1)
    assert np.all(np.diff(F) <= 0)
    assert abs(F[500] / 0.1 - 0.5 * (np.cos(np.pi / 4) + 1) * 0.95) < 1e-6
    assert abs(F[-1] / 0.1 - 0.4) < 2e-3          # (0 + 1)/2 * 0.8 at the end of the run
    c.f_schedule = 0
    assert all(orc.F_of(c, g) == np.float32(0.1) for g in (0, 10, 999))
    # the schedule reaches the trials: F = 0 at every step reduces rand/1 to copying donor r1
    c0 = _cfg(orc, NP=10, N=30, CR=1.0, F=0.0)
    c0.f_schedule = 1
    X = orc.init_population(c0)
    U = orc.de_trials(c0, 3, X)
    r1 = orc.de_indices(c0.seed, 0, 3, 2, 10, 30)[0]
    assert np.array_equal(U[2], X[r1])


def test_philox_known_answers_of_the_random123_distribution(orc):
    """Philox4x32-10 against the known-answer vectors published with Random123
    (Salmon, Moraes, Dror, Shaw, SC'11), read from tests/golden: they include the
    all-ones counter and a counter whose fourth word is set, the word that carries
    (instance << 8) | tag in this implementation's random-number contract."""
    import numpy as np
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        ctr, key, want = v[0:4], v[4:6], v[6:10]
        assert list(orc.philox(ctr, key)) == want, r


# ------------------------------------------------------------ adaptive F (Sec. 3.1.1)
def _acfg(orc, NP=64, G=100):
    return orc.make_cfg(NP, 16, G, 0.5, 0.9, 1, f_schedule=2)


def test_adaptive_F_spread_is_exact_and_matches_the_textbook_variance(orc):
    """The spread statistic is computed from fitness values quantised against the
    population maximum with integer operations only.  f = (1, 2, 3, 4) quantises to
    2^17 (1, 2, 3, 4) exactly, so cv^2 = (4 * 30 - 100) / 100 = 0.2 exactly; on random
    populations of every scale it agrees with numpy's variance / mean^2 to the
    quantisation's 2^-20 of the maximum."""
    import numpy as np
    cfg = orc.make_cfg(4, 16, 10, 0.5, 0.9, 1, f_schedule=2)
    _, _, st = orc.adaptive_F(cfg, 0, np.array([1, 2, 3, 4], np.float32), np.ones(4), 0.05)
    assert st[0] == 0.2 and st[1] == 1.0 and st[2] == 3.0
    rng = np.random.default_rng(3)
    for scale in (1e-30, 1e-3, 1.0, 7e5, 3e11, 1e30):
        for NP in (5, 64, 1000):
            f = (rng.random(NP) ** 3 * scale).astype(np.float32)
            cfg = orc.make_cfg(NP, 16, 10, 0.5, 0.9, 1, f_schedule=2)
            _, _, st = orc.adaptive_F(cfg, 3, f, np.ones(NP), 0.05)
            f64 = f.astype(np.float64)
            ref = f64.var() / f64.mean() ** 2
            assert abs(st[0] - ref) <= 1e-5 * max(ref, 1.0), (scale, NP)


def test_adaptive_F_takes_every_branch(orc):
    """Sec. 3.1.1: low diversity (cv < 0.05, or under 10 % of the trials improved)
    raises F by 1.25 up to 0.1; high diversity (cv > 0.5) or a fitness range under
    10^3 lowers it by 0.8 down to 0.01; otherwise F follows the schedule
    0.1 (cos(pi g / 2G) + 1) / 2 (1 - 0.2 (g / G)^2) of the next generation."""
    import numpy as np
    rng = np.random.default_rng(11)
    NP, G = 64, 100
    cfg = _acfg(orc, NP, G)
    imp = np.zeros(NP, np.uint8)
    imp[:10] = 1  # 10 of 64 improved: a convergence rate above 0.1
    moderate = (1e6 * (1.0 + rng.random(NP))).astype(np.float32)  # cv ~ 0.19, range ~ 1e6
    narrow = (1e6 * (1.0 + 0.01 * rng.random(NP))).astype(np.float32)  # cv ~ 0.002
    wide = (1e6 * rng.random(NP) ** 6).astype(np.float32)  # cv > 1
    flat = (1000.0 + 400.0 * rng.random(NP)).astype(np.float32)  # cv ~ 0.1, range < 1e3
    g, Fg = 40, np.float32(0.05)
    br, Fn, st = orc.adaptive_F(cfg, g, moderate, imp, Fg)
    assert br == 0 and 0.0025 < st[0] < 0.25 and Fn == orc.F_of(cfg, g + 1)
    x = (g + 1) / G
    sched = 0.1 * (math.cos(math.pi * (g + 1) / (2 * G)) + 1) / 2 * (1 - 0.2 * x * x)
    assert Fn == np.float32(sched)
    br, Fn, _ = orc.adaptive_F(cfg, g, narrow, imp, Fg)
    assert br == 1 and Fn == np.float32(Fg * np.float32(1.25))
    br, Fn, _ = orc.adaptive_F(cfg, g, moderate, np.zeros(NP, np.uint8), Fg)  # stagnating
    assert br == 1 and Fn == np.float32(Fg * np.float32(1.25))
    br, Fn, st = orc.adaptive_F(cfg, g, wide, imp, Fg)
    assert br == 2 and st[0] > 0.25 and Fn == np.float32(Fg * np.float32(0.8))
    br, Fn, st = orc.adaptive_F(cfg, g, flat, imp, Fg)
    assert br == 2 and st[2] < 1000.0 and st[0] > 0.0025 and Fn == np.float32(Fg * np.float32(0.8))
    # the bounds of [0.01, 0.1]
    assert orc.adaptive_F(cfg, g, narrow, imp, np.float32(0.09))[1] == np.float32(0.1)
    assert orc.adaptive_F(cfg, g, wide, imp, np.float32(0.011))[1] == np.float32(0.01)
    # a population of zero fitness has no spread: low
    assert orc.adaptive_F(cfg, g, np.zeros(NP, np.float32), imp, Fg)[0] == 1


def test_adaptive_F_schedule_end_points(orc):
    cfg = _acfg(orc, 8, 200)
    assert orc.F_of(cfg, 0) == np.float32(0.1)
    assert abs(orc.F_of(cfg, 200) - 0.1 * 0.5 * 0.8) < 1e-8


def test_adaptive_F_run_equals_its_generations(orc):
    """hwsda_run with the adaptive F equals the same loop taken generation by
    generation (population bit for bit, and the F history); every F stays in
    [0.01, 0.1] and the first is the schedule's 0.1."""
    import numpy as np
    from paper_2511_01255_gb300 import workloads as W
    c = W.SMALL
    G = 25
    cfg = orc.make_cfg(c["NP"], c["N"], G, c["F"], c["CR"], c["seed"], f_schedule=2)
    X, f, Fh = orc.hwsda_run(cfg, c["kappa1"], c["kappa2"], want_F=True)
    assert Fh[0] == np.float32(0.1) and np.all((Fh >= 0.01) & (Fh <= 0.1))
    Xg = orc.init_population(cfg)
    f64 = np.abs(orc.deff_genes(Xg, c["kappa1"], c["kappa2"])) ** 2
    fdec = f64.astype(np.float32)
    F = np.float32(orc.F_of(cfg, 0))
    branches = set()
    for g in range(G):
        assert F == Fh[g]
        Xg, fdec, f64, _, _, _, F, br = orc.hwsda_generation(cfg, c["kappa1"], c["kappa2"], g, Xg,
                                                             fdec, f64, F=F)
        branches.add(br)
    assert F == Fh[G]
    assert np.array_equal(X, Xg)
    assert 1 in branches  # the rule does fire on this problem


# ------------------------------------------------- the loop's objectives (Sec. 2.1, Sec. 5)
KAPPAS3 = [(2 * math.pi / 6.5, 2 * math.pi / 1.4), (2 * math.pi / 6.9, 2 * math.pi / 1.55),
           (2 * math.pi / 7.4, 2 * math.pi / 1.7)]


def test_objective_rows_equal_the_field_integrals(orc):
    """Every objective the loop can optimise, row by row, from the separately pinned
    field integrals: |d_eff|^2 (cascaded), |E|^2 (SHG), and sum_k |G0 - G_k| +
    beta (G_max - G_min) with G_k the cascaded or SHG field magnitude (Sec. 5)."""
    import numpy as np
    from paper_2511_01255_gb300 import workloads as W
    N, NP = 300, 7
    X = W.random_genes(NP, N, seed=9)
    k1, k2 = KAPPAS3[1]
    G0, beta = 3.0e4, 0.6
    cfg0 = orc.make_cfg(NP, N, 5, 0.5, 0.9, 1)
    assert np.allclose(orc.objective_rows(cfg0, X, k1, k2), np.abs(orc.deff_genes(X, k1, k2)) ** 2,
                       rtol=1e-13, atol=0)
    cfg1 = orc.make_cfg(NP, N, 5, 0.5, 0.9, 1, obj=1)
    assert np.allclose(orc.objective_rows(cfg1, X, k1, k2), np.abs(orc.shg_genes(X, k1)) ** 2,
                       rtol=1e-13, atol=0)
    for obj in (2, 3):
        cfg = orc.make_cfg(NP, N, 5, 0.5, 0.9, 1, obj=obj, kappas=KAPPAS3, G0=G0, beta=beta)
        if obj == 2:
            G = np.abs(np.stack([orc.deff_genes(X, a, b) for a, b in KAPPAS3], axis=1))
        else:
            G = np.abs(np.stack([orc.shg_genes(X, a) for a, _ in KAPPAS3], axis=1))
        want = np.abs(np.float32(G0) - G).sum(axis=1) + np.float32(beta) * (G.max(axis=1) - G.min(axis=1))
        assert np.allclose(orc.objective_rows(cfg, X), want, rtol=1e-12, atol=0), obj
    # the cascaded multi objective equals the multi_objective oracle used by qpm_eval_multi
    cfg = orc.make_cfg(NP, N, 5, 0.5, 0.9, 1, obj=2, kappas=KAPPAS3, G0=G0, beta=beta)
    _, ref = orc.multi_objective(X, KAPPAS3, np.float32(G0), np.float32(beta))
    assert np.allclose(orc.objective_rows(cfg, X), ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("obj", [1, 2, 3])
def test_objective_loops_keep_their_best_and_lead_with_it(orc, obj):
    """The loop maximises |E|^2 (obj 1) and minimises the multi-wavelength objectives
    (obj 2, 3): generation by generation the best value never gets worse, and the
    three leaders are the three best survivors in the objective's direction (ties to
    the lower index)."""
    import numpy as np
    N, NP, G = 40, 12, 15
    cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 2, obj=obj, kappas=KAPPAS3[:2], G0=200.0, beta=0.5)
    k1, k2 = KAPPAS3[0]
    X = orc.init_population(cfg)
    f64 = orc.objective_rows(cfg, X, k1, k2)
    fdec = f64.astype(np.float32)
    best = f64.min() if obj >= 2 else f64.max()
    for g in range(G):
        Xn, fdec_n, f64_n, _, _, lead = orc.hwsda_generation(cfg, k1, k2, g, X, fdec, f64)
        # leaders: from the DE survivors, i.e. recompute by replaying DE alone
        U = orc.de_trials(cfg, g, X)
        fu = orc.objective_rows(cfg, U, k1, k2)
        surv = np.where(fu <= f64, fu, f64) if obj >= 2 else np.where(fu >= f64, fu, f64)
        key = surv if obj >= 2 else -surv
        order = np.lexsort((np.arange(NP), key))
        assert list(lead) == list(order[:3])
        X, fdec, f64 = Xn, fdec_n, f64_n
        nb = f64.min() if obj >= 2 else f64.max()
        assert (nb <= best) if obj >= 2 else (nb >= best)
        best = nb
    assert np.allclose(f64, orc.objective_rows(cfg, X, k1, k2), rtol=0, atol=0)


def test_shg_multi_objective_against_exhaustive_search(orc):
    """A 10-domain, 3-wavelength SHG design: the loop's best objective after 60
    generations is no better than the exhaustive minimum over all 1024 patterns and
    no worse than the best of its initial population."""
    import itertools
    import numpy as np
    N, NP, G = 10, 16, 60
    kap = [(2 * math.pi / 2.3, 0.0), (2 * math.pi / 3.1, 0.0), (2 * math.pi / 4.2, 0.0)]
    cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 5, obj=3, kappas=kap, G0=8.0, beta=0.5)
    allX = np.array(list(itertools.product([-1.0, 1.0], repeat=N)), dtype=np.float32)
    cfg_all = orc.make_cfg(allX.shape[0], N, G, 0.5, 0.9, 5, obj=3, kappas=kap, G0=8.0, beta=0.5)
    fmin = orc.objective_rows(cfg_all, allX).min()
    X0 = orc.init_population(cfg)
    f0 = orc.objective_rows(cfg, X0).min()
    X, f = orc.hwsda_run(cfg, 0.0, 0.0)
    assert fmin - 1e-9 <= f.min() <= f0


# ------------------------------------------------ four-leader discrete GWO (Sec. 3.1.2)
def test_discrete_gwo_thresholds_at_both_ends(orc):
    """Start of the run (tau = 0): dispersion 0.5, social rate 0.3, disturbance 0.1 and
    P(+1) = 0.5 n/4 + 0.25; end (tau = 1): no dispersion, no social learning,
    disturbance 0.01 and the leaders' majority (a tie stays at 1/2)."""
    social, flip, plus = orc.discrete_thresholds(0, 100)
    assert social == 19660 and flip == 6553  # floor(65536 * 0.3), floor(65536 * 0.1)
    assert plus == [16384, 24576, 32768, 40960, 49152]
    social, flip, plus = orc.discrete_thresholds(100, 100)
    assert social == 0 and flip == 655 and plus == [0, 0, 32768, 65536, 65536]


def test_discrete_gwo_candidate_frequencies(orc):
    """Each candidate gene is +-1; for every count n of the four leaders at +1, the
    frequency of +1 over many genes equals what the rule implies:
      (1 - sigma) [(1 - mu) P_n + mu (1 - P_n)] + sigma [(1 - mu) n/4 + mu (1 - n/4)]
    (copy a random leader with probability sigma, else +1 with probability P_n, then
    flip with probability mu), within 5 binomial standard deviations."""
    import numpy as np
    NP, N, G, g = 6, 20000, 50, 20
    cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 3, combine=2)
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, (NP, N)).astype(np.float32)
    lead = np.array([0, 1, 2, 3], dtype=np.int32)
    Y = orc.gwo_candidates(cfg, g, X, lead)
    assert np.array_equal(Y[:4], X[:4])
    cand = Y[4:]
    assert np.all(np.abs(cand) == 1.0)
    n = (X[:4] >= 0).sum(axis=0)
    tau = g / G
    sigma, mu = 0.3 * (1 - tau), 0.1 * (1 - tau) + 0.01 * tau
    _, _, plus = orc.discrete_thresholds(g, G)
    for k in range(5):
        sel = n == k
        if sel.sum() < 200:
            continue
        Pn = plus[k] / 65536.0
        want = (1 - sigma) * ((1 - mu) * Pn + mu * (1 - Pn)) + sigma * ((1 - mu) * k / 4 + mu * (1 - k / 4))
        got = (cand[:, sel] > 0).mean()
        m = cand[:, sel].size
        assert abs(got - want) <= 5 * math.sqrt(want * (1 - want) / m), (k, got, want)


def test_discrete_gwo_loop(orc):
    """The hybrid loop with the discrete four-leader GWO: four leaders (a stable sort of
    the DE survivors), the best never lost, every moved wolf's accepted genes +-1."""
    import numpy as np
    from paper_2511_01255_gb300 import workloads as W
    c = W.SMALL
    G = 30
    cfg = orc.make_cfg(c["NP"], c["N"], G, c["F"], c["CR"], c["seed"], combine=2)
    X = orc.init_population(cfg)
    f64 = orc.objective_rows(cfg, X, c["kappa1"], c["kappa2"])  # re^2 + im^2, as the loop
    fdec = f64.astype(np.float32)
    best = f64.max()
    for g in range(G):
        U = orc.de_trials(cfg, g, X)
        fu = orc.objective_rows(cfg, U, c["kappa1"], c["kappa2"])
        surv = np.where(fu >= f64, fu, f64)
        Xn, fdec, f64n, _, _, lead = orc.hwsda_generation(cfg, c["kappa1"], c["kappa2"], g, X, fdec, f64)
        assert list(lead) == list(np.lexsort((np.arange(c["NP"]), -surv))[:4])
        moved = [i for i in range(c["NP"]) if i not in lead and f64n[i] != surv[i]]
        for i in moved:
            assert np.all(np.abs(Xn[i]) == 1.0)
        X, f64 = Xn, f64n
        assert f64.max() >= best
        best = f64.max()
