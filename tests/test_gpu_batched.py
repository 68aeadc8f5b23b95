"""GPU parity of the batched form (many independent instances in one launch).

Each instance k draws its random numbers with instance index k in the Philox
counter, so the oracle replays instance k with inst = k.  Bit-exact populations
in lockstep; fitness within tolerance; the batched launch equals the
launch-by-launch form on the same state, for every thread-block cluster size
(an instance run by 1, 2 or 4 CTAs gives the same bits).
"""
import math

import numpy as np
import pytest

from helpers import TOL_D, fit_err, lockstep_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01255_gb300 as q
    q.lib()
    return q


INSTANCES = [  # N, kappa1, kappa2, NP, compensated, combine
    (100, 2 * math.pi / 7.0, 2 * math.pi / 1.6, 8, 0, 0),
    (333, 2 * math.pi / 6.2, 2 * math.pi / 1.9, 24, 1, 0),
    (1000, 2 * math.pi / 6.9, 2 * math.pi / 1.55, 64, 1, 1),
    (64, 2 * math.pi / 7.7, 2 * math.pi / 1.35, 5, 0, 0),
    (2500, 2 * math.pi / 6.5, 2 * math.pi / 1.45, 40, 0, 0),
    (77, 2 * math.pi / 8.0, 2 * math.pi / 2.0, 4, 1, 1),
]


def build(q, G, seed=7):
    import torch
    probs = [(N, k1, k2) for N, k1, k2, NP, comp, comb in INSTANCES]
    prms = [q.Params(NP, G, 0.5, 0.9, seed, comb, comp) for N, k1, k2, NP, comp, comb in INSTANCES]
    st = q.State(probs, prms)
    traces = []
    for k, (N, k1, k2, NP, comp, comb) in enumerate(INSTANCES):
        tr = torch.full((NP * (1 + 2 * G),), float("nan"), dtype=torch.float32, device="cuda")
        q.qpm_set_trace(st.h, k, tr)
        traces.append(tr)
        assert q.qpm_team_of(st.h, k) == 32
    return st, traces


@pytest.mark.parametrize("ctas", [1, 2, 4])
def test_batched_lockstep_every_instance(q, orc, ctas):
    import torch
    G = 9
    st, traces = build(q, G)
    st.set_batch_cluster(ctas)
    st.init()
    st.run(4, q.RUN_BATCHED)
    st.run(G - 4, q.RUN_BATCHED)
    torch.cuda.synchronize()
    for k, (N, k1, k2, NP, comp, comb) in enumerate(INSTANCES):
        X, f, D = st.population(k)
        torch.cuda.synchronize()
        trace = traces[k].cpu().numpy()
        cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 7, k, comb)
        Xo, fo, tro = orc.hwsda_run(cfg, k1, k2, lockstep=trace, want_trace=True)
        assert np.array_equal(X.cpu().numpy(), Xo), k
        assert lockstep_errors(trace, tro, N).max() < 2 * TOL_D, k
    st.close()


def test_batched_equals_launches(q):
    import torch
    G = 6
    pops = []
    for mode, ctas in ((q.RUN_BATCHED, 1), (q.RUN_LAUNCHES, 1), (q.RUN_PERSISTENT, 1),
                       (q.RUN_BATCHED, 2), (q.RUN_BATCHED, 8)):
        st, traces = build(q, G, seed=11)
        st.set_batch_cluster(ctas)
        st.init()
        st.run(G, mode)
        torch.cuda.synchronize()
        pops.append([st.population(k)[0].cpu().numpy() for k in range(len(INSTANCES))])
        st.close()
    for other in pops[1:]:
        for a, b in zip(pops[0], other):
            assert np.array_equal(a, b)


def test_batched_states_of_different_sizes_take_turns(q):
    """Two batched states whose phasor tables in shared memory differ (8000 and 500
    domains: 125 KB and 8 KB) run in turns, each replaying its captured launch after
    the other was set up: the larger one's launch still fits, and every population
    equals that of the same state run alone."""
    import torch

    def make(N):
        probs = [(N, 2 * math.pi / 6.9, 2 * math.pi / 1.55), (N // 2, 2 * math.pi / 7.3, 2 * math.pi / 1.7)]
        prms = [q.Params(16, 6, 0.5, 0.9, 5, 0, 0), q.Params(8, 6, 0.5, 0.9, 5, 0, 0)]
        st = q.State(probs, prms)
        st.init()
        return st

    alone = {}
    for N in (8000, 500):
        st = make(N)
        st.run(2, q.RUN_BATCHED)
        st.run(2, q.RUN_BATCHED)
        st.run(2, q.RUN_BATCHED)
        alone[N] = [st.population(k)[0].cpu().numpy() for k in range(2)]
        st.close()
    big = make(8000)
    big.run(2, q.RUN_BATCHED)  # captured with the large tables
    small = make(500)
    small.run(2, q.RUN_BATCHED)
    big.run(2, q.RUN_BATCHED)  # replayed after the small state was set up
    small.run(2, q.RUN_BATCHED)
    big.run(2, q.RUN_BATCHED)
    small.run(2, q.RUN_BATCHED)
    torch.cuda.synchronize()
    for st, N in ((big, 8000), (small, 500)):
        for k in range(2):
            assert np.array_equal(st.population(k)[0].cpu().numpy(), alone[N][k]), (N, k)
        st.close()


def test_batched_full_size_sampled(q, orc):
    """512 instances (N ~ U[500, 8000], NP in {64..512}): two batched generations, then
    the third replayed by the oracle for three sampled instances."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    inst = W.batched_instances(512)
    probs = [(c["N"], c["kappa1"], c["kappa2"]) for c in inst]
    prms = [q.Params(c["NP"], c["G"], c["F"], c["CR"], c["seed"], 0, c["compensated"]) for c in inst]
    st = q.State(probs, prms)
    st.set_batch_cluster(2)
    sample = [0, 137, 511]
    traces = {}
    for k in sample:
        traces[k] = torch.full((inst[k]["NP"] * (1 + 2 * inst[k]["G"]),), float("nan"),
                               dtype=torch.float32, device="cuda")
        q.qpm_set_trace(st.h, k, traces[k])
    st.init()
    st.run(2, q.RUN_BATCHED)
    snaps = {k: st.population(k) for k in sample}
    torch.cuda.synchronize()
    snaps = {k: (v[0].cpu().numpy(), v[1].cpu().numpy()) for k, v in snaps.items()}
    st.run(1, q.RUN_BATCHED)
    torch.cuda.synchronize()
    g0 = 2
    for k in sample:
        c = inst[k]
        NP, N = c["NP"], c["N"]
        X1 = st.population(k)[0].cpu().numpy()
        tr = traces[k].cpu().numpy()
        lt = tr[NP * (1 + 2 * g0):NP * (2 + 2 * g0)]
        lc = tr[NP * (2 + 2 * g0):NP * (3 + 2 * g0)]
        cfg = orc.make_cfg(NP, N, c["G"], c["F"], c["CR"], c["seed"], k, 0)
        mask = np.zeros(NP, dtype=np.uint8)
        mask[[0, NP // 2, NP - 1]] = 1
        X0, f0 = snaps[k]
        Xn, fdec, _, t64, c64, lead = orc.hwsda_generation(cfg, c["kappa1"], c["kappa2"], g0, X0,
                                                           f0, lock_trial=lt, lock_cand=lc,
                                                           eval_mask=mask)
        assert np.array_equal(X1, Xn), k
        sel = mask.astype(bool)
        assert fit_err(lt[sel], t64[sel], N).max() < 2 * TOL_D
    st.close()


def test_batched_adaptive_F_lockstep(q, orc):
    """Instances with the adaptive F (f_schedule 2) next to constant-F instances in one
    batched launch on 2-CTA clusters: each adaptive instance's F history and population
    equal the oracle's lockstep replay."""
    import torch
    G = 10
    probs = [(N, k1, k2) for N, k1, k2, NP, comp, comb in INSTANCES]
    prms = [q.Params(NP, G, 0.5, 0.9, 3, comb, comp, 0, 2 if k % 2 == 0 else 0)
            for k, (N, k1, k2, NP, comp, comb) in enumerate(INSTANCES)]
    st = q.State(probs, prms)
    traces = []
    for k, (N, k1, k2, NP, comp, comb) in enumerate(INSTANCES):
        tr = torch.full((NP * (1 + 2 * G),), float("nan"), dtype=torch.float32, device="cuda")
        q.qpm_set_trace(st.h, k, tr)
        traces.append(tr)
    st.set_batch_cluster(2)
    st.init()
    st.run(G, q.RUN_BATCHED)
    for k, (N, k1, k2, NP, comp, comb) in enumerate(INSTANCES):
        X, f, D = st.population(k)
        Fg = q.qpm_get_F(st.h, k).cpu().numpy()
        torch.cuda.synchronize()
        cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 3, k, comb, 2 if k % 2 == 0 else 0)
        Xo, fo, tro, Fo = orc.hwsda_run(cfg, k1, k2, lockstep=traces[k].cpu().numpy(),
                                        want_trace=True, want_F=True)
        assert np.array_equal(X.cpu().numpy(), Xo), k
        if k % 2 == 0:
            assert np.array_equal(Fg, Fo), k
        else:
            assert np.all(Fg == np.float32(0.5))
    st.close()
