"""GPU parity of the HWSDA generation step (Sec. 3.2) against the oracle.

Bit-exact: the initial population, every DE trial / GWO candidate that survives,
the leaders, and therefore whole trajectories, when the oracle takes its
selection decisions from the GPU's FP32 fitness (lockstep).  Within tolerance:
every FP32 fitness the GPU computed, against the oracle's FP64 quadrature.
"""
import math

import numpy as np
import pytest

from helpers import TOL_D, deff_err, fit_err, lockstep_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01255_gb300 as q
    q.lib()
    return q


def make(q, N, k1, k2, NP, G, F=0.5, CR=0.9, seed=1, combine=0, comp=0, trace=True, team=0,
         f_schedule=0):
    import torch
    prm = q.Params(NP, G, F, CR, seed, combine, comp, team, f_schedule)
    st = q.State([(N, k1, k2)], [prm])
    tr = None
    if trace:
        tr = torch.full((NP * (1 + 2 * G),), float("nan"), dtype=torch.float32, device="cuda")
        q.qpm_set_trace(st.h, 0, tr)
    return st, tr


def snapshot(st):
    import torch
    X, f, D = st.population()
    torch.cuda.synchronize()
    return X.cpu().numpy(), f.cpu().numpy(), D.cpu().numpy()


def test_init_population_bit_exact(q, orc):
    N, NP = 333, 20
    k1, k2 = 2 * math.pi / 6.9, 2 * math.pi / 1.55
    st, tr = make(q, N, k1, k2, NP, 5, seed=77)
    st.init()
    X, f, D = snapshot(st)
    cfg = orc.make_cfg(NP, N, 5, 0.5, 0.9, 77)
    assert np.array_equal(X, orc.init_population(cfg))
    ref = orc.deff_genes(X, k1, k2)
    assert deff_err(D, ref, N).max() < TOL_D
    st.close()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_small_config_full_run_lockstep(q, orc, mode):
    """N = 16, kappa1 = 2pi/7, kappa2 = 2pi/1.6, NP = 32, 200 generations."""
    from paper_2511_01255_gb300 import workloads as W
    c = W.SMALL
    st, tr = make(q, c["N"], c["kappa1"], c["kappa2"], c["NP"], c["G"], seed=c["seed"])
    st.init()
    st.run(c["G"], mode)
    X, f, D = snapshot(st)
    x_best, d64, fb, idx = st.best()
    import torch
    torch.cuda.synchronize()
    trace = tr.cpu().numpy()
    cfg = orc.make_cfg(c["NP"], c["N"], c["G"], c["F"], c["CR"], c["seed"])
    Xo, fo, tro = orc.hwsda_run(cfg, c["kappa1"], c["kappa2"], lockstep=trace, want_trace=True)
    assert np.array_equal(X, Xo)
    assert lockstep_errors(trace, tro, c["N"]).max() < 2 * TOL_D
    # best individual, its FP64 re-check, and the gap to the exhaustive optimum
    i = int(idx.cpu().item())
    assert i == int(orc.top3(f)[0])
    assert np.array_equal(x_best.cpu().numpy(), X[i])
    ref = orc.deff_genes(X[i:i + 1], c["kappa1"], c["kappa2"])[0]
    d = d64.cpu().numpy()
    assert abs(complex(d[0], d[1]) - ref) <= 1e-9 * abs(ref)
    best, _ = orc.bruteforce(c["N"], c["kappa1"], c["kappa2"])
    assert abs(ref) ** 2 <= best * (1 + 1e-9)
    st.close()


@pytest.mark.parametrize("combine", [0, 1])
@pytest.mark.parametrize("comp", [0, 1])
def test_modes_agree_and_match_oracle_ragged(q, orc, combine, comp):
    """N = 333 (ragged against every team width), NP = 24: the three execution modes
    give bit-identical populations and the oracle's lockstep replay."""
    import torch
    N, NP, G = 333, 24, 12
    k1, k2 = 2 * math.pi / 7.3, 2 * math.pi / 1.4
    res = []
    for mode in (0, 1, 2):
        st, tr = make(q, N, k1, k2, NP, G, seed=5, combine=combine, comp=comp)
        st.init()
        st.run(4, mode)
        st.run(G - 4, mode)
        X, f, D = snapshot(st)
        res.append((X, f, tr.cpu().numpy()))
        st.close()
    for X, f, trace in res[1:]:
        assert np.array_equal(X, res[0][0]) and np.array_equal(f, res[0][1])
        assert np.array_equal(np.isnan(trace), np.isnan(res[0][2]))
    cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 5, 0, combine)
    Xo, fo, tro = orc.hwsda_run(cfg, k1, k2, lockstep=res[0][2], want_trace=True)
    assert np.array_equal(res[0][0], Xo)
    assert lockstep_errors(res[0][2], tro, N).max() < 2 * TOL_D


@pytest.mark.parametrize("mode", [0, 2, 3])
def test_decaying_F_lockstep(q, orc, mode):
    """The Sec. 3.1.1 F schedule (computed on the host in FP64) drives the trials bit
    for bit like the oracle's own evaluation of the same formula."""
    N, NP, G = 333, 24, 14
    k1, k2 = 2 * math.pi / 7.3, 2 * math.pi / 1.4
    st, tr = make(q, N, k1, k2, NP, G, F=0.1, seed=8, f_schedule=1, team=32)
    st.init()
    st.run(G, mode)
    X, f, D = snapshot(st)
    trace = tr.cpu().numpy()
    st.close()
    cfg = orc.make_cfg(NP, N, G, 0.1, 0.9, 8, 0, 0, 1)
    Xo, fo, tro = orc.hwsda_run(cfg, k1, k2, lockstep=trace, want_trace=True)
    assert np.array_equal(X, Xo)
    assert lockstep_errors(trace, tro, N).max() < 2 * TOL_D


@pytest.mark.parametrize("team", [32, 64, 256, 512])
def test_team_widths_lockstep(q, orc, team):
    """Every team width (threads per individual) follows the oracle bit for bit."""
    N, NP, G = 1000, 16, 6
    k1, k2 = 2 * math.pi / 6.9, 2 * math.pi / 1.55
    for mode in (1, 2):
        st, tr = make(q, N, k1, k2, NP, G, seed=3, comp=1, team=team)
        assert q.qpm_team_of(st.h) == team
        st.init()
        st.run(G, mode)
        X, f, D = snapshot(st)
        trace = tr.cpu().numpy()
        st.close()
        cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 3)
        Xo, fo, tro = orc.hwsda_run(cfg, k1, k2, lockstep=trace, want_trace=True)
        assert np.array_equal(X, Xo)
        assert lockstep_errors(trace, tro, N).max() < 2 * TOL_D


@pytest.mark.parametrize("N,team,mode", [(5000, 256, 2), (11000, 32, 3), (4500, 32, 3)])
def test_staged_long_rows_lockstep(q, orc, N, team, mode):
    """Long rows whose update stages rows one group ahead in shared memory: the
    persistent form with the phasor table too large for shared memory (N = 5000,
    so the table entries are staged with the rows), and the batched form with
    the table in global memory (N = 11000) and in shared memory (N = 4500)."""
    NP, G = 12, 4
    k1, k2 = 2 * math.pi / 7.1, 2 * math.pi / 1.45
    st, tr = make(q, N, k1, k2, NP, G, seed=11, comp=1, team=team)
    assert q.qpm_team_of(st.h) == team
    st.init()
    st.run(G, mode)
    X, f, D = snapshot(st)
    trace = tr.cpu().numpy()
    st.close()
    cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 11)
    Xo, fo, tro = orc.hwsda_run(cfg, k1, k2, lockstep=trace, want_trace=True)
    assert np.array_equal(X, Xo)
    assert lockstep_errors(trace, tro, N).max() < 2 * TOL_D


@pytest.mark.parametrize("N,team", [(3000, 512), (5000, 256)])
def test_persistent_several_individuals_per_cta_lockstep(q, orc, N, team):
    """NP = 400 individuals, more than the persistent grid holds CTAs (152 one-CTA
    slots of 512-thread teams, 304 of 256-thread teams), so CTAs loop over several
    individuals per phase: short rows (N = 3000, both slots read, redux leader
    search) and long rows (N = 5000, rows and table staged, warp-0 leader search)."""
    NP, G = 400, 3
    k1, k2 = 2 * math.pi / 6.7, 2 * math.pi / 1.5
    st, tr = make(q, N, k1, k2, NP, G, seed=13, comp=1, team=team)
    assert q.qpm_team_of(st.h) == team
    st.init()
    st.run(G, q.RUN_PERSISTENT)
    X, f, D = snapshot(st)
    trace = tr.cpu().numpy()
    st.close()
    cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 13)
    Xo, fo, tro = orc.hwsda_run(cfg, k1, k2, lockstep=trace, want_trace=True)
    assert np.array_equal(X, Xo)
    assert lockstep_errors(trace, tro, N).max() < 2 * TOL_D


@pytest.mark.parametrize("mode", [1, 2])
def test_solve_end_to_end_host_buffers(q, orc, mode):
    """qpm_solve (create, init, run, read back, destroy, with host buffers) returns
    what the state API returns for the same run, and its FP64 d_eff of the best
    genes matches the oracle's quadrature."""
    import torch
    N, NP, G = 333, 24, 12
    k1, k2 = 2 * math.pi / 7.3, 2 * math.pi / 1.4
    prm = q.Params(NP, G, 0.5, 0.9, 21, 0, 1)
    x_h = torch.empty(N, dtype=torch.float32)
    d_h = torch.empty(2, dtype=torch.float64)
    f_h = torch.empty(1, dtype=torch.float32)
    q.qpm_solve(N, k1, k2, prm, mode, x_h, d_h, f_h)
    with q.State([(N, k1, k2)], [prm]) as st:
        st.init()
        st.run(G, mode)
        x, d64, f, idx = st.best()
        torch.cuda.synchronize()
        assert np.array_equal(x_h.numpy(), x.cpu().numpy())
        assert np.array_equal(d_h.numpy(), d64.cpu().numpy())
        assert f_h.item() == f.item()
    ref = orc.deff_genes(x_h.numpy()[None], k1, k2)[0]
    assert abs(complex(d_h[0].item(), d_h[1].item()) - ref) <= 1e-9 * abs(ref)


def test_automatic_team_rule(q):
    """team = 0: at most 4 domains per thread up to 256 threads; a single long-row
    instance takes 512 threads when one CTA per SM fills the rounds of individuals
    better (1024 individuals on 152 SMs: 304 two-CTA slots leave the fourth round a
    third full, 152 one-CTA slots fill 6.7 of 7 rounds)."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    cases = [(16, 32, 32), (1000, 256, 256), (100000, 256, 256)]
    if nsm == 152:
        cases.append((100000, 1024, 512))
    for N, NP, want in cases:
        with q.State([(N, 1.0, 2.0)], [q.Params(NP, 2, 0.5, 0.9, 1, 0, 1)]) as st:
            assert q.qpm_team_of(st.h) == want, (N, NP)


def test_paper_scale_step_sampled(q, orc):
    """N = 1000, NP = 256, compensated scan: after 600 persistent generations one more
    generation is replayed by the oracle from the GPU's population (bit-exact result,
    FP64 fitness of 48 sampled trials and candidates)."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    c = W.PAPER_SCALE
    N, NP, G = c["N"], c["NP"], c["G"]
    st, tr = make(q, N, c["kappa1"], c["kappa2"], NP, G, seed=c["seed"], comp=1)
    st.init()
    g0 = 600
    st.run(g0, q.RUN_PERSISTENT)
    X0, f0, _ = snapshot(st)
    st.run(1, q.RUN_GRAPH)
    X1, f1, _ = snapshot(st)
    trace = tr.cpu().numpy()
    lt = trace[NP * (1 + 2 * g0):NP * (2 + 2 * g0)]
    lc = trace[NP * (2 + 2 * g0):NP * (3 + 2 * g0)]
    cfg = orc.make_cfg(NP, N, G, c["F"], c["CR"], c["seed"])
    mask = np.zeros(NP, dtype=np.uint8)
    mask[np.random.default_rng(0).choice(NP, 48, replace=False)] = 1
    Xn, fdec, _, t64, c64, lead = orc.hwsda_generation(cfg, c["kappa1"], c["kappa2"], g0, X0, f0,
                                                       lock_trial=lt, lock_cand=lc, eval_mask=mask)
    assert np.array_equal(X1, Xn)
    assert np.array_equal(f1, fdec)
    sel = mask.astype(bool)
    assert fit_err(lt[sel], t64[sel], N).max() < 2 * TOL_D
    ok = sel & ~np.isnan(c64)
    assert fit_err(lc[ok], c64[ok], N).max() < 2 * TOL_D
    # the final population of the whole run is still a valid FP64-checked design
    st.run(G - g0 - 1, q.RUN_PERSISTENT)
    x, d64, fb, idx = st.best()
    torch.cuda.synchronize()
    xb = x.cpu().numpy()[None]
    ref = orc.deff_genes(xb, c["kappa1"], c["kappa2"])[0]
    d = d64.cpu().numpy()
    assert abs(complex(d[0], d[1]) - ref) <= 1e-9 * abs(ref)
    assert abs(float(fb.cpu()) - abs(ref) ** 2) <= 2 * TOL_D * abs(ref) ** 2
    st.close()


def test_precision_scale_step_sampled(q, orc):
    """N = 1e5 domains, NP = 1024: two generations, then the third replayed by the
    oracle from the GPU's population; FP64 fitness of 4 sampled rows."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    c = W.PRECISION
    N, NP, G = c["N"], c["NP"], c["G"]
    st, tr = make(q, N, c["kappa1"], c["kappa2"], NP, G, seed=c["seed"], comp=1)
    st.init()
    st.run(2, q.RUN_PERSISTENT)
    X0, f0, _ = snapshot(st)
    st.run(1, q.RUN_LAUNCHES)
    X1, f1, _ = snapshot(st)
    trace = tr.cpu().numpy()
    g0 = 2
    lt = trace[NP * (1 + 2 * g0):NP * (2 + 2 * g0)]
    lc = trace[NP * (2 + 2 * g0):NP * (3 + 2 * g0)]
    cfg = orc.make_cfg(NP, N, G, c["F"], c["CR"], c["seed"])
    mask = np.zeros(NP, dtype=np.uint8)
    mask[[3, 400, 1000]] = 1
    Xn, fdec, _, t64, c64, lead = orc.hwsda_generation(cfg, c["kappa1"], c["kappa2"], g0, X0, f0,
                                                       lock_trial=lt, lock_cand=lc, eval_mask=mask)
    assert np.array_equal(X1, Xn)
    sel = mask.astype(bool)
    assert fit_err(lt[sel], t64[sel], N).max() < 2 * TOL_D
    st.close()
    del X0, X1, Xn


def test_persistent_wait_timeout_reports_status(q):
    """A device-side wait that runs out ends the kernel with QPM_ERR_TIMEOUT (no trap);
    the context stays usable."""
    import torch
    st, _ = make(q, 4000, 1.0, 2.0, 512, 10, trace=False)
    st.init()
    q.qpm_set_wait_timeout_ns(st.h, 0)
    with pytest.raises(q.QpmError) as e:
        st.run(3, q.RUN_PERSISTENT)
    assert e.value.status == 3
    st.close()
    X = torch.ones((2, 64), device="cuda")
    D = torch.empty((2, 2), device="cuda")
    q.qpm_eval(64, 0.0, 0.0, X, D)
    torch.cuda.synchronize()
    assert abs(D[0, 0].item() - 64 * 64 / 2) < 1e-3


def test_state_errors(q):
    st, _ = make(q, 64, 1.0, 2.0, 8, 3, trace=False)
    with pytest.raises(q.QpmError) as e:
        st.step()
    assert e.value.status == 5
    st.init()
    st.run(3)
    with pytest.raises(q.QpmError) as e:
        st.step()
    assert e.value.status == 1
    assert st.generation == 3
    st.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_checkpoint_resume_is_bit_exact(q, mode):
    """15 generations, checkpoint through qpm_get_population, a fresh state resumed with
    qpm_set_population at generation 15, 15 more: identical to 30 uninterrupted ones."""
    import torch
    N, NP, G = 700, 40, 30
    k1, k2 = 2 * math.pi / 6.9, 2 * math.pi / 1.55
    st, _ = make(q, N, k1, k2, NP, G, seed=21, comp=1, trace=False)
    st.init()
    st.run(G, mode)
    Xa, fa, Da = snapshot(st)
    st.close()
    st, _ = make(q, N, k1, k2, NP, G, seed=21, comp=1, trace=False)
    st.init()
    st.run(15, mode)
    Xc, fc, Dc = st.population()
    torch.cuda.synchronize()
    st.close()
    st2, _ = make(q, N, k1, k2, NP, G, seed=21, comp=1, trace=False)
    st2.init()
    q.qpm_set_population(st2.h, 0, Xc, 15)
    assert st2.generation == 15
    X2, f2, _ = snapshot(st2)
    assert np.array_equal(f2, fc.cpu().numpy())  # re-evaluated fitness is bit-identical
    st2.run(G - 15, mode)
    Xb, fb, Db = snapshot(st2)
    st2.close()
    assert np.array_equal(Xa, Xb) and np.array_equal(fa, fb)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_adaptive_F_lockstep(q, orc, mode):
    """The adaptive F of Sec. 3.1.1 (f_schedule 2): the GPU decides the F of every
    generation from its DE survivors' FP32 fitness and improvement flags; the oracle,
    replaying in lockstep, decides from the same values by the same exact integer
    statistics.  Population bit for bit, and the whole F history."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    for N, NP, G, k1, k2 in ((16, 32, 60, W.SMALL["kappa1"], W.SMALL["kappa2"]),
                             (1000, 256, 12, 2 * math.pi / 6.9, 2 * math.pi / 1.55)):
        st, tr = make(q, N, k1, k2, NP, G, seed=4, comp=1, f_schedule=2)
        st.init()
        st.run(G // 2, mode)
        st.run(G - G // 2, mode)
        X, f, D = snapshot(st)
        Fg = q.qpm_get_F(st.h, 0).cpu().numpy()
        trace = tr.cpu().numpy()
        st.close()
        cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 4, f_schedule=2)
        Xo, fo, tro, Fo = orc.hwsda_run(cfg, k1, k2, lockstep=trace, want_trace=True, want_F=True)
        assert np.array_equal(Fg, Fo), (N, np.nonzero(Fg != Fo))
        assert np.array_equal(X, Xo)
        assert lockstep_errors(trace, tro, N).max() < 2 * TOL_D
        assert Fg[0] == np.float32(0.1) and np.all((Fg >= 0.01) & (Fg <= 0.1))


KAP3 = [(2 * math.pi / 6.5, 2 * math.pi / 1.4), (2 * math.pi / 6.9, 2 * math.pi / 1.55),
        (2 * math.pi / 7.4, 2 * math.pi / 1.7)]
KAP5 = [(2 * math.pi / x, 0.0) for x in (2.1, 2.6, 3.2, 3.7, 4.4)]


@pytest.mark.parametrize("kind,N,NP,G,kap,G0,beta,modes,team,fs", [
    (1, 333, 24, 12, [(2 * math.pi / 6.9, 0.0)], 0.0, 0.0, (0, 1, 2, 3), 0, 0),
    (2, 3000, 32, 6, KAP3, 2.0e5, 0.5, (0, 1), 0, 0),
    (3, 3000, 32, 6, KAP5, 1.5e3, 0.5, (0, 1), 0, 0),
    # other team widths: more groups of 4 domains per thread (128), a team wider than
    # the rows need (512, N = 1001: padding domains), one CTA per individual of 64
    (2, 2999, 20, 4, KAP3[:2], 2.0e5, 0.5, (0,), 128, 0),
    (2, 1001, 12, 4, KAP3, 5.0e4, 0.5, (0,), 512, 0),
    (3, 3001, 20, 4, KAP5[:4], 1.5e3, 0.25, (0,), 64, 0),
    # four problems of 4096 padded domains: their tables (256 KB) do not fit shared
    # memory, so the one-team kernels read them through L1
    (2, 4000, 16, 3, KAP3 + [(2 * math.pi / 7.1, 2 * math.pi / 1.5)], 2.0e5, 0.5, (0, 1), 0, 0),
    # five SHG problems of 4096 padded domains in 512-thread teams: tables, staging and
    # scratch need exactly the opt-in limit, so the kernels' own static shared memory
    # sends them to the one-team kernels
    (3, 3000, 8, 3, KAP5, 1.5e3, 0.5, (0,), 512, 0),
    # one-warp teams, 16 to a CTA (no named barrier)
    (2, 1500, 40, 4, KAP3[:2], 1.0e5, 0.5, (0,), 32, 0),
    # the adaptive F of Sec. 3.1.1 on a minimised objective (teams share a CTA)
    (3, 2000, 40, 8, KAP5[:3], 1.0e3, 0.5, (0, 1), 64, 2),
])
def test_objective_lockstep(q, orc, kind, N, NP, G, kap, G0, beta, modes, team, fs):
    """The optimiser on the other objectives of the paper's designs: the SHG field
    (maximised), the multi-wavelength THG objective of Sec. 5 over three (kappa1,
    kappa2) pairs at N = 3000 and the multi-wavelength SHG objective over five (the
    paper's 9 mm / 3 um SHG designs have N = 3000 and five wavelengths), minimised.
    Populations bit for bit against the oracle's lockstep replay; every FP32 objective
    within tolerance of the oracle's FP64 one; the best individual's FP64 field
    re-check against the quadrature."""
    import torch
    k1, k2 = kap[0]
    for mode in modes:
        prm = q.Params(NP, G, 0.5, 0.9, 6, 0, 0, 32 if mode == 3 else team, fs)
        st = q.State([(N, k1, k2)], [prm])
        st.set_objective(kind, kap if kind >= 2 else (), G0, beta)
        tr = torch.full((NP * (1 + 2 * G),), float("nan"), dtype=torch.float32, device="cuda")
        q.qpm_set_trace(st.h, 0, tr)
        st.init()
        st.run(G, mode)
        X, f, D = snapshot(st)
        x, d64, fb, idx = st.best()
        torch.cuda.synchronize()
        trace = tr.cpu().numpy()
        st.close()
        cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 6, obj=kind, kappas=kap if kind >= 2 else (),
                           G0=G0, beta=beta, f_schedule=fs)
        Xo, fo, tro = orc.hwsda_run(cfg, k1, k2, lockstep=trace, want_trace=True)
        assert np.array_equal(X, Xo), mode
        ok = ~np.isnan(trace)
        if kind == 1:  # |E|^2: relative, floor at 1e-3 of the all-up |E|^2 = N^2
            err = np.abs(trace[ok] - tro[ok]) / np.maximum(tro[ok], 1e-6 * N * N)
            assert err.max() < 2 * TOL_D
        else:  # each |G0 - G_k| carries G_k's error: scale K G0
            assert np.max(np.abs(trace[ok] - tro[ok])) <= TOL_D * len(kap) * G0
        i = int(idx.cpu().item())
        assert i == (int(np.argmin(f)) if kind >= 2 else int(np.argmax(f)))
        xi = X[i][None]
        ref = orc.shg_genes(xi, k1)[0] if kind in (1, 3) else orc.deff_genes(xi, k1, k2)[0]
        z = complex(*d64.cpu().numpy())
        assert abs(z - ref) <= 1e-9 * abs(ref)


@pytest.mark.parametrize("mode", [0, 1])
def test_objectives_of_several_instances_lockstep(q, orc, mode):
    """A state of two instances with different multi-wavelength objectives (three
    cascaded problems, four SHG problems), one-warp teams 16 to a CTA: each instance
    bit for bit against the oracle's lockstep replay with its own instance index."""
    import torch
    inst = [(2000, KAP3, 16, 2, 1.0e5), (1500, KAP5[:4], 12, 3, 1.0e3)]
    G = 4
    probs = [(N, kap[0][0], kap[0][1]) for N, kap, NP, kind, G0 in inst]
    prms = [q.Params(NP, G, 0.5, 0.9, 13, 0, 0) for N, kap, NP, kind, G0 in inst]
    st = q.State(probs, prms)
    traces = []
    for k, (N, kap, NP, kind, G0) in enumerate(inst):
        st.set_objective(kind, kap, G0, 0.5, inst=k)
        tr = torch.full((NP * (1 + 2 * G),), float("nan"), dtype=torch.float32, device="cuda")
        q.qpm_set_trace(st.h, k, tr)
        traces.append(tr)
    st.init()
    st.run(G, mode)
    torch.cuda.synchronize()
    for k, (N, kap, NP, kind, G0) in enumerate(inst):
        X = st.population(k)[0].cpu().numpy()
        trace = traces[k].cpu().numpy()
        cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 13, inst=k, obj=kind, kappas=kap, G0=G0, beta=0.5)
        Xo, fo, tro = orc.hwsda_run(cfg, kap[0][0], kap[0][1], lockstep=trace, want_trace=True)
        assert np.array_equal(X, Xo), k
        ok = ~np.isnan(trace)
        assert np.max(np.abs(trace[ok] - tro[ok])) <= TOL_D * len(kap) * G0, k
    st.close()


@pytest.mark.parametrize("kind,kap", [(2, KAP3[:2]), (3, KAP5)])
def test_checkpoint_resume_multi_objective(q, kind, kap):
    """Checkpoint and resume of a multi-wavelength design (the multi-team kernels with
    shared-memory tables): the population re-evaluated by qpm_set_population has the
    same objective bits, and the resumed run ends exactly like the uninterrupted one."""
    import torch
    N, NP, G = 3000, 24, 10

    def make():
        st = q.State([(N, kap[0][0], kap[0][1])], [q.Params(NP, G, 0.5, 0.9, 9, 0, 0, 0)])
        st.set_objective(kind, kap, 1.0e5 if kind == 2 else 1.0e3, 0.5)
        st.init()
        return st

    st = make()
    st.run(G, 0)
    Xa, fa, _ = snapshot(st)
    st.close()
    st = make()
    st.run(5, 0)
    Xc, fc, _ = st.population()
    torch.cuda.synchronize()
    st.close()
    st2 = make()
    q.qpm_set_population(st2.h, 0, Xc, 5)
    X2, f2, _ = snapshot(st2)
    assert np.array_equal(f2, fc.cpu().numpy())
    st2.run(G - 5, 0)
    Xb, fb, _ = snapshot(st2)
    st2.close()
    assert np.array_equal(Xa, Xb) and np.array_equal(fa, fb)


def test_objective_states_of_different_sizes_take_turns(q):
    """Two multi-wavelength states whose shared-memory tables differ in size (147 KB and
    16 KB) set up one after the other and run in turns: the larger one's launches still
    fit, and each state's populations equal those of a run of that state alone."""
    import torch

    def make(N, kap):
        st = q.State([(N, kap[0][0], kap[0][1])], [q.Params(24, 6, 0.5, 0.9, 3, 0, 0, 0)])
        st.set_objective(2, kap, 1.0e5, 0.5)
        st.init()
        return st

    alone = {}
    for N, kap in ((3000, KAP3), (1000, KAP3[:1])):
        st = make(N, kap)
        st.run(6, 0)
        alone[N] = st.population()[0].cpu().numpy()
        st.close()
    big, small = make(3000, KAP3), make(1000, KAP3[:1])
    for _ in range(3):
        big.run(2, 0)
        small.run(2, 0)
    torch.cuda.synchronize()
    assert np.array_equal(big.population()[0].cpu().numpy(), alone[3000])
    assert np.array_equal(small.population()[0].cpu().numpy(), alone[1000])
    big.close()
    small.close()


def test_objective_errors(q):
    import torch
    st = q.State([(100, 1.0, 2.0)], [q.Params(8, 4, 0.5, 0.9, 1, 0, 0)])
    with pytest.raises(q.QpmError) as e:
        st.set_objective(2, [(1.0, 2.0)] * 5, 10.0, 0.5)
    assert e.value.status == 1
    with pytest.raises(q.QpmError) as e:
        st.set_objective(3, [(1.0, 0.0)], 10.0, -1.0)
    assert e.value.status == 1
    st.set_objective(2, [(1.0, 2.0), (1.5, 2.5)], 10.0, 0.5)
    st.init()
    with pytest.raises(q.QpmError) as e:
        st.set_objective(0)
    assert e.value.status == 5
    for mode in (2, 3):
        with pytest.raises(q.QpmError) as e:
            st.run(1, mode)
        assert e.value.status == 4
    with pytest.raises(q.QpmError) as e:
        q.qpm_polish_leaders(st.h, 0)
    assert e.value.status == 4
    st.run(2, q.RUN_GRAPH)
    torch.cuda.synchronize()
    st.close()


@pytest.mark.parametrize("comp", [0, 1])
def test_discrete_gwo_lockstep(q, orc, comp):
    """The four-leader discrete GWO of Sec. 3.1.2 (gwo_combine 2) follows the oracle bit
    for bit in the launches and graph forms (short rows read both slots, long rows
    stage them); the forms that do not support it say so."""
    import torch
    for N, NP, G in ((333, 24, 12), (5000, 20, 4)):
        k1, k2 = 2 * math.pi / 7.3, 2 * math.pi / 1.4
        for mode in (0, 1):
            st, tr = make(q, N, k1, k2, NP, G, seed=12, combine=2, comp=comp)
            st.init()
            st.run(G, mode)
            X, f, D = snapshot(st)
            trace = tr.cpu().numpy()
            st.close()
            cfg = orc.make_cfg(NP, N, G, 0.5, 0.9, 12, 0, 2)
            Xo, fo, tro = orc.hwsda_run(cfg, k1, k2, lockstep=trace, want_trace=True)
            assert np.array_equal(X, Xo), (N, mode)
            assert lockstep_errors(trace, tro, N).max() < 2 * TOL_D
            # four leaders per generation: four NaN entries in every candidate trace
            cand = trace[NP:].reshape(G, 2, NP)[:, 1]
            assert np.all(np.isnan(cand).sum(axis=1) == 4)
    st, _ = make(q, 100, 1.0, 2.0, 8, 4, combine=2, trace=False)
    st.init()
    with pytest.raises(q.QpmError) as e:
        st.run(1, q.RUN_PERSISTENT)
    assert e.value.status == 4
    st.close()


@pytest.mark.parametrize("mode", [0, 2])
def test_checkpoint_resume_with_adaptive_F(q, mode):
    """With the adaptive F the checkpoint also carries the F history (qpm_get_F); a fresh
    state given the population (qpm_set_population) and the history (qpm_set_F) at
    generation 15 continues exactly like the uninterrupted 30-generation run."""
    import torch
    N, NP, G = 700, 40, 30
    k1, k2 = 2 * math.pi / 6.9, 2 * math.pi / 1.55
    st, _ = make(q, N, k1, k2, NP, G, seed=22, comp=1, trace=False, f_schedule=2)
    st.init()
    st.run(G, mode)
    Xa, fa, _ = snapshot(st)
    Fa = q.qpm_get_F(st.h, 0).cpu().numpy()
    st.close()
    st, _ = make(q, N, k1, k2, NP, G, seed=22, comp=1, trace=False, f_schedule=2)
    st.init()
    st.run(15, mode)
    Xc, _, _ = st.population()
    Fc = q.qpm_get_F(st.h, 0).clone()
    torch.cuda.synchronize()
    st.close()
    st2, _ = make(q, N, k1, k2, NP, G, seed=22, comp=1, trace=False, f_schedule=2)
    st2.init()
    q.qpm_set_population(st2.h, 0, Xc, 15)
    q.qpm_set_F(st2.h, 0, Fc)
    st2.run(G - 15, mode)
    Xb, fb, _ = snapshot(st2)
    Fb = q.qpm_get_F(st2.h, 0).cpu().numpy()
    st2.close()
    assert np.array_equal(Xa, Xb) and np.array_equal(fa, fb) and np.array_equal(Fa, Fb)


def test_free_run_against_the_oracle(q, orc):
    """Free runs (no lockstep) of the 16-domain workload: the GPU decides in FP32, the
    oracle in FP64.  Both start from the same population; the first generation after
    which they differ is reported (a near-tie decided differently), and until then
    they agree bit for bit.  Both final bests are valid designs no better than the
    exhaustive optimum."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    c = W.SMALL
    prm = q.Params(c["NP"], c["G"], c["F"], c["CR"], c["seed"], 0, c["compensated"])
    cfg = orc.make_cfg(c["NP"], c["N"], c["G"], c["F"], c["CR"], c["seed"])
    with q.State([(c["N"], c["kappa1"], c["kappa2"])], [prm]) as st:
        st.init()
        pops = [st.population()[0].cpu().numpy()]
        for _ in range(c["G"]):
            st.step()
            pops.append(st.population()[0].cpu().numpy())
    X = orc.init_population(cfg)
    assert np.array_equal(X, pops[0])
    f64 = orc.objective_rows(cfg, X, c["kappa1"], c["kappa2"])
    fdec = f64.astype(np.float32)
    first = None
    for g in range(c["G"]):
        X, fdec, f64, _, _, _ = orc.hwsda_generation(cfg, c["kappa1"], c["kappa2"], g, X, fdec, f64)
        if first is None and not np.array_equal(X, pops[g + 1]):
            first = g
    best, _ = orc.bruteforce(c["N"], c["kappa1"], c["kappa2"])
    f_gpu = orc.objective_rows(cfg, pops[-1], c["kappa1"], c["kappa2"]).max()
    print(f"free run: first divergence at generation {first}; final best GPU {f_gpu:.6g}, "
          f"oracle {f64.max():.6g}, optimum {best:.6g}")
    assert f_gpu <= best * (1 + 1e-12) and f64.max() <= best * (1 + 1e-12)
