"""Benchmark: HWSDA design runs of the cascaded-THG QPM problem on one GB300.

One step = one whole HWSDA run of the paper-scale workload (N = 1000 domains,
kappa1 = 2pi/6.9, kappa2 = 2pi/1.55, NP = 256, G = 2000 generations, F = 0.5,
CR = 0.9, Kahan-compensated FP32 scan): phasor table, initial population and
its fitness, then 2000 generations of DE + GWO with greedy selection.  The
population (1 MB) lives in HBM/L2 throughout; L2 is flushed between timed steps
(a 256 MB write, then a 256 MB read of another buffer, so that no dirty line of the
flush is written back inside the timed region).

Metric: domain-evals/s = (NP + G * (2 NP - 3)) * N / step time (every fitness
evaluation scans N domains; a generation evaluates NP trials and NP - 3 GWO
candidates), plus HWSDA generations/s, for the plain form (two kernels per
generation, captured once into a CUDA graph) and the persistent form (one
cooperative kernel for all generations).  `value` is the faster form.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "domain-evals/s and HWSDA gen/s at N=1000,NP=256 vs roofline; batched vs plain"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def dist_env():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []     # (arrival time, line)
        self.t_mark = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self):
        """Start of the timed region: samples that arrive earlier are dropped."""
        self.t_mark = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in self.lines:
            if self.t_mark is not None and t < self.t_mark:
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- GPU arm
# DRAM bytes (read + write) of one k_persist launch of the 1000-domain workload
# (2000 generations), captured with
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none \
#       -k regex:k_persist -c 1 python -m paper_2511_01255_gb300.profile_run \
#       --workload paper --form persistent --gens 2000 --reps 1
# on the current kernel: 1501696 read + 329984 written.  The 2 MB population and
# the phasor table stay in L2; DRAM sees little more than the first touch.
K_PERSIST_DRAM_BYTES = 1501696 + 329984
# DRAM bytes of one relaxed forward (k_relaxed_fwd + k_relaxed_combine) and one backward
# at 4096 x 4096, read + write, from the ncu capture in profiles/k_relaxed_b4096_n4096.md
# (cold caches; the backward's last gradient lines are still in L2 when it ends)
K_RELAXED_DRAM_BYTES = (67191040 + 679424) + (4265984 + 0) + (71792896 + 14891776)


PHILOX_CALLS_PER_GENE_GEN = 0.25 + 0.75  # crossover word + three GWO words, 4 genes per call

# The packed-sign sweep appends a block of 4 domains per lookup in the sign-block
# table: per block 2 ops to take its 4 bits from the word, 3 to fold the pattern onto
# the 8 stored ones, 3 shared-memory loads of (A, B, C), 4 sign flips and the 10 of
# one monoid combination -> 22 issue slots per 4 domain-evals.  This is the
# implementation's own count.
PACKED_OPS_PER_DOMAIN = 22 / 4
# The method's count for one domain of a direct scan (no table): the complex
# multiply-add of a B into C (4 FFMA), A += a (2), B += b (2 FFMA), a = d p2 (2) ->
# 10 FP32 lane-ops; in FP32 flops (an FFMA counts 2) 6 FFMA + 4 others = 16 - 4 = 12.
DIRECT_SCAN_OPS_PER_DOMAIN = 10
DIRECT_SCAN_FLOPS_PER_DOMAIN = 12


def algorithmic_lane_ops_per_gene_gen(compensated):
    """Lane instructions the method needs per gene and generation: Philox4x32-10 at
    1.0 calls (80 ops each: a quarter for the crossover word, three quarters for
    the three GWO words, each giving one leader's r1 and r2); the GWO's r1 and 2 r2
    of three leaders (3 ops each: shift, mask-or into a significand, exact
    subtraction); the crossover test (1 integer compare); DE update (7: difference,
    product, sum, clamp 2, jrand compare, select); GWO update (28: per leader A in
    2, |C Xp - x| in 3, Xp - A D in 2; then two adds, the division by 3 in 3, clamp
    2); two fitness domain-evals (10 plain; 14.25 with Kahan compensation folded in
    every 8 domains)."""
    return (PHILOX_CALLS_PER_GENE_GEN * 80 + 6 * 3 + 1 + 7 + 28
            + 2 * (14.25 if compensated else 10))


def algorithmic_lane_ops_per_gene_gen_multi(kind, K):
    """The same count for the multi-wavelength objectives of Sec. 5 (plain scans): the
    updates as above, and per phase one scan of each of the K problems, 10 lane-ops a
    domain for a cascaded problem, 2 for an SHG problem (the running sum of d p1 as two
    FFMA)."""
    per_domain = DIRECT_SCAN_OPS_PER_DOMAIN if kind == 2 else 2
    return (algorithmic_lane_ops_per_gene_gen(0) - 2 * DIRECT_SCAN_OPS_PER_DOMAIN
            + 2 * K * per_domain)


def mix_ceiling_gene_gens(compensated, issue):
    """Gene-generations/s the work of a gene-generation allows on this GPU when every
    issue slot does useful work: the Philox4x32-10 calls at the measured rate of the
    library's own generator, the rest of the algorithmic lane-ops at the measured
    FFMA rate (they share the issue slots, so the times add)."""
    n_rest = algorithmic_lane_ops_per_gene_gen(compensated) - PHILOX_CALLS_PER_GENE_GEN * 80
    t = PHILOX_CALLS_PER_GENE_GEN / issue["philox_calls_per_s"] + n_rest / (issue["ffma"] * 1e12)
    return 1.0 / t


def phase_bound_s_per_gen(N, NP, compensated, issue, hbm_gbs):
    """Lower bound of one generation's time when each of the two phases runs at its
    own roofline, for populations far larger than L2: DE reads the target and three
    random donors and writes the trial (20 B of HBM per gene), GWO reads the target
    and writes the candidate (8 B per gene; the three leaders' rows stay in L2).
    Each phase takes the larger of its HBM time and its issue time (its Philox calls
    at the measured call rate, its other lane-ops at the FFMA rate); the grid
    barrier between the phases keeps them from overlapping."""
    ev = 14.25 if compensated else 10
    genes = N * NP
    de_issue = genes * (0.25 / issue["philox_calls_per_s"] + (1 + 7 + ev) / (issue["ffma"] * 1e12))
    gwo_issue = genes * (0.75 / issue["philox_calls_per_s"] + (6 * 3 + 28 + ev) / (issue["ffma"] * 1e12))
    de_hbm = 20.0 * genes / (hbm_gbs * 1e9)
    gwo_hbm = 8.0 * genes / (hbm_gbs * 1e9)
    return max(de_issue, de_hbm) + max(gwo_issue, gwo_hbm)


L2_NOTE = ("flushed between timed steps (256 MB written, then another 256 MB read, so L2 "
           "starts cold and clean)")


def workload_config(c, world):
    """The workload the metric is quoted on, identical in both arms' JSON lines."""
    return {"workload": c["name"], "N": c["N"], "NP": c["NP"], "G": c["G"],
            "kappa1": c["kappa1"], "kappa2": c["kappa2"], "F": c["F"], "CR": c["CR"],
            "compensated": bool(c["compensated"]), "l2": L2_NOTE,
            "parallelism": f"replicas{world}"}


def cpu_model():
    """The host CPU's model name (x86: /proc/cpuinfo; Arm: lscpu)."""
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def max_over_ranks(seconds, world, device=None):
    """Slowest rank's step time (the job's time); identity for one process."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds_max, world):
    """Whole-job throughput of independent replicas (weak scaling)."""
    return world * units_per_rank / seconds_max


class L2Flush:
    """Flush of the 129 MB L2 before a timed region: write a 256 MB buffer, then read
    another 256 MB buffer, so that the timed region starts with L2 holding neither
    the timed kernel's data nor dirty lines (whose write-back would otherwise land in
    the timed region and steal its DRAM bandwidth)."""

    def __init__(self, mb=256):
        import torch
        n = mb * 1024 * 1024 // 4
        self.w = torch.empty(n, dtype=torch.float32, device="cuda")
        self.r = torch.zeros(n, dtype=torch.float32, device="cuda")

    def __call__(self):
        self.w.fill_(1.0)
        self.r.sum()


def sample_best_rows(q, st, inst, prob, k, minimize=False):
    """The k fittest individuals of instance `inst` as left in the state: genes, the
    FP32 field and the objective the optimiser selected on, for the oracle to
    re-evaluate (outside any timed region)."""
    import numpy as np
    X, f, D = st.population(inst)
    fh = f.cpu().numpy()
    idx = np.argsort(fh if minimize else -fh, kind="stable")[:k]
    Xs = X[idx.tolist()].cpu().numpy()
    Ds = D[idx.tolist()].cpu().numpy()
    N, k1, k2 = prob
    return [{"N": int(N), "kappa1": float(k1), "kappa2": float(k2), "genes": Xs[j],
             "D": complex(Ds[j, 0], Ds[j, 1]), "objective": float(fh[idx[j]])}
            for j in range(len(idx))]


def _time_cuda(fn, reps, flush=None):
    """Mean seconds per call of fn() with CUDA events on the current stream."""
    import torch
    st = torch.cuda.current_stream()
    tot = 0.0
    for _ in range(reps):
        if flush is not None:
            flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        tot += e0.elapsed_time(e1) / 1e3
    return tot / reps


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2511_01255_gb300 as q
    from paper_2511_01255_gb300 import workloads as W

    rank, world, lrank = dist_env()
    torch.cuda.set_device(lrank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    q.lib()
    pk, pk_src = peaks()
    nsm = torch.cuda.get_device_properties(lrank).multi_processor_count
    peak_alu = nsm * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # T lane-ops/s
    # measured issue rates of this GPU (the library's microbenchmark), T lane-ops/s
    issue = {name: q.qpm_measure_issue_peak(k) / 1e12
             for k, name in enumerate(("ffma", "philox_mul_xor", "lop3"))}
    issue["philox_calls_per_s"] = q.qpm_measure_issue_peak(3)
    peak_hbm = pk.get("hbm_gbs", 6800.0)
    c = W.PAPER_SCALE
    N, NP, G = c["N"], c["NP"], c["G"]
    # independent replicas: each rank designs its own crystal (seed = 1 + rank)
    prm = q.Params(NP, G, c["F"], c["CR"], c["seed"] + rank, 0, c["compensated"])
    prob = (N, c["kappa1"], c["kappa2"])
    evals_per_run = (NP + G * (2 * NP - 3)) * N
    gene_gens = NP * N * G
    flush = L2Flush()
    stream = torch.cuda.current_stream()
    samples = {}  # rows the oracle re-evaluates in the CPU-baseline leg (error_vs_oracle)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------------------------------------------------- headline workload
    results = {}
    for mode_name, mode in (("persistent", q.RUN_PERSISTENT), ("plain_graph", q.RUN_GRAPH)):
        st = q.State([prob], [prm])
        sampler = ClockSampler(lrank)
        sampler.start()  # running before the timed region begins
        for _ in range(args.warmup):
            st.init()
            st.run(G, mode)
        torch.cuda.synchronize()
        times = []
        barrier()
        sampler.mark()
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st.init()
            st.run(G, mode)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        barrier()
        wall = time.perf_counter() - wall0
        clocks = sampler.stop()
        x, d64, fb, idx = st.best()
        torch.cuda.synchronize()
        best_f = float(fb.cpu())
        st.close()
        t = max_over_ranks(sum(times) / len(times), world, device="cuda")
        results[mode_name] = dict(s_per_step=t, wall=wall, clocks=clocks, best_f=best_f,
                                  launches_per_step=(3 + (2 * G if mode == q.RUN_GRAPH else 1)))

    # dominant kernel: the persistent generation kernel alone, on its stream
    st = q.State([prob], [prm])
    dur = []
    for _ in range(max(3, args.steps)):
        st.init()
        dur.append(_time_cuda(lambda: st.run(G, q.RUN_PERSISTENT), 1, flush))
    samples["headline"] = sample_best_rows(q, st, 0, prob, 3)
    grid_persist = min(NP, 2 * nsm)  # one 256-thread CTA per individual, two per SM
    st.close()
    # latency floor of one generation: two grid barriers, three dependent L2 round
    # trips (donor rows, survivor keys, leader rows) and the generation's issue time
    bar_ns = q.qpm_measure_latency(0, grid_persist)
    l2_ns = q.qpm_measure_latency(1)
    # the alternatives to the counter barrier, on the same grid
    sync_alt_ns = {"relaxed_counter_barrier_ns": q.qpm_measure_latency(2, grid_persist),
                   "fence_only_ns": q.qpm_measure_latency(3, grid_persist),
                   "tagged_word_exchange_ns": q.qpm_measure_latency(4, grid_persist)}
    kdur = statistics.median(dur)
    ops_gene_gen = algorithmic_lane_ops_per_gene_gen(c["compensated"])
    achieved = ops_gene_gen * gene_gens / kdur / 1e12
    issue_us = ops_gene_gen * NP * N / (peak_alu * 1e12) * 1e6
    floor_us = 2 * bar_ns / 1e3 + 3 * l2_ns / 1e3 + issue_us
    best_mode = min(results, key=lambda k: results[k]["s_per_step"])

    # ------------------------------------------------ batched: 512 instances
    inst = W.batched_instances(512)
    probs_b = [(ci["N"], ci["kappa1"], ci["kappa2"]) for ci in inst]
    prms_b = [q.Params(ci["NP"], ci["G"], ci["F"], ci["CR"], ci["seed"] + rank, 0, ci["compensated"])
              for ci in inst]
    Gb = inst[0]["G"]
    gg_b = sum(ci["NP"] * ci["N"] for ci in inst) * Gb
    ev_b = sum((2 * ci["NP"] - 3) * ci["N"] for ci in inst) * Gb + sum(ci["NP"] * ci["N"] for ci in inst)
    stb = q.State(probs_b, prms_b)
    stb.init()
    from paper_2511_01255_gb300 import autotune
    ctas = autotune.autotune_batch_cluster(stb, gens=10)  # CTAs per cluster, measured (cached)
    stb.run(3, q.RUN_BATCHED)  # warm-up (graph instantiation, caches)
    tb = []
    for _ in range(min(2, args.steps)):
        def one():
            stb.init()
            stb.run(Gb, q.RUN_BATCHED)
        tb.append(_time_cuda(one, 1, flush))
    t_batched = min(tb)
    samples["batched"] = []
    for inst_k in (0, 1, 2, 3):
        samples["batched"] += sample_best_rows(q, stb, inst_k, probs_b[inst_k], 1)
    # the same batch in the per-instance persistent form, timed over 3 generations
    stb.init()
    stb.run(1, q.RUN_PERSISTENT)
    t_inst3 = _time_cuda(lambda: stb.run(3, q.RUN_PERSISTENT), 1, flush)
    stb.close()
    batched = {
        "workload": "512 instances, N~U[500,8000], NP in {64,128,256,512}, G=1000, plain FP32 scan",
        "cluster_ctas": ctas,
        "s_per_run": t_batched, "domain_evals_per_s": ev_b / t_batched,
        "gene_gens_per_s": gg_b / t_batched,
        "per_instance_persistent_s_per_gen": t_inst3 / 3,
        "speedup_vs_per_instance_persistent_extrapolated": (t_inst3 / 3 * Gb) / t_batched,
        "speedup_note": "the per-instance persistent form timed over 3 generations of all 512 "
                        "instances and scaled to 1000 generations",
        "roofline": {"bound": "alu", "achieved": algorithmic_lane_ops_per_gene_gen(0) * gg_b / t_batched / 1e12,
                     "peak": peak_alu, "unit": "T lane-ops/s",
                     "frac": algorithmic_lane_ops_per_gene_gen(0) * gg_b / t_batched / 1e12 / peak_alu,
                     "frac_of_mix_ceiling": gg_b / t_batched / mix_ceiling_gene_gens(0, issue)},
    }

    # --------------------------------------- precision: N = 1e5, NP = 1024, G = 500
    cp = W.PRECISION
    prec = {}
    for comp in (1, 0):
        pr = q.Params(cp["NP"], cp["G"], cp["F"], cp["CR"], cp["seed"] + rank, 0, comp)
        stp = q.State([(cp["N"], cp["kappa1"], cp["kappa2"])], [pr])
        stp.init()
        stp.run(2, q.RUN_PERSISTENT)
        stp.init()
        tp = _time_cuda(lambda: stp.run(cp["G"], q.RUN_PERSISTENT), 1, None)
        samples["precision." + ("compensated" if comp else "plain")] = sample_best_rows(
            q, stp, 0, (cp["N"], cp["kappa1"], cp["kappa2"]), 2)
        stp.close()
        ggp = cp["NP"] * cp["N"] * cp["G"]
        prec["compensated" if comp else "plain"] = {
            "s_per_run": tp, "gene_gens_per_s": ggp / tp,
            "domain_evals_per_s": (2 * cp["NP"] - 3) * cp["N"] * cp["G"] / tp,
            "alu_frac": algorithmic_lane_ops_per_gene_gen(comp) * ggp / tp / 1e12 / peak_alu,
            "frac_of_mix_ceiling": ggp / tp / mix_ceiling_gene_gens(comp, issue),
            "phase_bound_us_per_gen": 1e6 * phase_bound_s_per_gen(cp["N"], cp["NP"], comp, issue,
                                                                  peak_hbm),
            "frac_of_phase_bound": phase_bound_s_per_gen(cp["N"], cp["NP"], comp, issue, peak_hbm)
                                   * cp["G"] / tp}
    prec["workload"] = cp["name"]

    # ---------------------------------- adjoint: B = 4096 rows of N = 4096, fwd + bwd
    cr = W.RELAXED
    th = torch.from_numpy(W.relaxed_theta(cr["B"], cr["N"], seed=cr["seed"])).cuda()
    Dr = torch.empty((cr["B"], 2), device="cuda")
    Ar = q.relaxed_saved(cr["B"], cr["N"])
    fr = torch.empty(cr["B"], device="cuda")
    gr = torch.empty_like(th)

    def fwd():
        q.qpm_deff_relaxed_fwd(cr["N"], cr["kappa1"], cr["kappa2"], th, Dr, fr, Ar)

    def bwd():
        q.qpm_deff_relaxed_bwd(cr["N"], cr["kappa1"], cr["kappa2"], th, Dr, Ar, None, gr)

    # row 0: a relaxed two-tone design (d = +-tanh 3), whose |d_eff| is a sizeable
    # fraction of L^2/2, so its error can be stated strictly relative
    th[0] = torch.from_numpy(3.0 * W.two_tone_signs(cr["N"], cr["kappa1"], cr["kappa2"])).cuda()
    for _ in range(3):
        fwd()
        bwd()
    t_f = _time_cuda(fwd, 10, flush)
    t_b = _time_cuda(bwd, 10, flush)
    fwd()
    bwd()
    cols = np.linspace(0, cr["N"] - 1, 16).astype(np.int64)
    samples["adjoint"] = {"N": cr["N"], "kappa1": cr["kappa1"], "kappa2": cr["kappa2"],
                          "theta": th[0].cpu().numpy(), "D": complex(*Dr[0].cpu().numpy()),
                          "cols": cols, "grad": gr[0, cols.tolist()].cpu().numpy()}
    elems = cr["B"] * cr["N"]
    adjoint = {"workload": cr["name"], "fwd_us": t_f * 1e6, "bwd_us": t_b * 1e6,
               "elements_per_s": elems / (t_f + t_b),
               "roofline": {"bound": "hbm", "achieved": 12 * elems / (t_f + t_b) / 1e9,
                            "peak": peak_hbm, "unit": "GB/s",
                            "frac": 12 * elems / (t_f + t_b) / 1e9 / peak_hbm,
                            "bytes_per_element": 12, "traffic": K_RELAXED_DRAM_BYTES,
                            "traffic_unit": "DRAM bytes of one fwd + combine + bwd (ncu)"}}

    # ------------------------------ qpm_eval: 1024 rows of N = 1e5 (genes, packed)
    Ne, NPe = 100000, 1024
    Xe = torch.rand((NPe, Ne), device="cuda") * 2 - 1
    We = torch.randint(-2 ** 31, 2 ** 31 - 1, (NPe, (Ne + 31) // 32), dtype=torch.int32, device="cuda")
    # row 0 a two-tone design (|d_eff| ~ 0.07 L^2/2), the others random (|d_eff| ~ N)
    tt = W.two_tone_signs(Ne, 1.0, 2.0)
    Xe[0] = torch.from_numpy(tt).cuda()
    We[0] = torch.from_numpy(W.pack_signs(tt[None], Ne).view(np.int32)[0]).cuda()
    De = torch.empty((NPe, 2), device="cuda")
    q.qpm_eval(Ne, 1.0, 2.0, Xe, De)
    q.qpm_eval_packed(Ne, 1.0, 2.0, We, De)
    t_g = _time_cuda(lambda: q.qpm_eval(Ne, 1.0, 2.0, Xe, De), 10, flush)
    t_p = _time_cuda(lambda: q.qpm_eval_packed(Ne, 1.0, 2.0, We, De), 10, flush)
    ev = NPe * Ne
    rows_e = [0, 1, 511, 1023]
    q.qpm_eval(Ne, 1.0, 2.0, Xe, De)
    samples["eval.genes"] = [{"N": Ne, "kappa1": 1.0, "kappa2": 2.0, "genes": Xe[r].cpu().numpy(),
                              "D": complex(*De[r].cpu().numpy())} for r in rows_e]
    q.qpm_eval_packed(Ne, 1.0, 2.0, We, De)
    samples["eval.packed"] = [{"N": Ne, "kappa1": 1.0, "kappa2": 2.0,
                               "words": We[r].cpu().numpy().view(np.uint32),
                               "D": complex(*De[r].cpu().numpy())} for r in rows_e]
    evaluate = {"workload": "1024 rows x 1e5 domains, plain scan",
                "genes": {"domain_evals_per_s": ev / t_g, "us": t_g * 1e6,
                          "roofline": {"bound": "hbm", "achieved": 4 * ev / t_g / 1e9, "peak": peak_hbm,
                                       "unit": "GB/s", "frac": 4 * ev / t_g / 1e9 / peak_hbm}},
                "packed": {"domain_evals_per_s": ev / t_p, "us": t_p * 1e6,
                           "roofline": {
                               "bound": "alu",
                               "achieved": DIRECT_SCAN_OPS_PER_DOMAIN * ev / t_p / 1e12,
                               "peak": peak_alu, "unit": "T lane-ops/s",
                               "ops_per_domain_eval": DIRECT_SCAN_OPS_PER_DOMAIN,
                               "frac": DIRECT_SCAN_OPS_PER_DOMAIN * ev / t_p / 1e12 / peak_alu,
                               "unit_note": "frac: the method's direct-scan work (10 FP32 "
                                            "lane-ops per domain-eval) at this rate, against the "
                                            "issue peak; the sign-block table does less work",
                               "frac_of_fp32_flops": DIRECT_SCAN_FLOPS_PER_DOMAIN * ev / t_p
                                                     / (2 * peak_alu * 1e12),
                               "fp32_flops_per_domain_eval": DIRECT_SCAN_FLOPS_PER_DOMAIN,
                               "frac_at_table_lookup_ops": PACKED_OPS_PER_DOMAIN * ev / t_p / 1e12
                                                           / peak_alu,
                               "table_lookup_ops_per_domain_eval": PACKED_OPS_PER_DOMAIN}}}
    del Xe, We

    # ------------------------------- the multi-wavelength designs of Sec. 5 (N = 3000)
    designs = {}
    from paper_2511_01255_gb300 import autotune
    for dc in (W.DESIGN_THG3, W.DESIGN_SHG5):
        k1d, k2d = dc["kappas"][0]
        obj_d = (dc["kind"], dc["kappas"], dc["G0"], dc["beta"])
        team_d = autotune.autotune_team(dc["N"], k1d, k2d, dc["NP"], 0, q.RUN_LAUNCHES, gens=4,
                                        objective=obj_d)  # measured, cached
        prm_d = q.Params(dc["NP"], dc["G"], dc["F"], dc["CR"], dc["seed"] + rank, 0, 0, team_d)
        std = q.State([(dc["N"], k1d, k2d)], [prm_d])
        std.set_objective(dc["kind"], dc["kappas"], dc["G0"], dc["beta"])
        std.init()
        std.run(2, q.RUN_LAUNCHES)  # warm-up: kernels loaded, tables built
        std.init()
        t_d = _time_cuda(lambda: std.run(dc["G"], q.RUN_LAUNCHES), 1, flush)
        K = len(dc["kappas"])
        ev_d = (2 * dc["NP"] - 3) * dc["N"] * dc["G"] * K
        rows = sample_best_rows(q, std, 0, (dc["N"], k1d, k2d), 1, minimize=True)
        rows[0]["cfg"] = dc
        samples["designs." + dc["name"]] = rows
        std.close()
        ops_d = algorithmic_lane_ops_per_gene_gen_multi(dc["kind"], K)
        gg_d = dc["NP"] * dc["N"] * dc["G"]  # gene-generations of the timed run
        designs[dc["name"]] = {
            "s_per_1000_iterations": t_d * 1000.0 / dc["G"],
            "domain_evals_per_s": ev_d / t_d,
            "domain_evals_note": "one domain of one problem's scan; K scans per evaluation",
            "best_objective": rows[0]["objective"], "form": "launches", "team": team_d,
            "roofline": {"bound": "alu", "achieved": ops_d * gg_d / t_d / 1e12,
                         "peak": peak_alu, "unit": "T lane-ops/s",
                         "frac": ops_d * gg_d / t_d / 1e12 / peak_alu,
                         "ops_per_gene_gen": ops_d},
            "paper_context": "about 21 s per 1000 iterations for the 5-wavelength SHG design at "
                             "N = 3000 on an RTX 4070 (Sec. 5); a different GPU and unknown NP, "
                             "context only"}

    # ------------- free run of the 16-domain workload: the population after every generation
    cs = W.SMALL
    prm_s = q.Params(cs["NP"], cs["G"], cs["F"], cs["CR"], cs["seed"], 0, cs["compensated"])
    sts = q.State([(cs["N"], cs["kappa1"], cs["kappa2"])], [prm_s])
    sts.init()
    pops = [sts.population()[0].cpu().numpy()]
    for _ in range(cs["G"]):
        sts.step()
        pops.append(sts.population()[0].cpu().numpy())
    sts.close()
    samples["free_run"] = pops

    # ---------------------------------------------- end to end through qpm_solve
    best_host = torch.empty(N, dtype=torch.float32).pin_memory()
    d64_host = torch.empty(2, dtype=torch.float64).pin_memory()
    f_host = torch.empty(1, dtype=torch.float32).pin_memory()
    mode_id = q.RUN_PERSISTENT if best_mode == "persistent" else q.RUN_GRAPH
    for _ in range(args.warmup):
        q.qpm_solve(N, c["kappa1"], c["kappa2"], prm, mode_id, best_host, d64_host, f_host)
    barrier()
    e2e = []
    for _ in range(args.steps):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q.qpm_solve(N, c["kappa1"], c["kappa2"], prm, mode_id, best_host, d64_host, f_host)
        e2e.append(time.perf_counter() - t0)
    e2e_t = sum(e2e) / len(e2e)

    if rank != 0:
        return
    best = results[best_mode]
    sm_mhz = best["clocks"].get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    value = job_throughput(evals_per_run, best["s_per_step"], world)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "domain-evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": best["s_per_step"] * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(c, world),
        "form": best_mode,
        "gen_per_s": world * G / best["s_per_step"],
        "forms": {k: {"ms_per_step": v["s_per_step"] * 1e3,
                      "domain_evals_per_s": world * evals_per_run / v["s_per_step"],
                      "gen_per_s": world * G / v["s_per_step"],
                      "best_f": v["best_f"]} for k, v in results.items()},
        "roofline": {"bound": "alu", "kernel": "k_persist",
                     "achieved": achieved, "peak": peak_alu, "unit": "T lane-ops/s",
                     "frac": achieved / peak_alu, "traffic": K_PERSIST_DRAM_BYTES,
                     "traffic_unit": "DRAM bytes per launch (2000 generations)",
                     "peak_note": f"{nsm} SMs x 128 lanes x {pk.get('sm_max_mhz', 2070.0)} MHz "
                                  f"(issue limit, derived; clocks {pk_src})",
                     "frac_at_median_clock": achieved / (nsm * 128 * sm_mhz * 1e6 / 1e12),
                     "frac_at_loaded_median_clock_of_peaks_file":
                         achieved / (nsm * 128 * pk.get("clocks_under_load", {}).get(
                             "sm_mhz_median", pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12),
                     "measured_issue_peaks": {k: v for k, v in issue.items()},
                     "frac_of_measured_ffma": achieved / issue["ffma"],
                     "frac_of_mix_ceiling": gene_gens / kdur / mix_ceiling_gene_gens(c["compensated"], issue),
                     "ops_per_gene_gen": ops_gene_gen, "launch_ms": kdur * 1e3,
                     "us_per_generation": kdur / G * 1e6,
                     "frac_of_latency_bound": floor_us / (kdur / G * 1e6),
                     "latency_floor": {
                         "us_per_generation": floor_us,
                         "grid_barrier_ns": bar_ns, "l2_load_ns": l2_ns, "issue_us": issue_us,
                         "grid_ctas": grid_persist,
                         "sync_alternatives": dict(sync_alt_ns, note=(
                             "per round on the same grid (qpm_measure_latency kinds 2-4): the "
                             "barrier without release/acquire, a lone gpu-scope fence, and a "
                             "counter-free exchange of tagged words that every CTA polls")),
                         "model": "2 grid barriers + 3 dependent L2 loads (donor rows, survivor "
                                  "keys, leader rows) + the generation's lane-ops at the issue "
                                  "peak; barrier and load latency measured by "
                                  "qpm_measure_latency in this run"}},
        "batched": batched,
        "precision": prec,
        "adjoint": adjoint,
        "eval": evaluate,
        "designs": designs,
        "e2e": {"value": world * evals_per_run / e2e_t, "unit": "domain-evals/s",
                "h2d_bytes_per_step": 24 + 40, "d2h_bytes_per_step": 4 * N + 16 + 4,
                "api": "qpm_solve (host buffers)", "form": best_mode},
        "gpu_launches": best["launches_per_step"] * args.steps,
        "clocks": best["clocks"],
    }
    if world == 1 and not args.no_cpu_baseline:
        # the CPU-baseline leg: the oracle timed on the host cores, and the oracle's
        # FP64 values of the rows sampled above (error of every sub-result)
        line["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_budget)
        line["cpu_baseline"]["closed_form_scan"] = cpu_closed_form()
        line["cpu_baseline"]["other_workloads"] = cpu_other_workloads()
        errs = oracle_errors(samples)
        line["error_vs_oracle"] = errs["headline"]
        line["batched"]["error_vs_oracle"] = errs["batched"]
        for k in ("compensated", "plain"):
            line["precision"][k]["error_vs_oracle"] = errs["precision." + k]
        line["eval"]["genes"]["error_vs_oracle"] = errs["eval.genes"]
        line["eval"]["packed"]["error_vs_oracle"] = errs["eval.packed"]
        line["adjoint"]["error_vs_oracle"] = errs["adjoint"]
        for name in designs:
            designs[name]["error_vs_oracle"] = errs["designs." + name]
        line["free_run"] = free_run_divergence(samples["free_run"])
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- CPU oracle
def cpu_baseline(budget_s=15.0, steps_cap=None):
    """The oracle (FP64 quadrature fitness, OpenMP) on the same workload, for as
    many whole generations as fit in the budget, starting from the initial
    population; throughput in the same unit."""
    import numpy as np

    import oracle
    from paper_2511_01255_gb300 import workloads as W
    c = W.PAPER_SCALE
    N, NP = c["N"], c["NP"]
    cfg = oracle.make_cfg(NP, N, c["G"], c["F"], c["CR"], c["seed"])
    X = oracle.init_population(cfg)
    t0 = time.perf_counter()
    f64 = np.abs(oracle.deff_genes(X, c["kappa1"], c["kappa2"])) ** 2
    fdec = f64.astype(np.float32)
    evals = NP * N
    g = 0
    while True:
        X, fdec, f64, _, _, _ = oracle.hwsda_generation(cfg, c["kappa1"], c["kappa2"], g, X, fdec,
                                                        f64)
        evals += (2 * NP - 3) * N
        g += 1
        el = time.perf_counter() - t0
        if el > budget_s or (steps_cap and g >= steps_cap):
            break
    return {"value": evals / el, "unit": "domain-evals/s", "cores": oracle.num_threads(),
            "cpu_model": cpu_model(), "kind": "oracle", "generations": g,
            "sample": f"init + {g} generations of {c['name']} ({el:.1f} s, FP64 quadrature, "
                      f"Q=16 Gauss-Legendre nodes per domain and level)"}


def cpu_other_workloads():
    """The oracle on the other workloads: the 16-domain run in full, and the
    1e5-domain and 512-instance runs extrapolated from the FP64 fitness of sampled
    rows (the oracle's time is its quadrature fitness; its FP32 updates take about
    2 % of it and are not timed), scaled by each run's domain-evals."""
    import oracle
    from paper_2511_01255_gb300 import workloads as W
    out = {}
    c = W.SMALL
    cfg = oracle.make_cfg(c["NP"], c["N"], c["G"], c["F"], c["CR"], c["seed"])
    t0 = time.perf_counter()
    oracle.hwsda_run(cfg, c["kappa1"], c["kappa2"])
    el = time.perf_counter() - t0
    ev = (c["NP"] + c["G"] * (2 * c["NP"] - 3)) * c["N"]
    out[c["name"]] = {"value": ev / el, "unit": "domain-evals/s", "s_per_run": el,
                      "kind": "full run (init + 200 generations)"}
    cp = W.PRECISION
    X = W.random_genes(16, cp["N"], seed=2)
    t0 = time.perf_counter()
    oracle.deff_genes(X, cp["kappa1"], cp["kappa2"])
    el = time.perf_counter() - t0
    rate = 16 * cp["N"] / el
    ev = (cp["NP"] + cp["G"] * (2 * cp["NP"] - 3)) * cp["N"]
    out[cp["name"]] = {"value": rate, "unit": "domain-evals/s", "kind": "extrapolated",
                       "extrapolated_s_per_run": ev / rate,
                       "sample": f"FP64 quadrature fitness of 16 random rows of {cp['N']} domains "
                                 f"({el:.2f} s), scaled to the run's {ev:.3g} domain-evals"}
    inst = W.batched_instances(512)
    pick = inst[::64]
    t0 = time.perf_counter()
    for ci in pick:
        oracle.deff_genes(W.random_genes(16, ci["N"], seed=ci["N"]), ci["kappa1"], ci["kappa2"])
    el = time.perf_counter() - t0
    rate = 16 * sum(ci["N"] for ci in pick) / el
    ev = sum((ci["NP"] + ci["G"] * (2 * ci["NP"] - 3)) * ci["N"] for ci in inst)
    out["batch512_g1000"] = {"value": rate, "unit": "domain-evals/s", "kind": "extrapolated",
                             "extrapolated_s_per_run": ev / rate,
                             "sample": f"FP64 quadrature fitness of 16 random rows of each of "
                                       f"{len(pick)} of the 512 instances ({el:.2f} s), scaled "
                                       f"to the batch's {ev:.3g} domain-evals"}
    return out


def oracle_errors(samples):
    """Relative error of the sampled GPU results against the oracle (FP64 quadrature
    of the Sec. 2.1 integral): |D_gpu - D_oracle| / |D_oracle| with no floor, and with
    the floor 1e-3 L^2/2 that random (cancelling) rows need; for the adjoint also
    the gradient error at 16 coordinates against the oracle's exact FP64 gradient,
    relative to its largest magnitude there."""
    import numpy as np

    import oracle

    def rows_err(rows):
        strict, floored, scale = [], [], []
        for r in rows:
            N = r["N"]
            if "genes" in r:
                ref = oracle.deff_genes(np.asarray(r["genes"][:N])[None], r["kappa1"], r["kappa2"])[0]
            else:
                d = oracle.signs_from_bits(np.asarray(r["words"])[None], N)[0]
                ref = oracle.deff(d, r["kappa1"], r["kappa2"])
            e = abs(r["D"] - ref)
            strict.append(e / abs(ref))
            floored.append(e / max(abs(ref), 1e-3 * N * N / 2))
            scale.append(abs(ref) / (N * N / 2))
        return {"max_rel": max(strict), "max_rel_with_floor": max(floored), "rows": len(rows),
                "deff_over_L2half": scale, "tolerance": 1e-5,
                "definition": "|D_gpu - D_oracle| / |D_oracle| (with floor: / max(|D_oracle|, "
                              "1e-3 L^2/2)); deff_over_L2half = |D_oracle| / (L^2/2) per row"}

    def design_err(rows):
        r = rows[0]
        dc = r["cfg"]
        cfg = oracle.make_cfg(1, r["N"], dc["G"], dc["F"], dc["CR"], dc["seed"], obj=dc["kind"],
                              kappas=dc["kappas"], G0=dc["G0"], beta=dc["beta"])
        ref = float(oracle.objective_rows(cfg, np.asarray(r["genes"])[None])[0])
        return {"objective_abs_err": abs(r["objective"] - ref), "objective_oracle": ref,
                "objective_rel_err": abs(r["objective"] - ref) / abs(ref),
                "tolerance_abs": 1e-5 * len(dc["kappas"]) * dc["G0"],
                "definition": "|f_gpu - f_oracle| of the best design (each |G0 - G_k| carries "
                              "G_k's error, so the scale is K G0)"}

    out = {k: (design_err(v) if k.startswith("designs.") else rows_err(v))
           for k, v in samples.items() if k not in ("adjoint", "free_run")}
    a = samples["adjoint"]
    g_ref, D_ref = oracle.grad_relaxed(a["theta"].astype(np.float64), a["kappa1"], a["kappa2"])
    g_ref = g_ref[a["cols"]]
    out["adjoint"] = {"d_eff_max_rel": abs(a["D"] - D_ref) / abs(D_ref),
                      "deff_over_L2half": abs(D_ref) / (a["N"] ** 2 / 2),
                      "grad_max_err": float(np.max(np.abs(a["grad"] - g_ref)) / np.max(np.abs(g_ref))),
                      "grad_coordinates": len(a["cols"]), "tolerance": {"d_eff": 1e-5, "grad": 1e-4},
                      "definition": "row: a relaxed two-tone design (theta = 3 sign pattern); "
                                    "grad error = max_k |g_gpu - g_oracle| / max_k |g_oracle|"}
    return out


def free_run_divergence(pops):
    """The GPU's free run of the 16-domain workload (its own FP32 decisions) against
    the oracle's free run (FP64 decisions) from the same initial population: the
    first generation after which the populations differ (a near-tie decided
    differently; None if they never do) and the gap between the two final bests'
    FP64 fitness."""
    import numpy as np

    import oracle
    from paper_2511_01255_gb300 import workloads as W
    c = W.SMALL
    cfg = oracle.make_cfg(c["NP"], c["N"], c["G"], c["F"], c["CR"], c["seed"])
    X = oracle.init_population(cfg)
    same_init = bool(np.array_equal(X, pops[0]))
    f64 = oracle.objective_rows(cfg, X, c["kappa1"], c["kappa2"])
    fdec = f64.astype(np.float32)
    first = None
    for g in range(c["G"]):
        X, fdec, f64, _, _, _ = oracle.hwsda_generation(cfg, c["kappa1"], c["kappa2"], g, X, fdec, f64)
        if first is None and not np.array_equal(X, pops[g + 1]):
            first = g
    f_gpu = oracle.objective_rows(cfg, pops[-1], c["kappa1"], c["kappa2"]).max()
    f_orc = f64.max()
    best, _ = oracle.bruteforce(c["N"], c["kappa1"], c["kappa2"])
    return {"workload": c["name"], "same_initial_population": same_init,
            "first_divergence_generation": first, "generations": c["G"],
            "final_best_f64_gpu": float(f_gpu), "final_best_f64_oracle": float(f_orc),
            "final_best_gap_rel": float(abs(f_gpu - f_orc) / f_orc),
            "exhaustive_optimum": float(best),
            "note": "free runs: each side decides selections and leaders in its own precision "
                    "(GPU FP32, oracle FP64); lockstep parity is tested separately"}


def cpu_closed_form(budget_s=2.0):
    """A fairer CPU throughput figure than the quadrature oracle: the oracle's FP64
    closed-form scan of the same fitness (all host cores), on the workload's row
    shape (NP rows of N domains), repeated for about budget_s."""
    import numpy as np

    import oracle
    from paper_2511_01255_gb300 import workloads as W
    c = W.PAPER_SCALE
    X = W.random_genes(c["NP"], c["N"], seed=1)
    oracle.deff_closed_genes(X, c["kappa1"], c["kappa2"])  # warm the rule and threads
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.deff_closed_genes(X, c["kappa1"], c["kappa2"])
        reps += 1
        el = time.perf_counter() - t0
        if el > budget_s:
            break
    return {"value": reps * c["NP"] * c["N"] / el, "unit": "domain-evals/s",
            "cores": oracle.num_threads(), "kind": "oracle closed-form FP64 scan",
            "sample": f"{reps} evaluations of {c['NP']} rows x {c['N']} domains ({el:.1f} s)"}


def run_reference(args):
    """The reference arm: the oracle itself, timed on the host cores on the same
    workload, metric and unit; every step is a bounded sample of the run (its initial
    population and as many whole generations as fit in the step's share of the CPU
    budget), and ms_per_step is the time of that sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2511_01255_gb300 import workloads as W
    c = W.PAPER_SCALE
    per_step, wall, gens = [], [], []
    cb = None
    for _ in range(args.warmup):
        cpu_baseline(budget_s=0.0, steps_cap=1)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(budget_s=args.cpu_budget / max(1, args.steps), steps_cap=None)
        wall.append(time.perf_counter() - t0)
        per_step.append(cb["value"])
        gens.append(cb["generations"])
    value = sum(per_step) / len(per_step)
    evals_per_run = (c["NP"] + c["G"] * (2 * c["NP"] - 3)) * c["N"]
    line = {
        "metric": METRIC, "value": value, "unit": "domain-evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(wall) / len(wall), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(c, world),
        "form": "oracle (CPU)",
        "step": f"init + {min(gens)}-{max(gens)} generations of the run per step (a bounded "
                f"sample; the GPU arm's step is the whole run of {c['G']} generations)",
        "extrapolated_ms_per_run": evals_per_run / value * 1e3,
        "l2_note": "the CPU oracle does not use the GPU; config.l2 describes the GPU arm",
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "domain-evals/s", "cores": cb["cores"],
                         "cpu_model": cb["cpu_model"], "kind": "oracle",
                         "sample": cb["sample"] + " per step"},
        "e2e": {"value": value, "unit": "domain-evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
