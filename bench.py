"""Benchmark: HWSDA design runs of the cascaded-THG QPM problem on one GB300.

One step = one whole HWSDA run of the paper-scale workload (N = 1000 domains,
kappa1 = 2pi/6.9, kappa2 = 2pi/1.55, NP = 256, G = 2000 generations, F = 0.5,
CR = 0.9, Kahan-compensated FP32 scan): phasor table, initial population and
its fitness, then 2000 generations of DE + GWO with greedy selection.  The
population (1 MB) lives in HBM/L2 throughout; L2 is flushed between timed steps.

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
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        for ln in self.lines:
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
def algorithmic_lane_ops_per_gene_gen(compensated):
    """Lane instructions the method needs per gene and generation (documented in
    the design doc): Philox4x32-10 at 1.75 calls (80 ops each), 7 uniforms (3 ops),
    DE update (7), GWO update (30), two fitness domain-evals (10 plain / 32 Kahan)."""
    return 1.75 * 80 + 7 * 3 + 7 + 30 + 2 * (32 if compensated else 10)


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
    c = W.PAPER_SCALE
    N, NP, G = c["N"], c["NP"], c["G"]
    # independent replicas: each rank designs its own crystal (seed = 1 + rank)
    prm = q.Params(NP, G, c["F"], c["CR"], c["seed"] + rank, 0, c["compensated"])
    prob = (N, c["kappa1"], c["kappa2"])
    evals_per_run = (NP + G * (2 * NP - 3)) * N
    gene_gens = NP * N * G
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    results = {}
    for mode_name, mode in (("plain_graph", q.RUN_GRAPH), ("persistent", q.RUN_PERSISTENT)):
        st = q.State([prob], [prm])
        for _ in range(args.warmup):
            st.init()
            st.run(G, mode)
        torch.cuda.synchronize()
        times = []
        sampler = ClockSampler(lrank)
        barrier()
        sampler.start()
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)
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
        t = sum(times) / len(times)
        if world > 1:
            import torch.distributed as dist
            tt = torch.tensor([t], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t = float(tt.item())
        results[mode_name] = dict(s_per_step=t, wall=wall, clocks=clocks, best_f=best_f,
                                  launches_per_step=(3 + (2 * G if mode == q.RUN_GRAPH else 1)))

    # dominant-kernel timing on its own stream: the persistent kernel alone
    st = q.State([prob], [prm])
    st.init()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    dur = []
    for _ in range(max(3, args.steps)):
        st.init()
        flush.fill_(1.0)
        e0.record(stream)
        st.run(G, q.RUN_PERSISTENT)
        e1.record(stream)
        e1.synchronize()
        dur.append(e0.elapsed_time(e1) / 1e3)
    st.close()
    kdur = statistics.median(dur)

    # end to end through the C ABI with host buffers (qpm_solve: create, init, run,
    # best genes + FP64 d_eff back to the host)
    best_host = torch.empty(N, dtype=torch.float32).pin_memory()
    d64_host = torch.empty(2, dtype=torch.float64).pin_memory()
    f_host = torch.empty(1, dtype=torch.float32).pin_memory()
    best_mode = min(results, key=lambda k: results[k]["s_per_step"])
    mode_id = q.RUN_PERSISTENT if best_mode == "persistent" else q.RUN_GRAPH
    for _ in range(args.warmup):
        q.qpm_solve(N, c["kappa1"], c["kappa2"], prm, mode_id, best_host, d64_host, f_host)
    barrier()
    e2e = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q.qpm_solve(N, c["kappa1"], c["kappa2"], prm, mode_id, best_host, d64_host, f_host)
        e2e.append(time.perf_counter() - t0)
    e2e_t = sum(e2e) / len(e2e)

    pk, pk_src = peaks()
    nsm = torch.cuda.get_device_properties(lrank).multi_processor_count
    sm_mhz = results[best_mode]["clocks"].get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    peak_max = nsm * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # T lane-ops/s
    ops = algorithmic_lane_ops_per_gene_gen(c["compensated"]) * gene_gens
    achieved = ops / kdur / 1e12

    if rank != 0:
        return
    best = results[best_mode]
    value = world * evals_per_run / best["s_per_step"]
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
        "config": {"workload": c["name"], "N": N, "NP": NP, "G": G,
                   "kappa1": c["kappa1"], "kappa2": c["kappa2"], "F": c["F"], "CR": c["CR"],
                   "compensated": bool(c["compensated"]), "form": best_mode,
                   "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"replicas{world}"},
        "gen_per_s": world * G / best["s_per_step"],
        "forms": {k: {"ms_per_step": v["s_per_step"] * 1e3,
                      "domain_evals_per_s": world * evals_per_run / v["s_per_step"],
                      "gen_per_s": world * G / v["s_per_step"],
                      "best_f": v["best_f"]} for k, v in results.items()},
        "roofline": {"bound": "alu", "kernel": "k_persist",
                     "achieved": achieved, "peak": peak_max, "unit": "T lane-ops/s",
                     "frac": achieved / peak_max, "traffic": None,
                     "peak_note": f"{nsm} SMs x 128 lanes x {pk.get('sm_max_mhz', 2070.0)} MHz "
                                  f"(issue limit, derived; clocks {pk_src})",
                     "frac_at_median_clock": achieved / (nsm * 128 * sm_mhz * 1e6 / 1e12),
                     "ops_per_gene_gen": algorithmic_lane_ops_per_gene_gen(c["compensated"]),
                     "launch_ms": kdur * 1e3},
        "e2e": {"value": world * evals_per_run / e2e_t, "unit": "domain-evals/s",
                "h2d_bytes_per_step": 24 + 40, "d2h_bytes_per_step": 4 * N + 16 + 4,
                "api": "qpm_solve (host buffers)", "form": best_mode},
        "gpu_launches": best["launches_per_step"] * args.steps,
        "clocks": best["clocks"],
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_budget)
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
            "kind": "oracle",
            "sample": f"init + {g} generations of {c['name']} ({el:.1f} s, FP64 quadrature, "
                      f"Q=16 Gauss-Legendre nodes per domain and level)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    per_step = []
    cb = None
    for _ in range(args.warmup):
        cpu_baseline(budget_s=0.0, steps_cap=1)
    for _ in range(args.steps):
        cb = cpu_baseline(budget_s=args.cpu_budget / max(1, args.steps), steps_cap=None)
        per_step.append(cb["value"])
    value = sum(per_step) / len(per_step)
    from paper_2511_01255_gb300 import workloads as W
    c = W.PAPER_SCALE
    evals_per_run = (c["NP"] + c["G"] * (2 * c["NP"] - 3)) * c["N"]
    line = {
        "metric": METRIC, "value": value, "unit": "domain-evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": evals_per_run / value * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": c["name"], "N": c["N"], "NP": c["NP"], "G": c["G"],
                   "form": "oracle (CPU)"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "domain-evals/s", "cores": cb["cores"],
                         "kind": "oracle", "sample": cb["sample"] + " per step"},
        "e2e": {"value": value, "unit": "domain-evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
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
