"""Run one workload of the library for a profiler (ncu) or a quick timing.

  python -m paper_2511_01255_gb300.profile_run --workload paper --form launches --gens 40

workloads: small (N=16, NP=32), paper (N=1000, NP=256, compensated),
precision (N=1e5, NP=1024, compensated), design_thg3 / design_shg5 (the
multi-wavelength designs of Sec. 5: N=3000, NP=5000, K=3 cascaded or K=5 SHG
problems), eval (qpm_eval of 1024 random rows of N=1e5), batch, relaxed, latency (the grid barrier of the persistent form over
several CTA counts and a dependent L2 load, from qpm_measure_latency).  forms:
launches, graph, persistent, batched.  Prints the mean time per repetition
measured with CUDA events.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import torch

    import paper_2511_01255_gb300 as q
    from paper_2511_01255_gb300 import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="paper",
                    choices=["small", "paper", "precision", "design_thg3", "design_shg5", "eval",
                             "batch", "relaxed", "latency"])
    ap.add_argument("--form", default="launches",
                    choices=["launches", "graph", "persistent", "batched"])
    ap.add_argument("--gens", type=int, default=20)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--comp", type=int, default=-1, help="override the compensated flag")
    ap.add_argument("--team", type=int, default=0, help="threads per individual (0 = automatic)")
    ap.add_argument("--instances", type=int, default=512, help="instances of the batch workload")
    ap.add_argument("--packed", type=int, default=0, help="eval workload: packed sign words")
    ap.add_argument("--cluster", type=int, default=1, help="batched form: CTAs per cluster")
    a = ap.parse_args()
    q.lib()
    if a.workload == "latency":
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        for ctas in (32, nsm, 256, 4 * nsm):
            best = min(q.qpm_measure_latency(0, ctas) for _ in range(max(1, a.reps)))
            print(f"grid barrier, {ctas} CTAs of 256 threads: {best / 1e3:.3f} us (best of {max(1, a.reps)})")
        best = min(q.qpm_measure_latency(1) for _ in range(max(1, a.reps)))
        print(f"dependent L2 load: {best:.1f} ns (best of {max(1, a.reps)})")
        names = {2: "counter barrier, relaxed arrival and polling",
                 3: "gpu-scope fence between two CTA barriers",
                 4: "tagged all-to-all word exchange"}
        for kind, name in names.items():
            for ctas in (32, nsm, 256):
                best = min(q.qpm_measure_latency(kind, ctas) for _ in range(max(1, a.reps)))
                print(f"{name}, {ctas} CTAs: {best / 1e3:.3f} us (best of {max(1, a.reps)})")
        return
    if a.workload == "relaxed":
        c = W.RELAXED
        th = torch.from_numpy(W.relaxed_theta(c["B"], c["N"], seed=c["seed"])).cuda()
        D = torch.empty((c["B"], 2), device="cuda")
        A = q.relaxed_saved(c["B"], c["N"])
        g = torch.empty_like(th)
        # clean flush, as in the bench: a 256 MB write, then a 256 MB read of another
        # buffer, so that neither theta nor dirty lines are left in the 129 MB L2
        fw = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        fr = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

        def fwd():
            q.qpm_deff_relaxed_fwd(c["N"], c["kappa1"], c["kappa2"], th, D, None, A)

        def bwd():
            q.qpm_deff_relaxed_bwd(c["N"], c["kappa1"], c["kappa2"], th, D, A, None, g)

        fwd()
        bwd()
        tot = {"fwd": 0.0, "bwd": 0.0}
        for _ in range(a.reps):
            for name, fn in (("fwd", fwd), ("bwd", bwd)):
                fw.fill_(1.0)
                fr.sum()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                tot[name] += e0.elapsed_time(e1)
        f_us, b_us = 1e3 * tot["fwd"] / a.reps, 1e3 * tot["bwd"] / a.reps
        print(f"relaxed B={c['B']} N={c['N']}: fwd {f_us:.1f} us, bwd {b_us:.1f} us "
              f"(L2 cleanly flushed before each call)")
        return
    if a.workload == "eval":
        N, NP = 100000, 1024
        D = torch.empty((NP, 2), device="cuda")
        comp = 0 if a.comp < 0 else a.comp
        if a.packed:
            X = torch.randint(-2 ** 31, 2 ** 31 - 1, (NP, (N + 31) // 32), dtype=torch.int32,
                              device="cuda")
            fn = q.qpm_eval_packed
        else:
            X = torch.rand((NP, N), device="cuda") * 2 - 1
            fn = q.qpm_eval
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn(N, 1.0, 2.0, X, D, None, comp)
        e0.record()
        for _ in range(a.reps):
            fn(N, 1.0, 2.0, X, D, None, comp)
        e1.record()
        torch.cuda.synchronize()
        print(f"eval N={N} NP={NP} packed={a.packed}: {e0.elapsed_time(e1) / a.reps:.3f} ms per call")
        return
    form = {"launches": q.RUN_LAUNCHES, "graph": q.RUN_GRAPH, "persistent": q.RUN_PERSISTENT,
            "batched": q.RUN_BATCHED}[a.form]
    if a.workload == "batch":
        inst = W.batched_instances(a.instances)
        comp = 0 if a.comp < 0 else a.comp
        st = q.State([(c["N"], c["kappa1"], c["kappa2"]) for c in inst],
                      [q.Params(c["NP"], c["G"], c["F"], c["CR"], c["seed"], 0, comp, a.team)
                       for c in inst])
        st.set_batch_cluster(a.cluster)
        c = {"name": f"batch{a.instances}_g1000_cluster{a.cluster}"}
    elif a.workload.startswith("design"):
        c = W.DESIGN_THG3 if a.workload == "design_thg3" else W.DESIGN_SHG5
        comp = 0
        prm = q.Params(c["NP"], c["G"], c["F"], c["CR"], c["seed"], 0, comp, a.team)
        k1, k2 = c["kappas"][0]
        st = q.State([(c["N"], k1, k2)], [prm])
        st.set_objective(c["kind"], c["kappas"], c["G0"], c["beta"])
    else:
        c = {"small": W.SMALL, "paper": W.PAPER_SCALE, "precision": W.PRECISION}[a.workload]
        comp = c["compensated"] if a.comp < 0 else a.comp
        prm = q.Params(c["NP"], c["G"], c["F"], c["CR"], c["seed"], 0, comp, a.team)
        st = q.State([(c["N"], c["kappa1"], c["kappa2"])], [prm])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(a.reps):
        st.init()
        e0.record()
        st.run(a.gens, form)
        e1.record()
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    st.close()
    print(f"{c['name']} form={a.form} comp={comp} team={a.team or 'auto'}: {a.gens} generations in "
          f"{tot / a.reps:.3f} ms ({tot / a.reps / a.gens * 1e3:.2f} us/generation)")


if __name__ == "__main__":
    main()
