"""Autotuner for the launch shapes of a workload.

Team width: the library's automatic choice (qpm_params.team = 0) is a fixed
rule, the smallest power of two in [32, 256] giving at most 4 domains per
thread.  autotune_team measures the candidates instead, through the C ABI, for a
given problem size, population and execution form, and caches the fastest in a
JSON file keyed by (device name, N bucket, NP, compensated, form).  Pass the
result as qpm_params.team.

Batched form: autotune_batch_cluster measures the CTAs per thread-block cluster
(qpm_set_batch_cluster) on the state itself, a few generations per candidate from
the initial population, and caches the fastest by (device, number of instances,
work buckets of the largest and of the mean instance).
"""
import json
import os
import time

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
CANDIDATES = (32, 64, 128, 256, 512)


def n_bucket(N):
    """Problems whose N rounds to the same power of two (in quarters) share an entry."""
    b = 1
    while b * 2 <= N:
        b *= 2
    q = (N - b) * 4 // b
    return f"{b}+{q}/4"


def _key(device, N, NP, compensated, form, objective=None):
    k = f"{device}|N{n_bucket(N)}|NP{NP}|c{int(bool(compensated))}|f{form}"
    if objective is not None:  # (kind, kappas, G0, beta): the kind and problem count
        k += f"|o{int(objective[0])}k{len(objective[1])}"
    return k


def load_cache(path=CACHE):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=CACHE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(timings):
    """Fastest candidate; ties go to the smaller team (fewer threads per row)."""
    return min(sorted(timings), key=lambda t: timings[t])


def measure_team(N, kappa1, kappa2, NP, team, compensated=0, form=None, gens=40, reps=3,
                 objective=None):
    """Seconds per generation of one instance with the given team width; objective:
    (kind, kappas, G0, beta) of qpm_set_objective, or None for the cascaded |d_eff|^2."""
    import torch

    import paper_2511_01255_gb300 as q
    form = q.RUN_PERSISTENT if form is None else form
    G = gens * (reps + 1) + 1
    prm = q.Params(NP, G, 0.5, 0.9, 1, 0, int(compensated), int(team))
    with q.State([(N, kappa1, kappa2)], [prm]) as st:
        if objective is not None:
            st.set_objective(*objective)
        st.init()
        st.run(gens, form)  # warm-up (graph instantiation, caches)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            st.run(gens, form)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3 / gens)
    return best


def autotune_team(N, kappa1, kappa2, NP, compensated=0, form=None, gens=40,
                  candidates=CANDIDATES, use_cache=True, path=CACHE, measure=None,
                  objective=None):
    """Return the fastest team width for this workload (cached).  objective: the
    (kind, kappas, G0, beta) of qpm_set_objective the instance will optimise, or None."""
    import torch

    import paper_2511_01255_gb300 as q
    form = q.RUN_PERSISTENT if form is None else form
    device = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    key = _key(device, N, NP, compensated, form, objective)
    cache = load_cache(path) if use_cache else {}
    if key in cache:
        return cache[key]["team"]
    measure = measure or measure_team
    timings = {}
    for t in candidates:
        if t > 32 and N <= 4 * (t // 2):
            continue  # more threads than 4 domains each would leave most of them idle
        if objective is None:
            timings[t] = measure(N, kappa1, kappa2, NP, t, compensated, form, gens)
        else:
            timings[t] = measure(N, kappa1, kappa2, NP, t, compensated, form, gens,
                                 objective=objective)
    best = choose(timings)
    cache[key] = {"team": best, "s_per_generation": {str(k): v for k, v in timings.items()},
                  "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if use_cache:
        save_cache(cache, path)
    return best


BATCH_CLUSTERS = (1, 2, 4)


def _batch_key(device, sizes):
    """sizes: N * NP of every instance; the makespan depends on the largest one."""
    mean = sum(sizes) / len(sizes)
    return f"{device}|batch|n{len(sizes)}|max{n_bucket(max(sizes))}|mean{n_bucket(int(mean))}"


def measure_batch_cluster(state, ctas, gens=20):
    """Seconds per generation of the batched form of `state` with clusters of `ctas`
    CTAs, measured from the initial population (the state is re-initialised first)."""
    import torch

    import paper_2511_01255_gb300 as q
    state.set_batch_cluster(ctas)
    state.init()
    state.run(1, q.RUN_BATCHED)  # capture and warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    state.run(gens, q.RUN_BATCHED)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3 / gens


def autotune_batch_cluster(state, gens=20, candidates=BATCH_CLUSTERS, use_cache=True, path=CACHE,
                           measure=None):
    """Set and return the fastest cluster size of the batched form for `state` (cached).
    Call it right after state.init(): the candidates run from the initial population
    and the state is initialised again at the end (init is deterministic, so the
    population is the same as before the call)."""
    import torch
    device = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    sizes = [state.problems[k][0] * state.params[k].NP for k in range(len(state.problems))]
    key = _batch_key(device, sizes)
    cache = load_cache(path) if use_cache else {}
    if key in cache:
        best = cache[key]["ctas"]
    else:
        measure = measure or measure_batch_cluster
        timings = {c: measure(state, c, gens) for c in candidates}
        best = choose(timings)
        cache[key] = {"ctas": best, "s_per_generation": {str(k): v for k, v in timings.items()},
                      "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
        if use_cache:
            save_cache(cache, path)
    state.set_batch_cluster(best)
    if hasattr(state, "init"):
        state.init()
    return best

