"""Host-side arithmetic of the benchmark's roofline fields (CPU only): the
algorithmic op count per gene-generation, the op-mix ceiling and the phase-wise
bound of a generation whose population exceeds L2."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

ISSUE = {"ffma": 38.0, "philox_calls_per_s": 4.0e11}


def test_op_count_per_gene_generation():
    # 80 Philox + 18 GWO uniforms + 1 crossover + 7 DE + 28 GWO + two domain-evals
    assert bench.algorithmic_lane_ops_per_gene_gen(0) == 154.0
    assert bench.algorithmic_lane_ops_per_gene_gen(1) == 162.5


def test_op_count_of_the_multi_wavelength_objectives():
    # the updates of the single count (134) and per phase one scan of each problem:
    # 10 lane-ops a domain for a cascaded problem, 2 for an SHG problem
    assert bench.algorithmic_lane_ops_per_gene_gen_multi(2, 1) == 154.0
    assert bench.algorithmic_lane_ops_per_gene_gen_multi(2, 3) == 194.0
    assert bench.algorithmic_lane_ops_per_gene_gen_multi(3, 5) == 154.0
    assert bench.algorithmic_lane_ops_per_gene_gen_multi(3, 1) == 138.0


def test_mix_ceiling_adds_generator_and_other_times():
    n_rest = 154.0 - 80.0
    t = 1.0 / ISSUE["philox_calls_per_s"] + n_rest / (ISSUE["ffma"] * 1e12)
    assert bench.mix_ceiling_gene_gens(0, ISSUE) == pytest.approx(1.0 / t)
    assert bench.mix_ceiling_gene_gens(1, ISSUE) < bench.mix_ceiling_gene_gens(0, ISSUE)


def test_phase_bound_takes_each_phase_limit():
    N, NP = 1000, 100
    genes = N * NP
    # unlimited issue: only the bytes remain, 20 B per gene in DE and 8 B in GWO
    fast = {"ffma": 1e30, "philox_calls_per_s": 1e42}
    assert bench.phase_bound_s_per_gen(N, NP, 0, fast, 1.0) == pytest.approx(28.0 * genes / 1e9)
    # unlimited bandwidth: the two phases' issue times add up to the mix-ceiling time
    t = bench.phase_bound_s_per_gen(N, NP, 0, ISSUE, 1e30)
    assert t == pytest.approx(genes / bench.mix_ceiling_gene_gens(0, ISSUE))
    t1 = bench.phase_bound_s_per_gen(N, NP, 1, ISSUE, 1e30)
    assert t1 == pytest.approx(genes / bench.mix_ceiling_gene_gens(1, ISSUE))
    # a bound never falls below either of its two limits
    for hbm in (100.0, 1000.0, 7000.0):
        tb = bench.phase_bound_s_per_gen(N, NP, 1, ISSUE, hbm)
        assert tb >= t1 * (1 - 1e-12) and tb >= 28.0 * genes / (hbm * 1e9) * (1 - 1e-12)


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one JSON line
    with the contract's keys, marked as the reference, with no GPU work."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--cpu-budget", "0.2"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e", "gpu_launches"):
        assert k in d, k
    assert d["impl"] == "reference" and d["gpu_launches"] == 0 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["config"]["workload"] == "n1000_np256_g2000"
