"""Strict relative parity at the precision-stress size: N = 1e5 domains (L = 100 mm at
w = 1 um), plain and Kahan-compensated FP32 scans, against the FP64 oracle (the
Sec. 2.1 double integral by nested quadrature) and against closed forms.

Random rows cancel (|d_eff| ~ N), so their comparison needs the tolerance floor of
tests/helpers.py.  The rows here have |d_eff| of 7-40 % of L^2/2, far above that
floor, and every comparison is a plain relative error with no floor:
  * all +1 at kappa1 = kappa2 = 0: d_eff = L^2/2 = 5e9 (the C sum of the scan exceeds
    2^24 many times over);
  * alternating at kappa1 = kappa2 = pi (first-order QPM of both steps):
    d_eff = -(2/pi)^2 L^2/2 exactly;
  * the two-tone row sign(cos kappa1 j + cos kappa2 j) at the paper-scale mismatches
    kappa1 = 2pi/6.9, kappa2 = 2pi/1.55: |d_eff| = 0.07 L^2/2 (oracle value);
  * the best individual of a 1e5-domain, 1024-individual run seeded with such rows.
Each goes through qpm_eval (16-byte aligned rows: the cp.async ring; other rows: the
register-prefetch sweep), qpm_eval_packed, and the optimiser's own team scan
(qpm_set_population recomputes every fitness with it) at 256 and 512 threads per
individual.
"""
import math

import numpy as np
import pytest

from helpers import TOL_D

pytestmark = pytest.mark.gpu

N = 100000
K1, K2 = 2 * math.pi / 6.9, 2 * math.pi / 1.55


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_01255_gb300 as q
    q.lib()
    return q


def _rows():
    from paper_2511_01255_gb300 import workloads as W
    tt = W.two_tone_signs(N, K1, K2)
    return {
        "ones_k0": (np.ones(N, np.float32), 0.0, 0.0, N * N / 2.0),
        "alt_pi": (W.alternating(N), math.pi, math.pi, -(2 / math.pi) ** 2 * N * N / 2.0),
        "two_tone": (tt, K1, K2, None),
    }


@pytest.fixture(scope="module")
def refs(orc):
    """FP64 oracle value of every row; the closed forms pin the oracle itself."""
    out = {}
    for name, (row, a, b, exact) in _rows().items():
        ref = orc.deff_genes(row[None], a, b)[0]
        if exact is not None:
            assert abs(ref - exact) <= 1e-9 * abs(exact)
        assert abs(ref) > 0.05 * N * N / 2  # far above the random-row floor
        out[name] = ref
    return out


def _strict(D, ref):
    z = D[:, 0].astype(np.float64) + 1j * D[:, 1].astype(np.float64)
    return np.abs(z - ref) / abs(ref)


def _eval(q, path, row, a, b, comp):
    import torch
    from paper_2511_01255_gb300 import workloads as W
    X = np.tile(row, (5, 1))
    D = torch.empty((5, 2), device="cuda")
    if path == "aligned":
        q.qpm_eval(N, a, b, torch.from_numpy(X).cuda(), D, None, comp)
    elif path == "unaligned":
        Xu = np.zeros((5, N + 1), np.float32)
        Xu[:, :N] = X
        q.qpm_eval(N, a, b, torch.from_numpy(Xu).cuda()[:, :N], D, None, comp)
    elif path == "packed":
        q.qpm_eval_packed(N, a, b, torch.from_numpy(W.pack_signs(X, N).view(np.int32)).cuda(), D,
                          None, comp)
    else:
        team = int(path[4:])
        prm = q.Params(5, 10, 0.5, 0.9, 1, 0, comp, team)
        with q.State([(N, a, b)], [prm]) as st:
            st.init()
            q.qpm_set_population(st.h, 0, torch.from_numpy(X).cuda(), 0)
            _, _, D = st.population()
    torch.cuda.synchronize()
    return D.cpu().numpy()


@pytest.mark.parametrize("comp", [0, 1])
@pytest.mark.parametrize("path", ["aligned", "unaligned", "packed", "team256", "team512"])
def test_strict_relative_at_1e5_domains(q, refs, path, comp):
    """Every fitness path, plain and compensated, within 1e-5 relative (no floor)."""
    errs = {}
    for name, (row, a, b, _) in _rows().items():
        errs[name] = float(_strict(_eval(q, path, row, a, b, comp), refs[name]).max())
    assert max(errs.values()) < TOL_D, errs


@pytest.mark.parametrize("comp", [0, 1])
def test_best_of_a_1e5_domain_run_is_strictly_within_tolerance(q, orc, comp):
    """A 1024 x 1e5 population (the precision-stress workload's shape) seeded with
    two-tone rows among random ones runs 2 persistent generations; the best
    individual's FP32 d_eff (the value the optimiser selected on) and its FP64
    re-check are compared with the oracle, strictly relative."""
    import torch
    from paper_2511_01255_gb300 import workloads as W
    NP = 1024
    X = W.random_genes(NP, N, seed=31)
    tt = W.two_tone_signs(N, K1, K2)
    for r in (3, 500, 1000):
        X[r] = tt * np.float32(0.75)
    X[500, ::97] *= -1  # a neighbour of the two-tone row
    prm = q.Params(NP, 500, 0.5, 0.9, 1, 0, comp)
    with q.State([(N, K1, K2)], [prm]) as st:
        st.init()
        q.qpm_set_population(st.h, 0, torch.from_numpy(X).cuda(), 0)
        st.run(2, q.RUN_PERSISTENT)
        Xg, f, D = st.population()
        xb, d64, fb, idx = st.best()
        torch.cuda.synchronize()
    i = int(idx.cpu()[0])
    assert float(f.cpu()[i]) == float(fb.cpu()[0])
    ref = orc.deff_genes(Xg.cpu().numpy()[i][None], K1, K2)[0]
    assert abs(ref) > 0.05 * N * N / 2
    assert _strict(D.cpu().numpy()[i][None], ref)[0] < TOL_D
    z64 = complex(*d64.cpu().numpy())
    assert abs(z64 - ref) <= 1e-9 * abs(ref)
