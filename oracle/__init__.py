"""CPU oracle for the cascaded-THG QPM design method -- TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package.  The CUDA library in `paper_2511_01255_gb300` shares no
code with it and never calls it.

Everything here is a thin ctypes layer over `qpm_oracle.c` (FP64 quadrature of
the d_eff double integral of Sec. 2.1, its exact derivative, the HWSDA loop of
Sec. 3.2 with FP32 genes, and Philox4x32-10).  See the C file for the readings
of the paper that the oracle takes.
"""
import ctypes
import os

import numpy as np

from . import build as _build

Q_DEFAULT = 16

_lib = None


class OrcCfg(ctypes.Structure):
    _fields_ = [("NP", ctypes.c_int32), ("N", ctypes.c_int32), ("ld", ctypes.c_int64),
                ("G", ctypes.c_int32), ("F", ctypes.c_float), ("CR", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("inst", ctypes.c_uint32),
                ("combine", ctypes.c_int32), ("f_schedule", ctypes.c_int32),
                ("obj", ctypes.c_int32), ("K", ctypes.c_int32),
                ("kap1", ctypes.c_double * 8), ("kap2", ctypes.c_double * 8),
                ("G0", ctypes.c_float), ("beta", ctypes.c_float)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64, u32, u64, dbl = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_double)
        L.orc_gauss_legendre.argtypes = [ctypes.c_int, P, P]
        L.orc_deff_quad.argtypes = [ctypes.c_int, ctypes.c_int, i64, dbl, dbl, P, ctypes.c_int, P]
        L.orc_deff_genes.argtypes = [ctypes.c_int, ctypes.c_int, i64, dbl, dbl, P, ctypes.c_int, P]
        L.orc_deff_closed.argtypes = [ctypes.c_int, ctypes.c_int, i64, dbl, dbl, P, ctypes.c_int, P]
        L.orc_bruteforce.argtypes = [ctypes.c_int, dbl, dbl, ctypes.c_int, P, P]
        L.orc_bruteforce.restype = dbl
        L.orc_shg_genes.argtypes = [ctypes.c_int, ctypes.c_int, i64, dbl, P, ctypes.c_int, P]
        L.orc_multi_objective.argtypes = [ctypes.c_int, ctypes.c_int, i64, ctypes.c_int, P, P, P,
                                          dbl, dbl, ctypes.c_int, P, P]
        L.orc_grad_relaxed.argtypes = [ctypes.c_int, dbl, dbl, P, ctypes.c_int, P, P]
        L.orc_fit_relaxed.argtypes = [ctypes.c_int, dbl, dbl, P, ctypes.c_int, P]
        L.orc_fit_relaxed.restype = dbl
        L.orc_fd_grad.argtypes = [ctypes.c_int, dbl, dbl, P, P, ctypes.c_int, dbl, ctypes.c_int, P]
        L.orc_philox.argtypes = [P, P, P]
        L.orc_uniform.argtypes = [u64, u32, u32, u32, u32, u32]
        L.orc_uniform.restype = ctypes.c_float
        L.orc_de_indices.argtypes = [u64, u32, u32, i32, i32, i32, P]
        L.orc_init_population.argtypes = [P, P]
        L.orc_de_trials.argtypes = [P, u32, P, P]
        L.orc_top3.argtypes = [i32, P, P]
        L.orc_F_of.argtypes = [P, i32]
        L.orc_F_of.restype = ctypes.c_float
        L.orc_a_of.argtypes = [i32, i32]
        L.orc_a_of.restype = ctypes.c_float
        L.orc_gwo_candidates.argtypes = [P, u32, P, P, P]
        L.orc_hwsda_generation.argtypes = [P, dbl, dbl, ctypes.c_int, i32, P, P, P, P, P, P, P, P, P,
                                           P, P]
        L.orc_hwsda_generation.restype = ctypes.c_int
        L.orc_adaptive_F.argtypes = [P, i32, P, P, ctypes.c_float, P, P]
        L.orc_objective_rows.argtypes = [P, dbl, dbl, ctypes.c_int, P, P]
        L.orc_discrete_thresholds.argtypes = [i32, i32, P]
        L.orc_adaptive_F.restype = ctypes.c_int
        L.orc_hwsda_run.argtypes = [P, dbl, dbl, ctypes.c_int, P, P, P, P, P]
        L.orc_hwsda_run.restype = ctypes.c_int
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads():
    return lib().orc_num_threads()


def gauss_legendre(Q):
    t = np.zeros(Q)
    w = np.zeros(Q)
    if lib().orc_gauss_legendre(Q, _p(t), _p(w)) != 0:
        raise ValueError("Q out of range")
    return t, w


def deff(d, kappa1, kappa2, Q=Q_DEFAULT):
    """d_eff (units of w^2) of each row of the real array d [NP, N] (or [N])."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    one = d.ndim == 1
    d2 = d.reshape(1, -1) if one else d
    NP, N = d2.shape
    out = np.zeros((NP, 2))
    lib().orc_deff_quad(NP, N, N, kappa1, kappa2, _p(d2), Q, _p(out))
    D = out[:, 0] + 1j * out[:, 1]
    return D[0] if one else D


def deff_genes(X, kappa1, kappa2, Q=Q_DEFAULT):
    """d_eff of FP32 gene rows X [NP, N] under the sign map d = (x < 0) ? -1 : +1."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    NP, N = X.shape
    out = np.zeros((NP, 2))
    lib().orc_deff_genes(NP, N, N, kappa1, kappa2, _p(X), Q, _p(out))
    return out[:, 0] + 1j * out[:, 1]


def deff_closed_genes(X, kappa1, kappa2, Q=Q_DEFAULT):
    """d_eff of FP32 gene rows by the closed form for unit domains (FP64 scan in
    index order; phi and psi by the Q-node rule) -- the CPU throughput reference."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    NP, N = X.shape
    out = np.zeros((NP, 2))
    lib().orc_deff_closed(NP, N, N, kappa1, kappa2, _p(X), Q, _p(out))
    return out[:, 0] + 1j * out[:, 1]


def shg_genes(X, kappa, Q=Q_DEFAULT):
    """SHG field integral int_0^L d(z) e^{-i k z} dz (units of w) of each gene row."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    NP, N = X.shape
    out = np.zeros((NP, 2))
    lib().orc_shg_genes(NP, N, N, kappa, _p(X), Q, _p(out))
    return out[:, 0] + 1j * out[:, 1]


def multi_objective(X, kappas, G0, beta, Q=Q_DEFAULT):
    """(d_eff [NP, K], objective [NP]) for the list of (kappa1, kappa2) pairs."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    NP, N = X.shape
    K = len(kappas)
    k1 = np.ascontiguousarray([k[0] for k in kappas], dtype=np.float64)
    k2 = np.ascontiguousarray([k[1] for k in kappas], dtype=np.float64)
    D = np.zeros((NP, K, 2))
    obj = np.zeros(NP)
    lib().orc_multi_objective(NP, N, N, K, _p(k1), _p(k2), _p(X), G0, beta, Q, _p(D), _p(obj))
    return D[..., 0] + 1j * D[..., 1], obj


def signs_from_bits(words, N):
    """Domain signs from packed bits (bit j of word j//32 set -> d_j = -1)."""
    words = np.asarray(words, dtype=np.uint32)
    NP = words.shape[0]
    bits = ((words[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(NP, -1)[:, :N]
    return np.where(bits == 1, -1.0, 1.0)


def bruteforce(N, kappa1, kappa2, Q=Q_DEFAULT, want_all=False):
    """Exhaustive optimum over all 2^N sign patterns: (best f, lowest best mask[, all f])."""
    fit = np.zeros(1 << N) if want_all else None
    m = ctypes.c_int64(0)
    best = lib().orc_bruteforce(N, kappa1, kappa2, Q, _p(fit), ctypes.byref(m))
    return (best, m.value, fit) if want_all else (best, m.value)


def grad_relaxed(theta, kappa1, kappa2, Q=Q_DEFAULT):
    """(df/dtheta [N], D) for f = |d_eff|^2, d = tanh(theta)."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    g = np.zeros_like(theta)
    D = np.zeros(2)
    lib().orc_grad_relaxed(theta.size, kappa1, kappa2, _p(theta), Q, _p(g), _p(D))
    return g, D[0] + 1j * D[1]


def fit_relaxed(theta, kappa1, kappa2, Q=Q_DEFAULT):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    D = np.zeros(2)
    f = lib().orc_fit_relaxed(theta.size, kappa1, kappa2, _p(theta), Q, _p(D))
    return f, D[0] + 1j * D[1]


def fd_grad(theta, kappa1, kappa2, idx, h=1e-6, Q=Q_DEFAULT):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.zeros(idx.size)
    lib().orc_fd_grad(theta.size, kappa1, kappa2, _p(theta), _p(idx), idx.size, h, Q, _p(out))
    return out


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c), _p(k), _p(o))
    return o


def uniform(seed, inst, tag, g, i, j):
    return lib().orc_uniform(seed, inst, tag, g, i, j)


def de_indices(seed, inst, g, i, NP, N):
    o = np.zeros(4, dtype=np.int32)
    lib().orc_de_indices(seed, inst, g, i, NP, N, _p(o))
    return o


def a_of(g, G):
    return lib().orc_a_of(g, G)


def make_cfg(NP, N, G, F, CR, seed, inst=0, combine=0, f_schedule=0, obj=0, kappas=(),
             G0=0.0, beta=0.0):
    """Loop configuration.  obj: 0 cascaded |d_eff|^2 (maximised), 1 SHG |E|^2 of
    kappa1 (maximised), 2 / 3 the multi-wavelength objective over the (kappa1, kappa2)
    pairs in `kappas` with the cascaded / SHG field (minimised)."""
    k1 = (ctypes.c_double * 8)(*[k[0] for k in kappas])
    k2 = (ctypes.c_double * 8)(*[k[1] for k in kappas])
    return OrcCfg(NP, N, N, G, F, CR, seed, inst, combine, f_schedule, obj, len(kappas), k1, k2,
                  G0, beta)


def objective_rows(cfg, X, kappa1=0.0, kappa2=0.0, Q=Q_DEFAULT):
    """The loop's objective (cfg.obj) of each gene row of X, in FP64."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    out = np.zeros(X.shape[0])
    lib().orc_objective_rows(ctypes.byref(cfg), kappa1, kappa2, Q, _p(X), _p(out))
    return out


def F_of(cfg, g):
    return lib().orc_F_of(ctypes.byref(cfg), g)


def init_population(cfg):
    X = np.zeros((cfg.NP, cfg.ld), dtype=np.float32)
    lib().orc_init_population(ctypes.byref(cfg), _p(X))
    return X


def de_trials(cfg, g, X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    U = np.zeros_like(X)
    lib().orc_de_trials(ctypes.byref(cfg), g, _p(X), _p(U))
    return U


def top3(f):
    f = np.ascontiguousarray(f, dtype=np.float32)
    o = np.zeros(3, dtype=np.int32)
    lib().orc_top3(f.size, _p(f), _p(o))
    return o


def discrete_thresholds(g, G):
    """(social, flip, plus[0..4]) 16-bit thresholds of the discrete GWO at generation g."""
    o = np.zeros(7, dtype=np.uint32)
    lib().orc_discrete_thresholds(g, G, _p(o))
    return int(o[0]), int(o[1]), [int(x) for x in o[2:]]


def gwo_candidates(cfg, g, X, lead):
    """Candidates of the omega wolves (leader rows copied unchanged); lead: three
    leaders, or four for the discrete GWO (cfg.combine == 2)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    lead = np.ascontiguousarray(lead, dtype=np.int32)
    Y = X.copy()
    lib().orc_gwo_candidates(ctypes.byref(cfg), g, _p(X), _p(lead), _p(Y))
    return Y


def adaptive_F(cfg, g, f, improved, F_g):
    """The adaptive F of Sec. 3.1.1 (see orc_adaptive_F): (branch, F of generation
    g + 1, (cv^2, improved fraction, fitness range)); branch 0 schedule, 1 raised,
    2 lowered."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    imp = np.ascontiguousarray(improved, dtype=np.uint8)
    out = ctypes.c_float()
    st = np.zeros(3)
    br = lib().orc_adaptive_F(ctypes.byref(cfg), g, _p(f), _p(imp), F_g, ctypes.byref(out), _p(st))
    return br, out.value, tuple(st)


def hwsda_generation(cfg, kappa1, kappa2, g, X, fdec, f64=None, lock_trial=None,
                     lock_cand=None, eval_mask=None, Q=Q_DEFAULT, F=None):
    """One generation (Sec. 3.2 Steps 2-6) from population X.

    Returns (X_next, fdec_next, f64_next, trial_f64, cand_f64, leaders), plus
    (F_next, branch) at the end when F (the adaptive F of generation g) is given
    (cfg.f_schedule == 2).  In lockstep mode (lock_trial/lock_cand given) the FP32
    values decide; eval_mask limits which rows get an FP64 fitness (NaN elsewhere)."""
    X = np.array(X, dtype=np.float32, order="C", copy=True)
    fdec = np.array(fdec, dtype=np.float32, copy=True)
    f64 = np.zeros(cfg.NP) if f64 is None else np.array(f64, dtype=np.float64, copy=True)
    lt = None if lock_trial is None else np.ascontiguousarray(lock_trial, dtype=np.float32)
    lc = None if lock_cand is None else np.ascontiguousarray(lock_cand, dtype=np.float32)
    em = None if eval_mask is None else np.ascontiguousarray(eval_mask, dtype=np.uint8)
    tt = np.zeros(cfg.NP)
    tc = np.zeros(cfg.NP)
    lead = np.zeros(4 if cfg.combine == 2 else 3, dtype=np.int32)
    Fio = None if F is None else ctypes.c_float(F)
    br = ctypes.c_int32(-1)
    rc = lib().orc_hwsda_generation(ctypes.byref(cfg), kappa1, kappa2, Q, g, _p(X), _p(fdec),
                                    _p(f64), _p(lt), _p(lc), _p(em), _p(tt), _p(tc), _p(lead),
                                    None if Fio is None else ctypes.byref(Fio), ctypes.byref(br))
    if rc == -1:
        raise ValueError("orc_hwsda_generation: eval_mask needs lockstep mode")
    if rc == -2:
        raise ValueError("orc_hwsda_generation: F is given exactly for the adaptive F")
    if Fio is not None:
        return X, fdec, f64, tt, tc, lead, Fio.value, br.value
    return X, fdec, f64, tt, tc, lead


def hwsda_run(cfg, kappa1, kappa2, lockstep=None, want_trace=False, Q=Q_DEFAULT, want_F=False):
    """Run the HWSDA loop of Sec. 3.2.  Returns (X_final, f64_final[, trace64][, F history
    of G + 1 values])."""
    X = np.zeros((cfg.NP, cfg.ld), dtype=np.float32)
    f = np.zeros(cfg.NP)
    n_tr = cfg.NP * (1 + 2 * cfg.G)
    ls = None
    if lockstep is not None:
        ls = np.ascontiguousarray(lockstep, dtype=np.float32).ravel()
        assert ls.size == n_tr
    tr = np.zeros(n_tr) if want_trace else None
    Fh = np.zeros(cfg.G + 1, dtype=np.float32) if want_F else None
    lib().orc_hwsda_run(ctypes.byref(cfg), kappa1, kappa2, Q, _p(X), _p(f), _p(ls), _p(tr), _p(Fh))
    out = (X, f)
    if want_trace:
        out += (tr,)
    if want_F:
        out += (Fh,)
    return out
