"""GB300 (sm_103a) quasi-phase-matching crystal design by HWSDA (arXiv 2511.01255).

Thin Python binding over the C ABI in ``include/qpm.h`` (library
``_build/libqpm.so``, built by ``build_lib.py``).  The functions keep the C
names; they only marshal arguments (torch CUDA tensors -> device pointers,
the current torch stream -> ``cudaStream_t``) and raise ``QpmError`` on a
non-zero status.  Every computation runs in the library's CUDA kernels; there is
no CPU path: if the library cannot be loaded, importing the binding's functions
raises.
"""
import ctypes
import os

from . import build_lib

__all__ = [
    "QpmError", "Problem", "Params", "lib", "qpm_eval", "qpm_eval_packed", "qpm_eval_noalloc", "qpm_eval_shg", "qpm_eval_multi",
    "qpm_release_caches", "qpm_measure_issue_peak", "qpm_measure_latency", "qpm_selfcheck", "qpm_relaxed_saved_floats", "relaxed_saved", "qpm_deff_relaxed_fwd",
    "qpm_deff_relaxed_bwd", "deff_relaxed",
    "qpm_create", "qpm_init", "qpm_step", "qpm_run", "qpm_destroy", "qpm_generation", "qpm_team_of",
    "qpm_instance_shape", "qpm_get_F", "qpm_set_F",
    "qpm_set_batch_cluster",
    "qpm_get_population", "qpm_set_population", "qpm_get_best", "qpm_polish_leaders", "qpm_set_trace", "qpm_set_wait_timeout_ns",
    "qpm_solve", "State", "RUN_LAUNCHES", "RUN_GRAPH", "RUN_PERSISTENT", "RUN_BATCHED",
    "Objective", "qpm_set_objective", "OBJ_THG", "OBJ_SHG", "OBJ_MULTI_THG", "OBJ_MULTI_SHG",
]

RUN_LAUNCHES, RUN_GRAPH, RUN_PERSISTENT, RUN_BATCHED = 0, 1, 2, 3
OBJ_THG, OBJ_SHG, OBJ_MULTI_THG, OBJ_MULTI_SHG = 0, 1, 2, 3
STATUS = {0: "QPM_OK", 1: "QPM_ERR_ARG", 2: "QPM_ERR_CUDA", 3: "QPM_ERR_TIMEOUT",
          4: "QPM_ERR_UNSUPPORTED", 5: "QPM_ERR_STATE"}


class QpmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("kappa1", ctypes.c_double), ("kappa2", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("NP", ctypes.c_int32), ("G", ctypes.c_int32), ("F", ctypes.c_float),
                ("CR", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("gwo_combine", ctypes.c_int32), ("compensated", ctypes.c_int32),
                ("team", ctypes.c_int32), ("f_schedule", ctypes.c_int32)]


class Objective(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("K", ctypes.c_int32),
                ("kappa1", ctypes.c_double * 8), ("kappa2", ctypes.c_double * 8),
                ("G0", ctypes.c_float), ("beta", ctypes.c_float)]


_lib = None
_P = ctypes.c_void_p


def lib(build=True):
    """Load libqpm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = build_lib.build() if build else build_lib.LIB
        if not os.path.exists(path):
            raise OSError(f"libqpm.so not found at {path}")
        L = ctypes.CDLL(path)
        i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        sig = {
            "qpm_last_error": ([], ctypes.c_char_p),
            "qpm_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "qpm_abi_version": ([], i32),
            "qpm_eval": ([_P, _P, i64, i32, _P, _P, i32, _P], ctypes.c_int),
            "qpm_eval_packed": ([_P, _P, i64, i32, _P, _P, i32, _P], ctypes.c_int),
            "qpm_eval_noalloc": ([_P, _P, i64, i32, _P, _P, i32, _P], ctypes.c_int),
            "qpm_eval_shg": ([_P, _P, i64, i32, _P, _P, _P], ctypes.c_int),
            "qpm_eval_multi": ([_P, i32, _P, i64, i32, ctypes.c_float, ctypes.c_float, _P, _P, _P,
                                ctypes.c_size_t, _P], ctypes.c_int),
            "qpm_eval_multi_scratch_bytes": ([i32, i32, i32], ctypes.c_size_t),
            "qpm_release_caches": ([], ctypes.c_int),
            "qpm_measure_issue_peak": ([i32, _P, _P], ctypes.c_int),
            "qpm_measure_latency": ([i32, i32, _P, _P], ctypes.c_int),
            "qpm_selfcheck": ([i32, _P, _P, _P], ctypes.c_int),
            "qpm_relaxed_saved_floats": ([i32], i64),
            "qpm_deff_relaxed_fwd": ([_P, _P, i64, i32, _P, _P, _P, _P], ctypes.c_int),
            "qpm_deff_relaxed_bwd": ([_P, _P, i64, i32, _P, _P, _P, _P, i64, _P], ctypes.c_int),
            "qpm_create": ([_P, _P, i32, _P], ctypes.c_int),
            "qpm_init": ([_P, _P], ctypes.c_int),
            "qpm_step": ([_P, _P], ctypes.c_int),
            "qpm_run": ([_P, i32, i32, _P], ctypes.c_int),
            "qpm_destroy": ([_P], ctypes.c_int),
            "qpm_generation": ([_P, _P], ctypes.c_int),
            "qpm_team_of": ([_P, i32, _P], ctypes.c_int),
            "qpm_instance_shape": ([_P, i32, _P, _P, _P], ctypes.c_int),
            "qpm_get_F": ([_P, i32, _P, _P], ctypes.c_int),
            "qpm_set_F": ([_P, i32, _P, _P], ctypes.c_int),
            "qpm_set_objective": ([_P, i32, _P], ctypes.c_int),
            "qpm_set_batch_cluster": ([_P, i32], ctypes.c_int),
            "qpm_get_population": ([_P, i32, _P, i64, _P, _P, _P], ctypes.c_int),
            "qpm_set_population": ([_P, i32, _P, i64, i32, _P], ctypes.c_int),
            "qpm_get_best": ([_P, i32, _P, _P, _P, _P, _P], ctypes.c_int),
            "qpm_set_trace": ([_P, i32, _P], ctypes.c_int),
            "qpm_set_wait_timeout_ns": ([_P, u64], ctypes.c_int),
            "qpm_solve": ([_P, _P, i32, _P, _P, _P], ctypes.c_int),
            "qpm_polish_leaders": ([_P, i32, i32, ctypes.c_float, ctypes.c_float, _P, _P],
                                   ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise QpmError(status, lib().qpm_last_error().decode(errors="replace"))


def _ptr(t):
    """Device (or host) address of a tensor, None for None."""
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _cuda(t, what, dtypes, min_numel=0, contiguous=True):
    """Check that t is a CUDA tensor on the current device with one of `dtypes`,
    at least `min_numel` elements and (if asked) contiguous, before its address
    goes to the library: a wrong pointer would otherwise become an out-of-bounds
    access on the device instead of a Python error."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: need a torch tensor, got {type(t).__name__}")
    if not t.is_cuda:
        raise ValueError(f"{what}: need a CUDA tensor, got one on {t.device}")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{what}: tensor is on {t.device}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    if t.dtype not in dtypes:
        raise ValueError(f"{what}: need dtype {' or '.join(str(d) for d in dtypes)}, got {t.dtype}")
    if contiguous and not t.is_contiguous():
        raise ValueError(f"{what}: need a contiguous tensor")
    if t.numel() < min_numel:
        raise ValueError(f"{what}: need at least {min_numel} elements, got {t.numel()}")
    return t


def _host(t, what, dtype, min_numel):
    """Same for the host (CPU) buffers of qpm_solve."""
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{what}: need a contiguous CPU tensor of dtype {dtype}")
    if t.numel() < min_numel:
        raise ValueError(f"{what}: need at least {min_numel} elements, got {t.numel()}")
    return t


def _f32():
    import torch
    return (torch.float32,)


def _i32():
    import torch
    return (torch.int32,)


def _rows(t, what, min_cols=0, dtypes=None):
    """(rows, leading dimension) of a row-major 2-D CUDA tensor with unit column
    stride and at least min_cols columns (float32 unless `dtypes` says otherwise)."""
    _cuda(t, what, dtypes or _f32(), contiguous=False)
    if t.dim() != 2 or (t.shape[1] > 1 and t.stride(1) != 1):
        raise ValueError(f"{what}: need a 2-D tensor with contiguous rows")
    if t.shape[1] < min_cols:
        raise ValueError(f"{what}: need at least {min_cols} columns, got {t.shape[1]}")
    if t.shape[0] < 1:
        raise ValueError(f"{what}: need at least one row")
    ld = t.stride(0) if t.shape[0] > 1 else max(t.stride(0), t.shape[1])
    return t.shape[0], ld


def _out(t, what, min_numel, dtypes=None, optional=True):
    """An output buffer: None (where allowed) or a contiguous CUDA tensor."""
    if t is None:
        if not optional:
            raise ValueError(f"{what}: required")
        return None
    return _cuda(t, what, dtypes or _f32(), min_numel)


def _problem(N, kappa1, kappa2):
    return Problem(int(N), float(kappa1), float(kappa2))


def qpm_eval(N, kappa1, kappa2, genes, d_eff, fit=None, compensated=0, stream=None):
    """d_eff (float32 [NP, 2]) and fit of the rows of genes (float32 CUDA [NP, ld])."""
    p = _problem(N, kappa1, kappa2)
    NP, ld = _rows(genes, "genes", N)
    _out(d_eff, "d_eff", 2 * NP, optional=False)
    _out(fit, "fit", NP)
    _check(lib().qpm_eval(ctypes.byref(p), _ptr(genes), ld, NP, _ptr(d_eff), _ptr(fit),
                          int(compensated), _stream(stream)))


def qpm_eval_packed(N, kappa1, kappa2, signs, d_eff, fit=None, compensated=0, stream=None):
    """Same from packed signs (int32/uint32 CUDA [NP, ld_words], bit set -> d = -1)."""
    import torch
    p = _problem(N, kappa1, kappa2)
    NP, ld = _rows(signs, "signs", (int(N) + 31) // 32,
                   (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ()))
    _out(d_eff, "d_eff", 2 * NP, optional=False)
    _out(fit, "fit", NP)
    _check(lib().qpm_eval_packed(ctypes.byref(p), _ptr(signs), ld, NP, _ptr(d_eff), _ptr(fit),
                                 int(compensated), _stream(stream)))


def qpm_eval_noalloc(N, kappa1, kappa2, genes, d_eff, fit=None, compensated=0, stream=None):
    """qpm_eval without any device allocation (fixed 16 MiB scratch inside the library)."""
    p = _problem(N, kappa1, kappa2)
    NP, ld = _rows(genes, "genes", N)
    _out(d_eff, "d_eff", 2 * NP, optional=False)
    _out(fit, "fit", NP)
    _check(lib().qpm_eval_noalloc(ctypes.byref(p), _ptr(genes), ld, NP, _ptr(d_eff), _ptr(fit),
                                  int(compensated), _stream(stream)))


def qpm_measure_issue_peak(kind, stream=None):
    """Measured lane-ops/s of the current device: 0 FFMA, 1 Philox multiply+xor, 2 xor."""
    v = ctypes.c_double()
    _check(lib().qpm_measure_issue_peak(int(kind), ctypes.byref(v), _stream(stream)))
    return v.value


def qpm_measure_latency(kind, ctas=256, stream=None):
    """Measured nanoseconds of 0: one grid barrier of the persistent kernel over `ctas`
    co-resident CTAs; 1: one dependent load served by L2."""
    v = ctypes.c_double()
    _check(lib().qpm_measure_latency(int(kind), int(ctas), ctypes.byref(v), _stream(stream)))
    return v.value


def qpm_selfcheck(kind, stream=None):
    """Exhaustive check of a library arithmetic shortcut against the operation it
    replaces (0: division by 3 of the GWO mean, 1: GWO uniforms built in the
    significand, 2: integer crossover test); returns (mismatches, first_bad)."""
    n = ctypes.c_uint64()
    first = ctypes.c_uint32()
    _check(lib().qpm_selfcheck(int(kind), ctypes.byref(n), ctypes.byref(first), _stream(stream)))
    return n.value, first.value


def qpm_relaxed_saved_floats(N):
    """Floats per row of the saved block the relaxed passes share."""
    return int(lib().qpm_relaxed_saved_floats(int(N)))


def relaxed_saved(B, N, device="cuda"):
    """A saved block for B rows of N domains (float32 [B, qpm_relaxed_saved_floats(N)])."""
    import torch
    return torch.empty((B, qpm_relaxed_saved_floats(N)), dtype=torch.float32, device=device)


def _check_saved(saved, B, N):
    _cuda(saved, "saved", _f32(), B * qpm_relaxed_saved_floats(N))
    if saved.data_ptr() % 16:
        raise ValueError("saved: need a 16-byte aligned block")


def qpm_deff_relaxed_fwd(N, kappa1, kappa2, theta, d_eff, fit, saved, stream=None):
    p = _problem(N, kappa1, kappa2)
    B, ld = _rows(theta, "theta", N)
    _out(d_eff, "d_eff", 2 * B, optional=False)
    _out(fit, "fit", B)
    _check_saved(saved, B, N)
    _check(lib().qpm_deff_relaxed_fwd(ctypes.byref(p), _ptr(theta), ld, B, _ptr(d_eff), _ptr(fit),
                                      _ptr(saved), _stream(stream)))


def qpm_deff_relaxed_bwd(N, kappa1, kappa2, theta, d_eff, saved, grad_fit, grad_theta,
                         stream=None):
    p = _problem(N, kappa1, kappa2)
    B, ld = _rows(theta, "theta", N)
    Bg, ldg = _rows(grad_theta, "grad_theta", N)
    if Bg < B:
        raise ValueError(f"grad_theta: need at least {B} rows, got {Bg}")
    _out(d_eff, "d_eff", 2 * B, optional=False)
    _out(grad_fit, "grad_fit", B)
    _check_saved(saved, B, N)
    _check(lib().qpm_deff_relaxed_bwd(ctypes.byref(p), _ptr(theta), ld, B, _ptr(d_eff),
                                      _ptr(saved), _ptr(grad_fit), _ptr(grad_theta), ldg,
                                      _stream(stream)))


def _relaxed_function():
    import torch

    class QpmDeff(torch.autograd.Function):
        """f = |d_eff|^2 of each row of theta (d = tanh(theta)); backward is the
        library's adjoint kernel (argument marshalling only)."""

        @staticmethod
        def forward(ctx, theta, kappa1, kappa2):
            theta = theta.contiguous()
            B, N = theta.shape
            D = torch.empty((B, 2), dtype=torch.float32, device=theta.device)
            f = torch.empty(B, dtype=torch.float32, device=theta.device)
            S = relaxed_saved(B, N, theta.device)
            qpm_deff_relaxed_fwd(N, kappa1, kappa2, theta, D, f, S)
            ctx.save_for_backward(theta, D, S)
            ctx.kappa = (kappa1, kappa2)
            return f

        @staticmethod
        def backward(ctx, gf):
            theta, D, S = ctx.saved_tensors
            B, N = theta.shape
            g = torch.empty_like(theta)
            qpm_deff_relaxed_bwd(N, ctx.kappa[0], ctx.kappa[1], theta, D, S,
                                 gf.contiguous().to(torch.float32), g)
            return g, None, None

    return QpmDeff


_QpmDeff = None


def deff_relaxed(theta, kappa1, kappa2):
    """Differentiable f = |d_eff|^2 per row of theta (float32 CUDA [B, N])."""
    global _QpmDeff
    if _QpmDeff is None:
        _QpmDeff = _relaxed_function()
    return _QpmDeff.apply(theta, float(kappa1), float(kappa2))


def qpm_eval_shg(N, kappa, genes, e_shg, fit=None, stream=None):
    """SHG field integral of each gene row (dk w = kappa)."""
    p = _problem(N, kappa, 0.0)
    NP, ld = _rows(genes, "genes", N)
    _out(e_shg, "e_shg", 2 * NP, optional=False)
    _out(fit, "fit", NP)
    _check(lib().qpm_eval_shg(ctypes.byref(p), _ptr(genes), ld, NP, _ptr(e_shg), _ptr(fit),
                              _stream(stream)))


def qpm_eval_multi(N, kappas, genes, G0, beta, objective, d_eff=None, stream=None):
    """Multi-wavelength objective for the (kappa1, kappa2) pairs in `kappas`."""
    import torch
    K = len(kappas)
    probs = (Problem * K)(*[_problem(N, k1, k2) for k1, k2 in kappas])
    NP, ld = _rows(genes, "genes", N)
    _out(objective, "objective", NP, optional=False)
    _out(d_eff, "d_eff", 2 * K * NP)
    nbytes = lib().qpm_eval_multi_scratch_bytes(K, N, NP)
    scratch = torch.empty(max(1, nbytes), dtype=torch.uint8, device=genes.device)
    _check(lib().qpm_eval_multi(probs, K, _ptr(genes), ld, NP, float(G0), float(beta),
                                _ptr(d_eff), _ptr(objective), _ptr(scratch), nbytes,
                                _stream(stream)))


def qpm_release_caches():
    _check(lib().qpm_release_caches())


def qpm_create(problems, params):
    """problems: list of (N, kappa1, kappa2); params: list of Params (same length)."""
    n = len(problems)
    pa = (Problem * n)(*[_problem(*p) for p in problems])
    qa = (Params * n)(*params)
    h = ctypes.c_void_p()
    _check(lib().qpm_create(pa, qa, n, ctypes.byref(h)))
    return h


def qpm_init(st, stream=None):
    _check(lib().qpm_init(st, _stream(stream)))


def qpm_step(st, stream=None):
    _check(lib().qpm_step(st, _stream(stream)))


def qpm_run(st, generations, mode=RUN_GRAPH, stream=None):
    _check(lib().qpm_run(st, int(generations), int(mode), _stream(stream)))


def qpm_destroy(st):
    _check(lib().qpm_destroy(st))


def qpm_generation(st):
    g = ctypes.c_int32()
    _check(lib().qpm_generation(st, ctypes.byref(g)))
    return g.value


def qpm_team_of(st, inst=0):
    t = ctypes.c_int32()
    _check(lib().qpm_team_of(st, int(inst), ctypes.byref(t)))
    return t.value


def qpm_set_batch_cluster(st, ctas):
    """CTAs per thread-block cluster of the batched form (1, 2, 4 or 8)."""
    _check(lib().qpm_set_batch_cluster(st, int(ctas)))


def qpm_instance_shape(st, inst=0):
    """(N, NP, G) of instance `inst`."""
    n, p, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().qpm_instance_shape(st, int(inst), ctypes.byref(n), ctypes.byref(p), ctypes.byref(g)))
    return n.value, p.value, g.value


def qpm_set_objective(st, inst, kind, kappas=(), G0=0.0, beta=0.0):
    """The fitness instance `inst` optimises (before qpm_init): OBJ_THG, OBJ_SHG, or a
    multi-wavelength kind over the (kappa1, kappa2) pairs in `kappas` (Sec. 5)."""
    if len(kappas) > 8:
        raise ValueError("kappas: at most 8 pairs")
    o = Objective(int(kind), len(kappas), (ctypes.c_double * 8)(*[float(k[0]) for k in kappas]),
                  (ctypes.c_double * 8)(*[float(k[1]) for k in kappas]), float(G0), float(beta))
    _check(lib().qpm_set_objective(st, int(inst), ctypes.byref(o)))


def qpm_get_F(st, inst=0, F_out=None, stream=None):
    """F of every generation of instance `inst` (float32 CUDA [G + 1]; allocated when
    F_out is None)."""
    import torch
    _, _, G = qpm_instance_shape(st, inst)
    if F_out is None:
        F_out = torch.empty(G + 1, dtype=torch.float32, device="cuda")
    _out(F_out, "F_out", G + 1, optional=False)
    _check(lib().qpm_get_F(st, int(inst), _ptr(F_out), _stream(stream)))
    return F_out


def qpm_set_F(st, inst, F_in, stream=None):
    """Restore the F history of instance `inst` (float32 CUDA [G + 1], from qpm_get_F)."""
    _, _, G = qpm_instance_shape(st, inst)
    _out(F_in, "F_in", G + 1, optional=False)
    _check(lib().qpm_set_F(st, int(inst), _ptr(F_in), _stream(stream)))


def qpm_get_population(st, inst, genes_out=None, fit_out=None, d_eff_out=None, stream=None):
    N, NP, _ = qpm_instance_shape(st, inst)
    ld = 0
    if genes_out is not None:
        rows, ld = _rows(genes_out, "genes_out", N)
        if rows < NP:
            raise ValueError(f"genes_out: need {NP} rows, got {rows}")
    _out(fit_out, "fit_out", NP)
    _out(d_eff_out, "d_eff_out", 2 * NP)
    _check(lib().qpm_get_population(st, int(inst), _ptr(genes_out), ld, _ptr(fit_out),
                                    _ptr(d_eff_out), _stream(stream)))


def qpm_set_population(st, inst, genes, generation, stream=None):
    N, NP, _ = qpm_instance_shape(st, inst)
    rows, ld = _rows(genes, "genes", N)
    if rows < NP:
        raise ValueError(f"genes: need {NP} rows, got {rows}")
    _check(lib().qpm_set_population(st, int(inst), _ptr(genes), ld, int(generation),
                                    _stream(stream)))


def qpm_get_best(st, inst, genes_out=None, d_eff64_out=None, fit_out=None, index_out=None,
                 stream=None):
    import torch
    N, _, _ = qpm_instance_shape(st, inst)
    _out(genes_out, "genes_out", N)
    _out(d_eff64_out, "d_eff64_out", 2, (torch.float64,))
    _out(fit_out, "fit_out", 1)
    _out(index_out, "index_out", 1, _i32())
    _check(lib().qpm_get_best(st, int(inst), _ptr(genes_out), _ptr(d_eff64_out), _ptr(fit_out),
                              _ptr(index_out), _stream(stream)))


def qpm_polish_leaders(st, inst=0, steps=8, lr=0.5, tau=3.0, accepted_out=None, stream=None):
    _out(accepted_out, "accepted_out", 3, _i32())
    _check(lib().qpm_polish_leaders(st, int(inst), int(steps), float(lr), float(tau),
                                    _ptr(accepted_out), _stream(stream)))


def qpm_set_trace(st, inst, trace):
    if trace is not None:
        _, NP, G = qpm_instance_shape(st, inst)
        _out(trace, "trace", NP * (1 + 2 * G))
    _check(lib().qpm_set_trace(st, int(inst), _ptr(trace)))


def qpm_set_wait_timeout_ns(st, ns):
    _check(lib().qpm_set_wait_timeout_ns(st, int(ns)))


def qpm_solve(N, kappa1, kappa2, params, mode, best_genes_host, best_deff64_host,
              best_fit_host=None):
    """End to end with host (CPU) tensors; synchronous."""
    import torch
    p = _problem(N, kappa1, kappa2)
    _host(best_genes_host, "best_genes_host", torch.float32, N)
    _host(best_deff64_host, "best_deff64_host", torch.float64, 2)
    if best_fit_host is not None:
        _host(best_fit_host, "best_fit_host", torch.float32, 1)
    _check(lib().qpm_solve(ctypes.byref(p), ctypes.byref(params), int(mode),
                           _ptr(best_genes_host), _ptr(best_deff64_host), _ptr(best_fit_host)))


class State:
    """Owning wrapper of a qpm_state (destroyed with the object or on close())."""

    def __init__(self, problems, params):
        self.problems = list(problems)
        self.params = list(params)
        self.h = qpm_create(self.problems, self.params)

    def close(self):
        if self.h is not None and self.h.value:
            qpm_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, stream=None):
        qpm_init(self.h, stream)

    def step(self, stream=None):
        qpm_step(self.h, stream)

    def run(self, generations, mode=RUN_GRAPH, stream=None):
        qpm_run(self.h, generations, mode, stream)

    def set_batch_cluster(self, ctas):
        qpm_set_batch_cluster(self.h, ctas)

    def set_objective(self, kind, kappas=(), G0=0.0, beta=0.0, inst=0):
        qpm_set_objective(self.h, inst, kind, kappas, G0, beta)
        if kind >= OBJ_MULTI_THG:  # the first pair becomes the instance's problem
            N = self.problems[inst][0]
            self.problems[inst] = (N, float(kappas[0][0]), float(kappas[0][1]))

    @property
    def generation(self):
        return qpm_generation(self.h)

    def population(self, inst=0):
        import torch
        N = self.problems[inst][0]
        NP = self.params[inst].NP
        X = torch.empty((NP, N), dtype=torch.float32, device="cuda")
        f = torch.empty(NP, dtype=torch.float32, device="cuda")
        D = torch.empty((NP, 2), dtype=torch.float32, device="cuda")
        qpm_get_population(self.h, inst, X, f, D)
        return X, f, D

    def best(self, inst=0):
        import torch
        N = self.problems[inst][0]
        x = torch.empty(N, dtype=torch.float32, device="cuda")
        d64 = torch.empty(2, dtype=torch.float64, device="cuda")
        f = torch.empty(1, dtype=torch.float32, device="cuda")
        idx = torch.empty(1, dtype=torch.int32, device="cuda")
        qpm_get_best(self.h, inst, x, d64, f, idx)
        return x, d64, f, idx
