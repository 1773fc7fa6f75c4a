"""Python binding of the PSMS GB300 library (C ABI in ``include/psms.h``).

Argument marshalling only: every function below forwards to the ``psms_*``
entry point of the same name in ``_lib/libpsms.so``.  Device buffers are
passed as CUDA torch tensors (their ``data_ptr()``); host results come back as
Python / numpy values.  There is no fallback: if the shared library is
missing or a call fails, an exception is raised.
"""
import ctypes
import os

import numpy as np

__all__ = [
    "PsmsError", "Context", "load_library",
    "psms_create", "psms_destroy", "psms_set_stream", "psms_geometry_info",
    "psms_gauge_init", "psms_gauge_set", "psms_gauge_get", "psms_gauge_copy", "psms_plaquette",
    "psms_gauge_sweep", "psms_gauge_translate", "psms_spinor_bytes", "psms_spinor_import",
    "psms_spinor_export", "psms_dw_apply", "psms_solve", "psms_logdet_ratio", "psms_filter_step",
    "psms_profile_enable", "psms_profile_read", "psms_block_solve_noalloc", "psms_domain_features",
    "psms_mlp_init", "psms_mlp_param_count", "psms_mlp_params", "psms_mlp_predict", "psms_mlp_grad",
    "psms_mlp_train", "psms_block_plan_create", "psms_block_plan_run", "psms_block_plan_schedule",
    "psms_block_plan_destroy", "BlockPlan", "psms_autotune", "psms_profile_read_block",
    "psms_domain_features_pair", "psms_checkpoint_save", "psms_checkpoint_load",
    "psms_relative_gauge_fix", "psms_profile_block_launches", "psms_hop_variant", "psms_full_solver",
    "psms_inner_reduction", "psms_shared_links",
    "psms_block_krylov", "SOLVER_CGNR", "SOLVER_BICGSTAB", "psms_level_covariance", "psms_level_coefficients",
    "psms_hyp_smear", "psms_hyp_block_action", "psms_block_action_change",
    "PREC_F64", "PREC_F32", "PREC_BF16", "OP_FULL", "OP_BLOCKS", "ACTIVE_BLOCKS", "ACTIVE_ALL",
    "LEVEL_BLOCK", "LEVEL_GLOBAL", "LEVEL_SUB", "EST_INTERP", "EST_INDEPENDENT", "psms_set_outer_blocks",
    "LEVEL_OUTER_GLOBAL", "psms_filter_record", "psms_max_chunk", "REC_H", "REC_DELTA_HYP", "REC_ACCEPT_BLOCK",
    "REC_DELTA_SUB", "REC_ACCEPT_SUB", "psms_block_logdet", "psms_scratch_bytes",
]

PREC_F64, PREC_F32, PREC_BF16 = 0, 1, 2
OP_FULL, OP_BLOCKS = -1, -2
ACTIVE_BLOCKS, ACTIVE_ALL = 0, 1
LEVEL_BLOCK, LEVEL_GLOBAL, LEVEL_SUB, LEVEL_OUTER_GLOBAL = 1, 2, 4, 6
REC_H, REC_DELTA_HYP, REC_ACCEPT_BLOCK, REC_DELTA_SUB, REC_ACCEPT_SUB = 0, 1, 2, 3, 4
EST_INTERP, EST_INDEPENDENT = 0, 1

STATUS = {0: "PSMS_OK", 1: "PSMS_EINVAL", 2: "PSMS_ENOMEM", 3: "PSMS_ECUDA", 4: "PSMS_ENOCONV",
          5: "PSMS_ETIMEOUT", 6: "PSMS_ESPECTRUM", 7: "PSMS_EHEATBATH"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libpsms.so")


class PsmsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class LatticeDesc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("block", ctypes.c_int * 4), ("kappa", ctypes.c_double),
                ("n_fields", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_longlong),
                ("true_residual", ctypes.c_double), ("n_systems", ctypes.c_int)]


class RelGFParams(ctypes.Structure):
    _fields_ = [("alpha0", ctypes.c_double), ("alpha_min", ctypes.c_double), ("dalpha", ctypes.c_double),
                ("theta_tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("prec", ctypes.c_int)]


def _relgf(alpha0=0.15, alpha_min=0.10, dalpha=0.01, theta_tol=1e-3, max_iter=1000, prec=None):
    return RelGFParams(float(alpha0), float(alpha_min), float(dalpha), float(theta_tol), int(max_iter),
                       int(PREC_F32 if prec is None else prec))


class FilterParams(ctypes.Structure):
    _fields_ = [("beta0", ctypes.c_double), ("n_iter", ctypes.c_int), ("n_or", ctypes.c_int),
                ("n_block", ctypes.c_int), ("beta_block", ctypes.c_double), ("n_global", ctypes.c_int),
                ("beta_global", ctypes.c_double), ("global_level", ctypes.c_int), ("tol", ctypes.c_double),
                ("inner_prec", ctypes.c_int), ("seed", ctypes.c_uint64), ("step", ctypes.c_uint64),
                ("learned", ctypes.c_int), ("gauge_fix", ctypes.c_int), ("relgf", RelGFParams),
                ("proposal_field", ctypes.c_int), ("translate", ctypes.c_int), ("hyp_level", ctypes.c_int),
                ("hyp_beta", ctypes.c_double * 2), ("beta_block_hyp", ctypes.c_double),
                ("beta_global_hyp", ctypes.c_double), ("n_sub", ctypes.c_int), ("beta_sub", ctypes.c_double),
                ("exact_block", ctypes.c_int), ("beta_block_det", ctypes.c_double),
                ("beta_global_blockdet", ctypes.c_double)]


class FilterResult(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int), ("n_accept_blocks", ctypes.c_int), ("accept_global", ctypes.c_int),
                ("shift", ctypes.c_int * 4), ("delta_global", ctypes.c_double),
                ("delta_block_sum", ctypes.c_double), ("solver_iters", ctypes.c_longlong),
                ("hb_failed", ctypes.c_int), ("n_accept_learned", ctypes.c_int), ("gf_steps", ctypes.c_longlong),
                ("n_accept_hyp", ctypes.c_int), ("n_accept_sub", ctypes.c_int)]


class BlockProblem(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("field", ctypes.c_int), ("n_rhs", ctypes.c_int),
                ("b_dev", ctypes.c_void_p), ("x_dev", ctypes.c_void_p)]


class TrainParams(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("weight_decay", ctypes.c_double), ("normalise", ctypes.c_int), ("seed", ctypes.c_uint64)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_U64 = ctypes.c_uint64
_SIGS = {
    "psms_create": [ctypes.POINTER(LatticeDesc), ctypes.POINTER(_P)],
    "psms_destroy": [_P],
    "psms_set_stream": [_P, _P],
    "psms_geometry_info": [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                           ctypes.POINTER(ctypes.c_longlong)],
    "psms_gauge_init": [_P, _I, _D, _U64],
    "psms_gauge_set": [_P, _I, _P],
    "psms_gauge_get": [_P, _I, _P],
    "psms_gauge_copy": [_P, _I, _I],
    "psms_plaquette": [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "psms_gauge_sweep": [_P, _I, _I, _I, _I, _D, _U64, _U64, ctypes.POINTER(_I)],
    "psms_gauge_translate": [_P, _I, ctypes.POINTER(_I)],
    "psms_spinor_import": [_P, _P, _P, _I],
    "psms_spinor_export": [_P, _P, _P, _I],
    "psms_dw_apply": [_P, _I, _I, _P, _P, _I],
    "psms_solve": [_P, _I, _I, _P, _P, _D, _I, _I, ctypes.POINTER(SolveInfo)],
    "psms_logdet_ratio": [_P, _I, _I, _I, _I, _I, _U64, _U64, _D, _I, ctypes.POINTER(_D)],
    "psms_filter_step": [_P, _I, ctypes.POINTER(FilterParams), ctypes.POINTER(FilterResult),
                         ctypes.POINTER(_D), ctypes.POINTER(_I)],
    "psms_block_solve_noalloc": [_P, _I, _I, _P, _P, _D, _I, ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(_D)],
    "psms_block_plan_create": [ctypes.POINTER(BlockProblem), _I, _D, _I, _I, ctypes.POINTER(_P)],
    "psms_block_plan_run": [_P, _P, ctypes.POINTER(SolveInfo)],
    "psms_block_plan_schedule": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D)],
    "psms_block_plan_destroy": [_P],
    "psms_domain_features": [_P, _I, _P],
    "psms_domain_features_pair": [_P, _I, _I, _P],
    "psms_mlp_init": [_P, _U64],
    "psms_mlp_params": [_P, ctypes.POINTER(ctypes.c_float), _I],
    "psms_mlp_predict": [_P, _P, _I, _P],
    "psms_mlp_grad": [_P, _P, _P, _I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_D)],
    "psms_mlp_train": [_P, _P, _P, _I, ctypes.POINTER(TrainParams), ctypes.POINTER(_D)],
    "psms_autotune": [_P, _I, _I],
    "psms_checkpoint_save": [_P, _I, ctypes.c_char_p, _U64, _U64],
    "psms_relative_gauge_fix": [_P, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P],
    "psms_profile_block_launches": [_P, _I, _P, _P, _P],
    "psms_hop_variant": [_P, _I, _P],
    "psms_full_solver": [_P, _I],
    "psms_inner_reduction": [_P, ctypes.c_double],
    "psms_shared_links": [_P, _I],
    "psms_block_krylov": [_P, _I],
    "psms_checkpoint_load": [_P, _I, ctypes.c_char_p, ctypes.POINTER(_U64), ctypes.POINTER(_U64)],
    "psms_profile_read_block": [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "psms_profile_enable": [_P, _I],
    "psms_profile_read": [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "psms_level_covariance": [_P, ctypes.c_longlong, _I, _P],
    "psms_hyp_smear": [_P, _I, _P, _P],
    "psms_block_action_change": [_P, _I, _I, _P],
    "psms_set_outer_blocks": [_P, _P],
    "psms_hyp_block_action": [_P, _I, _P, _P],
    "psms_level_coefficients": [_I, _P, _P, _P, _P],
    "psms_filter_record": [_P, _I, _P, _I, ctypes.POINTER(_I)],
    "psms_max_chunk": [_P, _I],
    "psms_block_logdet": [_P, _I, _P],
    "psms_scratch_bytes": [_P, ctypes.POINTER(ctypes.c_size_t)],
}

_lib = None


def load_library(path=LIB_PATH):
    """Load ``libpsms.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1204_1306_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.psms_last_error.argtypes = [_P]
    lib.psms_last_error.restype = ctypes.c_char_p
    lib.psms_spinor_bytes.argtypes = [_P, _I]
    lib.psms_spinor_bytes.restype = ctypes.c_size_t
    lib.psms_mlp_param_count.argtypes = []
    lib.psms_mlp_param_count.restype = ctypes.c_size_t
    lib.psms_kernel_launches.argtypes = []
    lib.psms_kernel_launches.restype = ctypes.c_longlong
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_cuda:
            raise ValueError("device buffers must be CUDA tensors")
        if not t.is_contiguous():
            raise ValueError("device buffers must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(int(t))


class Context:
    """Owns one ``psms_ctx``."""

    def __init__(self, dims, block, kappa, n_fields=4):
        self.lib = load_library()
        d = LatticeDesc((ctypes.c_int * 4)(*dims), (ctypes.c_int * 4)(*block), float(kappa), int(n_fields))
        h = _P()
        st = self.lib.psms_create(ctypes.byref(d), ctypes.byref(h))
        if st:
            raise PsmsError(st, "psms_create failed")
        self.handle = h
        self.dims = tuple(dims)
        self.block = tuple(block)
        self.kappa = kappa
        self.n_fields = n_fields
        self.V = int(np.prod(dims))
        self.outer = None  # outer blocks of the recursive decomposition

    def check(self, st):
        if st:
            raise PsmsError(st, self.lib.psms_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.psms_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def psms_create(dims, block, kappa, n_fields=4):
    return Context(dims, block, kappa, n_fields)


def psms_destroy(ctx):
    ctx.close()


def psms_set_stream(ctx, stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    raw = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    ctx.check(ctx.lib.psms_set_stream(ctx.handle, _P(raw)))


def psms_geometry_info(ctx):
    a, b, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    ctx.check(ctx.lib.psms_geometry_info(ctx.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def psms_gauge_init(ctx, field, eps, seed):
    ctx.check(ctx.lib.psms_gauge_init(ctx.handle, field, float(eps), int(seed)))


def psms_gauge_set(ctx, field, links_dev):
    ctx.check(ctx.lib.psms_gauge_set(ctx.handle, field, _ptr(links_dev)))


def psms_gauge_get(ctx, field, links_dev):
    ctx.check(ctx.lib.psms_gauge_get(ctx.handle, field, _ptr(links_dev)))


def psms_gauge_copy(ctx, dst, src):
    ctx.check(ctx.lib.psms_gauge_copy(ctx.handle, dst, src))


def psms_plaquette(ctx, field):
    a, b = _D(), _D()
    ctx.check(ctx.lib.psms_plaquette(ctx.handle, field, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def psms_gauge_sweep(ctx, field, active_set, n_iter, n_or, beta, seed, sweep0):
    f = _I()
    ctx.check(ctx.lib.psms_gauge_sweep(ctx.handle, field, active_set, n_iter, n_or, float(beta), int(seed),
                                       int(sweep0), ctypes.byref(f)))
    return f.value


def psms_gauge_translate(ctx, field, shift):
    ctx.check(ctx.lib.psms_gauge_translate(ctx.handle, field, (_I * 4)(*shift)))


def psms_spinor_bytes(ctx, prec):
    return int(ctx.lib.psms_spinor_bytes(ctx.handle, prec))


def psms_spinor_import(ctx, canonical_dev, native_dev, prec):
    ctx.check(ctx.lib.psms_spinor_import(ctx.handle, _ptr(canonical_dev), _ptr(native_dev), prec))


def psms_spinor_export(ctx, native_dev, canonical_dev, prec):
    ctx.check(ctx.lib.psms_spinor_export(ctx.handle, _ptr(native_dev), _ptr(canonical_dev), prec))


def psms_dw_apply(ctx, field, op, in_dev, out_dev, prec):
    ctx.check(ctx.lib.psms_dw_apply(ctx.handle, field, op, _ptr(in_dev), _ptr(out_dev), prec))


def psms_solve(ctx, field, op, b_dev, x_dev, tol, maxit, inner_prec):
    info = SolveInfo()
    ctx.check(ctx.lib.psms_solve(ctx.handle, field, op, _ptr(b_dev), _ptr(x_dev), float(tol), int(maxit),
                                 inner_prec, ctypes.byref(info)))
    return {"outer_iters": info.outer_iters, "inner_iters": info.inner_iters,
            "true_residual": info.true_residual, "n_systems": info.n_systems}


def psms_logdet_ratio(ctx, level, field_old, field_new, n, mode, seed, counter, tol, inner_prec):
    nb = int(np.prod([d // b for d, b in zip(ctx.dims, ctx.block)]))
    if level == LEVEL_SUB:
        outer = getattr(ctx, "outer", None)
        if outer is None:
            raise ValueError("LEVEL_SUB needs outer blocks (psms_set_outer_blocks)")
        nb = int(np.prod([d // b for d, b in zip(ctx.dims, outer)]))
    size = nb * n if level in (LEVEL_BLOCK, LEVEL_SUB) else n
    out = (_D * size)()
    ctx.check(ctx.lib.psms_logdet_ratio(ctx.handle, level, field_old, field_new, int(n), mode, int(seed),
                                        int(counter), float(tol), inner_prec, out))
    a = np.frombuffer(out, dtype=np.float64).copy()
    return a.reshape(nb, n) if level in (LEVEL_BLOCK, LEVEL_SUB) else a


def psms_filter_record(ctx, what):
    """Per-block record `what` (REC_*) of the last psms_filter_step."""
    n = ctypes.c_int()
    nb = int(np.prod([d // b for d, b in zip(ctx.dims, ctx.block)]))
    outer = getattr(ctx, "outer", None)
    no = nb if outer is None else int(np.prod([d // b for d, b in zip(ctx.dims, outer)]))
    out = np.zeros(max(nb, no), dtype=np.float64)
    ctx.check(ctx.lib.psms_filter_record(ctx.handle, int(what), out.ctypes.data, len(out), ctypes.byref(n)))
    return out[:n.value].copy()


def psms_block_logdet(ctx, field):
    """ln|det D_b| of every block (lexicographic block index), exact."""
    nb = int(psms_geometry_info(ctx)[0])
    out = np.empty(nb, dtype=np.float64)
    ctx.check(ctx.lib.psms_block_logdet(ctx.handle, field, out.ctypes.data))
    return out


def psms_scratch_bytes(ctx):
    """Bytes of device scratch the context holds."""
    v = ctypes.c_size_t()
    ctx.check(ctx.lib.psms_scratch_bytes(ctx.handle, ctypes.byref(v)))
    return v.value


def psms_max_chunk(ctx, n):
    """Cap on interpolation steps batched per estimator launch (0: automatic)."""
    ctx.check(ctx.lib.psms_max_chunk(ctx.handle, int(n)))


def psms_set_outer_blocks(ctx, outer):
    """Outer blocks of the recursive decomposition (None: off)."""
    arr = None if outer is None else (_I * 4)(*[int(v) for v in outer])
    ctx.check(ctx.lib.psms_set_outer_blocks(ctx.handle, arr))
    ctx.outer = None if outer is None else tuple(int(v) for v in outer)


def psms_filter_step(ctx, field, *, beta0, n_iter=1, n_or=0, n_block=4, n_global=4, beta_block=0.0,
                     beta_global=0.0, global_level=True, tol=1e-10, inner_prec=PREC_F64, seed=0, step=0,
                     learned=False, gauge_fix=None, proposal_field=-1, translate=True, hyp_level=None,
                     beta_block_hyp=0.0, beta_global_hyp=0.0, n_sub=0, beta_sub=0.0, exact_block=False,
                     beta_block_det=1.0, beta_global_blockdet=0.0):
    """gauge_fix: None (off) or a dict of relative gauge-fixing parameters
    (alpha0, alpha_min, dalpha, theta_tol, max_iter, prec; {} = defaults).
    proposal_field: -1 (domain sweep) or the slot of an external proposal.
    hyp_level: None (off) or the coefficients (b0, b1) of the HYP level."""
    hb = (0.0, 0.0) if hyp_level is None else tuple(float(v) for v in hyp_level)
    p = FilterParams(float(beta0), int(n_iter), int(n_or), int(n_block), float(beta_block), int(n_global),
                     float(beta_global), int(bool(global_level)), float(tol), int(inner_prec), int(seed), int(step),
                     int(bool(learned)), int(gauge_fix is not None), _relgf(**(gauge_fix or {})),
                     int(proposal_field), int(bool(translate)), int(hyp_level is not None), (_D * 2)(*hb),
                     float(beta_block_hyp), float(beta_global_hyp), int(n_sub), float(beta_sub),
                     int(bool(exact_block)), float(beta_block_det), float(beta_global_blockdet))
    r = FilterResult()
    nb = int(np.prod([d // b for d, b in zip(ctx.dims, ctx.block)]))
    db = (_D * nb)()
    ab = (_I * nb)()
    ctx.check(ctx.lib.psms_filter_step(ctx.handle, field, ctypes.byref(p), ctypes.byref(r), db, ab))
    return {"n_blocks": r.n_blocks, "n_accept_blocks": r.n_accept_blocks, "accept_global": bool(r.accept_global),
            "shift": tuple(r.shift), "delta_global": r.delta_global, "delta_block_sum": r.delta_block_sum,
            "solver_iters": r.solver_iters, "hb_failed": r.hb_failed, "n_accept_learned": r.n_accept_learned,
            "gf_steps": r.gf_steps, "n_accept_hyp": r.n_accept_hyp, "n_accept_sub": r.n_accept_sub,
            "delta_block": np.frombuffer(db, dtype=np.float64).copy(),
            "accept_block": np.frombuffer(ab, dtype=np.int32).astype(bool)}


def psms_block_solve_noalloc(ctx, field, op, b_dev, x_dev, tol, maxit):
    """Block solve with the library's static scratch (no device allocation)."""
    it, res = ctypes.c_longlong(), _D()
    ctx.check(ctx.lib.psms_block_solve_noalloc(ctx.handle, field, op, _ptr(b_dev), _ptr(x_dev), float(tol),
                                               int(maxit), ctypes.byref(it), ctypes.byref(res)))
    return {"inner_iters": it.value, "true_residual": res.value}


class BlockPlan:
    """Owns a psms_block_plan (see psms_block_plan_create)."""

    def __init__(self, problems, tol, maxit, inner_prec):
        self.lib = load_library()
        self.keep = problems
        arr = (BlockProblem * len(problems))()
        for i, (ctx, field, n_rhs, b, x) in enumerate(problems):
            arr[i] = BlockProblem(ctx.handle, int(field), int(n_rhs), _ptr(b), _ptr(x))
        h = _P()
        st = self.lib.psms_block_plan_create(arr, len(problems), float(tol), int(maxit), int(inner_prec),
                                             ctypes.byref(h))
        if st:
            raise PsmsError(st, self.lib.psms_last_error(problems[0][0].handle).decode())
        self.handle = h

    def run(self, stream=None):
        raw = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        info = SolveInfo()
        st = self.lib.psms_block_plan_run(self.handle, _P(raw), ctypes.byref(info))
        if st:
            raise PsmsError(st, "psms_block_plan_run failed")
        return {"inner_iters": info.inner_iters, "true_residual": info.true_residual, "n_systems": info.n_systems}

    def schedule(self):
        a, b, c = _I(), _I(), _D()
        self.lib.psms_block_plan_schedule(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return {"ctas": a.value, "order": b.value, "tuned_ms": c.value}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.psms_block_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def psms_block_plan_create(problems, tol, maxit, inner_prec):
    """problems: list of (ctx, field, n_rhs, b_dev, x_dev)."""
    return BlockPlan(problems, tol, maxit, inner_prec)


def psms_block_plan_run(plan, stream=None):
    return plan.run(stream)


def psms_block_plan_schedule(plan):
    return plan.schedule()


def psms_block_plan_destroy(plan):
    plan.close()


def psms_domain_features(ctx, field, out_dev):
    ctx.check(ctx.lib.psms_domain_features(ctx.handle, field, _ptr(out_dev)))


def psms_domain_features_pair(ctx, field_old, field_new, out_dev):
    ctx.check(ctx.lib.psms_domain_features_pair(ctx.handle, field_old, field_new, _ptr(out_dev)))


def psms_mlp_init(ctx, seed):
    ctx.check(ctx.lib.psms_mlp_init(ctx.handle, int(seed)))


def psms_mlp_param_count():
    return int(load_library().psms_mlp_param_count())


def psms_mlp_params(ctx, values=None):
    """Get (values None) or set the flat FP32 parameter block."""
    n = psms_mlp_param_count()
    buf = (ctypes.c_float * n)()
    if values is not None:
        buf[:] = [float(v) for v in np.asarray(values, dtype=np.float32)]
        ctx.check(ctx.lib.psms_mlp_params(ctx.handle, buf, 1))
        return None
    ctx.check(ctx.lib.psms_mlp_params(ctx.handle, buf, 0))
    return np.frombuffer(buf, dtype=np.float32).copy()


def psms_mlp_predict(ctx, feats_dev, n, h_dev):
    ctx.check(ctx.lib.psms_mlp_predict(ctx.handle, _ptr(feats_dev), int(n), _ptr(h_dev)))


def psms_mlp_grad(ctx, feats_dev, labels_dev, n):
    n_train = psms_mlp_param_count() - 129
    g = (ctypes.c_float * n_train)()
    loss = _D()
    ctx.check(ctx.lib.psms_mlp_grad(ctx.handle, _ptr(feats_dev), _ptr(labels_dev), int(n), g, ctypes.byref(loss)))
    return loss.value, np.frombuffer(g, dtype=np.float32).copy()


def psms_mlp_train(ctx, feats_dev, labels_dev, n, *, epochs=10, batch=256, lr=1e-3, beta1=0.9, beta2=0.999,
                   eps=1e-8, weight_decay=1e-4, normalise=True, seed=0):
    tp = TrainParams(int(epochs), int(batch), float(lr), float(beta1), float(beta2), float(eps), float(weight_decay),
                     int(bool(normalise)), int(seed))
    out = (_D * epochs)()
    ctx.check(ctx.lib.psms_mlp_train(ctx.handle, _ptr(feats_dev), _ptr(labels_dev), int(n), ctypes.byref(tp), out))
    return np.frombuffer(out, dtype=np.float64).copy()


def psms_profile_read_block(ctx):
    n, ms, by = ctypes.c_longlong(), _D(), _D()
    ctx.check(ctx.lib.psms_profile_read_block(ctx.handle, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
    return n.value, ms.value, by.value


SOLVER_CGNR, SOLVER_BICGSTAB = 0, 1


def psms_full_solver(ctx, kind):
    """Inner Krylov method of whole-lattice solves: SOLVER_CGNR or SOLVER_BICGSTAB."""
    ctx.check(ctx.lib.psms_full_solver(ctx.handle, int(kind)))


def psms_inner_reduction(ctx, delta):
    """Inner relative reduction per defect-correction step of whole-lattice
    solves (0 restores the defaults)."""
    ctx.check(ctx.lib.psms_inner_reduction(ctx.handle, float(delta)))


def psms_shared_links(ctx, on):
    """Shared-endpoint FP32 links in the estimators' whole-lattice solves
    (default on)."""
    ctx.check(ctx.lib.psms_shared_links(ctx.handle, int(on)))


def psms_block_krylov(ctx, kind):
    """Inner Krylov method of block solves: SOLVER_CGNR or SOLVER_BICGSTAB."""
    ctx.check(ctx.lib.psms_block_krylov(ctx.handle, int(kind)))


def psms_hop_variant(ctx, variant):
    """Force Wilson-hop variant `variant` (-1: autotuned); returns the count."""
    n = _I()
    ctx.check(ctx.lib.psms_hop_variant(ctx.handle, int(variant), ctypes.byref(n)))
    return n.value


def psms_profile_block_launches(ctx, n_max=4096):
    """[(ms, algorithmic bytes)] of the block-solver launches since profiling
    was enabled, in launch order."""
    n = _I()
    ms, by = (_D * n_max)(), (_D * n_max)()
    ctx.check(ctx.lib.psms_profile_block_launches(ctx.handle, int(n_max), ctypes.byref(n), ms, by))
    return [(ms[i], by[i]) for i in range(n.value)]


def psms_relative_gauge_fix(ctx, field_old, field_new, out_old, out_new, g_dev=None, **kw):
    """Relative gauge fixing of (field_old, field_new) into (out_old, out_new);
    returns per-block steps, alpha, theta, swapped (lexicographic order)."""
    nb = int(np.prod([d // b for d, b in zip(ctx.dims, ctx.block)]))
    st, al, th, sw = (_I * nb)(), (_D * nb)(), (_D * nb)(), (_I * nb)()
    p = _relgf(**kw)
    ctx.check(ctx.lib.psms_relative_gauge_fix(ctx.handle, field_old, field_new, out_old, out_new, ctypes.byref(p),
                                              st, al, th, sw, None if g_dev is None else _ptr(g_dev)))
    return {"steps": np.frombuffer(st, dtype=np.int32).copy(), "alpha": np.frombuffer(al, dtype=np.float64).copy(),
            "theta": np.frombuffer(th, dtype=np.float64).copy(),
            "swapped": np.frombuffer(sw, dtype=np.int32).astype(bool)}


def psms_checkpoint_save(ctx, field, path, step, seed):
    ctx.check(ctx.lib.psms_checkpoint_save(ctx.handle, field, str(path).encode(), int(step), int(seed)))


def psms_checkpoint_load(ctx, field, path):
    st, sd = _U64(), _U64()
    ctx.check(ctx.lib.psms_checkpoint_load(ctx.handle, field, str(path).encode(), ctypes.byref(st), ctypes.byref(sd)))
    return st.value, sd.value


def psms_autotune(ctx, enable=True, block_variant=-1):
    ctx.check(ctx.lib.psms_autotune(ctx.handle, int(bool(enable)), int(block_variant)))


def psms_profile_enable(ctx, enable):
    """0 off, 1 every full-operator hop launch, 10 + PREC_* only the launches
    of that storage precision."""
    ctx.check(ctx.lib.psms_profile_enable(ctx.handle, int(enable)))


def psms_profile_read(ctx):
    n, ms, by = ctypes.c_longlong(), _D(), _D()
    ctx.check(ctx.lib.psms_profile_read(ctx.handle, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
    return n.value, ms.value, by.value


def _host_check(st, name):
    if st != 0:
        raise PsmsError(st, name + " failed")


def psms_level_covariance(samples):
    """Covariance [n_actions, n_actions] of action-change samples
    [n_samples, n_actions] (host function of the library)."""
    x = np.ascontiguousarray(samples, dtype=np.float64)
    if x.ndim != 2:
        raise ValueError("samples must be [n_samples, n_actions]")
    out = np.empty((x.shape[1], x.shape[1]), dtype=np.float64)
    _host_check(load_library().psms_level_covariance(x.ctypes.data, x.shape[0], x.shape[1], out.ctypes.data),
                "psms_level_covariance")
    return out


def psms_level_coefficients(covs, targets, stochastic=None):
    """beta_i^(j) [n+1, n+1] of the parametrised levels from the level
    covariances covs[i-1] ((i+1) x (i+1), i = 1..n), the targets beta^(j)
    and optional stochastic flags per action (host function of the library)."""
    n = len(targets) - 1
    packed = np.concatenate([np.ascontiguousarray(c, dtype=np.float64).reshape(-1) for c in covs]) \
        if n >= 1 else np.zeros(0)
    for i, c in enumerate(covs, start=1):
        if np.shape(c) != (i + 1, i + 1):
            raise ValueError(f"covariance of level {i} must be {(i + 1, i + 1)}")
    if len(covs) != n:
        raise ValueError("one covariance per level 1..n")
    t = np.ascontiguousarray(targets, dtype=np.float64)
    st = None if stochastic is None else np.ascontiguousarray(stochastic, dtype=np.int32)
    out = np.empty((n + 1, n + 1), dtype=np.float64)
    _host_check(load_library().psms_level_coefficients(n, packed.ctypes.data, t.ctypes.data,
                                                       None if st is None else st.ctypes.data, out.ctypes.data),
                "psms_level_coefficients")
    return out


def _alpha(alpha):
    return None if alpha is None else (ctypes.c_double * 3)(*[float(a) for a in alpha])


def psms_hyp_smear(ctx, field, out_dev, alpha=None):
    """Fat links of one level of HYP smearing into out_dev (canonical layout,
    4V x 9 complex doubles on the device)."""
    ctx.check(ctx.lib.psms_hyp_smear(ctx.handle, field, _alpha(alpha), _ptr(out_dev)))


def psms_hyp_block_action(ctx, field, alpha=None):
    """S_HYP,b per block (lexicographic block index)."""
    nb = int(psms_geometry_info(ctx)[0])
    out = np.empty(nb, dtype=np.float64)
    ctx.check(ctx.lib.psms_hyp_block_action(ctx.handle, field, _alpha(alpha), out.ctypes.data))
    return out


def psms_block_action_change(ctx, field_old, field_new):
    """dS_w,b of field_old -> field_new per block (lexicographic block index)."""
    nb = int(psms_geometry_info(ctx)[0])
    out = np.empty(nb, dtype=np.float64)
    ctx.check(ctx.lib.psms_block_action_change(ctx.handle, field_old, field_new, out.ctypes.data))
    return out
