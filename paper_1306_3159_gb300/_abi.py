"""ctypes binding of libibrd (argument marshalling only).

Each ``ibrd_*`` function here has the name and argument order of the C entry
point in ``include/ibrd.h``; tensors are passed by device pointer.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libibrd.so")

IBRD_PESKIN4, IBRD_PESKIN3 = 4, 3
IBRD_FP64, IBRD_MIXED_FP32, IBRD_MIXED_REFINE = 0, 1, 2
IBRD_PRECOND_SCHUR, IBRD_PRECOND_DIAG, IBRD_PRECOND_AUTO, IBRD_PRECOND_BLOCK = 0, 1, 2, 3
IBRD_GUESS_NONE, IBRD_GUESS_UNIFORM, IBRD_GUESS_GIVEN, IBRD_GUESS_PENALTY = 0, 1, 2, 3

STATUS = {0: "IBRD_OK", 1: "IBRD_ERR_ARG", 2: "IBRD_ERR_CUDA", 3: "IBRD_ERR_OOM", 4: "IBRD_ERR_NOT_CONVERGED",
          5: "IBRD_ERR_BREAKDOWN", 6: "IBRD_ERR_NONFINITE", 7: "IBRD_ERR_TIMEOUT", 8: "IBRD_ERR_STATE"}

# Every entry point declared in include/ibrd.h.
EXPORTED = ["ibrd_default_opts", "ibrd_grid_create", "ibrd_grid_destroy", "ibrd_set_blobs", "ibrd_apply_L",
            "ibrd_residual", "ibrd_periodic_constant",
            "ibrd_vcycle", "ibrd_vcycle_f32", "ibrd_vcycle_f32_sweeps", "ibrd_vcycle_noalloc", "ibrd_spread", "ibrd_interp", "ibrd_solve_reaction", "ibrd_solve_saddle",
            "ibrd_solve_reaction_batch", "ibrd_solve_saddle_batch", "ibrd_solve_many", "ibrd_autotune", "ibrd_tune_set",
            "ibrd_tune_clear", "ibrd_set_wait_limit", "ibrd_gnn_num_params", "ibrd_gnn_create", "ibrd_gnn_destroy", "ibrd_gnn_last_error",
            "ibrd_gnn_set_params", "ibrd_gnn_get_params", "ibrd_gnn_init_params", "ibrd_gnn_neighbours", "ibrd_gnn_forward",
            "ibrd_gnn_predict", "ibrd_gnn_loss_grad", "ibrd_gnn_adam_step", "ibrd_gnn_train",
            "ibrd_last_error", "ibrd_status_string", "ibrd_profile_enable", "ibrd_profile_read",
            "ibrd_profile_class_name"]

PROF_NCLASS = 19


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("restart", ctypes.c_int),
                ("mg_cycles", ctypes.c_int), ("schur_inner", ctypes.c_int), ("precond", ctypes.c_int),
                ("zeta", ctypes.c_double), ("xi", ctypes.c_double), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("precision", ctypes.c_int), ("use_guess", ctypes.c_int),
                ("reorth_eta", ctypes.c_double), ("graphs", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("lambda_guess", ctypes.c_int), ("warm_cycles", ctypes.c_int),
                ("penalty_kappa", ctypes.c_double), ("penalty_tol", ctypes.c_double),
                ("block_cutoff", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("vcycles", ctypes.c_int), ("reorths", ctypes.c_int), ("rel_residual", ctypes.c_double), ("sum_lambda", ctypes.c_double),
                ("cbar", ctypes.c_double), ("rate_K", ctypes.c_double), ("seconds", ctypes.c_double),
                ("residual_history", ctypes.POINTER(ctypes.c_double)), ("history_len", ctypes.c_int),
                ("history_cap", ctypes.c_int), ("refinements", ctypes.c_int), ("a_L", ctypes.c_double),
                ("precond", ctypes.c_int)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("nclass", ctypes.c_int), ("overflow", ctypes.c_int),
                ("count", ctypes.c_longlong * PROF_NCLASS), ("timed", ctypes.c_longlong * PROF_NCLASS),
                ("ms", ctypes.c_double * PROF_NCLASS), ("bytes", ctypes.c_double * PROF_NCLASS),
                ("max_launch_bytes", ctypes.c_double * PROF_NCLASS), ("timed_bytes", ctypes.c_double * PROF_NCLASS)]


class SolveItem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("grid", ctypes.c_void_p), ("kappa", ctypes.c_void_p),
                ("rhs", ctypes.c_void_p), ("f", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("lam", ctypes.c_void_p), ("opts", ctypes.POINTER(SolveOpts)), ("info", ctypes.POINTER(SolveInfo)),
                ("q", ctypes.c_void_p), ("n_blobs", ctypes.c_int), ("c_host", ctypes.c_void_p),
                ("lambda_host", ctypes.c_void_p)]


IBRD_SOLVE_REACTION, IBRD_SOLVE_SADDLE = 0, 1


class TuneEntry(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("elem_bytes", ctypes.c_int),
                ("kind", ctypes.c_int), ("tx", ctypes.c_int), ("zc", ctypes.c_int), ("us_default", ctypes.c_double),
                ("us_tuned", ctypes.c_double), ("cached", ctypes.c_int)]


class IbrdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libibrd.so (built by ``paper_1306_3159_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libibrd.so not built at {path}; run paper_1306_3159_gb300/build.py")
    lib = ctypes.CDLL(path)
    vp, i, d, P = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER
    lib.ibrd_default_opts.argtypes = [P(SolveOpts)]
    lib.ibrd_default_opts.restype = None
    lib.ibrd_grid_create.argtypes = [P(vp), i, i, i, d, d, d, i, i, vp]
    lib.ibrd_grid_create.restype = i
    lib.ibrd_grid_destroy.argtypes = [vp]
    lib.ibrd_grid_destroy.restype = None
    lib.ibrd_set_blobs.argtypes = [vp, vp, i]
    lib.ibrd_set_blobs.restype = i
    lib.ibrd_apply_L.argtypes = [vp, vp, vp]
    lib.ibrd_apply_L.restype = i
    lib.ibrd_residual.argtypes = [vp, vp, vp, vp]
    lib.ibrd_residual.restype = i
    lib.ibrd_periodic_constant.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.ibrd_periodic_constant.restype = ctypes.c_double
    lib.ibrd_vcycle.argtypes = [vp, vp, vp, i]
    lib.ibrd_vcycle.restype = i
    lib.ibrd_vcycle_f32.argtypes = [vp, vp, vp, i]
    lib.ibrd_vcycle_f32.restype = i
    lib.ibrd_vcycle_f32_sweeps.argtypes = [vp, vp, vp, i, i, i]
    lib.ibrd_vcycle_f32_sweeps.restype = i
    lib.ibrd_spread.argtypes = [vp, vp, vp, i]
    lib.ibrd_spread.restype = i
    lib.ibrd_interp.argtypes = [vp, vp, vp]
    lib.ibrd_interp.restype = i
    lib.ibrd_solve_reaction.argtypes = [vp, vp, vp, vp, P(SolveOpts), P(SolveInfo)]
    lib.ibrd_solve_reaction.restype = i
    lib.ibrd_solve_saddle.argtypes = [vp, vp, vp, vp, vp, P(SolveOpts), P(SolveInfo)]
    lib.ibrd_solve_saddle.restype = i
    lib.ibrd_solve_reaction_batch.argtypes = [i, P(vp), P(vp), P(vp), P(vp), P(SolveOpts), P(SolveInfo), i]
    lib.ibrd_solve_reaction_batch.restype = i
    lib.ibrd_solve_saddle_batch.argtypes = [i, P(vp), P(vp), P(vp), P(vp), P(vp), P(SolveOpts), P(SolveInfo), i]
    lib.ibrd_solve_saddle_batch.restype = i
    lib.ibrd_solve_many.argtypes = [i, P(SolveItem), i]
    lib.ibrd_solve_many.restype = i
    lib.ibrd_autotune.argtypes = [vp, i, i, P(TuneEntry), i, P(i)]
    lib.ibrd_autotune.restype = i
    lib.ibrd_tune_set.argtypes = [vp, i, i, i, i, i, i, i]
    lib.ibrd_tune_set.restype = i
    lib.ibrd_tune_clear.argtypes = [vp]
    lib.ibrd_tune_clear.restype = i
    lib.ibrd_set_wait_limit.argtypes = [vp, ctypes.c_uint]
    lib.ibrd_set_wait_limit.restype = i
    lib.ibrd_gnn_num_params.argtypes = []
    lib.ibrd_gnn_num_params.restype = i
    lib.ibrd_gnn_create.argtypes = [P(vp), d, i, vp]
    lib.ibrd_gnn_create.restype = i
    lib.ibrd_gnn_destroy.argtypes = [vp]
    lib.ibrd_gnn_destroy.restype = None
    lib.ibrd_gnn_last_error.argtypes = [vp]
    lib.ibrd_gnn_last_error.restype = ctypes.c_char_p
    lib.ibrd_gnn_set_params.argtypes = [vp, vp, i]
    lib.ibrd_gnn_set_params.restype = i
    lib.ibrd_gnn_init_params.argtypes = [vp, ctypes.c_ulonglong]
    lib.ibrd_gnn_init_params.restype = i
    lib.ibrd_gnn_get_params.argtypes = [vp, vp]
    lib.ibrd_gnn_get_params.restype = i
    lib.ibrd_gnn_neighbours.argtypes = [vp, vp, i, d, d, d, vp, vp, vp]
    lib.ibrd_gnn_neighbours.restype = i
    lib.ibrd_gnn_forward.argtypes = [vp, vp, i, d, d, d, vp]
    lib.ibrd_gnn_forward.restype = i
    lib.ibrd_gnn_predict.argtypes = [vp, vp, i, d, d, d, d, vp]
    lib.ibrd_gnn_predict.restype = i
    lib.ibrd_gnn_loss_grad.argtypes = [vp, vp, i, d, d, d, vp, P(d), vp]
    lib.ibrd_gnn_loss_grad.restype = i
    lib.ibrd_gnn_adam_step.argtypes = [vp, vp, d]
    lib.ibrd_gnn_adam_step.restype = i
    lib.ibrd_gnn_train.argtypes = [vp, i, P(vp), P(i), P(d), P(vp), i, d, P(d)]
    lib.ibrd_gnn_train.restype = i
    lib.ibrd_last_error.argtypes = [vp]
    lib.ibrd_last_error.restype = ctypes.c_char_p
    lib.ibrd_status_string.argtypes = [i]
    lib.ibrd_status_string.restype = ctypes.c_char_p
    lib.ibrd_profile_enable.argtypes = [vp, ctypes.c_uint, d]
    lib.ibrd_profile_enable.restype = i
    lib.ibrd_profile_read.argtypes = [vp, P(Profile), i]
    lib.ibrd_profile_read.restype = i
    lib.ibrd_profile_class_name.argtypes = [i]
    lib.ibrd_profile_class_name.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(t, dtype="float64"):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or t.dtype != getattr(torch, dtype) or not t.is_contiguous():
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check(g, st: int):
    if st != 0:
        msg = ibrd_last_error(g) if g else ""
        raise IbrdError(st, msg)


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def ibrd_default_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    load_library().ibrd_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def ibrd_grid_create(nx, ny, nz, h=1.0, chi=1.0, alpha=0.0, kernel=IBRD_PESKIN4, precision=IBRD_FP64, stream=None):
    lib = load_library()
    g = ctypes.c_void_p()
    st = lib.ibrd_grid_create(ctypes.byref(g), int(nx), int(ny), int(nz), float(h), float(chi), float(alpha),
                              int(kernel), int(precision), _stream(stream))
    if st != 0:
        raise IbrdError(st, "ibrd_grid_create rejected its arguments")
    return g


def ibrd_grid_destroy(g):
    load_library().ibrd_grid_destroy(g)


def ibrd_last_error(g) -> str:
    return load_library().ibrd_last_error(g).decode()


def ibrd_set_blobs(g, q, n=None):
    n = int(q.shape[0]) if n is None else int(n)
    _check(g, load_library().ibrd_set_blobs(g, _ptr(q) if n else None, n))


def ibrd_apply_L(g, c, y):
    _check(g, load_library().ibrd_apply_L(g, _ptr(c), _ptr(y)))


def ibrd_periodic_constant(lx, ly, lz) -> float:
    return float(load_library().ibrd_periodic_constant(float(lx), float(ly), float(lz)))


def ibrd_residual(g, rhs, c, r):
    _check(g, load_library().ibrd_residual(g, _ptr(rhs), _ptr(c), _ptr(r)))


def ibrd_vcycle(g, rhs, x, zero_initial_guess=True):
    _check(g, load_library().ibrd_vcycle(g, _ptr(rhs), _ptr(x), int(bool(zero_initial_guess))))


def ibrd_vcycle_f32(g, rhs, x, zero_initial_guess=True):
    _check(g, load_library().ibrd_vcycle_f32(g, _ptr(rhs, "float32"), _ptr(x, "float32"),
                                             int(bool(zero_initial_guess))))

def ibrd_vcycle_f32_sweeps(g, rhs, x, zero_initial_guess=True, nu1=2, nu2=2):
    """FP32 V-cycle with nu1 / nu2 smoothing sweeps (the solves' counts)."""
    _check(g, load_library().ibrd_vcycle_f32_sweeps(g, _ptr(rhs, "float32"), _ptr(x, "float32"),
                                                    int(bool(zero_initial_guess)), int(nu1), int(nu2)))


def ibrd_spread(g, lam, out, accumulate=False):
    _check(g, load_library().ibrd_spread(g, _ptr(lam), _ptr(out), int(bool(accumulate))))


def ibrd_interp(g, c, out):
    _check(g, load_library().ibrd_interp(g, _ptr(c), _ptr(out)))


def _info(history_cap):
    import numpy as np
    info = SolveInfo()
    hist = np.zeros(max(1, history_cap), dtype=np.float64)
    info.residual_history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    info.history_cap = history_cap
    return info, hist


def _info_dict(info, hist):
    return {"status": info.status, "outer_iters": info.outer_iters, "inner_iters": info.inner_iters,
            "vcycles": info.vcycles, "reorths": info.reorths, "rel_residual": info.rel_residual, "sum_lambda": info.sum_lambda,
            "cbar": info.cbar, "rate_K": info.rate_K, "a_L": info.a_L, "seconds": info.seconds,
            "refinements": info.refinements, "precond": info.precond,
            "history": hist[:info.history_len].copy()}


def ibrd_solve_reaction(g, kappa, rhs, c, opts: SolveOpts | None = None, history_cap=4096, raise_on_error=True):
    info, hist = _info(history_cap)
    st = load_library().ibrd_solve_reaction(g, _ptr(kappa), _ptr(rhs), _ptr(c),
                                            ctypes.byref(opts) if opts is not None else None, ctypes.byref(info))
    if raise_on_error:
        _check(g, st)
    out = _info_dict(info, hist)
    out["status"] = st
    return out


def ibrd_solve_saddle(g, rhs, f, c, lam, opts: SolveOpts | None = None, history_cap=4096, raise_on_error=True):
    info, hist = _info(history_cap)
    st = load_library().ibrd_solve_saddle(g, _ptr(rhs), _ptr(f), _ptr(c), _ptr(lam),
                                          ctypes.byref(opts) if opts is not None else None, ctypes.byref(info))
    if raise_on_error:
        _check(g, st)
    out = _info_dict(info, hist)
    out["status"] = st
    return out


def _ptr_array(items, dtype="float64"):
    arr = (ctypes.c_void_p * max(1, len(items)))()
    for k, t in enumerate(items):
        p = _ptr(t, dtype)
        arr[k] = p.value if p is not None else None
    return arr


def _handles(grids):
    vals = [g.value if isinstance(g, ctypes.c_void_p) else g for g in grids]
    return (ctypes.c_void_p * max(1, len(vals)))(*vals)


def _batch_infos(count, history_cap):
    import numpy as np
    infos = (SolveInfo * max(1, count))()
    hists = []
    for k in range(count):
        h = np.zeros(max(1, history_cap), dtype=np.float64)
        infos[k].residual_history = h.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        infos[k].history_cap = history_cap
        hists.append(h)
    return infos, hists


def _batch_result(grids, st, infos, hists, raise_on_error):
    out = [_info_dict(infos[k], hists[k]) for k in range(len(grids))]
    if raise_on_error and st != 0:
        bad = next((k for k, r in enumerate(out) if r["status"] != 0), None)
        raise IbrdError(st, f"problem {bad}: " + (ibrd_last_error(grids[bad]) if bad is not None else ""))
    return out


def ibrd_solve_reaction_batch(grids, kappa, rhs, c, opts: SolveOpts | None = None, threads=0, history_cap=0,
                              raise_on_error=True):
    """Solve len(grids) reaction problems concurrently; lists of per-problem tensors."""
    n = len(grids)
    if not (len(kappa) == len(rhs) == len(c) == n):
        raise ValueError("one kappa, rhs and c per handle")
    infos, hists = _batch_infos(n, history_cap)
    hs = _handles(grids)
    st = load_library().ibrd_solve_reaction_batch(n, hs, _ptr_array(kappa), _ptr_array(rhs), _ptr_array(c),
                                                  ctypes.byref(opts) if opts is not None else None, infos,
                                                  int(threads))
    return _batch_result(grids, st, infos, hists, raise_on_error)


def ibrd_solve_saddle_batch(grids, rhs, f, c, lam, opts: SolveOpts | None = None, threads=0, history_cap=0,
                            raise_on_error=True):
    """Solve len(grids) saddle-point problems concurrently; f may be None."""
    n = len(grids)
    if not (len(rhs) == len(c) == len(lam) == n) or (f is not None and len(f) != n):
        raise ValueError("one rhs, c and lambda (and f) per handle")
    infos, hists = _batch_infos(n, history_cap)
    hs = _handles(grids)
    st = load_library().ibrd_solve_saddle_batch(n, hs, _ptr_array(rhs), _ptr_array(f) if f is not None else None,
                                                _ptr_array(c), _ptr_array(lam),
                                                ctypes.byref(opts) if opts is not None else None, infos,
                                                int(threads))
    return _batch_result(grids, st, infos, hists, raise_on_error)


def ibrd_solve_many(items, threads=0, history_cap=0, raise_on_error=True) -> list:
    """Independent solves of either kind at once. items: dicts with "kind"
    ("reaction" or "saddle"), "grid" (handle), "rhs", "c", and "kappa"
    (reaction) or "lam" and optionally "f" (saddle); optionally "opts", "q"
    (blob positions to set first) and "c_host" / "lam_host" (CPU float64
    tensors, pinned, that receive the solution after the solve)."""
    n = len(items)
    arr = (SolveItem * max(1, n))()
    infos, hists = _batch_infos(n, history_cap)
    keep = []
    for k, it in enumerate(items):
        kind = {"reaction": IBRD_SOLVE_REACTION, "saddle": IBRD_SOLVE_SADDLE}[it["kind"]]
        g = it["grid"]
        arr[k].kind = kind
        arr[k].grid = g.value if isinstance(g, ctypes.c_void_p) else g
        for name, key in (("kappa", "kappa"), ("rhs", "rhs"), ("f", "f"), ("c", "c"), ("lam", "lam")):
            ptr = _ptr(it.get(key))
            setattr(arr[k], name, ptr.value if ptr is not None else None)
        if it.get("q") is not None:
            arr[k].q = _ptr(it["q"]).value
            arr[k].n_blobs = int(it["q"].shape[0])
        for name, key in (("c_host", "c_host"), ("lambda_host", "lam_host")):
            t = it.get(key)
            if t is not None:
                if t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch.float64":
                    raise ValueError("host outputs are contiguous CPU float64 tensors (pinned for overlap)")
                setattr(arr[k], name, t.data_ptr())
        o = it.get("opts")
        if o is not None:
            keep.append(o)
            arr[k].opts = ctypes.pointer(o)
        arr[k].info = ctypes.pointer(infos[k])
    st = load_library().ibrd_solve_many(n, arr, int(threads))
    return _batch_result([it["grid"] for it in items], st, infos, hists, raise_on_error)


def ibrd_autotune(g, precision=-1, retune=False, cap=64) -> list:
    """Tune the sweep kernels' launch shapes for handle g; one dict per
    (level, precision, kernel) tuned."""
    arr = (TuneEntry * cap)()
    n = ctypes.c_int(0)
    _check(g, load_library().ibrd_autotune(g, int(precision), int(bool(retune)), arr, cap, ctypes.byref(n)))
    return [{f: getattr(arr[k], f) for f, _ in TuneEntry._fields_} for k in range(min(n.value, cap))]


def ibrd_tune_set(g, elem_bytes, kind, nx, ny, nz, tx, zc):
    _check(g, load_library().ibrd_tune_set(g, int(elem_bytes), int(kind), int(nx), int(ny), int(nz), int(tx),
                                           int(zc)))


def ibrd_tune_clear(g):
    _check(g, load_library().ibrd_tune_clear(g))


def ibrd_set_wait_limit(g, tries):
    """Polls each bounded device wait of handle g makes before it gives up."""
    _check(g, load_library().ibrd_set_wait_limit(g, int(tries)))


PROF_ALL = (1 << PROF_NCLASS) - 1


def profile_class_names():
    lib = load_library()
    return [lib.ibrd_profile_class_name(c).decode() for c in range(PROF_NCLASS)]


def ibrd_profile_enable(g, class_mask=PROF_ALL, min_bytes=0.0):
    """Time the kernel classes in class_mask (bit per class; True = all),
    only launches with at least min_bytes algorithmic bytes."""
    if class_mask is True:
        class_mask = PROF_ALL
    _check(g, load_library().ibrd_profile_enable(g, int(class_mask), float(min_bytes)))


def ibrd_profile_read(g, reset=True) -> dict:
    """Launch counts and event times per kernel class since the last reset."""
    lib = load_library()
    pr = Profile()
    _check(g, lib.ibrd_profile_read(g, ctypes.byref(pr), int(bool(reset))))
    classes = {}
    for c in range(pr.nclass):
        if pr.count[c]:
            classes[lib.ibrd_profile_class_name(c).decode()] = {
                "id": c, "launches": int(pr.count[c]), "timed": int(pr.timed[c]), "ms": float(pr.ms[c]),
                "bytes": float(pr.bytes[c]), "max_launch_bytes": float(pr.max_launch_bytes[c]),
                "timed_bytes": float(pr.timed_bytes[c])}
    return {"launches": int(pr.launches), "overflow": bool(pr.overflow), "classes": classes}


class Grid:
    """Owning wrapper of an ``ibrd_grid`` handle."""

    def __init__(self, nx, ny, nz, h=1.0, chi=1.0, alpha=0.0, kernel=IBRD_PESKIN4, precision=IBRD_FP64,
                 stream=None):
        self.dims = (int(nx), int(ny), int(nz))
        self.h, self.chi, self.alpha = float(h), float(chi), float(alpha)
        self.handle = ibrd_grid_create(nx, ny, nz, h, chi, alpha, kernel, precision, stream)
        self.n_blobs = 0

    def close(self):
        if self.handle is not None:
            ibrd_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field(self, fill=0.0):
        import torch
        nx, ny, nz = self.dims
        return torch.full((nz, ny, nx), float(fill), dtype=torch.float64, device="cuda")

    def set_blobs(self, q):
        self.n_blobs = int(q.shape[0])
        ibrd_set_blobs(self.handle, q)

    def apply_L(self, c, y=None):
        y = self.field() if y is None else y
        ibrd_apply_L(self.handle, c, y)
        return y

    def residual(self, rhs, c, r=None):
        r = self.field() if r is None else r
        ibrd_residual(self.handle, rhs, c, r)
        return r

    def vcycle(self, rhs, x=None, zero_initial_guess=True):
        x = self.field() if x is None else x
        ibrd_vcycle(self.handle, rhs, x, zero_initial_guess)
        return x

    def vcycle_f32(self, rhs, x=None, zero_initial_guess=True, nu1=2, nu2=2):
        import torch
        x = torch.zeros_like(rhs) if x is None else x
        if (nu1, nu2) == (2, 2):
            ibrd_vcycle_f32(self.handle, rhs, x, zero_initial_guess)
        else:
            ibrd_vcycle_f32_sweeps(self.handle, rhs, x, zero_initial_guess, nu1, nu2)
        return x

    def spread(self, lam, out=None, accumulate=False):
        out = self.field() if out is None else out
        ibrd_spread(self.handle, lam, out, accumulate)
        return out

    def interp(self, c, out=None):
        import torch
        out = torch.zeros(self.n_blobs, dtype=torch.float64, device="cuda") if out is None else out
        ibrd_interp(self.handle, c, out)
        return out

    def solve_reaction(self, kappa, rhs, c=None, **kw):
        c = self.field() if c is None else c
        info = ibrd_solve_reaction(self.handle, kappa, rhs, c, ibrd_default_opts(**kw))
        return c, info

    def solve_saddle(self, rhs, f=None, c=None, lam=None, **kw):
        import torch
        c = self.field() if c is None else c
        lam = torch.zeros(self.n_blobs, dtype=torch.float64, device="cuda") if lam is None else lam
        info = ibrd_solve_saddle(self.handle, rhs, f, c, lam, ibrd_default_opts(**kw))
        return c, lam, info


# ---------------------------------------------------------------- learned multiplier predictor
def ibrd_gnn_num_params() -> int:
    return int(load_library().ibrd_gnn_num_params())


def _gnn_check(m, st):
    if st != 0:
        raise IbrdError(st, load_library().ibrd_gnn_last_error(m).decode() if m else "")


class GNN:
    """Owning wrapper of an ``ibrd_gnn`` model (positions: CUDA FP64 (n, 3))."""

    def __init__(self, cutoff, max_neighbours=64, stream=None):
        lib = load_library()
        self.handle = ctypes.c_void_p()
        st = lib.ibrd_gnn_create(ctypes.byref(self.handle), float(cutoff), int(max_neighbours), _stream(stream))
        if st != 0:
            raise IbrdError(st, "ibrd_gnn_create rejected its arguments")
        self.cutoff, self.kmax = float(cutoff), int(max_neighbours)

    def close(self):
        if self.handle is not None:
            load_library().ibrd_gnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta, reset_optimizer=True):
        import numpy as np
        t = np.ascontiguousarray(theta, dtype=np.float32)
        if t.size != ibrd_gnn_num_params():
            raise ValueError("wrong parameter count")
        _gnn_check(self.handle, load_library().ibrd_gnn_set_params(self.handle, t.ctypes.data_as(ctypes.c_void_p),
                                                                    int(bool(reset_optimizer))))

    def init_params(self, seed):
        _gnn_check(self.handle, load_library().ibrd_gnn_init_params(self.handle, int(seed)))

    def get_params(self):
        import numpy as np
        t = np.zeros(ibrd_gnn_num_params(), dtype=np.float32)
        _gnn_check(self.handle, load_library().ibrd_gnn_get_params(self.handle, t.ctypes.data_as(ctypes.c_void_p)))
        return t

    def neighbours(self, q, box):
        import torch
        n = int(q.shape[0])
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        idx = torch.zeros((n, self.kmax), dtype=torch.int32, device="cuda")
        dist = torch.zeros((n, self.kmax), dtype=torch.float32, device="cuda")
        _gnn_check(self.handle, load_library().ibrd_gnn_neighbours(
            self.handle, _ptr(q), n, *map(float, box), _ptr(cnt, "int32"), _ptr(idx, "int32"),
            _ptr(dist, "float32")))
        return cnt, idx, dist

    def forward(self, q, box):
        import torch
        n = int(q.shape[0])
        y = torch.zeros(n, dtype=torch.float32, device="cuda")
        _gnn_check(self.handle, load_library().ibrd_gnn_forward(self.handle, _ptr(q), n, *map(float, box),
                                                                _ptr(y, "float32")))
        return y

    def predict(self, q, box, total, out=None):
        import torch
        n = int(q.shape[0])
        out = torch.zeros(n, dtype=torch.float64, device="cuda") if out is None else out
        _gnn_check(self.handle, load_library().ibrd_gnn_predict(self.handle, _ptr(q), n, *map(float, box),
                                                                float(total), _ptr(out)))
        return out

    def loss_grad(self, q, box, lam):
        import torch
        g = torch.zeros(ibrd_gnn_num_params(), dtype=torch.float32, device="cuda")
        loss = ctypes.c_double(0.0)
        _gnn_check(self.handle, load_library().ibrd_gnn_loss_grad(self.handle, _ptr(q), int(q.shape[0]),
                                                                  *map(float, box), _ptr(lam), ctypes.byref(loss),
                                                                  _ptr(g, "float32")))
        return loss.value, g

    def adam_step(self, grad, lr):
        _gnn_check(self.handle, load_library().ibrd_gnn_adam_step(self.handle, _ptr(grad, "float32"), float(lr)))

    def train(self, qs, boxes, lams, epochs, lr):
        """epochs passes over the configurations (lists of CUDA tensors); returns
        the mean loss of each epoch."""
        import numpy as np
        c = len(qs)
        qa, la = _ptr_array(qs), _ptr_array(lams)
        ns = (ctypes.c_int * c)(*[int(q.shape[0]) for q in qs])
        bx = (ctypes.c_double * (3 * c))(*[float(v) for b in boxes for v in b])
        out = (ctypes.c_double * epochs)()
        _gnn_check(self.handle, load_library().ibrd_gnn_train(self.handle, c, qa, ns, bx, la, int(epochs),
                                                              float(lr), out))
        return np.array(out[:])
