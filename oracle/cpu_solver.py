"""Iterative FP64 CPU solver (oracle side; test infrastructure only).

A plain C + OpenMP restatement of the paper's method -- flexible GMRES with
modified Gram-Schmidt, multigrid V-cycles, the reaction-limited operator and the
Appendix A preconditioner of the saddle point -- in ``cpu_solver.c``, compiled
with gcc by ``build()`` into ``oracle/libibrd_cpu.so``. It exists so that the
benchmark workload can be solved, not sampled, on the host cores: the direct
Schur solver in ``direct`` is exact but needs N Green's-function solves.

Only ``tests/``, ``__graft_entry__`` and ``bench.py``'s CPU legs load it. It is
pinned in ``tests/test_oracle_cpu_solver.py`` against the direct solutions of
``direct`` (themselves pinned by brute force) and its V-cycle against
``multigrid.vcycle``.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_solver.c")
LIB = os.path.join(HERE, "libibrd_cpu.so")
STAMP = os.path.join(HERE, "libibrd_cpu.arch")


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("vcycles", ctypes.c_long), ("threads", ctypes.c_int), ("rel_residual", ctypes.c_double)]


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return True
    if open(STAMP).read().strip() != platform.machine():
        return True
    return os.path.getmtime(SRC) > os.path.getmtime(LIB)


def build(force: bool = False) -> str:
    """Compile cpu_solver.c with gcc (C99, OpenMP, -O2) if needed."""
    if not force and not _stale():
        return LIB
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-std=gnu99", "-O2", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed on cpu_solver.c:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(platform.machine())
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.cpu_solve_reaction.argtypes = [i, i, i, d, d, d, i, p, i, p, p, p, d, i, i, i, i, i, i,
                                           ctypes.POINTER(_Info)]
        lib.cpu_solve_saddle.argtypes = [i, i, i, d, d, d, i, p, i, p, p, d, d, p, d, i, i, i, i, i, i, i,
                                         ctypes.POINTER(_Info)]
        lib.cpu_vcycle.argtypes = [i, i, i, d, d, d, i, i, p, p, i, i]
        for f in (lib.cpu_solve_reaction, lib.cpu_solve_saddle, lib.cpu_vcycle):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _info(s: _Info) -> dict:
    return dict(status=s.status, outer_iters=s.outer_iters, inner_iters=s.inner_iters, vcycles=int(s.vcycles),
                threads=s.threads, rel_residual=s.rel_residual)


def solve_reaction(q, kappa, g, h, chi, alpha, w=4, tol=1e-8, restart=30, max_iter=2000, mg_cycles=1, nu1=2,
                   nu2=2, threads=0, c0=None):
    """Iterative solve of (alpha I - chi L + S kappa J) c = g (Eqs.
    unsteady_system, steady_state); returns (c, info)."""
    lib = _load()
    g = _f64(g)
    nz, ny, nx = g.shape
    q = _f64(q).reshape(-1, 3)
    kappa = _f64(kappa)
    c = np.zeros_like(g) if c0 is None else _f64(c0).copy()
    info = _Info()
    lib.cpu_solve_reaction(nx, ny, nz, h, chi, alpha, w, _ptr(q), len(q), _ptr(kappa), _ptr(g), _ptr(c), tol,
                           restart, max_iter, mg_cycles, nu1, nu2, threads or host_threads(), ctypes.byref(info))
    return c, _info(info)


def solve_saddle(q, g, h, chi, alpha, zeta=1.0, xi=None, f=None, w=4, tol=1e-8, restart=30, max_iter=2000,
                 mg_cycles=1, schur_inner=5, nu1=2, nu2=2, threads=0):
    """Iterative solve of the saddle point of Eq. saddle_point with the
    Appendix A preconditioner; returns (c, lam, info)."""
    lib = _load()
    g = _f64(g)
    nz, ny, nx = g.shape
    q = _f64(q).reshape(-1, 3)
    n = len(q)
    if xi is None:
        xi = zeta / h ** 3
    fv = None if f is None else _f64(f)
    x = np.zeros(g.size + n)
    info = _Info()
    lib.cpu_solve_saddle(nx, ny, nz, h, chi, alpha, w, _ptr(q), n, _ptr(g), _ptr(fv), zeta, xi, _ptr(x), tol,
                         restart, max_iter, mg_cycles, schur_inner, nu1, nu2, threads or host_threads(),
                         ctypes.byref(info))
    return x[:g.size].reshape(g.shape), x[g.size:].copy(), _info(info)


def vcycle(b, h, chi, shift, x0=None, nu1=2, nu2=2, threads=0):
    """One V-cycle of (shift I - chi L) x = b (the multigrid readings of
    ``multigrid``); returns x."""
    lib = _load()
    b = _f64(b)
    nz, ny, nx = b.shape
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    rc = lib.cpu_vcycle(nx, ny, nz, h, chi, shift, nu1, nu2, _ptr(b), _ptr(x), 1 if x0 is None else 0,
                        threads or host_threads())
    if rc != 0:
        raise RuntimeError(f"cpu_vcycle failed ({rc})")
    return x
