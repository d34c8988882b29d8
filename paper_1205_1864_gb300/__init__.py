"""GB300 stochastic Galerkin solver with the hierarchical Schur complement
preconditioner (Sousedik, Ghanem, Phipps; arXiv 1205.1864).

Thin Python binding over the C ABI of ``libsghsc.so`` (``include/sghsc.h``).
The functions keep the C names (``sg_setup``, ``sg_apply``,
``hsc_precond_apply``, ``sg_solve``, ...) and only marshal arguments: every
step of the method runs in the library's CUDA kernels. PyTorch supplies
device memory and the current stream. There is no CPU fallback: importing the
package fails if the library has not been built.

Blocks are ``n x P`` row-major CUDA tensors (spatial index slow, chaos index
fast), ``torch.float64`` unless a call says otherwise.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import (SG_F32, SG_F32_ACC64, SG_F64, SG_HERMITE, SG_LEGENDRE, SG_M0_DIAG, SG_M0_VCYCLE, SG_PREC_BGS,
                   SG_PREC_HSC, SG_PREC_MEAN, SG_PREC_NONE, SGError, check)

__all__ = [
    "SGProblem", "sg_setup", "sg_apply", "sg_level_apply", "sg_vcycle_apply", "sg_inner_solve",
    "hsc_precond_apply", "mean_precond_apply", "bgs_precond_apply", "SG_PREC_BGS", "SG_M0_VCYCLE", "SG_M0_DIAG", "sg_solve", "sg_solve_host", "sg_qoi", "sg_qoi_grad", "prec_opts", "solve_opts",
    "sg_set_scales", "SGQoI", "SGGradBatch", "sg_kl_set_theta", "sg_kl_qoi_grad", "sg_qoi_value_and_grad_batch",
    "sg_autotune", "sg_autotune_forms", "sg_autotune_shapes", "sg_autotune_set", "sg_measure_alu_peak",
    "SGError", "SG_F32", "SG_F32_ACC64", "SG_F64", "SG_PREC_HSC", "SG_PREC_MEAN", "SG_PREC_NONE", "SG_LEGENDRE", "SG_HERMITE",
]

_DT = {torch.float64: SG_F64, torch.float32: SG_F32}


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _block(h: "SGProblem", t, name: str, cols: Optional[int] = None, dtypes=(torch.float64,)) -> None:
    """Refuse a block whose shape or element type is not what the call reads
    or writes: the library takes bare pointers and touches exactly n x cols
    elements (cols = P by default), so a smaller tensor would be overrun.
    ``None`` passes (optional arguments)."""
    if t is None:
        return
    want = (h.n, h.P if cols is None else cols)
    if tuple(t.shape) != want or t.dtype not in dtypes:
        kinds = " or ".join(str(d).replace("torch.", "") for d in dtypes)
        raise ValueError(f"{name}: expected a {want[0]} x {want[1]} {kinds} block, got "
                         f"{tuple(t.shape)} {str(t.dtype).replace('torch.', '')}")


def _ptr(t: Optional[torch.Tensor]) -> Optional[C.c_void_p]:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def prec_opts(**kw) -> _lib.sg_prec_opts:
    """Preconditioner options with the library defaults, overridden by ``kw``
    (precision, top_level_f64, inner_tol, inner_maxit, inner_fixed_iters, nu, omega)."""
    o = _lib.sg_prec_opts()
    _lib.LIB.sg_default_prec_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def solve_opts(prec: Optional[_lib.sg_prec_opts] = None, **kw) -> _lib.sg_solve_opts:
    """Outer solver options (precond, tol, maxit, flexible, use_x0) with defaults."""
    o = _lib.sg_solve_opts()
    _lib.LIB.sg_default_solve_opts(C.byref(o))
    if prec is not None:
        o.prec = prec
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@dataclass
class SolveStats:
    status: int
    iterations: int
    rel_res: float
    true_rel_res: float
    kappa_est: float
    inner_iters_total: int
    inner_iters_max: int
    solve_ms: float
    res_hist: list
    alpha: list
    beta: list


class SGProblem:
    """Owner of an ``sg_problem`` handle (``sg_setup`` / ``sg_destroy``)."""

    def __init__(self, ne_x: int, ne_y: int, M: int, p: int, rowptr, colidx, vals, mass=None,
                 family: int = SG_LEGENDRE, q: int = -1):
        """``q < 0``: the linear KL expansion (``vals`` is ``nnz x (M+1)``,
        ``sg_setup``); ``q >= 0``: a gPC coefficient of total degree ``q``
        (``vals`` is ``nnz x C(M+q, M)``, ``sg_setup_gpc``, Hermite chaos)."""
        import math
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        n = rowptr.shape[0] - 1
        nnz = colidx.shape[0]
        nterm = M + 1 if q < 0 else math.comb(M + q, M)
        if vals.shape != (nnz, nterm):
            raise ValueError(f"vals must have shape (nnz, terms) = ({nnz}, {nterm})")
        mesh = _lib.sg_mesh(ne_x, ne_y)
        mp = None
        if mass is not None:
            mass = np.ascontiguousarray(mass, dtype=np.float64)
            if mass.shape != (nnz,):
                raise ValueError(f"mass must hold one value per nonzero ({nnz})")
            mp = mass.ctypes.data_as(C.POINTER(C.c_double))
        h = C.c_void_p()
        torch.cuda.init()
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
        dp = vals.ctypes.data_as(C.POINTER(C.c_double))
        if q < 0:
            check(_lib.LIB.sg_setup(C.byref(mesh), M, p, family, n, nnz, ip(rowptr), ip(colidx), dp, mp, C.byref(h)),
                  "sg_setup")
        else:
            check(_lib.LIB.sg_setup_gpc(C.byref(mesh), M, p, q, family, n, nnz, ip(rowptr), ip(colidx), dp, mp,
                                        C.byref(h)), "sg_setup_gpc")
        self.h = h
        dims = [C.c_int() for _ in range(5)]
        check(_lib.LIB.sg_problem_dims(h, *[C.byref(x) for x in dims]), "sg_problem_dims")
        self.n, self.P, self.M, self.p, self.nnz = (d.value for d in dims)
        self.q, self.nterm = q, nterm
        self.off = [int(v) for v in self.chaos_table()[1]]   # degree d occupies columns off[d]:off[d+1]

    @classmethod
    def from_inputs(cls, prob, p: int, family: int = SG_LEGENDRE) -> "SGProblem":
        """From an ``sg_inputs.Problem`` (seeded synthetic problem); a gPC
        (lognormal) problem takes Hermite chaos."""
        q = getattr(prob, "coef_degree", -1)
        if q >= 0:
            family = SG_HERMITE
        return cls(prob.ne, prob.ne, prob.M, p, prob.rowptr, prob.colidx, prob.vals, prob.mass, family, q)

    @property
    def inner_cluster(self) -> bool:
        """True when the FP32 inner solves run on the cluster-resident solver."""
        return bool(_lib.LIB.sg_inner_cluster(self.h))

    def inner_path(self, w: int, dtype: int = SG_F32) -> int:
        """Solver of a batched inner solve of w columns: 0 stand-alone kernels,
        1 cluster solver on chip (clusters of 8), 3 the same with clusters of
        16, 2 cluster solver with the finest grid in HBM."""
        return int(_lib.LIB.sg_inner_path(self.h, w, dtype))

    def close(self):
        if getattr(self, "h", None):
            _lib.LIB.sg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def chaos_table(self):
        alpha = np.zeros(self.P * max(self.M, 1), dtype=np.int32)
        off = np.zeros(self.p + 2, dtype=np.int32)
        check(_lib.LIB.sg_chaos_table(self.h, alpha.ctypes.data_as(C.POINTER(C.c_int)),
                                      off.ctypes.data_as(C.POINTER(C.c_int))), "sg_chaos_table")
        return alpha[: self.P * self.M].reshape(self.P, self.M), off

    def empty(self, cols: Optional[int] = None, dtype=torch.float64):
        return torch.empty((self.n, self.P if cols is None else cols), dtype=dtype, device="cuda")


def sg_setup(ne_x, ne_y, M, p, rowptr, colidx, vals, mass=None, family=SG_LEGENDRE) -> SGProblem:
    return SGProblem(ne_x, ne_y, M, p, rowptr, colidx, vals, mass, family)


def sg_apply(h: SGProblem, U: torch.Tensor, Y: Optional[torch.Tensor] = None, df64: bool = False) -> torch.Tensor:
    """Y = sum_k A_k U G_k^T (K1). ``df64``: FP32 ``U``, sums in double-float
    arithmetic, FP64 ``Y`` (``SG_F32_ACCDF64``)."""
    if df64:
        if U.dtype != torch.float32:
            raise ValueError("sg_apply: df64 takes an FP32 U")
        _block(h, U, "sg_apply: U", dtypes=(torch.float32,))
        _block(h, Y, "sg_apply: Y", dtypes=(torch.float64,))
        Y = torch.empty(U.shape, dtype=torch.float64, device=U.device) if Y is None else Y
        code = _lib.SG_F32_ACCDF64
    else:
        _block(h, U, "sg_apply: U", dtypes=(torch.float64, torch.float32))
        _block(h, Y, "sg_apply: Y", dtypes=(U.dtype,))
        Y = torch.empty_like(U) if Y is None else Y
        code = _DT[U.dtype]
    check(_lib.LIB.sg_apply(h.h, _ptr(U), _ptr(Y), code, _stream()), "sg_apply")
    return Y


def sg_level_apply(h: SGProblem, lvl_out: int, lvl_in: int, X: torch.Tensor, Yin: Optional[torch.Tensor],
                   Yout: Optional[torch.Tensor] = None, df64: bool = False) -> torch.Tensor:
    """Yout = Yin - sum_k A_k X G_k[out, in]^T between adjacent degree levels (K2).
    An FP32 ``X`` with an FP64 ``Yin`` takes the FP64-accurate product of
    the mixed preconditioner's top level (``SG_F32_ACC64``, FP32 ``Yout``;
    ``df64``: double-float accumulation, ``SG_F32_ACCDF64``)."""
    mixed = X.dtype == torch.float32 and Yin is not None and Yin.dtype == torch.float64
    if 0 <= lvl_in <= h.p and 0 <= lvl_out <= h.p:   # other levels: refused by the library
        off = h.off
        w_in, w_out = off[lvl_in + 1] - off[lvl_in], off[lvl_out + 1] - off[lvl_out]
        _block(h, X, "sg_level_apply: X", w_in, (torch.float64, torch.float32))
        _block(h, Yin, "sg_level_apply: Yin", w_out, (torch.float64,) if mixed else (X.dtype,))
        _block(h, Yout, "sg_level_apply: Yout", w_out, (X.dtype,))
        if Yout is None:
            Yout = torch.empty((h.n, w_out), dtype=X.dtype, device="cuda")
    code = (_lib.SG_F32_ACCDF64 if df64 else SG_F32_ACC64) if mixed else _DT[X.dtype]
    check(_lib.LIB.sg_level_apply(h.h, lvl_out, lvl_in, _ptr(X), _ptr(Yin), _ptr(Yout), code, _stream()),
          "sg_level_apply")
    return Yout


def sg_vcycle_apply(h: SGProblem, B: torch.Tensor, opts=None) -> torch.Tensor:
    _block(h, B, "sg_vcycle_apply: B", B.shape[1] if len(B.shape) == 2 else -1, (torch.float64, torch.float32))
    X = torch.empty_like(B)
    o = opts or prec_opts()
    check(_lib.LIB.sg_vcycle_apply(h.h, _ptr(B), _ptr(X), B.shape[1], _DT[B.dtype], C.byref(o), _stream()),
          "sg_vcycle_apply")
    return X


def sg_inner_solve(h: SGProblem, B: torch.Tensor, opts=None):
    _block(h, B, "sg_inner_solve: B", B.shape[1] if len(B.shape) == 2 else -1, (torch.float64, torch.float32))
    X = torch.empty_like(B)
    o = opts or prec_opts()
    it = np.zeros(B.shape[1], dtype=np.int32)
    check(_lib.LIB.sg_inner_solve(h.h, _ptr(B), _ptr(X), B.shape[1], _DT[B.dtype], C.byref(o),
                                  it.ctypes.data_as(C.POINTER(C.c_int)), _stream()), "sg_inner_solve")
    return X, it


def hsc_precond_apply(h: SGProblem, R: torch.Tensor, opts=None, Z: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Z = M_P R (Algorithm 1)."""
    _block(h, R, "hsc_precond_apply: R")
    _block(h, Z, "hsc_precond_apply: Z")
    Z = torch.empty_like(R) if Z is None else Z
    o = opts or prec_opts()
    check(_lib.LIB.hsc_precond_apply(h.h, _ptr(R), _ptr(Z), C.byref(o), _stream()), "hsc_precond_apply")
    return Z


def bgs_precond_apply(h: SGProblem, R: torch.Tensor, opts=None, Z: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Z = M_bGS R (block symmetric Gauss-Seidel, zero initial guess)."""
    _block(h, R, "bgs_precond_apply: R")
    _block(h, Z, "bgs_precond_apply: Z")
    Z = torch.empty_like(R) if Z is None else Z
    o = opts or prec_opts()
    check(_lib.LIB.bgs_precond_apply(h.h, _ptr(R), _ptr(Z), C.byref(o), _stream()), "bgs_precond_apply")
    return Z


def mean_precond_apply(h: SGProblem, R: torch.Tensor, opts=None, Z: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Z = (I (x) A_0^{-1}) R with the inner PCG."""
    _block(h, R, "mean_precond_apply: R")
    _block(h, Z, "mean_precond_apply: Z")
    Z = torch.empty_like(R) if Z is None else Z
    o = opts or prec_opts()
    check(_lib.LIB.mean_precond_apply(h.h, _ptr(R), _ptr(Z), C.byref(o), _stream()), "mean_precond_apply")
    return Z


def _stats(status, st) -> "SolveStats":
    return SolveStats(status=status, iterations=st.iterations, rel_res=st.rel_res, true_rel_res=st.true_rel_res,
                      kappa_est=st.kappa_est, inner_iters_total=st.inner_iters_total,
                      inner_iters_max=st.inner_iters_max, solve_ms=st.solve_ms,
                      res_hist=list(st.res_hist[: st.n_hist]), alpha=list(st.alpha[: st.iterations]),
                      beta=list(st.beta[: max(st.iterations - 1, 0)]))


def sg_solve(h: SGProblem, F: torch.Tensor, opts=None, U: Optional[torch.Tensor] = None, raise_on_error=True):
    """Flexible CG on the SG system; returns ``(U, SolveStats)``."""
    _block(h, F, "sg_solve: F")
    _block(h, U, "sg_solve: U")
    U = torch.empty_like(F) if U is None else U
    o = opts or solve_opts()
    st = _lib.sg_solve_stats()
    status = _lib.LIB.sg_solve(h.h, _ptr(F), _ptr(U), C.byref(o), C.byref(st), _stream())
    stats = _stats(status, st)
    if raise_on_error:
        check(status, "sg_solve")
    return U, stats


def sg_solve_host(h: SGProblem, F: torch.Tensor, opts=None, U: Optional[torch.Tensor] = None,
                  raise_on_error=True):
    """``sg_solve`` on host (CPU) blocks: ``F`` in, ``U`` out, both contiguous
    FP64 CPU tensors (pinned ones are read and written by the library's
    kernels directly); returns ``(U, SolveStats)`` when ``U`` is filled."""
    if F.is_cuda or not F.is_contiguous() or F.dtype != torch.float64:
        raise ValueError("sg_solve_host: F must be a contiguous FP64 CPU tensor")
    _block(h, F, "sg_solve_host: F")
    U = torch.empty_like(F) if U is None else U
    if U.is_cuda or not U.is_contiguous() or U.dtype != torch.float64 or U.shape != F.shape:
        raise ValueError("sg_solve_host: U must be a contiguous FP64 CPU tensor shaped like F")
    o = opts or solve_opts()
    st = _lib.sg_solve_stats()
    status = _lib.LIB.sg_solve_host(h.h, C.c_void_p(F.data_ptr()), C.c_void_p(U.data_ptr()), C.byref(o),
                                    C.byref(st), _stream())
    stats = _stats(status, st)
    if raise_on_error:
        check(status, "sg_solve_host")
    return U, stats


def sg_autotune(h: SGProblem):
    """Time the SG product's candidate block sizes on this problem and keep the
    fastest; returns ``(threads_f64, threads_f32)``."""
    check(_lib.LIB.sg_autotune(h.h, _stream()), "sg_autotune")
    a, b = C.c_int(0), C.c_int(0)
    check(_lib.LIB.sg_autotune_result(h.h, C.byref(a), C.byref(b)), "sg_autotune_result")
    return a.value, b.value


def sg_autotune_forms(h: SGProblem):
    """Forms sg_autotune chose: ``(pairs_f64, pairs_f32, pairs_outer)``, 1 the
    pair form, 0 the gather form."""
    a, b, c = C.c_int(0), C.c_int(0), C.c_int(0)
    check(_lib.LIB.sg_autotune_forms(h.h, C.byref(a), C.byref(b), C.byref(c)), "sg_autotune_forms")
    return a.value, b.value, c.value


def sg_autotune_shapes(h: SGProblem):
    """All tuned shapes: ``(threads_f64, threads_f32, threads_outer, pairs_f64,
    pairs_f32, pairs_outer)`` (0 threads: the built-in choice)."""
    a, b, c = C.c_int(0), C.c_int(0), C.c_int(0)
    check(_lib.LIB.sg_autotune_result(h.h, C.byref(a), C.byref(b)), "sg_autotune_result")
    check(_lib.LIB.sg_autotune_outer_result(h.h, C.byref(c)), "sg_autotune_outer_result")
    return (a.value, b.value, c.value) + sg_autotune_forms(h)


def sg_autotune_set(h: SGProblem, threads_f64=0, threads_f32=0, threads_outer=0, pairs_f64=1, pairs_f32=1,
                    pairs_outer=1) -> None:
    """Pin the SG-product shapes without timing (``sg_autotune_set``)."""
    check(_lib.LIB.sg_autotune_set(h.h, threads_f64, threads_f32, threads_outer, pairs_f64, pairs_f32, pairs_outer),
          "sg_autotune_set")


def sg_measure_alu_peak(dtype: int = SG_F64, iters: Optional[int] = None) -> float:
    """Measured FMA throughput of the current device in FLOP/s (FP64 or FP32)."""
    it = iters if iters is not None else (4096 if dtype == SG_F64 else 131072)
    out = C.c_double(0.0)
    check(_lib.LIB.sg_measure_alu_peak(dtype, it, C.byref(out), _stream()), "sg_measure_alu_peak")
    return out.value


class SGBatch:
    """Many independent SG systems solved by one graph launch (``sg_batch_*``).
    The problems stay owned by the caller and must outlive the batch."""

    def __init__(self, problems):
        self.problems = list(problems)
        arr = (C.c_void_p * len(self.problems))(*[p.h for p in self.problems])
        out = C.c_void_p()
        check(_lib.LIB.sg_batch_create(len(self.problems), arr, C.byref(out)), "sg_batch_create")
        self.b = out.value

    def solve(self, Fs, opts=None, Us=None, raise_on_error=True):
        """Solve every system; returns ``(list of U, list of SolveStats)``."""
        count = len(self.problems)
        if len(Fs) != count or (Us is not None and len(Us) != count):
            raise ValueError(f"need {count} right-hand sides (and solution blocks)")
        for i, h in enumerate(self.problems):
            _block(h, Fs[i], f"SGBatch.solve: F[{i}]")
            _block(h, None if Us is None else Us[i], f"SGBatch.solve: U[{i}]")
        Us = [torch.empty_like(F) for F in Fs] if Us is None else list(Us)
        o = opts or solve_opts()
        st = (_lib.sg_solve_stats * count)()
        fp = (C.c_void_p * count)(*[_ptr(F) for F in Fs])
        up = (C.c_void_p * count)(*[_ptr(U) for U in Us])
        status = _lib.LIB.sg_batch_solve(self.b, fp, up, C.byref(o), st, _stream())
        stats = [_stats(st[i].status, st[i]) for i in range(count)]
        if raise_on_error:
            check(status, "sg_batch_solve")
        return Us, stats

    def solve_host(self, Fs, opts=None, Us=None, raise_on_error=True):
        """``solve`` on host blocks (contiguous FP64 CPU tensors; pinned ones
        are read and written by the library's kernels directly)."""
        count = len(self.problems)
        if len(Fs) != count or (Us is not None and len(Us) != count):
            raise ValueError(f"need {count} right-hand sides (and solution blocks)")
        Us = [torch.empty_like(F) for F in Fs] if Us is None else list(Us)
        for T in list(Fs) + Us:
            if T.is_cuda or not T.is_contiguous() or T.dtype != torch.float64:
                raise ValueError("solve_host: blocks must be contiguous FP64 CPU tensors")
        for i, h in enumerate(self.problems):
            _block(h, Fs[i], f"SGBatch.solve_host: F[{i}]")
            _block(h, Us[i], f"SGBatch.solve_host: U[{i}]")
        o = opts or solve_opts()
        st = (_lib.sg_solve_stats * count)()
        fp = (C.c_void_p * count)(*[C.c_void_p(F.data_ptr()) for F in Fs])
        up = (C.c_void_p * count)(*[C.c_void_p(U.data_ptr()) for U in Us])
        status = _lib.LIB.sg_batch_solve_host(self.b, fp, up, C.byref(o), st, _stream())
        stats = [_stats(st[i].status, st[i]) for i in range(count)]
        if raise_on_error:
            check(status, "sg_batch_solve_host")
        return Us, stats

    def close(self):
        if getattr(self, "b", None):
            _lib.LIB.sg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sg_qoi(h: SGProblem, U: torch.Tensor, want_grad: bool = True):
    """``Q = sum_j u_j^T M_h u_j`` (device scalar) and ``dQ/dU = 2 M_h U``."""
    _block(h, U, "sg_qoi: U")
    q = torch.empty(1, dtype=torch.float64, device="cuda")
    dq = torch.empty_like(U) if want_grad else None
    check(_lib.LIB.sg_qoi(h.h, _ptr(U), _ptr(dq), _ptr(q), _stream()), "sg_qoi")
    return q, dq


def sg_qoi_grad(h: SGProblem, U: torch.Tensor, Lam: torch.Tensor, W: np.ndarray):
    """``grad[t] = sum_k W[t,k] <Lam, A_k U G_k^T>``; returns ``(grad, h_k)``."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    if W.ndim != 2 or W.shape[1] != h.nterm or W.shape[0] < 1:
        raise ValueError(f"sg_qoi_grad: W must have shape (parameters, {h.nterm}) (one column per value term)")
    _block(h, U, "sg_qoi_grad: U")
    _block(h, Lam, "sg_qoi_grad: Lam")
    nparam = W.shape[0]
    grad = torch.empty(nparam, dtype=torch.float64, device="cuda")
    hk = torch.empty(h.nterm, dtype=torch.float64, device="cuda")
    check(_lib.LIB.sg_qoi_grad(h.h, _ptr(U), _ptr(Lam), nparam, W.ctypes.data_as(C.POINTER(C.c_double)),
                               _ptr(grad), _ptr(hk), _stream()), "sg_qoi_grad")
    return grad, hk


def sg_set_scales(h: SGProblem, scale) -> None:
    """``A_k := scale[k] * A_k`` (relative to the matrices given to sg_setup)."""
    sc = np.ascontiguousarray(scale, dtype=np.float64)
    if sc.shape != (h.nterm,):
        raise ValueError(f"need one scale per value term ({h.nterm}: M+1, or C(M+q, M) for a gPC coefficient)")
    check(_lib.LIB.sg_set_scales(h.h, sc.ctypes.data_as(C.POINTER(C.c_double))), "sg_set_scales")


# ---------------------------------------------------------------------------
# Quantity of interest Q = E[int u^2] and its adjoint gradient (K7)
# ---------------------------------------------------------------------------

def _theta_arg(h: SGProblem, theta) -> np.ndarray:
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1))
    if th.shape != (h.M + 2,):
        raise ValueError(f"theta must have M+2 = {h.M + 2} entries (a_mean, sigma, s_1..s_M)")
    return th


def sg_kl_set_theta(h: SGProblem, theta) -> None:
    """A_0 = a_mean L_h, A_k = sigma s_k Phi_k for theta = (a_mean, sigma,
    s_1..s_M) on a handle holding the unit-parameter matrices."""
    th = _theta_arg(h, theta)
    check(_lib.LIB.sg_kl_set_theta(h.h, th.ctypes.data_as(C.POINTER(C.c_double))), "sg_kl_set_theta")


def sg_kl_qoi_grad(h: SGProblem, U: torch.Tensor, Lam: torch.Tensor, theta) -> torch.Tensor:
    """dQ/dtheta (device, M+2) from the forward and adjoint solutions."""
    th = _theta_arg(h, theta)
    _block(h, U, "sg_kl_qoi_grad: U")
    _block(h, Lam, "sg_kl_qoi_grad: Lam")
    grad = torch.empty(h.M + 2, dtype=torch.float64, device="cuda")
    check(_lib.LIB.sg_kl_qoi_grad(h.h, _ptr(U), _ptr(Lam), th.ctypes.data_as(C.POINTER(C.c_double)), _ptr(grad),
                                  None, _stream()), "sg_kl_qoi_grad")
    return grad


class SGQoI(torch.autograd.Function):
    """Q(theta) = sum_j u_j^T M_h u_j with (sum_k G_k (x) A_k(theta)) u = f.

    Forward: one preconditioned solve and the mass contraction. Backward: the
    operator is symmetric, so the adjoint Lam solves the same system with the
    right-hand side dQ/du = 2 (M_h (x) I) u; the gradient is the fused K7
    contraction (sg_kl_qoi_grad). The handle must hold the unit-parameter
    matrices (a_mean = 1, sigma = 1, s_k = 1)."""

    @staticmethod
    def forward(ctx, theta, h, F, opts):
        th = theta.detach().double().cpu().numpy()
        sg_kl_set_theta(h, th)
        U, _ = sg_solve(h, F, opts)
        q, dq = sg_qoi(h, U)
        ctx.h, ctx.opts, ctx.th = h, opts, th
        ctx.save_for_backward(U, dq)
        return q[0].to(theta.dtype)

    @staticmethod
    def backward(ctx, gQ):
        U, dq = ctx.saved_tensors
        h = ctx.h
        sg_kl_set_theta(h, ctx.th)
        Lam, _ = sg_solve(h, dq, ctx.opts)
        grad = sg_kl_qoi_grad(h, U, Lam, ctx.th)
        return (gQ.to(grad.dtype) * grad).to(gQ.dtype), None, None, None


class SGGradBatch:
    """Q and dQ/dtheta for a batch of parameter sets, batched on the device:
    ``count`` handles of the same unit-parameter problem, each set to one
    theta, solved together in one graph launch (SGBatch) for the forward
    solves and in a second one for the adjoint solves, then the QoI and the K7
    contraction per set."""

    def __init__(self, ne_x: int, ne_y: int, M: int, p: int, rowptr, colidx, vals, mass, count: int,
                 family: int = SG_LEGENDRE):
        self.count = count
        self.hs = [SGProblem(ne_x, ne_y, M, p, rowptr, colidx, vals, mass, family) for _ in range(count)]
        self.batch = SGBatch(self.hs)
        self.M = M

    @classmethod
    def from_inputs(cls, prob, p: int, count: int, family: int = SG_LEGENDRE) -> "SGGradBatch":
        return cls(prob.ne, prob.ne, prob.M, p, prob.rowptr, prob.colidx, prob.vals, prob.mass, count, family)

    def autotune(self):
        """Tune the first handle; the others share its problem class (cached)."""
        for h in self.hs:
            sg_autotune(h)

    def value_and_grad(self, thetas, F: torch.Tensor, opts=None):
        """``(Q[count], dQ/dtheta[count, M+2])`` on the device for the rows of
        ``thetas``; ``F`` is the right-hand side shared by every set."""
        th = np.asarray(thetas, dtype=np.float64)
        if th.shape != (self.count, self.M + 2):
            raise ValueError(f"thetas must have shape ({self.count}, {self.M + 2})")
        o = opts or solve_opts()
        for h, t in zip(self.hs, th):
            sg_kl_set_theta(h, t)
        Us, _ = self.batch.solve([F] * self.count, o)
        qs, dqs = zip(*[sg_qoi(h, U) for h, U in zip(self.hs, Us)])
        Lams, _ = self.batch.solve(list(dqs), o)
        grads = [sg_kl_qoi_grad(h, U, Lam, t) for h, U, Lam, t in zip(self.hs, Us, Lams, th)]
        return torch.cat(qs), torch.stack(grads)

    def close(self):
        self.batch.close()
        for h in self.hs:
            h.close()


def sg_qoi_value_and_grad_batch(h: SGProblem, thetas, F: torch.Tensor, opts=None):
    """Q and dQ/dtheta for a batch of parameter sets (rows of ``thetas``) on
    one handle, one forward and one adjoint solve per set through SGQoI (the
    autograd path); SGGradBatch runs the same sets batched on the device."""
    o = opts or solve_opts()
    out_q, out_g = [], []
    for th in np.asarray(thetas, dtype=np.float64):
        t = torch.tensor(th, dtype=torch.float64, device=F.device, requires_grad=True)
        q = SGQoI.apply(t, h, F, o)
        q.backward()
        out_q.append(q.detach())
        out_g.append(t.grad.detach())
    return torch.stack(out_q), torch.stack(out_g)
