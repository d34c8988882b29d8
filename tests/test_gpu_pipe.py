"""The row-pipelined sweeps of the batched inner solver (grids of at least
60000 nodes, FP32 batches of 64 columns or more) against the FP64 oracle and
against the node-by-node kernels (SGHSC_NO_PIPE=1), on seeded inputs: fixed
iteration counts element by element, and a tolerance-driven solve by its true
residuals and iteration counts."""
import os

import numpy as np
import pytest

import sg_inputs as S
from oracle import gmg, krylov
from tests.gpu_common import problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1205_1864_gb300 as L
    return L


def _t(x, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype or torch.float64, device="cuda")


def _np(t):
    return t.double().cpu().numpy()


@pytest.fixture(scope="module")
def big(lib):
    """256 x 256 mesh (65025 nodes): a handle on the pipelined sweeps and one
    on the node-by-node kernels."""
    prob, A, G, off = problem(256, 2, 1)
    h1 = lib.SGProblem.from_inputs(prob, 1)
    os.environ["SGHSC_NO_PIPE"] = "1"
    try:
        h0 = lib.SGProblem.from_inputs(prob, 1)
    finally:
        del os.environ["SGHSC_NO_PIPE"]
    return prob, A, h1, h0


@pytest.mark.parametrize("w,nu", [(64, 2), (100, 3), (131, 1)])
def test_pipe_fixed_iterations_parity(lib, big, w, nu):
    """Two V-cycle-preconditioned CG steps per column (nu sweeps) against the
    column-wise oracle, for batch widths that fill 1, 2 and 3 column chunks
    (131: a partial last chunk); a zero column stays zero."""
    import torch
    prob, A, h1, h0 = big
    lv = gmg.hierarchy(A[0], 256)
    B = S.random_block(prob.n, w, seed=50 + w).astype(np.float32).astype(np.float64)
    B[:, 5] = 0.0
    o = lib.prec_opts(inner_fixed_iters=2, nu=nu)
    X, it = lib.sg_inner_solve(h1, _t(B, torch.float32), o)
    ref, it_ref = krylov.pcg_columns(lambda v: A[0] @ v, B, lambda r: gmg.vcycle(lv, r, nu=nu, omega=0.8),
                                     tol=0.0, maxit=2, fixed_iters=2)
    assert list(it) == list(it_ref)
    X = _np(X)
    scale = np.abs(ref).max(axis=0, keepdims=True) + 1e-300
    assert np.all(np.abs(X - ref) <= 1e-4 * scale)
    assert np.all(X[:, 5] == 0.0)
    X0, _ = lib.sg_inner_solve(h0, _t(B, torch.float32), o)
    assert np.all(np.abs(X - _np(X0)) <= 2e-5 * scale)


def test_pipe_tolerance_matches_node_by_node(lib, big):
    import torch
    prob, A, h1, h0 = big
    B = S.random_block(prob.n, 96, seed=61)
    B[:, ::7] *= 1e-3
    o = lib.prec_opts(inner_tol=1e-2)
    X1, it1 = lib.sg_inner_solve(h1, _t(B, torch.float32), o)
    X0, it0 = lib.sg_inner_solve(h0, _t(B, torch.float32), o)
    B32 = B.astype(np.float32).astype(np.float64)
    res = np.linalg.norm(B32 - A[0] @ _np(X1), axis=0) / np.linalg.norm(B32, axis=0)
    assert np.all(res <= 2e-2)
    assert np.all(np.abs(np.asarray(it1) - np.asarray(it0)) <= 1)
