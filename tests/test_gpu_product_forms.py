"""The product kernels chosen by shape: the FP32 row kernel (input columns in
registers, term sums in shared memory) for the full SG product (eq. (3)'s sum
over the KL terms) and the level products B_l, C_l of Algorithm 1 with at
least 512 input columns, or 128 input and 512 output columns; the
thread-per-output kernel for level products into at most 16 columns. Against
the oracle within the rounding bound, against the row-per-warp kernels (the
same products with the shape-specific kernels switched off), and inside the
FP32 preconditioner."""
import numpy as np
import pytest

import sg_inputs as S
from oracle import gmg, hsc, krylov, sg_operator as so
from tests.gpu_common import abs_bound, problem

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


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


# P = 1001, 924 and 680 columns; 9 x 9, 8 x 8 (not a power of two) and 5 x 5 nodes
SHAPES = [(8, 10, 4), (7, 6, 6), (4, 14, 3)]


@pytest.mark.parametrize("ne,M,p", SHAPES)
def test_rows32_full_product(lib, ne, M, p, monkeypatch):
    """Y = sum_k A_k U G_k^T in FP32: within m u sum|terms| of the exact
    product (m: the longest chain of roundings, nine nonzeros per pair sum
    plus the 2M + 1 couplings of an output), and within twice that of the
    row-per-warp kernel."""
    import torch
    prob, A, G, off = problem(ne, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    assert h.P >= 512
    U = S.random_block(prob.n, h.P, seed=11).astype(np.float32)
    Y = _np(lib.sg_apply(h, _t(U, torch.float32)))
    U = U.astype(np.float64)
    ref = so.sg_apply(A, G, U)
    bound = abs_bound(A, G, U)
    m = 9 + 2 * M + 2
    assert np.all(np.abs(Y - ref) <= m * U32 * bound + 1e-300)
    monkeypatch.setenv("SGHSC_GENERIC_PRODUCTS", "1")
    hg = lib.SGProblem.from_inputs(prob, p)
    Yg = _np(lib.sg_apply(hg, _t(U, torch.float32)))
    assert np.all(np.abs(Y - Yg) <= 2 * m * U32 * bound + 1e-300)
    h.close()
    hg.close()


@pytest.mark.parametrize("ne,M,p", [(8, 10, 4), (4, 14, 3)])
def test_rows32_wide_level_products(lib, ne, M, p):
    """Y = Yin - sum_k A_k X G_k[out, in]^T in FP32 between the two top
    levels in both directions (715 -> 220 and 220 -> 715 columns at M = 10,
    560 -> 120 at M = 14; 120 -> 560 stays on the row-per-warp kernel),
    within the FP32 bound of the exact value."""
    import torch
    prob, A, G, off = problem(ne, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    m = 9 + 2 * M + 3
    for lo, li in ((p - 1, p), (p, p - 1)):
        win, wout = off[li + 1] - off[li], off[lo + 1] - off[lo]
        X = S.random_block(prob.n, win, seed=lo + 10 * li).astype(np.float32)
        Yin = S.random_block(prob.n, wout, seed=5 + lo).astype(np.float32)
        Y = _np(lib.sg_level_apply(h, lo, li, _t(X, torch.float32), _t(Yin, torch.float32)))
        X, Yin = X.astype(np.float64), Yin.astype(np.float64)
        exact = Yin - so.level_apply(A, G, off, lo, li, X)
        bound = np.abs(Yin) + so.level_apply([abs(a) for a in A], [abs(g) for g in G], off, lo, li, np.abs(X))
        assert np.all(np.abs(Y - exact) <= m * U32 * bound + 1e-300), (lo, li)
    h.close()


def test_rows32_inside_the_fp32_preconditioner(lib):
    """Algorithm 1 in FP32 at P = 1001 (its level-4 products on the row
    kernel, the pre product in place) against the oracle's Algorithm 1 with the identical
    inner solver (four V-cycle-preconditioned CG steps per D_l solve)."""
    prob, A, G, off = problem(8, 10, 4)
    h = lib.SGProblem.from_inputs(prob, 4)
    lv = gmg.hierarchy(A[0], 8)

    def dsolve(l, X):
        return krylov.pcg_columns(lambda v: A[0] @ v, X, lambda r: gmg.vcycle(lv, r), tol=0.0, maxit=4,
                                  fixed_iters=4)[0]

    R = S.random_block(prob.n, h.P, seed=9)
    o = lib.prec_opts(precision=lib.SG_F32, inner_fixed_iters=4)
    Z = _np(lib.hsc_precond_apply(h, _t(R), o))
    ref = hsc.hsc_apply(A, G, off, R, dsolve=dsolve)
    assert np.abs(Z - ref).max() <= 2e-5 * np.abs(ref).max()
    h.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("ne,M,p", [(8, 10, 4), (7, 3, 3)])
def test_narrow_level_products(lib, ne, M, p, prec, monkeypatch):
    """The level products into at most 16 columns (one thread per row and
    output: B_1, C_1, B_2 at M = 10; every level at M = 3), in place as the
    preconditioner applies them, against the oracle within m u sum|terms| and
    against the staged kernels."""
    import torch
    prob, A, G, off = problem(ne, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    monkeypatch.setenv("SGHSC_GENERIC_PRODUCTS", "1")
    hg = lib.SGProblem.from_inputs(prob, p)
    dt, u = (torch.float64, 2.0 ** -53) if prec == "f64" else (torch.float32, U32)
    m = 9 * (2 * M + 1) + 2
    for lo, li in [(l - 1, l) for l in range(1, p + 1)] + [(l, l - 1) for l in range(1, p + 1)]:
        win, wout = off[li + 1] - off[li], off[lo + 1] - off[lo]
        if wout > 16:
            continue
        X = S.random_block(prob.n, win, seed=lo + 10 * li)
        Yin = S.random_block(prob.n, wout, seed=5 + lo)
        if prec == "f32":
            X, Yin = X.astype(np.float32).astype(np.float64), Yin.astype(np.float32).astype(np.float64)
        Yt = _t(Yin, dt)
        lib.sg_level_apply(h, lo, li, _t(X, dt), Yt, Yt)       # in place
        Y = _np(Yt)
        Yg = _np(lib.sg_level_apply(hg, lo, li, _t(X, dt), _t(Yin, dt)))
        exact = Yin - so.level_apply(A, G, off, lo, li, X)
        bound = np.abs(Yin) + so.level_apply([abs(a) for a in A], [abs(g) for g in G], off, lo, li, np.abs(X))
        assert np.all(np.abs(Y - exact) <= m * u * bound + 1e-300), (lo, li)
        assert np.all(np.abs(Y - Yg) <= 2 * m * u * bound + 1e-300), (lo, li)
    h.close()
    hg.close()


@pytest.mark.parametrize("M,p,n", [(6, 4, 203), (10, 4, 61)])
def test_ragged_rows_on_the_row_kernels(lib, M, p, n, monkeypatch):
    """Ragged CSR rows (empty rows, rows of up to 23 nonzeros: several chunks
    of nine) through the FP32 row kernel at every shape it takes (two rows per
    block at 56 <-> 126 columns, one row per block on the full product and at
    715 <-> 220), and the narrow kernel, against the oracle, with an odd row
    count so the last block holds a single row."""
    import torch
    from tests.gpu_common import random_csr
    from oracle import chaos
    rowptr, colidx = random_csr(n, seed=8, max_row=23)
    rng = np.random.default_rng(9)
    vals = rng.uniform(-1, 1, size=(len(colidx), M + 1))
    h = lib.SGProblem(0, 0, M, p, rowptr, colidx, vals)
    A = so.kl_matrices(rowptr, colidx, vals)
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    m = 23 + 2 * M + 3
    U = S.random_block(n, h.P, seed=3).astype(np.float32)
    Y = _np(lib.sg_apply(h, _t(U, torch.float32)))
    U = U.astype(np.float64)
    assert np.all(np.abs(Y - so.sg_apply(A, G, U)) <= m * U32 * abs_bound(A, G, U) + 1e-300)
    assert np.all(Y[3::7] == 0.0)
    for lo, li in [(l - 1, l) for l in range(1, p + 1)] + [(l, l - 1) for l in range(1, p + 1)]:
        win, wout = off[li + 1] - off[li], off[lo + 1] - off[lo]
        X = S.random_block(n, win, seed=lo + 10 * li).astype(np.float32).astype(np.float64)
        Yin = S.random_block(n, wout, seed=5 + lo).astype(np.float32).astype(np.float64)
        Yl = _np(lib.sg_level_apply(h, lo, li, _t(X, torch.float32), _t(Yin, torch.float32)))
        exact = Yin - so.level_apply(A, G, off, lo, li, X)
        bound = np.abs(Yin) + so.level_apply([abs(a) for a in A], [abs(g) for g in G], off, lo, li, np.abs(X))
        assert np.all(np.abs(Yl - exact) <= m * U32 * bound + 1e-300), (lo, li)
    h.close()
