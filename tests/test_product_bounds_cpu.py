"""The error bounds of the FP32 and double-float product parity tests,
checked on the CPU.

The GPU tests accept a double-float SG product entry when it lies within
m 2^-46 sum|terms| (+ 2^-52 |exact|) of the exact value, m the products of the
entry. This file checks that bar against the arithmetic it is derived from:
the kernel's sequence of FP32 operations for one output entry (nine-term
stencil sums of a double-float coefficient times an FP32 input, each sum then
times a double-float coupling weight and accumulated, normalised, finished in
FP64) is modelled with correctly rounded FP32 operations and a fused
multiply-add evaluated exactly and rounded once, and compared with the exact
rational value on rows and outputs of the 10-variable, degree-4 operator
(P = 1001). The model stays well inside the bar, and the same sums with the
low parts dropped (plain FP32 accumulation) break it, so the bar separates
the two arithmetics. The FP32 row kernel's bar is checked the same way.
"""
from fractions import Fraction as Fr

import numpy as np

import sg_inputs as S
from oracle import chaos

f32 = np.float32


def _round32(q: Fr) -> np.float32:
    """Round an exact rational to the nearest FP32 value, ties to even."""
    if q == 0:
        return f32(0.0)
    x = float(q)                     # correctly rounded to FP64
    f = f32(x)
    if float(f) != x:                # FP64 -> FP32 can round twice only at an FP32 midpoint
        lo = f if float(f) < x else np.nextafter(f, f32(-np.inf))
        hi = np.nextafter(lo, f32(np.inf))
        mid = (Fr(float(lo)) + Fr(float(hi))) / 2
        if Fr(x) == mid and q != mid:
            f = hi if q > mid else lo
    return f


def _fma(a, b, c):
    return _round32(Fr(float(a)) * Fr(float(b)) + Fr(float(c)))


def _split(v: float):
    h = f32(v)
    return h, f32(v - float(h))


def _mul_f(a, x):                    # double-float times FP32
    p = a[0] * x
    return p, _fma(a[1], x, _fma(a[0], x, -p))


def _mul(a, b):                      # double-float times double-float, lo * lo dropped
    p = a[0] * b[0]
    return p, _fma(a[1], b[0], _fma(a[0], b[1], _fma(a[0], b[0], -p)))


def _add(x, y, keep_lo=True):        # two-sum of the hi parts, lo parts in FP32
    s = x[0] + y[0]
    bb = s - x[0]
    e = (x[0] - (s - bb)) + (y[0] - bb)
    return (s, (x[1] + y[1]) + e) if keep_lo else (s, f32(0.0))


def _entry(A, U, l, coup, keep_lo):
    """One output entry Y(r, l) as the kernel forms it."""
    def dot(k, j):
        s = _mul_f(_split(A[0, k]), U[j][0])
        for e in range(1, A.shape[0]):
            s = _add(s, _mul_f(_split(A[e, k]), U[j][e]), keep_lo)
        return s if keep_lo else (s[0], f32(0.0))

    acc = dot(0, l)
    for k, j, c in coup:
        acc = _add(acc, _mul(_split(c), dot(k, j)), keep_lo)
    s = acc[0] + acc[1]
    acc = (s, acc[1] - (s - acc[0]))
    return float(acc[0]) + float(acc[1])


def test_double_float_product_error_within_the_parity_bar():
    M, p = 10, 4
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    P = G[0].shape[0]
    prob = S.make_problem(16, M, 0.3, 0.5)
    rng = np.random.default_rng(1864)
    worst, worst_fp32 = 0.0, 0.0
    for trial in range(120):
        r = int(rng.integers(0, prob.n))
        A = prob.vals[prob.rowptr[r]:prob.rowptr[r + 1]]          # (nz, M+1) FP64
        nz = A.shape[0]
        l = int(rng.integers(off[1], off[p])) if trial % 2 else int(rng.integers(0, P))
        coup = [(k, int(j), float(G[k][l, j])) for k in range(1, M + 1) for j in G[k][l].indices]
        scale = 10.0 ** rng.integers(-3, 4, size=P)                # columns over six decades, random signs
        U = {j: (rng.standard_normal(nz) * scale[j]).astype(np.float32) for j in [l] + [j for _, j, _ in coup]}
        exact, mag = Fr(0), Fr(0)
        for k, j, c in [(0, l, 1.0)] + coup:
            t = [Fr(float(A[e, k])) * Fr(float(U[j][e])) for e in range(nz)]
            exact += Fr(c) * sum(t)
            mag += abs(Fr(c)) * sum(abs(v) for v in t)
        m = nz * (len(coup) + 1)
        bar = m * Fr(2) ** -46 * mag + Fr(2) ** -52 * abs(exact)
        err = abs(Fr(_entry(A, U, l, coup, True)) - exact)
        worst = max(worst, float(err / bar))
        if trial < 20:
            worst_fp32 = max(worst_fp32, float(abs(Fr(_entry(A, U, l, coup, False)) - exact) / bar))
    assert worst < 0.25, worst            # the model's largest error is a small part of the bar
    assert worst_fp32 > 1e3, worst_fp32   # FP32 accumulation is far outside it


def test_fp32_row_product_error_within_the_parity_bar():
    """The FP32 product's bar, m u sum|terms| with u = 2^-24 and m = 9 + 2M + 2
    (nine stencil terms, up to 2M couplings and the diagonal term, and the FP32
    roundings of the matrix values and coupling weights), against the row
    kernel's operations: each term sum T(k, j) is a product followed by a
    chain of fused multiply-adds over the row's nonzeros, and an output is
    T(0, l) followed by one fused multiply-add c T(k, j) per coupling."""
    M, p = 10, 4
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    P = G[0].shape[0]
    prob = S.make_problem(16, M, 0.3, 0.5)
    rng = np.random.default_rng(1205)
    u, m = Fr(2) ** -24, 9 + 2 * M + 2
    worst = 0.0
    for trial in range(150):
        r = int(rng.integers(0, prob.n))
        A = prob.vals[prob.rowptr[r]:prob.rowptr[r + 1]]
        nz = A.shape[0]
        l = int(rng.integers(off[1], off[p])) if trial % 2 else int(rng.integers(0, P))
        coup = [(k, int(j), float(G[k][l, j])) for k in range(1, M + 1) for j in G[k][l].indices]
        U = {j: rng.standard_normal(nz).astype(np.float32) for j in [l] + [j for _, j, _ in coup]}

        def T(k, j):
            s = f32(A[0, k]) * U[j][0]
            for e in range(1, nz):
                s = _fma(f32(A[e, k]), U[j][e], s)
            return s

        acc = T(0, l)
        for k, j, c in coup:
            acc = _fma(f32(c), T(k, j), acc)
        exact, mag = Fr(0), Fr(0)
        for k, j, c in [(0, l, 1.0)] + coup:
            t = [Fr(float(A[e, k])) * Fr(float(U[j][e])) for e in range(nz)]
            exact += Fr(c) * sum(t)
            mag += abs(Fr(c)) * sum(abs(v) for v in t)
        worst = max(worst, float(abs(Fr(float(acc)) - exact) / (m * u * mag)))
    assert worst < 0.5, worst
