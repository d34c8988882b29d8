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
the two arithmetics. The FP32 row kernel's bar is checked the same way, and
so are the top-level products of Algorithm 1 (FP64 Yin converted to
double-float with integer operations, FP32 output): there the final FP32
rounding alone takes up to 2^-24 |exact| of the bar's 6e-8 |exact|, so the
model comes close to the bar without crossing it.
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


def _from_double(x: float):
    """FP64 -> double-float as the level products convert Yin, with integer
    operations only: hi keeps the sign, the exponent and the top 23 fraction
    bits (truncated, so exact), lo the next 29 bits renormalised from their
    leading one and truncated to 24 bits."""
    import struct
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    E = (b >> 52) & 0x7FF
    if E == 0:
        return f32(0.0), f32(0.0)
    eh = E - 1023 + 127
    if eh < 1 or eh > 254:
        return f32(x), f32(0.0)
    sign = (b >> 32) & 0x80000000
    as_f32 = lambda bits: np.frombuffer(struct.pack("<I", bits), dtype=np.float32)[0]
    hi = as_f32(sign | (eh << 23) | ((b >> 29) & 0x7FFFFF))
    m29 = b & 0x1FFFFFFF
    if m29 == 0:
        return hi, f32(0.0)
    t = m29.bit_length() - 1
    el = t + E - 1075 + 127
    if el < 1:
        return hi, f32(0.0)
    frac = (m29 >> (t - 23)) & 0x7FFFFF if t >= 23 else (m29 << (23 - t)) & 0x7FFFFF
    return hi, as_f32(sign | (el << 23) | frac)


def test_fp64_to_double_float_conversion_error():
    """The conversion's error: within 2^-47 |x| + 2^-125 of x over the normal
    FP32 range of hi (the part of lo that would fall under that range is
    dropped, which costs less than 2^-125), so within 2^-47 |x| from
    |x| >= 2^-79 up; sampled over the whole range and at the edges (a zero
    low part, low bits only just above or below the range)."""
    rng = np.random.default_rng(47)
    xs = list((1 + rng.random(3000)) * 2.0 ** rng.integers(-126, 128, size=3000) * rng.choice([-1, 1], 3000))
    xs += [1.0, -1.0, 3.0, 1.0 + 2.0 ** -30]
    xs += [(1 + 2.0 ** -k) * 2.0 ** e for e in (-126, -110, -100, -90, -80, -79) for k in (24, 30, 40, 45, 52)]
    for x in xs:
        hi, lo = _from_double(float(x))
        err = abs(Fr(float(hi)) + Fr(float(lo)) - Fr(float(x)))
        assert err <= Fr(2) ** -47 * abs(Fr(float(x))) + Fr(2) ** -125, x
        if abs(x) >= 2.0 ** -79:
            assert err <= Fr(2) ** -47 * abs(Fr(float(x))), x
    assert _from_double(0.0) == (0.0, 0.0)


def test_double_float_level_product_within_the_parity_bar():
    """The level products of Algorithm 1 at the top level, Y = Yin - sum (FP64
    Yin, FP32 X, FP32 output), as the kernel forms them: the sum in
    double-float, Yin converted exactly to 47 bits, the difference in
    double-float, one rounding to FP32. Against the GPU tests' bar
    m 2^-46 (|Yin| + sum|terms|) + 6e-8 |exact|."""
    M, p = 10, 4
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    prob = S.make_problem(16, M, 0.3, 0.5)
    rng = np.random.default_rng(4)
    m = 9 * (1 + 2 * M)
    worst = 0.0
    for trial in range(150):
        r = int(rng.integers(0, prob.n))
        A = prob.vals[prob.rowptr[r]:prob.rowptr[r + 1]]
        nz = A.shape[0]
        lo_, li = (p - 1, p) if trial % 2 else (p, p - 1)
        l = int(rng.integers(off[lo_], off[lo_ + 1]))
        coup = [(k, int(j), float(G[k][l, j])) for k in range(1, M + 1) for j in G[k][l].indices
                if off[li] <= j < off[li + 1]]
        X = {j: (rng.standard_normal(nz) * 10.0 ** rng.integers(-3, 4)).astype(np.float32) for _, j, _ in coup}
        yin = float(rng.standard_normal() * 10.0 ** rng.integers(-3, 4))
        acc, total, mag = (f32(0.0), f32(0.0)), Fr(0), Fr(0)
        for k, j, c in coup:
            s = _mul_f(_split(A[0, k]), X[j][0])
            for e in range(1, nz):
                s = _add(s, _mul_f(_split(A[e, k]), X[j][e]))
            acc = _add(acc, _mul(_split(c), s))
            t = [Fr(float(A[e, k])) * Fr(float(X[j][e])) for e in range(nz)]
            total += Fr(c) * sum(t)
            mag += abs(Fr(c)) * sum(abs(v) for v in t)
        s_ = acc[0] + acc[1]
        acc = (s_, acc[1] - (s_ - acc[0]))
        v = _add(_from_double(yin), (-acc[0], -acc[1]))
        y = v[0] + v[1]
        exact = Fr(yin) - total
        bar = m * Fr(2) ** -46 * (abs(Fr(yin)) + mag) + Fr(6e-8) * abs(exact)
        worst = max(worst, float(abs(Fr(float(y)) - exact) / bar))
    assert worst < 1.0, worst
