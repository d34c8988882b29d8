"""Host-side behaviour of the C ABI, on a machine without a GPU, through the
built libsghsc.so: the documented option defaults; every entry point that
takes a handle or a batch rejects a NULL one with SG_ERR_INVALID_ARG and a
message; sg_setup and sg_setup_gpc check the pattern, sizes, values and
chaos family before any device call; and where a device is needed and there
is none, the library reports SG_ERR_CUDA and hands out no handle (there is
no CPU fallback)."""
import ctypes as C
import importlib.util
import os

import numpy as np
import pytest

import sg_inputs as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SG_OK, SG_ERR_INVALID_ARG, SG_ERR_CUDA, SG_ERR_UNSUPPORTED = 0, 1, 2, 7
SG_F64, SG_F32 = 0, 1
SG_LEGENDRE, SG_HERMITE = 0, 1


@pytest.fixture(scope="module")
def L():
    spec = importlib.util.spec_from_file_location(
        "sghsc_build", os.path.join(ROOT, "paper_1205_1864_gb300", "build.py"))
    B = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(B)
    B.build()
    from paper_1205_1864_gb300 import _lib
    return _lib


def _err(L):
    msg = L.LIB.sg_last_error()
    return msg.decode() if msg else ""


def test_default_options_are_the_documented_ones(L):
    p = L.sg_prec_opts()
    L.LIB.sg_default_prec_opts(C.byref(p))
    assert (p.precision, p.top_level_f64, p.inner_tol, p.inner_maxit, p.inner_fixed_iters, p.nu, p.omega, p.m0,
            p.level_tol, p.level_maxit, p.md_m0, p.df64) == (SG_F32, 1, 1e-2, 200, 0, 2, 0.8, 0, 1e-8, 500, 0, 0)
    s = L.sg_solve_opts()
    L.LIB.sg_default_solve_opts(C.byref(s))
    assert (s.precond, s.tol, s.maxit, s.flexible, s.use_x0, s.check_true_residual, s.schur_reduced,
            s.schur_inner_tol) == (L.SG_PREC_HSC, 1e-8, 500, 1, 0, 1, 0, 1e-11)
    assert bytes(s.prec) == bytes(p)
    L.LIB.sg_default_prec_opts(None)             # ignored
    L.LIB.sg_default_solve_opts(None)


def test_null_handles_are_rejected(L):
    lib = L.LIB
    po, so, st = L.sg_prec_opts(), L.sg_solve_opts(), L.sg_solve_stats()
    lib.sg_default_prec_opts(C.byref(po))
    lib.sg_default_solve_opts(C.byref(so))
    buf = (C.c_double * 64)()
    dummy = C.cast(buf, C.c_void_p)
    i1, i2, i3 = C.c_int(), C.c_int(), C.c_int()
    d = (C.c_double * 16)()
    calls = {
        "sg_set_scales": lambda: lib.sg_set_scales(None, d),
        "sg_problem_dims": lambda: lib.sg_problem_dims(None, None, None, None, None, None),
        "sg_problem_terms": lambda: lib.sg_problem_terms(None, None, None),
        "sg_chaos_table": lambda: lib.sg_chaos_table(None, None, None),
        "sg_apply": lambda: lib.sg_apply(None, dummy, dummy, SG_F64, None),
        "sg_level_apply": lambda: lib.sg_level_apply(None, 0, 1, dummy, None, dummy, SG_F64, None),
        "sg_vcycle_apply": lambda: lib.sg_vcycle_apply(None, dummy, dummy, 1, SG_F64, C.byref(po), None),
        "sg_vcycle_apply_static": lambda: lib.sg_vcycle_apply_static(None, dummy, dummy, 1, SG_F64, C.byref(po),
                                                                     None),
        "sg_inner_solve": lambda: lib.sg_inner_solve(None, dummy, dummy, 1, SG_F64, C.byref(po), C.byref(i1), None),
        "hsc_precond_apply": lambda: lib.hsc_precond_apply(None, dummy, dummy, C.byref(po), None),
        "mean_precond_apply": lambda: lib.mean_precond_apply(None, dummy, dummy, C.byref(po), None),
        "bgs_precond_apply": lambda: lib.bgs_precond_apply(None, dummy, dummy, C.byref(po), None),
        "sg_solve": lambda: lib.sg_solve(None, dummy, dummy, C.byref(so), C.byref(st), None),
        "sg_solve_host": lambda: lib.sg_solve_host(None, dummy, dummy, C.byref(so), C.byref(st), None),
        "sg_qoi": lambda: lib.sg_qoi(None, dummy, None, dummy, None),
        "sg_qoi_grad": lambda: lib.sg_qoi_grad(None, dummy, dummy, 1, d, d, None, None),
        "sg_kl_set_theta": lambda: lib.sg_kl_set_theta(None, d),
        "sg_kl_qoi_grad": lambda: lib.sg_kl_qoi_grad(None, dummy, dummy, d, d, None, None),
        "sg_autotune": lambda: lib.sg_autotune(None, None),
        "sg_autotune_result": lambda: lib.sg_autotune_result(None, C.byref(i1), C.byref(i2)),
        "sg_autotune_forms": lambda: lib.sg_autotune_forms(None, C.byref(i1), C.byref(i2), C.byref(i3)),
        "sg_autotune_outer_result": lambda: lib.sg_autotune_outer_result(None, C.byref(i1)),
        "sg_autotune_set": lambda: lib.sg_autotune_set(None, 0, 0, 0, 0, 0, 0),
        "sg_batch_create": lambda: lib.sg_batch_create(1, None, C.byref(C.c_void_p())),
        "sg_batch_solve": lambda: lib.sg_batch_solve(None, None, None, C.byref(so), C.byref(st), None),
        "sg_batch_solve_host": lambda: lib.sg_batch_solve_host(None, None, None, C.byref(so), C.byref(st), None),
        "sg_measure_alu_peak": lambda: lib.sg_measure_alu_peak(SG_F64, 1, None, None),
    }
    for name, call in calls.items():
        assert call() == SG_ERR_INVALID_ARG, name
        assert _err(L), name
    # queries without a handle answer "no", destroy of NULL is a no-op
    assert lib.sg_inner_cluster(None) == 0 and lib.sg_inner_path(None, 8, SG_F32) == 0
    lib.sg_destroy(None)
    lib.sg_batch_destroy(None)
    # every entry point the header declares that takes a handle is covered above or is a query / destructor
    from test_library_cpu import _declared
    handled = set(calls) | {"sg_inner_cluster", "sg_inner_path", "sg_destroy", "sg_batch_destroy", "sg_setup",
                            "sg_setup_gpc", "sg_last_error", "sg_kernel_launches", "sg_default_prec_opts",
                            "sg_default_solve_opts"}
    assert set(_declared()) <= handled, set(_declared()) - handled


def _problem():
    prob = S.make_problem(4, 2, 0.3, 0.5)
    return prob, np.ascontiguousarray(prob.rowptr, np.int32), np.ascontiguousarray(prob.colidx, np.int32), \
        np.ascontiguousarray(prob.vals, np.float64)


def _setup(L, mesh, M, p, family, n, nnz, rowptr, colidx, vals, q=None):
    out = C.c_void_p(12345)
    P = C.POINTER
    ip = lambda a: a.ctypes.data_as(P(C.c_int)) if a is not None else None
    dp = lambda a: a.ctypes.data_as(P(C.c_double)) if a is not None else None
    if q is None:
        st = L.LIB.sg_setup(mesh, M, p, family, n, nnz, ip(rowptr), ip(colidx), dp(vals), None, C.byref(out))
    else:
        st = L.LIB.sg_setup_gpc(mesh, M, p, q, family, n, nnz, ip(rowptr), ip(colidx), dp(vals), None,
                                C.byref(out))
    return st, out.value


def test_setup_checks_its_inputs_before_any_device_call(L):
    prob, rp, ci, va = _problem()
    n, nnz = prob.n, prob.nnz
    mesh = C.byref(L.sg_mesh(4, 4))
    bad = []
    rp1 = rp.copy(); rp1[0] = 1
    bad.append(("rowptr[0] != 0", (mesh, 2, 3, SG_LEGENDRE, n, nnz, rp1, ci, va)))
    bad.append(("rowptr[n] != nnz", (mesh, 2, 3, SG_LEGENDRE, n, nnz - 1, rp, ci, va)))
    rp2 = rp.copy(); rp2[3], rp2[4] = rp2[4], rp2[3]
    bad.append(("rowptr not monotone", (mesh, 2, 3, SG_LEGENDRE, n, nnz, rp2, ci, va)))
    ci1 = ci.copy(); ci1[rp[2]] = n
    bad.append(("column out of range", (mesh, 2, 3, SG_LEGENDRE, n, nnz, rp, ci1, va)))
    ci2 = ci.copy(); ci2[rp[2]], ci2[rp[2] + 1] = ci2[rp[2] + 1], ci2[rp[2]]
    bad.append(("columns unsorted", (mesh, 2, 3, SG_LEGENDRE, n, nnz, rp, ci2, va)))
    va1 = va.copy(); va1[5, 1] = np.nan
    bad.append(("non-finite value", (mesh, 2, 3, SG_LEGENDRE, n, nnz, rp, ci, va1)))
    bad.append(("negative degree", (mesh, 2, -1, SG_LEGENDRE, n, nnz, rp, ci, va)))
    bad.append(("negative M", (mesh, -1, 3, SG_LEGENDRE, n, nnz, rp, ci, va)))
    bad.append(("unknown family", (mesh, 2, 3, 7, n, nnz, rp, ci, va)))
    bad.append(("no values", (mesh, 2, 3, SG_LEGENDRE, n, nnz, rp, ci, None)))
    for what, args in bad:
        st, h = _setup(L, *args)
        assert st == SG_ERR_INVALID_ARG and h is None, what
        assert "sg_setup" in _err(L), what
    assert L.LIB.sg_setup(mesh, 2, 3, SG_LEGENDRE, n, nnz, None, None, None, None, None) == SG_ERR_INVALID_ARG
    # the gPC coefficient: Hermite only, degree <= 16, at most 4096 terms
    st, h = _setup(L, mesh, 2, 2, SG_LEGENDRE, n, nnz, rp, ci, va, q=1)
    assert st == SG_ERR_UNSUPPORTED and h is None
    st, h = _setup(L, mesh, 2, 2, SG_HERMITE, n, nnz, rp, ci, va, q=17)
    assert st == SG_ERR_INVALID_ARG and h is None
    st, h = _setup(L, mesh, 2, 2, SG_HERMITE, n, nnz, rp, ci, va, q=-1)
    assert st == SG_ERR_INVALID_ARG and h is None
    big = np.zeros((nnz, 1), np.float64)       # C(10 + 6, 10) = 8008 terms: refused before the values are read
    st, h = _setup(L, mesh, 10, 2, SG_HERMITE, n, nnz, rp, ci, big, q=6)
    assert st == SG_ERR_UNSUPPORTED and "4096" in _err(L) and h is None


def test_without_a_gpu_setup_fails_loudly(L):
    """No CPU fallback: a valid problem on a machine without a CUDA device is
    refused with SG_ERR_CUDA and a message, and no handle is returned."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present: the GPU tests cover setup")
    prob, rp, ci, va = _problem()
    st, h = _setup(L, C.byref(L.sg_mesh(4, 4)), 2, 3, SG_LEGENDRE, prob.n, prob.nnz, rp, ci, va)
    assert st == SG_ERR_CUDA and h is None
    assert _err(L)
    out = C.c_double()
    assert L.LIB.sg_measure_alu_peak(SG_F64, 1, C.byref(out), None) == SG_ERR_CUDA


def test_batch_create_refuses_null_and_repeated_handles(L):
    """sg_batch_create checks its handle list on the host and leaves *out NULL:
    a NULL handle in any position (the first included) and a handle listed
    twice are refused before any device call. The non-NULL values here are
    never dereferenced: the check compares pointers only."""
    lib = L.LIB
    fake = C.c_void_p(0x1000)
    for count, hs in [(1, [None]), (2, [None, fake]), (2, [fake, None]), (2, [fake, fake]), (0, [fake])]:
        arr = (C.c_void_p * max(len(hs), 1))(*hs)
        out = C.c_void_p(12345)
        assert lib.sg_batch_create(count, arr, C.byref(out)) == SG_ERR_INVALID_ARG, hs
        assert out.value is None and "sg_batch_create" in _err(L)
    assert lib.sg_batch_create(1, None, None) == SG_ERR_INVALID_ARG


def _header_structs():
    """Field names and C types of the typedef'd structs in include/sghsc.h, in order."""
    import re
    src = open(os.path.join(ROOT, "include", "sghsc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(.+?)\s+(\w+(?:\s*,\s*\w+)*)\s*(\[[^\]]*\])?$", decl)
            ctype, names, arr = m.group(1), m.group(2), m.group(3)
            for nm in (x.strip() for x in names.split(",")):
                fields.append((nm, ctype, arr))
        out[name] = fields
    return out


def test_binding_structs_and_constants_match_the_header(L):
    """The ctypes mirrors of the option and statistics structs have the
    header's fields, in the header's order, with matching C types (a
    mismatch would shift every later field), and the status, precision and
    family constants have the header's values."""
    import re
    ctype_of = {"int": C.c_int, "double": C.c_double, "long long": C.c_longlong, "sg_prec_opts": L.sg_prec_opts}
    structs = _header_structs()
    for name in ("sg_mesh", "sg_prec_opts", "sg_solve_opts", "sg_solve_stats"):
        want = structs[name]
        got = getattr(L, name)._fields_
        assert [f[0] for f in got] == [f[0] for f in want], name
        for (fname, ftype), (_, ctype, arr) in zip(got, want):
            base = ctype_of[ctype]
            if arr:
                assert issubclass(ftype, C.Array) and ftype._type_ is base, (name, fname)
                n = eval(arr[1:-1].replace("SG_MAX_HIST", str(L.SG_MAX_HIST)))
                assert ftype._length_ == n, (name, fname)
            else:
                assert ftype is base, (name, fname)
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "sghsc.h")).read(), flags=re.S)
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(SG_[A-Z0-9_]+)\s*=\s*(\d+)", src))
    consts["SG_MAX_HIST"] = int(re.search(r"#define SG_MAX_HIST (\d+)", src).group(1))
    for k, v in consts.items():
        assert getattr(L, k) == v, k
    assert len(consts) >= 20


def test_binding_prototypes_match_the_header(L):
    """Every entry point's ctypes declaration takes as many arguments as the
    header's prototype, with the same kind (pointer, int, double, long long)
    in each position, and the same kind of result."""
    import re
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "sghsc.h")).read(), flags=re.S)
    protos = re.findall(r"^\s*([A-Za-z_][\w \*]*?)\s*\b((?:sg|hsc|mean|bgs)_\w+)\s*\(([^;{]*?)\)\s*;", src, flags=re.M | re.S)
    assert len(protos) >= 30

    def kind(ctype_text):
        t = " ".join(ctype_text.replace("const", " ").split())
        if "*" in t:
            return "ptr"
        return {"int": "int", "double": "double", "long long": "longlong", "void": "void"}[t]

    def ckind(ct):
        if ct is None:
            return "void"
        if ct in (C.c_int,):
            return "int"
        if ct is C.c_double:
            return "double"
        if ct is C.c_longlong:
            return "longlong"
        return "ptr"                       # c_void_p, c_char_p and POINTER(...)

    for ret, name, params in protos:
        fn = getattr(L.LIB, name)
        args = [] if params.strip() in ("", "void") else [a.strip() for a in params.split(",")]
        want = [kind(re.sub(r"\b\w+\s*$", "", a) if re.search(r"[\w\*]\s+\**\w+\s*$", a) else a) for a in args]
        assert [ckind(t) for t in fn.argtypes] == want, name
        assert ckind(fn.restype) == kind(ret), name
