"""Parity of the adjoint gradient (K7 behind torch.autograd) with the FP64
oracle's adjoint gradient and with central finite differences, and of the
parameter scaling of the KL matrices."""
import numpy as np
import pytest
import scipy.sparse as sp

import sg_inputs as S
from oracle import chaos, hsc, krylov, qoi, sg_operator as so

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1205_1864_gb300 as L
    return L


def _t(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _tight(L):
    return L.solve_opts(L.prec_opts(precision=L.SG_F64, inner_tol=1e-12), precond=L.SG_PREC_HSC, tol=1e-13,
                        maxit=200)


def _oracle_grad(prob_unit, theta, p):
    """Oracle: scaled KL matrices, forward and adjoint solves by the oracle's
    HSC-preconditioned CG to 1e-14, then the adjoint contraction."""
    A = so.kl_matrices(prob_unit.rowptr, prob_unit.colidx, prob_unit.vals)
    scales = np.concatenate([[theta[0]], theta[1] * theta[2:]])
    A = [s * a for s, a in zip(scales, A)]
    G = chaos.g_matrices(prob_unit.M, p)
    _, off = chaos.multi_indices(prob_unit.M, p)
    F = S.make_rhs(prob_unit, p)
    Mh = sp.csr_matrix((prob_unit.mass, prob_unit.colidx, prob_unit.rowptr), shape=(prob_unit.n, prob_unit.n))
    a0 = hsc.A0Solver(A[0])
    ap = lambda X: so.sg_apply(A, G, X)
    pre = lambda R: hsc.hsc_apply(A, G, off, R, a0solve=a0)
    U, _ = krylov.fcg(ap, F, pre, tol=1e-14, maxit=200)
    Lam, _ = krylov.fcg(ap, 2.0 * (Mh @ U), pre, tol=1e-14, maxit=200)
    return qoi.qoi(U, Mh), qoi.qoi_grad(A, G, U, Lam, theta[0], theta[1], theta[2:])


def test_set_scales_matches_reassembled_problem(lib):
    unit = S.make_unit_problem(16, 3, 0.5)
    real = S.make_problem(16, 3, 0.23, 0.5, a_mean=1.1)
    h = lib.SGProblem.from_inputs(unit, 2)
    lib.sg_kl_set_theta(h, S.theta_of(real))
    U = S.random_block(unit.n, h.P, seed=4)
    Y = lib.sg_apply(h, _t(U)).cpu().numpy()
    A = so.kl_matrices(real.rowptr, real.colidx, real.vals)
    ref = so.sg_apply(A, chaos.g_matrices(3, 2), U)
    assert np.abs(Y - ref).max() <= 1e-12 * np.abs(ref).max()
    # the multigrid hierarchy follows the mean scale: the preconditioned solve still converges
    F = _t(S.make_rhs(real, 2))
    _, st = lib.sg_solve(h, F, lib.solve_opts(tol=1e-10))
    assert st.iterations < 20


def test_autograd_gradient_matches_oracle(lib):
    import torch
    ne, M, p = 16, 3, 2
    unit = S.make_unit_problem(ne, M, 0.5)
    theta = S.theta_of(S.make_problem(ne, M, 0.2, 0.5, a_mean=1.05))
    h = lib.SGProblem.from_inputs(unit, p)
    F = _t(S.make_rhs(unit, p))
    t = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    q = lib.SGQoI.apply(t, h, F, _tight(lib))
    q.backward()
    q_ref, g_ref = _oracle_grad(unit, theta, p)
    assert float(q.item()) == pytest.approx(q_ref, rel=1e-10)
    g = t.grad.cpu().numpy()
    assert np.abs(g - g_ref).max() <= 1e-6 * np.abs(g_ref).max()


def test_gradient_matches_central_differences(lib):
    import torch
    ne, M, p = 8, 2, 2
    unit = S.make_unit_problem(ne, M, 0.6)
    theta = S.theta_of(S.make_problem(ne, M, 0.25, 0.6, a_mean=0.9))
    h = lib.SGProblem.from_inputs(unit, p)
    F = _t(S.make_rhs(unit, p))
    o = _tight(lib)
    t = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    q = lib.SGQoI.apply(t, h, F, o)
    q.backward()
    g = t.grad.cpu().numpy()
    step = 1e-6
    fd = np.zeros_like(theta)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += step
        tm[i] -= step
        qp = lib.SGQoI.apply(torch.tensor(tp, dtype=torch.float64, device="cuda"), h, F, o).item()
        qm = lib.SGQoI.apply(torch.tensor(tm, dtype=torch.float64, device="cuda"), h, F, o).item()
        fd[i] = (qp - qm) / (2 * step)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()


def test_gradient_batch_of_16_cfg4(lib):
    """Gradient workload: 64x64 grid, M = 4, p = 3, sixteen seeded parameter
    sets evaluated batched on the device (forward and adjoint solves of all
    sets in one graph launch each); every set against the oracle's adjoint
    gradient, and the batch against the one-set-at-a-time autograd path."""
    from concurrent.futures import ThreadPoolExecutor
    c = S.CONFIGS["cfg4_grad_64x64_M4_p3"]
    unit = S.make_unit_problem(c["ne"], c["M"], c["corr_len"])
    base_s = S.theta_of(S.make_problem(c["ne"], c["M"], 1.0, c["corr_len"]))[2:]
    sets = S.draw_grad_params(c["M"], 16)
    thetas = np.array([np.concatenate([[d["a_mean"], d["sigma"]], base_s * d["sqrt_lambda_scale"]]) for d in sets])
    F = _t(S.make_rhs(unit, c["p"]))
    gb = lib.SGGradBatch.from_inputs(unit, c["p"], 16)
    gb.autotune()
    Q, G = gb.value_and_grad(thetas, F, _tight(lib))
    Q, G = Q.cpu().numpy(), G.cpu().numpy()
    gb.close()
    assert Q.shape == (16,) and G.shape == (16, c["M"] + 2)
    with ThreadPoolExecutor(8) as ex:
        refs = list(ex.map(lambda th: _oracle_grad(unit, th, c["p"]), thetas))
    for i, (q_ref, g_ref) in enumerate(refs):
        assert Q[i] == pytest.approx(q_ref, rel=1e-10), i
        assert np.abs(G[i] - g_ref).max() <= 1e-6 * np.abs(g_ref).max(), i
    h = lib.SGProblem.from_inputs(unit, c["p"])
    Q1, G1 = lib.sg_qoi_value_and_grad_batch(h, thetas[:3], F, _tight(lib))
    assert np.allclose(Q1.cpu().numpy(), Q[:3], rtol=1e-12, atol=0)
    assert np.allclose(G1.cpu().numpy(), G[:3], rtol=1e-10, atol=1e-12 * np.abs(G).max())


def test_theta_entry_points_reject_bad_parameters(lib):
    unit = S.make_unit_problem(8, 2, 0.5)
    h = lib.SGProblem.from_inputs(unit, 2)
    for bad in ([0.0, 0.2, 1.0, 1.0], [-1.0, 0.2, 1.0, 1.0], [1.0, 0.0, 1.0, 1.0], [1.0, 0.2, np.nan, 1.0]):
        with pytest.raises(lib.SGError) as e:
            lib.sg_kl_set_theta(h, bad)
        assert e.value.status == 1
    with pytest.raises(ValueError):
        lib.sg_kl_set_theta(h, [1.0, 0.2, 1.0])
