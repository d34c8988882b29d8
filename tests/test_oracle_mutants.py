"""Planted mistakes in the oracle and in the seeded input generator that the
oracle and the CUDA path both consume: each case edits one line of one
function in memory (a dropped term, a wrong sign, a wrong index or operand
order, a loop run the wrong way), installs the edited function in place of the
original for the duration of the case, and runs the pins of that module
(the ``-m "not gpu"`` tests that tie it to closed forms, brute force, the
paper's printed numbers and identities of the mathematics). The case passes
only if one of those pins fails with an assertion, i.e. the pins are strong
enough to see that mistake. Nothing here touches the CUDA path. A mistake in
the input generator would reach both sides of a parity test alike, so its
pins (the KL pairs against a Nystrom discretisation, the stiffness matrices
against their integrals written out) are what keep the workload the paper's.

The edit is textual on the function's own source, so every case states the
exact fragment it replaces; a fragment that no longer occurs (the oracle was
rewritten) fails the case instead of passing it silently.
"""
from __future__ import annotations

import inspect
import textwrap
from dataclasses import dataclass
from typing import Callable, Sequence

import pytest

import sg_inputs
from oracle import chaos, gmg, hsc, krylov, qoi, sg_operator

import test_inputs as ti
import test_oracle_chaos as tc
import test_oracle_gmg as tg
import test_oracle_hsc as th
import test_oracle_krylov as tk
import test_oracle_operator as to
import test_oracle_qoi as tq


# The pins of each oracle module, cheapest first (each is a complete test of
# the module's own pin file, called with one of its parameter sets).
CHAOS_PINS: Sequence[Callable[[], None]] = (
    lambda: tc.test_xi_is_first_order_chaos_polynomial(),
    lambda: tc.test_multi_index_table_is_graded_complete_and_ordered(3, 3),
    lambda: tc.test_g_symmetric_and_lemma_diagonal_block(4, 4),
    lambda: tc.test_block_count_closed_forms(4, 3),
    lambda: tc.test_triple_products_match_brute_force_quadrature(chaos.LEGENDRE, 2, 3),
    lambda: tc.test_triple_products_match_brute_force_quadrature(chaos.HERMITE, 2, 3),
    lambda: tc.test_hermite_triple_products_against_quadrature(),
    lambda: tc.test_gpc_matrices_reduce_to_the_linear_expansion(2, 3),
    lambda: tc.test_gpc_triple_products_match_brute_force_quadrature(2, 2, 4),
    lambda: tc.test_block_counts_reproduce_table5_and_fig1(),
)
OPERATOR_PINS = (
    lambda: to.test_sg_apply_matches_block_matrix_of_the_paper(4, 2, 3),
    lambda: to.test_level_blocks_sum_to_operator_without_diagonal(),
    lambda: to.test_row_sampled_products_match_the_explicit_global_matrix(),
    lambda: to.test_direct_solve_residual_and_linearity(),
    lambda: to.test_global_matrix_symmetric_positive_definite_cfg1_small(),
    lambda: to.test_kl_matrices_hold_each_term_column(),
)
HSC_PINS = (
    lambda: th.test_block_inverse_with_true_schur_is_exact_inverse(),
    lambda: th.test_mean_preconditioner_is_blockwise_A0_inverse(),
    lambda: th.test_algorithm1_equals_recursive_block_inverse(4, 2, 3),
    lambda: th.test_algorithm1_gpc_equals_recursive_block_inverse(2, 2),
    lambda: th.test_hsc_symmetric_positive_definite(),
    lambda: th.test_general_prec_variants_match_the_paper_formula(),
    lambda: th.test_general_prec_factors_sit_where_the_paper_puts_them(),
    lambda: th.test_bgs_matches_block_triangular_solves(2, 2),
    lambda: th.test_theorem1_spectrum(4, 2, 3, 0.4),
    lambda: th.test_schur_reduced_solve_recovers_the_full_solution(2, 2),
    lambda: th.test_schur_reduced_iteration_is_preconditioned_by_algorithm1(2, 2),
    lambda: th.test_schur_constants_are_the_spectrum_of_one_level(2),
)
KRYLOV_PINS = (
    lambda: tk.test_cg_on_known_spectrum_and_lanczos_estimate(),
    lambda: tk.test_exact_preconditioner_converges_in_one_step(),
    lambda: tk.test_pcg_columns_conventions(),
    lambda: tk.test_flexible_cg_keeps_consecutive_directions_conjugate(),
    lambda: tk.test_pcg_iterates_minimise_the_energy_error_over_the_krylov_space(),
    lambda: tk.test_fcg_initial_guess_zero_right_hand_side_and_breakdown(),
    lambda: tk.test_fcg_sg_solution_matches_direct_solve(),
)
GMG_PINS = (
    lambda: tg.test_prolongation_is_bilinear_interpolation(8),
    lambda: tg.test_galerkin_coarse_operator_is_coarse_q1_matrix(8),
    lambda: tg.test_vcycle_symmetric_positive_definite(),
    lambda: tg.test_vcycle_columns_independent(),
    lambda: tg.test_vcycle_contraction_h_independent(16),
    lambda: tg.test_vcycle_equals_error_propagation_recursion(8, 2, 0.8, "kl"),
    lambda: tg.test_vcycle_equals_error_propagation_recursion(8, 2, 0.8, "lognormal"),
)
QOI_PINS = (
    lambda: tq.test_adjoint_gradient_matches_central_differences(),
)
INPUT_PINS = (
    lambda: ti.test_kl_2d_products_sorted(),
    lambda: ti.test_q1_mean_matrix_is_textbook_stencil(),
    lambda: ti.test_kl_stiffness_is_weighted_laplacian(),
    lambda: tq.test_mass_matrix_integrates_constants(),
    lambda: ti.test_kl_1d_closed_form_matches_nystrom(0.5),
    lambda: ti.test_kl_stiffness_matrices_match_direct_integration(),
    lambda: ti.test_lognormal_matrices_expand_the_stiffness_of_exp_g(),
)


@dataclass(frozen=True)
class Mutant:
    id: str
    module: object
    func: str
    old: str
    new: str
    pins: Sequence[Callable[[], None]]
    what: str


MUTANTS = [
    # --- chaos basis and triple products (Sec. 2 eq. (gPC-u), Sec. 3, Table 5)
    Mutant("chaos-order-ascending", chaos, "_compositions_desc", "range(d, -1, -1)", "range(0, d + 1)",
           CHAOS_PINS, "multi-indices of one degree in ascending instead of descending order"),
    Mutant("chaos-top-degree-dropped", chaos, "multi_indices", "for d in range(p + 1):", "for d in range(p):",
           CHAOS_PINS, "the degree-p block left out of the basis"),
    Mutant("legendre-triple-denominator", chaos, "xi_triple_1d", "(2 * m + 3)", "(2 * m + 1)",
           CHAOS_PINS, "wrong normalisation of the Legendre triple product"),
    Mutant("hermite-triple-index", chaos, "xi_triple_1d", "math.sqrt(m + 1.0)", "math.sqrt(m + 2.0)",
           CHAOS_PINS, "Hermite E[xi psi_m psi_m+1] at the wrong degree"),
    Mutant("g-min-to-max", chaos, "g_matrices", "min(a[k], b[k])", "max(a[k], b[k])",
           CHAOS_PINS, "triple product evaluated at the larger of the two degrees"),
    Mutant("g-one-sided", chaos, "g_matrices", "for step in (+1, -1):", "for step in (+1,):",
           CHAOS_PINS, "only the upper neighbour coupled (G_k not symmetric)"),
    Mutant("g-wrong-coordinate", chaos, "g_matrices", "b[k] += step", "b[(k + 1) % M] += step",
           CHAOS_PINS, "G_k built from the neighbour in the next coordinate"),
    Mutant("table5-diagonal-dropped", chaos, "block_counts", "sum(abs(G) for G in Gs)",
           "sum(abs(G) for G in Gs[1:])", CHAOS_PINS, "n_b counted without the diagonal blocks of G_0"),
    Mutant("table5-solves", chaos, "block_counts", "n_ds=2 * (n_db - 1) + 1", "n_ds=2 * n_db + 1",
           CHAOS_PINS, "one block solve too many per level"),
    Mutant("hermite-product-formula", chaos, "hermite_triple_1d", "math.factorial(s2 - c))",
           "math.factorial(s2 - b))", CHAOS_PINS, "wrong factorial in the Hermite product formula"),
    Mutant("gpc-coefficient-truncated", chaos, "gpc_g_matrices", "gamma, _ = multi_indices(M, q)",
           "gamma, _ = multi_indices(M, min(q, p))", CHAOS_PINS,
           "coefficient expanded to degree p instead of q = 2p"),
    Mutant("chaos-count", chaos, "chaos_count", "math.comb(M + p, M)", "math.comb(M + p, M - 1)", CHAOS_PINS,
           "(M+p)!/((M-1)!(p+1)!) polynomials"),
    Mutant("gpc-wrong-index", chaos, "gpc_g_matrices", "int(alpha[l][k])", "int(alpha[j][k])",
           CHAOS_PINS, "second polynomial index read as the first"),
    # --- SG operator (eq. (global-system), (global-matrix), (global-matrix-hierarchy))
    Mutant("kl-matrix-term-column", sg_operator, "kl_matrices", "vals[:, k]", "vals[:, min(k, 1)]", OPERATOR_PINS,
           "every A_k with k >= 1 read from the first KL term's values"),
    Mutant("apply-last-term-dropped", sg_operator, "sg_apply", "zip(A, G)", "zip(A[:-1], G[:-1])",
           OPERATOR_PINS, "the k = M term of sum_k A_k U G_k^T left out"),
    Mutant("apply-rows-last-term-dropped", sg_operator, "sg_apply_rows", "zip(A, G)", "zip(A[:-1], G[:-1])",
           OPERATOR_PINS, "the k = M term left out of the row-sampled product"),
    Mutant("apply-rows-shifted", sg_operator, "sg_apply_rows", "Ak[rows]", "Ak[(rows + 1) % Ak.shape[0]]",
           OPERATOR_PINS, "the row sample read one row off"),
    Mutant("block-coefficient-dropped", sg_operator, "global_matrix_chaos_major",
           "blk = c * Ak if blk is None else blk + c * Ak", "blk = Ak if blk is None else blk + Ak",
           OPERATOR_PINS, "K^(j,l) = sum_i K_i without the coefficients c_ijl"),
    Mutant("layout-permutation", sg_operator, "chaos_major_to_space_major", "(l * n + r)", "(r * P + l)",
           OPERATOR_PINS, "the chaos-major / space-major permutation inverted"),
    Mutant("kron-operands-swapped", sg_operator, "global_matrix_space_major", "sp.kron(Ak, Gk",
           "sp.kron(Gk, Ak", OPERATOR_PINS, "G_k (x) A_k instead of A_k (x) G_k for the space-major layout"),
    Mutant("direct-solve-layout", sg_operator, "direct_solve", "F.ravel()", "F.T.ravel()",
           OPERATOR_PINS, "right-hand side flattened chaos-major into a space-major solve"),
    Mutant("level-last-term-dropped", sg_operator, "level_apply", "zip(A, G)", "zip(A[:-1], G[:-1])",
           OPERATOR_PINS, "the k = M term left out of B_l / C_l"),
    # --- Algorithm 1 and the comparators (Sec. 4, 5, 6)
    Mutant("offdiag-sign", hsc, "_offdiag_apply", "Y += ", "Y -= ", HSC_PINS,
           "B_l / C_l applied with the wrong sign"),
    Mutant("pre-correction-unsolved", hsc, "hsc_apply",
           "r[:, :lo] -= _offdiag_apply(A, G, slice(0, lo), slice(lo, hi), y)",
           "r[:, :lo] -= _offdiag_apply(A, G, slice(0, lo), slice(lo, hi), r[:, lo:hi])", HSC_PINS,
           "pre-correction with B_l r_l instead of B_l D_l^-1 r_l"),
    Mutant("post-correction-sign", hsc, "hsc_apply", "t = r[:, lo:hi] - _offdiag_apply",
           "t = r[:, lo:hi] + _offdiag_apply", HSC_PINS, "post-correction r_l + C_l u instead of r_l - C_l u"),
    Mutant("pre-loop-direction", hsc, "hsc_apply", "for l in range(p, 0, -1):", "for l in range(1, p + 1):",
           HSC_PINS, "pre-correction swept from the lowest degree up"),
    Mutant("mean-solve-input", hsc, "hsc_apply", "dsolve(0, r[:, 0:off[1]])", "dsolve(0, R[:, 0:off[1]])",
           HSC_PINS, "mean problem solved with r_0 instead of g_0"),
    Mutant("pre-correction-adjacent-level", hsc, "hsc_apply",
           "r[:, :lo] -= _offdiag_apply(A, G, slice(0, lo), slice(lo, hi), y)",
           "r[:, off[l - 1]:lo] -= _offdiag_apply(A, G, slice(off[l - 1], lo), slice(lo, hi), y)", HSC_PINS,
           "B_l taken as coupling degree l with degree l - 1 only (true for the linear expansion alone)"),
    Mutant("post-correction-adjacent-level", hsc, "hsc_apply",
           "_offdiag_apply(A, G, slice(lo, hi), slice(0, lo), u[:, :lo])",
           "_offdiag_apply(A, G, slice(lo, hi), slice(off[l - 1], lo), u[:, off[l - 1]:lo])", HSC_PINS,
           "C_l taken as coupling degree l with degree l - 1 only"),
    Mutant("general-D-mean-term-only", hsc, "_diag_block_solver", "for Ak, Gk in zip(A, G):",
           "for Ak, Gk in zip(A[:1], G[:1]):", HSC_PINS,
           "assembled D_l from the mean term alone (the Lemma of Sec. 3, which needs the linear expansion)"),
    Mutant("general-D-layout", hsc, "_diag_block_solver", "sp.kron(Ak, sub", "sp.kron(sub, Ak", HSC_PINS,
           "assembled D_l in the wrong Kronecker order"),
    Mutant("block-inverse-transposed", hsc, "block_inverse", "np.linalg.inv(A - B @ Dinv @ C)",
           "np.linalg.inv(A - C.T @ Dinv @ B.T)", HSC_PINS, "Schur complement with transposed couplings"),
    Mutant("block-inverse-pre-sign", hsc, "block_inverse", "[np.eye(na), -B @ Dinv]", "[np.eye(na), B @ Dinv]",
           HSC_PINS, "pre-correction factor with the wrong sign"),
    Mutant("general-prec-factor", hsc, "general_prec", "[-MD3 @ C, np.eye(nd)]", "[-MD1 @ C, np.eye(nd)]",
           HSC_PINS, "M_D^1 used in the post-correction factor of eq. (general-prec)"),
    Mutant("general-prec-middle", hsc, "general_prec", "[np.zeros((nd, na)), MD2]", "[np.zeros((nd, na)), MD3]",
           HSC_PINS, "M_D^3 in the middle factor of eq. (general-prec)"),
    Mutant("recursion-exact-schur", hsc, "hsc_dense_recursive", "S_inv=M(l - 1)", "S_inv=None", HSC_PINS,
           "dense recursion with the exact Schur complement instead of M_l-1"),
    Mutant("schur-constants-no-pencil", hsc, "schur_constants",
           "sla.eigh(0.5 * (S + S.T), 0.5 * (A_l + A_l.T), eigvals_only=True)",
           "sla.eigh(0.5 * (S + S.T), eigvals_only=True)", HSC_PINS,
           "eigenvalues of S_l alone instead of the pencil (S_l, A_l)"),
    Mutant("schur-rhs-sign", hsc, "schur_reduced_solve", "g = F[:, :lo] - _offdiag_apply",
           "g = F[:, :lo] + _offdiag_apply", HSC_PINS, "g_p-1 = f + B D^-1 f^p"),
    Mutant("schur-recovery", hsc, "schur_reduced_solve",
           "dsolve(F[:, lo:] - _offdiag_apply(A, G, slice(lo, off[p + 1]), slice(0, lo), u_r))",
           "dsolve(F[:, lo:])", HSC_PINS, "u^p recovered without the C_p u_p-1 correction"),
    Mutant("schur-preconditioner-mean", hsc, "schur_reduced_solve", "hsc_apply(A, sub_G, off_r, R, a0solve=a0)",
           "mean_apply(A, R, a0)", HSC_PINS, "reduced system preconditioned with the mean-based M_m"),
    Mutant("schur-constant-upper", hsc, "schur_constants", "out.append((float(mu[0]), float(mu[-1])))",
           "out.append((float(mu[0]), float(mu[-2])))", HSC_PINS, "c_l,2 read one eigenvalue below the largest"),
    Mutant("bgs-backward-stale", hsc, "bgs_apply", "(fwd[:, l] if l < j else u[:, l])", "fwd[:, l]",
           HSC_PINS, "backward sweep reads the forward values for l > j"),
    Mutant("bgs-forward-upper", hsc, "bgs_apply", "            if l < j:\n", "            if l > j:\n",
           HSC_PINS, "forward sweep subtracts the upper instead of the lower blocks"),
    Mutant("bgs-dense-order", hsc, "bgs_dense", "np.linalg.solve(D + Up, D @ np.linalg.inv(D + Lo))",
           "np.linalg.solve(D + Lo, D @ np.linalg.inv(D + Up))", HSC_PINS,
           "dense M_bGS with the sweeps in the opposite order"),
    Mutant("mean-wrong-matrix", hsc, "mean_apply", "A0Solver(A[0])", "A0Solver(A[1])", HSC_PINS,
           "mean-based preconditioner with A_1 instead of A_0"),
    # --- flexible CG, Lanczos estimate, inner PCG (Sec. 5, 6)
    Mutant("fcg-initial-residual-sign", krylov, "fcg", "r = f - apply_A(x) if x0 is not None",
           "r = f + apply_A(x) if x0 is not None", KRYLOV_PINS, "initial residual f + A x0"),
    Mutant("fcg-no-breakdown-check", krylov, "fcg", "if not pq > 0:", "if pq < -1e300:", KRYLOV_PINS,
           "p^T A p <= 0 not detected"),
    Mutant("fcg-zero-rhs", krylov, "fcg", "converged=res[0] <= tol", "converged=False", KRYLOV_PINS,
           "a zero right-hand side iterated instead of solved at entry"),
    Mutant("lanczos-no-steps", krylov, "lanczos_kappa", "if m == 0:\n        return 1.0", "if m == 0:\n        return 0.0",
           KRYLOV_PINS, "condition estimate 0 without a CG step"),
    Mutant("fcg-direction", krylov, "fcg", "p = z + beta * p", "p = z + beta * z", KRYLOV_PINS,
           "search direction not conjugated (steepest descent)"),
    Mutant("fcg-beta-denominator", krylov, "fcg", "if flexible else rho_new) / rho",
           "if flexible else rho_new) / pq", KRYLOV_PINS, "beta divided by p^T q instead of rho"),
    Mutant("fcg-standard-beta", krylov, "fcg", "np.vdot(z, r - r_old)", "np.vdot(z, r)", KRYLOV_PINS,
           "flexible beta replaced by the standard one (wrong for a changing preconditioner)"),
    Mutant("fcg-update-z", krylov, "fcg", "x += alpha * p", "x += alpha * z", KRYLOV_PINS,
           "iterate moved along z instead of p"),
    Mutant("lanczos-diagonal", krylov, "lanczos_kappa",
           "1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)", "1.0 / alphas[j]",
           KRYLOV_PINS, "Lanczos diagonal without the beta / alpha term"),
    Mutant("lanczos-offdiagonal", krylov, "lanczos_kappa", "np.sqrt(max(betas[j], 0.0)) / alphas[j]",
           "max(betas[j], 0.0) / alphas[j]", KRYLOV_PINS, "Lanczos off-diagonal without the square root"),
    Mutant("pcg-stop-test", krylov, "pcg_columns", "tol * tol * bb", "tol * bb", KRYLOV_PINS,
           "column stop test ||r||^2 <= tol ||b||^2"),
    Mutant("pcg-beta-inverted", krylov, "pcg_columns", "beta = rho_new / rho", "beta = rho / rho_new",
           KRYLOV_PINS, "inner beta inverted"),
    Mutant("pcg-preconditioner-once", krylov, "pcg_columns", "            z = apply_M0(r)\n",
           "            z = r.copy()\n", KRYLOV_PINS, "inner M_0 applied at the first step only"),
    Mutant("pcg-rho-unpreconditioned", krylov, "pcg_columns", "rho_new = float(r @ z)", "rho_new = float(r @ r)",
           KRYLOV_PINS, "inner rho = r^T r instead of r^T z"),
    Mutant("fcg-preconditioner-once", krylov, "fcg", "        z = M(r)\n        rho_new",
           "        z = r.copy()\n        rho_new", KRYLOV_PINS, "outer preconditioner applied at the first step only"),
    Mutant("pcg-count-off-by-one", krylov, "pcg_columns", "iters[s] = it", "iters[s] = it - 1", KRYLOV_PINS,
           "per-column iteration count one short"),
    # --- multigrid V-cycle for A_0 (the inner M_0)
    Mutant("w1d-weight", gmg, "_w1d", "0.5 if d == 1", "0.25 if d == 1", GMG_PINS,
           "full-weighting 1/4 where bilinear interpolation has 1/2"),
    Mutant("prolongation-xy-swapped", gmg, "prolongation", "rows.append((j - 1) * m + (i - 1))",
           "rows.append((i - 1) * m + (j - 1))", GMG_PINS, "fine nodes ordered y fastest"),
    Mutant("galerkin-scaled", gmg, "hierarchy", "(P.T @ fine.A @ P)", "(0.25 * P.T @ fine.A @ P)", GMG_PINS,
           "coarse operator with a scaled restriction"),
    Mutant("vcycle-no-post-smoothing", gmg, "vcycle",
           "x = x + L.P @ xc\n    for _ in range(nu):", "x = x + L.P @ xc\n    for _ in range(0):",
           GMG_PINS, "post-smoothing left out (non-symmetric cycle)"),
    Mutant("vcycle-coarse-sweeps", gmg, "vcycle", "xc = vcycle(levels, L.P.T @ r, nu, omega, g + 1)",
           "xc = vcycle(levels, L.P.T @ r, 1, omega, g + 1)", GMG_PINS, "one smoothing step on the coarser grids"),
    Mutant("jacobi-first-diagonal", gmg, "vcycle", "dinv = L.dinv if b.ndim == 1 else L.dinv[:, None]",
           "dinv = L.dinv if b.ndim == 1 else L.dinv[None, :1]", GMG_PINS,
           "Jacobi scaled by the first diagonal entry (right only for a constant diagonal)"),
    Mutant("vcycle-restrict-rhs", gmg, "vcycle", "L.P.T @ r", "L.P.T @ b", GMG_PINS,
           "restriction of b instead of the residual"),
    Mutant("jacobi-no-accumulate", gmg, "vcycle", "x = x + omega * dinv * (b - L.A @ x)",
           "x = omega * dinv * (b - L.A @ x)", GMG_PINS, "pre-smoothing step overwrites x"),
    # --- quantity of interest and its adjoint gradient
    Mutant("chain-sigma-sign", qoi, "chain_weights", "W[1, 1:] = -1.0 / sigma", "W[1, 1:] = 1.0 / sigma",
           QOI_PINS, "dQ/dsigma with the wrong sign"),
    Mutant("chain-s-index", qoi, "chain_weights", "W[2 + k, 1 + k]", "W[2 + k, k]", QOI_PINS,
           "dA_k/ds_k attached to A_k-1"),
    Mutant("qoi-mass-dropped", qoi, "qoi", "np.sum(U * (Mh @ U))", "np.sum(U * U)", QOI_PINS,
           "Q without the mass matrix"),
    Mutant("k-products-operand", qoi, "k_resolved_products", "sg_apply([Ak], [Gk], U)",
           "sg_apply([Ak], [Gk], Lam)", QOI_PINS, "h_k = <Lam, A_k Lam G_k^T>"),
    # --- seeded inputs: KL expansion (eq. (cov), (KL-expansion)), Q1 assembly, lognormal gPC coefficient
    Mutant("kl-eigenvalue", sg_inputs, "kl_1d", "out.append((2 * c / (w * w + c * c), w, 0, nrm))",
           "out.append((c / (w * w + c * c), w, 0, nrm))", INPUT_PINS, "even KL eigenvalues halved"),
    Mutant("kl-odd-normalisation", sg_inputs, "kl_1d", "a - math.sin(2 * w * a) / (2 * w)",
           "a + math.sin(2 * w * a) / (2 * w)", INPUT_PINS, "odd KL modes normalised with the even modes' norm"),
    Mutant("kl-2d-ascending", sg_inputs, "kl_2d", "-round(t[0], 14)", "round(t[0], 14)", INPUT_PINS,
           "2-D KL pairs kept from the smallest eigenvalue"),
    Mutant("q1-gradient", sg_inputs, "_shape", ", sa * (1 + sb * eta) / 4.0", ", sa * (1 + sb * eta) / 2.0",
           INPUT_PINS, "x derivative of the bilinear shape function twice too large"),
    Mutant("q1-mass-table", sg_inputs, "_element_tables", "Mm[g, p, q] = vals[p][0] * vals[q][0]",
           "Mm[g, p, q] = vals[p][0]", INPUT_PINS, "mass integrand N_p instead of N_p N_q"),
    Mutant("stencil-slot-xy", sg_inputs, "_assemble_stencils", "slot = (bq - bp + 1) * 3 + (aq - ap + 1)",
           "slot = (aq - ap + 1) * 3 + (bq - bp + 1)", INPUT_PINS, "stencil offsets with x and y exchanged"),
    Mutant("csr-column-xy", sg_inputs, "_interior_csr", "cols.append((cy - 1) * m + (cx - 1))",
           "cols.append((cx - 1) * m + (cy - 1))", INPUT_PINS, "column nodes numbered y fastest"),
    Mutant("load-scale", sg_inputs, "make_problem", "f0 = np.full(n, h * h)", "f0 = np.full(n, h)", INPUT_PINS,
           "load vector of f = 1 scaled by h instead of h^2"),
    Mutant("mass-scale", sg_inputs, "make_problem", "h * h / 4.0)", "h * h)", INPUT_PINS,
           "mass matrix without the reference-element Jacobian"),
    Mutant("gauss-point-location", sg_inputs, "make_problem", "gx = np.stack([(ex + (1 + xi) / 2) * h",
           "gx = np.stack([(ex + xi / 2) * h", INPUT_PINS, "KL functions evaluated at shifted x Gauss points"),
    Mutant("kl-mode-xy", sg_inputs, "make_problem", "fy[:, None, :] * fx[None, :, :]",
           "fx[:, None, :] * fy[None, :, :]", INPUT_PINS, "phi_k(x, y) = e_a(y) e_b(x)"),
    Mutant("kl-amplitude", sg_inputs, "make_problem", "kappa[k] = sigma * s[k - 1] *",
           "kappa[k] = sigma * s[k - 1] ** 2 *", INPUT_PINS, "KL term scaled by lambda_k instead of sqrt(lambda_k)"),
    Mutant("lognormal-mean", sg_inputs, "make_lognormal_problem", "sig_g, mu_g = math.sqrt(sig2), -0.5 * sig2",
           "sig_g, mu_g = math.sqrt(sig2), 0.0", INPUT_PINS, "Gaussian field without the -sigma_g^2/2 shift"),
]


def _mutated(m: Mutant):
    """The function ``m.func`` of ``m.module`` compiled from its own source with
    the first occurrence of ``m.old`` replaced by ``m.new``; its globals are a
    copy of the module's, so it sees the module's other functions as they are."""
    src = textwrap.dedent(inspect.getsource(getattr(m.module, m.func)))
    assert m.old in src, f"{m.id}: fragment not found in {m.module.__name__}.{m.func}"
    src = src.replace(m.old, m.new, 1)
    ns = dict(vars(m.module))
    exec(compile(src, f"<mutant {m.id}>", "exec"), ns)
    return ns[m.func]


def test_mutant_ids_unique():
    ids = [m.id for m in MUTANTS]
    assert len(ids) == len(set(ids))


@pytest.mark.parametrize("m", MUTANTS, ids=lambda m: m.id)
def test_planted_mistake_fails_a_pin(m, monkeypatch):
    monkeypatch.setattr(m.module, m.func, _mutated(m))
    for pin in m.pins:
        try:
            pin()
        except AssertionError:
            return                    # caught
    pytest.fail(f"no pin of {m.module.__name__} fails with the planted mistake: {m.what}")


@pytest.mark.parametrize("module,func", sorted({(m.module, m.func) for m in MUTANTS}, key=lambda t: (t[0].__name__, t[1])),
                         ids=lambda v: v if isinstance(v, str) else v.__name__.split(".")[-1])
def test_recompiled_unchanged_function_passes_every_pin(module, func, monkeypatch):
    """The harness itself changes nothing: the same function recompiled from
    its unedited source passes all pins of its module, so a caught mutant is
    caught because of its edit."""
    pins = next(m.pins for m in MUTANTS if m.module is module and m.func == func)
    same = Mutant("unchanged", module, func, "def ", "def ", pins, "")
    monkeypatch.setattr(module, func, _mutated(same))
    for pin in pins:
        pin()
