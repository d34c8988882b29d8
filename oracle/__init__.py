"""FP64 CPU oracle for the stochastic Galerkin solve with the hierarchical
Schur complement (HSC) preconditioner.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it. The product path (the CUDA
library and its Python binding) never imports, links or calls anything here,
and the oracle shares no code with it: it re-derives every table (multi-indices,
triple products, multigrid transfer operators) from the definitions.

Each function states the passage of the paper it follows:

* ``chaos``        -- total-degree chaos basis, triple products ``c_ijk``,
                      block counts (Sec. 2 eq. (gPC-u), (global-system);
                      Sec. 3 and its Lemma; Sec. 6 Table 5, Fig. 1).
* ``sg_operator``  -- the SG matrix-vector product (eq. (global-system),
                      (global-matrix-block) and the MAT-VEC remark), the
                      explicit global matrix, the direct solve.
* ``hsc``          -- Algorithm 1 (Sec. 4), the block inverse
                      (eq. (block-LU), (block-inverse)), the Schur complements
                      and the constants of eq. (AS-ineq) / Theorem 1.
* ``krylov``       -- flexible CG (Sec. 5, Sec. 6), the Lanczos condition
                      estimate (Sec. 6), the inner batched PCG on ``A_0``.
* ``gmg``          -- geometric multigrid V-cycle for the mean problem (the
                      paper leaves ``M_0`` open, Sec. 5; this is the reading
                      used for the inner solves).
* ``qoi``          -- ``Q = E[int u^2]`` and its adjoint gradient.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against a closed form, a brute-force computation, a worked number printed in
the paper or an identity of the mathematics, except where its docstring says
"parity unpinned".
"""
