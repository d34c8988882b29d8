"""Shared helpers of the GPU tests: seeded problems, the oracle-side
operators, and the tolerance bounds. Imported only by ``-m gpu`` tests."""
import numpy as np
import scipy.sparse as sp

import sg_inputs as S
from oracle import chaos, sg_operator as so

# Rounding-error bounds of a gather sum of m terms in precision u: |err| <= m u sum|terms|.
# The SG product sums at most 9 nonzeros x (1 + 2M) couplings per entry; with M <= 10
# that is m <= 189, so 2e-5 (FP32) and 5e-14 (FP64) relative to the absolute-value
# product bound hold with margin.
TOL32 = 2e-5
TOL64 = 5e-14


def problem(ne, M, p, sigma=0.3, corr=0.5, a_mean=1.0, scale=None):
    prob = S.make_problem(ne, M, sigma, corr, a_mean=a_mean, sqrt_lambda_scale=scale)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    return prob, A, G, off


def abs_bound(A, G, U):
    """Elementwise sum of |terms| of sum_k A_k U G_k^T."""
    return so.sg_apply([abs(a) for a in A], [abs(g) for g in G], np.abs(U))


def random_csr(n, seed, max_row=14, empty_every=7):
    """Seeded random sorted CSR pattern with ragged rows (some empty, some longer
    than the 9-point stencil)."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for r in range(n):
        if empty_every and r % empty_every == 3:
            continue
        k = int(rng.integers(1, max_row + 1))
        c = np.unique(rng.integers(0, n, size=k))
        rows.extend([r] * len(c))
        cols.extend(c.tolist())
    m = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    m.sort_indices()
    return m.indptr.astype(np.int32), m.indices.astype(np.int32)


def oracle_rel_residual(A, G, F, U, threads=16, block=8192):
    """``||F - sum_k A_k U G_k^T|| / ||F||`` in FP64 by the oracle, one block of
    spatial rows per task (row ``r`` of the product needs only row ``r`` of
    each ``A_k``), the blocks on a thread pool (scipy's sparse products
    release the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor
    n = F.shape[0]
    starts = list(range(0, n, block))

    def part(s):
        rows = np.arange(s, min(s + block, n))
        R = F[rows] - so.sg_apply_rows(A, G, U, rows)
        return float(np.sum(R * R))

    with ThreadPoolExecutor(threads) as ex:
        ss = sum(ex.map(part, starts))
    return float(np.sqrt(ss) / np.linalg.norm(F))


def sample_rows(n, count=48, seed=0):
    """Sorted spatial rows for element checks at full size: the first and last
    rows, the rows next to them and a seeded spread over the rest."""
    rng = np.random.default_rng(seed)
    fixed = [0, 1, n // 2, n - 2, n - 1]
    rest = rng.choice(n, size=max(count - len(fixed), 0), replace=False)
    return np.unique(np.concatenate([fixed, rest]).astype(np.int64))
