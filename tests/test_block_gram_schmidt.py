"""The Gram-Schmidt orders of the GPU's FGMRES against the oracle's modified Gram-Schmidt, on the
CPU.

The GPU takes the dots of a block of b basis vectors (b = 2 by default, 4 or 8 as options) on one
w and subtracts the block in one pass. Since the vectors of a block are orthonormal to working
accuracy, that equals MGS up to rounding. This test writes that ordering out in numpy (a model of
the kernel's arithmetic order, not the kernel) and checks that the residual history and the
iterate equal those of the oracle's MGS FGMRES on the paper's operator and preconditioner.
"""

import numpy as np
import pytest

import workloads
from oracle import krylov, problem, schwarz
from oracle.problem import HeatKKT


def block_fgmres_history(matvec, precond, f, k, b, wts):
    """k steps of FGMRES from x = 0 with block-b Gram-Schmidt, on (wts K) x = wts f."""
    mv = lambda v: wts * matvec(v)          # noqa: E731
    pc = lambda q: precond(q / wts)         # noqa: E731
    f = wts * f
    n = f.size
    fnorm = np.linalg.norm(f)
    V = np.zeros((k + 1, n))
    Z = np.zeros((k, n))
    H = np.zeros((k + 1, k))
    V[0] = f / fnorm
    hist = []
    for j in range(k):
        Z[j] = pc(V[j])
        w = mv(Z[j])
        for s in range(0, j + 1, b):                 # one pass per block: dots on the same w
            blk = range(s, min(s + b, j + 1))
            d = [np.dot(V[i], w) for i in blk]
            for i, di in zip(blk, d):
                H[i, j] = di
                w = w - di * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = w / H[j + 1, j]
        g = np.zeros(j + 2)
        g[0] = fnorm
        y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], g, rcond=None)
        hist.append(np.linalg.norm(g - H[:j + 2, :j + 1] @ y) / fnorm)
    return np.array(hist), Z[:k].T @ y


@pytest.mark.parametrize("b", [2, 4, 8])
def test_block_gram_schmidt_equals_mgs_on_the_kkt_system(b):
    w = workloads.CFG_SMALL
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    f = problem.assemble_rhs(p, workloads.make_target(w), None)
    K = problem.assemble_K(p)
    d = problem.l2_residual_weights(p)
    pre = schwarz.schur_preconditioner(p, w.n_sub)
    apply_pre = lambda r: schwarz.block_preconditioner_apply(p, pre, r)   # noqa: E731
    k = 12
    ref = krylov.fgmres(lambda v: K @ v, apply_pre, f, fixed_iterations=k, row_scale=d)
    hist, x = block_fgmres_history(lambda v: K @ v, apply_pre, f, k, b, d)
    np.testing.assert_allclose(hist, ref.history, rtol=1e-9, atol=1e-15)
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) < 1e-9
