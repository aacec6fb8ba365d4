"""Right-preconditioned flexible GMRES (Section 4: "right preconditioned GMRES").

TEST INFRASTRUCTURE ONLY (see the package docstring).

Saad's FGMRES(m): Arnoldi with modified Gram-Schmidt on the vectors K z_j, z_j = P^{-1} v_j,
the least-squares problem reduced by Givens rotations, x = x_0 + Z y at the end of each
cycle. The stopping test is the relative residual ||f - K x||_2 / ||f||_2 <= tol on the
unscaled Euclidean norm over all three blocks (the paper states "relative residual" only).
With a fixed linear preconditioner FGMRES produces the same iterates as right-preconditioned
GMRES.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class KrylovResult:
    x: np.ndarray
    iterations: int
    converged: bool
    rel_residual: float
    history: list = field(default_factory=list)   # relative residual estimate per iteration


def fgmres(matvec, precond, f, x0=None, *, tol=1e-8, restart=30, maxit=420, fixed_iterations=None,
           row_scale=None):
    """Solve K x = f. ``matvec(x)`` = K x, ``precond(r)`` = P^{-1} r.

    ``fixed_iterations``: stop after exactly this many Arnoldi steps (a single cycle), whatever
    the residual; used to compare iterates of two implementations after the same k.
    ``row_scale`` (a positive vector d): minimise and test ||d * (f - K x)|| / ||d * f|| instead
    of the Euclidean residual, i.e. run FGMRES on (d K) x = d f with the preconditioner applied
    to the unscaled residual, P^{-1}(r / d).
    """
    f = np.asarray(f, dtype=np.float64)
    if row_scale is not None:
        wts = np.asarray(row_scale, dtype=np.float64)
        inner_mv, inner_pc = matvec, precond
        matvec = lambda v: wts * inner_mv(v)        # noqa: E731
        precond = lambda q: inner_pc(q / wts)       # noqa: E731
        f = wts * f
    n = f.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    fnorm = np.linalg.norm(f)
    if fnorm == 0.0:
        return KrylovResult(np.zeros(n), 0, True, 0.0, [])
    history = []
    its = 0
    r = f - matvec(x)
    beta = np.linalg.norm(r)
    if fixed_iterations is None and beta / fnorm <= tol:
        return KrylovResult(x, 0, True, beta / fnorm, [])
    m = restart if fixed_iterations is None else fixed_iterations
    while True:
        V = np.zeros((m + 1, n))
        Zs = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_used = 0
        for j in range(m):
            Zs[j] = precond(V[j])
            w = matvec(Zs[j])
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                           # apply earlier rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / d
            sn[j] = H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_used = j + 1
            history.append(abs(g[j + 1]) / fnorm)
            if fixed_iterations is None and (abs(g[j + 1]) / fnorm <= tol or its >= maxit):
                break
            if H[j, j] == 0.0:
                break
        y = np.linalg.solve(np.triu(H[:j_used, :j_used]), g[:j_used])
        x = x + Zs[:j_used].T @ y
        r = f - matvec(x)
        beta = np.linalg.norm(r)
        rel = beta / fnorm
        if fixed_iterations is not None:
            return KrylovResult(x, its, rel <= tol, rel, history)
        if rel <= tol:
            return KrylovResult(x, its, True, rel, history)
        if its >= maxit:
            return KrylovResult(x, its, False, rel, history)
