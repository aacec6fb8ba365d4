"""Exact per-mode direct solve of the KKT system, and per-mode views of S-hat.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every spatial block of K (Eq 5) is a polynomial in the 5-point Laplacian A of Eq 2, and
the orthonormal DST-I (scipy.fft.dstn, type 1, norm 'ortho') diagonalises A: the sampled
sine mode sin(k pi x / Lx) sin(l pi y / Ly) is an eigenvector with eigenvalue
lambda_kl = 4/dx^2 sin^2(k pi / 2 nx) + 4/dy^2 sin^2(l pi / 2 ny). So K splits into N
independent 3Nt x 3Nt banded systems, one per mode. Solving them is a textbook special
case that pins the final answer of the whole solver; it is not a step of the method.

The same change of basis turns S-hat into the Nt x Nt tridiagonal T(mu)/h per mode,
with mu = 1 + dt/sqrt(omega) + dt nu lambda_kl (the diagonal of Jhat under the sign
reading of ``schwarz``), which is how the oracle reaches grids too large for its
physical-space sparse coarse solve.
"""

from __future__ import annotations

import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla

from .problem import HeatKKT


def mode_eigenvalues(p: HeatKKT) -> np.ndarray:
    """lambda_kl of A on the [My][Mx] grid of modes (l along y, k along x)."""
    k = np.arange(1, p.nx)
    l = np.arange(1, p.ny)
    lx = 4.0 / p.dx**2 * np.sin(k * np.pi / (2 * p.nx)) ** 2
    ly = 4.0 / p.dy**2 * np.sin(l * np.pi / (2 * p.ny)) ** 2
    return ly[:, None] + lx[None, :]


def dst2(block: np.ndarray, p: HeatKKT) -> np.ndarray:
    """Orthonormal 2D DST-I of every time slice of a [Nt][My][Mx] block (involutory)."""
    X = np.asarray(block, dtype=np.float64).reshape(-1, p.My, p.Mx)
    return sfft.dstn(X, type=1, axes=(1, 2), norm="ortho")


def kkt_exact_mode_solve(p: HeatKKT, lam: float, fu: np.ndarray, fz: np.ndarray, fw: np.ndarray):
    """The exact solution's time series (u, z, w) on one sine mode with eigenvalue lam, given the
    right-hand side's time series of that mode (each [Nt]).

    With mu0 = 1 + dt nu lam the unknowns u_n, z_n, w_n obey
      h u_n + mu0 w_n - w_{n+1}        = fu_n
      omega h z_n - dt w_n             = fz_n
      mu0 u_n - u_{n-1} - dt z_n       = fw_n
    z is eliminated, and (u_1, w_1, u_2, w_2, ...) is solved as a banded system.
    """
    Nt = p.Nt
    c = p.dt * p.dt / (p.omega * p.h)
    nunk = 2 * Nt
    mu0 = 1.0 + p.dt * p.nu * lam
    ab = np.zeros((7, nunk))                      # band storage, 3 sub- and 3 super-diagonals
    rhs = np.empty(nunk)

    def put(row, col, val):
        ab[3 + row - col, col] = val

    for n in range(Nt):
        iu, iw = 2 * n, 2 * n + 1
        put(iu, iu, p.h)
        put(iu, iw, mu0)
        if n + 1 < Nt:
            put(iu, iw + 2, -1.0)
        rhs[iu] = fu[n]
        put(iw, iu, mu0)
        if n > 0:
            put(iw, iu - 2, -1.0)
        put(iw, iw, -c)
        rhs[iw] = fw[n] + p.dt * fz[n] / (p.omega * p.h)
    sol = sla.solve_banded((3, 3), ab, rhs)
    U = sol[0::2]
    W = sol[1::2]
    Z = (fz + p.dt * W) / (p.omega * p.h)
    return U, Z, W


def kkt_exact_solve(p: HeatKKT, f: np.ndarray) -> np.ndarray:
    """x = K^{-1} f by per-mode banded solves (kkt_exact_mode_solve on every sine mode)."""
    V, Nt = p.V, p.Nt
    fu = dst2(f[:V], p).reshape(Nt, -1)
    fz = dst2(f[V : 2 * V], p).reshape(Nt, -1)
    fw = dst2(f[2 * V :], p).reshape(Nt, -1)
    lam = mode_eigenvalues(p).ravel()
    U = np.empty((Nt, lam.size))
    Z = np.empty((Nt, lam.size))
    W = np.empty((Nt, lam.size))
    for q, lq in enumerate(lam):
        U[:, q], Z[:, q], W[:, q] = kkt_exact_mode_solve(p, lq, fu[:, q], fz[:, q], fw[:, q])
    u = dst2(U, p).ravel()
    z = dst2(Z, p).ravel()
    w = dst2(W, p).ravel()
    return np.concatenate([u, z, w])


def jhat_mode_diagonal(p: HeatKKT, jhat_sign: int = -1) -> np.ndarray:
    """mu_kl: the eigenvalue of Jhat's diagonal block on each sine mode ([My][Mx])."""
    return 1.0 - jhat_sign * p.dt / np.sqrt(p.omega) + p.dt * p.nu * mode_eigenvalues(p)
