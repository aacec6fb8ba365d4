"""Block preconditioner and the two-level time-domain-decomposition Schur inverse.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Section 2 (Eq 7) and Section 3 (Eqs 9-15) step by step:

* S-hat = Jhat M_u^{-1} Jhat^T with Jhat the block lower-bidiagonal matrix whose diagonal
  block is Bhat and whose sub-diagonal block is -I (Eq 7).
* Time subdomains overlap in one time node, not in time steps (Section 3, the Nt = 9,
  N_D = 3 example); R_s restricts to a subdomain's nodes, D_s is a boolean partition of
  unity, Q_s = [W_s; R_s] adds the node one step earlier (Eq 10).
* RAS (Eq 9), RASQ (Eq 13), the Nicolaides coarse space Z (Eq 14), the coarse operator
  S_0 = R_0 S-hat R_0^T with R_0 = Z^T, and the two-level composition (Eq 15).

Readings taken where the paper is silent or garbled (each is a constructor option, the
default named first):

* Sign of Jhat. Eq 7 prints Jhat = J + omega^{-1/2} L, and Eq 3 gives L = -dt I, so the
  literal diagonal block is (1 - dt/sqrt(omega)) I + dt nu A, which is indefinite or
  near-singular for the paper's own omega range. The cited Pearson-Wathen construction pairs
  the state operator with the control term so that the cross term of Jhat M^{-1} Jhat^T is
  positive; with L = -dt I that is Jhat = J - omega^{-1/2} L, diagonal block
  Bhat = (1 + dt/sqrt(omega)) I + dt nu A. ``jhat_sign=-1`` (default) takes this reading,
  ``jhat_sign=+1`` the literal one.
* D_s (Section 3 cites a definition not printed in the paper). ``pou='left'``: a node shared by
  subdomains s and s+1 belongs to s, the subdomain whose last step ends on it, so subdomain s
  owns nodes b_{s-1}+1 .. b_s. ``pou='right'`` gives it to s+1.
* Nt not divisible by N_D (Section 4 mentions such sequences): balanced split, subdomain s
  covers the steps b_{s-1}+1 .. b_s with b_s = floor(s Nt / N_D).
* Z (Eq 14, printed with a garbled block layout): column block s is R_s^T D_s (Phi_s kron I_N),
  Phi_s the constant and the linear function -1 + 2k/m_s on the subdomain's nodes
  k = 0..m_s; D_s removes the rows of nodes the subdomain does not own.
* Two-level composition (Eq 15 prints a product of rank at most 2 N_D N): multiplicative,
  coarse first: x_0 = R_0^T S_0^{-1} R_0 r, y = x_0 + S_RASQ^{-1} (r - S-hat x_0).
  ``variant='additive'`` gives x_0 + S_RASQ^{-1} r and ``variant='one-level'`` the RASQ alone.
  ``variant='ras'`` is RAS of Eq 9 alone and ``variant='ras-multiplicative'`` the same
  coarse-first composition with Eq 9's local solves in place of RASQ (an ablation).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .problem import HeatKKT, laplacian, time_stepping_matrix


def congruence(J, m_scale: float) -> sp.csr_matrix:
    """J M^{-1} J^T for M = m_scale * I: the Schur-complement product of Section 2 and of the
    three-step Euler example of Section 3."""
    J = sp.csr_matrix(J)
    return (J @ J.T / m_scale).tocsr()


@dataclass(frozen=True)
class Subdomain:
    """One time subdomain; nodes are 1-based time nodes, ranges inclusive."""

    s: int          # 1-based subdomain index
    first: int      # first time node (p_s)
    last: int       # last time node (q_s)
    m: int          # number of time steps covered, m_s
    k0: int         # Phi_s row index of the first node (1 when node 0 is excluded)
    owned_first: int
    owned_last: int

    @property
    def nodes(self) -> np.ndarray:
        return np.arange(self.first, self.last + 1)

    @property
    def owned(self) -> np.ndarray:
        return np.arange(self.owned_first, self.owned_last + 1)

    @property
    def extended_first(self) -> int:
        """First node of Q_s: one node before the subdomain when that node exists (Eq 10)."""
        return self.first - 1 if self.first - 1 >= 1 else self.first


def split_points(Nt: int, n_sub: int) -> np.ndarray:
    """b_s = floor(s Nt / N_D), s = 0..N_D (balanced split of the Nt time steps)."""
    return np.array([(s * Nt) // n_sub for s in range(n_sub + 1)], dtype=np.int64)


def subdomains(Nt: int, n_sub: int, pou: str = "left") -> list[Subdomain]:
    """Time subdomains of Section 3: steps b_{s-1}+1..b_s, nodes b_{s-1}..b_s minus node 0."""
    if n_sub < 1 or Nt < n_sub:
        raise ValueError("need 1 <= n_sub <= Nt")
    b = split_points(Nt, n_sub)
    out = []
    for s in range(1, n_sub + 1):
        lo, hi = int(b[s - 1]), int(b[s])
        first = max(lo, 1)
        if pou == "left":
            of, ol = lo + 1, hi
        elif pou == "right":
            of = first
            ol = hi if s == n_sub else hi - 1
        else:
            raise ValueError(pou)
        out.append(Subdomain(s=s, first=first, last=hi, m=hi - lo, k0=first - lo,
                             owned_first=of, owned_last=ol))
    return out


def jhat_diagonal_block(p: HeatKKT, jhat_sign: int = -1) -> sp.csr_matrix:
    """Diagonal block Bhat of Jhat = J + jhat_sign * omega^{-1/2} L (Eq 7, sign reading above).

    J's diagonal block is I + dt nu A and L = -dt I (Eqs 2-4). With the default reading
    (jhat_sign=-1) the block is (1 + dt/sqrt(omega)) I + dt nu A; with the literal sign
    (jhat_sign=+1) it is (1 - dt/sqrt(omega)) I + dt nu A.
    """
    shift = -jhat_sign * p.dt / np.sqrt(p.omega)
    return ((1.0 + shift) * sp.identity(p.N) + p.dt * p.nu * laplacian(p)).tocsr()


class SchurPreconditioner:
    """S-hat and its approximate inverses for one diagonal block Bhat (N x N).

    For the physical problem Bhat is N x N sparse; for one spatial sine mode it is the 1 x 1
    matrix [mu]. Everything below is generic in N.
    """

    def __init__(self, Bhat, Nt: int, n_sub: int, h: float, *, pou: str = "left",
                 variant: str = "multiplicative", build_coarse: bool = True, mode_diagonal=None,
                 mode_transform=None):
        self.Bhat = sp.csr_matrix(Bhat, dtype=np.float64)
        self.N = self.Bhat.shape[0]
        self.Nt = Nt
        self.n_sub = n_sub
        self.h = float(h)
        self.pou = pou
        self.variant = variant
        self.subs = subdomains(Nt, n_sub, pou)
        self._lu = spla.splu(self.Bhat.tocsc())
        self._Jhat = None
        self._S = None
        self._Z = None
        self._S0_lu = None
        # Optional per-mode coarse solve (for grids where the sparse coarse LU does not fit):
        # mode_diagonal[q] is Bhat's eigenvalue on mode q and mode_transform(X) applies the
        # orthonormal, involutory transform that diagonalises Bhat to each row X[t] (length N).
        self.mode_diagonal = None if mode_diagonal is None else np.asarray(mode_diagonal, np.float64).ravel()
        self.mode_transform = mode_transform
        if build_coarse and variant not in ("one-level", "ras") and self.mode_diagonal is None:
            self._build_coarse()

    # ----- S-hat = Jhat M_u^{-1} Jhat^T (Eq 7) ---------------------------------------------
    @property
    def Jhat(self) -> sp.csr_matrix:
        if self._Jhat is None:
            self._Jhat = time_stepping_matrix(self.Bhat, -sp.identity(self.N), self.Nt)
        return self._Jhat

    @property
    def S_hat(self) -> sp.csr_matrix:
        """Jhat M_u^{-1} Jhat^T with M_u = h I."""
        if self._S is None:
            self._S = congruence(self.Jhat, self.h)
        return self._S

    def jhat_apply(self, x):
        """(Jhat x)_n = Bhat x_n - x_{n-1}, one time node at a time."""
        X = x.reshape(self.Nt, self.N)
        Y = (self.Bhat @ X.T).T
        Y[1:] -= X[:-1]
        return Y.ravel()

    def jhat_T_apply(self, x):
        """(Jhat^T x)_n = Bhat^T x_n - x_{n+1}."""
        X = x.reshape(self.Nt, self.N)
        Y = (self.Bhat.T @ X.T).T
        Y[:-1] -= X[1:]
        return Y.ravel()

    def schur_apply(self, x):
        """S-hat x = Jhat (Jhat^T x) / h."""
        return self.jhat_apply(self.jhat_T_apply(x)) / self.h

    # ----- local solves --------------------------------------------------------------------
    def _bhat_solve(self, b, trans="N"):
        return self._lu.solve(np.ascontiguousarray(b), trans=trans)

    def _jhat_local_solve(self, rhs):
        """Jhat_s^{-1} on an extended subdomain: forward backward-Euler sweep, zero IC before."""
        out = np.empty_like(rhs)
        prev = np.zeros(self.N)
        for k in range(rhs.shape[0]):
            prev = self._bhat_solve(rhs[k] + prev)
            out[k] = prev
        return out

    def _jhat_local_solve_T(self, rhs):
        """Jhat_s^{-T}: backward (adjoint) sweep, zero terminal condition after the last node."""
        out = np.empty_like(rhs)
        nxt = np.zeros(self.N)
        for k in range(rhs.shape[0] - 1, -1, -1):
            nxt = self._bhat_solve(rhs[k] + nxt, trans="T")
            out[k] = nxt
        return out

    def rasq(self, r):
        """One-level RASQ of Eq 13: sum_s R_s^T D_s R_s Q_s^T Jhat_s^{-T} M_s Jhat_s^{-1} Q_s R_s^T R_s r."""
        R = r.reshape(self.Nt, self.N)
        y = np.zeros_like(R)
        for sd in self.subs:
            ext = np.arange(sd.extended_first, sd.last + 1)       # nodes of Q_s
            x_s = R[sd.nodes - 1]                                  # R_s r
            e = np.zeros((ext.size, self.N))                       # Q_s R_s^T x_s
            e[np.searchsorted(ext, sd.nodes)] = x_s
            v = self._jhat_local_solve(e)                          # Jhat_s^{-1}
            g = self.h * v                                         # M_s = Q_s M_u Q_s^T = h I
            yy = self._jhat_local_solve_T(g)                       # Jhat_s^{-T}
            y_s = yy[np.searchsorted(ext, sd.nodes)]               # R_s Q_s^T
            keep = (sd.nodes >= sd.owned_first) & (sd.nodes <= sd.owned_last)   # D_s
            y[sd.nodes[keep] - 1] += y_s[keep]                     # R_s^T
        return y.ravel()

    def ras(self, r):
        """RAS of Eq 9 with the explicitly formed local Schur matrices R_s S-hat R_s^T."""
        R = r.reshape(self.Nt, self.N)
        y = np.zeros_like(R)
        S = self.S_hat
        for sd in self.subs:
            idx = ((sd.nodes - 1)[:, None] * self.N + np.arange(self.N)[None, :]).ravel()
            Ss = S[idx][:, idx].tocsc()
            y_s = spla.spsolve(Ss, r[idx]).reshape(sd.nodes.size, self.N)
            keep = (sd.nodes >= sd.owned_first) & (sd.nodes <= sd.owned_last)
            y[sd.nodes[keep] - 1] += y_s[keep]
        return y.ravel()

    # ----- Nicolaides coarse space (Eq 14) -------------------------------------------------
    def phi(self, sd: Subdomain) -> np.ndarray:
        """Phi_s: rows k = 0..m_s, columns (1, -1 + 2k/m_s) (Eq 14)."""
        k = np.arange(sd.m + 1, dtype=np.float64)
        return np.stack([np.ones_like(k), -1.0 + 2.0 * k / sd.m], axis=1)

    def coarse_time_basis(self) -> sp.csr_matrix:
        """Z_t (Nt x 2 N_D): column 2(s-1)+c is D_s Phi_s[:, c] placed on subdomain s's nodes."""
        rows, cols, vals = [], [], []
        for sd in self.subs:
            ph = self.phi(sd)
            lo = sd.first - sd.k0                      # node of Phi_s row 0
            for node in sd.owned:
                k = node - lo
                for c in range(2):
                    rows.append(node - 1)
                    cols.append(2 * (sd.s - 1) + c)
                    vals.append(ph[k, c])
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.Nt, 2 * self.n_sub))

    @property
    def Z(self) -> sp.csr_matrix:
        """Z = Z_t kron I_N: coarse column index (2(s-1)+c) * N + spatial dof."""
        if self._Z is None:
            self._Z = sp.kron(self.coarse_time_basis(), sp.identity(self.N)).tocsr()
        return self._Z

    def _build_coarse(self):
        Z = self.Z
        S0 = (Z.T @ self.S_hat @ Z).tocsc()          # S_0 = R_0 S-hat R_0^T, R_0 = Z^T
        self._S0 = S0
        self._S0_lu = spla.splu(S0)

    def coarse_matrix(self) -> sp.csc_matrix:
        if self._S0_lu is None:
            self._build_coarse()
        return self._S0

    def coarse(self, r):
        """R_0^T S_0^{-1} R_0 r."""
        if self.mode_diagonal is not None:
            return self.coarse_per_mode(r)
        if self._S0_lu is None:
            self._build_coarse()
        return self.Z @ self._S0_lu.solve(self.Z.T @ r)

    def coarse_per_mode(self, r, chunk: int = 1024, mode_limit: int | None = None):
        """R_0^T S_0^{-1} R_0 r with S_0 solved mode by mode.

        Z = Z_t kron I_N commutes with the spatial transform Q, and Q Bhat Q = diag(mu), so
        S_0 = (I kron Q) blockdiag_q(Z_t^T T(mu_q) Z_t / h) (I kron Q), where
        T(mu) = Jhat Jhat^T for the scalar diagonal mu: mu^2 I + D - mu E, D = diag(0, 1, .., 1)
        and E the time shift in both directions. Each mode's 2 N_D x 2 N_D system is solved
        densely (numpy.linalg.solve), in batches of modes.
        """
        Zt = self.coarse_time_basis().toarray()
        Nt = self.Nt
        D = np.ones(Nt)
        D[0] = 0.0
        E = np.eye(Nt, k=1) + np.eye(Nt, k=-1)
        G1 = Zt.T @ Zt
        G2 = Zt.T @ (D[:, None] * Zt)
        G3 = Zt.T @ E @ Zt
        R = r.reshape(Nt, self.N)
        c = Zt.T @ R                                   # R_0 r: [2 N_D][N]
        chat = self.mode_transform(c)                  # into the sine basis, row by row
        out = np.zeros_like(chat)
        mu = self.mode_diagonal
        for q0 in range(0, self.N if mode_limit is None else min(mode_limit, self.N), chunk):
            m = mu[q0:q0 + chunk]
            S0 = (m[:, None, None] ** 2 * G1[None] + G2[None] - m[:, None, None] * G3[None]) / self.h
            out[:, q0:q0 + chunk] = np.linalg.solve(S0, chat[:, q0:q0 + chunk].T[:, :, None])[:, :, 0].T
        x = self.mode_transform(out)
        return (Zt @ x).ravel()

    # ----- two-level composition (Eq 15) ---------------------------------------------------
    def apply(self, r):
        r = np.asarray(r, dtype=np.float64)
        if self.variant == "one-level":
            return self.rasq(r)
        if self.variant == "ras":
            return self.ras(r)
        x0 = self.coarse(r)
        if self.variant == "ras-multiplicative":
            # Eq 15's coarse-first composition with Eq 9's local solves in place of RASQ
            return x0 + self.ras(r - self.schur_apply(x0))
        if self.variant == "multiplicative":
            return x0 + self.rasq(r - self.schur_apply(x0))
        if self.variant == "additive":
            return x0 + self.rasq(r)
        raise ValueError(self.variant)


def schur_preconditioner(p: HeatKKT, n_sub: int, *, jhat_sign: int = -1, coarse_solver: str = "sparse-lu",
                         **kw) -> SchurPreconditioner:
    """The approximate Schur inverse of the physical problem (Bhat from jhat_diagonal_block).

    coarse_solver="sparse-lu" factors Z^T S-hat Z as a sparse matrix (the literal definition);
    "per-mode" solves it in the sine basis (see SchurPreconditioner.coarse_per_mode), which a
    test checks against the sparse factorisation.
    """
    if coarse_solver == "per-mode":
        from . import spectral

        mu = spectral.jhat_mode_diagonal(p, jhat_sign)

        def transform(X):
            return spectral.dst2(X, p).reshape(X.shape[0], -1)

        kw = dict(kw, mode_diagonal=mu, mode_transform=transform)
    return SchurPreconditioner(jhat_diagonal_block(p, jhat_sign), p.Nt, n_sub, p.h, **kw)


def block_preconditioner_apply(p: HeatKKT, schur: SchurPreconditioner, r):
    """P^{-1} r of Eq 7: P = diag(M_u, omega M_z, S-hat), S-hat^{-1} replaced by ``schur``."""
    r = np.asarray(r, dtype=np.float64)
    V = p.V
    yu = r[:V] / p.h
    yz = r[V : 2 * V] / (p.omega * p.h)
    yw = schur.apply(r[2 * V :])
    return np.concatenate([yu, yz, yw])
