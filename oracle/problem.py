"""Discrete heat-equation optimal-control problem and its KKT system (Section 2, Eqs 2-5).

TEST INFRASTRUCTURE ONLY (see the package docstring): a literal FP64 restatement used
to check the CUDA path, never imported by it.

Index conventions (used by every side of the project):
* ``nx, ny`` are numbers of grid *intervals*; the interior indices are i = 1..nx-1 and
  j = 1..ny-1 (Section 2, below Eq 2), the boundary values are eliminated (they are 0).
  The paper's "17 x 17 mesh points, 15 x 15 unknowns" (Section 4) fixes this reading.
* A space-time block is stored [n][j][i], n = 1..Nt the time node, i fastest.
* dx = Lx/nx, dy = Ly/ny, dt = T/Nt and h = dt*dx*dy, the scale of M_u = M_z (Eq 5).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass(frozen=True)
class HeatKKT:
    """Sizes and coefficients of one KKT instance (Eq 1 discretised as in Section 2)."""

    nx: int
    ny: int
    Nt: int
    T: float = 1.0
    nu: float = 1.0
    omega: float = 1e-4
    Lx: float = 1.0
    Ly: float = 1.0

    @property
    def Mx(self) -> int:
        return self.nx - 1

    @property
    def My(self) -> int:
        return self.ny - 1

    @property
    def N(self) -> int:
        """Spatial unknowns per time node."""
        return self.Mx * self.My

    @property
    def V(self) -> int:
        """Unknowns per space-time block (u, z or w)."""
        return self.N * self.Nt

    @property
    def dx(self) -> float:
        return self.Lx / self.nx

    @property
    def dy(self) -> float:
        return self.Ly / self.ny

    @property
    def dt(self) -> float:
        return self.T / self.Nt

    @property
    def h(self) -> float:
        """M_u = M_z = dt*dx*dy * I (Eq 5 and the sentence after it)."""
        return self.dt * self.dx * self.dy

    def interior_points(self):
        """Coordinates (x_i, y_j) of the interior nodes, arrays of shape [My][Mx]."""
        x = self.dx * np.arange(1, self.nx)
        y = self.dy * np.arange(1, self.ny)
        return np.meshgrid(x, y, indexing="xy")


def second_difference(n_intervals: int, d: float) -> sp.csr_matrix:
    """tridiag(-1, 2, -1)/d^2 on the n_intervals-1 interior nodes (Dirichlet 0 eliminated)."""
    m = n_intervals - 1
    main = np.full(m, 2.0)
    off = np.full(max(m - 1, 0), -1.0)
    return (sp.diags([off, main, off], [-1, 0, 1], shape=(m, m)) / (d * d)).tocsr()


def laplacian(p: HeatKKT) -> sp.csr_matrix:
    """The 5-point negative Laplacian A of Eq 2: the bracket multiplying dt*nu there.

    With i fastest, the x-second-difference acts inside each j-row (kron(I_y, T_x)) and the
    y-second-difference couples rows j and j+-1 (kron(T_y, I_x)).
    """
    tx = second_difference(p.nx, p.dx)
    ty = second_difference(p.ny, p.dy)
    return (sp.kron(sp.identity(p.My), tx) + sp.kron(ty, sp.identity(p.Mx))).tocsr()


def state_block(p: HeatKKT) -> sp.csr_matrix:
    """J_{(n+1)(n+1)} of Eq 3: I + dt*nu*A (the implicit backward-Euler operator)."""
    return (sp.identity(p.N) + p.dt * p.nu * laplacian(p)).tocsr()


def time_stepping_matrix(diag_block, sub_block, Nt: int) -> sp.csr_matrix:
    """Block lower-bidiagonal space-time matrix: diag_block on the diagonal, sub_block below.

    This is the shape of J in Eqs 3-4 (one block row per time node n = 1..Nt; the block
    coupling node 1 to the initial condition u^0 is moved to the right-hand side). It is also
    the shape of the three-step Euler example of Section 3.
    """
    diag_block = sp.csr_matrix(diag_block)
    sub_block = sp.csr_matrix(sub_block)
    d = sp.kron(sp.identity(Nt), diag_block)
    s = sp.kron(sp.eye(Nt, k=-1), sub_block)
    return (d + s).tocsr()


def assemble_J(p: HeatKKT) -> sp.csr_matrix:
    """J of Eq 4: J_{nn} = I + dt*nu*A, J_{n,n-1} = -I (Eq 2 rearranged as Eq 3)."""
    return time_stepping_matrix(state_block(p), -sp.identity(p.N), p.Nt)


def assemble_L(p: HeatKKT) -> sp.csr_matrix:
    """L of Eq 4: block diagonal, L_{nn} = -dt*I (the dt*z^{n+1} term of Eq 2 moved left)."""
    return (-p.dt * sp.identity(p.V)).tocsr()


def assemble_K(p: HeatKKT) -> sp.csr_matrix:
    """The KKT matrix of Eq 5 on the unknown (u, z, w)."""
    J = assemble_J(p)
    L = assemble_L(p)
    Mu = p.h * sp.identity(p.V)
    Mz = p.h * sp.identity(p.V)
    return sp.bmat([[Mu, None, J.T], [None, p.omega * Mz, L.T], [J, L, None]]).tocsr()


def assemble_rhs(p: HeatKKT, u_target: np.ndarray, u0: np.ndarray | None) -> np.ndarray:
    """Right-hand side (f_u, f_z, f) of Eq 5.

    The paper states only that f carries the initial condition (below Eq 4). Taking the
    first-order conditions of the rectangle-rule discretisation of Eq 1,
    1/2 (u - u~)^T M_u (u - u~) + omega/2 z^T M_z z subject to J u + L z = f, gives
    f_u = M_u u~ and f_z = 0; moving the known u^0 of the first step of Eq 2 to the right gives
    f = (u_0, 0, ..., 0).
    """
    u_target = np.asarray(u_target, dtype=np.float64).reshape(p.V)
    fu = p.h * u_target
    fz = np.zeros(p.V)
    fw = np.zeros(p.V)
    if u0 is not None:
        fw[: p.N] = np.asarray(u0, dtype=np.float64).reshape(p.N)
    return np.concatenate([fu, fz, fw])


def kkt_apply_blockwise(p: HeatKKT, x: np.ndarray) -> np.ndarray:
    """K x of Eq 5, one time node at a time (same operator as assemble_K, O(V) memory).

    Used where the full sparse K does not fit; a test checks it against assemble_K.
    """
    B0 = state_block(p)
    Nt, N = p.Nt, p.N
    u = x[: p.V].reshape(Nt, N)
    z = x[p.V : 2 * p.V].reshape(Nt, N)
    w = x[2 * p.V :].reshape(Nt, N)
    yu = np.empty_like(u)
    yz = np.empty_like(z)
    yw = np.empty_like(w)
    for n in range(Nt):
        # row block n of M_u u + J^T w: J^T has B0^T on the diagonal and -I above it
        t = p.h * u[n] + B0.T @ w[n]
        if n + 1 < Nt:
            t = t - w[n + 1]
        yu[n] = t
        # omega M_z z + L^T w
        yz[n] = p.omega * p.h * z[n] - p.dt * w[n]
        # J u + L z
        t = B0 @ u[n] - p.dt * z[n]
        if n > 0:
            t = t - u[n - 1]
        yw[n] = t
    return np.concatenate([yu.ravel(), yz.ravel(), yw.ravel()])


def l2_residual_weights(p: HeatKKT) -> np.ndarray:
    """Row weights of the residual norm used to stop the solve.

    The rows of Eq 5 are, per time node and grid point, a gradient of the discrete objective
    (u and z rows: the residual is a functional, measured in the dual L2 norm, weight
    h^{-1/2}) and the state equation (w rows: a function, measured in the space-time L2 norm
    with the mass h, weight h^{1/2}). This is the discrete L2(0,T; L2(Omega)) norm pair; the
    paper states only "relative residual".
    """
    V = p.V
    return np.concatenate([np.full(V, p.h ** -0.5), np.full(V, p.h ** -0.5), np.full(V, p.h ** 0.5)])
