"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a value the paper
prints (tests/golden), a closed form, a brute-force loop over Eq 2, an independent
formulation (reduced-space least squares, dense LU, per-mode DST solve) or an exact
invariant. Together they are chosen so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them.
"""

import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import krylov, problem, schwarz, spectral
from oracle.problem import HeatKKT
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]


def _tiny(nx=5, ny=4, Nt=8, omega=1e-2, nu=0.7, T=1.0, Lx=1.0, Ly=1.3):
    return HeatKKT(nx=nx, ny=ny, Nt=Nt, T=T, nu=nu, omega=omega, Lx=Lx, Ly=Ly)


# ---------------------------------------------------------------------------------------
# Values printed in the paper
# ---------------------------------------------------------------------------------------

def _poly_matrix(lines, section, dt, n=3):
    M = np.zeros((n, n))
    on = False
    for ln in lines:
        if ln.startswith("["):
            on = ln == f"[{section}]"
            continue
        if on:
            r, c, c0, c1, c2 = ln.split()
            M[int(r), int(c)] = float(c0) + float(c1) * dt + float(c2) * dt * dt
    return M


@pytest.mark.parametrize("dt", [0.1, 0.37, 1.5])
def test_three_step_euler_schur_matches_printed_example(dt):
    """Section 3 example: the oracle's time-stepping assembly and Schur product give the
    printed J and J J^T of the three-step forward-Euler discretisation of y' = -y."""
    lines = _golden_lines("ode3_schur.txt")
    J_printed = _poly_matrix(lines, "J", dt)
    S_printed = _poly_matrix(lines, "JJT", dt)
    # forward Euler y^{n+1} - y^n + dt y^n = 0: diagonal block 1, sub-diagonal block -1 + dt
    J = problem.time_stepping_matrix([[1.0]], [[-1.0 + dt]], 3).toarray()
    np.testing.assert_allclose(J, J_printed, rtol=0, atol=1e-15)
    S = schwarz.congruence(J, 1.0).toarray()
    np.testing.assert_allclose(S, S_printed, rtol=0, atol=1e-14)


def test_subdomain_nodes_match_printed_example():
    """Section 3: Nt = 9, N_D = 3 gives nodes {1,2,3}, {3,4,5,6}, {6,7,8,9}."""
    lines = _golden_lines("subdomains_nt9_nd3.txt")
    subs = schwarz.subdomains(9, 3)
    for ln in lines:
        head, vals = ln.split(":")
        kind, s = head.split()
        want = [int(v) for v in vals.split()]
        if kind == "nodes":
            assert list(subs[int(s) - 1].nodes) == want


def test_extended_range_matches_printed_example():
    """Section 3: the range of Jhat^T R_s^T for the subdomain {3,4,5,6} is nonzero on {2..6}.

    Read from the sparsity of the oracle's Jhat (N = 2 spatial dofs, Nt = 9)."""
    lines = _golden_lines("subdomains_nt9_nd3.txt")
    want = [int(v) for v in [ln for ln in lines if ln.startswith("range")][0].split(":")[1].split()]
    N = 2
    pre = schwarz.SchurPreconditioner(np.array([[2.0, -0.3], [-0.3, 2.5]]), 9, 3, 1.0,
                                      variant="one-level")
    sd = pre.subs[1]
    cols = ((sd.nodes - 1)[:, None] * N + np.arange(N)[None, :]).ravel()
    block = pre.Jhat.T.tocsc()[:, cols]
    rows = np.unique(block.nonzero()[0] // N) + 1
    assert list(rows) == want
    assert sd.extended_first == want[0]


def test_phi_columns_match_printed_formula():
    """Eq 14: Phi_s rows (1, -1 + 2k/N_s); the oracle's Phi for N_s = 4."""
    want = np.array([[float(v) for v in ln.split()] for ln in _golden_lines("phi_ns4.txt")])
    pre = schwarz.SchurPreconditioner(np.array([[3.0]]), 8, 2, 1.0, variant="one-level")
    sd = pre.subs[1]
    assert sd.m == 4
    np.testing.assert_allclose(pre.phi(sd), want, rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------------------
# Closed forms and brute force for the discretisation (Section 2)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("k,l", [(1, 1), (2, 3), (4, 1)])
def test_laplacian_sine_modes_closed_form(k, l):
    """A sin(k pi x/Lx) sin(l pi y/Ly) = lambda_kl (same), lambda from the closed form."""
    p = _tiny(nx=6, ny=5, Lx=1.0, Ly=1.7)
    X, Y = p.interior_points()
    phi = (np.sin(k * np.pi * X / p.Lx) * np.sin(l * np.pi * Y / p.Ly)).ravel()
    lam = 4 / p.dx**2 * np.sin(k * np.pi / (2 * p.nx)) ** 2 + 4 / p.dy**2 * np.sin(l * np.pi / (2 * p.ny)) ** 2
    np.testing.assert_allclose(problem.laplacian(p) @ phi, lam * phi, rtol=1e-12, atol=1e-11)
    np.testing.assert_allclose(spectral.mode_eigenvalues(p)[l - 1, k - 1], lam, rtol=1e-14)


def test_backward_euler_step_decay_of_sine_modes():
    """One backward-Euler step of Eq 2 (z = 0) scales a sine mode by 1/(1 + dt nu lambda_kl)."""
    p = _tiny(nx=8, ny=6, Ly=2.0, nu=1.3, Nt=5)
    X, Y = p.interior_points()
    B0 = problem.state_block(p).toarray()
    lam = spectral.mode_eigenvalues(p)
    for k, l in [(1, 1), (3, 2), (7, 5)]:
        phi = (np.sin(k * np.pi * X / p.Lx) * np.sin(l * np.pi * Y / p.Ly)).ravel()
        nxt = np.linalg.solve(B0, phi)
        np.testing.assert_allclose(nxt, phi / (1 + p.dt * p.nu * lam[l - 1, k - 1]), rtol=1e-12, atol=1e-14)


def test_state_equation_rows_match_eq2_by_brute_force():
    """J u + L z - f evaluated by the oracle equals Eq 2 written out point by point."""
    p = _tiny(nx=5, ny=4, Nt=4, Lx=1.0, Ly=1.5, nu=0.9)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((p.Nt, p.My, p.Mx))
    z = rng.standard_normal((p.Nt, p.My, p.Mx))
    u0 = rng.standard_normal((p.My, p.Mx))
    f = problem.assemble_rhs(p, np.zeros(p.V), u0)
    got = problem.assemble_J(p) @ u.ravel() + problem.assemble_L(p) @ z.ravel() - f[2 * p.V:]

    def U(n, j, i):                       # 1-based indices, 0 on the boundary, u0 at n = 0
        if i < 1 or i > p.Mx or j < 1 or j > p.My:
            return 0.0
        return u0[j - 1, i - 1] if n == 0 else u[n - 1, j - 1, i - 1]

    want = np.zeros_like(u)
    for n in range(0, p.Nt):              # row of Eq 2 for the step n -> n+1
        for j in range(1, p.My + 1):
            for i in range(1, p.Mx + 1):
                lap = ((-U(n + 1, j, i + 1) + 2 * U(n + 1, j, i) - U(n + 1, j, i - 1)) / p.dx**2
                       + (-U(n + 1, j + 1, i) + 2 * U(n + 1, j, i) - U(n + 1, j - 1, i)) / p.dy**2)
                want[n, j - 1, i - 1] = (U(n + 1, j, i) - U(n, j, i) + p.dt * p.nu * lap
                                         - p.dt * z[n, j - 1, i - 1])
    np.testing.assert_allclose(got, want.ravel(), rtol=1e-13, atol=1e-12)


def test_kkt_solution_minimises_reduced_objective():
    """The KKT solution (Eq 5) equals the minimiser of the discrete Eq 1 found independently:
    eliminate u = J^{-1}(f - L z) and solve the reduced least-squares problem in z."""
    p = _tiny(nx=4, ny=5, Nt=5, omega=3e-2, nu=0.8, Ly=1.2)
    rng = np.random.default_rng(7)
    ut = rng.standard_normal(p.V)
    u0 = rng.standard_normal(p.N)
    K = problem.assemble_K(p)
    f = problem.assemble_rhs(p, ut, u0)
    x = np.linalg.solve(K.toarray(), f)
    J = problem.assemble_J(p).toarray()
    L = problem.assemble_L(p).toarray()
    fw = np.zeros(p.V)
    fw[: p.N] = u0
    # objective 1/2 h |u - ut|^2 + omega/2 h |z|^2 with u = J^{-1} fw - J^{-1} L z
    Ji = np.linalg.inv(J)
    G = -Ji @ L
    c = Ji @ fw - ut
    A = np.vstack([np.sqrt(p.h) * G, np.sqrt(p.omega * p.h) * np.eye(p.V)])
    b = np.concatenate([-np.sqrt(p.h) * c, np.zeros(p.V)])
    z = np.linalg.lstsq(A, b, rcond=None)[0]
    u = Ji @ (fw - L @ z)
    np.testing.assert_allclose(x[: p.V], u, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(x[p.V: 2 * p.V], z, rtol=1e-9, atol=1e-10)


def test_blockwise_matvec_matches_sparse_K():
    p = _tiny(nx=6, ny=5, Nt=7)
    x = workloads.random_vector(3 * p.V, 11)
    np.testing.assert_allclose(problem.kkt_apply_blockwise(p, x), problem.assemble_K(p) @ x,
                               rtol=1e-13, atol=1e-13)


def test_block_ldu_factorisation_and_schur_complement():
    """Section 2: K = L D U with S = J M_u^{-1} J^T + omega^{-1} L M_z^{-1} L^T."""
    p = _tiny(nx=4, ny=4, Nt=3)
    J = problem.assemble_J(p).toarray()
    L = problem.assemble_L(p).toarray()
    Mu = p.h * np.eye(p.V)
    Mz = p.h * np.eye(p.V)
    I = np.eye(p.V)
    O = np.zeros((p.V, p.V))
    S = J @ np.linalg.inv(Mu) @ J.T + L @ np.linalg.inv(Mz) @ L.T / p.omega
    Lf = np.block([[I, O, O], [O, I, O], [J @ np.linalg.inv(Mu), L @ np.linalg.inv(Mz) / p.omega, I]])
    D = np.block([[Mu, O, O], [O, p.omega * Mz, O], [O, O, -S]])
    Uf = np.block([[I, O, np.linalg.inv(Mu) @ J.T], [O, I, np.linalg.inv(Mz) @ L.T / p.omega], [O, O, I]])
    np.testing.assert_allclose(Lf @ D @ Uf, problem.assemble_K(p).toarray(), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------------------
# Solves: dense LU and the per-mode exact solve
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("nx,Nt,nd", [(4, 8, 2), (5, 8, 4), (4, 16, 4)])
def test_fgmres_two_level_matches_dense_lu(nx, Nt, nd):
    p = HeatKKT(nx=nx, ny=nx, Nt=Nt, nu=1.0, omega=1e-3)
    w = workloads.Workload("t", nx=nx, ny=nx, Nt=Nt, n_sub=nd, omega=1e-3, seed=5)
    f = problem.assemble_rhs(p, workloads.make_target(w), workloads.random_vector(p.N, 2))
    K = problem.assemble_K(p)
    pre = schwarz.schur_preconditioner(p, nd)
    res = krylov.fgmres(lambda v: K @ v, lambda r: schwarz.block_preconditioner_apply(p, pre, r),
                        f, tol=1e-13, restart=30, maxit=300)
    assert res.converged
    x = np.linalg.solve(K.toarray(), f)
    assert np.linalg.norm(res.x - x) <= 1e-10 * np.linalg.norm(x)


def test_per_mode_exact_solve_matches_dense_lu():
    p = _tiny(nx=5, ny=4, Nt=6, Ly=1.4, omega=2e-3)
    f = workloads.random_vector(3 * p.V, 21)
    x = np.linalg.solve(problem.assemble_K(p).toarray(), f)
    np.testing.assert_allclose(spectral.kkt_exact_solve(p, f), x, rtol=1e-10, atol=1e-10 * np.abs(x).max())


# ---------------------------------------------------------------------------------------
# The preconditioner: invariants and identities (Section 3)
# ---------------------------------------------------------------------------------------

def test_single_subdomain_gives_exact_schur_inverse():
    """N_D = 1: RASQ, RAS (Eq 9) and their two-level compositions all equal S-hat^{-1} exactly."""
    p = _tiny(nx=5, ny=6, Nt=9, omega=1e-3)
    x = workloads.random_vector(p.V, 4)
    for variant in ("one-level", "multiplicative", "ras", "ras-multiplicative"):
        pre = schwarz.schur_preconditioner(p, 1, variant=variant)
        r = pre.S_hat @ x
        np.testing.assert_allclose(pre.apply(r), x, rtol=1e-11, atol=1e-11 * np.abs(x).max())
    # the additive composition is not exact here, which separates the two readings
    pre = schwarz.schur_preconditioner(p, 1, variant="additive")
    assert np.linalg.norm(pre.apply(pre.S_hat @ x) - x) > 1e-3 * np.linalg.norm(x)


def test_schur_apply_matches_assembled_product():
    p = _tiny(nx=4, ny=5, Nt=6)
    pre = schwarz.schur_preconditioner(p, 2)
    x = workloads.random_vector(p.V, 9)
    np.testing.assert_allclose(pre.schur_apply(x), pre.S_hat @ x, rtol=1e-13, atol=1e-10)
    Jh = pre.Jhat.toarray()
    np.testing.assert_allclose(pre.S_hat.toarray(), Jh @ Jh.T / p.h, rtol=1e-13, atol=1e-8)


def _restriction_matrices(pre, sd):
    Nt, N = pre.Nt, pre.N
    I = np.eye(Nt * N)
    rows_R = np.concatenate([np.arange((n - 1) * N, n * N) for n in sd.nodes])
    ext = np.arange(sd.extended_first, sd.last + 1)
    rows_Q = np.concatenate([np.arange((n - 1) * N, n * N) for n in ext])
    return I[rows_R], I[rows_Q]


def test_extended_restriction_identities_eqs_10_to_12():
    """Q_s Q_s^T = I, Q_s^T Q_s Jhat^T R_s^T = Jhat^T R_s^T, R_s = R_s Q_s^T Q_s, Eq 11 = Eq 12,
    and the RASQ local operator equals (R_s Jhat R_s^T)^{-T} M (R_s Jhat R_s^T)^{-1}."""
    p = _tiny(nx=4, ny=4, Nt=9, omega=1e-2)
    pre = schwarz.schur_preconditioner(p, 3, variant="one-level")
    Jh = pre.Jhat.toarray()
    Minv = np.eye(p.V) / p.h
    for sd in pre.subs:
        R, Q = _restriction_matrices(pre, sd)
        np.testing.assert_allclose(Q @ Q.T, np.eye(Q.shape[0]), atol=0)
        np.testing.assert_allclose(Q.T @ Q @ Jh.T @ R.T, Jh.T @ R.T, atol=1e-13)
        np.testing.assert_allclose(R @ Q.T @ Q, R, atol=0)
        lhs = R @ Jh @ Minv @ Jh.T @ R.T
        eq11 = R @ Jh @ Q.T @ (Q @ Minv @ Q.T) @ Q @ Jh.T @ R.T
        Js = Q @ Jh @ Q.T
        Ms_inv = Q @ Minv @ Q.T
        eq12 = R @ Q.T @ Js @ Ms_inv @ Js.T @ Q @ R.T
        np.testing.assert_allclose(eq11, lhs, rtol=1e-12, atol=1e-6)
        np.testing.assert_allclose(eq12, lhs, rtol=1e-12, atol=1e-6)
        # RASQ local operator (Eq 13 parenthesis) against the sweep implementation
        Ms = np.linalg.inv(Ms_inv)
        local = R @ Q.T @ np.linalg.inv(Js).T @ Ms @ np.linalg.inv(Js) @ Q @ R.T
        Jloc = R @ Jh @ R.T
        np.testing.assert_allclose(local, np.linalg.inv(Jloc).T @ (p.h * np.eye(R.shape[0])) @ np.linalg.inv(Jloc),
                                   rtol=1e-10, atol=1e-14)
        rs = workloads.random_vector(R.shape[0], sd.s)
        # the oracle's sweep implementation of the same local operator
        e = np.zeros((Q.shape[0] // p.N, p.N))
        e[np.searchsorted(np.arange(sd.extended_first, sd.last + 1), sd.nodes)] = rs.reshape(-1, p.N)
        v = pre._jhat_local_solve(e)
        yy = pre._jhat_local_solve_T(p.h * v)
        y_s = yy[np.searchsorted(np.arange(sd.extended_first, sd.last + 1), sd.nodes)].ravel()
        np.testing.assert_allclose(y_s, local @ rs, rtol=1e-10, atol=1e-12 * np.abs(y_s).max())


def test_galerkin_orthogonality_of_coarse_correction():
    """R_0 (r - S-hat x_0) = 0 for x_0 = R_0^T S_0^{-1} R_0 r, and r = S-hat Z c gives x_0 = Z c."""
    p = _tiny(nx=5, ny=4, Nt=12, omega=1e-3)
    pre = schwarz.schur_preconditioner(p, 4)
    r = workloads.random_vector(p.V, 13)
    x0 = pre.coarse(r)
    np.testing.assert_allclose(pre.Z.T @ (r - pre.schur_apply(x0)), 0, atol=1e-9 * np.abs(r).max())
    c = workloads.random_vector(pre.Z.shape[1], 14)
    np.testing.assert_allclose(pre.coarse(pre.schur_apply(pre.Z @ c)), pre.Z @ c, rtol=1e-9, atol=1e-9)
    # the multiplicative composition reproduces the coarse range exactly (coarse first)
    np.testing.assert_allclose(pre.apply(pre.schur_apply(pre.Z @ c)), pre.Z @ c, rtol=1e-9, atol=1e-9)


def test_coarse_basis_columns_are_constant_and_linear_on_owned_nodes():
    pre = schwarz.SchurPreconditioner(np.array([[2.0]]), 12, 3, 1.0)
    Zt = pre.coarse_time_basis().toarray()
    assert Zt.shape == (12, 6)
    np.testing.assert_allclose(Zt[:, 0], [1, 1, 1, 1] + [0] * 8)
    np.testing.assert_allclose(Zt[:4, 1], [-0.5, 0.0, 0.5, 1.0])
    np.testing.assert_allclose(Zt[4:8, 3], [-0.5, 0.0, 0.5, 1.0])
    # every node is owned once: the columns of constants sum to one
    np.testing.assert_allclose(Zt[:, 0::2].sum(axis=1), 1.0)


def test_literal_jhat_sign_is_indefinite_at_the_small_configuration():
    """The literal sign of Eq 7 gives diagonal blocks with negative eigenvalues at the
    32 x 32, Nt = 64, omega = 1e-4 problem; the adopted sign keeps them above 1."""
    p = HeatKKT(nx=32, ny=32, Nt=64, nu=1.0, omega=1e-4)
    lit = spectral.jhat_mode_diagonal(p, +1)
    ado = spectral.jhat_mode_diagonal(p, -1)
    assert lit.min() < 0 < lit.max()
    assert ado.min() > 1.0


def test_per_mode_scalar_oracle_matches_physical_oracle():
    """The physical-space preconditioner applied to a block living on one sine mode equals the
    same preconditioner built for the scalar diagonal mu_kl, times the mode."""
    w = workloads.Workload("t", nx=6, ny=5, Nt=12, n_sub=3, Ly=1.5, omega=1e-3, nu=0.8)
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega, Ly=w.Ly)
    mu = spectral.jhat_mode_diagonal(p)
    for variant in ("multiplicative", "one-level"):
        phys = schwarz.schur_preconditioner(p, w.n_sub, variant=variant)
        for (k, l) in [(1, 1), (3, 2)]:
            blk, coeff = workloads.random_mode_block(w, [(k, l)], seed=k * 10 + l)
            y = phys.apply(blk.ravel()).reshape(w.Nt, -1)
            scal = schwarz.SchurPreconditioner(np.array([[mu[l - 1, k - 1]]]), w.Nt, w.n_sub, p.h,
                                               variant=variant)
            ys = scal.apply(coeff[:, 0])
            shape = blk[0] / coeff[0, 0]
            np.testing.assert_allclose(y, ys[:, None] * shape.ravel()[None, :], rtol=1e-10,
                                       atol=1e-10 * np.abs(y).max())


def test_two_level_iterations_flat_one_level_growing():
    """Section 4 trends on a small grid: two-level counts stay flat as N_D grows, one-level
    counts grow (the printed figures are missing, so only the trend is pinned)."""
    its = {}
    for nd in (2, 8, 16):
        p = HeatKKT(nx=8, ny=8, Nt=64, nu=1.0, omega=1e-2)
        w = workloads.Workload("t", nx=8, ny=8, Nt=64, n_sub=nd, omega=1e-2, target="paper")
        f = problem.assemble_rhs(p, workloads.make_target(w), None)
        K = problem.assemble_K(p)
        for variant in ("multiplicative", "one-level"):
            pre = schwarz.schur_preconditioner(p, nd, variant=variant)
            res = krylov.fgmres(lambda v: K @ v, lambda r: schwarz.block_preconditioner_apply(p, pre, r),
                                f, tol=1e-6, restart=30, maxit=400)
            its[(variant, nd)] = res.iterations
    assert its[("multiplicative", 16)] <= its[("multiplicative", 2)] + 3
    assert its[("one-level", 16)] > its[("one-level", 2)]
    assert its[("multiplicative", 16)] < its[("one-level", 16)]


def test_ras_and_rasq_differ_only_through_the_first_node():
    """Eq 9 vs Eq 13: R_s S-hat R_s^T minus (R_s Jhat R_s^T) M^{-1} (...)^T is nonzero only in the
    first node's diagonal block (the missing -I coupling to the node before)."""
    p = _tiny(nx=4, ny=4, Nt=9)
    pre = schwarz.schur_preconditioner(p, 3, variant="one-level")
    Jh = pre.Jhat.toarray()
    S = pre.S_hat.toarray()
    sd = pre.subs[1]
    R, _ = _restriction_matrices(pre, sd)
    Jloc = R @ Jh @ R.T
    diff = R @ S @ R.T - Jloc @ Jloc.T / p.h
    N = p.N
    np.testing.assert_allclose(diff[:N, :N], np.eye(N) / p.h, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(diff[N:, :], 0, atol=1e-9)
    np.testing.assert_allclose(diff[:, N:], 0, atol=1e-9)


@pytest.mark.parametrize("pou", ["left", "right"])
def test_per_mode_coarse_solve_matches_sparse_factorisation(pou):
    """The per-mode coarse solve (used where the sparse coarse LU does not fit) equals the
    literal sparse R_0^T (Z^T S-hat Z)^{-1} R_0."""
    p = HeatKKT(nx=8, ny=6, Nt=24, nu=0.9, omega=1e-3, Ly=1.5)
    a = schwarz.schur_preconditioner(p, 4, pou=pou)
    b = schwarz.schur_preconditioner(p, 4, pou=pou, coarse_solver="per-mode")
    r = workloads.random_vector(p.V, 31)
    np.testing.assert_allclose(b.coarse(r), a.coarse(r), rtol=1e-11, atol=1e-11 * np.abs(a.coarse(r)).max())
    np.testing.assert_allclose(b.apply(r), a.apply(r), rtol=1e-10, atol=1e-10 * np.abs(a.apply(r)).max())


def test_weighted_residual_norm_reaches_the_exact_solution():
    """In the L2-weighted norm the exact solution's relative residual is at rounding level and a
    1e-12 FGMRES solve is within 1e-10 of it; the Euclidean residual of the exact solution is
    already far above 1e-12 (the w rows carry O(1) coefficients against an O(h) right side)."""
    w = workloads.CFG_SMALL
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    f = problem.assemble_rhs(p, workloads.make_target(w), workloads.make_u0(w))
    K = problem.assemble_K(p)
    d = problem.l2_residual_weights(p)
    xe = spectral.kkt_exact_solve(p, f)
    assert np.linalg.norm(d * (f - K @ xe)) / np.linalg.norm(d * f) < 1e-13
    assert np.linalg.norm(f - K @ xe) / np.linalg.norm(f) > 1e-11
    pre = schwarz.schur_preconditioner(p, w.n_sub)
    res = krylov.fgmres(lambda v: K @ v, lambda r: schwarz.block_preconditioner_apply(p, pre, r), f,
                        tol=1e-12, restart=30, maxit=200, row_scale=d)
    assert res.converged
    assert np.linalg.norm(res.x - xe) <= 1e-10 * np.linalg.norm(xe)


# ---------------------------------------------------------------------------------------
# Learned coarse correction: the network reference (not in the paper)
# ---------------------------------------------------------------------------------------

def test_mlp_backward_matches_central_differences():
    from oracle import mlp
    rng = np.random.default_rng(0)
    params = mlp.init_params(6, 5, 4, seed=1)
    for k in ("b1", "b2", "b3"):
        params[k] = 0.1 * rng.standard_normal(params[k].shape)   # avoid kinks at zero
    X = rng.standard_normal((7, 6))
    T = rng.standard_normal((7, 4))
    Y, cache = mlp.forward(params, X)
    g = mlp.backward(params, cache, Y, T)
    for k, P in params.items():
        fd = np.zeros_like(P)
        for idx in np.ndindex(P.shape):
            old = P[idx]
            P[idx] = old + 1e-6
            lp = mlp.loss(mlp.forward(params, X)[0], T)
            P[idx] = old - 1e-6
            lm = mlp.loss(mlp.forward(params, X)[0], T)
            P[idx] = old
            fd[idx] = (lp - lm) / 2e-6
        np.testing.assert_allclose(g[k], fd, rtol=1e-6, atol=1e-8)


def test_adam_first_step_moves_each_parameter_by_lr():
    """With zero moments, the bias-corrected first Adam step is lr * g / (|g| + eps)."""
    from oracle import mlp
    params = {"w": np.array([1.0, -2.0, 3.0])}
    grads = {"w": np.array([0.5, -4.0, 1e-3])}
    state = {}
    mlp.adam_step(params, grads, state, t=1, lr=0.01)
    g = np.array([0.5, -4.0, 1e-3])
    np.testing.assert_allclose(params["w"], np.array([1.0, -2.0, 3.0]) - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_coarse_operator_inverse_reproduces_the_per_mode_coarse_solve():
    """The network's target, (h S_0(mu))^{-1} c, equals the coarse correction of the scalar oracle."""
    from oracle import mlp
    mu, Nt, nd = 1.7, 24, 4
    G = mlp.coarse_operator(mu, Nt, nd)
    pre = schwarz.SchurPreconditioner(np.array([[mu]]), Nt, nd, 1.0)
    r = workloads.random_vector(Nt, 5)
    c = pre.Z.T @ r
    np.testing.assert_allclose(pre.Z @ np.linalg.solve(G, c), pre.coarse(r), rtol=1e-12, atol=1e-12)


def test_mlp_forward_matches_hand_computed_network():
    """A 2-3-3-2 network with hand-picked weights, evaluated by hand:
    x = (1, 2): a1 = W1 x + b1 = (-1, 1, 2.5), h1 = (0, 1, 2.5); a2 = W2 h1 + b2 = (0.5, 3.5, -3),
    h2 = (0.5, 3.5, 0); y = W3 h2 + b3 = (7.5, -1.5).
    x = (-1, 0.5): a1 = (-1.5, -3, 1), h1 = (0, 0, 1); a2 = (0.5, 1, -2), h2 = (0.5, 1, 0);
    y = (2.5, -1.5).
    A dropped bias, a ReLU on the output or a transposed weight changes one of the outputs."""
    from oracle import mlp
    params = {"W1": np.array([[1.0, -1.0], [2.0, 0.0], [0.0, 1.0]]), "b1": np.array([0.0, -1.0, 0.5]),
              "W2": np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 1.0], [1.0, -1.0, 0.0]]), "b2": np.array([0.5, 0.0, -2.0]),
              "W3": np.array([[1.0, 2.0, 3.0], [-1.0, 0.0, 1.0]]), "b3": np.array([0.0, -1.0])}
    Y, _ = mlp.forward(params, np.array([[1.0, 2.0], [-1.0, 0.5]]))
    np.testing.assert_array_equal(Y, np.array([[7.5, -1.5], [2.5, -1.5]]))


def _coarse_batch(B=5, Nt=24, nd=4, seed=3):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    mus = 1.0 + rng.uniform(0.02, 3.0, B)
    G = [mlp.coarse_operator(float(m), Nt, nd) for m in mus]
    C = rng.standard_normal((B, 2 * nd))
    D = rng.standard_normal((B, 2 * nd))
    return G, C, D


def test_coarse_residual_loss_is_the_least_squares_residual():
    """Per sample, min over alpha of ||c - alpha G d|| from numpy's least squares, squared and
    divided by ||c||^2, averaged over the batch; and zero at the exact coarse solve d = G^-1 c."""
    from oracle import mlp
    G, C, D = _coarse_batch()
    want = 0.0
    for b in range(len(G)):
        g = (G[b] @ D[b])[:, None]
        _, res, _, _ = np.linalg.lstsq(g, C[b], rcond=None)
        want += float(res[0]) / float(C[b] @ C[b])
    loss, _ = mlp.coarse_residual_loss(D, C, G)
    np.testing.assert_allclose(loss, want / len(G), rtol=1e-12)
    exact = np.stack([3.7 * np.linalg.solve(G[b], C[b]) for b in range(len(G))])
    loss0, grad0 = mlp.coarse_residual_loss(exact, C, G)
    assert loss0 < 1e-24 and np.abs(grad0).max() < 1e-10


def test_coarse_residual_loss_gradient_matches_central_differences():
    from oracle import mlp
    G, C, D = _coarse_batch(seed=4)
    _, g = mlp.coarse_residual_loss(D, C, G)
    fd = np.zeros_like(D)
    for idx in np.ndindex(D.shape):
        old = D[idx]
        D[idx] = old + 1e-6
        lp, _ = mlp.coarse_residual_loss(D, C, G)
        D[idx] = old - 1e-6
        lm, _ = mlp.coarse_residual_loss(D, C, G)
        D[idx] = old
        fd[idx] = (lp - lm) / 2e-6
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_coarse_data_restriction_by_brute_force():
    """c = R_0 r for one mode's time series: per subdomain s with steps lo+1..hi (balanced split,
    left partition of unity), the sum of r_n and of r_n (-1 + 2 (n - lo) / (hi - lo)); x solves
    the coarse system."""
    from oracle import mlp
    Nt, nd = 30, 7
    rng = np.random.default_rng(8)
    r = rng.standard_normal((Nt, 3))
    mu = np.array([1.05, 1.6, 4.0])
    C, X = mlp.coarse_data(r, mu, Nt, nd)
    for b in range(3):
        for s in range(nd):
            lo, hi = s * Nt // nd, (s + 1) * Nt // nd
            c0 = sum(r[n - 1, b] for n in range(lo + 1, hi + 1))
            c1 = sum(r[n - 1, b] * (-1.0 + 2.0 * (n - lo) / (hi - lo)) for n in range(lo + 1, hi + 1))
            np.testing.assert_allclose(C[b, 2 * s], c0, rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(C[b, 2 * s + 1], c1, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(mlp.coarse_operator(mu[b], Nt, nd) @ X[b], C[b], rtol=1e-10, atol=1e-10)
