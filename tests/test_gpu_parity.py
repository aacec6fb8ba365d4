"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 tolerance: relative error 1e-10; every comparison below is a norm-wise relative error
||gpu - oracle|| / ||oracle|| against that bar (tighter where the arithmetic allows). Sizes
span several DST tiles and a ragged tail (31 x 31 lines in 32-line tiles, 255 columns in 8
tiles), odd and even sizes, non-power-of-two grids (direct transform), Nt not divisible by
N_D, both D_s readings and every composition variant.

Solves are compared where the comparison is well conditioned. An FGMRES iterate after a fixed
k at a stagnating step moves by 1e-6 when the preconditioner output is perturbed by 1e-14
(measured with the oracle), so iterates of two FP64 implementations cannot agree to 1e-10
there; the tests compare residual histories, and converged solutions against the exact
per-mode solve. The default residual norm is the discrete L2 pair (u, z rows weighted
h^-1/2, state rows h^1/2), in which the exact solution's relative residual is 1e-14; in the
unweighted Euclidean norm it is already 6.7e-10 at 32 x 32, Nt = 64, so Euclidean solves are
compared at 1e-8 only.
"""

import numpy as np
import pytest

import workloads
from oracle import krylov, problem, schwarz, spectral
from oracle.problem import HeatKKT

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def close(got, want, tol, n_slices):
    """Norm-wise relative error below tol, and element by element per time slice: each slice's
    largest error below tol times the larger of that slice's largest value and 1e-3 of the
    whole output's (so an error confined to a few small entries or slices cannot hide under
    the norm of the rest)."""
    got, want = np.asarray(got), np.asarray(want)
    assert rel(got, want) < tol
    g = got.reshape(n_slices, -1)
    w = want.reshape(n_slices, -1)
    err = np.abs(g - w).max(axis=1)
    scale = np.maximum(np.abs(w).max(axis=1), 1e-3 * np.abs(w).max())
    bad = np.nonzero(err > tol * scale)[0]
    assert bad.size == 0, f"slices {bad[:8]}: error {err[bad[:8]]}, scale {scale[bad[:8]]}"


@pytest.fixture(scope="module")
def kkt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_04421_gb300.kkt as k
    k.load_library()
    return k


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = [
    # nx, ny, Nt, n_sub, omega, nu, Lx, Ly
    (32, 32, 64, 4, 1e-4, 1.0, 1.0, 1.0),      # the small FP64 configuration
    (16, 8, 30, 4, 1e-2, 0.7, 1.0, 2.0),       # Nt not divisible by N_D, anisotropic
    (12, 20, 18, 3, 1e-3, 1.3, 1.0, 1.0),      # non-power-of-two grids (direct DST)
    (8, 8, 9, 1, 1e-3, 1.0, 1.0, 1.0),         # a single subdomain
    (4, 4, 4, 2, 1e-2, 1.0, 1.0, 1.0),         # two steps per subdomain (minimum)
    (64, 16, 40, 20, 1e-6, 2.0, 1.0, 1.0),     # many subdomains, small omega
]


def _problem(c):
    nx, ny, Nt, nd, om, nu, Lx, Ly = c
    return HeatKKT(nx=nx, ny=ny, Nt=Nt, nu=nu, omega=om, Lx=Lx, Ly=Ly), nd


def _solver(kkt, c, **opt):
    nx, ny, Nt, nd, om, nu, Lx, Ly = c
    if opt.get("pou") == "right" and Nt // nd < 3:
        with pytest.raises(kkt.KKTError):
            kkt.Solver(nx, ny, Nt, 1.0, nu, om, nd, Lx=Lx, Ly=Ly, **opt)
        pytest.skip("pou=right needs three steps in the first subdomain")
    return kkt.Solver(nx, ny, Nt, 1.0, nu, om, nd, Lx=Lx, Ly=Ly, **opt)


@pytest.mark.parametrize("c", CASES)
def test_dst2d_matches_scipy_dst(kkt, c):
    p, _ = _problem(c)
    s = _solver(kkt, c)
    x = workloads.random_vector(p.V, 3)
    got = host(s.dst2d(dev(x)))
    want = spectral.dst2(x, p).ravel()
    close(got, want, 1e-13, p.Nt)
    # involution: applying it twice gives the input back; in-place call allowed
    t = dev(x)
    s.dst2d(t, out=t)
    s.dst2d(t, out=t)
    assert rel(host(t), x) < 1e-13


@pytest.mark.parametrize("c", [c for c in CASES if max(c[0], c[1]) <= 32] + [(16, 16, 200, 40, 1e-4, 1.0, 1.0, 2.0)])
@pytest.mark.parametrize("method", ["tiles", "lane"])
def test_dst_methods_match_scipy_dst(kkt, c, method):
    """Both FP64 transform methods on grids with at most 31 points per direction (power-of-two
    and other interval counts, rows and columns, in place), and a preconditioner apply with each
    against the oracle."""
    p, nd = _problem(c)
    s = _solver(kkt, c)
    s.set_dst_method(method)
    x = workloads.random_vector(p.V, 13)
    assert rel(host(s.dst2d(dev(x))), spectral.dst2(x, p).ravel()) < 1e-13
    t = dev(x)
    s.dst2d(t, out=t)
    s.dst2d(t, out=t)
    assert rel(host(t), x) < 1e-13
    pre = schwarz.schur_preconditioner(p, nd)
    assert rel(host(s.schur_precond_apply(dev(x))), pre.apply(x)) < TOL


def test_lane_dst_refused_for_long_lines(kkt):
    s = kkt.Solver(64, 16, 8, 1.0, 1.0, 1e-3, 2)
    with pytest.raises(kkt.KKTError):
        s.set_dst_method("lane")
    s.set_dst_method("tiles")
    s.set_dst_method("auto")
    s.close()


@pytest.mark.parametrize("c", CASES)
def test_matvec_matches_sparse_kkt(kkt, c):
    p, _ = _problem(c)
    s = _solver(kkt, c)
    x = workloads.random_vector(3 * p.V, 5)
    got = host(s.matvec(dev(x)))
    close(got, problem.assemble_K(p) @ x, 1e-13, 3 * p.Nt)


@pytest.mark.parametrize("c", CASES)
def test_schur_apply_matches_oracle(kkt, c):
    p, nd = _problem(c)
    s = _solver(kkt, c)
    pre = schwarz.schur_preconditioner(p, nd, variant="one-level")
    x = workloads.random_vector(p.V, 6)
    close(host(s.schur_apply(dev(x))), pre.schur_apply(x), 1e-12, p.Nt)


@pytest.mark.parametrize("c", CASES)
@pytest.mark.parametrize("pou", ["left", "right"])
def test_coarse_correction_matches_oracle(kkt, c, pou):
    p, nd = _problem(c)
    s = _solver(kkt, c, pou=pou)
    pre = schwarz.schur_preconditioner(p, nd, pou=pou)
    r = workloads.random_vector(p.V, 7)
    close(host(s.coarse_apply(dev(r))), pre.coarse(r), TOL, p.Nt)


@pytest.mark.parametrize("c", CASES)
@pytest.mark.parametrize("variant,coarse", [("multiplicative", "exact"), ("additive", "exact"),
                                            ("multiplicative", "none")])
@pytest.mark.parametrize("pou", ["left", "right"])
def test_schur_preconditioner_matches_oracle(kkt, c, variant, coarse, pou):
    p, nd = _problem(c)
    s = _solver(kkt, c, variant=variant, coarse=coarse, pou=pou)
    ov = "one-level" if coarse == "none" else variant
    pre = schwarz.schur_preconditioner(p, nd, variant=ov, pou=pou)
    r = workloads.random_vector(p.V, 8)
    close(host(s.schur_precond_apply(dev(r))), pre.apply(r), TOL, p.Nt)


@pytest.mark.parametrize("c", CASES)
@pytest.mark.parametrize("coarse", ["none", "exact"])
@pytest.mark.parametrize("pou", ["left", "right"])
def test_ras_local_solves_match_oracle(kkt, c, coarse, pou):
    """RAS (Eq 9): the tridiagonal local Schur solves per mode, alone and inside the
    coarse-first composition, against the oracle's sparse local Schur matrices."""
    p, nd = _problem(c)
    s = _solver(kkt, c, coarse=coarse, pou=pou, local="ras")
    pre = schwarz.schur_preconditioner(p, nd, variant="ras" if coarse == "none" else "ras-multiplicative", pou=pou)
    r = workloads.random_vector(p.V, 18)
    close(host(s.schur_precond_apply(dev(r))), pre.apply(r), TOL, p.Nt)


def test_ras_local_solves_in_fp64_solves_and_tensor_core_forms(kkt):
    """A 1e-8 solve with RAS locals reaches the exact solution, and the TF32 form runs them too."""
    w = workloads.CFG_SMALL
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    f = problem.assemble_rhs(p, workloads.make_target(w), None)
    exact = spectral.kkt_exact_solve(p, f)
    for prec in ("fp64", "tf32"):
        s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, local="ras", precision=prec)
        res = s.solve(dev(f), tol=1e-12 if prec == "fp64" else 1e-8, maxit=420)
        assert res.status == kkt.KKT_OK
        assert rel(host(res.x), exact) < (TOL if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("c", CASES[:3])
def test_block_preconditioner_matches_oracle(kkt, c):
    p, nd = _problem(c)
    s = _solver(kkt, c)
    pre = schwarz.schur_preconditioner(p, nd)
    r = workloads.random_vector(3 * p.V, 9)
    close(host(s.precond_apply(dev(r))), schwarz.block_preconditioner_apply(p, pre, r), TOL, 3 * p.Nt)


def test_literal_sign_option_matches_oracle(kkt):
    c = (16, 16, 32, 4, 1e-2, 1.0, 1.0, 1.0)
    p, nd = _problem(c)
    s = _solver(kkt, c, jhat_sign=+1)
    pre = schwarz.schur_preconditioner(p, nd, jhat_sign=+1)
    r = workloads.random_vector(p.V, 10)
    assert rel(host(s.schur_precond_apply(dev(r))), pre.apply(r)) < 1e-8


def test_build_rhs_matches_oracle_device_and_host(kkt):
    w = workloads.CFG_SMALL
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub)
    ut = workloads.make_target(w).ravel()
    u0 = workloads.random_vector(p.N, 2)
    want = problem.assemble_rhs(p, ut, u0)
    assert rel(host(s.build_rhs(dev(ut), dev(u0))), want) < 1e-15
    f_host = torch.empty(3 * p.V, dtype=torch.float64)
    s.build_rhs(torch.from_numpy(ut), torch.from_numpy(u0), out=f_host)
    assert rel(f_host.numpy(), want) < 1e-15


@pytest.mark.parametrize("norm", ["l2", "euclidean"])
def test_solve_small_configuration_matches_oracle_and_exact(kkt, norm):
    """The 32 x 32, Nt = 64, N_D = 4 problem to 1e-8: GPU FGMRES reaches the tolerance in the
    oracle's iteration count (same residual norm); in the L2 norm a 1e-12 solve equals the
    per-mode exact solve within 1e-10, in the Euclidean norm the iterate after 60 steps does."""
    w = workloads.CFG_SMALL
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    f = problem.assemble_rhs(p, workloads.make_target(w), workloads.make_u0(w))
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, residual_norm=norm)
    d = problem.l2_residual_weights(p) if norm == "l2" else np.ones(3 * p.V)
    res = s.solve(dev(f), tol=1e-8, maxit=420)
    assert res.status == kkt.KKT_OK and res.rel_residual <= 1e-8
    K = problem.assemble_K(p)
    x = host(res.x)
    assert np.linalg.norm(d * (f - K @ x)) / np.linalg.norm(d * f) <= 1.01e-8
    # the Euclidean relative residual itself carries a rounding floor of about 7e-10 here
    np.testing.assert_allclose(res.rel_residual_euclid, np.linalg.norm(f - K @ x) / np.linalg.norm(f),
                               rtol=1e-6, atol=2e-9)
    pre = schwarz.schur_preconditioner(p, w.n_sub)
    ref = krylov.fgmres(lambda v: K @ v, lambda r: schwarz.block_preconditioner_apply(p, pre, r), f,
                        tol=1e-8, restart=30, maxit=420, row_scale=d)
    assert abs(res.iterations - ref.iterations) <= 1
    exact = spectral.kkt_exact_solve(p, f)
    if norm == "l2":
        tight = s.solve(dev(f), tol=1e-12, maxit=420)
        assert tight.status == kkt.KKT_OK
    else:
        tight = s.solve(dev(f), tol=1e-14, maxit=60)
        assert tight.status == kkt.KKT_NOT_CONVERGED and tight.iterations == 60
    assert rel(host(tight.x), exact) < TOL


@pytest.mark.parametrize("orth", ["mgs", "cgs2", "mgs2", "mgs4", "mgs8"])
@pytest.mark.parametrize("k", [1, 5, 12, 30])
def test_fixed_iteration_residuals_match_oracle(kkt, k, orth):
    """After the same k Arnoldi steps (one cycle), GPU and oracle agree on every residual
    estimate and on the true residual of the iterate, with either orthogonalisation (the
    oracle uses MGS; CGS2 differs from it by rounding only)."""
    w = workloads.CFG_SMALL
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    f = problem.assemble_rhs(p, workloads.make_target(w), None)
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, orth=orth)
    res = s.solve(dev(f), tol=1e-300, maxit=k)
    assert res.status == kkt.KKT_NOT_CONVERGED and res.iterations == k
    K = problem.assemble_K(p)
    d = problem.l2_residual_weights(p)
    pre = schwarz.schur_preconditioner(p, w.n_sub)
    ref = krylov.fgmres(lambda v: K @ v, lambda r: schwarz.block_preconditioner_apply(p, pre, r), f,
                        fixed_iterations=k, row_scale=d)
    np.testing.assert_allclose(res.history, ref.history, rtol=1e-7, atol=1e-13)
    x = host(res.x)
    np.testing.assert_allclose(np.linalg.norm(d * (f - K @ x)) / np.linalg.norm(d * f), ref.rel_residual,
                               rtol=1e-6, atol=1e-13)
    if k == 1:
        assert rel(x, ref.x) < TOL       # one step: x = y_1 z_1, well conditioned


@pytest.mark.parametrize("orth", ["mgs", "cgs2", "mgs2", "mgs4", "mgs8"])
def test_spectral_basis_solve_matches_oracle(kkt, orth):
    """FGMRES on sine-mode coefficients (transforms only at entry and exit): the same residual
    history as the oracle's physical-space FGMRES after 12 steps, the oracle's iteration count
    to 1e-8, and the exact solution after a 1e-12 solve, from a nonzero initial guess and with
    host buffers."""
    w = workloads.CFG_SMALL
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    f = problem.assemble_rhs(p, workloads.make_target(w), workloads.make_u0(w))
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, orth=orth, basis="spectral")
    K = problem.assemble_K(p)
    d = problem.l2_residual_weights(p)
    pre = schwarz.schur_preconditioner(p, w.n_sub)
    ref = krylov.fgmres(lambda v: K @ v, lambda r: schwarz.block_preconditioner_apply(p, pre, r), f,
                        fixed_iterations=12, row_scale=d)
    res = s.solve(dev(f), tol=1e-300, maxit=12)
    assert res.status == kkt.KKT_NOT_CONVERGED and res.iterations == 12
    np.testing.assert_allclose(res.history, ref.history, rtol=1e-7, atol=1e-13)
    x = host(res.x)
    np.testing.assert_allclose(np.linalg.norm(d * (f - K @ x)) / np.linalg.norm(d * f), ref.rel_residual,
                               rtol=1e-6, atol=1e-13)
    full = krylov.fgmres(lambda v: K @ v, lambda r: schwarz.block_preconditioner_apply(p, pre, r), f,
                         tol=1e-8, restart=30, maxit=420, row_scale=d)
    res = s.solve(dev(f), tol=1e-8, maxit=420)
    assert res.status == kkt.KKT_OK and abs(res.iterations - full.iterations) <= 1
    exact = spectral.kkt_exact_solve(p, f)
    x0 = torch.from_numpy(0.5 * exact + workloads.random_vector(3 * p.V, 3) * 1e-3)   # host, nonzero
    tight = s.solve(torch.from_numpy(f), x0, tol=1e-12, maxit=420)
    assert tight.status == kkt.KKT_OK
    assert rel(x0.numpy(), exact) < TOL


@pytest.mark.parametrize("orth", ["mgs", "cgs2", "mgs2", "mgs4", "mgs8"])
def test_restarted_fgmres_matches_oracle(kkt, orth):
    """FGMRES(5): several restart cycles; the oracle's FGMRES(5) takes the same iteration count
    within 1, and a 1e-12 solve reaches the exact solution."""
    w = workloads.CFG_SMALL
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    f = problem.assemble_rhs(p, workloads.make_target(w), None)
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, restart=5, orth=orth)
    K = problem.assemble_K(p)
    pre = schwarz.schur_preconditioner(p, w.n_sub)
    ref = krylov.fgmres(lambda v: K @ v, lambda r: schwarz.block_preconditioner_apply(p, pre, r), f,
                        tol=1e-8, restart=5, maxit=420, row_scale=problem.l2_residual_weights(p))
    res = s.solve(dev(f), tol=1e-8, maxit=420)
    assert res.status == kkt.KKT_OK and res.restarts >= 3
    assert abs(res.iterations - ref.iterations) <= 1, (res.iterations, ref.iterations)
    tight = s.solve(dev(f), tol=1e-12, maxit=600)
    assert tight.status == kkt.KKT_OK
    assert rel(host(tight.x), spectral.kkt_exact_solve(p, f)) < TOL


def test_spectral_basis_rejects_reduced_precision(kkt):
    with pytest.raises(kkt.KKTError) as e:
        kkt.Solver(32, 32, 64, 1.0, 1.0, 1e-4, 4, precision="tf32", basis="spectral")
    assert e.value.status == kkt.KKT_ERR_UNSUPPORTED


def test_solve_with_host_buffers_and_initial_guess(kkt):
    w = workloads.Workload("t", nx=16, ny=16, Nt=24, n_sub=3, omega=1e-3, seed=4)
    p = HeatKKT(nx=16, ny=16, Nt=24, omega=1e-3)
    f = problem.assemble_rhs(p, workloads.make_target(w), None)
    s = kkt.Solver(16, 16, 24, 1.0, 1.0, 1e-3, 3)
    exact = spectral.kkt_exact_solve(p, f)
    x = torch.zeros(3 * p.V, dtype=torch.float64)          # host tensor
    res = s.solve(torch.from_numpy(f), x, tol=1e-12, maxit=300)
    assert res.status == kkt.KKT_OK
    assert rel(x.numpy(), exact) < TOL
    # starting from the solution: converged at once
    res2 = s.solve(dev(f), dev(exact), tol=1e-8, maxit=10)
    assert res2.status == kkt.KKT_OK and res2.iterations == 0


def test_host_staging_modes_give_identical_solves(kkt):
    """Host vectors reach the device by the copy kernel (pinned buffers, 16-byte aligned or
    not) or by cudaMemcpyAsync (pageable buffers, or the copy-engine mode): the solve and the
    returned x are bit-identical to a device-memory solve. 3V is odd here (15 x 15 x 3 points),
    so the vector copy has a scalar tail."""
    w = workloads.Workload("t", nx=16, ny=16, Nt=3, n_sub=1, omega=1e-3, seed=6)
    p = HeatKKT(nx=16, ny=16, Nt=3, omega=1e-3)
    f = problem.assemble_rhs(p, workloads.make_target(w), None)
    n = 3 * p.V
    assert n % 2 == 1
    x0 = workloads.random_vector(n, 9) * 1e-3
    s = kkt.Solver(16, 16, 3, 1.0, 1.0, 1e-3, 1)
    ref = s.solve(dev(f), dev(x0), tol=1e-10, maxit=100)
    big_f = torch.zeros(n + 1, dtype=torch.float64).pin_memory()
    big_x = torch.zeros(n + 1, dtype=torch.float64).pin_memory()
    layouts = {"pinned": (torch.from_numpy(f).pin_memory(), lambda: torch.from_numpy(x0.copy()).pin_memory()),
               "pinned+8B": (big_f[1:].copy_(torch.from_numpy(f)), lambda: big_x[1:].copy_(torch.from_numpy(x0))),
               "pageable": (torch.from_numpy(f.copy()), lambda: torch.from_numpy(x0.copy()))}
    for mode in ("auto", "copy_engine"):
        s.set_staging(mode)
        for name, (fh, make_x) in layouts.items():
            xh = make_x()
            res = s.solve(fh, xh, tol=1e-10, maxit=100)
            assert res.status == kkt.KKT_OK and res.iterations == ref.iterations, (mode, name)
            assert np.array_equal(xh.numpy(), host(ref.x)), (mode, name)
    with pytest.raises(kkt.KKTError):
        kkt.kkt_set_staging(s.h, 2)
    s.close()


def test_zero_guess_solve_ignores_the_contents_of_x(kkt):
    """kkt_solve_zero_guess starts from 0 whatever x holds (NaN here), for host and device x,
    and takes the same steps as kkt_solve from a zeroed x."""
    w = workloads.Workload("t", nx=16, ny=16, Nt=24, n_sub=3, omega=1e-3, seed=5)
    p = HeatKKT(nx=16, ny=16, Nt=24, omega=1e-3)
    f = problem.assemble_rhs(p, workloads.make_target(w), None)
    s = kkt.Solver(16, 16, 24, 1.0, 1.0, 1e-3, 3)
    ref = s.solve(dev(f), dev(np.zeros(3 * p.V)), tol=1e-10, maxit=300)
    for x in (torch.full((3 * p.V,), float("nan"), dtype=torch.float64),
              torch.full((3 * p.V,), float("nan"), dtype=torch.float64, device="cuda")):
        res = s.solve(dev(f) if x.is_cuda else torch.from_numpy(f), x, tol=1e-10, maxit=300, zero_guess=True)
        assert res.status == kkt.KKT_OK and res.iterations == ref.iterations
        assert np.array_equal(host(x) if x.is_cuda else x.numpy(), host(ref.x))


def test_full_size_preconditioner_on_sampled_modes(kkt):
    """256 x 256, Nt = 1024, N_D = 64 (the benchmark size): an input living on a few sine modes
    is mapped mode by mode; each mode's time series must equal the scalar oracle's."""
    w = workloads.CFG_GPU
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    modes = [(1, 1), (3, 7), (200, 5), (255, 255)]
    blk, coeff = workloads.random_mode_block(w, modes, seed=17)
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub)
    y = s.schur_precond_apply(dev(blk.ravel()))
    yhat = host(s.dst2d(y)).reshape(w.Nt, w.ny - 1, w.nx - 1)
    mu = spectral.jhat_mode_diagonal(p)
    # the orthonormal DST of the sampled mode sin(k pi x) sin(l pi y) is its norm in slot (l, k)
    norm = np.sqrt((w.nx / 2.0) * (w.ny / 2.0))
    wants, gots = [], []
    for q, (k, l) in enumerate(modes):
        scal = schwarz.SchurPreconditioner(np.array([[mu[l - 1, k - 1]]]), w.Nt, w.n_sub, p.h)
        wants.append(scal.apply(coeff[:, q]))
        gots.append(yhat[:, l - 1, k - 1] / norm)
    # rounding of the transforms is relative to the whole output, whose norm the lowest mode sets
    total = np.sqrt(sum(np.linalg.norm(v) ** 2 for v in wants))
    for got, want in zip(gots, wants):
        assert np.linalg.norm(got - want) / total < TOL
    assert rel(gots[0], wants[0]) < TOL
    # everything else stays zero up to rounding
    mask = np.ones((w.ny - 1, w.nx - 1), bool)
    for (k, l) in modes:
        mask[l - 1, k - 1] = False
    assert np.linalg.norm(yhat[:, mask]) / norm < TOL * total


def test_full_size_matvec_sampled_points(kkt):
    w = workloads.CFG_GPU
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub)
    x = torch.randn(3 * p.V, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    y = s.matvec(x)
    xs = x.view(3, p.Nt, p.My, p.Mx)
    ys = host(y).reshape(3, p.Nt, p.My, p.Mx)
    rng = np.random.default_rng(1)
    for _ in range(40):
        n, j, i = int(rng.integers(p.Nt)), int(rng.integers(p.My)), int(rng.integers(p.Mx))
        # the oracle's blockwise matvec on the 3 neighbouring time slices around n
        lo, hi = max(n - 1, 0), min(n + 2, p.Nt)
        sub = HeatKKT(nx=w.nx, ny=w.ny, Nt=hi - lo, nu=w.nu, omega=w.omega, T=p.dt * (hi - lo))
        xw = host(xs[:, lo:hi].reshape(-1))
        yw = problem.kkt_apply_blockwise(sub, xw).reshape(3, hi - lo, p.My, p.Mx)
        t = n - lo
        # the window cuts the couplings at its ends: u^{lo-1} and w^{hi} are added back
        want = yw[:, t, j, i].copy()
        if t == 0 and lo > 0:
            want[2] -= float(xs[0, lo - 1, j, i])
        if t == hi - lo - 1 and hi < p.Nt:
            want[0] -= float(xs[2, hi, j, i])
        np.testing.assert_allclose(ys[:, n, j, i], want, rtol=1e-12, atol=1e-9)


def test_invalid_arguments_raise(kkt):
    with pytest.raises(kkt.KKTError):
        kkt.Solver(1, 8, 8, 1.0, 1.0, 1e-3, 2)
    with pytest.raises(kkt.KKTError):
        kkt.Solver(8, 8, 8, 1.0, 1.0, 1e-3, 5)     # Nt / n_sub < 2
    with pytest.raises(kkt.KKTError):
        kkt.Solver(8, 8, 8, 1.0, -1.0, 1e-3, 2)
    s = kkt.Solver(8, 8, 8, 1.0, 1.0, 1e-3, 2)
    with pytest.raises(kkt.KKTError):
        s.set_options(restart=0)
    bad = torch.full((3 * s.V,), float("nan"), dtype=torch.float64, device="cuda")
    with pytest.raises(kkt.KKTError) as ei:
        s.solve(bad)
    assert ei.value.status == kkt.KKT_ERR_NONFINITE
    with pytest.raises(kkt.KKTError):
        s.matvec(torch.zeros(3 * s.V, dtype=torch.float64))   # host pointer where device is required


@pytest.mark.parametrize("count,n", [(1, 1), (5, 1000), (17, 123457), (32, 300001)])
def test_multidot_matches_numpy(kkt, count, n):
    """The Gram-Schmidt multi-dot (FP64, deterministic) against numpy dots; repeated calls are
    bit-identical."""
    s = kkt.Solver(8, 8, 8, 1.0, 1.0, 1e-3, 2)
    stride = n + 3
    rng = np.random.default_rng(count)
    V = rng.standard_normal(count * stride)
    w = rng.standard_normal(n)
    out = torch.empty(count + 1, dtype=torch.float64, device="cuda")
    Vd, wd = dev(V), dev(w)
    kkt.kkt_multidot(s.h, Vd, stride, count, wd, n, out)
    got = host(out)
    want = np.array([np.dot(V[k * stride:k * stride + n], w) for k in range(count)] + [np.dot(w, w)])
    scale = np.sqrt(np.sum(V.reshape(count, stride)[:, :n] ** 2, axis=1).tolist() + [np.dot(w, w)]) * np.sqrt(np.dot(w, w))
    assert np.all(np.abs(got - want) <= 1e-13 * scale)
    out2 = torch.empty_like(out)
    kkt.kkt_multidot(s.h, Vd, stride, count, wd, n, out2)
    assert torch.equal(out, out2)
