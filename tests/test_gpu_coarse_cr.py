"""The two coarse solvers (block Thomas, and the multilevel cyclic-reduction hierarchy in time)
against the FP64 oracle's exact coarse correction and against each other.

Both solve S_0 c' = R_0 r exactly, so both meet the FP64 bar of 1e-10 against the oracle's
sparse factorisation of Z^T S-hat Z (the literal definition). Cases cover one, two and
non-power-of-two numbers of subdomains (ragged levels), both D_s readings, the paper's five
steps per subdomain with many subdomains, and the largest N_D whose blocks fit in shared
memory. Above that size, and with the learned correction, the cyclic request falls back to
Thomas.
"""

import numpy as np
import pytest

import workloads
from oracle import problem, schwarz, spectral
from oracle.problem import HeatKKT

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


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
    # nx, ny, Nt, n_sub, omega, Lx, Ly
    (8, 8, 9, 1, 1e-3, 1.0, 1.0),        # one block: no level
    (8, 8, 8, 2, 1e-2, 1.0, 1.0),        # one level
    (12, 10, 30, 7, 1e-4, 1.0, 2.0),     # ragged levels (7 -> 4 -> 2 -> 1), anisotropic
    (16, 16, 65, 13, 1e-3, 1.0, 1.0),    # Nt not divisible by N_D
    (16, 16, 100, 20, 1e-4, 1.0, 2.0),   # the paper's 5 steps per subdomain, 17 x 17 points
    (8, 8, 330, 33, 1e-6, 1.0, 1.0),     # 2^5 + 1 blocks
]


@pytest.mark.parametrize("c", CASES)
@pytest.mark.parametrize("solver", ["cyclic", "thomas"])
@pytest.mark.parametrize("pou", ["left", "right"])
def test_coarse_solvers_match_oracle(kkt, c, solver, pou):
    nx, ny, Nt, nd, om, Lx, Ly = c
    if pou == "right" and Nt // nd < 3:
        pytest.skip("pou=right needs three steps in the first subdomain")
    p = HeatKKT(nx=nx, ny=ny, Nt=Nt, nu=1.0, omega=om, Lx=Lx, Ly=Ly)
    s = kkt.Solver(nx, ny, Nt, 1.0, 1.0, om, nd, pou=pou, Lx=Lx, Ly=Ly, coarse_solve=solver)
    pre = schwarz.schur_preconditioner(p, nd, pou=pou)
    r = workloads.random_vector(p.V, 31)
    assert rel(host(s.coarse_apply(dev(r))), pre.coarse(r)) < TOL
    # and inside the full two-level Schur preconditioner (the coarse solve feeds the sweeps)
    assert rel(host(s.schur_precond_apply(dev(r))), pre.apply(r)) < TOL
    s.close()


def test_cyclic_equals_thomas_at_many_subdomains(kkt):
    """640 subdomains of 5 steps (the paper's largest Nt with m = 5) on the 17 x 17 mesh, and
    1900 subdomains (the largest N_D whose 13 doubles per block fit in 200 KB of shared
    memory): the two solvers agree to rounding."""
    for nx, Nt, nd in ((16, 3200, 640), (8, 3800, 1900)):
        s = kkt.Solver(nx, nx, Nt, 1.0, 1.0, 1e-4, nd, coarse_solve="thomas")
        r = dev(workloads.random_vector(s.V, 5))
        a = host(s.coarse_apply(r))
        s.set_options(coarse_solve="cyclic")
        b = host(s.coarse_apply(r))
        assert rel(b, a) < 1e-12
        s.close()


def test_cyclic_request_falls_back_above_shared_memory(kkt):
    """2000 blocks need 208 KB per mode: the cyclic request runs block Thomas instead and
    still matches the exact solve."""
    nx, Nt, nd = 4, 4000, 2000
    s = kkt.Solver(nx, nx, Nt, 1.0, 1.0, 1e-4, nd, coarse_solve="cyclic")
    p = HeatKKT(nx=nx, ny=nx, Nt=Nt, nu=1.0, omega=1e-4)
    pre = schwarz.schur_preconditioner(p, nd)
    r = workloads.random_vector(p.V, 6)
    assert rel(host(s.coarse_apply(dev(r))), pre.coarse(r)) < TOL
    s.close()


@pytest.mark.parametrize("solver", ["cyclic", "thomas"])
def test_solves_with_either_coarse_solver_reach_the_exact_solution(kkt, solver):
    w = workloads.Workload("paper-like", nx=16, ny=16, Nt=200, n_sub=40, omega=1e-4)
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    f = problem.assemble_rhs(p, workloads.make_target(w), None)
    exact = spectral.kkt_exact_solve(p, f)
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, coarse_solve=solver)
    res = s.solve(dev(f), tol=1e-12, maxit=420)
    assert res.status == kkt.KKT_OK
    assert rel(host(res.x), exact) < TOL
    s.close()


def test_tensor_core_form_with_cyclic_coarse_solve(kkt):
    """The TF32 form's coarse solve takes FP32 coefficients; both solvers see the same sums,
    so their preconditioner outputs agree far below the form's own error."""
    nx, Nt, nd = 32, 160, 32
    s = kkt.Solver(nx, nx, Nt, 1.0, 1.0, 1e-4, nd, precision="tf32", coarse_solve="thomas")
    r = dev(workloads.random_vector(s.V, 8))
    a = host(s.schur_precond_apply(r))
    s.set_options(precision="tf32", coarse_solve="cyclic")
    b = host(s.schur_precond_apply(r))
    assert rel(b, a) < 1e-9
    s.close()


def test_invalid_coarse_solve_rejected(kkt):
    s = kkt.Solver(8, 8, 8, 1.0, 1.0, 1e-3, 2)
    opt = kkt.KKTOptions()
    import ctypes
    assert kkt.load_library().kkt_default_options(ctypes.byref(opt)) == 0
    opt.coarse_solve = 3
    with pytest.raises(kkt.KKTError):
        kkt.kkt_set_options(s.h, opt)
    s.close()


def test_fp64_after_a_mixed_form_keeps_its_cyclic_factors(kkt):
    """Switching a cyclic-coarse FP64 handle to TF32 and back re-derives the stored
    cyclic-reduction factors in memory the handle still owns: the Schur preconditioner then
    equals a fresh FP64 handle's."""
    nx, Nt, nd = 32, 128, 16
    r = dev(workloads.random_vector((nx - 1) ** 2 * Nt, 9))
    fresh = kkt.Solver(nx, nx, Nt, 1.0, 1.0, 1e-4, nd, coarse_solve="cyclic")
    want = host(fresh.schur_precond_apply(r))
    fresh.close()
    s = kkt.Solver(nx, nx, Nt, 1.0, 1.0, 1e-4, nd, coarse_solve="cyclic")
    s.set_options(precision="tf32", coarse_solve="cyclic")
    s.set_options(precision="fp64", coarse_solve="cyclic")
    assert rel(host(s.schur_precond_apply(r)), want) < 1e-12
    s.close()


def test_closed_handles_return_their_device_memory(kkt):
    """Twenty cyclic-coarse FP64 handles created and closed in turn leave the device's free
    memory where it was (each holds about 38 MB of stored factors at this size)."""
    def once():
        s = kkt.Solver(64, 64, 1024, 1.0, 1.0, 1e-4, 64, coarse_solve="cyclic")
        s.close()

    once()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        once()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 32 * 2**20, f"{(free0 - free1) / 2**20:.1f} MiB not returned"
