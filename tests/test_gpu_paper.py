"""Section 4's experiment on the GPU against the FP64 oracle, cell by cell.

The problem is Eq 16: Omega = (0,1) x (0,2), T = 1, nu = 1, u_0 = -x y (x-1)(y-2),
u~ = sin 2 pi t sin 2 pi x sin 2 pi y, 17 x 17 mesh points (15 x 15 unknowns), right-preconditioned
FGMRES(30) to a 1e-6 relative residual (the unweighted Euclidean norm, as the paper states it),
at most 420 iterations. Each cell (Nt, m steps per subdomain, omega) is solved one-level (RASQ
alone) and two-level (coarse first, Eq 15), the two-level one with both coarse solvers (block
Thomas, and the cyclic-reduction hierarchy in time). The GPU's iteration counts must equal the
oracle's within one: the two FGMRES implementations differ only in rounding (the GPU pairs
its modified Gram-Schmidt steps), which can move the step at which the 1e-6 test first passes.

The paper's figures are missing from its source, so the counts themselves are not pinned to
printed values; the trends they show (two-level flat, one-level growing with the subdomain
count) are pinned on the oracle by tests/test_oracle_pins.py.
"""

import numpy as np
import pytest

import workloads
from oracle import krylov, problem, schwarz
from oracle.problem import HeatKKT

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kkt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_04421_gb300.kkt as k
    k.load_library()
    return k


CELLS = [(Nt, m, omega) for Nt in (100, 200) for m in (20, 5) for omega in (1e-2, 1e-4)]


def _paper_problem(Nt, n_sub, omega):
    w = workloads.Workload("paper", nx=16, ny=16, Nt=Nt, n_sub=n_sub, Lx=1.0, Ly=2.0, omega=omega,
                           target="paper", u0="paper")
    p = HeatKKT(nx=16, ny=16, Nt=Nt, nu=1.0, omega=omega, Lx=1.0, Ly=2.0)
    f = problem.assemble_rhs(p, workloads.make_target(w), workloads.make_u0(w))
    return w, p, f


@pytest.mark.parametrize("Nt,m,omega", CELLS)
def test_section4_iteration_counts_match_oracle(kkt, Nt, m, omega):
    nd = max(1, round(Nt / m))
    w, p, f = _paper_problem(Nt, nd, omega)
    K = problem.assemble_K(p)
    fd = torch.from_numpy(f).cuda()
    # the GPU's own right-hand side of Eq 16 equals the oracle's
    s0 = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, Lx=1.0, Ly=2.0)
    fg = s0.build_rhs(torch.from_numpy(workloads.make_target(w).ravel()).cuda(),
                      torch.from_numpy(workloads.make_u0(w).ravel()).cuda())
    np.testing.assert_allclose(fg.cpu().numpy(), f, rtol=1e-14, atol=1e-300)
    s0.close()
    counts = {}
    for level, coarse, variant in (("one", "none", "one-level"), ("two", "exact", "multiplicative")):
        pre = schwarz.schur_preconditioner(p, nd, variant=variant)
        ref = krylov.fgmres(lambda v: K @ v, lambda r: schwarz.block_preconditioner_apply(p, pre, r), f,
                            tol=1e-6, restart=30, maxit=420)
        assert ref.converged, (level, ref.iterations)
        solvers = ("thomas", "cyclic") if coarse == "exact" else ("auto",)
        for cs in solvers:
            s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, coarse=coarse, residual_norm="euclidean",
                           Lx=1.0, Ly=2.0, coarse_solve=cs)
            res = s.solve(fd, tol=1e-6, maxit=420)
            s.close()
            assert res.status == kkt.KKT_OK, (level, cs)
            assert abs(res.iterations - ref.iterations) <= 1, (level, cs, res.iterations, ref.iterations)
            counts[(level, cs)] = res.iterations
        counts[(level, "oracle")] = ref.iterations
    # the paper's claim on these cells: the coarse level never needs more iterations than RASQ
    # alone beyond rounding, and it needs fewer once there are many subdomains
    assert counts[("two", "oracle")] <= counts[("one", "oracle")] + 1
    if nd >= 20:
        assert counts[("two", "oracle")] < counts[("one", "oracle")]
