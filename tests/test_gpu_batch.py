"""Batched form: many uneven KKT instances solved together (waves, lockstep FGMRES, one launch
per phase over all instances, CUDA-graph replay of the preconditioner + matvec phase).

Each instance must behave exactly as its own kkt_solve up to rounding order: the same
iteration count (+-1) and a solution that matches the oracle's exact solve (Eq 5 diagonalised
by the sine transform) at the tight tolerance.
"""

import numpy as np
import pytest

import workloads
from oracle import problem, spectral
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


# uneven sizes: powers of two and not, non-square grids, short and long subdomains, and a spread
# of nu and omega (several tiles of every batched kernel, ragged tails in each)
SMALL = [
    workloads.Workload("b0", nx=32, ny=32, Nt=64, n_sub=4, nu=1.0, omega=1e-4, target="sine-series", seed=11),
    workloads.Workload("b1", nx=64, ny=64, Nt=128, n_sub=8, nu=0.3, omega=1e-3, target="sine-series", seed=12),
    workloads.Workload("b2", nx=48, ny=40, Nt=96, n_sub=6, nu=2.0, omega=1e-5, target="cos-mode-noise", seed=13),
    workloads.Workload("b3", nx=32, ny=64, Nt=64, n_sub=16, nu=0.1, omega=1e-2, target="sine-series", seed=14),
    workloads.Workload("b4", nx=16, ny=16, Nt=24, n_sub=3, nu=1.0, omega=1e-3, target="cos-mode-noise", seed=15),
    workloads.Workload("b5", nx=128, ny=128, Nt=32, n_sub=8, nu=5.0, omega=1e-6, target="sine-series", seed=16),
]


def rhs(w):
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    return p, problem.assemble_rhs(p, workloads.make_target(w), None)


@pytest.fixture(scope="module")
def small_case(kkt):
    ps, fs = zip(*[rhs(w) for w in SMALL])
    return list(ps), [dev(f) for f in fs]


def single(kkt, w, f, tol, coarse="exact", orth="mgs", basis="physical"):
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, coarse=coarse, orth=orth, basis=basis)
    r = s.solve(f, tol=tol, maxit=420)
    s.close()
    return r


@pytest.mark.parametrize("coarse,orth,basis", [("exact", "mgs", "physical"), ("none", "mgs", "physical"),
                                               ("exact", "cgs2", "physical"), ("exact", "mgs", "spectral"),
                                               ("exact", "mgs2", "physical"), ("none", "mgs2", "spectral")])
def test_batch_matches_single_instance_solves(kkt, small_case, coarse, orth, basis):
    ps, fs = small_case
    b = kkt.Batch(SMALL, coarse=coarse, orth=orth, basis=basis)
    b.set_single_threshold(0)          # every instance through the batched kernels
    res = b.solve(fs, tol=1e-8, maxit=420)
    assert res.status == kkt.KKT_OK
    for i, w in enumerate(SMALL):
        ref = single(kkt, w, fs[i], 1e-8, coarse, orth, basis)
        assert res.statuses[i] == kkt.KKT_OK
        assert abs(res.iterations[i] - ref.iterations) <= 1, (w.name, res.iterations[i], ref.iterations)
        assert res.rel_residual[i] <= 1e-8
        assert rel(host(res.xs[i]), host(ref.x)) < 1e-5
    # graphs: one per step index taken while every instance of the wave was running (later
    # steps run only the instances still iterating, launched directly)
    assert res.waves == 1
    assert 1 <= res.graphs <= min(min(res.iterations), 30)
    assert res.graph_launches >= res.graphs
    assert res.tile_lines in (8, 16, 32) and res.sweep_block in (64, 128, 256)


@pytest.mark.parametrize("basis", ["physical", "spectral"])
def test_batch_tight_solutions_match_the_oracle(kkt, small_case, basis):
    ps, fs = small_case
    b = kkt.Batch(SMALL, basis=basis)
    res = b.solve(fs, tol=1e-12, maxit=420)
    assert res.status == kkt.KKT_OK
    for i in range(len(SMALL)):
        exact = spectral.kkt_exact_solve(ps[i], host(fs[i]))
        assert rel(host(res.xs[i]), exact) < TOL, SMALL[i].name


# the paper's mesh (15 x 15 interior points) with 5 steps per subdomain: the batched waves run the
# cyclic-reduction coarse solve for these instances (and Thomas when told to)
PAPER_LIKE = [workloads.Workload(f"p{Nt}", nx=16, ny=16, Nt=Nt, n_sub=Nt // 5, omega=om, target="sine-series",
                                 seed=30 + q)
              for q, (Nt, om) in enumerate([(100, 1e-2), (400, 1e-4), (1600, 1e-3), (3200, 1e-4)])]


def test_batch_cyclic_coarse_solve_on_paper_like_instances(kkt):
    ps, fs = zip(*[rhs(w) for w in PAPER_LIKE])
    fs = [dev(f) for f in fs]
    out = {}
    for solver in ("auto", "thomas"):
        b = kkt.Batch(PAPER_LIKE, coarse_solve=solver)
        b.set_single_threshold(0)
        out[solver] = b.solve(fs, tol=1e-12, maxit=420)
        assert out[solver].status == kkt.KKT_OK
        b.close()
    for i, w in enumerate(PAPER_LIKE):
        assert out["auto"].iterations[i] == out["thomas"].iterations[i], w.name
        exact = spectral.kkt_exact_solve(ps[i], host(fs[i]))
        assert rel(host(out["auto"].xs[i]), exact) < TOL, w.name
        assert rel(host(out["thomas"].xs[i]), exact) < TOL, w.name


def test_batch_waves_give_the_same_results(kkt, small_case):
    ps, fs = small_case
    one = kkt.Batch(SMALL).solve(fs, tol=1e-8, maxit=420)
    b = kkt.Batch(SMALL)
    # the largest instance's storage: several waves, first-fit by decreasing size
    biggest = max(4 * (31 * 3 + 30) * 2 * w.V for w in SMALL)
    b.set_memory_limit(biggest)
    many = b.solve(fs, tol=1e-8, maxit=420)
    assert many.waves > 1
    assert many.status == kkt.KKT_OK
    for i in range(len(SMALL)):
        assert many.iterations[i] == one.iterations[i]
        assert rel(host(many.xs[i]), host(one.xs[i])) < 1e-12
    b.set_memory_limit(1 << 20)            # smaller than any instance: refused, nothing launched
    with pytest.raises(kkt.KKTError) as e:
        b.solve(fs, tol=1e-8, maxit=420)
    assert e.value.status == kkt.KKT_ERR_OOM


def test_batch_initial_guess_zero_rhs_and_maxit(kkt, small_case):
    ps, fs = small_case
    b = kkt.Batch(SMALL[:3])
    # the first instance starts from its exact solution, the second has f = 0
    exact0 = dev(spectral.kkt_exact_solve(ps[0], host(fs[0])))
    f1 = torch.zeros_like(fs[1])
    xs = [exact0.clone(), torch.zeros_like(f1), torch.zeros_like(fs[2])]
    res = b.solve([fs[0], f1, fs[2]], xs, tol=1e-8, maxit=420)
    assert res.statuses[0] == kkt.KKT_OK and res.iterations[0] == 0
    assert res.statuses[1] == kkt.KKT_OK and res.iterations[1] == 0
    assert float(host(res.xs[1]).__abs__().max()) == 0.0
    assert res.statuses[2] == kkt.KKT_OK and res.iterations[2] > 0
    # maxit: every instance stops at exactly 3 steps
    res = b.solve(fs[:3], tol=1e-14, maxit=3)
    assert res.status == kkt.KKT_NOT_CONVERGED
    assert res.iterations == [3, 3, 3]


def test_batch_rejects_unsupported_options(kkt):
    opt = kkt.KKTOptions()
    kkt.load_library().kkt_default_options(opt)
    opt.precision = kkt.PREC["bf16"]
    with pytest.raises(kkt.KKTError):
        kkt.kkt_batch_create([(32, 32, 64, 4, 1.0, 1.0, 1e-4)], opt)
    with pytest.raises(kkt.KKTError):
        kkt.kkt_batch_create([(32, 32, 64, 0, 1.0, 1.0, 1e-4)])   # n_sub 0
    for orth in ("mgs4", "mgs8"):   # the batched kernels orthogonalise pairs at most
        kkt.load_library().kkt_default_options(opt)
        opt.orth = kkt.ORTH[orth]
        with pytest.raises(kkt.KKTError, match="orthogonalises"):   # (a null handle: no status)
            kkt.kkt_batch_create([(32, 32, 64, 4, 1.0, 1.0, 1e-4)], opt)


def test_batch_replays_count_their_kernels(kkt, small_case):
    ps, fs = small_case
    b = kkt.Batch(SMALL[:2])
    kkt.kkt_profile_read(reset=True)
    res = b.solve(fs[:2], tol=1e-8, maxit=420)
    prof = kkt.kkt_profile_read(reset=True)
    steps = max(res.iterations)
    # per step (replayed graph or direct launches): 4 transform passes, coarse, sweeps, matvec
    assert prof["graph"]["launches"] == res.graph_launches
    assert prof["dst"]["launches"] >= 4 * steps
    assert prof["matvec"]["launches"] >= steps
    assert prof["coarse"]["launches"] >= steps and prof["sweep"]["launches"] >= steps


def test_batch_restart_cycles_and_ras_locals(kkt, small_case):
    """FGMRES(5) in the batched form (several lockstep restart cycles, instances finishing in
    different cycles) with RAS local solves: each instance matches its own kkt_solve."""
    ps, fs = small_case
    b = kkt.Batch(SMALL, restart=5)
    opt = kkt.KKTOptions()
    kkt.load_library().kkt_default_options(opt)
    res = b.solve(fs, tol=1e-8, maxit=420)
    assert res.status == kkt.KKT_OK
    for i, w in enumerate(SMALL):
        s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, restart=5)
        ref = s.solve(fs[i], tol=1e-8, maxit=420)
        s.close()
        assert abs(res.iterations[i] - ref.iterations) <= 1, (w.name, res.iterations[i], ref.iterations)
        assert rel(host(res.xs[i]), host(ref.x)) < 1e-5
    exact = [spectral.kkt_exact_solve(ps[i], host(fs[i])) for i in range(len(SMALL))]
    for local_opt in ("ras",):
        descs = [(w.nx, w.ny, w.Nt, w.n_sub, w.T, w.nu, w.omega) for w in SMALL]
        opt.local = kkt.LOCAL[local_opt]
        bh = kkt.kkt_batch_create(descs, opt)
        xs = [torch.zeros_like(f) for f in fs]
        st = kkt.KKTBatchStats()
        assert kkt.kkt_batch_solve(bh, fs, xs, 1e-12, 420, st) == kkt.KKT_OK
        kkt.kkt_batch_destroy(bh)
        for i in range(len(SMALL)):
            assert rel(host(xs[i]), exact[i]) < TOL, SMALL[i].name


def test_batch_large_instances_take_the_single_solve_path(kkt, small_case):
    """With a threshold below the largest instance, those instances are solved one by one
    (kkt_solve's path) and the rest in waves; every instance still matches its own solve."""
    ps, fs = small_case
    b = kkt.Batch(SMALL)
    biggest = max(w.V for w in SMALL)
    b.set_single_threshold(biggest)
    res = b.solve(fs, tol=1e-12, maxit=420)
    assert res.status == kkt.KKT_OK
    assert res.solo == sum(1 for w in SMALL if w.V >= biggest) and res.waves == 1
    for i in range(len(SMALL)):
        exact = spectral.kkt_exact_solve(ps[i], host(fs[i]))
        assert rel(host(res.xs[i]), exact) < TOL, SMALL[i].name
    b.set_single_threshold(1)          # every instance alone: no waves
    res = b.solve(fs, tol=1e-8, maxit=420)
    assert res.status == kkt.KKT_OK and res.solo == len(SMALL) and res.waves == 0


TENSOR_SET = [
    workloads.Workload("t0", nx=128, ny=128, Nt=128, n_sub=8, nu=1.0, omega=1e-4, target="sine-series", seed=21),
    workloads.Workload("t1", nx=64, ny=64, Nt=32, n_sub=4, nu=0.5, omega=1e-3, target="cos-mode-noise", seed=22),
    workloads.Workload("t2", nx=128, ny=128, Nt=96, n_sub=12, nu=2.0, omega=1e-5, target="cos-mode-noise", seed=23),
]


def test_batch_with_tensor_core_transforms(kkt):
    """Every instance on the tensor-core FP64 transform, all in the batched waves: the two whose
    GEMM passes fill the GPU (128 x 128 grids) are transformed alone inside the step graphs, the
    64 x 64 one stays in the line-tile launches. Each matches the oracle's exact solve at 1e-12
    and its own single solve's iteration count within 1; the physical and spectral bases."""
    ps, fs = zip(*[rhs(w) for w in TENSOR_SET])
    fs = [dev(f) for f in fs]
    for basis in ("physical", "spectral"):
        b = kkt.Batch(TENSOR_SET, basis=basis)
        b.set_dst_method("tensor")
        b.set_single_threshold(0)
        res = b.solve(fs, tol=1e-12, maxit=420)
        assert res.status == kkt.KKT_OK and res.solo == 0
        for i, w in enumerate(TENSOR_SET):
            assert rel(host(res.xs[i]), spectral.kkt_exact_solve(ps[i], host(fs[i]))) < TOL, (basis, w.name)
        res8 = b.solve(fs, tol=1e-8, maxit=420)
        for i, w in enumerate(TENSOR_SET):
            s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, basis=basis)
            s.set_dst_method("tensor")
            r = s.solve(fs[i], tol=1e-8, maxit=420)
            s.close()
            assert abs(r.iterations - res8.iterations[i]) <= 1, (basis, w.name, r.iterations, res8.iterations[i])
        b.close()
