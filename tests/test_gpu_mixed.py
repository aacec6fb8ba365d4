"""Reduced-precision forms: DST transforms on tcgen05 tensor cores (BF16 or TF32 operands, FP32
accumulation), FP32 sweeps, FP64 coarse solve and FP64 FGMRES.

By default every transform uses split operands (x = x_hi + x_lo, Q = Q_hi + Q_lo, three
products accumulated in FP32); tc_split = 0 selects single operands.

Errors against FP64, per result (norm-wise relative):
* BF16 2D transform vs an exact NumPy emulation of the same splits and roundings (FP64 sums):
  <= 2e-5 (FP32 accumulation order, rare tie flips of the rounded intermediate); vs the FP64
  transform: <= 1e-4 (the dropped lo x lo products, about 2^-16).
* TF32 2D transform vs the FP64 transform: <= 2e-5.
* preconditioner apply vs the FP64 oracle: split <= 1e-3 (BF16), <= 1e-4 (TF32); single
  operands <= 2e-2 (BF16), <= 3e-3 (TF32), dominated by the inverse transform (about 2^-9 and
  2^-11 of the output).
* solves: the same 1e-8 weighted relative residual as FP64, checked against the exact solution.
"""

import numpy as np
import pytest

import workloads
from oracle import problem, schwarz, spectral
from oracle.problem import HeatKKT

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


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


def bf16(x):
    """Round-to-nearest-even to 8 significant bits (BF16), computed exactly in FP64."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def split_bf16(x):
    hi = bf16(x)
    return hi, bf16(x - hi)


def split_f32_bf16(x):
    """hi/lo split of FP32 values as the kernel forms it: hi = bf16(v), lo = bf16(fl32(v - hi))."""
    v = np.asarray(x, dtype=np.float32).astype(np.float64)
    hi = bf16(v)
    return hi, bf16((v - hi).astype(np.float32).astype(np.float64))


def dst_matrix(n):
    j = np.arange(1, n)
    return np.sqrt(2.0 / n) * np.sin(np.pi * np.outer(j, j) / n)


@pytest.mark.parametrize("n,Nt", [(16, 3), (128, 5), (200, 2), (256, 4)])
def test_bf16_tensor_core_transform_matches_emulation(kkt, n, Nt):
    p = HeatKKT(nx=n, ny=n, Nt=Nt)
    s = kkt.Solver(n, n, Nt, 1.0, 1.0, 1e-3, 1, precision="bf16")
    x = workloads.random_vector(p.V, 40 + n).reshape(Nt, n - 1, n - 1)
    got = host(s.dst2d(dev(x.ravel()))).reshape(Nt, n - 1, n - 1)       # [t][l][k]
    Qh, Ql = split_bf16(dst_matrix(n))
    xh, xl = split_bf16(x.astype(np.float32).astype(np.float64))   # the pack splits the FP32-rounded input
    y1 = (np.einsum("tji,ik->tkj", xh, Qh) + np.einsum("tji,ik->tkj", xh, Ql)
          + np.einsum("tji,ik->tkj", xl, Qh))      # along x -> [t][k][j], accumulated in FP32
    yh, yl = split_f32_bf16(y1)
    want = (np.einsum("tkj,jl->tlk", yh, Qh) + np.einsum("tkj,jl->tlk", yh, Ql)
            + np.einsum("tkj,jl->tlk", yl, Qh))    # along y -> [t][l][k]
    assert rel(got, want) < 2e-5
    exact = spectral.dst2(x, p)
    assert rel(got, exact) < 1e-4


@pytest.mark.parametrize("n,Nt", [(16, 3), (130, 2), (256, 4)])
def test_tf32_tensor_core_transform_close_to_fp64(kkt, n, Nt):
    p = HeatKKT(nx=n, ny=n, Nt=Nt)
    s = kkt.Solver(n, n, Nt, 1.0, 1.0, 1e-3, 1, precision="tf32")
    x = workloads.random_vector(p.V, 50 + n)
    got = host(s.dst2d(dev(x)))
    assert rel(got, spectral.dst2(x, p).ravel()) < 2e-5


@pytest.mark.parametrize("prec,split,tol", [("bf16", True, 1e-3), ("tf32", True, 1e-4),
                                            ("bf16", False, 2e-2), ("tf32", False, 3e-3)])
@pytest.mark.parametrize("variant,coarse", [("multiplicative", "exact"), ("multiplicative", "none")])
def test_mixed_schur_preconditioner_error_vs_fp64_oracle(kkt, prec, split, tol, variant, coarse):
    w = workloads.CFG_SMALL
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, precision=prec, variant=variant, coarse=coarse,
                   tc_split=split)
    pre = schwarz.schur_preconditioner(p, w.n_sub, variant="one-level" if coarse == "none" else variant)
    r = workloads.random_vector(p.V, 61)
    err = rel(host(s.schur_precond_apply(dev(r))), pre.apply(r))
    assert err < tol, err


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_mixed_solve_reaches_tolerance_and_exact_solution(kkt, prec):
    w = workloads.CFG_SMALL
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    f = problem.assemble_rhs(p, workloads.make_target(w), workloads.make_u0(w))
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, precision=prec)
    res = s.solve(dev(f), tol=1e-8, maxit=420)
    assert res.status == kkt.KKT_OK and res.rel_residual <= 1e-8
    K = problem.assemble_K(p)
    d = problem.l2_residual_weights(p)
    x = host(res.x)
    assert np.linalg.norm(d * (f - K @ x)) / np.linalg.norm(d * f) <= 1.01e-8
    assert rel(x, spectral.kkt_exact_solve(p, f)) < 1e-6
    tight = s.solve(dev(f), tol=1e-12, maxit=420)
    assert tight.status == kkt.KKT_OK
    assert rel(host(tight.x), spectral.kkt_exact_solve(p, f)) < 1e-10


def test_mixed_preconditioner_full_grid_vs_fp64_gpu(kkt):
    """512 x 512 grid (the mixed workload's spatial size), a short time axis: the BF16 and TF32
    applies against the FP64 apply on the same GPU."""
    n, Nt, nd = 512, 16, 4
    r = torch.randn((n - 1) ** 2 * Nt, dtype=torch.float64, device="cuda",
                    generator=torch.Generator("cuda").manual_seed(3))
    ref = kkt.Solver(n, n, Nt, 1.0, 0.1, 1e-4, nd).schur_precond_apply(r)
    for prec, split, tol in (("bf16", True, 1e-3), ("tf32", True, 1e-4), ("bf16", False, 2e-2), ("tf32", False, 3e-3)):
        got = kkt.Solver(n, n, Nt, 1.0, 0.1, 1e-4, nd, precision=prec, tc_split=split).schur_precond_apply(r)
        err = float(torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref))
        assert err < tol, (prec, err)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_mixed_solve_converges_on_a_large_grid(kkt, prec):
    """256 x 256, Nt = 64, N_D = 8, nu = 0.1: a high mu_max / mu_min ratio, where an unsplit BF16
    forward transform stalls FGMRES; with split transforms both forms reach 1e-8. TF32 keeps
    the FP64 iteration count (+2); BF16's split operands still carry about 2^-16 relative error
    per transform, which costs a few iterations at this ratio (measured 27 against 21): bound
    1.5x + 2."""
    w = workloads.Workload("t", nx=256, ny=256, Nt=64, n_sub=8, nu=0.1, omega=1e-4, target="sine-series", seed=2)
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, precision=prec)
    ref = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub)
    ut = dev(workloads.make_target(w).ravel())
    f = ref.build_rhs(ut)
    a = ref.solve(f, tol=1e-8, maxit=420)
    b = s.solve(f, tol=1e-8, maxit=420)
    assert a.status == kkt.KKT_OK and b.status == kkt.KKT_OK
    bound = a.iterations + 2 if prec == "tf32" else int(1.5 * a.iterations) + 2
    assert b.iterations <= bound
    assert float(torch.linalg.vector_norm(b.x - a.x) / torch.linalg.vector_norm(a.x)) < 1e-6


def test_pipeline_timeout_flag_is_reported_and_cleared(kkt):
    """The tensor-core transforms' timeout path, injected from the host (the device flag a
    bounded pipeline wait sets when it runs out; no kernel is made to wait): the next solve
    returns KKT_ERR_TIMEOUT, and the one after it, with the flag cleared, converges."""
    w = workloads.Workload("t", nx=32, ny=32, Nt=32, n_sub=4, omega=1e-4)
    s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, precision="tf32")
    ut = torch.from_numpy(workloads.make_target(w).ravel()).cuda()
    f = s.build_rhs(ut)
    kkt.load_library().kkt_inject_tc_timeout(s.h)
    with pytest.raises(kkt.KKTError) as ei:
        s.solve(f, tol=1e-8, maxit=100)
    assert ei.value.status == kkt.KKT_ERR_TIMEOUT
    res = s.solve(f, tol=1e-8, maxit=100)
    assert res.status == kkt.KKT_OK
    s.close()
    fp64 = kkt.Solver(8, 8, 8, 1.0, 1.0, 1e-3, 2)
    assert kkt.load_library().kkt_inject_tc_timeout(fp64.h) == kkt.KKT_ERR_INVALID_ARG
    fp64.close()
