"""Learned coarse correction: the network's GPU kernels against the NumPy reference, GPU
training, and what the trained network adds to the preconditioner.

Tolerances (FP32 kernels against the FP64 reference): forward 1e-5, gradients 1e-4, one Adam
step 1e-5 (relative, per parameter block); BF16-weight inference vs FP32 weights 2e-2.
"""

import numpy as np
import pytest

import workloads
from oracle import mlp as ref
from oracle import problem
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


ORDER = ["W1", "b1", "W2", "b2", "W3", "b3"]


def flat(params):
    return np.concatenate([params[k].ravel() for k in ORDER]).astype(np.float32)


def unflat(v, like):
    out, o = {}, 0
    for k in ORDER:
        n = like[k].size
        out[k] = v[o:o + n].reshape(like[k].shape)
        o += n
    return out


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) / max(np.linalg.norm(b), 1e-300)


def small_net(kkt, **kw):
    cfg = dict(nx=16, Nt=16, n_sub=4, modes=4, width=16, seed=3)
    cfg.update(kw)
    return kkt.Mlp(**cfg)


def test_forward_gradients_and_adam_match_reference(kkt):
    net = small_net(kkt)
    d_out = 2 * net.cfg.n_sub
    params = ref.init_params(d_out + 2, net.cfg.width, d_out, seed=11)
    rng = np.random.default_rng(2)
    for k in ("b1", "b2", "b3"):
        params[k] = 0.1 * rng.standard_normal(params[k].shape)
    params = {k: v.astype(np.float32).astype(np.float64) for k, v in params.items()}
    net.set_params(flat(params))
    assert np.array_equal(net.get_params(), flat(params))
    X = rng.standard_normal((37, d_out + 2)).astype(np.float32)
    T = rng.standard_normal((37, d_out)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    Y, cache = ref.forward(params, X.astype(np.float64))
    assert rel(net.forward(Xd).cpu().numpy(), Y) < 1e-5
    assert rel(net.forward(Xd, use_bf16=True).cpu().numpy(), Y) < 2e-2
    loss, g = net.loss_grad(Xd, Td)
    gref = ref.backward(params, cache, Y, T.astype(np.float64))
    np.testing.assert_allclose(loss, ref.loss(Y, T.astype(np.float64)), rtol=1e-5)
    gg = unflat(g.cpu().numpy(), params)
    for k in ORDER:
        assert rel(gg[k], gref[k]) < 1e-4, k
    net.adam_step(Xd, Td, lr=1e-3)
    state = {}
    ref.adam_step(params, gref, state, t=1, lr=1e-3)
    got = unflat(net.get_params(), params)
    for k in ORDER:
        assert rel(got[k], params[k]) < 1e-5, k


def test_coarse_residual_loss_and_gradients_match_reference(kkt):
    """The guard's quantity as a training loss: ||c - alpha G d||^2 / ||c||^2 with the
    minimal-residual alpha, per sample mu, on the network's own decomposition (Nt = 16,
    N_D = 4); loss and every parameter gradient against the FP64 reference."""
    net = small_net(kkt)
    nc = 2 * net.cfg.n_sub
    params = ref.init_params(nc + 2, net.cfg.width, nc, seed=12)
    rng = np.random.default_rng(21)
    for k in ("b1", "b2", "b3"):
        params[k] = 0.1 * rng.standard_normal(params[k].shape)
    params = {k: v.astype(np.float32).astype(np.float64) for k, v in params.items()}
    net.set_params(flat(params))
    B = 29
    C = rng.standard_normal((B, nc))
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    X = np.concatenate([C, rng.standard_normal((B, 2))], axis=1).astype(np.float32)
    mu = 1.0 + rng.uniform(0.01, 3.0, B)
    loss, g = net.resid_loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(mu).cuda())
    Y, cache = ref.forward(params, X.astype(np.float64))
    G = [ref.coarse_operator(float(m), net.cfg.Nt, net.cfg.n_sub) for m in mu]
    want, dY = ref.coarse_residual_loss(Y, X[:, :nc].astype(np.float64), G)
    np.testing.assert_allclose(loss, want, rtol=1e-5)
    gref = ref.backward_from(params, cache, dY)
    gg = unflat(g.cpu().numpy(), params)
    for k in ORDER:
        assert rel(gg[k], gref[k]) < 1e-4, k


def test_training_pairs_match_reference(kkt):
    """The coarse right-hand sides R_0 r and exact coarse solutions the network is trained on,
    generated by the GPU's restriction and block-Thomas elimination, against the reference's
    restriction matrix and dense solve (ragged split: Nt = 30, N_D = 7), element by element."""
    net = small_net(kkt, nx=16, Nt=30, n_sub=7, modes=4)
    rng = np.random.default_rng(9)
    count = 50
    r = rng.standard_normal((30, count))
    mu = 1.0 + np.concatenate([rng.uniform(0.005, 0.05, count // 2), rng.uniform(0.05, 6.0, count - count // 2)])
    c, x = net.coarse_data(torch.from_numpy(r).cuda(), torch.from_numpy(mu).cuda())
    c, x = c.cpu().numpy(), x.cpu().numpy()
    C, Xr = ref.coarse_data(r, mu, 30, 7)
    for b in range(count):
        np.testing.assert_allclose(c[b], C[b], rtol=0, atol=1e-13 * np.abs(C[b]).max())
        np.testing.assert_allclose(x[b], Xr[b], rtol=0, atol=1e-10 * np.abs(Xr[b]).max())


def test_save_and_load_round_trip(kkt, tmp_path):
    net = small_net(kkt, seed=5)
    path = str(tmp_path / "net.bin")
    net.save(path)
    back = kkt.Mlp.load(path)
    assert np.array_equal(back.get_params(), net.get_params())
    assert back.cfg.n_sub == net.cfg.n_sub and back.cfg.width == net.cfg.width


def _solve_counts(kkt, w, net):
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    f = problem.assemble_rhs(p, workloads.make_target(w), None)
    fd = torch.from_numpy(f).cuda()
    its = {}
    for name, coarse, mode in [("exact", "exact", None), ("one-level", "none", None),
                               ("learned", "learned", "learned"), ("without-network", "learned", "none"),
                               ("network-only", "learned", "network")]:
        s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub)
        if mode is not None:
            s.attach_mlp(net, mode)
        s.set_options(coarse=coarse)
        res = s.solve(fd, tol=1e-8, maxit=420)
        assert res.status == kkt.KKT_OK, name
        its[name] = res.iterations
        if name == "learned":
            its["kept"], its["fallback"] = s.learned_stats()
        if name == "network-only":
            its["net_applied"], its["net_beyond_guard"] = s.learned_stats()
    return its


@pytest.fixture(scope="module")
def trained(kkt):
    """A network trained on the GPU for the 32 x 32, Nt = 128, N_D = 16 geometry (modes k, l < 8)."""
    w = workloads.Workload("t", nx=32, ny=32, Nt=128, n_sub=16, nu=1.0, omega=1e-4, target="sine-series", seed=7)
    net = kkt.Mlp(nx=32, Nt=128, n_sub=16, modes=8, width=128, seed=4, samples=8192, epochs=40, batch=128,
                  nu_lo=0.5, nu_hi=2.0, omega_lo=3e-5, omega_hi=3e-4, lr=2e-3)
    st = net.train()
    return w, net, st


def test_trained_network_reduces_iterations(kkt, trained):
    """Solve with the exact coarse solve, none, the learned correction (guarded), the network's
    corrections alone (no guard, no exact fallback), and the learned modes left without coarse
    correction: the network alone must beat that ablation, so the gain is the network's and not
    the exact solve's."""
    w, net, st = trained
    assert st.val_cosine > 0.8, st.val_cosine
    its = _solve_counts(kkt, w, net)
    assert its["kept"] > 0
    assert its["net_applied"] > 0
    assert its["learned"] < its["without-network"], its
    assert its["network-only"] < its["without-network"], its
    assert its["exact"] <= its["learned"], its


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_learned_coarse_with_tensor_core_transforms(kkt, trained, prec):
    """The learned correction inside the reduced-precision preconditioner (padded mode grid):
    converges to 1e-8, keeps learned corrections, and matches the FP64 learned solve."""
    w, net, _ = trained
    p = HeatKKT(nx=w.nx, ny=w.ny, Nt=w.Nt, nu=w.nu, omega=w.omega)
    fd = torch.from_numpy(problem.assemble_rhs(p, workloads.make_target(w), None)).cuda()
    out = {}
    for form in ("fp64", prec):
        s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub, precision=form)
        s.attach_mlp(net, "learned")
        s.set_options(precision=form, coarse="learned")
        r = s.solve(fd, tol=1e-8, maxit=420)
        assert r.status == kkt.KKT_OK, form
        kept, _ = s.learned_stats()
        assert kept > 0, form
        out[form] = r
    bound = out["fp64"].iterations + 2 if prec == "tf32" else int(1.5 * out["fp64"].iterations) + 2
    assert out[prec].iterations <= bound
    assert float(torch.linalg.vector_norm(out[prec].x - out["fp64"].x) / torch.linalg.vector_norm(out["fp64"].x)) < 1e-6
