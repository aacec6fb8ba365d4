"""Guard bands around every buffer an entry point touches, a check for out-of-range writes
that needs no memory-checking tool: each vector is a view into a larger device allocation whose
margins hold a sentinel bit pattern, and after the call the margins must be untouched and the
inputs unchanged. Sizes are odd and ragged (tails in every kernel's tiling),
both coarse solvers and both transform methods run, and so do the reduced-precision forms
and the batched form.
"""

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

G = 4099   # guard doubles on each side (odd: shifts the view off any 16-byte alignment of the margin)
SENTINEL = 0x7FF4DEADBEEF0123   # a signalling-NaN bit pattern no kernel writes


@pytest.fixture(scope="module")
def kkt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_04421_gb300.kkt as k
    k.load_library()
    return k


class Guarded:
    """A device vector of n doubles inside margins of G sentinels."""

    def __init__(self, n, values=None):
        self.n = n
        self.buf = torch.empty(n + 2 * G, dtype=torch.int64, device="cuda")
        self.buf.fill_(SENTINEL)
        self.view = self.buf.view(torch.float64)[G:G + n]
        if values is not None:
            self.view.copy_(torch.from_numpy(np.ascontiguousarray(values, dtype=np.float64)))

    def margins_intact(self):
        torch.cuda.synchronize()
        b = self.buf.cpu().numpy()
        return bool((b[:G] == SENTINEL).all() and (b[G + self.n:] == SENTINEL).all())

    def values(self):
        torch.cuda.synchronize()
        return self.view.cpu().numpy().copy()


CASES = [
    # nx, ny, Nt, n_sub, options
    (17, 9, 23, 4, {}),                                  # non-power-of-two transforms, ragged tiles
    (16, 16, 65, 13, {"coarse_solve": "cyclic"}),
    (16, 16, 65, 13, {"coarse_solve": "thomas"}),
    (64, 64, 21, 5, {"local": "ras", "variant": "additive"}),
    (32, 32, 12, 3, {"precision": "tf32"}),
    (32, 32, 12, 3, {"precision": "bf16", "tc_split": False}),
]


@pytest.mark.parametrize("c", CASES)
def test_entry_points_write_only_their_outputs(kkt, c):
    nx, ny, Nt, nd, opts = c
    s = kkt.Solver(nx, ny, Nt, 1.0, 1.0, 1e-3, nd, **opts)
    V = s.V
    calls = [("matvec", 3 * V, 3 * V), ("precond_apply", 3 * V, 3 * V), ("dst2d", V, V), ("schur_apply", V, V),
             ("schur_precond_apply", V, V)]
    if opts.get("precision", "fp64") == "fp64":
        calls.append(("coarse_apply", V, V))
    for name, n_in, n_out in calls:
        x = workloads.random_vector(n_in, 40)
        gin, gout = Guarded(n_in, x), Guarded(n_out)
        getattr(s, name)(gin.view, out=gout.view)
        assert gin.margins_intact() and gout.margins_intact(), name
        assert np.array_equal(gin.values(), x), name + " changed its input"
        assert np.isfinite(gout.values()).all(), name + " left part of its output unwritten"
    # a solve: f read only, x written in place, and the right-hand side builder
    ut = Guarded(V, workloads.random_vector(V, 41))
    f = Guarded(3 * V)
    s.build_rhs(ut.view, out=f.view)
    assert ut.margins_intact() and f.margins_intact()
    f0 = f.values()
    x = Guarded(3 * V, np.zeros(3 * V))
    res = s.solve(f.view, x.view, tol=1e-8, maxit=60)
    assert res.status in (kkt.KKT_OK, kkt.KKT_NOT_CONVERGED)
    assert f.margins_intact() and x.margins_intact()
    assert np.array_equal(f.values(), f0)
    s.close()


def test_batched_solve_writes_only_its_outputs(kkt):
    ws = [workloads.Workload("g0", nx=17, ny=9, Nt=23, n_sub=4, omega=1e-3, target="sine-series", seed=1),
          workloads.Workload("g1", nx=16, ny=16, Nt=65, n_sub=13, omega=1e-4, target="sine-series", seed=2),
          workloads.Workload("g2", nx=32, ny=32, Nt=40, n_sub=8, omega=1e-2, target="sine-series", seed=3)]
    fs, xs = [], []
    for w in ws:
        s = kkt.Solver(w.nx, w.ny, w.Nt, w.T, w.nu, w.omega, w.n_sub)
        g = Guarded(3 * s.V)
        s.build_rhs(torch.from_numpy(workloads.make_target(w).ravel()).cuda(), out=g.view)
        fs.append(g)
        xs.append(Guarded(3 * s.V, np.zeros(3 * s.V)))
        s.close()
    f0 = [g.values() for g in fs]
    b = kkt.Batch(ws)
    b.set_single_threshold(0)
    res = b.solve([g.view for g in fs], [g.view for g in xs], tol=1e-8, maxit=420)
    assert res.status == kkt.KKT_OK
    for g, v in zip(fs, f0):
        assert g.margins_intact() and np.array_equal(g.values(), v)
    for g in xs:
        assert g.margins_intact()
    b.close()
