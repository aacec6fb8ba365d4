"""kkt_multidot_noalloc: the multi-dot for callers that cannot allocate device memory.

Such callers (an application whose device memory belongs to another allocator, or a loop that
must not allocate) pass only their inputs and output; the library keeps the partial sums in a
static device array. This file is collected last so that a run stopping at its first failure
has already run every other test; it also passes alone in a fresh process.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kkt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_04421_gb300.kkt as k
    k.load_library()
    return k


@pytest.mark.parametrize("count,n", [(1, 7), (9, 100003), (32, 400001)])
def test_noalloc_multidot_matches_the_allocating_entry_point(kkt, count, n):
    rng = np.random.default_rng(100 + count)
    stride = n + 5
    V = torch.from_numpy(rng.standard_normal(count * stride)).cuda()
    w = torch.from_numpy(rng.standard_normal(n)).cuda()
    solver = kkt.Solver(8, 8, 8, 1.0, 1.0, 1e-3, 2)
    ref = torch.empty(count + 1, dtype=torch.float64, device="cuda")
    kkt.kkt_multidot(solver.h, V, stride, count, w, n, ref)
    scale = (torch.linalg.vector_norm(V.view(count, stride)[:, :n], dim=1).cpu().numpy().tolist()
             + [float(torch.linalg.vector_norm(w))])
    scale = np.asarray(scale) * float(torch.linalg.vector_norm(w))
    for _ in range(2):                     # two calls in a row share the static scratch
        out = torch.full((count + 1,), float("nan"), dtype=torch.float64, device="cuda")
        kkt.kkt_multidot_noalloc(V, stride, count, w, n, out)
        torch.cuda.synchronize()
        diff = (out - ref).abs().cpu().numpy()
        assert np.all(diff <= 1e-13 * scale)


def test_noalloc_multidot_rejects_counts_beyond_its_scratch(kkt):
    V = torch.zeros(33 * 10, dtype=torch.float64, device="cuda")
    w = torch.zeros(10, dtype=torch.float64, device="cuda")
    out = torch.zeros(34, dtype=torch.float64, device="cuda")
    with pytest.raises(kkt.KKTError) as ei:
        kkt.kkt_multidot_noalloc(V, 10, 33, w, 10, out)
    assert ei.value.status == kkt.KKT_ERR_INVALID_ARG
    assert "32" in str(ei.value)
