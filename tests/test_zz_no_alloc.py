"""fp_apply_projection_noalloc: the allocation-free variant of the coarse projection.

Some callers cannot allocate device memory at call time: an application that has reserved
the device memory for its own pool, or a latency-bound loop that cannot take cudaMalloc's
implicit device synchronisation.  This entry point serves them: its scratch is a fixed
device array compiled into the library.  The tests call it through the C ABI, twice in a row
and in place, compare it with fp_apply_projection at the FP64 parity tolerance and with the
oracle's projector P = I - G (G^T G)^{-1} G^T, check that repeated calls change neither
torch's allocator nor the device's free memory, that a problem without floating subdomains
gets a plain copy, and that a problem above the array's limit (8192 floating subdomains) is
refused with FP_ERR_INVALID.  The file is collected last so that a run stopping at its first
failure has run every other test."""
import numpy as np
import pytest

from paper_2509_06673_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def F():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06673_gb300 import build
    build.build()
    from paper_2509_06673_gb300 import fetipe
    return fetipe


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_projection_noalloc_matches_projection_and_oracle(F):
    import torch
    from oracle.monolithic import Discretization
    from oracle.feti import FETI
    case = W.small_case(4, 4, 3, k=2, lame_lambda=49.0, tau=1e-3)   # 4 floating subdomains
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    assert sol.sizes.n_floating == 4
    fe = FETI(case, Discretization(case))
    rng = np.random.default_rng(7)
    out = torch.empty(sol.sizes.n_lambda, dtype=torch.float64, device="cuda")
    for _ in range(2):   # two calls in a row share the array
        v = rng.normal(size=sol.sizes.n_lambda)
        ref = sol.apply_projection(v)
        got = sol.apply_projection_noalloc(torch.from_numpy(v).cuda(), out).cpu().numpy()
        assert _rel(got, ref) <= TOL
        assert _rel(got, fe.P(v)) <= TOL
    # in place (v and out alias)
    v = rng.normal(size=sol.sizes.n_lambda)
    vt = torch.from_numpy(v).cuda()
    got = sol.apply_projection_noalloc(vt, vt).cpu().numpy()
    assert _rel(got, sol.apply_projection(v)) <= TOL
    sol.close()


def test_projection_noalloc_allocates_nothing(F):
    import torch
    case = W.small_case(4, 4, 3, k=2, lame_lambda=49.0, tau=1e-3)
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    n = sol.sizes.n_lambda
    v = torch.randn(n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(v)
    sol.apply_projection_noalloc(v, out)   # first call on the device: looks up the array
    first = out.clone()
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        sol.apply_projection_noalloc(v, out)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(out, first)
    sol.close()


def test_projection_noalloc_without_floating_subdomains_copies(F):
    import torch
    case = W.small_case(2, 2, 3, k=1, lame_lambda=3.0, tau=1e-2)   # every subdomain touches the boundary
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    assert sol.sizes.n_floating == 0
    v = torch.randn(sol.sizes.n_lambda, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(v)
    sol.apply_projection_noalloc(v, out)
    assert torch.equal(out, v)
    sol.close()


def test_projection_noalloc_rejects_more_than_8192_floating_subdomains(F):
    import torch
    case = W.grid_case("94x94 x 2 cells P1", 94, 94, 2, 2, order_k=1)   # 92^2 = 8464 floating
    assert F.plan(case).n_floating == 8464
    sol = F.Solver(case)
    v = torch.zeros(sol.sizes.n_lambda, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FetipeError) as ei:
        sol.apply_projection_noalloc(v, v)
    assert ei.value.status == F.FP_ERR_INVALID and "8192" in str(ei.value)
    sol.close()


def test_projection_noalloc_checks_tensors(F):
    import torch
    case = W.small_case(4, 4, 3, k=2, lame_lambda=49.0, tau=1e-3)
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    n = sol.sizes.n_lambda
    good = torch.zeros(n, dtype=torch.float64, device="cuda")
    for bad in (torch.zeros(n, dtype=torch.float32, device="cuda"), torch.zeros(n - 1, dtype=torch.float64,
                device="cuda"), torch.zeros(n, dtype=torch.float64), torch.zeros(2 * n, dtype=torch.float64,
                device="cuda")[::2]):
        with pytest.raises(ValueError):
            sol.apply_projection_noalloc(bad, good)
        with pytest.raises(ValueError):
            sol.apply_projection_noalloc(good, bad)
    sol.close()
