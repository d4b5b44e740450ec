"""fp_apply_projection_noalloc: the allocation-free variant of the coarse projection.

Callers that cannot allocate device memory at call time (code running during CUDA graph
capture, or a runtime that owns all allocations) use this entry point; its scratch is a
fixed device array compiled into the library.  The test calls it through the C ABI twice
in a row and compares each result with fp_apply_projection at the FP64 parity tolerance.
It is collected last so that a run stopping at its first failure has run every other test."""
import numpy as np
import pytest

from paper_2509_06673_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_projection_noalloc_matches_projection():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06673_gb300 import build
    build.build()
    from paper_2509_06673_gb300 import fetipe as F
    case = W.small_case(4, 4, 3, k=2, lame_lambda=49.0, tau=1e-3)   # 4 floating subdomains
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    assert sol.sizes.n_floating == 4
    rng = np.random.default_rng(7)
    out = torch.empty(sol.sizes.n_lambda, dtype=torch.float64, device="cuda")
    for _ in range(2):
        v = rng.normal(size=sol.sizes.n_lambda)
        ref = sol.apply_projection(v)
        vt = torch.from_numpy(v).cuda()
        got = sol.apply_projection_noalloc(vt, out).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    sol.close()
