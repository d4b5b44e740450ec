"""The seeded synthetic inputs shared by the oracle and the CUDA path: the counter-based
SplitMix64 stream against its published definition, and the structure of the workloads
(uneven meshes, log-normal permeability, point-source placement)."""
import numpy as np

from paper_2509_06673_gb300 import workloads as W


def _splitmix64_scalar(seed, i):
    """SplitMix64 (Steele, Lea & Flood 2014), value i of the stream started at `seed`:
    state = seed + (i + 1) * golden gamma, then the two xor-shift-multiply rounds."""
    m = (1 << 64) - 1
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def test_splitmix64_matches_definition():
    idx = np.array([0, 1, 2, 1000, 2 ** 40], dtype=np.uint64)
    for seed in (0, 1, 12345):
        got = W.splitmix64(seed, idx)
        ref = [_splitmix64_scalar(seed, int(i)) for i in idx]
        assert [int(v) for v in got] == ref
    u = W.uniform01(7, np.arange(100000, dtype=np.uint64))
    assert u.min() > 0.0 and u.max() <= 1.0 and abs(u.mean() - 0.5) < 0.01


def test_uneven_cells_and_lognormal_perm():
    cx = W.uneven_cells(32, seed=0)
    assert cx == W.uneven_cells(32, seed=0) and len(cx) == 32
    assert all(16 <= c <= 48 for c in cx) and len(set(cx)) > 10
    c = W.grid_case("p", 4, 4, 24, 24)
    perm = W.lognormal_perm(c, sigma=1.0, seed=0)
    assert len(perm) == 16 and all(p.size == 2 * 24 * 24 for p in perm)
    g = np.log(np.concatenate(perm))
    assert abs(g.mean()) < 0.05 and abs(g.std() - 1.0) < 0.05


def test_point_source_node_inside_one_poroelastic_subdomain():
    c = W.config4(seed=0)
    for seed in range(1000, 1010):
        i, j = W.point_source_node(c, seed)
        # P1 vertex indices on the global grid, strictly inside the poroelastic half
        bx = np.cumsum([0] + list(c.cells_x))
        by = np.cumsum([0] + list(c.cells_y))
        assert 0 < i < bx[-1] and 0 < j < by[c.poro_rows]
        assert i not in bx and j not in by          # off partition lines: one owner
