"""Seeded synthetic workloads: the only module both the CUDA path and the oracle consume.

It holds no arithmetic of the method: only partition shapes, physical parameters, and
seeded random inputs (uneven cell counts, permeability field, point-source location).
Random numbers come from SplitMix64 (Steele, Lea & Flood 2014), used as a counter-based
generator: value i of stream ``seed`` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15).

Workloads (unit square, poroelastic below y = 1/2, elastic above, u = 0 on the boundary,
p = 0 on the outer boundary of the poroelastic region):

* ``config1``  1 x 2 subdomains of 16 x 16 cells, P1, lambda = mu = alpha = c0 = K = 1,
               manufactured solution of Test Case 1 (Sec. 4.1), 10 steps of dt = 0.01.
  Configs 2, 3 and 5 use the same closed form times (1 + t) so that every step changes
  the solution and the Krylov solve has work to do.
* ``config2``  8 x 8 subdomains of 32 x 32 cells, P2, nu = 0.49 (lambda = 49, mu = 1),
               50 steps of dt = 1e-3, Dirichlet preconditioner.
* ``config3``  32 x 32 subdomains, cells per partition column / row uniform on {16..48}
               (SplitMix64 seed 0), P2, nu = 0.49, dt = 1e-3, 100 steps.
* ``config4``  config-3 geometry with a point fluid source q(t) = sin(omega t) at a
               seeded node (seed 0 for training, 1 for evaluation), 400 + 200 steps.
* ``config5``  64 x 64 subdomains of 24 x 24 cells, P2, nu = 0.499 (lambda = 499),
               log-normal permeability exp(sigma g), g ~ N(0,1) per element (Box-Muller on
               SplitMix64 seed 0, sigma = 1), 200 steps.
"""
from dataclasses import dataclass, field, replace
from typing import Optional, Sequence

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, idx):
    """Counter-based SplitMix64: uint64 array for counters ``idx`` of stream ``seed``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed, idx):
    """Uniform doubles in (0, 1]."""
    z = splitmix64(seed, idx)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(seed, n, offset=0):
    """Standard normals by Box-Muller on consecutive pairs of the stream."""
    i = np.arange(n, dtype=np.uint64) + np.uint64(offset)
    u1 = uniform01(seed, 2 * i)
    u2 = uniform01(seed, 2 * i + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class Case:
    name: str
    nsub_x: int
    nsub_y: int
    cells_x: Sequence[int]
    cells_y: Sequence[int]
    poro_rows: int
    order_k: int = 2
    lame_lambda: float = 1.0
    mu: float = 1.0
    alpha: float = 1.0
    c0: float = 1.0
    perm_k: float = 1.0
    mu_f: float = 1.0
    tau: float = 1e-3
    n_steps: int = 1
    perm: Optional[list] = None          # per subdomain: per-element permeability (or None)
    source: str = "manufactured"         # "manufactured" | "manufactured_t" | "point" | "barry_mercer"
    src_node: tuple = (0, 0)             # global P1 grid indices of the point source
    q_omega: float = 0.0
    bc: str = "clamped"                  # "clamped" | "barry_mercer" (oracle only)
    tol: float = 1e-10
    max_it: int = 1000
    precision: str = "fp64"              # "fp64" | "mixed"
    precond: str = "dirichlet"           # "dirichlet" | "lumped" | "none" | "auto"
    extra: dict = field(default_factory=dict)

    @property
    def nsub(self):
        return self.nsub_x * self.nsub_y

    def is_poro(self, s):
        return (s // self.nsub_x) < self.poro_rows

    def with_(self, **kw):
        return replace(self, **kw)


def lame_from_nu(nu, mu=1.0):
    """lambda for a given Poisson ratio at fixed mu (plain definition of nu)."""
    return 2.0 * mu * nu / (1.0 - 2.0 * nu)


def grid_case(name, nsub_x, nsub_y, cells_x, cells_y, **kw):
    if np.isscalar(cells_x):
        cells_x = [int(cells_x)] * nsub_x
    if np.isscalar(cells_y):
        cells_y = [int(cells_y)] * nsub_y
    assert nsub_y % 2 == 0, "the interface y = 1/2 must be a partition line"
    return Case(name=name, nsub_x=nsub_x, nsub_y=nsub_y, cells_x=list(cells_x),
                cells_y=list(cells_y), poro_rows=nsub_y // 2, **kw)


def uneven_cells(n, seed=0, lo=16, hi=48, offset=0):
    z = splitmix64(seed, np.arange(n, dtype=np.uint64) + np.uint64(offset))
    return [int(lo + int(v % np.uint64(hi - lo + 1))) for v in z]


def lognormal_perm(case, sigma=1.0, seed=0):
    perms, off = [], 0
    for s in range(case.nsub):
        ne = 2 * case.cells_x[s % case.nsub_x] * case.cells_y[s // case.nsub_x]
        perms.append(np.exp(sigma * normal(seed, ne, offset=off)))
        off += ne
    return perms


def point_source_node(case, seed):
    """Seeded source location in [0.05, 0.95] x [0.05, 0.45], snapped to the nearest P1
    vertex and moved off partition lines (so exactly one subdomain owns it)."""
    u = uniform01(seed, np.arange(2, dtype=np.uint64))
    xs = 0.05 + 0.90 * u[0]
    ys = 0.05 + 0.40 * u[1]

    def snap(v, nsub, cells):
        c = min(int(v * nsub), nsub - 1)
        h = 1.0 / (nsub * cells[c])
        i = int(round((v - c / nsub) / h))
        if i == 0:
            i = 1
        if i == cells[c]:
            i = cells[c] - 1
        return int(sum(cells[:c])) + i
    return (snap(xs, case.nsub_x, case.cells_x), snap(ys, case.nsub_y, case.cells_y))


def config1(**kw):
    c = grid_case("config1: 1x2 subdomains, 16x16 cells, P1, manufactured", 1, 2, 16, 16,
                  order_k=1, tau=0.01, n_steps=10, tol=1e-10)
    return c.with_(**kw)


def config2(**kw):
    c = grid_case("config2: 8x8 subdomains, 32x32 cells, P2, nu=0.49", 8, 8, 32, 32,
                  order_k=2, lame_lambda=lame_from_nu(0.49), tau=1e-3, n_steps=50, tol=1e-10,
                  source="manufactured_t")
    return c.with_(**kw)


def config3(**kw):
    c = grid_case("config3: 32x32 subdomains, uneven 16..48 cells, P2, nu=0.49", 32, 32,
                  uneven_cells(32, seed=0), uneven_cells(32, seed=0, offset=32),
                  order_k=2, lame_lambda=lame_from_nu(0.49), tau=1e-3, n_steps=100,
                  tol=1e-8, precision="mixed", source="manufactured_t")
    return c.with_(**kw)


def config4(seed=0, **kw):
    c = config3(name=f"config4: config-3 geometry, point source seed {seed}", source="point",
                n_steps=400 if seed == 0 else 200)
    c = c.with_(src_node=point_source_node(c, seed + 1000),
                q_omega=2.0 * 2.0 * np.pi / (600 * c.tau))
    return c.with_(**kw)


def config5(**kw):
    c = grid_case("config5: 64x64 subdomains, 24x24 cells, P2, nu=0.499, log-normal K", 64, 64,
                  24, 24, order_k=2, lame_lambda=lame_from_nu(0.499), tau=1e-3, n_steps=200,
                  tol=1e-8, precision="mixed", source="manufactured_t")
    c = c.with_(perm=lognormal_perm(c, sigma=1.0, seed=0))
    return c.with_(**kw)


def small_case(nsub_x=2, nsub_y=2, cells=4, k=2, **kw):
    """Small multi-subdomain case for parity tests (several tiles, floating subdomains
    appear from 3 x 4 upwards)."""
    return grid_case(f"small {nsub_x}x{nsub_y} x {cells} cells P{k}", nsub_x, nsub_y,
                     cells, cells, order_k=k, **kw)
