"""Seeded synthetic workloads for the SCSF eigenvalue-dataset pipeline.

This module is shared by the CPU oracle, the tests and the benchmark. It only
*defines the inputs* (coefficient fields sampled on the grid); it holds none of
the method's arithmetic (no discretisation, no DFT, no sort, no eigensolver).

The paper's datasets (App. D.2: generalized Poisson -div(K grad h) = lambda h
with K from a Gaussian random field; Helmholtz-type operators) are not
available, so smooth random fields of the same kind stand in for them:

    f(x, y) = sum_{p<M} sum_{q<M} xi_pq cos(p pi x) cos(q pi y),  xi_pq ~ N(0, 1)

drawn p-major from ``numpy.random.default_rng(seed)`` one operator after the
other, with the (0, 0) mode included and no decay weighting.

* div-a-grad workloads (generalized Poisson, App. D.2 item 1):
  a = exp(0.5 f / M) with M = 8. The mode sum is normalised by 1/M: the
  plain sum of 64 unit-variance modes has a standard deviation of about 4,
  which makes a span 10^5-10^6 (far outside the moderate-contrast random
  fields of the paper's Poisson data); with the 1/M factor f/M has a standard
  deviation of about 0.5 and a spans a factor of about 4-6.
* Laplacian-plus-potential workloads (stand-in for the Helmholtz family,
  App. D.2 item 3): V = 10 f with M = 12.
* thin-plate vibration workloads (App. D.2 item 4, div(grad(D lap u)) = lambda rho u):
  flexural rigidity D = exp(0.5 f / M) and density rho = exp(0.5 g / M), M = 8, with
  f and g drawn one after the other (f's modes first), both at the n x n nodes.

Grid convention (Sec. 2.1, row-major node order): the unit square holds an
n x n interior grid with spacing h = 1/(n+1); node (i, j) sits at
x = (i+1) h, y = (j+1) h and has linear index I = i*n + j (j fastest).
Face coefficients are the field evaluated at face midpoints:

* ``ax[f, j]`` = a((f + 1/2) h, (j+1) h), f = 0..n   (the x-face between
  node (f-1, j) and node (f, j); f = 0 and f = n touch the boundary)
* ``ay[i, g]`` = a((i+1) h, (g + 1/2) h), g = 0..n

The sort's parameter matrix P (Alg. 2) is the field at the n x n nodes.

General sparse operators (the solver's CSR operator kind) have no grid: there
the matrix itself is the input. ``knn_graph_chain`` stands in for operators on
unstructured meshes: a weighted k-nearest-neighbour graph Laplacian on a random
point cloud (irregular row lengths, 7 to 14 entries a row) plus a quadratic
potential whose centre moves along the chain.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

__all__ = [
    "DivAGradOp", "LapPlusVOp", "mode_coefficients", "cosine_field",
    "div_a_grad_chain", "lap_plus_v_chain", "constant_div_a_grad",
    "separable_div_a_grad", "gaussian_block", "batched_chain_specs",
    "SparseOp", "knn_graph_chain", "PlateOp", "plate_chain", "constant_plate", "WORKLOADS",
]


@dataclass
class DivAGradOp:
    """-div(a grad u) on the n x n interior grid, Dirichlet boundary."""
    n: int
    ax: np.ndarray  # [n+1, n] float64
    ay: np.ndarray  # [n, n+1] float64
    P: np.ndarray   # [n, n]   float64, a at the nodes (sort input)

    @property
    def N(self) -> int:
        return self.n * self.n


@dataclass
class LapPlusVOp:
    """-Lap u + V u on the n x n interior grid, Dirichlet boundary."""
    n: int
    V: np.ndarray   # [n, n] float64, V at the nodes (also the sort input)

    @property
    def N(self) -> int:
        return self.n * self.n

    @property
    def P(self) -> np.ndarray:
        return self.V


@dataclass
class PlateOp:
    """Thin-plate vibration problem on the n x n interior grid: rigidity D and density rho
    at the nodes."""
    n: int
    D: np.ndarray    # [n, n] float64
    rho: np.ndarray  # [n, n] float64

    @property
    def N(self) -> int:
        return self.n * self.n

    @property
    def P(self) -> np.ndarray:
        """Sort input: the local ratio D / rho (the eigenvalues scale with it)."""
        return self.D / self.rho


def mode_coefficients(rng: np.random.Generator, M: int) -> np.ndarray:
    """xi[p, q] ~ N(0, 1), drawn p-major (q fastest)."""
    return rng.standard_normal((M, M))


def cosine_field(xi: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """f(x_r, y_s) = sum_pq xi_pq cos(p pi x_r) cos(q pi y_s) on a tensor grid."""
    M = xi.shape[0]
    cx = np.cos(np.pi * np.outer(x, np.arange(M)))  # [len(x), M]
    cy = np.cos(np.pi * np.outer(y, np.arange(M)))  # [len(y), M]
    return cx @ xi @ cy.T


def _grids(n: int):
    h = 1.0 / (n + 1)
    nodes = (np.arange(n) + 1.0) * h
    faces = (np.arange(n + 1) + 0.5) * h
    return nodes, faces


def _div_a_grad_from_xi(n: int, xi: np.ndarray, scale: float | None = None) -> DivAGradOp:
    """a = exp(scale * f); the default scale is 0.5 / M (normalised mode sum)."""
    if scale is None:
        scale = 0.5 / xi.shape[0]
    nodes, faces = _grids(n)
    ax = np.exp(scale * cosine_field(xi, faces, nodes))
    ay = np.exp(scale * cosine_field(xi, nodes, faces))
    P = np.exp(scale * cosine_field(xi, nodes, nodes))
    return DivAGradOp(n, np.ascontiguousarray(ax), np.ascontiguousarray(ay),
                      np.ascontiguousarray(P))


def div_a_grad_chain(n: int, n_ops: int, seed: int, M: int = 8) -> List[DivAGradOp]:
    """n_ops operators -div(a grad u), a = exp(0.5 f / M), f with M x M modes."""
    rng = np.random.default_rng(seed)
    return [_div_a_grad_from_xi(n, mode_coefficients(rng, M)) for _ in range(n_ops)]


def perturbed_div_a_grad_chain(n: int, n_ops: int, seed: int, eps: float, M: int = 8) -> List[DivAGradOp]:
    """Operators whose mode coefficients are xi0 + eps * xi_i: a family of similar
    problems around one base field (the shape of the paper's perturbation study)."""
    rng = np.random.default_rng(seed)
    xi0 = mode_coefficients(rng, M)
    return [_div_a_grad_from_xi(n, xi0 + eps * mode_coefficients(rng, M)) for _ in range(n_ops)]


def lap_plus_v_chain(n: int, n_ops: int, seed: int, M: int = 12,
                     amplitude: float = 10.0) -> List[LapPlusVOp]:
    """n_ops operators -Lap u + V u, V = amplitude * f, f with M x M modes."""
    rng = np.random.default_rng(seed)
    nodes, _ = _grids(n)
    out = []
    for _ in range(n_ops):
        xi = mode_coefficients(rng, M)
        out.append(LapPlusVOp(n, np.ascontiguousarray(amplitude * cosine_field(xi, nodes, nodes))))
    return out


def plate_chain(n: int, n_ops: int, seed: int, M: int = 8) -> List[PlateOp]:
    """n_ops plate problems: D = exp(0.5 f / M), rho = exp(0.5 g / M), f then g drawn per
    problem."""
    rng = np.random.default_rng(seed)
    nodes, _ = _grids(n)
    out = []
    for _ in range(n_ops):
        f = cosine_field(mode_coefficients(rng, M), nodes, nodes)
        g = cosine_field(mode_coefficients(rng, M), nodes, nodes)
        out.append(PlateOp(n, np.ascontiguousarray(np.exp(0.5 * f / M)),
                           np.ascontiguousarray(np.exp(0.5 * g / M))))
    return out


def constant_plate(n: int, D: float = 1.0, rho: float = 1.0) -> PlateOp:
    """Uniform plate: D and rho constant."""
    return PlateOp(n, np.full((n, n), D), np.full((n, n), rho))


def constant_div_a_grad(n: int, value: float = 1.0) -> DivAGradOp:
    """a == value everywhere (the Dirichlet Laplacian when value == 1)."""
    return DivAGradOp(n, np.full((n + 1, n), value), np.full((n, n + 1), value),
                      np.full((n, n), value))


def separable_lap_plus_v(n: int, seed: int, M: int = 12, amplitude: float = 10.0) -> LapPlusVOp:
    """-Lap u + V u with V = amplitude (g1(x) + g2(y)), g = sum_p xi_p cos(p pi x),
    xi ~ N(0, 1) (g1's M coefficients drawn first)."""
    rng = np.random.default_rng(seed)
    xi1 = rng.standard_normal(M)
    xi2 = rng.standard_normal(M)
    nodes, _ = _grids(n)
    c = np.cos(np.pi * np.outer(nodes, np.arange(M)))
    V = amplitude * ((c @ xi1)[:, None] + (c @ xi2)[None, :])
    return LapPlusVOp(n, np.ascontiguousarray(V))


def separable_div_a_grad(n: int, seed: int, M: int = 8) -> DivAGradOp:
    """a = a(x) only: a = exp(0.5 g(x) / M), g = sum_p xi_p cos(p pi x)."""
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal(M)
    nodes, faces = _grids(n)
    gx_faces = np.cos(np.pi * np.outer(faces, np.arange(M))) @ xi
    gx_nodes = np.cos(np.pi * np.outer(nodes, np.arange(M))) @ xi
    s = 0.5 / M
    ax = np.repeat(np.exp(s * gx_faces)[:, None], n, axis=1)
    ay = np.repeat(np.exp(s * gx_nodes)[:, None], n + 1, axis=1)
    P = np.repeat(np.exp(s * gx_nodes)[:, None], n, axis=1)
    return DivAGradOp(n, ax, ay, P)


@dataclass
class SparseOp:
    """A symmetric sparse matrix in CSR form (rows sorted, columns ascending in each row)."""
    rows: int
    row_ptr: np.ndarray  # [rows + 1] int32
    col: np.ndarray      # [nnz] int32
    val: np.ndarray      # [nnz] float64

    @property
    def N(self) -> int:
        return self.rows


def knn_graph_chain(N: int, n_ops: int, seed: int, neighbours: int = 6,
                    amplitude: float = 10.0) -> List[SparseOp]:
    """n_ops operators L + diag(V_t) on one random point cloud.

    N points uniform in the unit square; each is joined to its `neighbours` nearest
    points, the edge set is symmetrised and every edge gets a weight uniform in
    [0.5, 1.5). L = D - W is the weighted graph Laplacian and
    V_t(x, y) = amplitude ((x - c_x)^2 + (y - c_y)^2) with the centre
    c = (0.5 + 0.2 cos(2 pi t / 64), 0.5 + 0.2 sin(2 pi t / 64)) for problem t (a slow
    walk, so consecutive problems are close).
    """
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    pts = rng.random((N, 2))
    _, nb = cKDTree(pts).query(pts, k=neighbours + 1)
    i = np.repeat(np.arange(N), neighbours)
    j = nb[:, 1:].reshape(-1)
    edges = np.unique(np.stack([np.minimum(i, j), np.maximum(i, j)], axis=1), axis=0)
    w = 0.5 + rng.random(len(edges))
    r = np.concatenate([edges[:, 0], edges[:, 1]])
    c = np.concatenate([edges[:, 1], edges[:, 0]])
    ww = np.concatenate([w, w])
    deg = np.bincount(r, weights=ww, minlength=N)
    out = []
    for t in range(n_ops):
        ang = 2.0 * np.pi * t / 64.0
        cx, cy = 0.5 + 0.2 * np.cos(ang), 0.5 + 0.2 * np.sin(ang)
        V = amplitude * ((pts[:, 0] - cx) ** 2 + (pts[:, 1] - cy) ** 2)
        rows = np.concatenate([r, np.arange(N)])
        cols = np.concatenate([c, np.arange(N)])
        vals = np.concatenate([-ww, deg + V])
        order = np.lexsort((cols, rows))
        rows, cols, vals = rows[order], cols[order], vals[order]
        row_ptr = np.zeros(N + 1, dtype=np.int64)
        np.cumsum(np.bincount(rows, minlength=N), out=row_ptr[1:])
        out.append(SparseOp(N, row_ptr.astype(np.int32), cols.astype(np.int32),
                            vals.astype(np.float64)))
    return out


def gaussian_block(N: int, k: int, seed: int) -> np.ndarray:
    """A seeded N x k block of N(0, 1) entries, row-major (k fastest)."""
    return np.random.default_rng(seed).standard_normal((N, k))


@dataclass
class ChainSpec:
    n: int
    k: int
    seed: int
    n_ops: int


def batched_chain_specs(n_chains: int, n_ops: int, seed: int, n_lo: int = 64,
                        n_hi: int = 192, k_lo: int = 32, k_hi: int = 256) -> List[ChainSpec]:
    """Per-chain grid side and k drawn uniformly (inclusive), one seed per chain."""
    rng = np.random.default_rng(seed)
    specs = []
    for c in range(n_chains):
        n = int(rng.integers(n_lo, n_hi + 1))
        k = int(rng.integers(k_lo, k_hi + 1))
        specs.append(ChainSpec(n=n, k=k, seed=int(seed * 1000 + c), n_ops=n_ops))
    return specs


@dataclass
class Workload:
    name: str
    kind: str           # "div_a_grad" | "lap_plus_v"
    n: int
    n_ops: int
    k: int
    degree: int
    tol: float
    seed: int
    p0: int = 8
    extra: dict = field(default_factory=dict)

    def operators(self, n_ops: int | None = None):
        cnt = self.n_ops if n_ops is None else n_ops
        if self.kind == "div_a_grad":
            return div_a_grad_chain(self.n, cnt, self.seed)
        return lap_plus_v_chain(self.n, cnt, self.seed)


# The five workload laws: shapes, sizes and seeds.
WORKLOADS = {
    "poisson32_k20": Workload("poisson32_k20", "div_a_grad", n=32, n_ops=16, k=20,
                              degree=16, tol=1e-8, seed=0),
    "poisson128_k100": Workload("poisson128_k100", "div_a_grad", n=128, n_ops=200, k=100,
                                degree=20, tol=1e-8, seed=1),
    "lapv256_k400": Workload("lapv256_k400", "lap_plus_v", n=256, n_ops=1000, k=400,
                             degree=20, tol=1e-8, seed=2),
}
