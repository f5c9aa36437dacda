"""Graph and node-set generators (inputs only; no Krylov arithmetic lives here).

Each generator returns a :class:`CSRGraph` holding the CSR form of a graph Laplacian
L = D - W (Section 2.1): off-diagonal entries -w_ij < 0 for every edge, diagonal
L_ii = sum_j w_ij, zero elsewhere.  Rows are sorted by column index and contain the
diagonal entry.  Indices are int32, values float32 (the weights are drawn or given in
float32 and the diagonal is their float32 sum, so the float32 matrix is exactly what
both the oracle (promoted to float64) and the CUDA path see).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSRGraph:
    n: int
    rowptr: np.ndarray  # int32, n+1
    col: np.ndarray     # int32, nnz
    val: np.ndarray     # float32, nnz
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def unit_weight(self) -> bool:
        off = self.col != np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.rowptr))
        return bool(np.all(self.val[off] == -1.0))


def from_edges(n: int, src: np.ndarray, dst: np.ndarray, w: np.ndarray | None = None,
               meta: dict | None = None) -> CSRGraph:
    """Laplacian CSR from an undirected edge list (each edge listed once, src != dst).

    Duplicate edges are rejected (the graph is simple, Section 2.1)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if w is None:
        w = np.ones(src.shape[0], dtype=np.float32)
    w = np.asarray(w, dtype=np.float32)
    if np.any(src == dst):
        raise ValueError("self loops are not allowed")
    if np.any(w <= 0):
        raise ValueError("edge weights must be positive")
    r = np.concatenate([src, dst])
    c = np.concatenate([dst, src])
    ww = np.concatenate([w, w])
    key = r * n + c
    order = np.argsort(key, kind="stable")
    key = key[order]
    if key.size and np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate edges")
    r = r[order]
    c = c[order]
    ww = ww[order]
    # float32 diagonal = float32 sum of the row's float32 weights (summed in float64, rounded once)
    deg = np.zeros(n, dtype=np.float64)
    np.add.at(deg, r, ww.astype(np.float64))
    deg32 = deg.astype(np.float32)
    # merge the diagonal into the sorted rows
    rr = np.concatenate([r, np.arange(n, dtype=np.int64)])
    cc = np.concatenate([c, np.arange(n, dtype=np.int64)])
    vv = np.concatenate([-ww, deg32])
    order = np.argsort(rr * n + cc, kind="stable")
    rr = rr[order]
    cc = cc[order]
    vv = vv[order]
    counts = np.bincount(rr, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 indexing")
    return CSRGraph(n=n, rowptr=rowptr.astype(np.int32), col=cc.astype(np.int32),
                    val=vv.astype(np.float32), meta=dict(meta or {}))


def path_graph(n: int) -> CSRGraph:
    """Path P_n: node i joined to i+1."""
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, meta={"kind": "path", "n": n})


def cycle_graph(n: int) -> CSRGraph:
    """Cycle C_n (n >= 3)."""
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, meta={"kind": "cycle", "n": n})


def grid_graph(dims: tuple[int, ...]) -> CSRGraph:
    """Non-periodic 2-D/3-D grid with nearest-neighbour edges; row-major node index
    (the last coordinate varies fastest)."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    idx = np.arange(n).reshape(dims)
    src, dst = [], []
    for ax in range(len(dims)):
        a = np.take(idx, np.arange(dims[ax] - 1), axis=ax).ravel()
        b = np.take(idx, np.arange(1, dims[ax]), axis=ax).ravel()
        src.append(a)
        dst.append(b)
    return from_edges(n, np.concatenate(src), np.concatenate(dst),
                      meta={"kind": "grid", "dims": list(dims)})


def random_geometric_graph(n: int, mean_degree: float = 10.0, seed: int = 0,
                           permute: bool = False) -> CSRGraph:
    """Random geometric graph: n uniform points in the unit square, an edge when the
    distance is below r with (n-1) * pi * r^2 = mean_degree.  Nodes are numbered in
    row-major order of square cells of side r (cell-sorted), or randomly when permute."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    r = float(np.sqrt(mean_degree / (np.pi * max(n - 1, 1))))
    ncell = max(int(np.floor(1.0 / r)), 1)
    cx = np.minimum((pts[:, 0] * ncell).astype(np.int64), ncell - 1)
    cy = np.minimum((pts[:, 1] * ncell).astype(np.int64), ncell - 1)
    order = np.lexsort((pts[:, 0], cx, cy))
    if permute:
        order = order[rng.permutation(n)]
    pts = pts[order]
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    g = from_edges(n, pairs[:, 0], pairs[:, 1],
                   meta={"kind": "rgg", "n": n, "mean_degree": mean_degree, "radius": r,
                         "seed": seed, "permuted": permute})
    g.meta["realised_mean_degree"] = 2.0 * pairs.shape[0] / n
    return g


_BA_LIB = None


def _ba_lib():
    global _BA_LIB
    if _BA_LIB is not None:
        return _BA_LIB
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "ba.c")
    so = os.path.join(here, "_ba.so")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.ba_edges.restype = ctypes.c_int64
    lib.ba_edges.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                             ctypes.c_void_p, ctypes.c_void_p]
    _BA_LIB = lib
    return lib


def barabasi_albert_graph(n: int, edges_per_node: int = 5, seed: int = 0,
                          weighted: bool = False) -> CSRGraph:
    """Barabasi-Albert preferential attachment: a seed clique on edges_per_node + 1
    nodes, then each new node joins edges_per_node distinct earlier nodes drawn from the
    list of edge endpoints (probability proportional to degree).  Weights, when asked
    for, are uniform in [0.5, 1.5] (float32)."""
    k = int(edges_per_node)
    if n <= k + 1:
        raise ValueError("n must exceed edges_per_node + 1")
    ne = (k + 1) * k // 2 + (n - k - 1) * k
    src = np.empty(ne, dtype=np.int32)
    dst = np.empty(ne, dtype=np.int32)
    got = _ba_lib().ba_edges(n, k, np.uint64(seed), src.ctypes.data, dst.ctypes.data)
    assert got == ne, (got, ne)
    w = None
    if weighted:
        rng = np.random.default_rng(seed + 0x5EED)
        w = rng.uniform(0.5, 1.5, size=ne).astype(np.float32)
    return from_edges(n, src, dst, w, meta={"kind": "ba", "n": n, "edges_per_node": k,
                                            "seed": seed, "weighted": weighted})


def random_weighted_graph(n: int, p: float, seed: int = 0) -> CSRGraph:
    """Erdos-Renyi G(n, p) with float32 weights uniform in [0.5, 1.5]; small cases only."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    w = rng.uniform(0.5, 1.5, size=int(keep.sum())).astype(np.float32)
    return from_edges(n, iu[keep], ju[keep], w, meta={"kind": "gnp", "n": n, "p": p, "seed": seed})


def sample_nodes(n: int, M: int, seed: int = 0) -> np.ndarray:
    """M distinct nodes drawn uniformly without replacement (int32)."""
    if M > n:
        raise ValueError("M > n")
    rng = np.random.default_rng(seed)
    return rng.choice(n, size=M, replace=False).astype(np.int32)
