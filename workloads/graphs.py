"""Seeded synthetic graphs in CSR form.

Every generator returns a :class:`CSRGraph` describing a simple undirected
graph: symmetric adjacency, sorted column indices per row, no duplicate
entries and no self-loops.  The paper's inputs are symmetrised as A + A^T + I
and reduced to their largest connected component (Sec. 6.1); the diagonal
``I`` is the Laplacian's business, so the adjacency stored here carries only
off-diagonal entries and the structure count with the diagonal is
``nnz + n``.

Random draws come from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) so that a
graph is the same bit for bit on every machine and numpy version.
"""

from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

# graphs at least this large use the C helpers of _gen.c when gcc is available
_NATIVE_MIN = 1 << 22


def _native_lib():
    from . import _native
    return _native.lib()


_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied element-wise (uint64, wrapping)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        base = np.array([(seed * 0x632BE59BD9B4E019 + stream * 0x9E3779B97F4A7C15 + 0x5851F42D4C957F2D)
                         & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return _mix64(base)[0]


def uniform01(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` doubles in [0, 1) from counter ``offset .. offset+count-1``."""
    key = _stream_key(seed, stream)
    ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix64(key + ctr * _GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class CSRGraph:
    """Undirected simple graph: ``row_ptr`` int64 (n+1), ``col`` int32 (nnz)."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: Optional[np.ndarray] = None  # float32 per stored entry, symmetric
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def rows(self) -> np.ndarray:
        """Row index of every stored entry (int64)."""
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))


def _from_sorted_pairs(n: int, rows: np.ndarray, cols: np.ndarray, w=None, name="") -> CSRGraph:
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSRGraph(n=n, row_ptr=row_ptr, col=cols.astype(np.int32), w=w, name=name)


def symmetrize_edges(n: int, src: np.ndarray, dst: np.ndarray, name: str = "") -> CSRGraph:
    """Simple undirected graph from a directed edge list: A + A^T with
    self-loops dropped and duplicate entries merged."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    a = np.minimum(src[keep], dst[keep])
    b = np.maximum(src[keep], dst[keep])
    key = np.unique(a * n + b)
    a = key // n
    b = key % n
    del key
    rows = np.concatenate([a, b])
    cols = np.concatenate([b, a])
    del a, b
    order = np.argsort(rows * n + cols, kind="stable")
    rows = rows[order]
    cols = cols[order]
    return _from_sorted_pairs(n, rows, cols, name=name)


def _offsets_csr(shape, offsets, periodic: bool, name: str) -> CSRGraph:
    """CSR of a structured grid whose vertex (x, y, z, ...) is numbered
    x + nx*(y + ny*z ...), connected to every listed offset."""
    dims = list(shape)
    n = int(np.prod(dims))
    coords = np.indices(dims[::-1]).reshape(len(dims), -1)[::-1]  # coords[d] of vertex i
    strides = np.cumprod([1] + dims[:-1])
    rows_l, cols_l = [], []
    for off in offsets:
        valid = np.ones(n, dtype=bool)
        nbr = np.zeros(n, dtype=np.int64)
        for d, o in enumerate(off):
            c = coords[d] + o
            if periodic:
                c = np.mod(c, dims[d])
            else:
                valid &= (c >= 0) & (c < dims[d])
            nbr += np.clip(c, 0, dims[d] - 1) * strides[d]
        idx = np.nonzero(valid)[0]
        rows_l.append(idx)
        cols_l.append(nbr[idx])
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    keep = rows != cols
    rows, cols = rows[keep], cols[keep]
    key = np.unique(rows * n + cols)
    rows = key // n
    cols = key % n
    g = _from_sorted_pairs(n, rows, cols, name=name)
    g.meta["shape"] = tuple(dims)
    g.meta["periodic"] = periodic
    return g


def _grid3d_fast(nx: int, ny: int, nz: int, offsets, name: str) -> CSRGraph:
    """Non-periodic grid built row by row without a global sort (large meshes)."""
    n = nx * ny * nz
    offs = sorted(offsets, key=lambda o: o[0] + nx * (o[1] + ny * o[2]))
    x = np.tile(np.arange(nx, dtype=np.int32), ny * nz)
    y = np.tile(np.repeat(np.arange(ny, dtype=np.int32), nx), nz)
    z = np.repeat(np.arange(nz, dtype=np.int32), nx * ny)
    masks = []
    for dx, dy, dz in offs:
        m = np.ones(n, dtype=bool)
        if dx:
            m &= (x + dx >= 0) & (x + dx < nx)
        if dy:
            m &= (y + dy >= 0) & (y + dy < ny)
        if dz:
            m &= (z + dz >= 0) & (z + dz < nz)
        masks.append(m)
    del x, y, z
    counts = np.zeros(n, dtype=np.int64)
    for m in masks:
        counts += m
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = np.empty(int(row_ptr[-1]), dtype=np.int32)
    run = row_ptr[:-1].copy()
    ids = np.arange(n, dtype=np.int64)
    for (dx, dy, dz), m in zip(offs, masks):
        idx = ids[m]
        col[run[m]] = (idx + dx + nx * (dy + ny * dz)).astype(np.int32)
        run[m] += 1
    g = CSRGraph(n=n, row_ptr=row_ptr, col=col, name=name)
    g.meta["shape"] = (nx, ny, nz)
    g.meta["periodic"] = False
    return g


def path_graph(n: int) -> CSRGraph:
    return _offsets_csr((n,), [(-1,), (1,)], False, f"path{n}")


def cycle_graph(n: int) -> CSRGraph:
    if n < 3:
        raise ValueError("cycle needs n >= 3")
    return _offsets_csr((n,), [(-1,), (1,)], True, f"cycle{n}")


def grid2d(nx: int, ny: int, periodic: bool = False) -> CSRGraph:
    """5-point grid graph (4-neighbour mesh) on nx x ny vertices."""
    if periodic and min(nx, ny) < 3:
        raise ValueError("periodic grid needs every side >= 3")
    return _offsets_csr((nx, ny), [(-1, 0), (1, 0), (0, -1), (0, 1)], periodic,
                        f"grid2d_{nx}x{ny}{'_torus' if periodic else ''}")


def _stencil3d(points: int):
    if points == 7:
        return [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    if points == 27:
        return [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                if (dx, dy, dz) != (0, 0, 0)]
    raise ValueError("stencil must be 7 or 27")


def grid3d(nx: int, ny: int, nz: int, points: int = 27, periodic: bool = False) -> CSRGraph:
    """3D structured mesh graph with a 7- or 27-point stencil (the 27-point
    box is the structure of the Brick3D meshes of Sec. 6.1)."""
    offs = _stencil3d(points)
    name = f"grid3d{points}_{nx}x{ny}x{nz}{'_torus' if periodic else ''}"
    if periodic:
        if min(nx, ny, nz) < 3:
            raise ValueError("periodic grid needs every side >= 3")
        return _offsets_csr((nx, ny, nz), offs, True, name)
    return _grid3d_fast(nx, ny, nz, offs, name)


def star_graph(n: int) -> CSRGraph:
    """Vertex 0 joined to vertices 1..n-1 (a maximally irregular degree profile)."""
    src = np.zeros(n - 1, dtype=np.int64)
    dst = np.arange(1, n, dtype=np.int64)
    return symmetrize_edges(n, src, dst, name=f"star{n}")


def erdos_renyi(n: int, p: float, seed: int) -> CSRGraph:
    """G(n, p) on small n (all n(n-1)/2 pairs are drawn)."""
    iu, ju = np.triu_indices(n, k=1)
    u = uniform01(seed, 11, iu.size)
    keep = u < p
    return symmetrize_edges(n, iu[keep], ju[keep], name=f"er{n}_{p}_{seed}")


def largest_component(g: CSRGraph, native: Optional[bool] = None) -> CSRGraph:
    """Induced subgraph on the largest connected component, vertices kept in
    their original relative order (Sec. 6.1 keeps the largest component)."""
    native = _native_lib() if (native or (native is None and g.nnz >= _NATIVE_MIN)) else None
    if native is not None:
        return _largest_component_native(native, g)
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    data = np.ones(g.nnz, dtype=np.int8)
    a = sp.csr_matrix((data, g.col, g.row_ptr), shape=(g.n, g.n))
    ncomp, labels = connected_components(a, directed=False)
    if ncomp == 1:
        g.meta["n_before_lcc"] = g.n
        return g
    big = np.argmax(np.bincount(labels))
    keep = np.nonzero(labels == big)[0]
    newid = -np.ones(g.n, dtype=np.int64)
    newid[keep] = np.arange(keep.size)
    rows = g.rows()
    m = labels[rows] == big
    r2 = newid[rows[m]]
    c2 = newid[g.col[m].astype(np.int64)]
    w2 = None if g.w is None else g.w[m]
    out = _from_sorted_pairs(int(keep.size), r2, c2, w=w2, name=g.name + "_lcc")
    out.meta = dict(g.meta)
    out.meta["n_before_lcc"] = g.n
    out.meta["components"] = int(ncomp)
    return out


def _largest_component_native(L, g: CSRGraph) -> CSRGraph:
    """largest_component through the C helpers: same components, same
    tie rule (the component whose smallest vertex comes first)."""
    labels = np.empty(g.n, dtype=np.int64)
    ncomp = L.gen_components(g.n, g.row_ptr.ctypes.data, g.col.ctypes.data, labels.ctypes.data)
    if ncomp < 0:
        raise MemoryError("components")
    if ncomp == 1:
        g.meta["n_before_lcc"] = g.n
        return g
    sizes = np.bincount(labels)
    big = int(np.argmax(sizes))
    nk = int(sizes[big])
    kept = int(np.sum(np.diff(g.row_ptr)[labels == big]))
    rp = np.empty(nk + 1, dtype=np.int64)
    col = np.empty(kept, dtype=np.int32)
    w = None if g.w is None else np.empty(kept, dtype=np.float32)
    e = L.gen_induced(g.n, g.row_ptr.ctypes.data, g.col.ctypes.data, None if g.w is None else g.w.ctypes.data,
                      labels.ctypes.data, big, rp.ctypes.data, col.ctypes.data, None if w is None else w.ctypes.data)
    if e != kept:
        raise RuntimeError("induced subgraph size mismatch")
    out = CSRGraph(n=nk, row_ptr=rp, col=col, w=w, name=g.name + "_lcc")
    out.meta = dict(g.meta)
    out.meta["n_before_lcc"] = g.n
    out.meta["components"] = int(ncomp)
    return out


def _rmat_native(L, scale: int, m: int, a: float, ab: float, abc: float, seed: int, name: str) -> CSRGraph:
    n = 1 << scale
    keys = np.empty(m, dtype=np.uint64)
    L.gen_rmat_keys(scale, m, a, ab, abc, seed, keys.ctypes.data)
    tmp = np.empty(m, dtype=np.uint64)
    u = L.gen_sort_unique(keys.ctypes.data, tmp.ctypes.data, m, 2 * scale)
    del tmp
    if u < 0:
        raise MemoryError("sort")
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(2 * u, dtype=np.int32)
    if L.gen_csr_from_keys(n, keys.ctypes.data, u, row_ptr.ctypes.data, col.ctypes.data) != 0:
        raise MemoryError("csr")
    return CSRGraph(n=n, row_ptr=row_ptr, col=col, name=name)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 3, lcc: bool = True, chunk: int = 1 << 24,
         native: Optional[bool] = None) -> CSRGraph:
    """R-MAT graph (Chakrabarti, Zhan, Faloutsos 2004): ``edge_factor * 2^scale``
    edge draws, each descending ``scale`` quadrant choices with probabilities
    (a, b, c, d).  Symmetrised, deduplicated, self-loops dropped and reduced to
    the largest component.  Vertex ids are not permuted.  ``native`` selects
    the C helpers (same graph; default: for large graphs when available)."""
    n = 1 << scale
    m = edge_factor * n
    ab, abc = a + b, a + b + c
    L = _native_lib() if (native or (native is None and m >= _NATIVE_MIN)) else None
    if native and L is None:
        raise RuntimeError("native graph helpers unavailable")
    if L is not None:
        g = _rmat_native(L, scale, m, a, ab, abc, seed, f"rmat{scale}_ef{edge_factor}_s{seed}")
        g.meta["edge_draws"] = m
        return _largest_component_native(L, g) if lcc else g
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        s = np.zeros(hi - lo, dtype=np.int64)
        d = np.zeros(hi - lo, dtype=np.int64)
        for lvl in range(scale):
            u = uniform01(seed, 100 + lvl, hi - lo, offset=lo)
            sb = u >= ab
            db = ((u >= a) & (u < ab)) | (u >= abc)
            bit = np.int64(1) << np.int64(scale - 1 - lvl)
            s |= sb.astype(np.int64) * bit
            d |= db.astype(np.int64) * bit
        src[lo:hi] = s
        dst[lo:hi] = d
    g = symmetrize_edges(n, src, dst, name=f"rmat{scale}_ef{edge_factor}_s{seed}")
    del src, dst
    g.meta["edge_draws"] = m
    return largest_component(g, native=native) if lcc else g


def rgg(n: int, radius: Optional[float] = None, seed: int = 4, lcc: bool = True,
        native: Optional[bool] = None) -> CSRGraph:
    """Random geometric graph: n points uniform in the unit square, joined
    when at most ``radius`` apart (default sqrt(8 / (pi n)), mean degree ~8).
    ``native`` selects the C helpers (same graph; default: when available)."""
    if radius is None:
        radius = float(np.sqrt(8.0 / (np.pi * n)))
    L = _native_lib() if (native or native is None) else None
    if native and L is None:
        raise RuntimeError("native graph helpers unavailable")
    if L is not None:
        cap = 16 * n + 1024
        while True:
            keys = np.empty(cap, dtype=np.uint64)
            m = L.gen_rgg_keys(n, radius, seed, keys.ctypes.data, cap)
            if m >= 0:
                break
            cap *= 2
        keys = keys[:m].copy()
        tmp = np.empty(max(m, 1), dtype=np.uint64)
        u = L.gen_sort_unique(keys.ctypes.data, tmp.ctypes.data, m, 2 * max(1, int(n - 1).bit_length()))
        row_ptr = np.empty(n + 1, dtype=np.int64)
        col = np.empty(2 * u, dtype=np.int32)
        L.gen_csr_from_keys(n, keys.ctypes.data, u, row_ptr.ctypes.data, col.ctypes.data)
        g = CSRGraph(n=n, row_ptr=row_ptr, col=col, name=f"rgg{n}_s{seed}")
        g.meta["radius"] = radius
        return _largest_component_native(L, g) if lcc else g
    from scipy.spatial import cKDTree
    x = uniform01(seed, 21, n)
    y = uniform01(seed, 22, n)
    pts = np.stack([x, y], axis=1)
    pairs = cKDTree(pts).query_pairs(radius, output_type="ndarray")
    g = symmetrize_edges(n, pairs[:, 0], pairs[:, 1], name=f"rgg{n}_s{seed}")
    g.meta["radius"] = radius
    return largest_component(g) if lcc else g


def rgg_batch(count: int = 2000, n_min: float = 1e3, n_max: float = 2e5, seed: int = 4) -> list:
    """The batch workload: ``count`` random geometric graphs with sizes
    log-uniform in [n_min, n_max] (n_i = floor(exp(ln n_min + u_i ln(n_max /
    n_min))), u_i draw i + 1 of stream 61), radius sqrt(8 / (pi n_i)) (mean
    degree about 8), graph i drawn with seed + i and reduced to its largest
    component."""
    u = uniform01(seed, 61, count)
    sizes = np.floor(np.exp(np.log(n_min) + u * np.log(n_max / n_min))).astype(np.int64)
    return [rgg(int(n), seed=seed + i) for i, n in enumerate(sizes)]


def concat_graphs(graphs) -> tuple:
    """Block-diagonal union of graphs (vertex ids shifted, weights kept when
    every graph has them) and the offsets graph_ptr[count + 1] of each
    graph's vertex range: the input of a batched partition."""
    gptr = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        gptr[i + 1] = gptr[i] + g.n
    eptr = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        eptr[i + 1] = eptr[i] + g.nnz
    row_ptr = np.zeros(int(gptr[-1]) + 1, dtype=np.int64)
    col = np.empty(int(eptr[-1]), dtype=np.int32)
    weighted = all(g.w is not None for g in graphs)
    w = np.empty(int(eptr[-1]), dtype=np.float32) if weighted else None
    for i, g in enumerate(graphs):
        row_ptr[gptr[i] + 1:gptr[i + 1] + 1] = g.row_ptr[1:] + eptr[i]
        col[eptr[i]:eptr[i + 1]] = g.col + np.int32(gptr[i])
        if weighted:
            w[eptr[i]:eptr[i + 1]] = g.w
    out = CSRGraph(n=int(gptr[-1]), row_ptr=row_ptr, col=col, w=w, name=f"batch{len(graphs)}")
    return out, gptr


def random_edge_weights(g: CSRGraph, lo: float = 0.5, hi: float = 1.5, seed: int = 5,
                        native: Optional[bool] = None) -> CSRGraph:
    """Attach FP32 weights uniform in [lo, hi), one draw per undirected edge
    (keyed by the unordered pair, so the weight matrix is symmetric)."""
    L = _native_lib() if (native or (native is None and g.nnz >= _NATIVE_MIN)) else None
    if L is not None:
        w = np.empty(g.nnz, dtype=np.float32)
        L.gen_edge_weights(g.n, g.row_ptr.ctypes.data, g.col.ctypes.data, float(lo), float(hi), seed, w.ctypes.data)
        return dataclasses.replace(g, w=w, name=g.name + "_w", meta=dict(g.meta))
    rows = g.rows()
    cols = g.col.astype(np.int64)
    a = np.minimum(rows, cols)
    b = np.maximum(rows, cols)
    key = _stream_key(seed, 31)
    with np.errstate(over="ignore"):
        z = _mix64(key + (a.astype(np.uint64) * np.uint64(g.n) + b.astype(np.uint64) + np.uint64(1)) * _GOLDEN)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    w = (lo + (hi - lo) * u).astype(np.float32)
    return dataclasses.replace(g, w=w, name=g.name + "_w", meta=dict(g.meta))


def random_vertex_weights(n: int, lo: int = 1, hi: int = 10, seed: int = 6) -> np.ndarray:
    """int64 vertex weights uniform in [lo, hi]."""
    u = uniform01(seed, 41, n)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def random_coords(n: int, dim: int, seed: int, dtype=np.float64, ties: bool = False) -> np.ndarray:
    """Row-major n x dim coordinates uniform in [-1, 1); with ``ties`` the
    values are snapped to a coarse lattice so that many coordinates repeat and
    signed zeros appear."""
    u = uniform01(seed, 51, n * dim).reshape(n, dim)
    x = 2.0 * u - 1.0
    if ties:
        x = np.round(x * 4.0) / 4.0
        neg = uniform01(seed, 52, n * dim).reshape(n, dim) < 0.5
        x = np.where((x == 0.0) & neg, -0.0, x)
    return np.ascontiguousarray(x.astype(dtype))
