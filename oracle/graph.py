"""Graph estimate, core/halo partition, gather and collect (CPU reference).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* graph_build: Sec. "Estimating the connectivity graph" -- an edge (i, j),
  i != j, when |H_ij| > tau or |D_prev,ij| > tau, symmetrised; optionally the
  paths of length two of that graph are added (the favourite estimate) which is
  also the "H^m with m = 2" ad hoc estimate when no D_prev is given.
* partition: Fig. 1 and Sec. "Choosing the graph partitioning" -- disjoint
  cores; each subgraph is its core plus the halo of directly connected
  vertices; vertices of a subgraph are kept in ascending global order.
* gather / collect_columns: Eq. sub_f and Eq. dCollect -- principal
  submatrices x^(i) = X[S_i, S_i] and the column-by-column collect of the
  core columns (each core column carries the core rows and the halo rows).
* polynomial_on_graph: Fig. 0 / Eq. f_tau -- a matrix polynomial built by
  left multiplication, with everything outside the graph removed after every
  single product.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Adjacency:
    n: int
    indptr: np.ndarray   # int64 (n+1)
    indices: np.ndarray  # int32, ascending per row, no self loops

    def neighbours(self, i: int) -> np.ndarray:
        return self.indices[self.indptr[i]:self.indptr[i + 1]]

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n), dtype=bool)
        rows = np.repeat(np.arange(self.n), np.diff(self.indptr))
        a[rows, self.indices] = True
        return a


@dataclass
class Partition:
    n: int
    core_ptr: np.ndarray   # int64 (n_sub+1)
    core_idx: np.ndarray   # int32, ascending per core
    sub_ptr: np.ndarray    # int64 (n_sub+1)
    sub_idx: np.ndarray    # int32, ascending per subgraph (core and halo)
    core_pos: np.ndarray   # int32, local position in S_i of every core vertex (aligned with core_idx)

    @property
    def n_sub(self) -> int:
        return len(self.core_ptr) - 1

    def core(self, i: int) -> np.ndarray:
        return self.core_idx[self.core_ptr[i]:self.core_ptr[i + 1]]

    def sub(self, i: int) -> np.ndarray:
        return self.sub_idx[self.sub_ptr[i]:self.sub_ptr[i + 1]]

    def local_core(self, i: int) -> np.ndarray:
        return self.core_pos[self.core_ptr[i]:self.core_ptr[i + 1]]

    def sizes(self) -> np.ndarray:
        return np.diff(self.sub_ptr)


def _pattern(n, indptr, indices, data, tau):
    rows = np.repeat(np.arange(n), np.diff(np.asarray(indptr)))
    keep = np.abs(np.asarray(data)) > tau
    r, c = rows[keep], np.asarray(indices)[keep]
    off = r != c
    return r[off], c[off]


def graph_build(n, h_indptr, h_indices, h_data, tau, *, paths2=False, d_prev=None) -> Adjacency:
    """Thresholded, symmetrised graph of H (and of D_prev), optionally squared.

    ``d_prev`` is ``(ptr, idx, val)`` of a compressed sparse matrix (rows or
    columns -- the result is symmetrised, so the orientation does not matter).
    The threshold is strict: |x| > tau.  Self loops are never edges.
    """
    r, c = _pattern(n, h_indptr, h_indices, h_data, tau)
    rs, cs = [r, c], [c, r]
    if d_prev is not None:
        dr, dc = _pattern(n, *d_prev, tau)
        rs += [dr, dc]
        cs += [dc, dr]
    rr = np.concatenate(rs)
    cc = np.concatenate(cs)
    a = sp.csr_matrix((np.ones(len(rr), dtype=np.int64), (rr, cc)), shape=(n, n))
    a.sum_duplicates()
    a.data[:] = 1
    if paths2:
        a2 = (a @ a).tocsr()
        a = (a + a2).tocsr()
        a.sum_duplicates()
        a.setdiag(0)
        a.eliminate_zeros()
        a.data[:] = 1
    a.sort_indices()
    return Adjacency(n, a.indptr.astype(np.int64), a.indices.astype(np.int32))


def partition(adj: Adjacency, groups=None, target_core_size: int = 6) -> Partition:
    """Cores from group ids (ascending id, empty ids skipped) or consecutive blocks.

    halo_i = (union of the neighbours of core_i) minus core_i, and
    S_i = sorted(core_i + halo_i).
    """
    n = adj.n
    if groups is None:
        gid = np.arange(n) // int(target_core_size)
    else:
        gid = np.asarray(groups, dtype=np.int64)
    order = np.lexsort((np.arange(n), gid))
    uniq, start = np.unique(gid[order], return_index=True)
    bounds = list(start) + [n]
    core_ptr, core_idx, sub_ptr, sub_idx, core_pos = [0], [], [0], [], []
    for i in range(len(uniq)):
        core = np.sort(order[bounds[i]:bounds[i + 1]])
        halo = set()
        for v in core:
            halo.update(int(u) for u in adj.neighbours(int(v)))
        s = np.array(sorted(set(int(v) for v in core) | halo), dtype=np.int64)
        core_idx.append(core)
        sub_idx.append(s)
        core_pos.append(np.searchsorted(s, core))
        core_ptr.append(core_ptr[-1] + len(core))
        sub_ptr.append(sub_ptr[-1] + len(s))
    return Partition(n, np.array(core_ptr, dtype=np.int64),
                     np.concatenate(core_idx).astype(np.int32),
                     np.array(sub_ptr, dtype=np.int64),
                     np.concatenate(sub_idx).astype(np.int32),
                     np.concatenate(core_pos).astype(np.int32))


def partition_capped(adj: Adjacency, groups, subgroups, max_sub: int) -> Partition:
    """Cores from group ids, with a cap on the subgraph size.

    The paper leaves the partition free (Sec. "Choosing the graph
    partitioning").  Rule: partition by group (key g); every core whose
    subgraph holds more than ``max_sub`` vertices is replaced by one core per
    subgroup id among its vertices (key G + subgroup, G above every group
    id); every such core still over the cap is replaced by one core per
    vertex (key G + S + v, S above every subgroup id).  Cores are ordered by
    ascending key.
    """
    key = np.asarray(groups, dtype=np.int64)
    sub = np.asarray(subgroups, dtype=np.int64)
    n = adj.n
    part = partition(adj, key)
    for level, base in ((1, int(key.max()) + 1), (2, int(key.max()) + 1 + int(sub.max()) + 1)):
        sizes = np.diff(part.sub_ptr)
        big = {int(key[part.core_idx[part.core_ptr[k]]]) for k in np.nonzero(sizes > max_sub)[0]}
        if not big:
            break
        piece = sub if level == 1 else np.arange(n)
        key = np.array([base + piece[v] if int(key[v]) in big else key[v] for v in range(n)], dtype=np.int64)
        part = partition(adj, key)
    return part


def gather(X, s: np.ndarray) -> np.ndarray:
    """Principal submatrix X[S, S] (X dense, or a scipy sparse matrix)."""
    if sp.issparse(X):
        return X[s][:, s].toarray()
    return np.asarray(X)[np.ix_(s, s)]


def collect_columns(core_blocks, part: Partition):
    """Column collect {x_c^(i)}: a ragged CSC matrix (col_ptr, row_idx, val).

    ``core_blocks[i]`` holds the core columns of block i, shape
    (|S_i|, |core_i|), in the order of ``part.core(i)``.  Column j (a core
    vertex of subgraph i) of the result holds that column on the rows S_i.
    """
    n = part.n
    owner = np.empty(n, dtype=np.int64)
    slot = np.empty(n, dtype=np.int64)
    for i in range(part.n_sub):
        c = part.core(i)
        owner[c] = i
        slot[c] = np.arange(len(c))
    sizes = part.sizes()
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    col_ptr[1:] = np.cumsum(sizes[owner])
    row_idx = np.empty(col_ptr[-1], dtype=np.int32)
    val = np.empty(col_ptr[-1])
    for j in range(n):
        i = owner[j]
        a, b = col_ptr[j], col_ptr[j + 1]
        row_idx[a:b] = part.sub(i)
        val[a:b] = core_blocks[i][:, slot[j]]
    return col_ptr, row_idx, val


def csc_to_dense(n, col_ptr, row_idx, val) -> np.ndarray:
    out = np.zeros((n, n))
    cols = np.repeat(np.arange(n), np.diff(col_ptr))
    out[row_idx, cols] = val
    return out


def column_mask(part: Partition) -> np.ndarray:
    """M[r, j] = 1 when row r lies in the subgraph whose core holds column j."""
    m = np.zeros((part.n, part.n), dtype=bool)
    for i in range(part.n_sub):
        s = part.sub(i)
        m[np.ix_(s, part.core(i))] = True
    return m


def polynomial_on_graph(X: np.ndarray, mask: np.ndarray, coeffs) -> np.ndarray:
    """p_G(X) = sum_k a_k T_k with T_0 = I|_G, T_k = (X T_{k-1})|_G (Fig. 0)."""
    t = np.eye(X.shape[0]) * mask
    out = coeffs[0] * t
    for a in coeffs[1:]:
        t = (X @ t) * mask
        out = out + a * t
    return out


def dense_polynomial(x: np.ndarray, coeffs) -> np.ndarray:
    """The same polynomial on a dense principal submatrix, with no mask."""
    t = np.eye(x.shape[0])
    out = coeffs[0] * t
    for a in coeffs[1:]:
        t = x @ t
        out = out + a * t
    return out
