"""Seeded synthetic hypergraphs and vectors shaped like the paper's workloads.

This module only draws random structure (edge sizes, members, x vectors) and
prepares it (largest connected component, relabelling).  It contains none of
the S^3TTVc arithmetic, so both the CPU oracle and the CUDA path can take
their inputs from it without sharing any of the method's code.

Hypergraphs are returned as ``(n, edge_ptr, members)``: ``edge_ptr`` is int64
of length m+1, ``members`` is int32 of length edge_ptr[-1]; edge ``i`` owns
``members[edge_ptr[i]:edge_ptr[i+1]]`` (0-based node ids, no repeats inside an
edge, arbitrary order).

Workload recipes (sizes and distributions of the paper's Sec. V data, Table I):
  * ``uniform_sizes``      -- sizes uniform on {lo..hi}, members uniform.
  * ``zipf_sizes``         -- P(s) proportional to s^-alpha on {lo..hi}.
  * ``geometric_sizes``    -- P(s) proportional to (1-p)^(s-lo) on {lo..hi}.
  * ``chung_lu_members``   -- node weights w_i ~ i^(-1/(gamma-1)) over a random
                              id permutation (power-law degree, exponent gamma);
                              members drawn by weight, repeats inside an edge
                              redrawn (rejection).
  * ``sunflower`` / ``nested`` -- the sub-structures of Fig. 3.
  * ``paper_s_family``     -- the synthetic S1-S4 family of Table I.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Hypergraph", "uniform_sizes", "zipf_sizes", "geometric_sizes",
    "uniform_members", "chung_lu_members", "largest_component",
    "random_uniform_hypergraph", "config_small", "config_powerlaw",
    "config_large_rank", "config_batched", "tiny_case", "fig1_example",
    "sunflower", "nested", "paper_s_family", "x_uniform", "x_constant", "x_degree_like",
]


class Hypergraph:
    """A plain container: node count, CSR edge pointer and members."""

    def __init__(self, n, edge_ptr, members, rank=None, name=""):
        self.n = int(n)
        self.edge_ptr = np.ascontiguousarray(edge_ptr, dtype=np.int64)
        self.members = np.ascontiguousarray(members, dtype=np.int32)
        sizes = np.diff(self.edge_ptr)
        self.rank = int(rank) if rank is not None else (int(sizes.max()) if sizes.size else 0)
        self.name = name

    @property
    def m(self):
        return self.edge_ptr.size - 1

    @property
    def nnz(self):
        return int(self.edge_ptr[-1])

    def sizes(self):
        return np.diff(self.edge_ptr)

    def edges(self):
        """List of tuples (slow; for small cases)."""
        p, mem = self.edge_ptr, self.members
        return [tuple(int(v) for v in mem[p[i]:p[i + 1]]) for i in range(self.m)]

    def degrees(self):
        return np.bincount(self.members, minlength=self.n).astype(np.int64)

    def __repr__(self):
        return f"Hypergraph({self.name!r}, n={self.n}, m={self.m}, nnz={self.nnz}, rank={self.rank})"


# ----------------------------------------------------------------- sizes ---

def _force_max(sizes, hi, rng):
    """Make sure the realised maximum size equals ``hi`` (the configured rank)."""
    if sizes.size and sizes.max() < hi:
        sizes[rng.integers(0, sizes.size)] = hi
    return sizes


def uniform_sizes(m, lo, hi, rng):
    return _force_max(rng.integers(lo, hi + 1, size=m).astype(np.int64), hi, rng)


def zipf_sizes(m, alpha, lo, hi, rng):
    vals = np.arange(lo, hi + 1)
    p = vals.astype(np.float64) ** (-alpha)
    p /= p.sum()
    return _force_max(rng.choice(vals, size=m, p=p).astype(np.int64), hi, rng)


def geometric_sizes(m, prob, lo, hi, rng):
    vals = np.arange(lo, hi + 1)
    p = (1.0 - prob) ** (vals - lo).astype(np.float64)
    p /= p.sum()
    return _force_max(rng.choice(vals, size=m, p=p).astype(np.int64), hi, rng)


# --------------------------------------------------------------- members ---

def _fix_repeats(edge_of, draw, resample, rng, max_rounds=1000):
    """Redraw members that repeat inside their edge until none do.

    Every later occurrence of a node inside an edge is redrawn (in position
    order); after the first pass only the edges that had a repeat are checked
    again.  ``edge_of`` is non-decreasing (edges are contiguous)."""
    span = int(draw.max()) + 1 if draw.size else 1
    m = int(edge_of[-1]) + 1 if edge_of.size else 0
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(edge_of, minlength=m), out=ptr[1:])
    idx = np.arange(draw.size, dtype=np.int64)
    for _ in range(max_rounds):
        key = edge_of[idx] * span + draw[idx]
        order = np.argsort(key, kind="stable")
        ks = key[order]
        same = ks[1:] == ks[:-1]
        if not same.any():
            return draw
        dup = np.sort(idx[order[1:][same]])
        new = resample(dup.size)
        span = max(span, int(new.max()) + 1)
        draw[dup] = new
        bad = np.unique(edge_of[dup])
        lens = ptr[bad + 1] - ptr[bad]
        starts = np.repeat(ptr[bad] - np.concatenate(([0], np.cumsum(lens)[:-1])), lens)
        idx = starts + np.arange(int(lens.sum()), dtype=np.int64)
    raise RuntimeError("could not draw members without repeats")


def uniform_members(sizes, n, rng):
    sizes = np.asarray(sizes, dtype=np.int64)
    if sizes.size and sizes.max() > n:
        raise ValueError("edge larger than node count")
    total = int(sizes.sum())
    edge_of = np.repeat(np.arange(sizes.size, dtype=np.int64), sizes)
    draw = rng.integers(0, n, size=total).astype(np.int64)
    draw = _fix_repeats(edge_of, draw, lambda k: rng.integers(0, n, size=k), rng)
    ptr = np.zeros(sizes.size + 1, dtype=np.int64)
    np.cumsum(sizes, out=ptr[1:])
    return ptr, draw.astype(np.int32)


def chung_lu_members(sizes, n, gamma, rng):
    """Preferential membership: weight of the node of rank i is i^(-1/(gamma-1))."""
    sizes = np.asarray(sizes, dtype=np.int64)
    ranks = np.arange(1, n + 1, dtype=np.float64)
    w = ranks ** (-1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    perm = rng.permutation(n).astype(np.int64)

    def draw_k(k):
        r = np.searchsorted(cdf, rng.random(k), side="right")
        return perm[np.minimum(r, n - 1)]

    total = int(sizes.sum())
    edge_of = np.repeat(np.arange(sizes.size, dtype=np.int64), sizes)
    draw = _fix_repeats(edge_of, draw_k(total), draw_k, rng)
    ptr = np.zeros(sizes.size + 1, dtype=np.int64)
    np.cumsum(sizes, out=ptr[1:])
    return ptr, draw.astype(np.int32)


def largest_component(hg):
    """Restrict to the largest connected component and relabel nodes 0..n'-1.

    Connectivity is taken on the node/edge incidence graph; nodes keep their
    relative order.  Returns (Hypergraph, kept_node_ids).
    """
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    n, m = hg.n, hg.m
    edge_of = np.repeat(np.arange(m, dtype=np.int64), hg.sizes())
    rows = hg.members.astype(np.int64)
    cols = n + edge_of
    a = sp.coo_matrix((np.ones(rows.size, dtype=np.int8), (rows, cols)), shape=(n + m, n + m))
    ncomp, lab = connected_components(a, directed=False)
    node_lab = lab[:n]
    deg = hg.degrees()
    # the largest component counted in nodes that belong to at least one edge
    counts = np.bincount(node_lab[deg > 0], minlength=ncomp)
    big = int(np.argmax(counts))
    keep_node = (node_lab == big) & (deg > 0)
    keep_edge = lab[n:] == big
    new_id = -np.ones(n, dtype=np.int64)
    kept = np.nonzero(keep_node)[0]
    new_id[kept] = np.arange(kept.size)
    sizes = hg.sizes()[keep_edge]
    ptr = np.zeros(sizes.size + 1, dtype=np.int64)
    np.cumsum(sizes, out=ptr[1:])
    mask = np.repeat(keep_edge, hg.sizes())
    mem = new_id[hg.members[mask].astype(np.int64)]
    assert (mem >= 0).all()
    out = Hypergraph(kept.size, ptr, mem.astype(np.int32), rank=hg.rank, name=hg.name + "-lcc")
    return out, kept


# ------------------------------------------------------------- workloads ---

def random_uniform_hypergraph(n, m, lo, hi, seed, name=""):
    rng = np.random.default_rng(seed)
    sizes = uniform_sizes(m, lo, hi, rng)
    ptr, mem = uniform_members(sizes, n, rng)
    return Hypergraph(n, ptr, mem, rank=hi, name=name or f"uniform-n{n}-m{m}-s{lo}..{hi}")


def config_small(seed=1):
    """n=1000, m=5000, sizes uniform in {2..5} (rank 5), uniform members."""
    return random_uniform_hypergraph(1000, 5000, 2, 5, seed, name="small-n1000-m5000-r5")


def config_powerlaw(n=1_000_000, m=5_000_000, rank=25, alpha=2.5, gamma=2.1, seed=2, lcc=False):
    """Zipf(alpha) sizes on {2..rank}, Chung-Lu membership with degree exponent gamma."""
    rng = np.random.default_rng(seed)
    sizes = zipf_sizes(m, alpha, 2, rank, rng)
    ptr, mem = chung_lu_members(sizes, n, gamma, rng)
    hg = Hypergraph(n, ptr, mem, rank=rank, name=f"powerlaw-n{n}-m{m}-r{rank}")
    if lcc:
        hg, _ = largest_component(hg)
    return hg


def config_large_rank(n=200_000, m=1_000_000, rank=100, prob=0.1, seed=3):
    """Geometric(prob) sizes on {2..rank}, uniform members."""
    rng = np.random.default_rng(seed)
    sizes = geometric_sizes(m, prob, 2, rank, rng)
    ptr, mem = uniform_members(sizes, n, rng)
    return Hypergraph(n, ptr, mem, rank=rank, name=f"largerank-n{n}-m{m}-r{rank}")


def config_batched(count=64, n_lo=10_000, n_hi=500_000, seed=4, scale=1.0):
    """``count`` independent power-law hypergraphs: n log-uniform, m=5n, rank U{8..32}.

    ``scale`` shrinks every n (for tests); the recipe itself is unchanged.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))) * scale))
        n = max(n, 64)
        r = int(rng.integers(8, 33))
        out.append(config_powerlaw(n=n, m=5 * n, rank=r, seed=int(rng.integers(1 << 30))))
    return out


def tiny_case(seed=0, n=12, m=20, rank=4):
    """n=12, m=20, sizes uniform on {1..rank} with at least one of each size 2..rank."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1, rank + 1, size=m).astype(np.int64)
    sizes[: rank - 1] = np.arange(2, rank + 1)
    rng.shuffle(sizes)
    ptr, mem = uniform_members(sizes, n, rng)
    return Hypergraph(n, ptr, mem, rank=rank, name=f"tiny-{seed}")


def fig1_example():
    """The 8-node, 6-edge hypergraph of Fig. 1 (ids shifted to 0-based)."""
    edges = [(2, 3, 4, 7), (1, 3, 4, 6), (1, 2, 3, 8), (4, 5, 6, 7), (1, 4, 6), (5, 7)]
    return from_edges(8, [tuple(v - 1 for v in e) for e in edges], rank=4, name="fig1")


def from_edges(n, edges, rank=None, name=""):
    sizes = np.array([len(e) for e in edges], dtype=np.int64)
    ptr = np.zeros(len(edges) + 1, dtype=np.int64)
    np.cumsum(sizes, out=ptr[1:])
    mem = np.array([v for e in edges for v in e], dtype=np.int32)
    return Hypergraph(n, ptr, mem, rank=rank, name=name)


def sunflower(petals, k, core, n, seed=5):
    """``petals`` edges of size k sharing a common core of ``core`` nodes (Fig. 3, left)."""
    rng = np.random.default_rng(seed)
    if core + petals * (k - core) > n:
        raise ValueError("not enough nodes")
    ids = rng.permutation(n)
    c = list(ids[:core])
    edges = []
    pos = core
    for _ in range(petals):
        edges.append(tuple(int(v) for v in c + list(ids[pos:pos + k - core])))
        pos += k - core
    return from_edges(n, edges, rank=k, name=f"sunflower-{petals}x{k}-core{core}")


def nested(chains, length, start, step, n, seed=6):
    """``chains`` nested families e_1 < e_2 < ... (sizes start, start+step, ...) (Fig. 3, right)."""
    rng = np.random.default_rng(seed)
    top = start + step * (length - 1)
    edges = []
    for _ in range(chains):
        ids = rng.choice(n, size=top, replace=False)
        for j in range(length):
            edges.append(tuple(int(v) for v in ids[: start + step * j]))
    return from_edges(n, edges, rank=top, name=f"nested-{chains}x{length}")


def paper_s_family(rank, n=2500, m=25000, seed=7):
    """Table I synthetic family: sizes 5,10,...,rank, about m/k edges each, uniform members."""
    rng = np.random.default_rng(seed)
    sizes_set = np.arange(5, rank + 1, 5)
    k = sizes_set.size
    sizes = np.repeat(sizes_set, m // k)
    ptr, mem = uniform_members(sizes, n, rng)
    return Hypergraph(n, ptr, mem, rank=rank, name=f"S-family-r{rank}")


# --------------------------------------------------------------- vectors ---

def x_uniform(n, lo, hi, seed, dtype=np.float64):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n).astype(dtype)


def x_constant(n, value, dtype=np.float64):
    return np.full(n, value, dtype=dtype)


def x_degree_like(hg, seed=5):
    """A positive vector shaped like a centrality: degree^(1/(N-1)) of each node (degree
    0 counts as 1), times a U(0.9, 1.1) jitter, rescaled to maximum 1.  This is the x of
    the power-law benchmark workload."""
    rng = np.random.default_rng(seed)
    d = np.maximum(hg.degrees(), 1).astype(np.float64)
    x = d ** (1.0 / (hg.rank - 1)) * rng.uniform(0.9, 1.1, hg.n)
    return x / x.max()
