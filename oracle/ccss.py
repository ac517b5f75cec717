"""The CCSS forest of Sec. III, enumerated from its definition -- test infrastructure.

For a hypergraph whose edges are sorted node lists, the (untrimmed) CCSS is a
forest whose root-to-level-l paths are exactly the sorted proper sub-sequences
of length l of the edges.  Every pair (e, v) with v in e is a special leaf
hanging below the path e minus v (so at depth |e|, Fig. 2).  Trimming keeps
only paths that lead to a special leaf, i.e. the prefixes of the sequences
e minus v (the "easy optimisation" at the end of Sec. IV-B).
"""
from __future__ import annotations

import itertools


def untrimmed_levels(edges):
    """{level l: set of sorted tuples of length l} over all proper sub-sequences."""
    levels = {}
    for e in edges:
        e = tuple(sorted(e))
        for l in range(1, len(e)):
            for sub in itertools.combinations(e, l):
                levels.setdefault(l, set()).add(sub)
    return levels


def special_leaves(edges):
    """{path (sorted tuple): [(dropped node, edge index), ...]}."""
    out = {}
    for i, e in enumerate(edges):
        e = tuple(sorted(e))
        for v in e:
            path = tuple(u for u in e if u != v)
            out.setdefault(path, []).append((v, i))
    return out


def trimmed_levels(edges):
    """Levels of the forest after removing sub-trees without special leaves."""
    levels = {}
    for path in special_leaves(edges):
        for l in range(1, len(path) + 1):
            levels.setdefault(l, set()).add(path[:l])
    return levels


def level_counts(levels):
    return [len(levels[l]) for l in sorted(levels)]
