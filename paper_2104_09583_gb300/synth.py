"""Seeded synthetic workloads: random decision forests and query feature
vectors, as text and integer arrays.  This module holds no part of the
method's arithmetic; both the CUDA path's tests and the CPU oracle's tests
draw their inputs from it.

The paper's microbenchmarks are randomly generated forests (Section 8.1,
Table 6); its real-world models (income, soccer) were trained with
scikit-learn on datasets that are not available here, so seeded random forests
of the stated shapes stand in for every workload.

Forest text format (one line of class names, then one line per tree in
preorder): a branch is ``b <feature> <threshold>`` followed by its left and
right subtrees, a leaf is ``l <class>``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def random_tree_tokens(rng, depth, n_features, precision, n_classes, p_split, complete):
    toks = []

    def grow(level):
        split = level < depth and (complete or level == 0 or rng.random() < p_split)
        if split:
            toks.extend(["b", str(int(rng.integers(n_features))), str(int(rng.integers(1 << precision)))])
            grow(level + 1)
            grow(level + 1)
        else:
            toks.extend(["l", str(int(rng.integers(n_classes)))])

    grow(0)
    return toks


def random_forest(seed, n_trees, depth, n_features, precision, n_classes,
                  complete=True, p_split=0.9, branches=None):
    """A forest as text.  Complete trees of the given depth, or trees whose
    non-root nodes above the depth limit split with probability p_split; with
    ``branches=(lo, hi)`` whole forests are redrawn until the branch count is
    in range."""
    rng = np.random.default_rng(seed)
    while True:
        lines = [" ".join(f"c{i}" for i in range(n_classes))]
        nb = 0
        for _ in range(n_trees):
            toks = random_tree_tokens(rng, depth, n_features, precision, n_classes, p_split, complete)
            nb += toks.count("b")
            lines.append(" ".join(toks))
        if branches is None or branches[0] <= nb <= branches[1]:
            return "\n".join(lines) + "\n"


def random_queries(seed, n, n_features, precision):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 1 << precision, size=(n, n_features), dtype=np.int64).astype(np.uint32)


@dataclass(frozen=True)
class Workload:
    name: str
    log_n: int
    bits: int
    primes: int          # ciphertext primes (chain length)
    dnum: int
    forests: tuple       # (seed, n_trees, depth, n_features, precision, n_classes, complete, branches)
    queries: tuple       # queries per forest

    def forest_texts(self):
        return [random_forest(s, nt, dp, nf, p, nc, complete=c, branches=br)
                for (s, nt, dp, nf, p, nc, c, br) in self.forests]

    def precision(self, k=0):
        return self.forests[k][4]

    def n_features(self, k=0):
        return self.forests[k][3]

    def query_arrays(self):
        return [random_queries(7 * (1000 + k) + 1, nq, self.forests[k][3], self.forests[k][4])
                for k, nq in enumerate(self.queries)]


# Chain lengths: the circuit drops 3 + ceil(log2 p) + ceil(log2 d) primes and
# decryption needs one more, so the toy workload carries 8 primes (not 4) and
# the N=2^14 workload 10 (not 8).
WORKLOADS = {
    # 1 complete tree of depth 3, 2 features, 4-bit, 2 classes; N = 2^10, 50-bit primes; 1 query
    "toy-n1024": Workload("toy-n1024", 10, 50, 8, 3,
                          ((1001, 1, 3, 2, 4, 2, True, None),), (1,)),
    # 4 random trees of depth <= 5 with 90..110 branches, 8 features, 8-bit, 4 classes;
    # N = 2^14, 55-bit primes; 1 query
    "forest100-n16384": Workload("forest100-n16384", 14, 55, 10, 3,
                                 ((2001, 4, 5, 8, 8, 4, False, (90, 110)),), (1,)),
    # batching: 256 queries over three forests (1 x depth 3, 4 x depth 5, 16 x depth 6)
    "batch3-n16384": Workload("batch3-n16384", 14, 55, 10, 3,
                              ((3001, 1, 3, 8, 8, 4, True, None),
                               (3002, 4, 5, 16, 8, 4, False, None),
                               (3003, 16, 6, 32, 8, 4, True, None)),
                              (32, 96, 128)),
}
