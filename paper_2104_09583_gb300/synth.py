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


def exact_tree_tokens(rng, n_branches, depth, n_features, precision, n_classes):
    """One tree with exactly n_branches branches whose longest root-to-leaf
    path crosses exactly min(depth, n_branches) of them: a random spine of
    that length, then leaves above the depth limit, drawn uniformly, turned
    into branches until the count is reached."""
    depth = min(depth, n_branches)
    if n_branches > (1 << depth) - 1:
        raise ValueError("a binary tree of this depth cannot hold that many branches")
    root = {"d": 0, "kids": None}
    node = root
    for _ in range(depth):                       # the spine
        node["kids"] = [{"d": node["d"] + 1, "kids": None}, {"d": node["d"] + 1, "kids": None}]
        node = node["kids"][int(rng.integers(2))]
    count = depth

    def open_leaves(n, out):
        if n["kids"] is None:
            if n["d"] < depth:
                out.append(n)
        else:
            for k in n["kids"]:
                open_leaves(k, out)
        return out

    while count < n_branches:
        cand = open_leaves(root, [])
        leaf = cand[int(rng.integers(len(cand)))]
        leaf["kids"] = [{"d": leaf["d"] + 1, "kids": None}, {"d": leaf["d"] + 1, "kids": None}]
        count += 1
    toks = []

    def emit(n):
        if n["kids"] is None:
            toks.extend(["l", str(int(rng.integers(n_classes)))])
        else:
            toks.extend(["b", str(int(rng.integers(n_features))), str(int(rng.integers(1 << precision)))])
            emit(n["kids"][0])
            emit(n["kids"][1])

    emit(root)
    return toks


# The eight microbenchmark forests of Section 8.4 (Table 6): max depth,
# precision and branches per tree.  Every forest has 2 features and 3 labels.
# The printed table gives the total branch count (15, 10 or 20); the names
# width55 / width78 / width677 give the split over the trees, and the other
# models split 15 branches as 7 + 8 like width78.
TABLE6 = {
    "depth4": (4, 8, (7, 8)),
    "depth5": (5, 8, (7, 8)),
    "depth6": (6, 8, (7, 8)),
    "width55": (5, 8, (5, 5)),
    "width78": (5, 8, (7, 8)),
    "width677": (5, 8, (6, 7, 7)),
    "prec8": (5, 8, (7, 8)),
    "prec16": (5, 16, (7, 8)),
}
TABLE6_FEATURES = 2
TABLE6_CLASSES = 3


def table6_forest(name, seed=6000):
    """A Table 6 microbenchmark forest as text, redrawn from its own seed."""
    depth, precision, per_tree = TABLE6[name]
    rng = np.random.default_rng(seed + sorted(TABLE6).index(name))
    lines = [" ".join(f"c{i}" for i in range(TABLE6_CLASSES))]
    for nb in per_tree:
        lines.append(" ".join(exact_tree_tokens(rng, nb, depth, TABLE6_FEATURES, precision, TABLE6_CLASSES)))
    return "\n".join(lines) + "\n"


def shuffle_plan(seed, leaf_classes, n_pad, n_classes):
    """A server-side label shuffle with padding (the option of Section 7.2, "Returning
    classification bitvectors"): a uniform permutation of the L leaves and n_pad padding slots.
    Returns (src, codebook): output slot j carries leaf src[j] (-1 = a padding slot, whose bit
    is always 0), codebook[j] its class (padding slots get uniform random classes)."""
    rng = np.random.default_rng(seed)
    L = len(leaf_classes)
    src = np.concatenate([np.arange(L), -np.ones(n_pad, dtype=np.int64)])
    rng.shuffle(src)
    code = np.array([leaf_classes[i] if i >= 0 else int(rng.integers(n_classes)) for i in src], dtype=np.uint32)
    return src.astype(np.int32), code


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
    bsgs: tuple = (128, 256)  # baby-step sizes of an encrypted-model run (reshuffle, levels)

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
    # encrypted model: 32 complete trees of depth 8 (8160 branches, 8192 leaves; the query
    # spans both slot rows of N = 2^15 as two row segments of 16 trees), 32 features, 16-bit,
    # 10 classes; 16 primes; 64 queries
    "encmodel32-n32768": Workload("encmodel32-n32768", 15, 55, 16, 3,
                                  ((4001, 32, 8, 32, 16, 10, True, None),), (64,)),
    # a small case of the encrypted-model products at the same ring and chain (1 complete tree of
    # depth 6, 8 features, 16-bit; 16 query ciphertexts of 128 queries): a few GB on the device,
    # for detailed counter captures of the multiply-accumulate kernel
    "encmodel1-n32768": Workload("encmodel1-n32768", 15, 55, 16, 3,
                                 ((4011, 1, 6, 8, 16, 10, True, None),), (2048,), (32, 32)),
    # batching: 256 queries over three forests (1 x depth 3, 4 x depth 5, 16 x depth 6)
    "batch3-n16384": Workload("batch3-n16384", 14, 55, 10, 3,
                              ((3001, 1, 3, 8, 8, 4, True, None),
                               (3002, 4, 5, 16, 8, 4, False, None),
                               (3003, 16, 6, 32, 8, 4, True, None)),
                              (32, 96, 128)),
}
