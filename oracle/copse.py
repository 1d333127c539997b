"""COPSE in the CPU oracle: the forest compiler, plaintext classification, the
vectorised inference circuit over slot vectors (cleartext) and over BGV
ciphertexts (through ``oracle.bgv``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; the product never imports it.

Each function names the part of the paper (Malik et al., "Vectorized Secure
Evaluation of Decision Forests", PLDI'21) it follows.  Readings of passages the
paper leaves open are stated where they are used.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import bgv as B


# ---------------------------------------------------------------------------
# Forest model and its serialisation (Section 5, "Input Representation"):
# a line of label names, then one line per tree; a leaf gives its label index,
# a branch gives its feature index, threshold, then left and right subtrees.
# Token syntax (this implementation's): "l <label>" and "b <feature> <threshold>".
# ---------------------------------------------------------------------------
@dataclass
class Node:
    leaf: bool
    label: int = -1
    feature: int = -1
    threshold: int = 0
    left: "Node" = None
    right: "Node" = None


def parse_forest(text: str):
    lines = [ln for ln in text.strip().splitlines() if ln.strip()]
    if len(lines) < 2:
        raise ValueError("forest needs a label line and at least one tree")
    labels = lines[0].split()
    trees = []
    for ln in lines[1:]:
        toks = ln.split()
        pos = 0

        def rec():
            nonlocal pos
            kind = toks[pos]
            if kind == "l":
                n = Node(True, label=int(toks[pos + 1]))
                pos += 2
                return n
            if kind == "b":
                n = Node(False, feature=int(toks[pos + 1]), threshold=int(toks[pos + 2]))
                pos += 3
                n.left = rec()
                n.right = rec()
                return n
            raise ValueError(f"bad token {kind!r}")

        t = rec()
        if pos != len(toks):
            raise ValueError("trailing tokens in tree line")
        trees.append(t)
    # a leaf names its class by its index in the label line (Section 5, Input Representation)
    if any(not 0 <= c < len(labels) for c in _leaf_labels(trees)):
        raise ValueError("class index out of range")
    return labels, trees


def _leaf_labels(trees):
    out = []

    def walk(n):
        if n.leaf:
            out.append(n.label)
        else:
            walk(n.left)
            walk(n.right)
    for t in trees:
        walk(t)
    return out


def classify_plain(trees, x):
    """Plaintext evaluation (Section 2.1): at a branch compare x[f] < threshold;
    false goes left, true goes right.  Returns one bit per leaf (leaves in
    preorder, continued across trees), 1 for the leaf each tree reaches."""
    bits = []
    for t in trees:
        def walk(n, on):
            if n.leaf:
                bits.append(1 if on else 0)
                return
            d = x[n.feature] < n.threshold
            walk(n.left, on and not d)
            walk(n.right, on and d)
        walk(t, True)
    return bits


# ---------------------------------------------------------------------------
# Compiler (Section 4.1-4.2)
# ---------------------------------------------------------------------------
@dataclass
class Model:
    n_features: int
    precision: int
    labels_per_leaf: list          # class index of each leaf (preorder)
    br_feature: list               # f vector (Section 4.1.1)
    br_threshold: list             # t vector
    br_level: list                 # level of each branch (Section 4.1.1)
    K: int                         # maximum multiplicity
    q: int                         # quantised branching K * n_features
    b: int                         # branching
    L: int                         # number of leaves (slots of the result)
    d: int                         # number of levels
    thr_slot: list                 # padded threshold vector (sentinel 0)
    slot_branch: list              # branch held by each padded slot, -1 = sentinel
    R: np.ndarray                  # reshuffling matrix b x q
    lvl: list                      # level matrices L x b, k = 1..d
    mask: list                     # level masks, length L, k = 1..d
    block: int = 0                 # slots per query block
    extras: dict = field(default_factory=dict)
    # Row segments (a layout reading of this implementation, not of the paper): a forest
    # whose query block would not fit a slot row is split into n_seg contiguous groups of
    # trees, each compiled alike with a common K, q and d; query j then owns blocks
    # j*n_seg .. j*n_seg + n_seg - 1, block s holding segment s.  b and L are then the
    # largest segment's (the block layout); b_total and L_total count the whole forest.
    n_seg: int = 1
    segs: list = None
    b_total: int = 0
    L_total: int = 0

    @property
    def m1(self):                  # rows of the extended reshuffle: L + b - 1
        return self.L + self.b - 1

    @property
    def pd(self):                  # slots that must hold the periodic decision vector
        return self.m1 + self.q - 1


def _branches(n) -> int:
    return 0 if n.leaf else 1 + _branches(n.left) + _branches(n.right)


def compile_forest(text: str, precision: int, n_features: int = 0, slots_per_row: int = 0) -> Model:
    """Compile a forest (Sections 4.1-4.2).  With slots_per_row (= N/2) given, a forest whose
    query block would exceed a slot row is compiled in row segments: the smallest power of
    two S such that, with tree t in group floor(S * (branches of the trees before t) /
    (all branches)), no group is empty and the common block fits a row (and S blocks fit
    the ring)."""
    labels, trees = parse_forest(text)
    if any(t < 0 or t >= (1 << precision) for t in _thresholds(trees)):
        raise ValueError("threshold out of range for the precision")
    feats = _features(trees)
    if not feats:
        raise ValueError("forest has no branches")
    nf = n_features if n_features else max(feats) + 1
    m = _build(trees, precision, nf)
    m.b_total, m.L_total = m.b, m.L
    if not slots_per_row or m.block <= slots_per_row:
        if slots_per_row and m.block > slots_per_row:
            raise ValueError("model does not fit one slot row")
        return m
    counts = [_branches(t) for t in trees]
    total = sum(counts)
    S = 2
    while S <= min(64, len(trees)):
        before = np.concatenate([[0], np.cumsum(counts)[:-1]])
        gi = [min(S - 1, (S * int(b)) // total) for b in before]
        groups = [[t for t, g in zip(trees, gi) if g == k] for k in range(S)]
        if all(groups):
            first = [_build(g, precision, nf) for g in groups]
            K, d = max(x.K for x in first), max(x.d for x in first)
            segs = [_build(g, precision, nf, K, d) for g in groups]
            bp, Lp = max(x.b for x in segs), max(x.L for x in segs)
            need = Lp + bp - 1 + K * nf - 1
            blk = 1
            while blk < need:
                blk <<= 1
            if blk <= slots_per_row and S * blk <= 2 * slots_per_row:
                for x in segs:
                    x.block = blk
                    x.b_total, x.L_total = x.b, x.L
                return Model(nf, precision, m.labels_per_leaf, m.br_feature, m.br_threshold, m.br_level, K, K * nf,
                             bp, Lp, d, None, None, None, None, None, blk, n_seg=S, segs=segs,
                             b_total=m.b, L_total=m.L)
        S *= 2
    raise ValueError("model does not fit one slot row")


def _thresholds(trees):
    out = []

    def walk(n):
        if not n.leaf:
            out.append(n.threshold)
            walk(n.left)
            walk(n.right)
    for t in trees:
        walk(t)
    return out


def _features(trees):
    out = []

    def walk(n):
        if not n.leaf:
            out.append(n.feature)
            walk(n.left)
            walk(n.right)
    for t in trees:
        walk(t)
    return out


def _build(trees, precision: int, nf: int, K_min: int = 0, d_min: int = 0) -> Model:
    """Sections 4.1.1-4.2.4 for a list of trees: K at least K_min, levels 1..max(d, d_min)."""
    # Section 4.1.1: branches and leaves indexed in preorder, continuing across trees.
    br_f, br_t, br_lvl, leaf_cls = [], [], [], []
    leaf_anc = []   # per leaf: list of (branch index, leaf is under its true child)

    def walk(n, anc):
        if n.leaf:
            leaf_cls.append(n.label)
            leaf_anc.append(list(anc))
            return 0
        i = len(br_f)
        br_f.append(n.feature)
        br_t.append(n.threshold)
        br_lvl.append(0)
        hl = walk(n.left, anc + [(i, False)])
        hr = walk(n.right, anc + [(i, True)])
        # level = branches on the longest path from the node to a label, itself included
        br_lvl[i] = 1 + max(hl, hr)
        return br_lvl[i]

    for t in trees:
        walk(t, [])
    b = len(br_f)
    if b == 0:
        raise ValueError("forest has no branches")
    if max(br_f) >= nf or min(br_f) < 0:
        raise ValueError("feature index out of range")
    L, d = len(leaf_cls), max(max(br_lvl), d_min)
    # Section 4.1.1: multiplicity, maximum multiplicity K, quantised branching q = K * n_features.
    kappa = [br_f.count(f) for f in range(nf)]
    K = max(max(kappa), K_min)
    q = K * nf
    # Section 4.2.1: thresholds grouped by feature, each group padded to K with S = 0.
    # Reading: within a group, branches keep their preorder order.
    thr_slot = [0] * q
    slot_branch = [-1] * q
    seen = [0] * nf
    for i, f in enumerate(br_f):
        s = K * f + seen[f]
        seen[f] += 1
        thr_slot[s] = br_t[i]
        slot_branch[s] = i
    # Section 4.2.2: R[i][j] = 1 iff padded slot j holds branch i.
    R = np.zeros((b, q), dtype=np.int64)
    for j, i in enumerate(slot_branch):
        if i >= 0:
            R[i, j] = 1
    # Section 4.2.3-4.2.4: level matrices and masks.  For label l and level k pick
    # the ancestor whose level is k, else the ancestor of greatest level below k
    # ("the highest branch not exceeding that level"); reading where every
    # ancestor is above k: pick the parent.  A leaf that is a whole tree has no
    # ancestor: its row stays empty and its mask is 1.
    lvl, mask = [], []
    for k in range(1, d + 1):
        M = np.zeros((L, b), dtype=np.int64)
        mk = np.ones(L, dtype=np.int64)
        for l, anc in enumerate(leaf_anc):
            if not anc:
                continue
            exact = [(i, tr) for i, tr in anc if br_lvl[i] == k]
            below = [(i, tr) for i, tr in anc if br_lvl[i] < k]
            if exact:
                i, tr = exact[0]
            elif below:
                i, tr = max(below, key=lambda a: br_lvl[a[0]])
            else:
                i, tr = anc[-1]
            M[l, i] = 1
            mk[l] = 0 if tr else 1     # 0 under the true path, 1 otherwise
        lvl.append(M)
        mask.append(mk)
    m = Model(nf, precision, leaf_cls, br_f, br_t, br_lvl, K, q, b, L, d, thr_slot, slot_branch, R, lvl, mask)
    need = m.pd
    blk = 1
    while blk < need:
        blk <<= 1
    m.block = blk
    return m


# ---------------------------------------------------------------------------
# Slot layout.  Query j owns block j (slots j*B .. j*B+B-1; a row of N/2 slots
# holds N/(2B) blocks).  Inside a block the replicated feature vector
# (Section 3.3, Step 0) repeats with period q over the first pd slots so that
# rotations by up to q-1 and b-1 stay inside the block (the cyclic extension
# of the diagonal method, Section 4.1.2).
# ---------------------------------------------------------------------------
def parts(m: Model):
    """The compiled forests whose blocks make up one query's slots: the model itself, or
    its row segments in order."""
    return m.segs if m.n_seg > 1 else [m]


def feature_planes(m: Model, queries, N: int):
    """p bit-planes (Section 4.1.2) of the replicated feature vectors; query j's features
    fill each of its blocks j*n_seg + s."""
    nb = N // (m.block * m.n_seg)
    if len(queries) > nb:
        raise ValueError("too many queries for one ciphertext")
    planes = np.zeros((m.precision, N), dtype=np.int64)
    pos = np.arange(m.pd)
    feat_of = (pos % m.q) // m.K
    for j, x in enumerate(queries):
        x = np.asarray(x, dtype=np.int64)
        vals = x[feat_of]
        for s in range(m.n_seg):
            for i in range(m.precision):
                planes[i, (j * m.n_seg + s) * m.block + pos] = (vals >> i) & 1
    return planes


def tile_blocks(m: Model, block_vec, N: int):
    """Repeat a per-block slot pattern (length <= block) in every block.  For a model in row
    segments the pattern is an array [n_seg, length]: row s goes to every block of segment s."""
    v = np.asarray(block_vec, dtype=np.int64)
    if v.ndim == 1:
        v = np.broadcast_to(v, (m.n_seg, v.shape[0]))
    blk = np.zeros((m.n_seg, m.block), dtype=np.int64)
    blk[:, : v.shape[1]] = v
    return np.tile(blk.reshape(-1), N // (m.block * m.n_seg))


def threshold_planes(m: Model, N: int):
    pos = np.arange(m.pd)
    vals = np.stack([np.asarray(sg.thr_slot, dtype=np.int64)[pos % m.q] for sg in parts(m)])
    return np.stack([tile_blocks(m, (vals >> i) & 1, N) for i in range(m.precision)])


def generalized_diagonal(M: np.ndarray, i: int, rows: int) -> np.ndarray:
    """d_i[j] = M[j mod m][(j + i) mod n], j < rows (Section 4.1.2, generalised
    diagonals, with rows cyclically extended past m)."""
    m, n = M.shape
    j = np.arange(rows)
    return M[j % m, (j + i) % n]


def _padded(M: np.ndarray, rows: int, cols: int) -> np.ndarray:
    """A segment's matrix inside the common block layout: zero rows and columns appended."""
    out = np.zeros((rows, cols), dtype=np.int64)
    out[: M.shape[0], : M.shape[1]] = M
    return out


def reshuffle_diagonal(m: Model, i: int) -> np.ndarray:
    """Diagonal i of the extended reshuffle R_ext (rows L+b-1, row j = R[j mod b]); for a model
    in row segments an array [n_seg, L+b-1], segment s's R padded to b rows."""
    if m.n_seg == 1:
        return generalized_diagonal(m.R, i, m.m1)
    return np.stack([generalized_diagonal(_padded(sg.R, m.b, m.q), i, m.m1) for sg in m.segs])


def level_diagonal(m: Model, k: int, i: int, t: int) -> np.ndarray:
    """Signed diagonal i of level k: (1 - 2 Mask_k) * d_i(Lvl_k), values in {0,1,t-1}; per
    segment (array [n_seg, L]) for a model in row segments, each level matrix padded to
    L x b with zeros."""
    if m.n_seg == 1:
        return ((1 - 2 * m.mask[k - 1]) * generalized_diagonal(m.lvl[k - 1], i, m.L)) % t
    return np.stack([((1 - 2 * _padded(sg.mask[k - 1][:, None], m.L, 1)[:, 0]) *
                      generalized_diagonal(_padded(sg.lvl[k - 1], m.L, m.b), i, m.L)) % t
                     * (np.arange(m.L) < sg.L) for sg in m.segs])


def mask_vector(m: Model, k: int) -> np.ndarray:
    """Mask_k as a block pattern ([n_seg, L] for row segments, zero past a segment's leaves)."""
    if m.n_seg == 1:
        return m.mask[k - 1]
    return np.stack([_padded(sg.mask[k - 1][:, None], m.L, 1)[:, 0] for sg in m.segs])


def fused_matrix(m: Model, k: int, sg: Model = None) -> np.ndarray:
    """The reshuffle folded into level k (Algorithm 1 multiplies Decisions by R, then
    Branches by Lvl_k; the product is associative): F_k = S_k R, S_k = (1 - 2 Mask_k) Lvl_k,
    an L x q matrix with entries in {0, 1, -1}.  For a model in row segments, segment sg's."""
    sg = sg or m
    return ((1 - 2 * sg.mask[k - 1])[:, None] * sg.lvl[k - 1]) @ sg.R


def fused_diagonal(m: Model, k: int, i: int, t: int) -> np.ndarray:
    """Diagonal i < q of F_k, values mod t (per segment [n_seg, L] for row segments, each F
    padded to L x q)."""
    if m.n_seg == 1:
        return generalized_diagonal(fused_matrix(m, k), i, m.L) % t
    return np.stack([generalized_diagonal(_padded(fused_matrix(m, k, sg), m.L, m.q), i, m.L) % t for sg in m.segs])


def fused_diagonals(m: Model, k: int, t: int):
    """Nonzero diagonals of the fused level-k matrix F_k = S_k R."""
    out = {}
    for i in range(m.q):
        dg = fused_diagonal(m, k, i, t)
        if dg.any():
            out[i] = dg
    return out


def reshuffle_diagonals(m: Model):
    """Nonzero diagonals of the extended reshuffle R_ext (rows L+b-1, row j = R[j mod b]):
    multiplying by it leaves the branch vector repeated with period b, ready for
    the level products without further rotation."""
    out = {}
    for i in range(m.q):
        dg = reshuffle_diagonal(m, i)
        if dg.any():
            out[i] = dg
    return out


def level_diagonals(m: Model, k: int, t: int):
    """Signed diagonals of level k: (1 - 2 Mask_k) * d_i(Lvl_k), values in {0,1,t-1};
    adding Mask_k afterwards computes Lvl_k * Branches XOR Mask_k (Section 4.2.4)
    as m + (1-2m) z."""
    out = {}
    for i in range(m.b):
        dg = level_diagonal(m, k, i, t)
        if dg.any():
            out[i] = dg
    return out


def bsgs_split(diags: dict, g: int, block: int):
    """Baby-step / giant-step grouping of the diagonal method (Halevi and Shoup's
    BSGS form of the MatMul of Section 4.1.2): diagonal i = k g + j, 0 <= j < g,
    joins giant step k g with baby step j, its block-local slot vector shifted
    by k g,  d'_{k,j}[s] = d_i[s - k g],  so that
        M v = sum_k rot( sum_j d'_{k,j} * rot(v, j), k g ).
    The shift stays inside the query's block (k g + rows <= block), so no
    product reaches another block.  Returns {k g: {j: d'}}."""
    out = {}
    for i in sorted(diags):
        k, j = divmod(i, g)
        d = np.asarray(diags[i])
        assert k * g + d.shape[-1] <= block, "shifted diagonal leaves the block"
        sh = np.zeros(d.shape[:-1] + (k * g + d.shape[-1],), dtype=np.int64)
        sh[..., k * g:] = d
        out.setdefault(k * g, {})[j] = sh
    return out


def _rots(diag_sets, g, block):
    if not g:
        return set(i for d in diag_sets for i in d if i)
    r = set()
    for d in diag_sets:
        for kg, babies in bsgs_split(d, g, block).items():
            r |= set(j for j in babies if j)
            if kg:
                r.add(kg)
    return r


def rotation_sets(m: Model, g=(0, 0), fused=False):
    """Rotation amounts used by the reshuffle and by the level products (0 excluded);
    g = (baby-step size of the reshuffle, of the levels), 0 = the plain diagonal method.
    fused: the fused level products over Decisions only (baby-step size g[0])."""
    if fused:
        return [], sorted(_rots([fused_diagonals(m, k, 65537) for k in range(1, m.d + 1)], g[0], m.block))
    rs = _rots([reshuffle_diagonals(m)], g[0], m.block)
    ls = _rots([level_diagonals(m, k, 65537) for k in range(1, m.d + 1)], g[1], m.block)
    return sorted(rs), sorted(ls)


# ---------------------------------------------------------------------------
# The circuit (Algorithm 1, Section 4.3), written once over an abstract
# "engine" so that the cleartext slot simulation and the BGV evaluation follow
# the same steps in the same order.
# ---------------------------------------------------------------------------
def pairwise(items, combine):
    """Balanced reduction: combine adjacent pairs, carry an odd last element."""
    while len(items) > 1:
        nxt = [combine(items[k], items[k + 1], len(items) == 2) for k in range(0, len(items) - 1, 2)]
        if len(items) % 2:
            nxt.append(items[-1])
        items = nxt
    return items[0]


def seccomp(E, X, Y_planes, p):
    """SecComp (Section 4.1.2, Integer Comparison): D = [x < y] slotwise, bit-sliced,
    most significant plane p-1.  The paper gives only operation counts; reading:
    per plane lt_i = (1 - x_i) y_i and eq_i = [x_i == y_i], combined over planes
    MSB-first by the associative operator
        (lt_h, eq_h) o (lt_l, eq_l) = (lt_h + eq_h lt_l, eq_h eq_l)
    as a balanced tree (ceil(log2 p) multiplicative levels).  With plaintext
    thresholds, lt_i = y_i - y_i x_i and eq_i = (1 - y_i) + (2 y_i - 1) x_i."""
    leaves = []
    for i in reversed(range(p)):
        y = Y_planes[i]
        if E.encrypted_model:
            xy = E.mul(X[i], y)
            lt = E.sub(y, xy)
            eq = E.add_const(E.sub(E.add(xy, xy), E.add(X[i], y)), 1)
        else:
            lt = E.affine(X[i], (-y) % E.t, y)
            eq = E.affine(X[i], (2 * y - 1) % E.t, (1 - y) % E.t)
        leaves.append((lt, eq))

    def combine(hi, lo, root):
        lt = E.add(hi[0], E.mul(hi[1], lo[0]))
        eq = None if root else E.mul(hi[1], lo[1])
        return (lt, eq)

    return pairwise(leaves, combine)[0]


def matmul(E, v, diag_sets, add_vecs, m: Model, N: int, g: int = 0):
    """Diagonal method (Section 4.1.2, Matrix Multiplication) for several matrices
    applied to the same vector: for each matrix a, the sum over its nonzero
    diagonals of d_i * rot(v, i), plus an optional plaintext, then one modulus
    switch.  Rotations of v by the same amount serve every matrix.  diag_sets
    hold block-local diagonals.  With g > 0 the sum is taken in baby-step /
    giant-step form (bsgs_split): the baby-step sums of every (matrix, giant
    step) share the rotations of v, and each matrix's giant steps are rotated
    and summed (E.rot_sum)."""
    if not g:
        sums = E.diag_sums(v, [{i: tile_blocks(m, d, N) for i, d in ds.items()} for ds in diag_sets])
    else:
        groups = [bsgs_split(ds, g, m.block) for ds in diag_sets]
        inner_sets = [{j: tile_blocks(m, d, N) for j, d in grp[kg].items()} for grp in groups for kg in sorted(grp)]
        inner = iter(E.diag_sums(v, inner_sets))
        sums = [E.rot_sum([(kg, next(inner)) for kg in sorted(grp)]) for grp in groups]
    out = []
    for acc, add in zip(sums, add_vecs):
        if add is not None:
            acc = E.add_plain(acc, add)
        out.append(E.rescale(acc))
    return out


def infer(E, m: Model, X, N: int, g=(0, 0), shuffle=None, fused=False):
    """Algorithm 1: SecComp, reshuffle, per-level product XOR mask, MultAll.
    Reading: the level products use Branches (the reshuffled vector, as the
    text of Section 4.3 says), not Decisions as the listing prints.
    g = (baby-step size of the reshuffle, of the levels); 0 = plain diagonal method.
    shuffle = src of a label shuffle (shuffle_diagonals), applied to the result.
    fused: each level's product taken with F_k = S_k R on Decisions (fused_matrix), baby-step
    size g[0]; no Branches vector."""
    t = E.t
    Y = E.thresholds(m)
    D = seccomp(E, X, Y, m.precision)
    if fused:
        Fd = [fused_diagonals(m, k, t) for k in range(1, m.d + 1)]
        res = matmul(E, D, Fd, [tile_blocks(m, mask_vector(m, k), N) for k in range(1, m.d + 1)], m, N, g[0])
    elif E.encrypted_model:
        em = E.enc_model
        Br = matmul_enc(E, D, [em["R"]], [None], em["g"][0])[0]
        res = matmul_enc(E, Br, em["levels"], em["masks"], em["g"][1])
    else:
        Br = matmul(E, D, [reshuffle_diagonals(m)], [None], m, N, g[0])[0]
        Ld = [level_diagonals(m, k, t) for k in range(1, m.d + 1)]
        res = matmul(E, Br, Ld, [tile_blocks(m, mask_vector(m, k), N) for k in range(1, m.d + 1)], m, N, g[1])
    out = pairwise(res, lambda a, b, root: E.mul(a, b))
    if shuffle is not None:
        out = matmul(E, out, [shuffle_diagonals(m, shuffle, N)], [None], m, N)[0]
    return out


def shuffle_diagonals(m: Model, src, N: int):
    """A server-side label shuffle with padding (Section 7.2, "Returning classification
    bitvectors": a permutation of the result bitvector by a plaintext matrix product, the
    codebook permuted alike, padded with extra labels).  Output slot j of a block takes leaf
    src[j] (-1: a padding slot, always 0).  Diagonal method over signed shifts: the term with
    shift k = src[j] - j is the rotation by k mod N/2 (a negative shift reads backwards inside
    the block, since src[j] >= 0).  Returns {rotation amount: block-local diagonal}."""
    assert len(src) <= m.block
    h = N // 2
    out = {}
    for j, i in enumerate(src):
        if i < 0:
            continue
        a = (int(i) - j) % h
        out.setdefault(a, np.zeros(len(src), dtype=np.int64))[j] = 1
    return out


def shuffle_galois(m: Model, src, logN: int):
    return sorted(set(B.galois_rot(logN, a) for a in shuffle_diagonals(m, src, 1 << logN) if a))


# ---------------------------------------------------------------------------
# Encrypted model (Section 3.1 with Maurice = Diane; Section 8.3): the model
# owner encrypts the threshold planes, every diagonal of the reshuffle and
# level matrices (zero ones included, so their number p + q + d(b+1) of
# Table 1d reveals only the sizes) and the masks, and the products become
# ciphertext x ciphertext.
# ---------------------------------------------------------------------------
def model_ct_index(m: Model, kind: str, k: int = 0, i: int = 0) -> int:
    """Canonical numbering of the encrypted model's ciphertexts: threshold planes,
    reshuffle diagonals, level k diagonals (k = 1..d), masks."""
    if kind == "thr":
        return i
    if kind == "R":
        return m.precision + i
    if kind == "lvl":
        return m.precision + m.q + (k - 1) * m.b + i
    return m.precision + m.q + m.d * m.b + (k - 1)


def _clog2(x):
    return (x - 1).bit_length() if x > 1 else 0


def encrypt_model(bgv: B.Bgv, sk, m: Model, N: int, seed: int, g=(0, 0)):
    """Every ciphertext of the encrypted model, under the secret key with seeded
    masks (Bgv.encrypt_sk), each at the level where the circuit uses it:
    thresholds at L, reshuffle diagonals at the level of Decisions, level
    diagonals and masks at the level of Branches.  With a baby-step size g the
    diagonal i is stored shifted by its giant step (bsgs_split)."""
    P = bgv.P
    lvl_D = P.L - 1 - _clog2(m.precision)
    lvl_B = lvl_D - 1

    def enc(vec, idx, ell):
        return bgv.encrypt_sk(sk, B.encode(P, vec % P.t), seed, idx, ell)

    def shifted(d, i, gg):
        kg = i - i % gg if gg else 0
        d = np.asarray(d)
        v = np.zeros(d.shape[:-1] + (kg + d.shape[-1],), dtype=np.int64)
        v[..., kg:] = d
        return v

    thr = [enc(y, model_ct_index(m, "thr", i=i), P.L) for i, y in enumerate(threshold_planes(m, N))]
    R = {i: enc(tile_blocks(m, shifted(reshuffle_diagonal(m, i), i, g[0]), N),
                model_ct_index(m, "R", i=i), lvl_D) for i in range(m.q)}
    levels, masks = [], []
    for k in range(1, m.d + 1):
        levels.append({i: enc(tile_blocks(m, shifted(level_diagonal(m, k, i, P.t), i, g[1]), N),
                              model_ct_index(m, "lvl", k, i), lvl_B)
                       for i in range(m.b)})
        masks.append(enc(tile_blocks(m, mask_vector(m, k), N), model_ct_index(m, "mask", k), lvl_B))
    return {"thresholds": thr, "R": R, "levels": levels, "masks": masks, "g": tuple(g)}


def encrypted_rotation_sets(m: Model, g=(0, 0)):
    """Rotation amounts of the encrypted-model products: every diagonal index is present."""
    def amounts(n, gg):
        if not gg:
            return set(range(1, n))
        return set(i % gg for i in range(n)) - {0} | set(i - i % gg for i in range(n)) - {0}
    return sorted(amounts(m.q, g[0])), sorted(amounts(m.b, g[1]))


def matmul_enc(E, v, enc_sets, add_cts, g: int = 0):
    """MatMul with encrypted diagonals: for each matrix, per giant step k g the sum
    over baby steps j of Enc(d'_{k,j}) x rot(v, j) as 3-component tensors,
    relinearised once (lazy relinearisation); the giant steps rotated and summed
    (E.rot_sum); plus the encrypted mask; then one modulus switch."""
    sums = E.enc_diag_sums(v, enc_sets, g)
    out = []
    for acc, add in zip(sums, add_cts):
        if add is not None:
            acc = E.add(acc, add)
        out.append(E.rescale(acc))
    return out


class SlotEngine:
    """Cleartext slot arithmetic mod t: the values the encrypted circuit must decrypt to."""

    def __init__(self, N: int, t: int = B.T_DEFAULT, encrypted_model=False, model=None):
        self.N, self.t, self.encrypted_model = N, t, encrypted_model

    def thresholds(self, m):
        return threshold_planes(m, self.N)

    def rot(self, v, i):
        h = self.N // 2
        return np.concatenate([np.roll(v[:h], -i), np.roll(v[h:], -i)])

    def mul(self, a, b):
        return (a * b) % self.t

    def mul_plain(self, a, p):
        return (a * p) % self.t

    def add(self, a, b):
        return (a + b) % self.t

    def sub(self, a, b):
        return (a - b) % self.t

    def add_const(self, a, c):
        return (a + c) % self.t

    def add_plain(self, a, p):
        return (a + p) % self.t

    def affine(self, x, mult, addv):
        return (x * mult + addv) % self.t

    def rescale(self, a):
        return a

    def rot_sum(self, terms):
        acc = np.zeros(self.N, dtype=np.int64)
        for k, c in terms:
            acc = (acc + self.rot(c, k)) % self.t
        return acc

    def diag_sums(self, v, diag_sets):
        out = []
        for diags in diag_sets:
            acc = np.zeros(self.N, dtype=np.int64)
            for i in sorted(diags):
                acc = (acc + diags[i] * self.rot(v, i)) % self.t
            out.append(acc)
        return out


class BgvEngine:
    """The same circuit on BGV ciphertexts with the canonical policy: after every
    multiplication (ct x ct after relinearisation; after each affine plaintext
    step and after each matrix product) drop one prime; before a binary
    operation bring the operand at the higher level down.  The products of one
    vector with several matrices share its rotations, and each sum of
    diagonal products takes the modulus-down step of key switching once
    (Bgv.matmul)."""

    def __init__(self, bgv: B.Bgv, keys: B.Keys, encrypted_model=False, enc_model=None):
        self.b, self.k = bgv, keys
        self.P = bgv.P
        self.N, self.t = self.P.N, self.P.t
        self.encrypted_model = encrypted_model
        self.enc_model = enc_model
        self.counts = {"rot": 0, "mul": 0, "mul_plain": 0, "modswitch_ops": 0}

    def thresholds(self, m):
        if self.encrypted_model:
            return self.enc_model["thresholds"]
        return threshold_planes(m, self.N)

    def rot(self, v, i):
        """One rotation with its own modulus-down step (equal, bit for bit, to a hoisted one)."""
        if i == 0:
            return v
        g = B.galois_rot(self.P.logN, i)
        return self.b.rotate(v, g, self.k.gk[g])

    def diag_sums(self, v, diag_sets):
        rots = sorted(set(i for d in diag_sets for i in d))
        galois = [B.galois_rot(self.P.logN, i) if i else 1 for i in rots]
        gks = [self.k.gk[g] if g != 1 else None for g in galois]
        pts = [[B.encode(self.P, d[i]) if i in d else None for i in rots] for d in diag_sets]
        self.counts["rot"] += sum(1 for i in rots if i)
        self.counts["mul_plain"] += sum(len(d) for d in diag_sets)
        return self.b.matmul(v, galois, gks, pts)

    def enc_diag_sums(self, v, enc_sets, g):
        """Per matrix {diagonal index: ciphertext}: baby rotations of v shared by every
        matrix (each with its own key switch, identical to hoisting), per giant step
        the tensor products summed and relinearised once, then the giant-step sum."""
        babies = sorted(set((i % g if g else i) for es in enc_sets for i in es))
        R = {j: self.rot(v, j) for j in babies}
        self.counts["rot"] += sum(1 for j in babies if j)
        out = []
        for es in enc_sets:
            groups = {}
            for i in sorted(es):
                groups.setdefault(i - i % g if g else 0, []).append((i % g if g else i, es[i]))
            terms = []
            for kg in sorted(groups):
                acc = None
                for j, d in groups[kg]:
                    t3 = self.b.tensor(d, R[j])
                    acc = t3 if acc is None else self.b.add(acc, t3)
                self.counts["mul"] += len(groups[kg])
                terms.append((kg, self.b.relin(acc, self.k.rlk)))
            out.append(self.rot_sum(terms))
        return out

    def rot_sum(self, terms):
        """Giant steps: sum_k rot(c_k, k) with one modulus-down step (Bgv.rotsum)."""
        if all(k == 0 for k, _ in terms) and len(terms) == 1:
            return terms[0][1]
        galois = [B.galois_rot(self.P.logN, k) if k else 1 for k, _ in terms]
        self.counts["rot"] += sum(1 for k, _ in terms if k)
        return self.b.rotsum([c for _, c in terms], galois, [self.k.gk[g] if g != 1 else None for g in galois])

    def mul(self, a, b):
        self.counts["mul"] += 1
        return self.b.mul(a, b, self.k.rlk)

    def mul_plain(self, a, p):
        self.counts["mul_plain"] += 1
        return self.b.mul_plain(a, B.encode(self.P, p))

    def add(self, a, b):
        return self.b.add(a, b)

    def sub(self, a, b):
        return self.b.sub(a, b)

    def add_const(self, a, c):
        return self.b.add_plain(a, B.encode(self.P, np.full(self.N, c)))

    def add_plain(self, a, p):
        return self.b.add_plain(a, B.encode(self.P, p))

    def affine(self, x, mult, addv):
        r = self.b.add_plain(self.b.mul_plain(x, B.encode(self.P, mult)), B.encode(self.P, addv))
        return self.b.modswitch(r)

    def rescale(self, a):
        return self.b.modswitch(a)


def galois_elements(m: Model, logN: int, g=(0, 0), fused=False):
    rs, ls = rotation_sets(m, g, fused)
    return sorted(set(B.galois_rot(logN, i) for i in rs + ls))


def encrypt_queries(bgv: B.Bgv, keys: B.Keys, m: Model, queries, seed: int, index0: int = 0):
    """The p feature planes of one query ciphertext, plane i as encryption index0 + i
    (query ciphertext c of a larger batch uses index0 = c p)."""
    planes = feature_planes(m, queries, bgv.P.N)
    return [bgv.encrypt_slots(keys.pk, planes[i], seed, index0 + i) for i in range(m.precision)]


def decode_labels(m: Model, slots, n_queries: int, n_out: int = 0):
    """Result slots -> per query, one bit per leaf (Section 4.1.2, Classification Result);
    n_out output slots per query when the result was shuffled and padded."""
    out = []
    for j in range(n_queries):
        if m.n_seg > 1:
            v = np.concatenate([np.asarray(slots[(j * m.n_seg + s) * m.block: (j * m.n_seg + s) * m.block + sg.L],
                                           dtype=np.int64) for s, sg in enumerate(m.segs)])
        else:
            n = n_out or m.L
            v = np.asarray(slots[j * m.block: j * m.block + n], dtype=np.int64)
        out.append(v.tolist())
    return out


def levels_needed(m: Model, encrypted_model=False, shuffle=False, fused=False) -> int:
    """Primes dropped by the circuit under the canonical policy (plaintext model):
    1 (SecComp leaves) + ceil(log2 p) + 1 (reshuffle) + 1 (levels) + ceil(log2 d);
    the fused level products drop the reshuffle's prime."""
    def clog2(x):
        return (x - 1).bit_length() if x > 1 else 0
    return 1 + clog2(m.precision) + (1 if fused else 2) + clog2(m.d) + (1 if shuffle else 0)
