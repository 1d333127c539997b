// Host-side COPSE forest compiler: parses the forest text and builds the
// vectorised structures of Section 4.2 of the paper (padded threshold vector,
// reshuffling matrix, level matrices and masks) plus the slot layout the
// device circuit uses.  Pure C++; no CUDA.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

struct ForestNode {
    bool leaf = true;
    int label = -1;       // class index (leaf)
    int feature = -1;     // branch
    uint32_t threshold = 0;
    int left = -1, right = -1;  // node indices
};

// Baby-step / giant-step split of the diagonal method for a group of matrices
// applied to one vector: diagonal i = k g + j of matrix a is multiplied, shifted
// by k g inside the query block, with rot(v, j) into accumulator (a, k g); each
// matrix's accumulators are then rotated by their giant step and summed.  g = 0
// keeps the plain method: all nonzero diagonals are baby steps, one
// accumulator per matrix with giant step 0.
struct BsgsGroup {
    struct Acc {
        uint32_t mat = 0, giant = 0;
        std::vector<int32_t> diag;  // per baby step: diagonal index giant + baby, or -1 (zero)
    };
    std::vector<uint32_t> baby;     // ascending, may include 0
    std::vector<Acc> acc;           // matrices in order, giant steps ascending within a matrix
    uint32_t n_mat = 0;
    bool plain() const;             // one accumulator per matrix, every giant step 0
    void rotations(std::vector<uint32_t> &out) const;  // nonzero baby and giant amounts, ascending
};
BsgsGroup bsgs_group(const std::vector<std::vector<uint32_t>> &nonzero, uint32_t g);

struct CompiledForest {
    // forest
    std::vector<std::string> classes;
    std::vector<ForestNode> nodes;
    std::vector<int> roots;
    // Section 4.1.1
    uint32_t n_features = 0, precision = 0, K = 0, q = 0, b = 0, L = 0, d = 0;
    std::vector<int> br_feature, br_level;
    std::vector<uint32_t> br_threshold;
    std::vector<int> leaf_class;
    // Section 4.2.1: padded threshold vector; slot_branch = -1 marks the sentinel S = 0
    std::vector<uint32_t> thr_slot;
    std::vector<int32_t> slot_branch;
    // Section 4.2.2-4.2.4, row-major
    std::vector<uint8_t> R;     // b x q
    std::vector<uint8_t> lvl;   // d x L x b
    std::vector<uint8_t> mask;  // d x L
    // slot layout: query block size (power of two >= L + b - 1 + q - 1)
    uint32_t block = 0;
    uint32_t log_n = 0;
    // nonzero diagonal indices
    std::vector<uint32_t> rot_reshuffle;  // ascending, may include 0
    std::vector<uint32_t> rot_level;      // union over levels, ascending, may include 0
    std::vector<std::vector<uint32_t>> lvl_nonzero;  // per level: nonzero diagonal indices
    // baby-step sizes of the reshuffle and of the level products (0 = plain method)
    uint32_t g_reshuffle = 0, g_level = 0;
    // encrypted model (every diagonal is a ciphertext, zero ones included, so the
    // products run over all q reshuffle and all b level diagonals)
    bool encrypted = false;
    BsgsGroup group_reshuffle() const;
    BsgsGroup group_level() const;

    // label shuffle with padding (Section 7.2): output slot j takes leaf shuffle_src[j]
    // (-1 = padding, always 0); codebook[j] is its class.  Empty = no shuffle.
    std::vector<int32_t> shuffle_src;
    std::vector<uint32_t> codebook;
    uint32_t n_out() const { return shuffle_src.empty() ? L_total : (uint32_t)shuffle_src.size(); }
    // rotation amounts of the shuffle product (signed shifts src[j] - j taken mod N/2), ascending
    void shuffle_rotations(std::vector<uint32_t> &out) const;
    // its diagonal for one rotation amount, block-local over n_out() slots
    void shuffle_diagonal(uint32_t amount, std::vector<uint32_t> &out) const;

    uint32_t m1() const { return L + b - 1; }       // rows of the extended reshuffle
    uint32_t pd() const { return m1() + q - 1; }    // slots carrying the periodic decisions
    uint32_t levels_used() const;

    // Row segments.  When one query block of the whole forest would not fit a slot row,
    // the trees are split into n_seg contiguous groups (segments) compiled alike: a common
    // K (so q), a common depth d, and per-block sizes b, L = the largest segment's.  Query j
    // then owns the n_seg blocks j n_seg + s, block s holding segment s; rotations never
    // cross a block, so each block's diagonals are its segment's.  b_total and L_total count
    // the whole forest (L_total leaf bits per query, in preorder across the trees).
    uint32_t n_seg = 1;
    std::vector<CompiledForest> seg;  // the segments when n_seg > 1
    uint32_t b_total = 0, L_total = 0;
    uint32_t span() const { return n_seg * block; }  // slots of one query (its blocks)
    const CompiledForest &part(uint32_t s) const { return n_seg > 1 ? seg[s] : *this; }
    // threshold bit of plane i at block-local slot x of segment s's block
    uint32_t thr_bit(uint32_t s, uint32_t x, uint32_t i) const;
    // diagonal i of segment s's extended reshuffle matrix (rows m1(), period b), block-local
    void reshuffle_diagonal(uint32_t i, std::vector<uint8_t> &out, uint32_t s = 0) const;
    // signed diagonal i of segment s's level k (1-based), values in {0, 1, t-1}; L rows, block-local
    void level_diagonal(uint32_t k, uint32_t i, uint64_t t, std::vector<uint64_t> &out, uint32_t s = 0) const;
    // level-k mask at block-local slot x of segment s's block (0 past the segment's leaves)
    uint32_t mask_at(uint32_t k, uint32_t x, uint32_t s) const;

    // Fused level products: the reshuffle folded into every level matrix, F_k = S_k R with
    // S_k = (1 - 2 Mask_k) Lvl_k (L x q, entries 0 / +-1): one product per level over the
    // rotations of Decisions, no Branches vector and one prime fewer.  Row x of F_k holds
    // its one nonzero at the padded slot of the branch Lvl_k picks for leaf x.  Plaintext
    // model only; the plan's baby-step size is g_reshuffle (the products are q wide).
    bool fused = false;
    std::vector<int32_t> fslot;                        // [d][L]: that slot, -1 = empty row
    std::vector<std::vector<uint32_t>> fused_nonzero;  // per level: nonzero diagonals of F_k
    void build_fused();                                // fslot of every part, fused_nonzero
    // signed diagonal i < q of segment s's F_k, values {0, 1, t-1}; L rows, block-local
    void fused_diagonal(uint32_t k, uint32_t i, uint64_t t, std::vector<uint64_t> &out, uint32_t s = 0) const;
};

// 0 on success; otherwise a COPSE_E* code and a message in `err`.
int compile_forest(const char *text, size_t len, uint32_t precision, uint32_t n_features, uint32_t log_n,
                   CompiledForest &out, std::string &err);

// one bit per leaf for query x (x has n_features entries)
void classify_plain(const CompiledForest &m, const uint32_t *x, uint8_t *bits);
