// COPSE forest compiler (host).  Section references are to Malik et al.,
// "Vectorized Secure Evaluation of Decision Forests" (PLDI'21).
#include "forest.h"

#include <algorithm>
#include <cstring>
#include <sstream>

#include "../../include/copse.h"

namespace {

struct Parser {
    std::vector<std::string> toks;
    size_t pos = 0;
    CompiledForest *f;
    std::string err;

    int node() {
        if (pos >= toks.size()) { err = "tree line ends early"; return -1; }
        const std::string &k = toks[pos];
        ForestNode n;
        if (k == "l") {
            if (pos + 1 >= toks.size()) { err = "leaf without a class"; return -1; }
            char *end = nullptr;
            long c = strtol(toks[pos + 1].c_str(), &end, 10);
            if (*end || c < 0) { err = "bad class index '" + toks[pos + 1] + "'"; return -1; }
            n.leaf = true;
            n.label = (int)c;
            pos += 2;
            f->nodes.push_back(n);
            return (int)f->nodes.size() - 1;
        }
        if (k == "b") {
            if (pos + 2 >= toks.size()) { err = "branch without feature and threshold"; return -1; }
            char *e1 = nullptr, *e2 = nullptr;
            long fe = strtol(toks[pos + 1].c_str(), &e1, 10);
            long long th = strtoll(toks[pos + 2].c_str(), &e2, 10);
            if (*e1 || *e2 || fe < 0 || th < 0 || th > 0xFFFFFFFFLL) { err = "bad branch fields"; return -1; }
            n.leaf = false;
            n.feature = (int)fe;
            n.threshold = (uint32_t)th;
            pos += 3;
            f->nodes.push_back(n);
            int me = (int)f->nodes.size() - 1;
            int l = node();
            if (l < 0) return -1;
            int r = node();
            if (r < 0) return -1;
            f->nodes[me].left = l;
            f->nodes[me].right = r;
            return me;
        }
        err = "unexpected token '" + k + "'";
        return -1;
    }
};

uint32_t clog2(uint32_t x) {
    uint32_t r = 0;
    while ((1u << r) < x) r++;
    return r;
}

}  // namespace

uint32_t CompiledForest::levels_used() const {
    return 1 + clog2(precision) + (fused ? 1 : 2) + clog2(d) + (shuffle_src.empty() ? 0 : 1);
}

void CompiledForest::build_fused() {
    for (uint32_t sgi = 0; sgi < n_seg; sgi++) {
        CompiledForest &P = n_seg > 1 ? seg[sgi] : *this;
        std::vector<int32_t> slot_of(P.b, -1);
        for (uint32_t j = 0; j < q; j++)
            if (P.slot_branch[j] >= 0) slot_of[P.slot_branch[j]] = (int32_t)j;
        P.fslot.assign((size_t)d * P.L, -1);
        for (uint32_t k = 1; k <= d; k++)
            for (uint32_t x = 0; x < P.L; x++) {
                const uint8_t *row = &P.lvl[((size_t)(k - 1) * P.L + x) * P.b];
                for (uint32_t j = 0; j < P.b; j++)
                    if (row[j]) { P.fslot[(size_t)(k - 1) * P.L + x] = slot_of[j]; break; }
            }
    }
    fused_nonzero.assign(d, {});
    for (uint32_t k = 1; k <= d; k++) {
        std::vector<char> nz(q, 0);
        for (uint32_t sgi = 0; sgi < n_seg; sgi++) {
            const CompiledForest &P = part(sgi);
            for (uint32_t x = 0; x < P.L; x++) {
                const int32_t c = P.fslot[(size_t)(k - 1) * P.L + x];
                if (c >= 0) nz[((uint32_t)c + q - x % q) % q] = 1;
            }
        }
        for (uint32_t i = 0; i < q; i++)
            if (nz[i]) fused_nonzero[k - 1].push_back(i);
    }
}

void CompiledForest::fused_diagonal(uint32_t k, uint32_t i, uint64_t t, std::vector<uint64_t> &out,
                                    uint32_t s) const {
    const CompiledForest &P = part(s);
    out.assign(L, 0);
    for (uint32_t x = 0; x < P.L; x++) {
        const int32_t c = P.fslot[(size_t)(k - 1) * P.L + x];
        if (c < 0 || (x + i) % q != (uint32_t)c) continue;
        out[x] = P.mask[(size_t)(k - 1) * P.L + x] ? t - 1 : 1;  // (1 - 2 mask) * entry, mod t
    }
}

uint32_t CompiledForest::thr_bit(uint32_t s, uint32_t x, uint32_t i) const {
    return x < pd() ? (part(s).thr_slot[x % q] >> i) & 1u : 0u;
}

void CompiledForest::reshuffle_diagonal(uint32_t i, std::vector<uint8_t> &out, uint32_t s) const {
    // extended reshuffle: row x is R[x mod b] (zero for rows past the segment's branches);
    // diagonal entry x is R_ext[x][(x+i) mod q]
    const CompiledForest &P = part(s);
    out.assign(m1(), 0);
    for (uint32_t x = 0; x < m1(); x++) {
        const uint32_t row = x % b;
        if (row < P.b) out[x] = P.R[(size_t)row * q + (x + i) % q];
    }
}

void CompiledForest::level_diagonal(uint32_t k, uint32_t i, uint64_t t, std::vector<uint64_t> &out,
                                    uint32_t s) const {
    // segment s's level matrix as L_s x b (zero columns past its branches), diagonal i
    const CompiledForest &P = part(s);
    out.assign(L, 0);
    const uint8_t *M = &P.lvl[(size_t)(k - 1) * P.L * P.b];
    const uint8_t *mk = &P.mask[(size_t)(k - 1) * P.L];
    for (uint32_t x = 0; x < P.L; x++) {
        const uint32_t col = (x + i) % b;
        if (col >= P.b || !M[(size_t)x * P.b + col]) continue;
        out[x] = mk[x] ? t - 1 : 1;  // (1 - 2 mask) * entry, mod t
    }
}

uint32_t CompiledForest::mask_at(uint32_t k, uint32_t x, uint32_t s) const {
    const CompiledForest &P = part(s);
    return x < P.L ? P.mask[(size_t)(k - 1) * P.L + x] : 0u;
}

namespace {

// Sections 4.1.1-4.2.4 for the trees `roots` of f.nodes (f.n_features and f.precision set):
// preorder indices, levels, K and q (at least forced_K), the padded threshold vector, the
// reshuffling matrix, the level matrices and masks for levels 1..max(d, forced_d).
int build_structures(CompiledForest &f, const std::vector<int> &roots, uint32_t forced_K, uint32_t forced_d,
                     std::string &err) {
    f.br_feature.clear();
    f.br_threshold.clear();
    f.br_level.clear();
    f.leaf_class.clear();
    // Section 4.1.1: preorder indices of branches and of labels, continued across trees
    struct Anc { int br; bool right; };
    std::vector<std::vector<Anc>> leaf_anc;
    std::vector<int> node_br(f.nodes.size(), -1);
    for (int root : roots) {
        std::vector<std::pair<int, std::vector<Anc>>> stack;
        stack.push_back({root, {}});
        while (!stack.empty()) {
            auto [n, anc] = stack.back();
            stack.pop_back();
            const ForestNode &nd = f.nodes[n];
            if (nd.leaf) {
                f.leaf_class.push_back(nd.label);
                leaf_anc.push_back(anc);
                continue;
            }
            int bi = (int)f.br_feature.size();
            node_br[n] = bi;
            f.br_feature.push_back(nd.feature);
            f.br_threshold.push_back(nd.threshold);
            f.br_level.push_back(0);
            auto ra = anc, la = anc;
            la.push_back({bi, false});
            ra.push_back({bi, true});
            stack.push_back({nd.right, ra});  // popped after the left subtree
            stack.push_back({nd.left, la});
        }
    }
    f.b = (uint32_t)f.br_feature.size();
    f.L = (uint32_t)f.leaf_class.size();
    if (f.b == 0) { err = "forest has no branches"; return COPSE_EINVAL; }
    // level: branches on the longest path to a label, itself included (labels: 0)
    {
        std::vector<int> lev(f.nodes.size(), 0);
        for (int n = (int)f.nodes.size() - 1; n >= 0; n--) {  // children follow parents in `nodes`
            const ForestNode &nd = f.nodes[n];
            if (!nd.leaf) lev[n] = 1 + std::max(lev[nd.left], lev[nd.right]);
        }
        for (size_t n = 0; n < f.nodes.size(); n++)
            if (node_br[n] >= 0) f.br_level[node_br[n]] = lev[n];
    }
    f.d = std::max(forced_d, (uint32_t)*std::max_element(f.br_level.begin(), f.br_level.end()));
    int maxf = *std::max_element(f.br_feature.begin(), f.br_feature.end());
    if ((uint32_t)maxf >= f.n_features) { err = "feature index out of range"; return COPSE_EINVAL; }
    for (uint32_t th : f.br_threshold)
        if (f.precision < 32 && th >= (1u << f.precision)) { err = "threshold needs more bits than the precision"; return COPSE_EINVAL; }
    for (int c : f.leaf_class)
        if (c >= (int)f.classes.size()) { err = "class index out of range"; return COPSE_EINVAL; }
    // multiplicities, K, q = K * n_features
    std::vector<uint32_t> kappa(f.n_features, 0);
    for (int fe : f.br_feature) kappa[fe]++;
    f.K = std::max(forced_K, *std::max_element(kappa.begin(), kappa.end()));
    f.q = f.K * f.n_features;
    // Section 4.2.1: thresholds grouped by feature in preorder, padded to K with S = 0
    f.thr_slot.assign(f.q, 0);
    f.slot_branch.assign(f.q, -1);
    std::vector<uint32_t> seen(f.n_features, 0);
    for (uint32_t i = 0; i < f.b; i++) {
        uint32_t fe = (uint32_t)f.br_feature[i];
        uint32_t slot = f.K * fe + seen[fe]++;
        f.thr_slot[slot] = f.br_threshold[i];
        f.slot_branch[slot] = (int32_t)i;
    }
    // Section 4.2.2: R[i][j] = 1 iff padded slot j holds branch i
    f.R.assign((size_t)f.b * f.q, 0);
    for (uint32_t j = 0; j < f.q; j++)
        if (f.slot_branch[j] >= 0) f.R[(size_t)f.slot_branch[j] * f.q + j] = 1;
    // Section 4.2.3-4.2.4.  Branch for label l at level k: the ancestor at level k;
    // else the ancestor with the greatest level below k; else (every ancestor above
    // k) the parent.  A leaf that is a whole tree keeps an empty row and mask 1.
    f.lvl.assign((size_t)f.d * f.L * f.b, 0);
    f.mask.assign((size_t)f.d * f.L, 1);
    for (uint32_t k = 1; k <= f.d; k++) {
        for (uint32_t l = 0; l < f.L; l++) {
            const auto &anc = leaf_anc[l];
            if (anc.empty()) continue;
            int pick = -1, best_below = -1;
            for (size_t a = 0; a < anc.size(); a++) {
                int lv = f.br_level[anc[a].br];
                if ((uint32_t)lv == k) pick = (int)a;
                else if ((uint32_t)lv < k && (best_below < 0 || lv > f.br_level[anc[best_below].br])) best_below = (int)a;
            }
            if (pick < 0) pick = best_below >= 0 ? best_below : (int)anc.size() - 1;
            f.lvl[((size_t)(k - 1) * f.L + l) * f.b + anc[pick].br] = 1;
            f.mask[(size_t)(k - 1) * f.L + l] = anc[pick].right ? 0 : 1;
        }
    }
    return 0;
}

uint32_t pow2_at_least(uint32_t need) {
    uint32_t blk = 1;
    while (blk < need) blk <<= 1;
    return blk;
}

// branch count of one tree
uint32_t tree_branches(const CompiledForest &f, int root) {
    uint32_t n = 0;
    std::vector<int> st{root};
    while (!st.empty()) {
        const int c = st.back();
        st.pop_back();
        if (f.nodes[c].leaf) continue;
        n++;
        st.push_back(f.nodes[c].left);
        st.push_back(f.nodes[c].right);
    }
    return n;
}

}  // namespace

int compile_forest(const char *text, size_t len, uint32_t precision, uint32_t n_features, uint32_t log_n,
                   CompiledForest &f, std::string &err) {
    f = CompiledForest();
    if (!text || precision < 1 || precision > 32 || log_n < 2 || log_n > 17) {
        err = "invalid compile arguments";
        return COPSE_EINVAL;
    }
    // Section 5, Input Representation: label names, then one tree per line
    std::string s(text, len);
    std::istringstream in(s);
    std::string line;
    std::vector<std::string> lines;
    while (std::getline(in, line)) {
        bool blank = line.find_first_not_of(" \t\r") == std::string::npos;
        if (!blank) lines.push_back(line);
    }
    if (lines.size() < 2) {
        err = "forest needs a label line and at least one tree";
        return COPSE_EPARSE;
    }
    {
        std::istringstream ls(lines[0]);
        std::string w;
        while (ls >> w) f.classes.push_back(w);
    }
    for (size_t li = 1; li < lines.size(); li++) {
        Parser p;
        p.f = &f;
        std::istringstream ts(lines[li]);
        std::string w;
        while (ts >> w) p.toks.push_back(w);
        int root = p.node();
        if (root < 0) { err = "tree " + std::to_string(li) + ": " + p.err; return COPSE_EPARSE; }
        if (p.pos != p.toks.size()) { err = "tree " + std::to_string(li) + ": trailing tokens"; return COPSE_EPARSE; }
        f.roots.push_back(root);
    }
    f.precision = precision;
    int maxf = -1;
    for (const ForestNode &nd : f.nodes)
        if (!nd.leaf) maxf = std::max(maxf, nd.feature);
    f.n_features = n_features ? n_features : (uint32_t)(maxf + 1);
    int st = build_structures(f, f.roots, 0, 0, err);
    if (st) return st;
    f.b_total = f.b;
    f.L_total = f.L;
    f.log_n = log_n;
    const uint32_t row = 1u << (log_n - 1);
    f.block = pow2_at_least(f.pd());
    if (f.block > row) {
        // row segments: the trees in n_seg contiguous groups, tree t in group
        // floor(n_seg * (branches of the trees before t) / total branches); the smallest
        // power of two whose common block fits a row (and whose blocks fit the ring)
        std::vector<uint32_t> before(f.roots.size() + 1, 0);
        for (size_t t = 0; t < f.roots.size(); t++) before[t + 1] = before[t] + tree_branches(f, f.roots[t]);
        bool ok = false;
        for (uint32_t S = 2; S <= 64 && S <= f.roots.size() && !ok; S *= 2) {
            std::vector<std::vector<int>> groups(S);
            for (size_t t = 0; t < f.roots.size(); t++)
                groups[std::min<uint64_t>(S - 1, (uint64_t)S * before[t] / f.b_total)].push_back(f.roots[t]);
            if (std::any_of(groups.begin(), groups.end(), [](const std::vector<int> &g) { return g.empty(); })) continue;
            std::vector<CompiledForest> segs(S);
            uint32_t K = 0, d = 0;
            for (int pass = 0; pass < 2; pass++) {
                for (uint32_t g = 0; g < S; g++) {
                    CompiledForest &sg = segs[g];
                    sg.classes = f.classes;
                    sg.nodes = f.nodes;
                    sg.roots = groups[g];
                    sg.n_features = f.n_features;
                    sg.precision = precision;
                    sg.log_n = log_n;
                    st = build_structures(sg, sg.roots, pass ? K : 0, pass ? d : 0, err);
                    if (st) return st;
                    if (!pass) {
                        K = std::max(K, sg.K);
                        d = std::max(d, sg.d);
                    }
                }
            }
            uint32_t bp = 0, Lp = 0;
            for (const CompiledForest &sg : segs) {
                bp = std::max(bp, sg.b);
                Lp = std::max(Lp, sg.L);
            }
            const uint32_t blk = pow2_at_least(Lp + bp - 1 + K * f.n_features - 1);
            if (blk > row || (uint64_t)S * blk > (1ull << log_n)) continue;
            for (CompiledForest &sg : segs) {
                sg.b_total = sg.b;
                sg.L_total = sg.L;
                sg.block = blk;
            }
            f.n_seg = S;
            f.seg = std::move(segs);
            f.K = K;
            f.q = K * f.n_features;
            f.d = d;
            f.b = bp;
            f.L = Lp;
            f.block = blk;
            // the whole-forest arrays are not the layout's: each segment holds its own
            f.thr_slot.clear();
            f.slot_branch.clear();
            f.R.clear();
            f.lvl.clear();
            f.mask.clear();
            ok = true;
        }
        if (!ok) {
            err = "query block of " + std::to_string(f.block) + " slots exceeds a slot row";
            return COPSE_EFIT;
        }
    }
    // nonzero diagonals (of any segment)
    std::vector<uint8_t> dg;
    for (uint32_t i = 0; i < f.q; i++) {
        bool nz = false;
        for (uint32_t sgi = 0; sgi < f.n_seg && !nz; sgi++) {
            f.reshuffle_diagonal(i, dg, sgi);
            nz = std::any_of(dg.begin(), dg.end(), [](uint8_t v) { return v != 0; });
        }
        if (nz) f.rot_reshuffle.push_back(i);
    }
    f.lvl_nonzero.assign(f.d, {});
    std::vector<uint64_t> dl;
    for (uint32_t i = 0; i < f.b; i++) {
        bool any = false;
        for (uint32_t k = 0; k < f.d; k++) {
            bool nz = false;
            for (uint32_t sgi = 0; sgi < f.n_seg && !nz; sgi++) {
                f.level_diagonal(k + 1, i, 2, dl, sgi);
                nz = std::any_of(dl.begin(), dl.end(), [](uint64_t v) { return v != 0; });
            }
            if (nz) f.lvl_nonzero[k].push_back(i);
            any |= nz;
        }
        if (any) f.rot_level.push_back(i);
    }
    return 0;
}

void CompiledForest::shuffle_rotations(std::vector<uint32_t> &out) const {
    const int64_t h = (int64_t)1 << (log_n - 1);
    out.clear();
    for (size_t j = 0; j < shuffle_src.size(); j++)
        if (shuffle_src[j] >= 0) out.push_back((uint32_t)((((int64_t)shuffle_src[j] - (int64_t)j) % h + h) % h));
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
}

void CompiledForest::shuffle_diagonal(uint32_t amount, std::vector<uint32_t> &out) const {
    const int64_t h = (int64_t)1 << (log_n - 1);
    out.assign(shuffle_src.size(), 0u);
    for (size_t j = 0; j < shuffle_src.size(); j++)
        if (shuffle_src[j] >= 0 && (uint32_t)((((int64_t)shuffle_src[j] - (int64_t)j) % h + h) % h) == amount)
            out[j] = 1u;
}

BsgsGroup CompiledForest::group_reshuffle() const {
    if (fused) return BsgsGroup();  // no reshuffle product: folded into the level matrices
    if (!encrypted) return bsgs_group({rot_reshuffle}, g_reshuffle);
    std::vector<uint32_t> all(q);
    for (uint32_t i = 0; i < q; i++) all[i] = i;
    return bsgs_group({all}, g_reshuffle);
}

BsgsGroup CompiledForest::group_level() const {
    if (fused) return bsgs_group(fused_nonzero, g_reshuffle);
    if (!encrypted) return bsgs_group(lvl_nonzero, g_level);
    std::vector<uint32_t> all(b);
    for (uint32_t i = 0; i < b; i++) all[i] = i;
    return bsgs_group(std::vector<std::vector<uint32_t>>(d, all), g_level);
}

bool BsgsGroup::plain() const {
    if (acc.size() != n_mat) return false;
    for (const Acc &a : acc)
        if (a.giant != 0) return false;
    return true;
}

void BsgsGroup::rotations(std::vector<uint32_t> &out) const {
    std::vector<uint32_t> r;
    for (uint32_t b : baby)
        if (b) r.push_back(b);
    for (const Acc &a : acc)
        if (a.giant) r.push_back(a.giant);
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    out = r;
}

BsgsGroup bsgs_group(const std::vector<std::vector<uint32_t>> &nonzero, uint32_t g) {
    BsgsGroup G;
    G.n_mat = (uint32_t)nonzero.size();
    std::vector<uint32_t> babies;
    for (const auto &nz : nonzero)
        for (uint32_t i : nz) babies.push_back(g ? i % g : i);
    std::sort(babies.begin(), babies.end());
    babies.erase(std::unique(babies.begin(), babies.end()), babies.end());
    G.baby = babies;
    auto baby_pos = [&](uint32_t j) {
        return (int)(std::lower_bound(G.baby.begin(), G.baby.end(), j) - G.baby.begin());
    };
    for (uint32_t a = 0; a < G.n_mat; a++) {
        // giant steps of this matrix, ascending (the nonzero lists are ascending)
        std::vector<BsgsGroup::Acc> accs;
        for (uint32_t i : nonzero[a]) {
            const uint32_t giant = g ? i - i % g : 0, j = g ? i % g : i;
            if (accs.empty() || accs.back().giant != giant) {
                BsgsGroup::Acc x;
                x.mat = a;
                x.giant = giant;
                x.diag.assign(G.baby.size(), -1);
                accs.push_back(std::move(x));
            }
            accs.back().diag[baby_pos(j)] = (int32_t)i;
        }
        if (accs.empty()) {  // a zero matrix still yields its (zero) product
            BsgsGroup::Acc x;
            x.mat = a;
            x.diag.assign(G.baby.size(), -1);
            accs.push_back(std::move(x));
        }
        for (auto &x : accs) G.acc.push_back(std::move(x));
    }
    return G;
}

void classify_plain(const CompiledForest &m, const uint32_t *x, uint8_t *bits) {
    size_t leaf = 0;
    for (int root : m.roots) {
        // reached leaf of this tree
        int n = root;
        while (!m.nodes[n].leaf) n = x[m.nodes[n].feature] < m.nodes[n].threshold ? m.nodes[n].right : m.nodes[n].left;
        // number the tree's leaves in preorder
        std::vector<int> st{root};
        while (!st.empty()) {
            int c = st.back();
            st.pop_back();
            if (m.nodes[c].leaf) { bits[leaf++] = c == n ? 1 : 0; continue; }
            st.push_back(m.nodes[c].right);
            st.push_back(m.nodes[c].left);
        }
    }
}
