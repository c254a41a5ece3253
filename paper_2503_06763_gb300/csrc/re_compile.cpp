// Host compiler: regular expression -> segments -> parser NFA -> forward and
// reverse DFA / multi-entry DFA tables (arXiv 2503.06763, Sects. 2.2-3.1,
// App. A).  Runs once per RE; not on the parse path.
//
// Differences in method from a literal reading of the paper (same results):
//  * Classic followers (Eq. classicfollowers) are built by per-operator rules:
//    every numbered sub-expression of e_# starts with its own open parenthesis
//    (or is a single leaf) and ends with its close parenthesis, so each one has
//    exactly one first and one last symbol.
//  * Segments (Fig. segmentalgo) are enumerated forwards: a segment starts at
//    the first symbol of the LST or at a follower of a numbered terminal and
//    extends along Fol through parentheses and ε symbols up to the first
//    end-letter.  The paper extends meta-prefixes backwards; both give the set
//    of maximal meta-prefix + end-letter substrings of LSTs.
//  * NFA transitions out of a segment depend only on its end-letter
//    (Eq. folsegdef), so the image of a segment set S under byte class c is the
//    union of D_p = {σ : first(σ) ∈ Fol(p)} over end-letters p of S matching c,
//    and the reverse image is the union of End_p = {q : end(q) = p} over the
//    matching p with D_p ∩ S ≠ ∅.
//  * The ME-DFA's initial singletons {q} are stepped once at compile time: after
//    its first byte a run from {q} is in D_end(q) (forward) or in the reverse
//    image of {q}, which depends on first(q) only.  Speculative runs therefore
//    start from those sets, one per distinct set ("slot"), and the tables hold
//    the states reachable from I, F and those start sets.
#include <algorithm>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <set>
#include <unordered_map>

#include "re_internal.h"

namespace slpf {
namespace {

// ---------------------------------------------------------------- RE syntax
struct Node {
    enum Kind { TERM, EPS, CAT, ALT, STAR, PLUS, REP } kind;
    std::vector<int> kids;
    uint64_t set[4] = {0, 0, 0, 0};   // byte set for TERM
    uint32_t count = 0;               // REP: lower bound h of e{h}, e{h,k}, e{h,}
    uint32_t hi = 0;                  // REP: upper bound (= count for e{h}; kUnbounded for e{h,})
    uint32_t num = 0;
};

constexpr uint32_t kUnbounded = 0xFFFFFFFFu;
constexpr uint64_t kMaxRepeat = 4096;

struct SyntaxError {
    std::string msg;
};

class Parser {
   public:
    Parser(const unsigned char *s, size_t n, std::vector<Node> &nodes) : s_(s), n_(n), nodes_(nodes) {}
    int parse() {
        int r = alt();
        if (i_ != n_) throw SyntaxError{"unbalanced ')' at offset " + std::to_string(i_)};
        return r;
    }

   private:
    const unsigned char *s_;
    size_t n_, i_ = 0;
    std::vector<Node> &nodes_;

    int make(Node::Kind k, std::vector<int> kids = {}) {
        Node nd;
        nd.kind = k;
        nd.kids = std::move(kids);
        nodes_.push_back(nd);
        return (int)nodes_.size() - 1;
    }
    int term(const uint64_t set[4]) {
        int id = make(Node::TERM);
        std::memcpy(nodes_[id].set, set, sizeof(uint64_t) * 4);
        return id;
    }
    static void add(uint64_t set[4], unsigned b) { set[b >> 6] |= 1ull << (b & 63); }

    unsigned escape() {
        if (i_ >= n_) throw SyntaxError{"dangling backslash"};
        unsigned c = s_[i_++];
        switch (c) {
            case 'n': return 10;
            case 't': return 9;
            case 'r': return 13;
            case 'x': {
                if (i_ + 2 > n_) throw SyntaxError{"bad \\x escape"};
                unsigned v = 0;
                for (int k = 0; k < 2; ++k) {
                    unsigned h = s_[i_++];
                    if (h >= '0' && h <= '9') v = v * 16 + (h - '0');
                    else if (h >= 'a' && h <= 'f') v = v * 16 + (h - 'a' + 10);
                    else if (h >= 'A' && h <= 'F') v = v * 16 + (h - 'A' + 10);
                    else throw SyntaxError{"bad \\x escape"};
                }
                return v;
            }
            default: return c;
        }
    }
    int charset() {  // after '['
        uint64_t set[4] = {0, 0, 0, 0};
        bool neg = false;
        if (i_ < n_ && s_[i_] == '^') { neg = true; ++i_; }
        bool first = true;
        for (;;) {
            if (i_ >= n_) throw SyntaxError{"unterminated '['"};
            unsigned c = s_[i_];
            if (c == ']' && !first) { ++i_; break; }
            first = false;
            unsigned lo;
            if (c == '\\') { ++i_; lo = escape(); } else { lo = c; ++i_; }
            if (i_ + 1 < n_ && s_[i_] == '-' && s_[i_ + 1] != ']') {
                ++i_;
                unsigned hi;
                if (s_[i_] == '\\') { ++i_; hi = escape(); } else { hi = s_[i_++]; }
                if (hi < lo) throw SyntaxError{"reversed range in '['"};
                for (unsigned b = lo; b <= hi; ++b) add(set, b);
            } else {
                add(set, lo);
            }
        }
        if (neg) for (int w = 0; w < 4; ++w) set[w] = ~set[w];
        if (!(set[0] | set[1] | set[2] | set[3])) throw SyntaxError{"empty character set"};
        return term(set);
    }
    int atom() {
        unsigned c = s_[i_];
        if (c == '(') {
            ++i_;
            int r = alt();
            if (i_ >= n_ || s_[i_] != ')') throw SyntaxError{"missing ')'"};
            ++i_;
            return r;
        }
        if (c == '[') { ++i_; return charset(); }
        uint64_t set[4] = {0, 0, 0, 0};
        if (c == '.') {
            ++i_;
            for (int w = 0; w < 4; ++w) set[w] = ~0ull;
            set[0] &= ~(1ull << 10);
            return term(set);
        }
        if (c == '\\') { ++i_; add(set, escape()); return term(set); }
        if (c == '*' || c == '+' || c == '?' || c == '{') throw SyntaxError{"operator without operand"};
        if (c == ']') throw SyntaxError{"unbalanced ']'"};
        ++i_;
        add(set, c);
        return term(set);
    }
    int postfix() {
        int nd = atom();
        while (i_ < n_) {
            unsigned c = s_[i_];
            if (c == '*') { ++i_; nd = make(Node::STAR, {nd}); }
            else if (c == '+') { ++i_; nd = make(Node::PLUS, {nd}); }
            else if (c == '?') { ++i_; int e = make(Node::EPS); nd = make(Node::ALT, {nd, e}); }
            else if (c == '{') {                   // e{h}, e{h,k}, e{h,} (App. A, bounded repetition)
                size_t j = i_ + 1;
                auto number = [&](uint64_t &v) {
                    const size_t j0 = j;
                    v = 0;
                    while (j < n_ && s_[j] >= '0' && s_[j] <= '9' && v <= kMaxRepeat) v = v * 10 + (s_[j++] - '0');
                    return j > j0;
                };
                uint64_t lo = 0, hi = 0;
                bool ok = number(lo);
                bool comma = false, has_hi = false;
                if (ok && j < n_ && s_[j] == ',') { comma = true; ++j; has_hi = number(hi); }
                ok = ok && j < n_ && s_[j] == '}' && lo <= kMaxRepeat && hi <= kMaxRepeat;
                if (ok && !comma) ok = lo >= 1;
                if (ok && has_hi) ok = lo < hi;
                if (!ok)
                    throw SyntaxError{"bounded repetition is e{h} (1 <= h), e{h,k} (h < k) or e{h,}, "
                                      "with bounds up to 4096"};
                i_ = j + 1;
                nd = make(Node::REP, {nd});
                nodes_[nd].count = (uint32_t)lo;
                nodes_[nd].hi = !comma ? (uint32_t)lo : has_hi ? (uint32_t)hi : kUnbounded;
            } else break;
        }
        return nd;
    }
    int seq() {
        std::vector<int> items;
        while (i_ < n_ && s_[i_] != '|' && s_[i_] != ')') items.push_back(postfix());
        if (items.empty()) return make(Node::EPS);
        if (items.size() == 1) return items[0];
        return make(Node::CAT, items);
    }
    int alt() {
        std::vector<int> br{seq()};
        while (i_ < n_ && s_[i_] == '|') { ++i_; br.push_back(seq()); }
        if (br.size() == 1) return br[0];
        return make(Node::ALT, br);
    }
};

// Deep copy (for bounded-repetition expansion).
int clone(std::vector<Node> &nodes, int id) {
    Node cp = nodes[id];
    const std::vector<int> src = nodes[id].kids;   // nodes grows below
    std::vector<int> kids;
    for (int k : src) kids.push_back(clone(nodes, k));
    cp.kids = kids;
    nodes.push_back(cp);
    return (int)nodes.size() - 1;
}

// Bounded repetition (App. A): the node's children become fresh copies of
// its body, so every iteration has its own numbered symbols.  e{h}: h copies;
// e{h,k}: then copies h+1 .. k as nested optionals (e (e (... e?)?)?)?, so a
// tree with j iterations uses copies 1 .. j in order; e{h,}: then copy h+1
// under a star.  With h = 0 the node is the outermost optional (or the star)
// itself, so e{0,1} is the optional e? = (e|ε) and e{0,} the star e*, as App. A
// states for the optional (e? = e{0,1}).
void expand(std::vector<Node> &nodes, int id) {
    for (size_t i = 0; i < nodes[id].kids.size(); ++i) expand(nodes, nodes[id].kids[i]);
    if (nodes[id].kind != Node::REP) return;
    const int body = nodes[id].kids[0];
    const uint32_t h = nodes[id].count, hi = nodes[id].hi;
    bool body_used = false;
    auto fresh = [&]() {                            // the body itself first, then clones
        if (!body_used) { body_used = true; return body; }
        return clone(nodes, body);
    };
    auto add = [&](Node::Kind k, std::vector<int> kids) {
        Node nd;
        nd.kind = k;
        nd.kids = std::move(kids);
        nodes.push_back(nd);
        return (int)nodes.size() - 1;
    };
    std::vector<int> reps;
    for (uint32_t c = 0; c < h; ++c) reps.push_back(fresh());
    if (hi == kUnbounded) {
        const int copy = fresh();
        reps.push_back(add(Node::STAR, {copy}));
    } else if (hi > h) {
        int copy = fresh();
        int tail = add(Node::ALT, {copy, add(Node::EPS, {})});                 // copy k
        for (uint32_t j = 0; j + 1 < hi - h; ++j) {                           // copies k-1 .. h+1 around it
            copy = fresh();
            const int cat = add(Node::CAT, {copy, tail});
            tail = add(Node::ALT, {cat, add(Node::EPS, {})});
        }
        reps.push_back(tail);
    }
    if (h == 0) {                                   // the optional / starred iterations are the node
        const Node only = nodes[reps[0]];
        nodes[id] = only;
        return;
    }
    nodes[id].kids = reps;
}

bool empty_text(const std::vector<Node> &nodes, int id) {
    const Node &n = nodes[id];
    switch (n.kind) {
        case Node::TERM: return false;
        case Node::EPS: return true;
        case Node::STAR: return true;
        case Node::PLUS: return empty_text(nodes, n.kids[0]);
        case Node::ALT:
            for (int k : n.kids) if (empty_text(nodes, k)) return true;
            return false;
        default:
            for (int k : n.kids) if (!empty_text(nodes, k)) return false;
            return true;
    }
}

bool finitely_ambiguous(const std::vector<Node> &nodes, int id) {
    const Node &n = nodes[id];
    if ((n.kind == Node::STAR || n.kind == Node::PLUS) && empty_text(nodes, n.kids[0])) return false;
    for (int k : n.kids) if (!finitely_ambiguous(nodes, k)) return false;
    return true;
}

// ---------------------------------------------------------------- numbered symbols
enum SymKind { OPEN = 0, CLOSE = 1, LEAF_T = 2, LEAF_E = 3, ENDMARK = 4 };
struct Sym {
    SymKind kind;
    uint32_t num;
    int node;
};

struct Bits {  // helpers over W-word bitsets
    static void set(uint64_t *b, uint32_t i) { b[i >> 6] |= 1ull << (i & 63); }
    static bool get(const uint64_t *b, uint32_t i) { return (b[i >> 6] >> (i & 63)) & 1; }
    static bool any_and(const uint64_t *a, const uint64_t *b, uint32_t W) {
        for (uint32_t w = 0; w < W; ++w) if (a[w] & b[w]) return true;
        return false;
    }
    static bool any(const uint64_t *a, uint32_t W) {
        for (uint32_t w = 0; w < W; ++w) if (a[w]) return true;
        return false;
    }
};

// Interning table of segment bitsets -> ids.
class StateTable {
   public:
    explicit StateTable(uint32_t W) : W_(W) { bits_.assign(W, 0); index_.assign(1024, 0); }
    uint32_t size() const { return (uint32_t)(bits_.size() / W_); }  // incl. row 0 (empty)
    const uint64_t *row(uint32_t id) const { return &bits_[(size_t)id * W_]; }
    // Returns id; inserts if absent.  Row 0 is the empty set.
    uint32_t intern(const uint64_t *b, bool &inserted) {
        inserted = false;
        if (!Bits::any(b, W_)) return 0;
        uint64_t mask = index_.size() - 1;
        uint64_t h = bits_hash(b, W_) & mask;
        for (;;) {
            uint32_t id = index_[h];
            if (id == 0) break;
            if (std::memcmp(row(id), b, W_ * 8) == 0) return id;
            h = (h + 1) & mask;
        }
        uint32_t id = size();
        bits_.insert(bits_.end(), b, b + W_);
        index_[h] = id;
        inserted = true;
        if ((uint64_t)size() * 2 > index_.size()) rehash();
        return id;
    }
    const std::vector<uint64_t> &bits() const { return bits_; }

   private:
    void rehash() {
        std::vector<uint32_t> idx(index_.size() * 2, 0);
        uint64_t mask = idx.size() - 1;
        for (uint32_t id = 1; id < size(); ++id) {
            uint64_t h = bits_hash(row(id), W_) & mask;
            while (idx[h]) h = (h + 1) & mask;
            idx[h] = id;
        }
        index_.swap(idx);
    }
    uint32_t W_;
    std::vector<uint64_t> bits_;
    std::vector<uint32_t> index_;
};

std::vector<uint32_t> build_device_hash(const std::vector<uint64_t> &bits, uint32_t n, uint32_t W,
                                        uint32_t &mask_out) {
    uint64_t cap = 16;
    while (cap < (uint64_t)n * 2) cap <<= 1;
    std::vector<uint32_t> h(cap, 0);
    for (uint32_t id = 1; id < n; ++id) {
        uint64_t x = bits_hash(&bits[(size_t)id * W], W) & (cap - 1);
        while (h[x]) x = (x + 1) & (cap - 1);
        h[x] = id;
    }
    mask_out = (uint32_t)(cap - 1);
    return h;
}

}  // namespace

re_status compile_pattern(const char *pattern, size_t len, const re_compile_opts *opts,
                          Compiled &C, std::string &err) {
    uint32_t max_states = (opts && opts->max_states) ? opts->max_states : (1u << 20);
    uint64_t max_dict = (opts && opts->max_dict) ? opts->max_dict : (1ull << 24);
    if (opts && (opts->flags & ~(RE_COMPILE_HOST_ONLY | RE_COMPILE_DFA_STARTS | RE_COMPILE_DFA_STARTS_BWD))) {
        err = "unknown re_compile_opts.flags";
        return RE_E_INVALID_ARG;
    }

    // ---- parse and number (Sects. 2.1, 2.2)
    std::vector<Node> nodes;
    int root;
    try {
        Parser p((const unsigned char *)pattern, len, nodes);
        root = p.parse();
    } catch (const SyntaxError &e) {
        err = "syntax: " + e.msg;
        return RE_E_SYNTAX;
    }
    const uint32_t sample_limit = opts ? opts->sample_limit : 0;
    if (sample_limit > RE_SAMPLE_LIMIT_MAX) {
        err = "re_compile_opts.sample_limit above RE_SAMPLE_LIMIT_MAX";
        return RE_E_INVALID_ARG;
    }
    expand(nodes, root);
    C.inf_amb = !finitely_ambiguous(nodes, root);
    C.sample_limit = sample_limit;
    if (C.inf_amb && sample_limit == 0) {
        err = "an iterated sub-expression derives the empty text (infinitely ambiguous)";
        return RE_E_INFINITE_AMBIGUITY;
    }
    std::vector<Sym> syms;              // all numbered symbols of e_# ⊣
    std::vector<int> first_sym(nodes.size(), -1), last_sym(nodes.size(), -1);
    uint32_t counter = 0;
    std::function<void(int)> number = [&](int id) {
        Node &n = nodes[id];
        n.num = ++counter;
        if (n.kind == Node::TERM || n.kind == Node::EPS) {
            syms.push_back({n.kind == Node::TERM ? LEAF_T : LEAF_E, n.num, id});
            first_sym[id] = last_sym[id] = (int)syms.size() - 1;
            return;
        }
        syms.push_back({OPEN, n.num, id});
        first_sym[id] = (int)syms.size() - 1;
        for (int k : n.kids) number(k);
        syms.push_back({CLOSE, n.num, id});
        last_sym[id] = (int)syms.size() - 1;
    };
    number(root);
    syms.push_back({ENDMARK, 0, -1});
    const int endsym = (int)syms.size() - 1;
    const uint32_t nsym = (uint32_t)syms.size();

    // ---- classic followers, per-operator rules (Eq. classicfollowers)
    std::vector<std::vector<int>> fol(nsym);
    auto link = [&](int a, int b) { fol[a].push_back(b); };
    std::function<void(int)> rules = [&](int id) {
        const Node &n = nodes[id];
        if (n.kind == Node::TERM || n.kind == Node::EPS) return;
        int o = first_sym[id], c = last_sym[id];
        const auto &k = n.kids;
        switch (n.kind) {
            case Node::CAT:
            case Node::REP:
                link(o, first_sym[k[0]]);
                for (size_t i = 0; i + 1 < k.size(); ++i) link(last_sym[k[i]], first_sym[k[i + 1]]);
                link(last_sym[k.back()], c);
                break;
            case Node::ALT:
                for (int ch : k) { link(o, first_sym[ch]); link(last_sym[ch], c); }
                break;
            case Node::STAR:
                link(o, first_sym[k[0]]); link(o, c);
                link(last_sym[k[0]], first_sym[k[0]]); link(last_sym[k[0]], c);
                break;
            case Node::PLUS:
                link(o, first_sym[k[0]]);
                link(last_sym[k[0]], first_sym[k[0]]); link(last_sym[k[0]], c);
                break;
            default: break;
        }
        for (int ch : k) rules(ch);
    };
    rules(root);
    link(last_sym[root], endsym);
    const int lst_first = first_sym[root];
    auto is_end_letter = [&](int s) { return syms[s].kind == LEAF_T || syms[s].kind == ENDMARK; };

    // ---- segments: forward enumeration from every segment start.  Each
    // symbol may occur once on a path (finite ambiguity), or up to
    // sample_limit times when an infinitely ambiguous RE is sampled (App. A,
    // "Infinite ambiguity": counters for the numbered symbols).
    std::set<std::vector<int>> segset;
    std::vector<int> path;
    std::vector<uint32_t> onpath(nsym, 0);
    const uint32_t per_symbol = sample_limit ? sample_limit : 1;
    bool amb = false, over = false;
    size_t budget = 0;
    std::function<void(int)> extend = [&](int s) {
        if (amb || over) return;
        if (++budget > 50000000) { over = true; return; }
        path.push_back(s);
        ++onpath[s];
        if (is_end_letter(s)) {
            segset.insert(path);
        } else {
            for (int nx : fol[s]) {
                if (onpath[nx] >= per_symbol) {
                    if (!sample_limit) { amb = true; break; }
                    continue;
                }
                extend(nx);
            }
        }
        --onpath[s];
        path.pop_back();
    };
    std::vector<char> is_start(nsym, 0);
    is_start[lst_first] = 1;
    for (uint32_t s = 0; s < nsym; ++s)
        if (syms[s].kind == LEAF_T) for (int nx : fol[s]) is_start[nx] = 1;
    for (uint32_t s = 0; s < nsym; ++s) if (is_start[s]) extend((int)s);
    if (amb) { err = "segment enumeration did not terminate (infinite ambiguity)"; return RE_E_INFINITE_AMBIGUITY; }
    if (over) { err = "segment enumeration exceeds its step budget"; return RE_E_TOO_MANY_STATES; }

    // canonical order: lexicographic over symbol keys (number, kind), ⊣ last
    auto key = [&](int s) -> std::pair<uint64_t, int> {
        if (syms[s].kind == ENDMARK) return {1ull << 40, 3};
        int kk = syms[s].kind == OPEN ? 0 : syms[s].kind == CLOSE ? 1 : 2;
        return {syms[s].num, kk};
    };
    std::vector<std::vector<int>> segs(segset.begin(), segset.end());
    std::sort(segs.begin(), segs.end(), [&](const std::vector<int> &a, const std::vector<int> &b) {
        size_t m = std::min(a.size(), b.size());
        for (size_t i = 0; i < m; ++i) {
            auto ka = key(a[i]), kb = key(b[i]);
            if (ka != kb) return ka < kb;
        }
        return a.size() < b.size();
    });
    const uint32_t ell = (uint32_t)segs.size();
    const uint32_t W = (ell + 63) / 64;
    C.ell = ell;
    C.W = W;
    C.names.clear();
    for (auto &sg : segs) {
        std::string nm;
        for (size_t i = 0; i < sg.size(); ++i) {
            const Sym &y = syms[sg[i]];
            if (i) nm += ' ';
            switch (y.kind) {
                case OPEN: nm += std::to_string(y.num) + "("; break;
                case CLOSE: nm += ")" + std::to_string(y.num); break;
                case LEAF_T: nm += "t" + std::to_string(y.num); break;
                case LEAF_E: nm += "e" + std::to_string(y.num); break;
                case ENDMARK: nm += "$"; break;
            }
        }
        C.names.push_back(nm);
        std::vector<int32_t> pr;
        for (int sy : sg) {
            const Sym &y = syms[sy];
            if (y.kind == OPEN) pr.push_back(y.num);
            else if (y.kind == CLOSE) pr.push_back(-y.num);
            if (y.kind == OPEN || y.kind == CLOSE) C.max_group = std::max<uint32_t>(C.max_group, y.num);
        }
        C.parens.push_back(std::move(pr));
    }

    // ---- positions (numbered terminals) and byte classes (App. A)
    std::vector<int> pos_of_sym(nsym, -1), pos_sym;
    for (uint32_t s = 0; s < nsym; ++s)
        if (syms[s].kind == LEAF_T) { pos_of_sym[s] = (int)pos_sym.size(); pos_sym.push_back((int)s); }
    const uint32_t P = (uint32_t)pos_sym.size();
    C.npos = P;
    {
        std::map<std::vector<uint64_t>, uint32_t> sig2cls;
        std::vector<uint64_t> sig((P + 63) / 64 + 1);
        for (unsigned b = 0; b < 256; ++b) {
            std::fill(sig.begin(), sig.end(), 0);
            for (uint32_t p = 0; p < P; ++p) {
                const Node &n = nodes[syms[pos_sym[p]].node];
                if ((n.set[b >> 6] >> (b & 63)) & 1) sig[p >> 6] |= 1ull << (p & 63);
            }
            auto it = sig2cls.find(sig);
            if (it == sig2cls.end()) it = sig2cls.emplace(sig, (uint32_t)sig2cls.size()).first;
            C.cls[b] = (uint8_t)it->second;
        }
        C.ncls = (uint32_t)sig2cls.size();
    }
    const uint32_t ncls = C.ncls;
    std::vector<uint8_t> pos_match((size_t)P * ncls, 0);   // p matches class c
    for (unsigned b = 0; b < 256; ++b)
        for (uint32_t p = 0; p < P; ++p) {
            const Node &n = nodes[syms[pos_sym[p]].node];
            if ((n.set[b >> 6] >> (b & 63)) & 1) pos_match[(size_t)p * ncls + C.cls[b]] = 1;
        }

    // ---- per-position masks: End_p = {q : end(q) = p},  D_p = {σ : first(σ) ∈ Fol(p)}
    std::vector<uint64_t> End((size_t)P * W, 0), D((size_t)P * W, 0);
    std::vector<int> seg_end_pos(ell), seg_first(ell);
    std::vector<uint64_t> Iset(W, 0), Fset(W, 0);
    for (uint32_t q = 0; q < ell; ++q) {
        int e = segs[q].back();
        seg_end_pos[q] = pos_of_sym[e];
        seg_first[q] = segs[q].front();
        if (seg_end_pos[q] >= 0) Bits::set(&End[(size_t)seg_end_pos[q] * W], q);
        if (segs[q].front() == lst_first) Bits::set(Iset.data(), q);
        if (e == endsym) Bits::set(Fset.data(), q);
    }
    for (uint32_t p = 0; p < P; ++p) {
        std::vector<char> f(nsym, 0);
        for (int nx : fol[pos_sym[p]]) f[nx] = 1;
        for (uint32_t q = 0; q < ell; ++q) if (f[seg_first[q]]) Bits::set(&D[(size_t)p * W], q);
    }
    // FolSeg(q) = D_end(q) (Eq. folsegdef); a segment ending in ⊣ has no follower
    C.folseg.assign((size_t)ell * W, 0);
    for (uint32_t q = 0; q < ell; ++q)
        if (seg_end_pos[q] >= 0)
            std::copy(&D[(size_t)seg_end_pos[q] * W], &D[(size_t)seg_end_pos[q] * W] + W, &C.folseg[(size_t)q * W]);
    std::vector<std::vector<uint32_t>> match_pos(ncls);
    for (uint32_t c = 0; c < ncls; ++c)
        for (uint32_t p = 0; p < P; ++p) if (pos_match[(size_t)p * ncls + c]) match_pos[c].push_back(p);

    auto fwd_image = [&](const uint64_t *S, uint32_t c, uint64_t *out) {
        std::fill(out, out + W, 0);
        for (uint32_t p : match_pos[c])
            if (Bits::any_and(S, &End[(size_t)p * W], W))
                for (uint32_t w = 0; w < W; ++w) out[w] |= D[(size_t)p * W + w];
    };
    auto bwd_image = [&](const uint64_t *S, uint32_t c, uint64_t *out) {
        std::fill(out, out + W, 0);
        for (uint32_t p : match_pos[c])
            if (Bits::any_and(S, &D[(size_t)p * W], W))
                for (uint32_t w = 0; w < W; ++w) out[w] |= End[(size_t)p * W + w];
    };

    // ---- powerset exploration (Sect. 3.1): classic DFA first, then the ME-DFA part
    auto explore = [&](StateTable &tab, std::vector<uint32_t> &T, const std::vector<uint64_t> &seeds,
                       size_t nseeds_dfa, uint32_t &ndfa, bool reverse) -> bool {
        std::vector<uint64_t> tmp(W);
        size_t next = 1;  // BFS over ids
        auto run_bfs = [&]() -> bool {
            while (next < tab.size()) {
                uint32_t id = (uint32_t)next++;
                std::vector<uint64_t> S(tab.row(id), tab.row(id) + W);
                for (uint32_t c = 0; c < ncls; ++c) {
                    if (reverse) bwd_image(S.data(), c, tmp.data());
                    else fwd_image(S.data(), c, tmp.data());
                    bool ins;
                    uint32_t t = tab.intern(tmp.data(), ins);
                    if (T.size() < (size_t)(id + 1) * ncls) T.resize((size_t)(id + 1) * ncls, 0);
                    T[(size_t)id * ncls + c] = t;
                    if (tab.size() > max_states) return false;
                }
            }
            return true;
        };
        T.assign(ncls, 0);  // row 0: empty set stays empty
        bool ins;
        for (size_t s = 0; s < nseeds_dfa; ++s) tab.intern(&seeds[s * W], ins);
        if (!run_bfs()) return false;
        ndfa = tab.size() - 1;
        for (size_t s = nseeds_dfa; s < seeds.size() / W; ++s) tab.intern(&seeds[s * W], ins);
        if (!run_bfs()) return false;
        T.resize((size_t)tab.size() * ncls, 0);
        return true;
    };

    // forward seeds: I, then every D_p
    std::vector<uint64_t> fseeds(Iset);
    for (uint32_t p = 0; p < P; ++p) fseeds.insert(fseeds.end(), &D[(size_t)p * W], &D[(size_t)(p + 1) * W]);
    // reverse seeds: F, then the reverse image of {q} for every first symbol and class
    std::vector<int> bkey_syms;     // distinct first symbols of segments
    std::vector<int> bkey_of_sym(nsym, -1);
    for (uint32_t q = 0; q < ell; ++q)
        if (bkey_of_sym[seg_first[q]] < 0) { bkey_of_sym[seg_first[q]] = (int)bkey_syms.size(); bkey_syms.push_back(seg_first[q]); }
    const uint32_t K = (uint32_t)bkey_syms.size();
    // Pred_f image under class c: ∪ End_p over p matching c with f ∈ Fol(p)
    std::vector<uint64_t> bstart((size_t)K * ncls * W, 0);
    for (uint32_t kf = 0; kf < K; ++kf)
        for (uint32_t c = 0; c < ncls; ++c)
            for (uint32_t p : match_pos[c]) {
                bool fo = false;
                for (int nx : fol[pos_sym[p]]) if (nx == bkey_syms[kf]) { fo = true; break; }
                if (fo) for (uint32_t w = 0; w < W; ++w) bstart[((size_t)kf * ncls + c) * W + w] |= End[(size_t)p * W + w];
            }
    std::vector<uint64_t> bseeds(Fset);
    bseeds.insert(bseeds.end(), bstart.begin(), bstart.end());

    StateTable ftab(W), btab(W);
    uint32_t nfd = 0, nbd = 0;
    if (!explore(ftab, C.fT, fseeds, 1, nfd, false) || !explore(btab, C.bT, bseeds, 1, nbd, true) ||
        ftab.size() + btab.size() > max_states) {
        err = "automaton exceeds max_states";
        return RE_E_TOO_MANY_STATES;
    }
    C.nf = ftab.size(); C.nb = btab.size(); C.nfd = nfd; C.nbd = nbd;
    C.fBits = ftab.bits(); C.bBits = btab.bits();
    uint32_t fI, bF;
    { bool ins; fI = ftab.intern(Iset.data(), ins); bF = btab.intern(Fset.data(), ins); }
    if (fI != 1 || bF != 1) { err = "internal: I / F ids"; return RE_E_INTERNAL; }

    // ---- speculation slots per (class before the boundary, class after it)
    // Forward keys: end positions p matching the first byte whose segments can
    // follow a byte of the previous class (the last-character filter of PaREM,
    // Sect. 6); grouped by start set D_p.
    std::vector<uint64_t> succ((size_t)ncls * W, 0);   // ∪ D_p over p matching c
    for (uint32_t c = 0; c < ncls; ++c)
        for (uint32_t p : match_pos[c]) for (uint32_t w = 0; w < W; ++w) succ[(size_t)c * W + w] |= D[(size_t)p * W + w];
    // Backward keys: first symbols f of segments whose end-letter matches the
    // next class, with a non-empty reverse image under the last class.
    std::vector<std::vector<std::pair<uint32_t, std::vector<uint64_t>>>> fsl(ncls * ncls), bsl(ncls * ncls);
    uint32_t msf = 1, msb = 1;
    for (uint32_t cp = 0; cp < ncls; ++cp)
        for (uint32_t cf = 0; cf < ncls; ++cf) {
            auto &L = fsl[cp * ncls + cf];
            std::map<uint32_t, size_t> by_start;
            for (uint32_t p : match_pos[cf]) {
                if (!Bits::any_and(&End[(size_t)p * W], &succ[(size_t)cp * W], W)) continue;
                bool ins;
                uint32_t st = ftab.intern(&D[(size_t)p * W], ins);
                if (ins) { err = "internal: forward start set missing"; return RE_E_INTERNAL; }
                if (st == 0) continue;   // D_p empty: the run dies on the next byte; contributes nothing
                auto it = by_start.find(st);
                if (it == by_start.end()) { it = by_start.emplace(st, L.size()).first; L.push_back({st, std::vector<uint64_t>(W, 0)}); }
                for (uint32_t w = 0; w < W; ++w) L[it->second].second[w] |= End[(size_t)p * W + w];
            }
            msf = std::max<uint32_t>(msf, (uint32_t)L.size());
        }
    // Note on forward keys with empty D_p: only ⊣-ending segments have no
    // followers and they end in ⊣, which matches no byte; a terminal always has
    // at least one follower, so D_p is never empty for a position p.
    for (uint32_t cl = 0; cl < ncls; ++cl)
        for (uint32_t cn = 0; cn < ncls; ++cn) {
            auto &L = bsl[cl * ncls + cn];
            std::map<uint32_t, size_t> by_start;
            for (uint32_t kf = 0; kf < K; ++kf) {
                std::vector<uint64_t> segmask(W, 0);
                for (uint32_t q = 0; q < ell; ++q)
                    if (seg_first[q] == bkey_syms[kf] && seg_end_pos[q] >= 0 &&
                        pos_match[(size_t)seg_end_pos[q] * ncls + cn])
                        Bits::set(segmask.data(), q);
                if (!Bits::any(segmask.data(), W)) continue;
                const uint64_t *st_bits = &bstart[((size_t)kf * ncls + cl) * W];
                bool ins;
                uint32_t st = btab.intern(st_bits, ins);
                if (ins) { err = "internal: reverse start set missing"; return RE_E_INTERNAL; }
                if (st == 0) continue;
                auto it = by_start.find(st);
                if (it == by_start.end()) { it = by_start.emplace(st, L.size()).first; L.push_back({st, std::vector<uint64_t>(W, 0)}); }
                for (uint32_t w = 0; w < W; ++w) L[it->second].second[w] |= segmask[w];
            }
            msb = std::max<uint32_t>(msb, (uint32_t)L.size());
        }
    if (opts && (opts->flags & RE_COMPILE_DFA_STARTS)) {
        // Ablation: forward runs from every classic DFA state s (ids 1..nfd,
        // reachable from I), one slot per distinct state after the first
        // byte; an input state enters exactly the slot of its own successor.
        const uint32_t nf = ftab.size();
        C.fSlotOf.assign((size_t)ncls * ncls * nf, 0xFF);
        msf = 1;
        for (uint32_t cp = 0; cp < ncls; ++cp)
            for (uint32_t cf = 0; cf < ncls; ++cf) {
                const uint32_t pr = cp * ncls + cf;
                auto &L = fsl[pr];
                L.clear();
                std::map<uint32_t, size_t> by_start;
                for (uint32_t st = 1; st <= nfd; ++st) {
                    const uint32_t nx = C.fT[(size_t)st * ncls + cf];
                    if (nx == 0) continue;                 // the text cannot continue from st
                    auto it = by_start.find(nx);
                    if (it == by_start.end()) {
                        it = by_start.emplace(nx, L.size()).first;
                        L.push_back({nx, std::vector<uint64_t>(W, 0)});   // keys unused: exact lookup
                    }
                    if (it->second < 0xFF) C.fSlotOf[(size_t)pr * nf + st] = (uint8_t)it->second;
                }
                msf = std::max<uint32_t>(msf, (uint32_t)L.size());
            }
    }
    if (opts && (opts->flags & RE_COMPILE_DFA_STARTS_BWD)) {
        // The same ablation backwards: runs from every reverse DFA state
        // (ids 1..nbd, reachable from F), one slot per distinct state after
        // the chunk's last byte (class cl); the class after the chunk plays
        // no part, so every pair (cl, cn) has the same slots.
        const uint32_t nb = btab.size();
        C.bSlotOf.assign((size_t)ncls * ncls * nb, 0xFF);
        msb = 1;
        for (uint32_t cl = 0; cl < ncls; ++cl)
            for (uint32_t cn = 0; cn < ncls; ++cn) {
                const uint32_t pr = cl * ncls + cn;
                auto &L = bsl[pr];
                L.clear();
                std::map<uint32_t, size_t> by_start;
                for (uint32_t st = 1; st <= nbd; ++st) {
                    const uint32_t nx = C.bT[(size_t)st * ncls + cl];
                    if (nx == 0) continue;                 // no text continues leftwards from st
                    auto it = by_start.find(nx);
                    if (it == by_start.end()) {
                        it = by_start.emplace(nx, L.size()).first;
                        L.push_back({nx, std::vector<uint64_t>(W, 0)});   // keys unused: exact lookup
                    }
                    if (it->second < 0xFF) C.bSlotOf[(size_t)pr * nb + st] = (uint8_t)it->second;
                }
                msb = std::max<uint32_t>(msb, (uint32_t)L.size());
            }
    }
    C.msf = msf; C.msb = msb;
    C.fSlotStart.assign((size_t)ncls * ncls * msf, 0);
    C.fSlotMask.assign((size_t)ncls * ncls * msf * W, 0);
    C.fSlotCount.assign((size_t)ncls * ncls, 0);
    C.bSlotStart.assign((size_t)ncls * ncls * msb, 0);
    C.bSlotMask.assign((size_t)ncls * ncls * msb * W, 0);
    C.bSlotCount.assign((size_t)ncls * ncls, 0);
    for (uint32_t pr = 0; pr < ncls * ncls; ++pr) {
        C.fSlotCount[pr] = (uint32_t)fsl[pr].size();
        for (size_t j = 0; j < fsl[pr].size(); ++j) {
            C.fSlotStart[(size_t)pr * msf + j] = fsl[pr][j].first;
            std::copy(fsl[pr][j].second.begin(), fsl[pr][j].second.end(), &C.fSlotMask[((size_t)pr * msf + j) * W]);
        }
        C.bSlotCount[pr] = (uint32_t)bsl[pr].size();
        for (size_t j = 0; j < bsl[pr].size(); ++j) {
            C.bSlotStart[(size_t)pr * msb + j] = bsl[pr][j].first;
            std::copy(bsl[pr][j].second.begin(), bsl[pr][j].second.end(), &C.bSlotMask[((size_t)pr * msb + j) * W]);
        }
    }

    // ---- column dictionary: every non-empty B ∩ B̂ over classic-DFA state pairs
    C.has_dict = false;
    C.dict.clear(); C.pt.clear(); C.dict_size = 0;
    if ((uint64_t)C.nf * C.nb <= max_dict) {
        StateTable cols(W);
        // raw pair table over all states; pairs the parse can produce are
        // (DFA state reachable from I, reverse DFA state reachable from F)
        std::vector<uint32_t> raw((size_t)C.nf * C.nb, 0xFFFFFFFFu);
        std::vector<uint64_t> tmp(W);
        for (uint32_t f = 0; f < C.nf; ++f)
            for (uint32_t b = 0; b < C.nb; ++b) {
                if (f == 0 || b == 0) { raw[(size_t)f * C.nb + b] = 0; continue; }   // an empty side
                if (f > nfd || b > nbd) continue;                                  // never produced
                for (uint32_t w = 0; w < W; ++w) tmp[w] = ftab.row(f)[w] & btab.row(b)[w];
                bool ins;
                raw[(size_t)f * C.nb + b] = cols.intern(tmp.data(), ins);
            }
        uint32_t D0 = cols.size() - 1;
        if (D0 < 0xFFFFFFF0u) {
            // canonical order: ascending segment-id lists compared lexicographically
            std::vector<uint32_t> order(D0);
            for (uint32_t i = 0; i < D0; ++i) order[i] = i + 1;
            // x < y iff, at the lowest segment id where they differ, the list
            // that continues with the larger id is y, or x has no more ids.
            auto list_less = [&](uint32_t a, uint32_t b) {
                const uint64_t *x = cols.row(a), *y = cols.row(b);
                for (uint32_t w = 0; w < W; ++w) {
                    uint64_t d = x[w] ^ y[w];
                    if (!d) continue;
                    uint32_t bit = (uint32_t)__builtin_ctzll(d);
                    const uint64_t *has = ((x[w] >> bit) & 1) ? x : y;     // owns id d
                    const uint64_t *other = has == x ? y : x;
                    // does `other` have any id above d?
                    bool other_more = (bit < 63 && (other[w] >> (bit + 1)) != 0);
                    for (uint32_t v = w + 1; v < W && !other_more; ++v) other_more = other[v] != 0;
                    bool has_smaller = other_more;   // `has` continues with d < other's next id
                    return has == x ? has_smaller : !has_smaller;
                }
                return false;
            };
            std::sort(order.begin(), order.end(), list_less);
            std::vector<uint32_t> rank(D0 + 1, 0);
            for (uint32_t i = 0; i < D0; ++i) rank[order[i]] = i + 1;
            C.pt.resize(raw.size());
            for (size_t i = 0; i < raw.size(); ++i) C.pt[i] = raw[i] == 0xFFFFFFFFu ? 0xFFFFFFFFu : rank[raw[i]];
            C.dict.resize((size_t)D0 * W);
            for (uint32_t i = 0; i < D0; ++i) std::copy(cols.row(order[i]), cols.row(order[i]) + W, &C.dict[(size_t)i * W]);
            C.dict_size = D0;
            C.has_dict = true;
        }
    }

    // ---- device probe tables
    // ---- two-byte tables for small class alphabets: one lookup per byte pair.
    // Forward entry (s, c1, c2): mid = δ(s, c1), end = δ(mid, c2); backward
    // entry: mid = δ̂(s, c2), end = δ̂(mid, c1) (the right byte is read first).
    C.f2.clear(); C.b2.clear();
    if (ncls <= 16 && C.nf < 65536 && C.nb < 65536 &&
        (uint64_t)(C.nf + C.nb) * ncls * ncls * 4 <= 48 * 1024) {
        const uint32_t nc2 = ncls * ncls;
        C.f2.resize((size_t)C.nf * nc2);
        C.b2.resize((size_t)C.nb * nc2);
        for (uint32_t st = 0; st < C.nf; ++st)
            for (uint32_t c1 = 0; c1 < ncls; ++c1)
                for (uint32_t c2 = 0; c2 < ncls; ++c2) {
                    const uint32_t mid = C.fT[(size_t)st * ncls + c1];
                    C.f2[(size_t)st * nc2 + c1 * ncls + c2] = mid | (C.fT[(size_t)mid * ncls + c2] << 16);
                }
        for (uint32_t st = 0; st < C.nb; ++st)
            for (uint32_t c1 = 0; c1 < ncls; ++c1)
                for (uint32_t c2 = 0; c2 < ncls; ++c2) {
                    const uint32_t mid = C.bT[(size_t)st * ncls + c2];
                    C.b2[(size_t)st * nc2 + c1 * ncls + c2] = mid | (C.bT[(size_t)mid * ncls + c1] << 16);
                }
    }
    // ---- byte-indexed one-byte tables (states fit a byte): the reach looks a
    // transition up by the text byte itself, with no class lookup first.
    C.fbyte.clear(); C.bbyte.clear();
    if (C.nf <= 256 && C.nb <= 256) {
        C.fbyte.resize((size_t)C.nf * 256);
        C.bbyte.resize((size_t)C.nb * 256);
        for (uint32_t st = 0; st < C.nf; ++st)
            for (uint32_t b = 0; b < 256; ++b) C.fbyte[(size_t)st * 256 + b] = (uint8_t)C.fT[(size_t)st * ncls + C.cls[b]];
        for (uint32_t st = 0; st < C.nb; ++st)
            for (uint32_t b = 0; b < 256; ++b) C.bbyte[(size_t)st * 256 + b] = (uint8_t)C.bT[(size_t)st * ncls + C.cls[b]];
    }
    // ---- bytes 128..255 folded onto bytes below 128 of the same class: when
    // every class holding a byte >= 128 also holds one below, the byte-indexed
    // rows need only their first 128 entries (half the shared memory, so a
    // reach block holds more warps), and a byte >= 128 is replaced by the
    // smallest byte of its class before the lookup.
    C.hirep.clear();
    if (!C.fbyte.empty()) {
        int rep[256];
        for (int &r : rep) r = -1;
        for (int b = 127; b >= 0; --b) rep[C.cls[b]] = b;
        C.hirep.resize(128);
        for (int b = 128; b < 256; ++b) {
            if (rep[C.cls[b]] < 0) { C.hirep.clear(); break; }
            C.hirep[b - 128] = (uint8_t)rep[C.cls[b]];
        }
    }
    C.fHash = build_device_hash(C.fBits, C.nf, W, C.fHashMask);
    C.bHash = build_device_hash(C.bBits, C.nb, W, C.bHashMask);
    return RE_OK;
}

}  // namespace slpf
