// Query compilation: regular expression over labels and inverse labels ->
// minimised DFA with the dead state removed (section 5.2 of the paper turns
// every query into a minimised DFA; section 4 explains why: with a DFA each
// N^a has at most |Q| non-zero entries, so the product with G^a is cheap).
//
// Route: parse -> push inverses down to the symbols (R^- reverses words and
// inverts symbols, section 4) -> Glushkov position automaton (epsilon-free)
// -> subset construction over the symbols that occur -> Moore partition
// refinement -> drop states that cannot reach a final state.
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>

#include "rpq_internal.h"

namespace rpq {
namespace {

enum Kind { SYM, CAT, ALT, STAR, PLUS, OPT, INV };

struct Node {
    Kind k;
    int sym;   // SYM
    int a, b;  // children
};

struct Parser {
    const char *s;
    size_t i = 0, n;
    int32_t L;
    std::vector<Node> nodes;
    std::string err;
    rpq_status err_status = RPQ_ERR_PARSE;

    Parser(const char *t, int32_t L_) : s(t), n(strlen(t)), L(L_) {}

    int add(Node x) {
        nodes.push_back(x);
        return (int)nodes.size() - 1;
    }
    void skip_ws() {
        while (i < n && (s[i] == ' ' || s[i] == '\t' || s[i] == '\n' || s[i] == '\r')) i++;
    }
    // Concatenation separators: '/', '.', U+00B7 (UTF-8 C2 B7).
    bool take_cat() {
        skip_ws();
        if (i < n && (s[i] == '/' || s[i] == '.')) { i++; return true; }
        if (i + 1 < n && (unsigned char)s[i] == 0xC2 && (unsigned char)s[i + 1] == 0xB7) {
            i += 2;
            return true;
        }
        return false;
    }
    bool starts_atom() {
        skip_ws();
        return i < n && (isdigit((unsigned char)s[i]) || s[i] == '^' || s[i] == '(');
    }
    int fail_at(const char *what) {
        if (err.empty()) err = std::string(what) + " at offset " + std::to_string(i);
        return -1;
    }
    int alt() {
        int x = seq();
        if (x < 0) return -1;
        for (;;) {
            skip_ws();
            if (i < n && s[i] == '|') {
                i++;
                int y = seq();
                if (y < 0) return -1;
                x = add({ALT, 0, x, y});
            } else {
                return x;
            }
        }
    }
    int seq() {
        int x = post();
        if (x < 0) return -1;
        for (;;) {
            if (take_cat()) {
                int y = post();
                if (y < 0) return -1;
                x = add({CAT, 0, x, y});
            } else if (starts_atom()) {
                int y = post();
                if (y < 0) return -1;
                x = add({CAT, 0, x, y});
            } else {
                return x;
            }
        }
    }
    int post() {
        int x = atom();
        if (x < 0) return -1;
        for (;;) {
            skip_ws();
            if (i < n && s[i] == '*') { i++; x = add({STAR, 0, x, -1}); }
            else if (i < n && s[i] == '+') { i++; x = add({PLUS, 0, x, -1}); }
            else if (i < n && s[i] == '?') { i++; x = add({OPT, 0, x, -1}); }
            else return x;
        }
    }
    int atom() {
        skip_ws();
        if (i >= n) return fail_at("unexpected end of expression");
        char c = s[i];
        if (isdigit((unsigned char)c)) {
            int64_t v = 0;
            while (i < n && isdigit((unsigned char)s[i])) {
                v = v * 10 + (s[i] - '0');
                if (v > 0x7fffffff) v = 0x7fffffff;
                i++;
            }
            if (v >= L) {
                err_status = RPQ_ERR_INVALID;
                err = "label " + std::to_string(v) + " outside [0, " + std::to_string(L) + ")";
                return -1;
            }
            return add({SYM, (int)v, -1, -1});
        }
        if (c == '^') {
            i++;
            int x = atom();
            if (x < 0) return -1;
            return add({INV, 0, x, -1});
        }
        if (c == '(') {
            i++;
            int x = alt();
            if (x < 0) return -1;
            skip_ws();
            if (i >= n || s[i] != ')') return fail_at("expected ')'");
            i++;
            return x;
        }
        return fail_at("unexpected character");
    }
};

// Rewrites node x (under `inv` inversions) into a tree without INV nodes.
int push_inverse(std::vector<Node> &in, std::vector<Node> &out, int x, bool inv, int32_t L) {
    const Node nd = in[x];
    auto add = [&](Node y) { out.push_back(y); return (int)out.size() - 1; };
    switch (nd.k) {
        case SYM: return add({SYM, inv ? nd.sym + L : nd.sym, -1, -1});
        case INV: return push_inverse(in, out, nd.a, !inv, L);
        case CAT: {
            int l = push_inverse(in, out, inv ? nd.b : nd.a, inv, L);
            int r = push_inverse(in, out, inv ? nd.a : nd.b, inv, L);
            return add({CAT, 0, l, r});
        }
        case ALT: {
            int l = push_inverse(in, out, nd.a, inv, L);
            int r = push_inverse(in, out, nd.b, inv, L);
            return add({ALT, 0, l, r});
        }
        default: {
            int c = push_inverse(in, out, nd.a, inv, L);
            return add({nd.k, 0, c, -1});
        }
    }
}

using PosSet = std::vector<int>;

void set_union(PosSet &dst, const PosSet &src) {
    PosSet r;
    r.reserve(dst.size() + src.size());
    std::set_union(dst.begin(), dst.end(), src.begin(), src.end(), std::back_inserter(r));
    dst.swap(r);
}

struct Glushkov {
    std::vector<Node> &t;
    std::vector<int> pos_sym;          // symbol of each position
    std::vector<PosSet> follow;        // follow set of each position
    std::vector<int> node_pos;         // position of each SYM node
    struct Info { bool nullable; PosSet first, last; };

    explicit Glushkov(std::vector<Node> &tree) : t(tree), node_pos(tree.size(), -1) {}

    Info run(int x) {
        const Node nd = t[x];
        switch (nd.k) {
            case SYM: {
                int p = (int)pos_sym.size();
                pos_sym.push_back(nd.sym);
                follow.emplace_back();
                return {false, {p}, {p}};
            }
            case CAT: {
                Info X = run(nd.a), Y = run(nd.b);
                for (int p : X.last) set_union(follow[p], Y.first);
                Info r;
                r.nullable = X.nullable && Y.nullable;
                r.first = X.first;
                if (X.nullable) set_union(r.first, Y.first);
                r.last = Y.last;
                if (Y.nullable) set_union(r.last, X.last);
                return r;
            }
            case ALT: {
                Info X = run(nd.a), Y = run(nd.b);
                Info r;
                r.nullable = X.nullable || Y.nullable;
                r.first = X.first; set_union(r.first, Y.first);
                r.last = X.last; set_union(r.last, Y.last);
                return r;
            }
            case STAR:
            case PLUS: {
                Info X = run(nd.a);
                for (int p : X.last) set_union(follow[p], X.first);
                if (nd.k == STAR) X.nullable = true;
                return X;
            }
            case OPT: {
                Info X = run(nd.a);
                X.nullable = true;
                return X;
            }
            default: return {false, {}, {}};
        }
    }
};

}  // namespace

rpq_status compile_regex(const char *text, int32_t n_labels, Automaton *out) {
    if (!text || !out) return fail(RPQ_ERR_INVALID, "null argument");
    if (n_labels <= 0) return fail(RPQ_ERR_INVALID, "n_labels must be positive");
    if (strlen(text) > 65536) return fail(RPQ_ERR_INVALID, "expression longer than 65536 bytes");
    Parser ps(text, n_labels);
    int root = ps.alt();
    ps.skip_ws();
    if (root >= 0 && ps.i != ps.n) root = ps.fail_at("trailing input");
    if (root < 0) return fail(ps.err_status, "regex: %s", ps.err.c_str());

    std::vector<Node> tree;
    int r2 = push_inverse(ps.nodes, tree, root, false, n_labels);
    Glushkov G(tree);
    Glushkov::Info top = G.run(r2);
    const int P = (int)G.pos_sym.size();
    if (P > 8192) return fail(RPQ_ERR_INVALID, "expression has more than 8192 label occurrences");

    // Glushkov NFA: state 0 initial, state p+1 for position p.
    // Alphabet: symbols that occur.
    std::vector<int> alphabet(G.pos_sym.begin(), G.pos_sym.end());
    std::sort(alphabet.begin(), alphabet.end());
    alphabet.erase(std::unique(alphabet.begin(), alphabet.end()), alphabet.end());
    const int A = (int)alphabet.size();
    std::vector<int> sym_index(2 * (size_t)n_labels, -1);
    for (int k = 0; k < A; k++) sym_index[alphabet[k]] = k;
    std::vector<char> is_last(P, 0);
    for (int p : top.last) is_last[p] = 1;

    // Subset construction.  A DFA state is a sorted set of NFA states.
    const int kMaxDfa = 4096;
    std::map<PosSet, int> ids;
    std::vector<PosSet> sets;
    std::vector<std::vector<int>> dtrans;  // [state][symbol index] -> state or -1
    std::vector<char> dfinal;
    auto intern = [&](const PosSet &s, bool fin) -> int {
        auto it = ids.find(s);
        if (it != ids.end()) return it->second;
        int id = (int)sets.size();
        ids.emplace(s, id);
        sets.push_back(s);
        dtrans.emplace_back(A, -1);
        dfinal.push_back(fin ? 1 : 0);
        return id;
    };
    // NFA state 0 is the initial state; we represent it as -1 in sets.
    intern(PosSet{-1}, top.nullable);
    for (size_t cur = 0; cur < sets.size(); cur++) {
        if ((int)sets.size() > kMaxDfa)
            return fail(RPQ_ERR_INVALID, "subset construction exceeded %d states", kMaxDfa);
        std::vector<PosSet> next(A);
        for (int q : sets[cur]) {
            const PosSet &succ = (q < 0) ? top.first : G.follow[q];
            for (int p : succ) next[sym_index[G.pos_sym[p]]].push_back(p);
        }
        for (int k = 0; k < A; k++) {
            PosSet &s = next[k];
            if (s.empty()) continue;
            std::sort(s.begin(), s.end());
            s.erase(std::unique(s.begin(), s.end()), s.end());
            bool fin = false;
            for (int p : s) fin = fin || is_last[p];
            int id = intern(s, fin);
            dtrans[cur][k] = id;
        }
    }

    // Moore refinement on the completed DFA (missing transitions -> sink).
    const int D = (int)sets.size();
    const int SINK = D;
    std::vector<int> cls(D + 1);
    for (int q = 0; q < D; q++) cls[q] = dfinal[q] ? 1 : 0;
    cls[SINK] = 0;
    int ncls = 0;
    for (;;) {
        std::map<std::vector<int>, int> sig;
        std::vector<int> ncl(D + 1);
        for (int q = 0; q <= D; q++) {
            std::vector<int> key;
            key.reserve(A + 1);
            key.push_back(cls[q]);
            for (int k = 0; k < A; k++) {
                int t = (q == SINK) ? SINK : dtrans[q][k];
                key.push_back(cls[t < 0 ? SINK : t]);
            }
            auto it = sig.find(key);
            if (it == sig.end()) it = sig.emplace(key, (int)sig.size()).first;
            ncl[q] = it->second;
        }
        int nn = (int)sig.size();
        cls.swap(ncl);
        if (nn == ncls) break;
        ncls = nn;
    }
    // Class of the sink = dead class; also drop classes that cannot reach a
    // final class (they are equivalent to the sink after refinement).
    const int dead = cls[SINK];
    std::vector<std::vector<int>> ctrans(ncls, std::vector<int>(A, -1));
    std::vector<char> cfinal(ncls, 0);
    for (int q = 0; q < D; q++) {
        int c = cls[q];
        cfinal[c] = dfinal[q];
        for (int k = 0; k < A; k++) {
            int t = dtrans[q][k];
            int tc = t < 0 ? dead : cls[t];
            ctrans[c][k] = tc;
        }
    }
    // Renumber live classes in BFS order from the start class.
    const int start_c = cls[0];
    std::vector<int> newid(ncls, -1);
    std::deque<int> bfs;
    int S = 0;
    if (start_c != dead || true) {
        newid[start_c] = S++;
        bfs.push_back(start_c);
    }
    while (!bfs.empty()) {
        int c = bfs.front();
        bfs.pop_front();
        for (int k = 0; k < A; k++) {
            int t = ctrans[c][k];
            if (t == dead || t < 0 || newid[t] >= 0) continue;
            newid[t] = S++;
            bfs.push_back(t);
        }
    }
    if (S > kMaxStates)
        return fail(RPQ_ERR_INVALID, "minimised automaton has %d states (limit %d)", S, kMaxStates);

    Automaton a;
    a.S = S;
    a.L = n_labels;
    a.start_mask = 1ull << 0;
    for (int c = 0; c < ncls; c++) {
        if (newid[c] < 0) continue;
        if (cfinal[c] && c != dead) a.final_mask |= 1ull << newid[c];
        if (c == dead) continue;
        for (int k = 0; k < A; k++) {
            int t = ctrans[c][k];
            if (t == dead || t < 0 || newid[t] < 0) continue;
            a.from.push_back(newid[c]);
            a.to.push_back(newid[t]);
            a.sym.push_back(alphabet[k]);
        }
    }
    *out = std::move(a);
    return RPQ_OK;
}

bool automaton_accepts(const Automaton &a, const int32_t *word, int32_t len) {
    uint64_t cur = a.start_mask;
    for (int32_t i = 0; i < len && cur; i++) {
        uint64_t nxt = 0;
        for (size_t t = 0; t < a.from.size(); t++)
            if (((cur >> a.from[t]) & 1) && a.sym[t] == word[i]) nxt |= 1ull << a.to[t];
        cur = nxt;
    }
    return (cur & a.final_mask) != 0;
}

Automaton automaton_reverse(const Automaton &a) {
    Automaton r;
    r.S = a.S;
    r.L = a.L;
    r.start_mask = a.final_mask;
    r.final_mask = a.start_mask;
    for (size_t t = 0; t < a.from.size(); t++) {
        r.from.push_back(a.to[t]);
        r.to.push_back(a.from[t]);
        int s = a.sym[t];
        r.sym.push_back(s < a.L ? s + a.L : s - a.L);
    }
    return r;
}

}  // namespace rpq
