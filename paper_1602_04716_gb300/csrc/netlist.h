/*
 * netlist.h -- records a bitslice circuit of circuit.cuh as a netlist of
 * 3-input gates (host code only).
 *
 * The circuits of circuit.cuh are templates over the word type.  Instantiated
 * with GW, a word that records each gate into a DAG instead of computing it,
 * they yield the circuit as a netlist in which every gate is a function of at
 * most three words given by its truth table (one LOP3 on sm_103a).  The
 * recorder absorbs inversions into the truth table, folds constants and
 * repeated inputs, shares identical gates, and the live set keeps only the
 * gates that reach an output.  lut3_map then re-covers the live netlist by
 * 3-input functions.  gatecount.cpp counts the mapped gates; circuitgen.cpp
 * prints them as device code.
 *
 * Each translation unit that includes this header gets its own recorder.
 */
#pragma once
#include <stdint.h>

#include <algorithm>
#include <unordered_map>
#include <vector>

#include "circuit.cuh"

namespace bsfp {
namespace gc {
/* internal linkage: each per-E translation unit keeps its own recorder */
namespace {

struct Graph {
    int ninputs = 0;
    std::vector<int32_t> in[3];   /* input value refs (id << 1 | inv); -1 = unused */
    std::vector<uint8_t> lut;
    std::unordered_map<uint64_t, int32_t> cse;
};

static thread_local Graph* g_graph = nullptr;

/* A recorded word: id 0 is the constant 0 (ref 1 = all ones), ids
 * 1..ninputs are circuit inputs, larger ids are gates. */
struct GW {
    int32_t ref;
    GW() : ref(0) {}
    explicit GW(int32_t r, int) : ref(r) {}
    GW(uint32_t v) : ref(v ? 1 : 0) {}  /* constants 0 and ~0 only */
};

static inline int bit(unsigned L, int i) { return (L >> i) & 1; }

/* Record f(x, y, z) given by truth table L (bit 4a+2b+c). */
static GW lop(unsigned L, GW x, GW y, GW z) {
    int32_t r[3] = {x.ref, y.ref, z.ref};
    const int sh[3] = {2, 1, 0};
    /* absorb inversions */
    for (int k = 0; k < 3; ++k)
        if (r[k] & 1) {
            unsigned N = 0;
            for (int i = 0; i < 8; ++i) N |= (unsigned)bit(L, i ^ (1 << sh[k])) << i;
            L = N;
            r[k] &= ~1;
        }
    /* constant zero inputs: restrict to that input = 0 */
    bool live[3];
    for (int k = 0; k < 3; ++k) {
        live[k] = true;
        if (r[k] == 0) {
            unsigned N = 0;
            for (int i = 0; i < 8; ++i) N |= (unsigned)bit(L, i & ~(1 << sh[k])) << i;
            L = N;
            live[k] = false;
        }
    }
    /* repeated inputs: input j := input k */
    for (int k = 0; k < 3; ++k)
        for (int j = k + 1; j < 3; ++j)
            if (live[k] && live[j] && r[k] == r[j]) {
                unsigned N = 0;
                for (int i = 0; i < 8; ++i) {
                    int a = (i >> sh[k]) & 1;
                    int idx = (i & ~(1 << sh[j])) | (a << sh[j]);
                    N |= (unsigned)bit(L, idx) << i;
                }
                L = N;
                live[j] = false;
            }
    /* drop inputs the function does not depend on */
    for (int k = 0; k < 3; ++k)
        if (live[k]) {
            bool dep = false;
            for (int i = 0; i < 8; ++i) dep |= bit(L, i) != bit(L, i ^ (1 << sh[k]));
            if (!dep) live[k] = false;
        }
    int nlive = 0, only = -1;
    for (int k = 0; k < 3; ++k)
        if (live[k]) {
            ++nlive;
            only = k;
        }
    if (nlive == 0) return GW(bit(L, 0) ? 1 : 0, 0);
    if (nlive == 1) {
        /* identity or complement of one input */
        int inv = bit(L, 0);   /* value when that input (and the rest) is 0 */
        return GW(r[only] | inv, 0);
    }
    /* canonical form: live inputs in id order into slots a, b, (c); dead
     * slots fixed at 0; output inverted so that f(0,0,0) = 0 */
    int32_t ids[3] = {-1, -1, -1};
    int slot[3] = {-1, -1, -1};
    {
        int order[3], n = 0;
        for (int k = 0; k < 3; ++k)
            if (live[k]) order[n++] = k;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q)
                if (r[order[q]] < r[order[p]]) {
                    int t = order[p];
                    order[p] = order[q];
                    order[q] = t;
                }
        for (int p = 0; p < n; ++p) {
            ids[p] = r[order[p]];
            slot[order[p]] = p;
        }
    }
    unsigned N = 0;
    for (int i = 0; i < 8; ++i) {
        int a = (i >> 2) & 1, b = (i >> 1) & 1, c = i & 1;
        int v[3] = {a, b, c};
        int src = 0;
        for (int k = 0; k < 3; ++k)
            if (live[k]) src |= v[slot[k]] << sh[k];
        N |= (unsigned)bit(L, src) << i;
    }
    /* slots beyond the live count are don't-cares: keep only the c=0 / b=0 half */
    if (nlive == 2) {
        unsigned M2 = 0;
        for (int i = 0; i < 8; ++i) M2 |= (unsigned)bit(N, i & ~1) << i;
        N = M2;
    }
    int oinv = N & 1;
    if (oinv) N = ~N & 0xFFu;
    Graph& g = *g_graph;
    uint64_t key = (uint64_t)N << 56 ^ (uint64_t)(uint32_t)ids[0] << 36 ^ (uint64_t)(uint32_t)(ids[1] + 1) << 18 ^
                   (uint64_t)(uint32_t)(ids[2] + 1);
    auto it = g.cse.find(key);
    int32_t id;
    if (it != g.cse.end()) {
        id = it->second;
    } else {
        id = (int32_t)(g.ninputs + 1 + g.lut.size());
        for (int k = 0; k < 3; ++k) g.in[k].push_back(ids[k]);
        g.lut.push_back((uint8_t)N);
        g.cse.emplace(key, id);
    }
    return GW((id << 1) | oinv, 0);
}

/* The gate primitives for recorded words (chosen over the templates of
 * circuit.cuh by overload resolution).  Truth tables use a=0xF0, b=0xCC,
 * c=0xAA. */
inline GW operator~(GW a) { return GW(a.ref ^ 1, 0); }
inline GW NOT(GW a) { return ~a; }
inline GW AND(GW a, GW b) { return lop(0xC0, a, b, a); }
inline GW OR(GW a, GW b) { return lop(0xFC, a, b, a); }
inline GW XOR(GW a, GW b) { return lop(0x3C, a, b, a); }
inline GW ANDN(GW a, GW b) { return lop(0x30, a, b, a); }
inline GW XOR3(GW a, GW b, GW c) { return lop(0x96, a, b, c); }
inline GW MAJ(GW a, GW b, GW c) { return lop(0xE8, a, b, c); }
inline GW MUX(GW s, GW t, GW f) { return lop(0xCA, s, t, f); }
inline GW OR3(GW a, GW b, GW c) { return lop(0xFE, a, b, c); }
inline GW AND3(GW a, GW b, GW c) { return lop(0x80, a, b, c); }
inline GW ANDOR(GW a, GW b, GW c) { return lop(0xEA, a, b, c); }
inline GW ANDNN(GW a, GW b, GW c) { return lop(0x10, a, b, c); }
template <unsigned L> inline GW F3(GW a, GW b, GW c) { return lop(L, a, b, c); }

/* Live gates reachable from the outputs (mark[i] for gate id first+i). */
static std::vector<char> live_set(const Graph& g, const GW* out, int nout) {
    const int first = g.ninputs + 1;
    std::vector<char> mark(g.lut.size(), 0);
    std::vector<int32_t> stack;
    for (int i = 0; i < nout; ++i) stack.push_back(out[i].ref >> 1);
    while (!stack.empty()) {
        int32_t id = stack.back();
        stack.pop_back();
        if (id < first) continue;
        int idx = id - first;
        if (mark[idx]) continue;
        mark[idx] = 1;
        for (int k = 0; k < 3; ++k)
            if (g.in[k][idx] >= 0) stack.push_back(g.in[k][idx] >> 1);
    }
    return mark;
}

static long count_live(const Graph& g, const GW* out, int nout) {
    long n = 0;
    for (char m : live_set(g, out, nout)) n += m;
    return n;
}

/* ------------------------------------------------------ LUT3 re-mapping --- *
 * The recorder keeps the gates in the grouping the templates wrote them in.
 * A gate whose only use is a neighbouring gate can often be merged into it:
 * the pair is one 3-input function whenever the two together read at most
 * three distinct values (a partial product AND feeding a half adder's XOR,
 * say).  lut3_map covers the live netlist with 3-input functions by cut
 * enumeration: every gate's 3-feasible cuts (sets of at most three values
 * that determine it) are merged from its inputs' cuts, a cover is chosen by
 * area flow (each value's cost shared among its uses), then refined by exact
 * local area (the gates a choice adds to or removes from the cover), and
 * each chosen cut becomes one gate whose truth table is that of the cone
 * over the cut.  Inputs, outputs and the function computed are unchanged;
 * only gates disappear. */
namespace lut3 {

constexpr int MAX_CUTS = 48;

struct Cut {
    int n = 0;
    int32_t leaf[3];   /* value ids, ascending */
};

static inline bool cut_subset(const Cut& a, const Cut& b) {   /* a within b */
    for (int i = 0; i < a.n; ++i) {
        bool f = false;
        for (int j = 0; j < b.n; ++j) f |= a.leaf[i] == b.leaf[j];
        if (!f) return false;
    }
    return true;
}

static inline bool cut_merge(const Cut& a, const Cut& b, Cut* o) {
    int i = 0, j = 0, n = 0;
    while (i < a.n || j < b.n) {
        int32_t v;
        if (j >= b.n || (i < a.n && a.leaf[i] < b.leaf[j])) v = a.leaf[i++];
        else if (i >= a.n || b.leaf[j] < a.leaf[i]) v = b.leaf[j++];
        else { v = a.leaf[i]; ++i; ++j; }
        if (n == 3) return false;
        o->leaf[n++] = v;
    }
    o->n = n;
    return true;
}

struct Mapper {
    const Graph& g;
    int first;                                  /* id of the first gate */
    std::vector<char> live;
    std::vector<std::vector<Cut>> cuts;         /* per gate index */
    std::vector<int> best;                      /* chosen cut per gate index */
    std::vector<int> refs;                      /* per value id: uses in the current cover */
    std::vector<double> flow;                   /* area flow per value id */

    explicit Mapper(const Graph& gr) : g(gr), first(gr.ninputs + 1) {}

    bool is_gate(int32_t id) const { return id >= first; }
    int fanins(int idx, int32_t* f) const {
        int n = 0;
        for (int k = 0; k < 3; ++k) {
            const int32_t r = g.in[k][idx];
            if (r < 0) continue;
            const int32_t id = r >> 1;
            if (id == 0) continue;   /* constants are folded into the truth tables */
            bool dup = false;
            for (int q = 0; q < n; ++q) dup |= f[q] == id;
            if (!dup) f[n++] = id;
        }
        return n;
    }

    void enumerate() {
        const size_t ng = g.lut.size();
        cuts.assign(ng, {});
        for (size_t idx = 0; idx < ng; ++idx) {
            if (!live[idx]) continue;
            int32_t f[3];
            const int nf = fanins((int)idx, f);
            /* candidate cut sets of each fanin: its own trivial cut, plus its cuts if a gate */
            std::vector<Cut> lists[3];
            for (int q = 0; q < nf; ++q) {
                Cut t;
                t.n = 1;
                t.leaf[0] = f[q];
                lists[q].push_back(t);
                if (is_gate(f[q]))
                    for (const Cut& c : cuts[f[q] - first]) lists[q].push_back(c);
            }
            std::vector<Cut> out;
            Cut acc;
            acc.n = 0;
            combine(lists, nf, 0, acc, out);
            /* drop dominated cuts, keep the smallest first */
            std::sort(out.begin(), out.end(), [](const Cut& a, const Cut& b) {
                if (a.n != b.n) return a.n < b.n;
                for (int i = 0; i < a.n; ++i)
                    if (a.leaf[i] != b.leaf[i]) return a.leaf[i] < b.leaf[i];
                return false;
            });
            std::vector<Cut> keep;
            for (const Cut& c : out) {
                bool dom = false;
                for (const Cut& k : keep) dom |= cut_subset(k, c);
                if (!dom) keep.push_back(c);
                if ((int)keep.size() >= MAX_CUTS) break;
            }
            cuts[idx] = keep;
        }
    }

    void combine(const std::vector<Cut>* lists, int nf, int q, const Cut& acc, std::vector<Cut>& out) {
        if (q == nf) {
            out.push_back(acc);
            return;
        }
        for (const Cut& c : lists[q]) {
            Cut m;
            if (cut_merge(acc, c, &m)) combine(lists, nf, q + 1, m, out);
        }
    }

    /* area-flow selection in topological order */
    void select_flow(const std::vector<int>& fanout) {
        const size_t ng = g.lut.size();
        flow.assign(first + ng, 0.0);
        best.assign(ng, -1);
        for (size_t idx = 0; idx < ng; ++idx) {
            if (!live[idx]) continue;
            double bv = 1e300;
            int bi = -1;
            for (int ci = 0; ci < (int)cuts[idx].size(); ++ci) {
                const Cut& c = cuts[idx][ci];
                double v = 1.0;
                for (int i = 0; i < c.n; ++i) {
                    const int32_t l = c.leaf[i];
                    v += flow[l] / (fanout[l] > 0 ? fanout[l] : 1);
                }
                if (v < bv - 1e-9) {
                    bv = v;
                    bi = ci;
                }
            }
            best[idx] = bi;
            flow[first + idx] = bv;
        }
    }

    int deref(int idx) {   /* gates freed by dropping gate idx's cut */
        int a = 1;
        const Cut& c = cuts[idx][best[idx]];
        for (int i = 0; i < c.n; ++i) {
            const int32_t l = c.leaf[i];
            if (is_gate(l) && --refs[l] == 0) a += deref(l - first);
        }
        return a;
    }
    int ref(int idx) {     /* gates added by taking gate idx's cut */
        int a = 1;
        const Cut& c = cuts[idx][best[idx]];
        for (int i = 0; i < c.n; ++i) {
            const int32_t l = c.leaf[i];
            if (is_gate(l) && refs[l]++ == 0) a += ref(l - first);
        }
        return a;
    }

    /* reference counts of the cover reachable from the outputs */
    void count_cover(const GW* out, int nout) {
        refs.assign(first + g.lut.size(), 0);
        for (int i = 0; i < nout; ++i) {
            const int32_t id = out[i].ref >> 1;
            if (is_gate(id) && refs[id]++ == 0) ref(id - first);
        }
    }

    void refine(const GW* out, int nout, int rounds) {
        for (int r = 0; r < rounds; ++r) {
            count_cover(out, nout);
            for (size_t idx = 0; idx < g.lut.size(); ++idx) {
                if (!live[idx] || refs[first + idx] == 0) continue;
                const int a0 = deref((int)idx);
                int bi = best[idx], ba = a0;
                for (int ci = 0; ci < (int)cuts[idx].size(); ++ci) {
                    best[idx] = ci;
                    const int a = ref((int)idx);
                    deref((int)idx);
                    if (a < ba) {
                        ba = a;
                        bi = ci;
                    }
                }
                best[idx] = bi;
                ref((int)idx);
            }
        }
        count_cover(out, nout);
    }

    /* truth table (8 bits, leaves on a = 0xF0, b = 0xCC, c = 0xAA) of value id over a cut */
    unsigned cone(int32_t id, const Cut& c, std::unordered_map<int32_t, unsigned>& memo) const {
        static const unsigned pat[3] = {0xF0u, 0xCCu, 0xAAu};
        for (int i = 0; i < c.n; ++i)
            if (c.leaf[i] == id) return pat[i];
        if (id == 0) return 0u;
        auto it = memo.find(id);
        if (it != memo.end()) return it->second;
        const int idx = id - first;
        unsigned v[3] = {0u, 0u, 0u};
        for (int k = 0; k < 3; ++k) {
            const int32_t r = g.in[k][idx];
            if (r >= 0) v[k] = cone(r >> 1, c, memo) ^ ((r & 1) ? 0xFFu : 0u);
        }
        unsigned t = 0u;
        const unsigned L = g.lut[idx];
        for (int i = 0; i < 8; ++i)
            if ((L >> i) & 1u)
                t |= ((i & 4) ? v[0] : ~v[0]) & ((i & 2) ? v[1] : ~v[1]) & ((i & 1) ? v[2] : ~v[2]);
        t &= 0xFFu;
        memo.emplace(id, t);
        return t;
    }
};

}  // namespace lut3

/* Re-map g's live netlist (outputs out[0..nout)) into ng; mapped[i] are the
 * outputs in ng.  ng has the same inputs. */
static void lut3_map(const Graph& g, const GW* out, int nout, Graph& ng, GW* mapped) {
    lut3::Mapper m(g);
    m.live = live_set(g, out, nout);
    const int first = g.ninputs + 1;
    /* fanout of every value among live gates and outputs */
    std::vector<int> fanout(first + g.lut.size(), 0);
    for (size_t idx = 0; idx < g.lut.size(); ++idx) {
        if (!m.live[idx]) continue;
        int32_t f[3];
        const int nf = m.fanins((int)idx, f);
        for (int q = 0; q < nf; ++q) ++fanout[f[q]];
    }
    for (int i = 0; i < nout; ++i) ++fanout[out[i].ref >> 1];
    m.enumerate();
    m.select_flow(fanout);
    m.refine(out, nout, 4);
    /* rebuild: every gate in the cover becomes one recorded gate */
    ng = Graph();
    ng.ninputs = g.ninputs;
    Graph* saved = g_graph;
    g_graph = &ng;
    std::vector<GW> newref(first + g.lut.size());
    for (int32_t id = 0; id < first; ++id) newref[id] = GW(id << 1, 0);
    for (size_t idx = 0; idx < g.lut.size(); ++idx) {
        const int32_t id = first + (int32_t)idx;
        if (!m.live[idx] || m.refs[id] == 0) continue;
        const lut3::Cut& c = m.cuts[idx][m.best[idx]];
        std::unordered_map<int32_t, unsigned> memo;
        const unsigned L = m.cone(id, c, memo);
        GW x[3] = {GW(0u), GW(0u), GW(0u)};
        for (int i = 0; i < c.n; ++i) x[i] = newref[c.leaf[i]];
        newref[id] = lop(L, x[0], x[1], x[2]);
    }
    for (int i = 0; i < nout; ++i) {
        const GW v = newref[out[i].ref >> 1];
        mapped[i] = GW(v.ref ^ (out[i].ref & 1), 0);
    }
    g_graph = saved;
}

/* Record fp_op<E, M, R, OP> (R: rounding mode, bit 0 toward zero, bit 1
 * flush to zero) over inputs a = ids 1..B, b = B+1..2B, c = 2B+1..3B into
 * g; the B output refs go to r. */
template <int E, int M, int R, int OP> static void record(Graph& g, GW* r) {
    constexpr int B = 1 + E + M;
    g.ninputs = 3 * B;
    g_graph = &g;
    GW a[B], b[B], c[B];
    for (int i = 0; i < B; ++i) {
        a[i] = GW((1 + i) << 1, 0);
        b[i] = GW((1 + B + i) << 1, 0);
        c[i] = GW((1 + 2 * B + i) << 1, 0);
    }
    fp_op<E, M, R, OP>(a, b, c, r);
    g_graph = nullptr;
}

/* Record int_op<w, OP> over inputs a = ids 1..w, b = w+1..2w. */
template <int w, int OP> static void record_int(Graph& g, GW* r) {
    g.ninputs = 2 * w;
    g_graph = &g;
    GW a[w], b[w];
    for (int i = 0; i < w; ++i) {
        a[i] = GW((1 + i) << 1, 0);
        b[i] = GW((1 + w + i) << 1, 0);
    }
    int_op<w, OP>(a, b, r);
    g_graph = nullptr;
}

}  // namespace
}  // namespace gc
}  // namespace bsfp
