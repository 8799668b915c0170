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
 * gates that reach an output.  gatecount.cpp counts the live gates;
 * circuitgen.cpp prints them as device code.
 *
 * Each translation unit that includes this header gets its own recorder.
 */
#pragma once
#include <stdint.h>

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
