// Team-cooperative builders of the per-group structures from a vertex's
// adjacency (Section 5.1, adaptive group representation).  Used when a graph
// is created and when an update batch converts a group to another kind or
// outgrows a capacity (Section 5.2, rebuild).
#pragma once

#include "bingo_internal.cuh"

namespace bingo {

// Order-preserving team compaction over [0, n): each thread takes IT consecutive elements per chunk,
// one team scan per chunk of IT * team size, and emit(j, position) for every j whose test passes,
// positions ascending with j.  Returns the count.  load(j) reads what the test of element j needs;
// the IT loads of a thread are issued before any test (indexes clamped into [0, n), the tail masked
// afterwards), so they are in flight together instead of one dependent round trip per element.
constexpr int COMPACT_IT = 4;
template <class Team, class Load, class Test, class Emit>
__device__ __forceinline__ uint32_t team_compact_lt(const Team& t, uint32_t n, Load load, Test test, Emit emit) {
    uint32_t pos = 0;
    const uint32_t chunk = COMPACT_IT * t.size();
    for (uint32_t base = 0; base < n; base += chunk) {
        const uint32_t j0 = base + t.rank() * COMPACT_IT;
        decltype(load(0u)) x[COMPACT_IT];
#pragma unroll
        for (int q = 0; q < COMPACT_IT; q++) x[q] = load(min(j0 + q, n - 1));
        bool p[COMPACT_IT];
        uint32_t c = 0;
#pragma unroll
        for (int q = 0; q < COMPACT_IT; q++) {
            p[q] = (j0 + q < n) && test(x[q], j0 + q);
            c += p[q] ? 1u : 0u;
        }
        uint32_t tot;
        uint32_t off = t.scan_excl(c, tot);
#pragma unroll
        for (int q = 0; q < COMPACT_IT; q++)
            if (p[q]) emit(j0 + q, pos + off++);
        pos += tot;
    }
    return pos;
}
// The same with a predicate that is cheap to evaluate once its operand is loaded.
template <class Team, class Pred, class Emit>
__device__ __forceinline__ uint32_t team_compact(const Team& t, uint32_t n, Pred pred, Emit emit) {
    return team_compact_lt(
        t, n, [&](uint32_t j) { return pred(j); }, [](bool v, uint32_t) { return v; }, emit);
}

// Group blocks hold [member destinations | member list | inverted index | spare], cap words each:
// a walker reads a uniform member's destination with one access at the block's start.

// Regular group k: member list of slots with bit k set, inverted index by slot.
template <class Team>
__device__ void build_regular(const Team& t, const DevGraph& G, uint64_t adj, uint32_t d, uint32_t k, uint64_t goff,
                              uint32_t capa) {
    const uint2* pairs = adj_pairs(G, adj);
    uint32_t* mdst = G.pool.base + goff;
    uint32_t* mem = mdst + capa;
    uint32_t* inv = mem + capa;
    team_compact(
        t, d, [&](uint32_t j) { return ((pairs[j].y >> k) & 1u) != 0; },
        [&](uint32_t j, uint32_t pos) {
            mem[pos] = j;
            inv[j] = pos;
            mdst[pos] = pairs[j].x;
        });
}

// Sparse neighbour list S: slots of edges with any bit of spmask set, S_inv by slot.
template <class Team>
__device__ uint32_t build_slist(const Team& t, const DevGraph& G, uint64_t adj, uint32_t d, uint32_t spmask,
                                uint64_t sref, uint32_t capa) {
    const uint2* pairs = adj_pairs(G, adj);
    uint32_t* S = G.pool.base + sref;
    uint32_t* Sinv = S + capa;
    return team_compact(
        t, d, [&](uint32_t j) { return (pairs[j].y & spmask) != 0u; },
        [&](uint32_t j, uint32_t pos) {
            S[pos] = j;
            Sinv[j] = pos;
        });
}

// Sparse group k: member list of positions in S, inverted index by S position.
template <class Team>
__device__ void build_sparse(const Team& t, const DevGraph& G, uint64_t adj, uint64_t sref, uint32_t nsp, uint32_t k,
                             uint64_t goff, uint32_t caps) {
    const uint2* pairs = adj_pairs(G, adj);
    const uint32_t* S = G.pool.base + sref;
    uint32_t* mdst = G.pool.base + goff;
    uint32_t* mem = mdst + caps;
    uint32_t* inv = mem + caps;
    team_compact(
        t, nsp, [&](uint32_t i) { return ((pairs[S[i]].y >> k) & 1u) != 0; },
        [&](uint32_t i, uint32_t pos) {
            mem[pos] = i;
            inv[i] = pos;
            mdst[pos] = pairs[S[i]].x;
        });
}

// Slot of the (unique) edge with bit k set; NONE32 if there is none.
template <class Team>
__device__ uint32_t find_one(const Team& t, const DevGraph& G, uint64_t adj, uint32_t d, uint32_t k) {
    const uint2* pairs = adj_pairs(G, adj);
    const uint32_t chunk = COMPACT_IT * t.size();
    for (uint32_t base = 0; base < d; base += chunk) {
        const uint32_t j0 = base + t.rank() * COMPACT_IT;
        uint32_t w[COMPACT_IT];
#pragma unroll
        for (int q = 0; q < COMPACT_IT; q++) w[q] = pairs[min(j0 + q, d - 1)].y;
        uint32_t cand = NONE32;
#pragma unroll
        for (int q = COMPACT_IT - 1; q >= 0; q--)
            if (j0 + q < d && ((w[q] >> k) & 1u)) cand = j0 + q;
        const uint32_t m = ~t.max(~cand);  // team minimum
        if (m != NONE32) return m;         // team-uniform
    }
    return NONE32;
}

}  // namespace bingo
