// Team-cooperative builders of the per-group structures from a vertex's
// adjacency (Section 5.1, adaptive group representation).  Used when a graph
// is created and when an update batch converts a group to another kind or
// outgrows a capacity (Section 5.2, rebuild).
#pragma once

#include "bingo_internal.cuh"

namespace bingo {

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
    uint32_t pos = 0;
    for (uint32_t b = 0; b < d; b += t.size()) {
        const uint32_t j = b + t.rank();
        const bool p = j < d && ((pairs[j].y >> k) & 1u);
        uint32_t tot;
        const uint32_t r = t.scan_pred(p, tot);
        if (p) {
            mem[pos + r] = j;
            inv[j] = pos + r;
            mdst[pos + r] = pairs[j].x;
        }
        pos += tot;
    }
}

// Sparse neighbour list S: slots of edges with any bit of spmask set, S_inv by slot.
template <class Team>
__device__ uint32_t build_slist(const Team& t, const DevGraph& G, uint64_t adj, uint32_t d, uint32_t spmask,
                                uint64_t sref, uint32_t capa) {
    const uint2* pairs = adj_pairs(G, adj);
    uint32_t* S = G.pool.base + sref;
    uint32_t* Sinv = S + capa;
    uint32_t pos = 0;
    for (uint32_t b = 0; b < d; b += t.size()) {
        const uint32_t j = b + t.rank();
        const bool p = j < d && (pairs[j].y & spmask) != 0u;
        uint32_t tot;
        const uint32_t r = t.scan_pred(p, tot);
        if (p) {
            S[pos + r] = j;
            Sinv[j] = pos + r;
        }
        pos += tot;
    }
    return pos;
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
    uint32_t pos = 0;
    for (uint32_t b = 0; b < nsp; b += t.size()) {
        const uint32_t i = b + t.rank();
        const uint2 e = i < nsp ? pairs[S[i]] : make_uint2(0, 0);
        const bool p = i < nsp && ((e.y >> k) & 1u);
        uint32_t tot;
        const uint32_t r = t.scan_pred(p, tot);
        if (p) {
            mem[pos + r] = i;
            inv[i] = pos + r;
            mdst[pos + r] = e.x;
        }
        pos += tot;
    }
}

// Slot of the (unique) edge with bit k set; NONE32 if there is none.
template <class Team>
__device__ uint32_t find_one(const Team& t, const DevGraph& G, uint64_t adj, uint32_t d, uint32_t k) {
    const uint2* pairs = adj_pairs(G, adj);
    uint32_t best = NONE32;
    for (uint32_t b = 0; b < d; b += t.size()) {
        const uint32_t j = b + t.rank();
        const bool p = j < d && ((pairs[j].y >> k) & 1u);
        const uint32_t cand = p ? j : NONE32;
        // team minimum via max of complements
        const uint32_t m = ~t.max(~cand);
        best = best < m ? best : m;
        if (best != NONE32) break;  // team-uniform
    }
    return best;
}

}  // namespace bingo
