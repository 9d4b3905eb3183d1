// Random-walk kernels: hierarchical sampling (Eq. group_prob for the group,
// Eq. pvp within it; dense groups by rejection on the neighbour list, Section
// 5.1), DeepWalk / PPR / node2vec policies (Section 2.2; node2vec by rejection
// against f(prev, x) of Eq. node2vec, as in KnightKing), and the node2vec edge
// index.
//
// Randomness: Philox4x32-10 keyed by the seed; walker w at step s draws from
// counters (w lo, w hi, s, 0), (w lo, w hi, s, 1), ... so results depend only
// on (graph state, seed, walker id) and never on the launch shape.
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "bingo_host.h"

using namespace bingo;

#define CK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

namespace {

constexpr int MAX_DENSE_TRIES = 1 << 14;
// Thread bound of the 64+-register walker instances: 768 threads a block leave each thread up to 80
// registers, which the cold-group scan needs without spilling (measured faster than 64 registers
// with spills at 1,024 threads).
constexpr int WALK_MAX_THREADS = 768;
constexpr int MAX_N2V_TRIES = 1 << 14;
constexpr uint32_t WF_PAD = 1u;  // pad path rows with 0xFFFFFFFF

struct WalkParams {
    uint64_t nwalkers;
    uint32_t hot_last;  // hot-line loads with an L2 evict-last policy (hot_policy)
    const uint32_t* starts;
    const uint32_t* lengths;
    const uint8_t* pids;
    uint2 key;
    uint32_t stride;
    uint32_t npol;
    uint32_t flags;
    uint32_t* paths;
    uint32_t* plen;
    unsigned long long* queue;
    uint32_t* status;
    const bingo_policy* pols;   // device [npol] (or [nreq] in request mode)
    // request mode (merged launch of independent requests): walker w belongs to request r with
    // req_off[r] <= w < req_off[r+1]; it uses key req_key[r], policy pols[r] and local id w - req_off[r]
    const uint64_t* req_off;
    const uint64_t* req_key;
    uint32_t nreq;
    // completion notices for downloads that overlap the walk (chunk_done null = off)
    uint32_t* chunk_done;
    uint32_t* host_flags;
    uint32_t chunk_shift, io_seq;
    // stepwise state
    uint32_t* s_cur;
    uint32_t* s_prev;
    // partitioned walks: this launch serves the graph's vertex range [G.base, G.base + G.n); walkers
    // come from `resume` records (global ids) and leave through `outbox` when their next vertex is
    // another partition's; node2vec probes the previous vertex's owner's edge index
    const PartRec* resume;
    PartRec* outbox;
    unsigned long long* nout;
    const PartEH* peh;
    const uint32_t* bounds;  // npart + 1 boundaries of the partitions (global ids)
    uint32_t npart;
};

// Live copies of (prev, x), global ids, in the edge index of prev's partition.
__device__ __forceinline__ uint32_t part_probe(const WalkParams& A, uint32_t prev, uint32_t x) {
    uint32_t lo = 0, hi = A.npart;  // last p with bounds[p] <= prev
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(A.bounds + mid) <= prev) lo = mid; else hi = mid;
    }
    const PartEH e = A.peh[lo];
    return e.mask ? eh_lookup_in(e.key, e.cnt, e.mask, prev - __ldg(A.bounds + lo), x) : 0u;
}

// Policy index of walker `wid`: its request in request mode, else policy_ids[wid] (default 0).
__device__ __forceinline__ uint32_t walker_pid(const WalkParams& A, uint64_t wid) {
    if (A.req_off) {
        uint32_t lo = 0, hi = A.nreq;  // last r with req_off[r] <= wid
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(A.req_off + mid) <= wid) lo = mid; else hi = mid;
        }
        return lo;
    }
    return A.pids ? __ldg(A.pids + wid) : 0u;
}
// Philox key and counter walker-id of walker `wid` (re-derived each step instead of kept live).
__device__ __forceinline__ void walker_stream(const WalkParams& A, uint64_t wid, uint32_t pid, uint2& key,
                                              uint64_t& lid) {
    if (A.req_off) {
        const uint64_t k = __ldg(A.req_key + pid);
        key = make_uint2((uint32_t)k, (uint32_t)(k >> 32));
        lid = wid - __ldg(A.req_off + pid);
    } else {
        key = A.key;
        lid = wid;
    }
}

// Hot lines are re-read at every visit of their vertex, while member reads and path stores mostly
// touch a line once: hot-line loads carry an L2 evict-last policy (hot_policy), unless the graph's
// configuration asks for the normal one.
__device__ __forceinline__ uint64_t hot_policy(uint32_t evict_last) {
    uint64_t pol;
    if (evict_last) asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    else asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint4 ld_hot(const uint4* q, uint64_t pol) {
    uint4 r;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(q), "l"(pol));
    return r;
}

// Hot part of a vertex record, one 64-byte line: the header, the total weight outside the hot pairs,
// the hot pairs a, b and copies of their groups.
struct Sec0 {
    uint32_t adj, deg, mask;
    uint32_t word;   // the caller's id of the vertex, and the cold scan order (WORD_DESC)
    uint64_t wcold;  // total weight of the groups outside the hot pairs
    uint32_t hp;     // a = hp & 15, b = (hp >> 4) & 15
    uint4 p0, p1;    // groups 2a, 2a+1 and 2b, 2b+1
};
__device__ __forceinline__ Sec0 ld_sec0(const DevGraph& G, uint32_t v, uint64_t pol) {
    const uint4* q = reinterpret_cast<const uint4*>(G.vh + v);
    const uint4 a = ld_hot(q, pol);
    const uint4 b = ld_hot(q + 1, pol);
    Sec0 s;
    s.adj = a.x;
    s.deg = a.y;
    s.mask = a.z;
    s.word = a.w;
    s.wcold = (uint64_t)b.x | ((uint64_t)b.y << 32);
    s.hp = b.z;
    s.p0 = ld_hot(q + 2, pol);
    s.p1 = ld_hot(q + 3, pol);
    return s;
}
// Groups 2i and 2i+1 of vertex v from its cold record as {c_2i, ref_2i, c_2i+1, ref_2i+1} (16-byte aligned).
__device__ __forceinline__ uint4 ld_pair(const DevGraph& G, uint32_t v, uint32_t i) {
    return __ldg(reinterpret_cast<const uint4*>(G.vc[v].g) + i);
}
// WM: the weight mode (slot_weight): integer base 2, real biases (every integer group counts 2^8
// times and slot 31, the second half of pair 15, carries the decimal total itself), or base 4.
template <int WM>
__device__ __forceinline__ uint64_t pair_w(uint4 x, uint32_t i) {
    return slot_weight<WM>(x.x, 2 * i) + slot_weight<WM>(x.z, 2 * i + 1);
}
// pairs with at least one nonempty group, as bits 2i of the result
__device__ __forceinline__ uint32_t pair_bits(uint32_t mask) { return (mask | (mask >> 1)) & 0x55555555u; }

// --------------------------------------------------------------------------------- group selection
// All variants pick the first group k* in the vertex's scan order whose running sum of
// W(p_k) = 2^k |G_k| exceeds r, r uniform in [0, sum_j W(p_j)): group k with probability
// W(p_k) / sum W (Eq. group_prob).  They differ only in how a team of T lanes shares the vertex
// record.  Outputs k*, |G_k*| and the group's ref.

template <int WM>
__device__ __forceinline__ bool scan_pair(uint4 x, uint32_t i, uint64_t r, uint64_t& acc, uint32_t& ks, uint32_t& cs,
                                          uint32_t& ref) {
    const uint64_t lo = acc + slot_weight<WM>(x.x, 2 * i);
    if (r < lo) { ks = 2 * i; cs = x.x; ref = x.y; return true; }
    acc = lo + slot_weight<WM>(x.z, 2 * i + 1);
    if (r < acc) { ks = 2 * i + 1; cs = x.z; ref = x.w; return true; }
    return false;
}
// The same with the pair's two groups in descending order (cold groups of a vertex scanned downwards).
template <int WM>
__device__ __forceinline__ bool scan_pair_desc(uint4 x, uint32_t i, uint64_t r, uint64_t& acc, uint32_t& ks,
                                               uint32_t& cs, uint32_t& ref) {
    const uint64_t hi = acc + slot_weight<WM>(x.z, 2 * i + 1);
    if (r < hi) { ks = 2 * i + 1; cs = x.z; ref = x.w; return true; }
    acc = hi + slot_weight<WM>(x.x, 2 * i);
    if (r < acc) { ks = 2 * i; cs = x.x; ref = x.y; return true; }
    return false;
}

// Scan order of the groups of a vertex: the hot pairs a then b (each pair's groups ascending), then
// the other pairs ascending, or descending (each pair's groups descending) when the hot word's
// WORD_DESC bit is set (hot_summary).  Any fixed order of the inverse CDF draws group k with
// probability W(p_k) / sum W; every team width uses this one, so all give the same k* for the same r.

// T = 1: one lane per walker.  The hot pairs and the total weight outside them came with the header,
// so r is drawn from one 64-byte line.  The cold pairs are read only when r falls beyond the hot
// pairs, in the vertex's scan order (hot_summary): upwards in the aligned batches of pairs [0, 4),
// [4, 8), [8, 12), [12, 16), or downwards in windows of four pairs from the highest nonempty cold
// pair; the loads of a batch are issued together and batches without a nonempty cold pair are skipped.
template <int WM>
__device__ __forceinline__ void select_group_1(const DevGraph& G, uint32_t v, const Sec0& h, StepRng& R,
                                               uint32_t& ks, uint32_t& cs, uint32_t& ref, uint32_t* status) {
    const uint32_t a = h.hp & 15u, b = (h.hp >> 4) & 15u;
    const uint64_t whot = pair_w<WM>(h.p0, a) + pair_w<WM>(h.p1, b);
    const uint64_t r = below64(R, whot + h.wcold, status);
    uint64_t acc = 0;
    if (scan_pair<WM>(h.p0, a, r, acc, ks, cs, ref)) return;
    if (scan_pair<WM>(h.p1, b, r, acc, ks, cs, ref)) return;
    // one loop for both directions: batch starts i0 = 0, 4, 8, 12 upwards, or top, top - 4, ...
    // downwards; a downward pair is scanned odd group first (its halves swapped)
    const bool desc = (h.word & WORD_DESC) != 0;
    const uint32_t cm = pair_bits(h.mask) & ~((1u << (2 * a)) | (1u << (2 * b)));  // nonempty cold pairs, bits 2i
    const int dir = desc ? -1 : 1;
#pragma unroll 1
    for (int i0 = desc ? (int)((31 - __clz(cm)) >> 1) : 0; desc ? i0 >= 0 : i0 < 16; i0 += 4 * dir) {
        const int low = desc ? i0 - 3 : i0;  // lowest pair of the batch (may be below 0 downwards)
        const uint32_t wbits = low >= 0 ? (cm >> (2 * low)) & 0xFFu : (cm << (-2 * low)) & 0xFFu;
        if (!wbits) continue;
        uint4 x[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int i = i0 + dir * j;
            x[j] = (i >= 0 && i < 16 && ((cm >> (2 * i)) & 1u)) ? ld_pair(G, v, (uint32_t)i) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t i = (uint32_t)(i0 + dir * j);
            const uint4 y = desc ? make_uint4(x[j].z, x[j].w, x[j].x, x[j].y) : x[j];
            const uint32_t k0 = desc ? 2 * i + 1 : 2 * i, k1 = desc ? 2 * i : 2 * i + 1;
            const uint64_t lo = acc + slot_weight<WM>(y.x, k0);
            if (r < lo) { ks = k0; cs = y.x; ref = y.y; return; }
            acc = lo + slot_weight<WM>(y.z, k1);
            if (r < acc) { ks = k1; cs = y.z; ref = y.w; return; }
        }
    }
    ks = 31;
    cs = 0;
    ref = 0;
    atomicOr(status, ST_STATE);  // r beyond every group: the cached total disagrees with the counts
}

// Pair at scan position p (0..15) of a vertex: the hot pairs a, b, then the q = p - 2-th of the other
// pairs, upwards or downwards.
__device__ __forceinline__ uint32_t pair_at(uint32_t p, uint32_t hp, bool desc) {
    const uint32_t a = hp & 15u, b = (hp >> 4) & 15u;
    if (p == 0) return a;
    if (p == 1) return b;
    uint32_t lo = min(a, b), hi = max(a, b);
    if (desc) {
        const uint32_t t = 15 - lo;
        lo = 15 - hi;
        hi = t;
    }
    uint32_t c = p - 2;  // rank among the 14 cold pairs in scan order; skip the two hot ones
    if (c >= lo) c++;
    if (c >= hi) c++;
    return desc ? 15 - c : c;
}

// T = 4: lane t of the team owns scan positions [4t, 4t+4) (pair_at); a two-level shuffle prefix
// over the team and a ballot find the lane holding k*, which searches its pairs again.
template <int WM>
__device__ __forceinline__ void select_group_4(const DevGraph& G, uint32_t v, const Sec0& h, StepRng& R,
                                               uint32_t& ks, uint32_t& cs, uint32_t& ref, uint32_t* status,
                                               uint32_t tl, uint32_t team_mask, uint32_t team_base) {
    const uint32_t pb = pair_bits(h.mask);
    const bool desc = (h.word & WORD_DESC) != 0;
    uint64_t s = 0;
#pragma unroll
    for (uint32_t j = 0; j < 4; j++) {
        const uint32_t p = 4 * tl + j, i = pair_at(p, h.hp, desc);
        if ((pb >> (2 * i)) & 1u) s += pair_w<WM>(p == 0 ? h.p0 : p == 1 ? h.p1 : ld_pair(G, v, i), i);
    }
    uint64_t incl = s;
#pragma unroll
    for (int d = 1; d < 4; d <<= 1) {
        const uint64_t y = __shfl_up_sync(team_mask, incl, d, 4);
        if (tl >= (uint32_t)d) incl += y;
    }
    const uint64_t tot = __shfl_sync(team_mask, incl, team_base + 3);
    const uint64_t r = below64(R, tot, status);
    const uint64_t excl = incl - s;
    const uint32_t b = __ballot_sync(team_mask, r < incl && r >= excl) & team_mask;
    if (b == 0) {  // r beyond every group: the counts disagree with the mask (never with a consistent state)
        ks = 31;
        cs = 0;
        ref = 0;
        if (tl == 0) atomicOr(status, ST_STATE);
        return;
    }
    const uint32_t owner = __ffs(b) - 1;
    uint32_t k_l = 0, c_l = 0, r_l = 0;
    if (lane_id() == owner) {
        uint64_t acc = excl;
        for (uint32_t j = 0; j < 4; j++) {
            const uint32_t p = 4 * tl + j, i = pair_at(p, h.hp, desc);
            if (!((pb >> (2 * i)) & 1u)) continue;
            const uint4 x = p == 0 ? h.p0 : p == 1 ? h.p1 : ld_pair(G, v, i);
            if ((p >= 2 && desc) ? scan_pair_desc<WM>(x, i, r, acc, k_l, c_l, r_l)
                                 : scan_pair<WM>(x, i, r, acc, k_l, c_l, r_l))
                break;
        }
    }
    ks = __shfl_sync(team_mask, k_l, owner);
    cs = __shfl_sync(team_mask, c_l, owner);
    ref = __shfl_sync(team_mask, r_l, owner);
}

// T = 32: lane l owns the group at scan position l (pair_at(l / 2), its lower group first unless
// the pair is a cold pair scanned downwards); a warp-wide shuffle prefix of W_k = 2^k |G_k| and a ballot of (prefix > r) give k*
// at the first set bit.
template <int WM>
__device__ __forceinline__ void select_group_32(const DevGraph& G, uint32_t v, const Sec0& h, StepRng& R,
                                                uint32_t& ks, uint32_t& cs, uint32_t& ref, uint32_t* status,
                                                uint32_t lane) {
    const bool desc = (h.word & WORD_DESC) != 0;
    // scan position lane: positions 0-3 the hot pairs' groups, then two positions per cold pair
    const uint32_t i = pair_at(lane >> 1, h.hp, desc);
    const uint32_t k = 2 * i + ((lane >= 4 && desc) ? 1u - (lane & 1u) : (lane & 1u));
    uint2 gk = make_uint2(0, 0);
    if (lane < 4) {
        const uint4 x = lane < 2 ? h.p0 : h.p1;
        gk = (lane & 1u) ? make_uint2(x.z, x.w) : make_uint2(x.x, x.y);
    } else if ((h.mask >> k) & 1u) {
        gk = __ldg(&G.vc[v].g[k]);
    }
    uint64_t incl = slot_weight<WM>(gk.x, k);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(FULL, incl, d);
        if (lane >= (uint32_t)d) incl += y;
    }
    const uint64_t tot = __shfl_sync(FULL, incl, 31);
    const uint64_t r = below64(R, tot, status);
    const uint32_t b = __ballot_sync(FULL, r < incl);
    if (b == 0) {  // only when the total is zero, which a vertex with out-edges never has
        ks = 31;
        cs = 0;
        ref = 0;
        if (lane == 0) atomicOr(status, ST_STATE);
        return;
    }
    const uint32_t owner = __ffs(b) - 1;
    ks = __shfl_sync(FULL, k, owner);
    cs = __shfl_sync(FULL, gk.x, owner);
    ref = __shfl_sync(FULL, gk.y, owner);
}

// --------------------------------------------------------------------------------- intra-group pick
// Uniform member of G_k* (Eq. pvp).  One-element groups store their member's destination; regular
// and sparse groups keep their members' destinations at the head of the group block, so a uniform
// position costs one access.  Dense groups use rejection over the whole neighbour list, accepting a
// slot whose bias has bit k* (Section 5.1).  Returns the destination vertex.
// Decimal group of a real-bias vertex (Section 4.3, step (iii)): neighbour j with probability
// q_j / Q_D.  Rejection over the d slots, a uniform slot accepted iff a uniform byte < q_j; after
// DEC_TRIES candidates, inverse transform over the decimal parts.  Either way the output law is
// q_j / Q_D, so the fallback keeps it exact.
// Inverse transform over the decimal parts: the first slot whose running sum of q exceeds r < Q_D.
static __device__ __noinline__ uint32_t decimal_its(const uint8_t* qb, const uint2* pairs, uint32_t d, uint32_t r) {
    uint32_t acc = 0;
    for (uint32_t j = 0; j < d; j++) {
        acc += __ldg(qb + j);
        if (r < acc) return __ldg(&pairs[j].x);
    }
    return NONE32;
}
// Decimal picks are rare (the decimal group carries a small share of the weight), so candidates go
// one at a time: few registers on this path.
constexpr int DEC_TRIES = 16;
__device__ __forceinline__ uint32_t pick_decimal(const DevGraph& G, const Sec0& h, uint32_t qd, uint32_t ref,
                                                 StepRng& R, uint32_t* status) {
    if (words_of(ref) >= G.pool.words || qd == 0) { atomicOr(status, ST_STATE); return NONE32; }
    const uint8_t* qb = dec_bytes(G, ref);
    const uint2* pairs = adj_pairs(G, words_of(h.adj));
    for (int t = 0; t < DEC_TRIES; t++) {
        const uint32_t j = below32(R, h.deg, status);
        if ((R.next() & 255u) < __ldg(qb + j)) return __ldg(&pairs[j].x);
    }
    const uint32_t x = decimal_its(qb, pairs, h.deg, below32(R, qd, status));
    if (x == NONE32) atomicOr(status, ST_STATE);
    return x;
}

template <int WM>
__device__ __forceinline__ uint32_t pick_member(const DevGraph& G, const Sec0& h, uint32_t ks, uint32_t cs,
                                                uint32_t ref, StepRng& R, uint32_t* status) {
    if constexpr (WM == WM_REAL)
        if (ks == DEC_SLOT) return pick_decimal(G, h, cs, ref, R, status);
    if (cs == 0) return NONE32;  // no group was selected (the selection flagged ST_STATE)
    const uint32_t kd = kind_of(cs, h.deg, G.alpha, G.beta);
    if (kd == K_DENSE) {
        const uint2* pairs = adj_pairs(G, words_of(h.adj));
        // Rejection in rounds of B candidates drawn in order, whose loads are in flight together; the
        // first accepted candidate in draw order is the one sequential rejection would return.
        // B grows as the acceptance rate |G_k|/d falls (it is > 0.4 for a dense group).
        const uint32_t B = (4ull * cs >= 3ull * h.deg) ? 1u : (2ull * cs >= h.deg) ? 2u : 3u;
        for (int t = 0; t < MAX_DENSE_TRIES; t += 3) {
            const uint32_t j0 = below32(R, h.deg, status);
            const uint32_t j1 = B > 1 ? below32(R, h.deg, status) : 0u;
            const uint32_t j2 = B > 2 ? below32(R, h.deg, status) : 0u;
            const uint2 e0 = __ldg(pairs + j0);
            const uint2 e1 = B > 1 ? __ldg(pairs + j1) : make_uint2(0, 0);
            const uint2 e2 = B > 2 ? __ldg(pairs + j2) : make_uint2(0, 0);
            if ((e0.y >> ks) & 1u) return e0.x;
            if ((e1.y >> ks) & 1u) return e1.x;
            if ((e2.y >> ks) & 1u) return e2.x;
        }
        atomicOr(status, ST_TIMEOUT);
        return NONE32;
    }
    if (kd == K_ONE) return ref;
    if (words_of(ref) >= G.pool.words) { atomicOr(status, ST_STATE); return NONE32; }  // never read past the pool
    const uint32_t pos = below32(R, cs, status);
    return __ldg(G.pool.base + words_of(ref) + pos);
}

// One step of a walker at `cur`.  Returns false if the walk ends here (PPR stop, no out-edge, error).
// PART: a partition graph's walker (previous vertex and the sampled vertex are global ids).
template <int T, int WM, bool PART>
__device__ __forceinline__ bool walk_step(const DevGraph& G, const WalkParams& A, uint64_t wid, uint32_t pid,
                                          uint32_t step, uint32_t& cur, uint32_t& prev, uint32_t tl,
                                          uint32_t team_mask, uint32_t team_base, uint32_t lane, uint32_t& hword) {
    const bingo_policy* P = A.pols + pid;
    const uint32_t kind = __ldg(&P->kind);
    StepRng R;
    {
        uint2 key;
        uint64_t lid;
        walker_stream(A, wid, pid, key, lid);
        R.init(key, lid, step);
    }
    hword = NONE32;
    if (kind == BINGO_PPR && R.next() < __ldg(&P->ppr_stop_u32)) return false;
    const Sec0 h = ld_sec0(G, cur, hot_policy(A.hot_last));
    hword = h.word & WORD_ID;
    if (h.deg == 0) return false;
    for (int attempt = 0; attempt < MAX_N2V_TRIES; attempt++) {
        uint32_t ks, cs, ref;
        if constexpr (T == 1) select_group_1<WM>(G, cur, h, R, ks, cs, ref, A.status);
        else if constexpr (T == 4) select_group_4<WM>(G, cur, h, R, ks, cs, ref, A.status, tl, team_mask, team_base);
        else select_group_32<WM>(G, cur, h, R, ks, cs, ref, A.status, lane);
        const uint32_t x = pick_member<WM>(G, h, ks, cs, ref, R, A.status);
        if (x >= G.dst_n) {
            if (x != NONE32) atomicOr(A.status, ST_STATE);
            return false;
        }
        if (kind == BINGO_NODE2VEC && prev != NONE32) {
            const uint64_t u = R.next();
            const unsigned long long* acc_t = reinterpret_cast<const unsigned long long*>(P->n2v_accept);
            bool acc;
            if (x == prev) {
                acc = u < __ldg(acc_t + 0);
            } else {
                const uint64_t a1 = __ldg(acc_t + 1), a2 = __ldg(acc_t + 2);
                const uint64_t lo = a1 < a2 ? a1 : a2, hi = a1 < a2 ? a2 : a1;
                if (u < lo) acc = true;        // accepted at either distance: no probe needed
                else if (u >= hi) acc = false; // rejected at either distance
                else acc = u < ((PART ? part_probe(A, prev, x) : eh_lookup(G, prev, x)) ? a1 : a2);
            }
            if (!acc) continue;
        }
        prev = PART ? cur + G.base : cur;  // partitioned walks keep the previous vertex's global id
        cur = x;                           // partitioned walks: a global id (the caller localises it)
        return true;
    }
    atomicOr(A.status, ST_TIMEOUT);
    return false;
}

// Completion notice of walker `wid`, whose row and length are written: the walker that completes its
// id chunk publishes io_seq in the chunk's host-mapped flag, after which the host may start a copy
// engine on the chunk while the walk goes on.  Each lane fences its own stores at system scope (the
// copy engine is the reader) before the team's count.
__device__ __forceinline__ void notify_done(const WalkParams& A, uint64_t wid, uint32_t tl, uint32_t team_mask) {
    __threadfence_system();
    __syncwarp(team_mask);
    if (tl != 0) return;
    const uint64_t c = wid >> A.chunk_shift, lo = c << A.chunk_shift;
    const uint64_t size = A.nwalkers - lo < (1ull << A.chunk_shift) ? A.nwalkers - lo : (1ull << A.chunk_shift);
    if (atomicAdd(A.chunk_done + c, 1u) + 1 == size) {
        __threadfence_system();
        *(volatile uint32_t*)(A.host_flags + c) = A.io_seq;
    }
}

__device__ __forceinline__ void finish_walker(const WalkParams& A, uint64_t wid, uint32_t steps, uint32_t tl,
                                              uint32_t T, uint32_t team_mask) {
    uint32_t* row = A.paths + wid * (uint64_t)A.stride;
    if (tl == 0) A.plen[wid] = steps + 1;
    if (A.flags & WF_PAD)
        for (uint32_t t = steps + 1 + tl; t < A.stride; t += T) row[t] = NONE32;
    if (A.chunk_done) notify_done(A, wid, tl, team_mask);
}

// OCC selects the register budget: 0 = up to 64 registers (1,024-thread bound), 1 = 40 registers
// (256-thread blocks, six per SM), trading spills to L1 for 50% more resident warps.
// WM: the graph's weight mode; each mode runs its own instance (integer graphs carry no code for the
// decimal group or the base-4 weights).
template <int T, int OCC, int WM, bool PART = false>
__global__ void __launch_bounds__(OCC ? 256 : WALK_MAX_THREADS, OCC ? 6 : 1) k_walk_persistent(DevGraph G, WalkParams A) {
    const uint32_t lane = threadIdx.x & 31, tl = lane % T, team = lane / T;
    const uint32_t team_base = team * T;
    const uint32_t team_mask = (T == 32) ? FULL : (((1u << T) - 1u) << team_base);
    uint64_t wid = 0;
    uint32_t pid = 0, cur = 0, prev = NONE32, step = 0, L = 0;
    bool have = false, drained = false;
    for (;;) {
        if (!drained) {
            const bool need = !have && tl == 0;
            const uint32_t nm = __ballot_sync(FULL, need);
            if (nm) {
                const int leader = __ffs(nm) - 1;
                unsigned long long base = 0;
                if ((int)lane == leader) base = atomicAdd(A.queue, (unsigned long long)__popc(nm));
                base = __shfl_sync(FULL, base, leader);
                uint64_t mine = base + __popc(nm & lanemask_lt());
                mine = __shfl_sync(FULL, mine, team_base);
                if (base + __popc(nm) >= A.nwalkers) drained = true;
                if (PART && !have && mine < A.nwalkers) {  // a walker arriving in this partition
                    const PartRec rc = A.resume[mine];
                    wid = rc.wid;
                    pid = walker_pid(A, wid);
                    if (pid >= A.npol) { pid = 0; atomicOr(A.status, ST_INVALID); }
                    L = A.lengths ? __ldg(A.lengths + wid) : __ldg(&A.pols[pid].max_len);
                    if (L + 1 > A.stride) { L = A.stride - 1; atomicOr(A.status, ST_INVALID); }
                    cur = rc.cur - G.base;
                    prev = rc.prev;
                    step = rc.step;
                    if (cur >= G.n) { L = step; atomicOr(A.status, ST_STATE); }  // routed to a wrong partition
                    have = true;
                    if (step == 0 && tl == 0) A.paths[wid * (uint64_t)A.stride] = rc.cur;
                    if (step >= L) {
                        finish_walker(A, wid, step, tl, T, team_mask);
                        have = false;
                    }
                } else if (!PART && !have && mine < A.nwalkers) {
                    wid = mine;
                    pid = walker_pid(A, wid);
                    if (pid >= A.npol) { pid = 0; atomicOr(A.status, ST_INVALID); }
                    cur = __ldg(A.starts + wid);
                    L = A.lengths ? __ldg(A.lengths + wid) : __ldg(&A.pols[pid].max_len);
                    if (L + 1 > A.stride) { L = A.stride - 1; atomicOr(A.status, ST_INVALID); }
                    if (cur >= G.n) { L = 0; atomicOr(A.status, ST_INVALID); }
                    prev = NONE32;
                    step = 0;
                    have = true;
                    if (tl == 0) A.paths[wid * (uint64_t)A.stride] = cur;
                    cur = to_internal(G, cur);
                    if (L == 0) {
                        finish_walker(A, wid, 0, tl, T, team_mask);
                        have = false;
                    }
                }
            }
        }
        if (!__any_sync(FULL, have)) {
            if (drained) break;
            continue;
        }
        if (have) {
            uint32_t hword;
            const bool took = walk_step<T, WM, PART>(G, A, wid, pid, step, cur, prev, tl, team_mask, team_base, lane, hword);
            uint32_t* row = A.paths + wid * (uint64_t)A.stride;
            // Path entry `step` is the vertex this step started from, whose hot line carries the
            // caller's id; it is read there (no extra load) except when the walk stopped before
            // reading it, and for the last vertex of a walk.
            if (step && tl == 0) row[step] = hword != NONE32 ? hword : to_caller(G, cur);
            bool remote = false;
            if (took) {
                step++;
                if (PART) {  // partitioned: the sampled vertex is a global id
                    remote = cur - G.base >= G.n;
                    if (!remote) cur -= G.base;
                }
                if (step == L && tl == 0) row[step] = remote ? cur : to_caller(G, cur);
            }
            if (!took || step == L) {
                finish_walker(A, wid, step, tl, T, team_mask);
                have = false;
            } else if (PART && remote) {  // continue in the owner's next launch
                if (tl == 0) {
                    row[step] = cur;
                    PartRec rc;
                    rc.wid = wid;
                    rc.cur = cur;
                    rc.prev = prev;
                    rc.step = step;
                    rc.pad = 0;
                    A.outbox[atomicAdd(A.nout, 1ull)] = rc;
                }
                have = false;
            }
        }
    }
}

// The paper's step-by-step form (Section 6 (iii)): one launch per step, one thread per walker.
template <int WM>
__global__ void k_walk_step(DevGraph G, WalkParams A, uint32_t s) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t wid = tid; wid < A.nwalkers; wid += nt) {
        uint32_t pid = walker_pid(A, wid);
        if (pid >= A.npol) pid = 0;
        uint32_t L = A.lengths ? __ldg(A.lengths + wid) : __ldg(&A.pols[pid].max_len);
        if (L + 1 > A.stride) L = A.stride - 1;
        uint32_t cur, prev;
        if (s == 0) {
            cur = __ldg(A.starts + wid);
            prev = NONE32;
            if (cur >= G.n) { L = 0; atomicOr(A.status, ST_INVALID); }
            A.paths[wid * (uint64_t)A.stride] = cur;
            cur = to_internal(G, cur);
            if (L == 0) {
                finish_walker(A, wid, 0, 0, 1, 1u << (threadIdx.x & 31));
                A.s_cur[wid] = NONE32;
                continue;
            }
        } else {
            cur = A.s_cur[wid];
            if (cur == NONE32) continue;
            prev = A.s_prev[wid];
        }
        uint32_t hword;
        const bool took = walk_step<1, WM, false>(G, A, wid, pid, s, cur, prev, 0, 0, 0, 0, hword);
        if (took) A.paths[wid * (uint64_t)A.stride + s + 1] = to_caller(G, cur);
        if (!took || s + 1 == L) {
            finish_walker(A, wid, took ? s + 1 : s, 0, 1, 1u << (threadIdx.x & 31));
            A.s_cur[wid] = NONE32;
        } else {
            A.s_cur[wid] = cur;
            A.s_prev[wid] = prev;
        }
    }
}

// ---------------------------------------------------------------------------------------- edge index

__global__ void k_eh_build(DevGraph G) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = warp; v < G.n; v += nwarps) {
        const VHdr h = load_hdr(G, v);
        const uint2* pairs = adj_pairs(G, h.adj);
        for (uint32_t j = lane; j < h.deg; j += 32) {
            const unsigned long long key = (v << 32) | pairs[j].x;
            uint64_t p = eh_hash(key) & G.eh_mask;
            for (uint64_t probe = 0; probe <= G.eh_mask; probe++) {
                const unsigned long long old = atomicCAS(G.eh_key + p, EH_EMPTY, key);
                if (old == EH_EMPTY || old == key) {
                    atomicAdd(G.eh_cnt + p, 1u);
                    break;
                }
                p = (p + 1) & G.eh_mask;
            }
        }
    }
}

}  // namespace

namespace bingo {

// Build (or rebuild) the node2vec edge index at load factor <= 1/2.
bingo_status edge_index_build(bingo_graph* g, cudaStream_t s) {
    uint64_t cap = 1024;
    while (cap < 2 * (g->m_live + 1)) cap <<= 1;
    if (g->d_eh) cudaFree(g->d_eh);
    g->d_eh = nullptr;
    g->G.eh_mask = 0;
    CK(cudaMalloc(&g->d_eh, cap * 12), "edge index");
    g->G.eh_key = (unsigned long long*)g->d_eh;
    g->G.eh_cnt = (uint32_t*)((char*)g->d_eh + cap * 8);
    g->G.eh_mask = cap - 1;
    CK(cudaMemsetAsync(g->G.eh_key, 0xFF, cap * 8, s), "edge index init");
    CK(cudaMemsetAsync(g->G.eh_cnt, 0, cap * 4, s), "edge index init");
    unsigned blocks = (unsigned)std::min<uint64_t>(((uint64_t)g->n * 32 + 255) / 256, (uint64_t)g->num_sms * 16);
    k_eh_build<<<blocks ? blocks : 1, 256, 0, s>>>(g->G);
    g->launches++;
    g->eh_distinct = g->m_live;
    CK(cudaGetLastError(), "edge index build");
    return BINGO_OK;
}

static int g_occ_cache[3][2][3][33];

static int weight_mode(const bingo_graph* g) { return g->G.fbits ? WM_REAL : g->G.base4 ? WM_B4 : WM_INT; }

template <int T, int OCC>
static void* walk_kernel_ptr(int wm) {
    return wm == WM_REAL ? (void*)k_walk_persistent<T, OCC, WM_REAL>
           : wm == WM_B4 ? (void*)k_walk_persistent<T, OCC, WM_B4>
                         : (void*)k_walk_persistent<T, OCC, WM_INT>;
}

static void* walk_kernel(int lanes, int occ, int wm) {
    if (occ)
        return lanes == 1 ? walk_kernel_ptr<1, 1>(wm) : lanes == 4 ? walk_kernel_ptr<4, 1>(wm)
                                                                   : walk_kernel_ptr<32, 1>(wm);
    return lanes == 1 ? walk_kernel_ptr<1, 0>(wm) : lanes == 4 ? walk_kernel_ptr<4, 0>(wm)
                                                               : walk_kernel_ptr<32, 0>(wm);
}

static int walk_blocks_per_sm(int lanes, int wpb, int occ, int wm) {
    const int li = lanes == 1 ? 0 : lanes == 4 ? 1 : 2;
    if (wpb < 1 || wpb > 32) return 1;
    int& c = g_occ_cache[wm][occ ? 1 : 0][li][wpb];
    if (c) return c;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, walk_kernel(lanes, occ, wm), wpb * 32, 0);
    c = nb < 1 ? 1 : nb;
    return c;
}

// Every walker instance of the graph's weight mode is launched once over zero walkers: the launch
// loads its module (lazy loading) and grows the context's local-memory reservation to the kernel's
// frame, so no later walk launch does either (both can allocate device memory).
cudaError_t walk_preload(bingo_graph* g, cudaStream_t s) {
    const int wm = weight_mode(g);
    WalkParams A;
    memset(&A, 0, sizeof(A));
    A.queue = (unsigned long long*)((uint64_t*)g->d_ctl + CTL_QUEUE);
    A.status = (uint32_t*)((uint64_t*)g->d_ctl + CTL_STATUS);
    A.stride = 1;
    A.npol = 1;
    void* args[] = {(void*)&g->G, (void*)&A};
    for (int occ = 0; occ < 2; occ++)
        for (int lanes : {1, 4, 32}) {
            const cudaError_t e = cudaLaunchKernel(walk_kernel(lanes, occ, wm), dim3(1), dim3(32), args, 0, s);
            if (e != cudaSuccess) return e;
            g->launches++;
        }
    if (wm == WM_REAL) k_walk_step<WM_REAL><<<1, 32, 0, s>>>(g->G, A, 0);
    else if (wm == WM_B4) k_walk_step<WM_B4><<<1, 32, 0, s>>>(g->G, A, 0);
    else k_walk_step<WM_INT><<<1, 32, 0, s>>>(g->G, A, 0);
    g->launches++;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), s);
}

// Launch the walk on device buffers (all pointers device).  Pre: policies validated.
bingo_status walk_launch(bingo_graph* g, const WalkReq& q, cudaStream_t s) {
    WalkParams A;
    memset(&A, 0, sizeof(A));
    A.hot_last = g->cfg.hot_l2_hint != BINGO_HOT_NORMAL;
    const uint64_t nwalkers = q.nwalkers;
    const uint32_t mode = q.mode, max_steps = q.max_steps;
    A.nwalkers = nwalkers;
    A.starts = q.starts;
    A.lengths = q.lengths;
    A.pids = q.pids;
    A.key = make_uint2((uint32_t)q.seed, (uint32_t)(q.seed >> 32));
    A.stride = q.stride;
    A.npol = q.npol;
    A.flags = q.pad ? WF_PAD : 0;
    A.paths = q.paths;
    A.plen = q.plen;
    A.queue = q.queue;
    A.status = (uint32_t*)((uint64_t*)g->d_ctl + CTL_STATUS);
    A.pols = q.dev_pols;
    A.req_off = q.req_off;
    A.req_key = q.req_key;
    A.nreq = q.nreq;
    A.chunk_done = q.chunk_done;
    A.host_flags = q.host_flags;
    A.chunk_shift = q.chunk_shift;
    A.io_seq = q.io_seq;
    A.resume = q.resume;
    A.outbox = q.outbox;
    A.nout = q.nout;
    A.peh = q.peh;
    A.bounds = q.bounds;
    A.npart = q.npart;
    if (nwalkers == 0) return BINGO_OK;
    if (mode == BINGO_WALK_STEPWISE) {
        CK(ensure(g->s_walk, 8 * nwalkers), "walk state");
        A.s_cur = (uint32_t*)g->s_walk.p;
        A.s_prev = A.s_cur + nwalkers;
        const unsigned blocks = (unsigned)std::min<uint64_t>((nwalkers + 255) / 256, (uint64_t)g->num_sms * 8);
        for (uint32_t st = 0; st < (max_steps ? max_steps : 1); st++) {
            const int wm = weight_mode(g);
            if (wm == WM_REAL) k_walk_step<WM_REAL><<<blocks, 256, 0, s>>>(g->G, A, st);
            else if (wm == WM_B4) k_walk_step<WM_B4><<<blocks, 256, 0, s>>>(g->G, A, st);
            else k_walk_step<WM_INT><<<blocks, 256, 0, s>>>(g->G, A, st);
            g->launches++;
        }
        CK(cudaGetLastError(), "stepwise walk launch");
        return BINGO_OK;
    }
    CK(cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), s), "walk queue reset");
    g->launches++;
    const int lanes = (int)g->tune.lanes, occ_mode = (int)g->tune.occ;
    int wpb = (int)g->tune.warps_per_block;
    if (occ_mode && wpb > 8) wpb = 8;  // the 40-register variant is bounded to 256-thread blocks
    if (wpb > WALK_MAX_THREADS / 32) wpb = WALK_MAX_THREADS / 32;
    if (wpb < 1) wpb = 1;
    int bps = (int)g->tune.blocks_per_sm;
    const int wm = weight_mode(g);
    const int occ = walk_blocks_per_sm(lanes, wpb, occ_mode, wm);
    if (bps <= 0 || bps > occ) bps = occ;
    uint64_t blocks = (uint64_t)g->num_sms * bps;
    const uint64_t walkers_per_block = (uint64_t)wpb * (32 / lanes);
    const uint64_t useful = (nwalkers + walkers_per_block - 1) / walkers_per_block;
    if (blocks > useful) blocks = useful;
    if (blocks == 0) blocks = 1;
    void* args[] = {(void*)&g->G, (void*)&A};
    void* fn = walk_kernel(lanes, occ_mode, wm);
    if (q.resume) {  // partitioned walks: one lane per walker, the 80-register build
        fn = wm == WM_REAL ? (void*)k_walk_persistent<1, 0, WM_REAL, true>
             : wm == WM_B4 ? (void*)k_walk_persistent<1, 0, WM_B4, true>
                           : (void*)k_walk_persistent<1, 0, WM_INT, true>;
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 8 * 32, 0);
        blocks = std::min<uint64_t>((uint64_t)g->num_sms * (nb < 1 ? 1 : nb), (nwalkers + 31) / 32);
        wpb = 8;
    }
    CK(cudaLaunchKernel(fn, dim3((unsigned)(blocks ? blocks : 1)), dim3(wpb * 32), args, 0, s), "walk launch");
    g->launches++;
    CK(cudaGetLastError(), "walk launch");
    return BINGO_OK;
}

}  // namespace bingo
