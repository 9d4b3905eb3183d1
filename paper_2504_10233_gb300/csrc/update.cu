// Batched and streaming edge updates applied in place to the radix groups.
//
// Batch (Section 5.2, Fig. update): records are grouped by source vertex on the
// GPU (stable radix sort on (src, is_delete, dst)); per vertex, insertions are
// appended, deletions resolved to the earliest live copy of (src, dst), the
// group counts updated by the bits of the inserted / deleted biases (Eq. dwi),
// members removed from regular and sparse groups by two-phase delete-and-swap,
// the adjacency compacted the same way (moved edges are renumbered in every
// group through the inverted indexes, Section 4.2), new members appended, and
// groups whose kind changed (Eq. group) rebuilt from the adjacency.
// Streaming (Section 4.2): the same per-vertex procedure, one record at a time,
// in order, inside one launch.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "bingo_host.h"
#include "groups.cuh"

using namespace bingo;

#define CK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

namespace {

constexpr unsigned long long INF64 = 0xFFFFFFFFFFFFFFFFull;
constexpr uint32_t ST_STOP = ST_INVALID | ST_OOM | ST_STATE;

// stats layout inside CTL_STATS: 0 inserted, 1 deleted, 2 not_found, 3 touched, 4 rebuilt, 5.. conv[5][5]
enum { S_INS = 0, S_DEL = 1, S_NF = 2, S_TOUCH = 3, S_REBUILT = 4, S_CONV = 5 };

// Source of a segment's records: insertions (dst, bias, edge id) and deletions (dst, sorted ascending).
struct BatchSrc {
    const uint4* rec;      // per insertion key: {edge id low, dst, bias, edge id high}
    const uint64_t* keys;
    uint64_t dmask;
    uint64_t start;  // first key of the segment
    uint32_t ni;
    const uint32_t* sdel;  // deletion destinations staged in shared memory (nullable)
    __device__ __forceinline__ uint4 ins(uint32_t i) const { return rec[start + i]; }
    __device__ __forceinline__ uint64_t ins_eid(uint32_t i) const {
        const uint4 r = rec[start + i];
        return (uint64_t)r.x | ((uint64_t)(r.w & 0xFFFFFFu) << 32);
    }
    __device__ __forceinline__ uint32_t ins_q(uint32_t i) const { return rec[start + i].w >> 24; }
    __device__ __forceinline__ uint32_t del_dst_global(uint32_t j) const {
        return (uint32_t)(keys[start + ni + j] & dmask);
    }
    __device__ __forceinline__ uint32_t del_dst(uint32_t j) const { return sdel ? sdel[j] : del_dst_global(j); }
};

struct OneSrc {
    uint32_t dst, bias, q;  // bias: the factorised (integer) part; q: decimal part of a real bias
    uint64_t eid;
    const uint32_t* sdel = nullptr;
    __device__ __forceinline__ uint32_t del_dst_global(uint32_t) const { return dst; }
    __device__ __forceinline__ uint4 ins(uint32_t) const { return make_uint4(0, dst, bias, 0); }
    __device__ __forceinline__ uint64_t ins_eid(uint32_t) const { return eid; }
    __device__ __forceinline__ uint32_t ins_q(uint32_t) const { return q; }
    __device__ __forceinline__ uint32_t del_dst(uint32_t) const { return dst; }
};

// team-shared state of one segment
struct SegSh {
    uint32_t cnt_old[32];
    uint32_t cnt_new[32];
    int32_t delta[32];
    uint32_t removed[32];      // dead pre-existing edges with bit k
    uint64_t gref_old[32];
    uint64_t gref_new[32];
    uint32_t tscratch[40];     // block-team scan scratch
    uint64_t adj;
    uint64_t alloc_off;
    uint32_t nsp_del, nsp_add;
    uint32_t rounds;
    uint32_t found;
    uint32_t kmask[8];
};

// Kind masks of the 32 groups from (cnt[k], d): lane k of the first warp evaluates Eq. group for
// group k and ballots form the masks (published through shared memory for block teams).
struct KindMasks {
    uint32_t sp, reg, one, nonempty;
};
template <bool REAL, class Team>
__device__ __forceinline__ KindMasks kind_masks(const Team& t, SegSh& sh, const uint32_t* cnt, uint32_t d,
                                                const DevGraph& G, int slot) {
    KindMasks km;
    constexpr bool warp_team = std::is_same<Team, WarpTeam>::value;
    if (warp_team || threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x & 31;
        const uint32_t c = cnt[lane];
        const uint32_t kd = (REAL && lane == DEC_SLOT) ? (uint32_t)K_EMPTY : kind_of(c, d, G.alpha, G.beta);
        km.sp = __ballot_sync(FULL, kd == K_SPARSE);
        km.reg = __ballot_sync(FULL, kd == K_REGULAR);
        km.one = __ballot_sync(FULL, kd == K_ONE);
        km.nonempty = __ballot_sync(FULL, c > 0);
    }
    if constexpr (!warp_team) {
        if (threadIdx.x == 0) {
            sh.kmask[4 * slot + 0] = km.sp;
            sh.kmask[4 * slot + 1] = km.reg;
            sh.kmask[4 * slot + 2] = km.one;
            sh.kmask[4 * slot + 3] = km.nonempty;
        }
        t.sync();
        km.sp = sh.kmask[4 * slot + 0];
        km.reg = sh.kmask[4 * slot + 1];
        km.one = sh.kmask[4 * slot + 2];
        km.nonempty = sh.kmask[4 * slot + 3];
    }
    return km;
}

// equal range of x among the segment's (sorted) deletion destinations
template <class Src>
__device__ __forceinline__ void del_range(const Src& B, uint32_t nd, uint32_t x, uint32_t& lo_out, uint32_t& hi_out) {
    uint32_t lo = 0, hi = nd;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (B.del_dst(mid) < x) lo = mid + 1; else hi = mid;
    }
    uint32_t a = lo;
    hi = nd;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (B.del_dst(mid) <= x) lo = mid + 1; else hi = mid;
    }
    lo_out = a;
    hi_out = lo;
}

// Two-phase parallel delete-and-swap (Section 5.2, Fig. update(b)) on a list L of length c.
// cand(i), i < ncand, yields a position to delete or NONE32.  Phase 1 marks the N deleted
// positions; the N tail positions [c-N, c) then hold gamma deleted entries and N-gamma survivors,
// and phase 2 moves the survivors (ascending) into the N-gamma holes below c-N (in candidate
// order), with their entries of the parallel array M (nullable).  move(value, from, to) patches the
// inverted index of each moved entry.
template <class Team, class Cand, class Move>
__device__ uint32_t dswap(const Team& t, uint32_t* L, uint32_t* M, uint32_t c, uint32_t ncand, Cand cand, Move move,
                          uint32_t* holes, uint32_t* surv, uint32_t* status) {
    uint32_t nrem = 0;
    for (uint32_t b = 0; b < ncand; b += t.size()) {
        const uint32_t i = b + t.rank();
        uint32_t p = i < ncand ? cand(i) : NONE32;
        if (p != NONE32 && p >= c) {  // inconsistent inverted index: record and skip
            atomicOr(status, ST_STATE);
            p = NONE32;
        }
        if (p != NONE32) L[p] = NONE32;
        nrem += t.sum(p != NONE32 ? 1u : 0u);
    }
    t.sync();
    if (nrem == 0) return c;
    const uint32_t c1 = c - nrem;
    uint32_t nh = 0;
    for (uint32_t b = 0; b < ncand; b += t.size()) {
        const uint32_t i = b + t.rank();
        uint32_t p = i < ncand ? cand(i) : NONE32;
        if (p != NONE32 && p >= c) p = NONE32;
        const bool pred = p != NONE32 && p < c1;
        uint32_t tot;
        const uint32_t r = t.scan_pred(pred, tot);
        if (pred) holes[nh + r] = p;
        nh += tot;
    }
    uint32_t ns = 0;
    for (uint32_t b = c1; b < c; b += t.size()) {
        const uint32_t q = b + t.rank();
        const bool pred = q < c && L[q] != NONE32;
        uint32_t tot;
        const uint32_t r = t.scan_pred(pred, tot);
        if (pred) surv[ns + r] = q;
        ns += tot;
    }
    t.sync();
    for (uint32_t b = 0; b < nh; b += t.size()) {
        const uint32_t r = b + t.rank();
        if (r < nh) {
            const uint32_t h = holes[r], s = (r < ns) ? surv[r] : NONE32;
            if (s == NONE32) {
                atomicOr(status, ST_STATE);
            } else {
                const uint32_t val = L[s];
                L[h] = val;
                if (M) M[h] = M[s];  // the member's destination travels with it
                move(val, s, h);
            }
        }
    }
    t.sync();
    return c1;
}

struct SegScratch {
    uint32_t* holes;          // >= nd entries
    uint32_t* surv;           // >= nd entries
    uint32_t* ins_final;      // [ni] final slot of each inserted edge (NONE32 if deleted in the batch)
    uint32_t* del_slot;       // [nd] slot removed by each deletion (NONE32 if not found)
    unsigned long long* best; // [nd]
};

constexpr uint32_t PRE_MULT = 4;             // candidate region per deletion key
constexpr uint32_t PRE_CHUNK = 256 * 8;      // slots of one pre-pass work item
constexpr uint32_t PRE_MIN_DEG = 1024;       // segments with deletions at vertices this large are pre-scanned
constexpr uint32_t NO_PRE = 0xFFFFFFFFu;

// Deletion candidates among the pre-existing slots [0, d0), collected for a big segment by the
// grid-wide pre-pass (k_cand_scan); list == nullptr when there is none.
struct PreCand {
    const uint32_t* list = nullptr;
    uint32_t count = 0, cap = 0;
};

// S3 of a segment: resolve each deletion to the earliest live copy (smallest edge id) of (v, dst);
// the r-th deletion of the same dst takes the r-th earliest copy (round r).  Marks the chosen slots
// dead (DEAD_BIT in the edge id), records them in X.del_slot and returns how many deletions found a copy.
template <class Team, class Src>
__device__ __forceinline__ uint32_t resolve_deletions(const Team& t, Src& B, const SegScratch& X, uint2* pairs,
                                                      uint64_t* eids, uint32_t d0, uint32_t ni, uint32_t nd,
                                                      uint32_t* sdel_buf, uint32_t sdel_cap, uint32_t* cand_buf,
                                                      uint32_t cand_cap, const PreCand& pre) {
    const uint32_t rank = t.rank(), T = t.size();
    const uint32_t dtot = d0 + ni;
    // The sorted deletion destinations are staged in shared memory when they fit, for the per-slot searches.
    if (nd && sdel_buf && nd <= sdel_cap) {
        for (uint32_t j = rank; j < nd; j += T) sdel_buf[j] = B.del_dst_global(j);
        t.sync();
        B.sdel = sdel_buf;
    }
    if (nd) {
        uint32_t mr = 0;
        for (uint32_t j = rank; j < nd; j += T) {
            uint32_t lo, hi;
            del_range(B, nd, B.del_dst(j), lo, hi);
            mr = max(mr, j - lo + 1);
        }
        const uint32_t rounds = t.max(mr);
        // Candidates: live slots whose destination is deleted in this segment, collected once (a
        // duplicated edge repeated in the batch needs one round per repetition, and RMAT hubs carry
        // many duplicates); the rounds then scan only the candidates.
        uint32_t ncand = 0;
        bool use_cand = cand_buf != nullptr;
        if (use_cand) {
            auto is_cand = [&](uint2 xe, uint32_t) {
                if (xe.y & (uint32_t)(DEAD_BIT >> 32)) return false;
                const uint32_t x = xe.x;
                uint32_t lo = 0, hi = nd;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (B.del_dst(mid) < x) lo = mid + 1; else hi = mid;
                }
                return lo < nd && B.del_dst(lo) == x;
            };
            if (pre.list && pre.count <= pre.cap) {
                // the pre-pass scanned [0, d0); only the appended slots are left to test
                const uint32_t n0 = pre.count;
                if (n0 <= cand_cap)
                    for (uint32_t i = rank; i < n0; i += T) cand_buf[i] = pre.list[i];
                const uint32_t n1 = team_compact_lt(
                    t, ni, [&](uint32_t j) { return make_uint2(pairs[d0 + j].x, (uint32_t)(eids[d0 + j] >> 32)); },
                    is_cand,
                    [&](uint32_t j, uint32_t pos) {
                        if (n0 + pos < cand_cap) cand_buf[n0 + pos] = d0 + j;
                    });
                ncand = n0 + n1;
            } else {
                ncand = team_compact_lt(
                    t, dtot, [&](uint32_t j) { return make_uint2(pairs[j].x, (uint32_t)(eids[j] >> 32)); }, is_cand,
                    [&](uint32_t j, uint32_t pos) {
                        if (pos < cand_cap) cand_buf[pos] = j;
                    });
            }
            use_cand = ncand <= cand_cap;
            t.sync();
        }
        if (use_cand) {
            for (uint32_t r = 0; r < rounds; r++) {
                for (uint32_t i = rank; i < ncand; i += T) {
                    const uint32_t j = cand_buf[i];
                    const uint64_t e = eids[j];
                    if (e & DEAD_BIT) continue;
                    uint32_t lo, hi;
                    del_range(B, nd, pairs[j].x, lo, hi);
                    if (hi - lo > r) atomicMin(&X.best[lo + r], (unsigned long long)e);
                }
                t.sync();
                for (uint32_t i = rank; i < ncand; i += T) {
                    const uint32_t j = cand_buf[i];
                    const uint64_t e = eids[j];
                    if (e & DEAD_BIT) continue;
                    uint32_t lo, hi;
                    del_range(B, nd, pairs[j].x, lo, hi);
                    if (hi - lo > r && X.best[lo + r] == e) {
                        eids[j] = e | DEAD_BIT;
                        X.del_slot[lo + r] = j;
                    }
                }
                t.sync();
            }
        }
        // Each thread takes RES_IT consecutive slots per iteration with their loads in flight together.
        constexpr int RES_IT = 4;
        for (uint32_t r = 0; r < (use_cand ? 0u : rounds); r++) {
            for (uint32_t j0 = rank * RES_IT; j0 < dtot; j0 += T * RES_IT) {
                uint32_t x[RES_IT];
                uint64_t e[RES_IT];
#pragma unroll
                for (int q = 0; q < RES_IT; q++) {
                    const bool in = j0 + q < dtot;
                    x[q] = in ? pairs[j0 + q].x : 0u;
                    e[q] = in ? eids[j0 + q] : DEAD_BIT;
                }
#pragma unroll
                for (int q = 0; q < RES_IT; q++) {
                    if (e[q] & DEAD_BIT) continue;
                    uint32_t lo, hi;
                    del_range(B, nd, x[q], lo, hi);
                    if (hi - lo > r) atomicMin(&X.best[lo + r], (unsigned long long)e[q]);
                }
            }
            t.sync();
            for (uint32_t j0 = rank * RES_IT; j0 < dtot; j0 += T * RES_IT) {
                uint32_t x[RES_IT];
                uint64_t e[RES_IT];
#pragma unroll
                for (int q = 0; q < RES_IT; q++) {
                    const bool in = j0 + q < dtot;
                    x[q] = in ? pairs[j0 + q].x : 0u;
                    e[q] = in ? eids[j0 + q] : DEAD_BIT;
                }
#pragma unroll
                for (int q = 0; q < RES_IT; q++) {
                    if (e[q] & DEAD_BIT) continue;
                    uint32_t lo, hi;
                    del_range(B, nd, x[q], lo, hi);
                    if (hi - lo > r && X.best[lo + r] == e[q]) {
                        eids[j0 + q] = e[q] | DEAD_BIT;
                        X.del_slot[lo + r] = j0 + q;
                    }
                }
            }
            t.sync();
        }
    }
    uint32_t found = 0;
    for (uint32_t b = 0; b < nd; b += T) {
        const uint32_t j = b + rank;
        found += t.sum(j < nd && X.del_slot[j] != NONE32 ? 1u : 0u);
    }
    return found;
}

// S11-S12 of a segment: the new groups (sh.cnt_new, sh.gref_new), the walker's hot-line summary and
// the header h1; then the batch statistics, kind conversions included.
template <bool REAL, class Team>
__device__ __forceinline__ void write_back(const Team& t, const DevGraph& G, const SegSh& sh, uint32_t v, const VHdr& h1,
                                           uint32_t d0, uint32_t ni, uint32_t nd, uint32_t found, uint32_t rebuilt,
                                           unsigned long long* stats) {
    const uint32_t rank = t.rank(), T = t.size();
    for (uint32_t k = rank; k < 32; k += T) grp(G, v, k) = make_uint2(sh.cnt_new[k], (uint32_t)sh.gref_new[k]);
    if (rank < 32)  // the team's first warp (the whole team for a warp team): the hot line
        write_hot(G, v, rank, sh.cnt_new[rank], (uint32_t)sh.gref_new[rank], h1.word);
    if (rank == 0) {
        store_hdr(G, v, h1);
        atomicAdd(stats + S_INS, (unsigned long long)ni);
        atomicAdd(stats + S_DEL, (unsigned long long)found);
        atomicAdd(stats + S_NF, (unsigned long long)(nd - found));
        atomicAdd(stats + S_TOUCH, 1ull);
        if (rebuilt) atomicAdd(stats + S_REBUILT, (unsigned long long)rebuilt);
    }
    for (uint32_t k = rank; k < 32; k += T) {
        const bool dec = REAL && k == DEC_SLOT;
        const uint32_t ko = dec ? (uint32_t)K_EMPTY : kind_of(sh.cnt_old[k], d0, G.alpha, G.beta);
        const uint32_t kn = dec ? (uint32_t)K_EMPTY : kind_of(sh.cnt_new[k], h1.deg, G.alpha, G.beta);
        if (ko != kn) atomicAdd(stats + S_CONV + ko * 5 + kn, 1ull);
    }
    t.sync();
}

// Apply one vertex's segment (ni insertions then nd deletions).  Returns false if the graph ran out of pool.
// REAL: real-bias graphs (decimal parts follow their edges, slot 31 holds the decimal total).
template <bool REAL, class Team, class Src>
__device__ void apply_segment(const Team& t, const DevGraph& G, SegSh& sh, uint32_t v, uint32_t ni, uint32_t nd,
                              Src B, const SegScratch& X, unsigned long long* stats, uint32_t* sdel_buf,
                              uint32_t sdel_cap, uint32_t* cand_buf = nullptr, uint32_t cand_cap = 0,
                              PreCand pre = PreCand()) {
    const uint32_t rank = t.rank(), T = t.size();
    const VHdr h0 = load_hdr(G, v);
    const uint32_t d0 = h0.deg, capa0 = capa_of(h0), caps0 = caps_of(h0);
    const uint32_t dtot = d0 + ni;
    for (uint32_t k = rank; k < 32; k += T) {
        const uint2 gk = grp(G, v, k);
        sh.cnt_old[k] = gk.x;
        sh.gref_old[k] = gk.y;
        sh.gref_new[k] = sh.gref_old[k];
        sh.delta[k] = 0;
        sh.removed[k] = 0;
    }
    if (rank == 0) {
        sh.adj = h0.adj;
        sh.nsp_del = 0;
        sh.nsp_add = 0;
        sh.found = 0;
        sh.rounds = 0;
    }
    t.sync();
    // old kinds
    const KindMasks kmo = kind_masks<REAL>(t, sh, sh.cnt_old, d0, G, 0);
    const uint32_t SPo = kmo.sp, REGo = kmo.reg, ONEo = kmo.one;

    // ---- S1: adjacency capacity for the insertions
    uint32_t capa1 = capa0;
    bool full = false;
    if (dtot > capa0) {
        capa1 = capa_for(dtot);
        full = true;
        if (rank == 0) sh.alloc_off = pool_alloc(G.pool, 4ull * capa1);
        t.sync();
        const uint64_t noff = sh.alloc_off;
        if (noff == 0) return;  // pool exhausted (flagged); the pre-check makes this unreachable
        if (d0) {
            const uint2* op = adj_pairs(G, h0.adj);
            const uint64_t* oe = adj_eids(G, h0.adj, capa0);
            uint2* np = adj_pairs(G, noff);
            uint64_t* ne = adj_eids(G, noff, capa1);
            for (uint32_t j = rank; j < d0; j += T) {
                np[j] = op[j];
                ne[j] = oe[j];
            }
        }
        if constexpr (REAL) {  // the decimal block follows the adjacency's capacity
            if (rank == 0) sh.alloc_off = pool_alloc(G.pool, dec_words(capa1));
            t.sync();
            const uint64_t qoff = sh.alloc_off;
            if (qoff == 0) return;
            uint8_t* nq = reinterpret_cast<uint8_t*>(G.pool.base + qoff);
            if (d0) {
                const uint8_t* oq = dec_bytes(G, (uint32_t)sh.gref_old[DEC_SLOT]);
                for (uint32_t j = rank; j < d0; j += T) nq[j] = oq[j];
            }
            t.sync();
            if (rank == 0) {
                if (capa0) pool_free(G.pool, words_of(sh.gref_old[DEC_SLOT]), dec_words(capa0));
                sh.gref_new[DEC_SLOT] = ref_of(qoff);
            }
        }
        t.sync();
        if (rank == 0) {
            if (capa0) pool_free(G.pool, h0.adj, 4ull * capa0);
            sh.adj = noff;
        }
        t.sync();
    }
    const uint64_t adj = sh.adj;
    uint2* pairs = adj_pairs(G, adj);
    uint64_t* eids = adj_eids(G, adj, capa1);
    // real biases: decimal part of each slot (moves with its edge)
    uint8_t* qbytes = nullptr;
    if constexpr (REAL)
        if (sh.gref_new[DEC_SLOT]) qbytes = dec_bytes(G, (uint32_t)sh.gref_new[DEC_SLOT]);

    // ---- S2: append insertions at slots d0 .. d0+ni-1
    for (uint32_t i = rank; i < ni; i += T) {
        const uint4 u = B.ins(i);
        pairs[d0 + i] = make_uint2(u.y, u.z);
        eids[d0 + i] = B.ins_eid(i);
        if (qbytes) qbytes[d0 + i] = (uint8_t)B.ins_q(i);
    }
    for (uint32_t j = rank; j < nd; j += T) {
        X.del_slot[j] = NONE32;
        X.best[j] = INF64;
    }
    t.sync();

    // ---- S3: resolve each deletion to the earliest live copy
    const uint32_t found = resolve_deletions(t, B, X, pairs, eids, d0, ni, nd, sdel_buf, sdel_cap, cand_buf, cand_cap, pre);
    const uint32_t d1 = dtot - found;

    // ---- S4: count deltas from the bits of deleted pre-existing and surviving new edges
    uint32_t deadbits_local = 0;
    for (uint32_t j = rank; j < nd; j += T) {
        const uint32_t s = X.del_slot[j];
        if (s != NONE32 && s < d0) {
            const uint32_t w = pairs[s].y;
            deadbits_local |= w;
            for (uint32_t b = w; b; b &= b - 1) {
                const int k = __ffs(b) - 1;
                atomicAdd(&sh.delta[k], -1);
                atomicAdd(&sh.removed[k], 1u);
            }
        }
    }
    for (uint32_t i = rank; i < ni; i += T) {
        if (!(eids[d0 + i] & DEAD_BIT)) {
            const uint32_t w = pairs[d0 + i].y;
            for (uint32_t b = w; b; b &= b - 1) atomicAdd(&sh.delta[__ffs(b) - 1], 1);
        }
    }
    uint32_t q_add = 0, q_sub = 0;  // decimal total: parts of surviving insertions minus deleted edges
    if (qbytes) {
        for (uint32_t b = 0; b < nd; b += T) {
            const uint32_t j = b + rank;
            const uint32_t s = j < nd ? X.del_slot[j] : NONE32;
            q_sub += t.sum(s != NONE32 && s < d0 ? (uint32_t)qbytes[s] : 0u);
        }
        for (uint32_t b = 0; b < ni; b += T) {
            const uint32_t i = b + rank;
            q_add += t.sum(i < ni && !(eids[d0 + i] & DEAD_BIT) ? (uint32_t)qbytes[d0 + i] : 0u);
        }
    }
    t.sync();
    for (uint32_t k = rank; k < 32; k += T)
        sh.cnt_new[k] = (qbytes && k == DEC_SLOT) ? sh.cnt_old[k] + q_add - q_sub
                                                  : (uint32_t)((int32_t)sh.cnt_old[k] + sh.delta[k]);
    t.sync();
    const KindMasks kmn = kind_masks<REAL>(t, sh, sh.cnt_new, d1, G, 1);
    const uint32_t SPn = kmn.sp, REGn = kmn.reg, ONEn = kmn.one, maskn = kmn.nonempty;
    // bits of the deleted pre-existing edges (the groups that lose members)
    const uint32_t deadbits = t.or_all(deadbits_local);
    const uint32_t REGk = full ? 0u : (REGo & REGn);              // regular groups updated in place
    const uint32_t ONEk = full ? 0u : (ONEo & ONEn & ~deadbits);   // one-element groups whose member survives
    bool keepS = !full && SPo == SPn && SPn != 0 && h0.sref != 0;
    uint32_t nsp1 = 0;
    if (keepS) {
        uint32_t del_s = 0, add_s = 0;
        for (uint32_t b = 0; b < nd; b += T) {
            const uint32_t j = b + rank;
            const uint32_t s = j < nd ? X.del_slot[j] : NONE32;
            del_s += t.sum(s != NONE32 && s < d0 && (pairs[s].y & SPo) ? 1u : 0u);
        }
        for (uint32_t b = 0; b < ni; b += T) {
            const uint32_t i = b + rank;
            const bool live = i < ni && !(eids[d0 + i] & DEAD_BIT);
            add_s += t.sum(live && (pairs[d0 + i].y & SPn) ? 1u : 0u);
        }
        nsp1 = h0.nsp - del_s + add_s;
        if (nsp1 > caps0) keepS = false;  // sparse capacity outgrown: rebuild S and sparse groups
    }

    // ---- S6: remove deleted members from regular groups kept in place
    for (uint32_t m = REGk & deadbits; m; m &= m - 1) {
        const uint32_t k = __ffs(m) - 1;
        uint32_t* M = G.pool.base + words_of(sh.gref_old[k]);
        uint32_t* L = M + capa0;
        uint32_t* inv = L + capa0;
        const uint32_t icap_guard = capa0;
        dswap(
            t, L, M, sh.cnt_old[k], nd,
            [&](uint32_t j) -> uint32_t {
                const uint32_t s = X.del_slot[j];
                return (s != NONE32 && s < d0 && ((pairs[s].y >> k) & 1u)) ? inv[s] : NONE32;
            },
            [&](uint32_t val, uint32_t, uint32_t to) { if (val < icap_guard) inv[val] = to; }, X.holes, X.surv, G.pool.status);
    }
    // ---- S7: sparse groups, then the sparse list itself
    uint32_t nsp_after_del = h0.nsp;
    if (keepS) {
        uint32_t* S = G.pool.base + h0.sref;
        uint32_t* Sinv = S + capa0;
        for (uint32_t m = SPn & deadbits; m; m &= m - 1) {
            const uint32_t k = __ffs(m) - 1;
            uint32_t* M = G.pool.base + words_of(sh.gref_old[k]);
            uint32_t* L = M + caps0;
            uint32_t* inv = L + caps0;
            const uint32_t icap_guard = caps0;
            dswap(
                t, L, M, sh.cnt_old[k], nd,
                [&](uint32_t j) -> uint32_t {
                    const uint32_t s = X.del_slot[j];
                    if (!(s != NONE32 && s < d0 && ((pairs[s].y >> k) & 1u))) return NONE32;
                    const uint32_t sp = Sinv[s];
                    return sp < caps0 ? inv[sp] : NONE32;
                },
                [&](uint32_t val, uint32_t, uint32_t to) { if (val < icap_guard) inv[val] = to; }, X.holes, X.surv, G.pool.status);
        }
        nsp_after_del = dswap(
            t, S, nullptr, h0.nsp, nd,
            [&](uint32_t j) -> uint32_t {
                const uint32_t s = X.del_slot[j];
                return (s != NONE32 && s < d0 && (pairs[s].y & SPo)) ? Sinv[s] : NONE32;
            },
            [&](uint32_t e, uint32_t from, uint32_t to) {
                if (e >= capa0) { atomicOr(G.pool.status, ST_STATE); return; }
                Sinv[e] = to;
                const uint32_t w = pairs[e].y & SPn;
                for (uint32_t b = w; b; b &= b - 1) {
                    const uint32_t k = __ffs(b) - 1;
                    uint32_t* L = G.pool.base + words_of(sh.gref_old[k]) + caps0;
                    uint32_t* inv = L + caps0;
                    const uint32_t mpos = inv[from];
                    if (mpos < caps0) {
                        L[mpos] = to;
                        inv[to] = mpos;
                    } else {
                        atomicOr(G.pool.status, ST_STATE);
                    }
                }
            },
            X.holes, X.surv, G.pool.status);
    }

    // ---- S8: compact the adjacency: surviving edges of the tail [d1, dtot) fill the holes below d1
    for (uint32_t i = rank; i < ni; i += T) X.ins_final[i] = (eids[d0 + i] & DEAD_BIT) ? NONE32 : d0 + i;
    t.sync();
    if (found) {
        uint32_t nh = 0, ns = 0;
        for (uint32_t b = 0; b < nd; b += T) {
            const uint32_t j = b + rank;
            const uint32_t s = j < nd ? X.del_slot[j] : NONE32;
            const bool pred = s != NONE32 && s < d1;
            uint32_t tot;
            const uint32_t r = t.scan_pred(pred, tot);
            if (pred) X.holes[nh + r] = s;
            nh += tot;
        }
        for (uint32_t b = d1; b < dtot; b += T) {
            const uint32_t q = b + rank;
            const bool pred = q < dtot && !(eids[q] & DEAD_BIT);
            uint32_t tot;
            const uint32_t r = t.scan_pred(pred, tot);
            if (pred) X.surv[ns + r] = q;
            ns += tot;
        }
        t.sync();
        uint32_t* S = h0.sref ? G.pool.base + h0.sref : nullptr;
        uint32_t* Sinv = S ? S + capa0 : nullptr;
        for (uint32_t b = 0; b < nh; b += T) {
            const uint32_t r = b + rank;
            if (r < nh) {
                const uint32_t q = X.holes[r], p = X.surv[r];
                const uint2 e = pairs[p];
                pairs[q] = e;
                eids[q] = eids[p];
                if (qbytes) qbytes[q] = qbytes[p];
                if (p < d0) {
                    for (uint32_t bb = e.y & REGk; bb; bb &= bb - 1) {
                        const uint32_t k = __ffs(bb) - 1;
                        uint32_t* L = G.pool.base + words_of(sh.gref_old[k]) + capa0;
                        uint32_t* inv = L + capa0;
                        const uint32_t mpos = inv[p];
                        if (mpos < capa0) {
                            L[mpos] = q;
                            inv[q] = mpos;
                        } else {
                            atomicOr(G.pool.status, ST_STATE);
                        }
                    }
                    if (keepS && (e.y & SPn)) {
                        const uint32_t sp = Sinv[p];
                        if (sp < capa0) {
                            S[sp] = q;
                            Sinv[q] = sp;
                        } else {
                            atomicOr(G.pool.status, ST_STATE);
                        }
                    }
                } else {
                    X.ins_final[p - d0] = q;
                }
            }
        }
        t.sync();
    }

    // ---- S9: append surviving new edges to the groups kept in place
    for (uint32_t m = REGk & REGn; m; m &= m - 1) {
        const uint32_t k = __ffs(m) - 1;
        uint32_t* M = G.pool.base + words_of(sh.gref_old[k]);
        uint32_t* L = M + capa0;
        uint32_t* inv = L + capa0;
        uint32_t pos = sh.cnt_old[k] - sh.removed[k];
        for (uint32_t b = 0; b < ni; b += T) {
            const uint32_t i = b + rank;
            const uint32_t s = i < ni ? X.ins_final[i] : NONE32;
            const bool pred = s != NONE32 && ((pairs[s].y >> k) & 1u);
            uint32_t tot;
            const uint32_t r = t.scan_pred(pred, tot);
            if (pred) {
                L[pos + r] = s;
                inv[s] = pos + r;
                M[pos + r] = pairs[s].x;
            }
            pos += tot;
        }
    }
    if (keepS) {
        uint32_t* S = G.pool.base + h0.sref;
        uint32_t* Sinv = S + capa0;
        uint32_t pos = nsp_after_del;
        for (uint32_t b = 0; b < ni; b += T) {
            const uint32_t i = b + rank;
            const uint32_t s = i < ni ? X.ins_final[i] : NONE32;
            const bool pred = s != NONE32 && (pairs[s].y & SPn);
            uint32_t tot;
            const uint32_t r = t.scan_pred(pred, tot);
            if (pred) {
                S[pos + r] = s;
                Sinv[s] = pos + r;
            }
            pos += tot;
        }
        t.sync();
        for (uint32_t m = SPn; m; m &= m - 1) {
            const uint32_t k = __ffs(m) - 1;
            uint32_t* M = G.pool.base + words_of(sh.gref_old[k]);
            uint32_t* L = M + caps0;
            uint32_t* inv = L + caps0;
            uint32_t gpos = sh.cnt_old[k] - sh.removed[k];
            for (uint32_t b = 0; b < ni; b += T) {
                const uint32_t i = b + rank;
                const uint32_t s = i < ni ? X.ins_final[i] : NONE32;
                const bool pred = s != NONE32 && ((pairs[s].y >> k) & 1u);
                uint32_t tot;
                const uint32_t r = t.scan_pred(pred, tot);
                if (pred) {
                    const uint32_t sp = Sinv[s];
                    L[gpos + r] = sp;
                    inv[sp] = gpos + r;
                    M[gpos + r] = pairs[s].x;
                }
                gpos += tot;
            }
        }
    }
    t.sync();

    // ---- S10: rebuild groups whose kind changed or whose capacity changed; free the rest
    uint32_t rebuilt = 0;
    // free blocks that are not kept
    if (rank == 0) {
        for (uint32_t m = REGo & ~REGk; m; m &= m - 1) pool_free(G.pool, words_of(sh.gref_old[__ffs(m) - 1]), 4ull * capa0);
        if (!keepS && h0.sref) {
            pool_free(G.pool, h0.sref, 2ull * capa0);
            for (uint32_t m = SPo; m; m &= m - 1) pool_free(G.pool, words_of(sh.gref_old[__ffs(m) - 1]), 4ull * caps0);
        }
    }
    for (int k = rank; k < 32; k += T) {
        const uint32_t bit = 1u << k;
        if (REAL && k == (int)DEC_SLOT) continue;  // the decimal block stays with the adjacency
        if (!(maskn & bit) || (!(REGn & bit) && !(SPn & bit) && !(ONEn & bit))) sh.gref_new[k] = 0;  // dense / empty
    }
    t.sync();
    for (uint32_t m = REGn & ~REGk; m; m &= m - 1) {
        const uint32_t k = __ffs(m) - 1;
        if (rank == 0) sh.alloc_off = pool_alloc(G.pool, 4ull * capa1);
        t.sync();
        const uint64_t off = sh.alloc_off;
        if (off) build_regular(t, G, adj, d1, k, off, capa1);
        if (rank == 0) sh.gref_new[k] = ref_of(off);
        rebuilt++;
        t.sync();
    }
    uint64_t sref1 = keepS ? h0.sref : 0;
    uint32_t caps1 = keepS ? caps0 : 0;
    if (!keepS && SPn) {
        if (rank == 0) sh.alloc_off = pool_alloc(G.pool, 2ull * capa1);
        t.sync();
        sref1 = sh.alloc_off;
        t.sync();
        if (sref1) {
            nsp1 = build_slist(t, G, adj, d1, SPn, sref1, capa1);
            t.sync();
            caps1 = caps_for(nsp1);
            for (uint32_t m = SPn; m; m &= m - 1) {
                const uint32_t k = __ffs(m) - 1;
                if (rank == 0) sh.alloc_off = pool_alloc(G.pool, 4ull * caps1);
                t.sync();
                const uint64_t off = sh.alloc_off;
                if (off) build_sparse(t, G, adj, sref1, nsp1, k, off, caps1);
                if (rank == 0) sh.gref_new[k] = ref_of(off);
                rebuilt++;
                t.sync();
            }
        }
    }
    for (uint32_t m = ONEn & ~ONEk; m; m &= m - 1) {
        const uint32_t k = __ffs(m) - 1;
        const uint32_t s = find_one(t, G, adj, d1, k);
        if (rank == 0) sh.gref_new[k] = s < d1 ? pairs[s].x : NONE32;  // one-element: the member's destination
        rebuilt++;
    }
    t.sync();

    // ---- S11-S12: write back, stats
    VHdr h1;
    h1.adj = adj;
    h1.deg = d1;
    h1.mask = maskn;
    h1.sref = SPn ? sref1 : 0;
    h1.nsp = SPn ? nsp1 : 0;
    h1.lcapa = capa1 ? (uint8_t)(log2_u32(capa1) + 1) : 0;
    h1.lcaps = SPn ? (uint8_t)(log2_u32(caps1) + 1) : 0;
    h1.pad = 0;
    h1.word = h0.word;
    write_back<REAL>(t, G, sh, v, h1, d0, ni, nd, found, rebuilt, stats);
}

// A segment whose groups are all dense or empty before it and stay so whatever its deletions find
// (k_seg_classify proves it from the counts, the degree range and the inserted bits; integer
// graphs only): no member list, sparse list or one-element reference exists before or after, so
// apply_segment reduces to the adjacency (capacity, append, resolution, compaction) and the counts.
// The same steps in the same order as apply_segment takes for such a segment, so the same result,
// in far less code: most segments of a batch on a graph with wide biases take this path.
template <class Team, class Src>
__device__ void apply_dense_segment(const Team& t, const DevGraph& G, SegSh& sh, uint32_t v, uint32_t ni, uint32_t nd,
                                    Src B, const SegScratch& X, unsigned long long* stats, uint32_t* sdel_buf,
                                    uint32_t sdel_cap, uint32_t* cand_buf, uint32_t cand_cap, PreCand pre) {
    const uint32_t rank = t.rank(), T = t.size();
    const VHdr h0 = load_hdr(G, v);
    const uint32_t d0 = h0.deg, capa0 = capa_of(h0);
    const uint32_t dtot = d0 + ni;
    for (uint32_t k = rank; k < 32; k += T) {
        sh.cnt_old[k] = grp(G, v, k).x;  // dense and empty groups carry no reference
        sh.gref_new[k] = 0;
        sh.delta[k] = 0;
    }
    // S1: adjacency capacity for the insertions
    uint32_t capa1 = capa0;
    uint64_t adj = h0.adj;
    if (dtot > capa0) {
        capa1 = capa_for(dtot);
        if (rank == 0) sh.alloc_off = pool_alloc(G.pool, 4ull * capa1);
        t.sync();
        const uint64_t noff = sh.alloc_off;
        if (noff == 0) return;  // pool exhausted (flagged); the pre-check makes this unreachable
        if (d0) {
            const uint2* op = adj_pairs(G, h0.adj);
            const uint64_t* oe = adj_eids(G, h0.adj, capa0);
            uint2* np = adj_pairs(G, noff);
            uint64_t* ne = adj_eids(G, noff, capa1);
            for (uint32_t j = rank; j < d0; j += T) {
                np[j] = op[j];
                ne[j] = oe[j];
            }
        }
        t.sync();
        if (rank == 0 && capa0) pool_free(G.pool, h0.adj, 4ull * capa0);
        adj = noff;
    }
    uint2* pairs = adj_pairs(G, adj);
    uint64_t* eids = adj_eids(G, adj, capa1);
    // S2: append insertions at slots d0 .. d0+ni-1
    for (uint32_t i = rank; i < ni; i += T) {
        const uint4 u = B.ins(i);
        pairs[d0 + i] = make_uint2(u.y, u.z);
        eids[d0 + i] = B.ins_eid(i);
    }
    for (uint32_t j = rank; j < nd; j += T) {
        X.del_slot[j] = NONE32;
        X.best[j] = INF64;
    }
    t.sync();
    // S3: resolution
    const uint32_t found = resolve_deletions(t, B, X, pairs, eids, d0, ni, nd, sdel_buf, sdel_cap, cand_buf, cand_cap, pre);
    const uint32_t d1 = dtot - found;
    // S4: count deltas from the bits of deleted pre-existing and surviving new edges
    for (uint32_t j = rank; j < nd; j += T) {
        const uint32_t s = X.del_slot[j];
        if (s != NONE32 && s < d0)
            for (uint32_t b = pairs[s].y; b; b &= b - 1) atomicAdd(&sh.delta[__ffs(b) - 1], -1);
    }
    for (uint32_t i = rank; i < ni; i += T)
        if (!(eids[d0 + i] & DEAD_BIT))
            for (uint32_t b = pairs[d0 + i].y; b; b &= b - 1) atomicAdd(&sh.delta[__ffs(b) - 1], 1);
    t.sync();
    for (uint32_t k = rank; k < 32; k += T) sh.cnt_new[k] = (uint32_t)((int32_t)sh.cnt_old[k] + sh.delta[k]);
    t.sync();
    const KindMasks kmn = kind_masks<false>(t, sh, sh.cnt_new, d1, G, 1);
    if ((kmn.sp | kmn.reg | kmn.one) && rank == 0) atomicOr(G.pool.status, ST_STATE);  // the classification was wrong
    // S8: compact the adjacency: surviving edges of the tail [d1, dtot) fill the holes below d1
    if (found) {
        uint32_t nh = 0, ns = 0;
        for (uint32_t b = 0; b < nd; b += T) {
            const uint32_t j = b + rank;
            const uint32_t s = j < nd ? X.del_slot[j] : NONE32;
            const bool pred = s != NONE32 && s < d1;
            uint32_t tot;
            const uint32_t r = t.scan_pred(pred, tot);
            if (pred) X.holes[nh + r] = s;
            nh += tot;
        }
        for (uint32_t b = d1; b < dtot; b += T) {
            const uint32_t q = b + rank;
            const bool pred = q < dtot && !(eids[q] & DEAD_BIT);
            uint32_t tot;
            const uint32_t r = t.scan_pred(pred, tot);
            if (pred) X.surv[ns + r] = q;
            ns += tot;
        }
        t.sync();
        for (uint32_t b = 0; b < nh; b += T) {
            const uint32_t r = b + rank;
            if (r < nh) {
                const uint32_t q = X.holes[r], p = X.surv[r];
                pairs[q] = pairs[p];
                eids[q] = eids[p];
            }
        }
        t.sync();
    }
    // S11-S12
    VHdr h1;
    h1.adj = adj;
    h1.deg = d1;
    h1.mask = kmn.nonempty;
    h1.sref = 0;
    h1.nsp = 0;
    h1.lcapa = capa1 ? (uint8_t)(log2_u32(capa1) + 1) : 0;
    h1.lcaps = 0;
    h1.pad = 0;
    h1.word = h0.word;
    write_back<false>(t, G, sh, v, h1, d0, ni, nd, found, 0u, stats);
}

// ------------------------------------------------------------------------------------------- batch kernels

struct BatchArgs {
    const uint4* ups;
    uint64_t count;                // record capacity (grid size); the live count is *count_dev when set
    const uint64_t* count_dev;
    uint32_t n, max_bits, bn;
    uint32_t dst_n;  // destinations are ids below dst_n (n for a whole graph; the global count for a partition)
    uint32_t fbits;       // real biases (Section 4.3) when nonzero
    double lambda;
    uint64_t* keys;
    uint32_t* vals;
    uint64_t* packed;     // per record: nkeys (low 32) | is_insert (high 32)
    uint64_t* pscan;      // exclusive scan of packed
    uint32_t* status;
    const uint32_t* perm; // caller -> internal vertex ids, or null (identity)
};

__device__ __forceinline__ uint32_t batch_id(const BatchArgs& A, uint32_t v) { return A.perm ? __ldg(A.perm + v) : v; }

__device__ __forceinline__ uint64_t live_count(const BatchArgs& A) { return A.count_dev ? *A.count_dev : A.count; }

__global__ void k_expand(BatchArgs A) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t cnt = live_count(A);
    bool bad = false;
    for (uint64_t i = tid; i < A.count; i += nt) {
        if (i >= cnt) {  // capacity tail: contributes nothing to the scans
            A.packed[i] = 0;
            continue;
        }
        const uint4 u = A.ups[i];
        const bool ins = u.w == BINGO_OP_INSERT || u.w == BINGO_OP_SET_BIAS;
        const bool del = u.w == BINGO_OP_DELETE || u.w == BINGO_OP_SET_BIAS;
        bad |= u.x >= A.n || u.y >= A.dst_n || u.w > 2;
        if (ins && A.fbits) {
            uint32_t I, q;
            bad |= !split_real_bias(u.z, A.lambda, I, q);
        } else if (ins) {
            bad |= u.z == 0 || (A.max_bits < 32 && (u.z >> A.max_bits) != 0);
        }
        A.packed[i] = (uint64_t)(ins ? 1 : 0) + (del ? 1 : 0) + ((uint64_t)(ins ? 1 : 0) << 32);
    }
    if (bad) atomicOr(A.status, ST_INVALID);
}

__global__ void k_make_keys(BatchArgs A) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t cnt = live_count(A);
    for (uint64_t i = tid; i < cnt; i += nt) {
        const uint4 u = A.ups[i];
        if (u.x >= A.n || u.y >= A.dst_n || u.w > 2) continue;
        uint64_t pos = A.pscan[i] & 0xFFFFFFFFull;
        const uint64_t sk = (uint64_t)batch_id(A, u.x) << (A.bn + 1);
        if (u.w == BINGO_OP_INSERT || u.w == BINGO_OP_SET_BIAS) {
            A.keys[pos] = sk;
            A.vals[pos] = (uint32_t)i;
            pos++;
        }
        if (u.w == BINGO_OP_DELETE || u.w == BINGO_OP_SET_BIAS) {
            A.keys[pos] = sk | (1ull << A.bn) | batch_id(A, u.y);
            A.vals[pos] = (uint32_t)i;
        }
    }
}

__global__ void k_key_count(const uint64_t* total, uint64_t* nkeys) { *nkeys = *total & 0xFFFFFFFFull; }

// Segment heads of the sorted keys; for each insertion key, the record it applies in key order
// ({edge id low, dst, factorised bias, edge id bits 32-55 | decimal part << 24}, the edge id from
// the insertion's batch rank), so the per-vertex pass reads its insertions contiguously.
__global__ void k_seg_flags(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t cap,
                            const uint64_t* __restrict__ nkeys_dev, uint32_t bn, const uint4* __restrict__ ups,
                            const uint64_t* __restrict__ pscan, const unsigned long long* __restrict__ eid_base,
                            uint32_t fbits, double lambda, uint32_t base4, const uint32_t* __restrict__ perm,
                            uint64_t* __restrict__ flag, uint4* __restrict__ rec) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t nkeys = nkeys_dev ? *nkeys_dev : cap;
    for (uint64_t i = tid; i < cap; i += nt) {
        const bool live = i < nkeys;
        const uint64_t k = live ? keys[i] : 0;
        flag[i] = live && (i == 0 || (k >> (bn + 1)) != (keys[i - 1] >> (bn + 1))) ? 1 : 0;
        if (rec && live && !((k >> bn) & 1ull)) {
            const uint32_t r = vals[i];
            const uint4 u = ups[r];
            const uint64_t eid = *eid_base + (pscan[r] >> 32);
            uint32_t I = u.z, q = 0;
            if (fbits) split_real_bias(u.z, lambda, I, q);
            if (base4) I = b4_mask(u.z);
            rec[i] = make_uint4((uint32_t)eid, perm ? perm[u.y] : u.y, I, ((uint32_t)(eid >> 32) & 0xFFFFFFu) | (q << 24));
        }
    }
}

__global__ void k_seg_write(const uint64_t* __restrict__ flag, const uint64_t* __restrict__ segid, uint64_t cap,
                            const uint64_t* __restrict__ nkeys_dev, uint32_t* __restrict__ seg_start) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t nkeys = nkeys_dev ? *nkeys_dev : cap;
    for (uint64_t i = tid; i < nkeys; i += nt) {
        if (flag[i]) seg_start[segid[i]] = (uint32_t)i;
        if (i == nkeys - 1) seg_start[segid[i] + flag[i]] = (uint32_t)nkeys;
    }
}

// Worst-case pool words a vertex can allocate when its counts move within [c - nd, c + ni_k] and its
// degree within [d + ni - nd, d + ni]: a new adjacency block if it grows, one group block (4 * capA
// words) for every group that can reach a list kind (Eq. group) other than its current kind, the
// blocks of every group that can be sparse when the set of sparse groups can change (they are
// rebuilt together), and a sparse list.
// The 32 group counts of vertex v, read as whole 16-byte pairs with every load in flight at once.
__device__ __forceinline__ void load_counts(const DevGraph& G, uint32_t v, uint32_t* cnt) {
    const uint4* cold = reinterpret_cast<const uint4*>(G.vc[v].g);
    uint4 x[16];
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = cold[i];
#pragma unroll
    for (int i = 0; i < 16; i++) {
        cnt[2 * i] = x[i].x;
        cnt[2 * i + 1] = x[i].z;
    }
}

// dense_only (nullable): set when every group is dense or empty now and can be nothing else after
// (no list kind and no one-element group reachable), on integer graphs with group adaption.
__device__ __forceinline__ unsigned long long pool_bound(const DevGraph& G, uint32_t v, const VHdr& h, uint32_t ni,
                                                         uint32_t nd, uint32_t insbits, bool* dense_only = nullptr) {
    uint32_t cnts[32];
    load_counts(G, v, cnts);
    const uint32_t d0 = h.deg, dmin = d0 + ni >= nd ? d0 + ni - nd : 0, dmax = d0 + ni;
    const bool grows = dmax > capa_of(h);
    const uint32_t capa1 = grows ? capa_for(dmax) : capa_of(h);
    uint32_t nblocks = 0, sp_possible = 0;
    bool sp_set_may_change = false, any_old_sp = false;
    const uint32_t nslots = G.fbits ? DEC_SLOT : 32u;  // the decimal slot is never a list
    bool dense = G.fbits == 0 && G.alpha != ALL_REGULAR;
    for (uint32_t k = 0; k < nslots; k++) {
        const uint32_t c = cnts[k];
        const uint32_t cmax = c + (((insbits >> k) & 1u) ? ni : 0u), cmin = c > nd ? c - nd : 0u;
        const uint32_t old = kind_of(c, d0, G.alpha, G.beta);
        if (old != K_EMPTY && old != K_DENSE) dense = false;
        // one-element reachable: a count of 1 at a degree where it is not dense (100 <= alpha d)
        if (cmin <= 1 && cmax >= 1 && 100ull <= (uint64_t)G.alpha * dmax) dense = false;
        const uint32_t min_list = G.alpha == ALL_REGULAR ? 1u : 2u;  // smallest count of a list kind
        if (cmax < min_list) continue;  // can never be a list kind (and is not one now)
        const uint32_t lo2 = cmin > min_list ? cmin : min_list;
        // sparse reachable: the smallest count >= 2 stays below beta% of the largest degree
        const bool can_sp = 100ull * lo2 < (uint64_t)G.beta * dmax;
        // regular reachable: [lo2, cmax] meets [ceil(beta dmin / 100), floor(alpha dmax / 100)]
        const uint64_t rlo = ((uint64_t)G.beta * dmin + 99) / 100, rhi = ((uint64_t)G.alpha * dmax) / 100;
        const bool can_reg = lo2 <= rhi && cmax >= rlo && rlo <= rhi;
        const bool can_dense = 100ull * cmax > (uint64_t)G.alpha * dmin;
        if (can_reg || can_sp) dense = false;
        if ((can_reg && (old != K_REGULAR || grows)) || (can_sp && (old != K_SPARSE || grows))) nblocks++;
        if (can_sp) sp_possible++;
        if (old == K_SPARSE) {
            any_old_sp = true;
            if (cmin <= 1 || can_reg || can_dense) sp_set_may_change = true;  // may leave the sparse set
        } else if (can_sp) {
            sp_set_may_change = true;  // may join it
        }
    }
    // the sparse list and all sparse groups are rebuilt together when the set changes, the adjacency
    // grows, or insertions may outgrow the sparse capacity
    const bool sp_rebuild = sp_set_may_change || grows || (ni > 0 && any_old_sp);
    unsigned long long words = grows ? 4ull * capa1 + (G.fbits ? dec_words(capa1) : 0ull) : 0ull;
    words += 4ull * capa1 * nblocks;
    if (sp_possible && sp_rebuild) words += 2ull * capa1 + 4ull * capa1 * sp_possible;
    if (dense_only) *dense_only = dense;
    return words;
}

struct SegArgs {
    BatchArgs B;
    const uint64_t* sorted_keys;
    const uint32_t* sorted_vals;
    const uint32_t* seg_start;
    const uint64_t* nseg_dev;
    uint32_t* small_list;
    uint32_t* big_list;
    uint32_t* dense_flag;         // [segment] 1: a small dense-only segment (k_apply_dense)
    unsigned long long* ndense;   // [0] count, [1] k_apply_dense work queue
    unsigned long long* counts;   // [0] small, [1] big, [2] pool bound
    unsigned long long* queue;    // [0] next small segment, [1] next big segment (k_apply work queues)
    uint32_t big_slots;           // segments above this many adjacency slots run on a block team
    uint4* rec;                   // per key: the insertion record {edge id low, dst, bias, edge id high}
    uint4* seginfo;               // per segment: {v, first key, ni, nd}
    uint32_t* gcand;              // big segments: deletion candidates from the pre-pass, region PRE_MULT * (first
                                  // deletion key) .. + PRE_MULT * nd
    uint32_t* gcand_cnt;          // per segment: candidates found (may exceed the region: then unused);
                                  // NO_PRE for segments the pre-pass does not scan
    uint32_t* huge_list;          // segments scanned by the pre-pass
    unsigned long long* nhuge;
    uint32_t* huge_coff;          // [nhuge + 1] first pre-pass chunk of each listed segment (k_cand_plan)
    uint32_t* huge_nch;           // [nhuge] pre-pass chunks of each listed segment (k_seg_classify)
    uint32_t* chunk_seg;          // [chunk_cap] listed segment of each pre-pass chunk (k_cand_plan)
    uint32_t chunk_cap;
    uint64_t eid_base;
    const unsigned long long* eid_base_dev;  // when set, the edge-id base is read on the device
    uint32_t* holes;
    uint32_t* surv;
    uint32_t* slot_scratch;
    unsigned long long* best;
    unsigned long long* stats;
};

// Per segment: insertion count, and the worst-case pool words the segment may allocate.
__global__ void k_seg_classify(DevGraph G, SegArgs S) {
    if (*G.pool.status & ST_STOP) return;  // an invalid batch may carry ids >= n
    const uint64_t nseg = *S.nseg_dev;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long bound = 0;
    for (uint64_t sidx = tid; sidx < nseg; sidx += nt) {
        S.dense_flag[sidx] = 0u;
        const uint32_t a = S.seg_start[sidx], b = S.seg_start[sidx + 1];
        const uint32_t v = (uint32_t)(S.sorted_keys[a] >> (S.B.bn + 1));
        if (v >= G.n) { atomicOr(G.pool.status, ST_INVALID); continue; }
        uint32_t lo = a, hi = b;  // first deletion key
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if ((S.sorted_keys[mid] >> S.B.bn) & 1ull) hi = mid; else lo = mid + 1;
        }
        const uint32_t ni = lo - a;
        S.seginfo[sidx] = make_uint4(v, a, ni, b - lo);
        const VHdr h = load_hdr(G, v);
        const uint32_t dtot = h.deg + ni;
        if (G.fbits && dtot >= REAL_MAX_DEG) { atomicOr(G.pool.status, ST_INVALID); continue; }
        uint32_t insbits = 0;
        for (uint32_t i = a; i < lo; i++) insbits |= S.rec[i].z;
        bool dense_only = false;
        bound += pool_bound(G, v, h, ni, b - lo, insbits, &dense_only);
        const bool big = dtot > S.big_slots || (b - a) > 256;
        if (!big && dense_only) S.dense_flag[sidx] = 1u;
        const bool huge = h.deg >= PRE_MIN_DEG && b > lo;  // deletions at a large vertex: grid-wide candidate scan
        S.gcand_cnt[sidx] = huge ? 0u : NO_PRE;
        if (huge) {
            const unsigned long long pos = atomicAdd(S.nhuge, 1ull);
            S.huge_list[pos] = (uint32_t)sidx;
            S.huge_nch[pos] = (h.deg + PRE_CHUNK - 1) / PRE_CHUNK;
        }
        if (big) S.big_list[atomicAdd(&S.counts[1], 1ull)] = (uint32_t)sidx;
        else if (dense_only) atomicAdd(S.ndense, 1ull);
        else S.small_list[atomicAdd(&S.counts[0], 1ull)] = (uint32_t)sidx;
    }
    if (bound) atomicAdd(&S.counts[2], bound);
}

__global__ void k_oom_check(DevGraph G, const unsigned long long* counts, unsigned long long* queue) {
    const unsigned long long top = *G.pool.top;
    if (top + counts[2] > G.pool.words) atomicOr(G.pool.status, ST_OOM);
    queue[0] = 0;
    queue[1] = 0;
}

// Grid-wide pre-pass: for every segment with deletions at a vertex of at least PRE_MIN_DEG edges, the
// pre-existing slots [0, d0) whose destination is deleted in the segment, found by the whole grid at
// once instead of by the segment's single team (an O(d) scan per touched large vertex).  The work is
// flattened into chunks of PRE_CHUNK slots over all listed segments (k_cand_plan numbers them), so
// every block takes chunks of any segment and no segment is a serial step.  Candidate order is
// irrelevant: resolution takes minima of edge ids.
__global__ void __launch_bounds__(1024) k_cand_plan(DevGraph G, SegArgs S) {
    __shared__ uint32_t sm[64];
    if (*(volatile uint32_t*)G.pool.status & ST_STOP) return;
    const uint64_t nhuge = *S.nhuge;
    uint32_t base = 0;
    for (uint64_t t0 = 0; t0 < nhuge; t0 += blockDim.x) {
        const uint64_t i = t0 + threadIdx.x;
        const uint32_t c = i < nhuge ? S.huge_nch[i] : 0u;
        const uint2 r = block_scan_excl(sm, c);
        if (i < nhuge) S.huge_coff[i] = base + r.x;
        base += r.y;
    }
    if (threadIdx.x == 0) S.huge_coff[nhuge] = base;
    // chunk -> segment map (when it fits; k_cand_scan searches the offsets otherwise)
    if (base > S.chunk_cap) return;
    __syncthreads();
    for (uint64_t i = threadIdx.x; i < nhuge; i += blockDim.x) {
        const uint32_t c0 = S.huge_coff[i], c1 = c0 + S.huge_nch[i];
        for (uint32_t c = c0; c < c1; c++) S.chunk_seg[c] = (uint32_t)i;
    }
}

constexpr uint32_t PRE_SDEL = 2048;  // deletion destinations of a chunk's segment staged in shared memory
__global__ void __launch_bounds__(256) k_cand_scan(DevGraph G, SegArgs S) {
    __shared__ uint32_t sdk[PRE_SDEL];
    if (*(volatile uint32_t*)G.pool.status & ST_STOP) return;  // block-uniform
    const unsigned long long nhuge = *S.nhuge;
    if (nhuge == 0) return;
    const uint32_t total = S.huge_coff[nhuge];
    const bool mapped = total <= S.chunk_cap;
    const uint64_t dmask = (1ull << S.B.bn) - 1;
    for (uint32_t c = blockIdx.x; c < total; c += gridDim.x) {
        uint32_t lo = 0;  // the listed segment holding chunk c: the last whose first chunk is <= c
        if (mapped) {
            lo = S.chunk_seg[c];
        } else {
            uint32_t hi = (uint32_t)nhuge;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (S.huge_coff[mid] <= c) lo = mid; else hi = mid;
            }
        }
        const uint32_t sidx = S.huge_list[lo];
        const uint4 info = S.seginfo[sidx];
        const uint32_t nd = info.w, v = info.x, first = info.y + info.z;
        const VHdr h = load_hdr(G, v);
        const uint32_t d0 = h.deg;
        const uint2* pairs = adj_pairs(G, h.adj);
        const uint64_t* dk = S.sorted_keys + first;  // the segment's deletion keys, ascending destination
        uint32_t* out = S.gcand + (uint64_t)PRE_MULT * first;
        const uint32_t cap = PRE_MULT * nd;
        const uint32_t c0 = (c - S.huge_coff[lo]) * PRE_CHUNK;
        uint32_t x[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint32_t j = c0 + q * 256 + threadIdx.x;
            x[q] = j < d0 ? pairs[j].x : NONE32;
        }
        const bool staged = nd <= PRE_SDEL;
        __syncthreads();  // the previous chunk's searches are done with sdk
        if (staged)
            for (uint32_t j = threadIdx.x; j < nd; j += blockDim.x) sdk[j] = (uint32_t)(__ldg(dk + j) & dmask);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint32_t j = c0 + q * 256 + threadIdx.x;
            if (j >= d0) continue;
            uint32_t a = 0, b = nd;
            while (a < b) {
                const uint32_t mid = (a + b) >> 1;
                const uint32_t y = staged ? sdk[mid] : (uint32_t)(__ldg(dk + mid) & dmask);
                if (y < x[q]) a = mid + 1; else b = mid;
            }
            if (a < nd && (staged ? sdk[a] : (uint32_t)(__ldg(dk + a) & dmask)) == x[q]) {
                const uint32_t pos = atomicAdd(S.gcand_cnt + sidx, 1u);
                if (pos < cap) out[pos] = j;
            }
        }
    }
}

// Per-team scratch in shared memory for segments of at most SMALL_X insertions and deletions, so the
// per-deletion and per-slot lists between phases stay on the SM instead of round-tripping to L2.
constexpr uint32_t SMALL_X = 32;
struct SmallScratch {
    uint32_t holes[SMALL_X], surv[SMALL_X], ins_final[SMALL_X], del_slot[SMALL_X];
    unsigned long long best[SMALL_X];
};

template <bool REAL, class Team>
__device__ __forceinline__ void run_segment(const Team& t, const DevGraph& G, const SegArgs& S, SegSh& sh, uint32_t sidx,
                                            uint32_t* sdel_buf, uint32_t sdel_cap, uint32_t* cand_buf,
                                            uint32_t cand_cap, SmallScratch* sx = nullptr,
                                            unsigned long long* stats = nullptr, bool pre_scanned = false,
                                            bool dense_only = false) {
    const uint4 info = S.seginfo[sidx];
    const uint32_t v = info.x, a = info.y, ni = info.z, nd = info.w;
    BatchSrc src;
    src.rec = S.rec;
    src.keys = S.sorted_keys;
    src.dmask = (1ull << S.B.bn) - 1;
    src.start = a;
    src.ni = ni;
    SegScratch X;
    if (sx && ni <= SMALL_X && nd <= SMALL_X) {
        X.holes = sx->holes;
        X.surv = sx->surv;
        X.ins_final = sx->ins_final;
        X.del_slot = sx->del_slot;
        X.best = sx->best;
    } else {
        X.holes = S.holes + a;
        X.surv = S.surv + a;
        X.ins_final = S.slot_scratch + a;
        X.del_slot = S.slot_scratch + a + ni;
        X.best = S.best + a + ni;
    }
    src.sdel = nullptr;
    PreCand pre;
    if (pre_scanned && nd && S.gcand_cnt[sidx] != NO_PRE) {
        pre.list = S.gcand + (uint64_t)PRE_MULT * (a + ni);
        pre.count = S.gcand_cnt[sidx];
        pre.cap = PRE_MULT * nd;
    }
    if (!REAL && dense_only)
        apply_dense_segment(t, G, sh, v, ni, nd, src, X, stats ? stats : S.stats, sdel_buf, sdel_cap, cand_buf, cand_cap,
                            pre);
    else
        apply_segment<REAL>(t, G, sh, v, ni, nd, src, X, stats ? stats : S.stats, sdel_buf, sdel_cap, cand_buf,
                            cand_cap, pre);
    // the edge-index pass (k_eh_apply) reads from the batch scratch which deletions found an edge
    if (G.eh_mask && X.del_slot != S.slot_scratch + a + ni)
        for (uint32_t j = t.rank(); j < nd; j += t.size()) S.slot_scratch[a + ni + j] = X.del_slot[j];
}

constexpr uint32_t DEFAULT_UPDATE_CHUNK = 4096;  // best of 1,024 .. 16,384 on RMAT-20 with 10^5-update batches
constexpr uint32_t SMALL_SDEL = 64;    // staged deletion destinations per warp team
constexpr uint32_t SMALL_CAND = 64;    // resolution candidates per warp team
constexpr uint32_t BIG_SDEL = 4096;    // per block team
constexpr uint32_t BIG_CAND = 4096;
constexpr uint32_t APPLY_THREADS = 512;
constexpr uint32_t APPLY_TEAMS = APPLY_THREADS / 32;

// One persistent launch for every segment (grid = resident blocks).  Each block first takes big
// segments, one at a time as a 512-thread team, from a shared queue (they are the long poles, so
// they start first); when that queue is empty its 16 warps become warp teams that pull small
// segments one by one, so no warp idles while work is left.
struct BigShared {
    SegSh sh;
    uint32_t sdel[BIG_SDEL];
    uint32_t cand[BIG_CAND];
};
struct SmallShared {
    SegSh sh[APPLY_TEAMS];
    uint32_t sdel[APPLY_TEAMS][SMALL_SDEL];
    uint32_t cand[APPLY_TEAMS][SMALL_CAND];
    SmallScratch x[APPLY_TEAMS];
};
union ApplyShared {
    BigShared big;
    SmallShared small;
};

template <bool REAL>
__global__ void __launch_bounds__(APPLY_THREADS, 2) k_apply(DevGraph G, SegArgs S) {
    __shared__ ApplyShared smem;
    __shared__ unsigned long long next;
    __shared__ unsigned long long bstats[S_CONV + 25];  // block totals, added to the batch's once at the end
    for (uint32_t i = threadIdx.x; i < S_CONV + 25; i += blockDim.x) bstats[i] = 0;
    const unsigned long long nbig = S.counts[1], nsmall = S.counts[0];
    {
        BlockTeam t;
        t.sm = smem.big.sh.tscratch;
        for (;;) {
            if (threadIdx.x == 0)
                next = (*(volatile uint32_t*)G.pool.status & ST_STOP) ? nbig : atomicAdd(S.queue + 1, 1ull);
            __syncthreads();
            const unsigned long long i = next;
            __syncthreads();
            if (i >= nbig) break;
            run_segment<REAL>(t, G, S, smem.big.sh, S.big_list[i], smem.big.sdel, BIG_SDEL, smem.big.cand, BIG_CAND, nullptr,
                        bstats, true);
        }
    }
    __syncthreads();  // shared memory changes from the big-segment to the warp-team layout
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTeam t;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0)
            i = (*(volatile uint32_t*)G.pool.status & ST_STOP) ? nsmall : atomicAdd(S.queue, 1ull);
        i = __shfl_sync(FULL, i, 0);
        if (i >= nsmall) break;
        run_segment<REAL>(t, G, S, smem.small.sh[w], S.small_list[i], smem.small.sdel[w], SMALL_SDEL, smem.small.cand[w],
                          SMALL_CAND, &smem.small.x[w], bstats, true);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < S_CONV + 25; i += blockDim.x)
        if (bstats[i]) atomicAdd(S.stats + i, bstats[i]);
}

// The small dense-only segments (integer graphs), after k_apply: the same warp teams and queue,
// on apply_dense_segment alone.  k_apply is bound by instruction fetch, and a launch that runs one
// short procedure on every SM keeps it in the instruction cache, where sharing k_apply's warps with
// the general procedure slowed both.
__global__ void __launch_bounds__(APPLY_THREADS, 2) k_apply_dense(DevGraph G, SegArgs S) {
    __shared__ SmallShared smem;
    __shared__ unsigned long long bstats[S_CONV + 25];
    for (uint32_t i = threadIdx.x; i < S_CONV + 25; i += blockDim.x) bstats[i] = 0;
    __syncthreads();
    // segments in their sorted order, which under the degree numbering puts the largest vertices
    // (the longest segments) first, so the launch does not end on a few long ones
    const unsigned long long n = S.ndense[0] ? *S.nseg_dev : 0ull;
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTeam t;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = (*(volatile uint32_t*)G.pool.status & ST_STOP) ? n : atomicAdd(S.ndense + 1, 1ull);
        i = __shfl_sync(FULL, i, 0);
        if (i >= n) break;
        if (!S.dense_flag[i]) continue;
        run_segment<false>(t, G, S, smem.sh[w], (uint32_t)i, smem.sdel[w], SMALL_SDEL, smem.cand[w], SMALL_CAND,
                           &smem.x[w], bstats, true, true);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < S_CONV + 25; i += blockDim.x)
        if (bstats[i]) atomicAdd(S.stats + i, bstats[i]);
}

// edge-index maintenance: +1 for every insertion record, -1 for every deletion that found an edge
__global__ void k_eh_apply(DevGraph G, SegArgs S, uint64_t cap, const uint64_t* nkeys_dev) {
    if (*G.pool.status & ST_STOP) return;
    const uint64_t nkeys = nkeys_dev ? *nkeys_dev : cap;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = tid; i < nkeys; i += nt) {
        const uint64_t key = S.sorted_keys[i];
        const bool del = (key >> S.B.bn) & 1ull;
        const uint32_t src = (uint32_t)(key >> (S.B.bn + 1));
        const uint4 u = S.B.ups[S.sorted_vals[i]];
        if (del && S.slot_scratch[i] == NONE32) continue;
        const unsigned long long k = ((unsigned long long)src << 32) | to_internal(G, u.y);
        uint64_t p = eh_hash(k) & G.eh_mask;
        for (uint64_t probe = 0; probe <= G.eh_mask; probe++) {
            if (!del) {
                const unsigned long long old = atomicCAS(G.eh_key + p, EH_EMPTY, k);
                if (old == EH_EMPTY || old == k) { atomicAdd(G.eh_cnt + p, 1u); break; }
            } else {
                const unsigned long long cur = G.eh_key[p];
                if (cur == k) { atomicSub(G.eh_cnt + p, 1u); break; }
                if (cur == EH_EMPTY) break;
            }
            p = (p + 1) & G.eh_mask;
        }
    }
}

// Make this batch's frees reusable: the free stacks' counts (a class's count goes negative while
// pops outrun its stack) are reset to zero, every pending block is pushed, and the counts clamped.
// The pushes run grid-wide with one atomic per size class and warp (warp-aggregated).
__global__ void k_pool_open(DevGraph G) {
    Pool P = G.pool;
    for (int c = threadIdx.x; c < NCLASS; c += blockDim.x)
        if (P.fcount[c] < 0) P.fcount[c] = 0;
}
__global__ void __launch_bounds__(256) k_pool_push(DevGraph G) {
    Pool P = G.pool;
    const unsigned long long np = *P.npending;
    const unsigned long long lim = np < P.pcap ? np : P.pcap;
    const uint32_t lane = threadIdx.x & 31;
    const unsigned long long nt = (unsigned long long)gridDim.x * blockDim.x;
    // every lane of a warp runs the same trips, so the warp stays converged for match and shuffle
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < lim; b += nt) {
        const unsigned long long i = b + lane;
        const bool live = i < lim;
        const uint64_t x = live ? P.pending[i] : 0ull;
        const uint32_t c = live ? (uint32_t)(x & 0xFF) : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(FULL, c);
        const uint32_t leader = __ffs(peers) - 1;
        unsigned long long base = 0;
        if (live && lane == leader)
            base = atomicAdd(reinterpret_cast<unsigned long long*>(&P.fcount[c]), (unsigned long long)__popc(peers));
        base = __shfl_sync(FULL, base, leader);
        if (live) {
            const uint64_t idx = base + __popc(peers & lanemask_lt());
            if (idx < P.fcap) P.fstack[(uint64_t)c * P.fcap + idx] = x >> 8;
            else atomicAdd(P.leaked, (unsigned long long)(8ull << c));
        }
    }
}
__global__ void k_pool_close(DevGraph G) {
    Pool P = G.pool;
    for (int c = threadIdx.x; c < NCLASS; c += blockDim.x)
        if ((uint64_t)P.fcount[c] > P.fcap) P.fcount[c] = (long long)P.fcap;
    if (threadIdx.x == 0) *P.npending = 0;
}

// Streaming (Section 4.2): every record is applied as a batch of one, in record order.  Records of
// different source vertices touch disjoint state and edge ids are fixed by record position, so the
// records are grouped by source (stable sort) and one team applies each vertex's records in order
// while vertices proceed in parallel: the result equals strict one-at-a-time application.  A warp
// applies the records of a vertex with fewer than STREAM_BIG_DEG edges; larger vertices (whose
// deletions scan the whole adjacency) are listed and applied afterwards by a 512-thread block each.
constexpr uint32_t STREAM_TEAMS = 16;
constexpr uint32_t STREAM_BIG_DEG = 4096;
constexpr uint32_t STREAM_BIG_THREADS = 512;
constexpr uint32_t STREAM_BIG_CAND = 4096;
struct StreamScratch {
    uint32_t holes[2], surv[2], ins_final[2], del_slot[2];
    unsigned long long best[2];
};

// Apply record r of the sorted stream with team t.  Returns false when processing must stop (pool
// exhausted or an invalid record; the status says which).
template <bool REAL, class Team>
__device__ bool stream_record(const Team& t, const DevGraph& G, const SegArgs& S, SegSh& sh, StreamScratch& xs,
                              uint32_t r, unsigned long long* reserved, uint32_t* cand_buf, uint32_t cand_cap) {
    const bool stop = t.rank() == 0 && (*(volatile uint32_t*)G.pool.status & ST_STOP);
    if (t.any(stop)) return false;  // one reader, so the whole team leaves together
    const uint32_t rec = S.sorted_vals[r];
    uint4 u = S.B.ups[rec];
    u.x = to_internal(G, u.x);
    u.y = to_internal(G, u.y);
    const uint32_t ni = (u.w == BINGO_OP_INSERT || u.w == BINGO_OP_SET_BIAS) ? 1u : 0u;
    const uint32_t nd = (u.w == BINGO_OP_DELETE || u.w == BINGO_OP_SET_BIAS) ? 1u : 0u;
    // reserve this record's worst-case pool growth so no allocation inside it can fail
    uint32_t I = u.z, qd = 0;
    if (REAL && ni) split_real_bias(u.z, G.lambda, I, qd);
    if (G.base4 && ni) I = b4_mask(u.z);
    const VHdr h = load_hdr(G, u.x);
    if (REAL && h.deg + ni >= REAL_MAX_DEG) {
        if (t.rank() == 0) atomicOr(G.pool.status, ST_INVALID);
        return false;
    }
    const unsigned long long need = pool_bound(G, u.x, h, ni, nd, ni ? I : 0u);
    bool fail = false;
    if (t.rank() == 0) {
        const unsigned long long prev = atomicAdd(reserved, need);
        if (*G.pool.top + prev + need > G.pool.words) {
            atomicAdd(reserved, 0ull - need);
            atomicOr(G.pool.status, ST_OOM);
            fail = true;
        }
    }
    if (t.any(fail)) return false;
    OneSrc src;
    src.dst = u.y;
    src.bias = I;
    src.q = qd;
    src.eid = S.eid_base + (S.B.pscan[rec] >> 32);
    SegScratch X;
    X.holes = xs.holes;
    X.surv = xs.surv;
    X.ins_final = xs.ins_final;
    X.del_slot = xs.del_slot;
    X.best = xs.best;
    apply_segment<REAL>(t, G, sh, u.x, ni, nd, src, X, S.stats, nullptr, 0u, cand_buf, cand_cap);
    if (G.eh_mask && t.rank() == 0) {  // edge index: +1 per insertion, -1 per deletion that found an edge
        const unsigned long long k = ((unsigned long long)u.x << 32) | u.y;
        if (ni) {
            uint64_t p = eh_hash(k) & G.eh_mask;
            for (uint64_t probe = 0; probe <= G.eh_mask; probe++) {
                const unsigned long long old = atomicCAS(G.eh_key + p, EH_EMPTY, k);
                if (old == EH_EMPTY || old == k) { atomicAdd(G.eh_cnt + p, 1u); break; }
                p = (p + 1) & G.eh_mask;
            }
        }
        if (nd && X.del_slot[0] != NONE32) {
            uint64_t p = eh_hash(k) & G.eh_mask;
            for (uint64_t probe = 0; probe <= G.eh_mask; probe++) {
                const unsigned long long cur = G.eh_key[p];
                if (cur == k) { atomicSub(G.eh_cnt + p, 1u); break; }
                if (cur == EH_EMPTY) break;
                p = (p + 1) & G.eh_mask;
            }
        }
    }
    if (t.rank() == 0) atomicAdd(reserved, 0ull - need);
    t.sync();
    return true;
}

template <bool REAL>
__global__ void __launch_bounds__(STREAM_TEAMS * 32) k_stream_apply(DevGraph G, SegArgs S, unsigned long long* reserved,
                                                                    uint32_t* big_list, unsigned long long* nbig) {
    __shared__ SegSh sh[STREAM_TEAMS];
    __shared__ StreamScratch xs[STREAM_TEAMS];
    const uint32_t w = threadIdx.x >> 5;
    WarpTeam t;
    const uint64_t nseg = *S.nseg_dev;
    for (uint64_t sidx = (uint64_t)blockIdx.x * STREAM_TEAMS + w; sidx < nseg; sidx += (uint64_t)gridDim.x * STREAM_TEAMS) {
        const uint32_t a = S.seg_start[sidx], b = S.seg_start[sidx + 1];
        // the vertex's degree before its first record decides the team (the block pass runs after)
        const uint32_t v = to_internal(G, S.B.ups[S.sorted_vals[a]].x);
        if (v < G.n && load_hdr(G, v).deg >= STREAM_BIG_DEG) {
            if (t.rank() == 0) big_list[atomicAdd(nbig, 1ull)] = (uint32_t)sidx;
            continue;
        }
        for (uint32_t r = a; r < b; r++)
            if (!stream_record<REAL>(t, G, S, sh[w], xs[w], r, reserved, nullptr, 0u)) return;
    }
}

// The listed large vertices, one 512-thread block team each, their records in order.
template <bool REAL>
__global__ void __launch_bounds__(STREAM_BIG_THREADS) k_stream_apply_big(DevGraph G, SegArgs S, unsigned long long* reserved,
                                                                         const uint32_t* big_list,
                                                                         const unsigned long long* nbig) {
    __shared__ SegSh sh;
    __shared__ StreamScratch xs;
    __shared__ uint32_t cand[STREAM_BIG_CAND];
    BlockTeam t;
    t.sm = sh.tscratch;
    const unsigned long long nb = *nbig;
    for (unsigned long long i = blockIdx.x; i < nb; i += gridDim.x) {
        const uint32_t sidx = big_list[i];
        const uint32_t a = S.seg_start[sidx], b = S.seg_start[sidx + 1];
        for (uint32_t r = a; r < b; r++)
            if (!stream_record<REAL>(t, G, S, sh, xs, r, reserved, cand, STREAM_BIG_CAND)) return;
    }
}

__global__ void k_stream_keys(BatchArgs A) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = tid; i < A.count; i += nt) {
        A.keys[i] = (uint64_t)A.ups[i].x << (A.bn + 1);
        A.vals[i] = (uint32_t)i;
    }
}

uint32_t bits_for(uint32_t n) {
    uint32_t b = 1;
    while (b < 31 && (1u << b) < n) b++;
    return b;
}

bingo_status read_stats(bingo_graph* g, cudaStream_t s, bingo_update_stats* stats, uint32_t* status_out) {
    uint64_t* ctl = (uint64_t*)g->d_ctl;
    uint64_t host[CTL_WORDS];
    CK(cudaMemcpyAsync(host, ctl, sizeof(host), cudaMemcpyDeviceToHost, s), "stats read");
    CK(cudaStreamSynchronize(s), "update");
    *status_out = (uint32_t)host[CTL_STATUS];
    const uint64_t* st = host + CTL_STATS;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->inserted = st[S_INS];
        stats->deleted = st[S_DEL];
        stats->not_found = st[S_NF];
        stats->vertices_touched = st[S_TOUCH];
        stats->groups_rebuilt = st[S_REBUILT];
        for (int a = 0; a < 5; a++)
            for (int b = 0; b < 5; b++) stats->conversions[a][b] = st[S_CONV + a * 5 + b];
    }
    return BINGO_OK;
}

}  // namespace

namespace bingo {
bingo_status edge_index_build(bingo_graph* g, cudaStream_t s);
}

static unsigned grid_cap(const bingo_graph* g, uint64_t items, unsigned block, unsigned per_sm = 16) {
    uint64_t b = (items + block - 1) / block;
    const uint64_t cap = (uint64_t)g->num_sms * per_sm;
    if (b > cap) b = cap;
    return b ? (unsigned)b : 1u;
}

static void launch_pool_merge(bingo_graph* g, cudaStream_t s) {
    k_pool_open<<<1, 64, 0, s>>>(g->G);
    k_pool_push<<<(unsigned)g->num_sms * 4, 256, 0, s>>>(g->G);
    k_pool_close<<<1, 64, 0, s>>>(g->G);
    g->launches += 3;
}

static bingo_status finish_batch(bingo_graph* g, cudaStream_t s, bingo_update_stats* stats, uint64_t inserts_expected,
                                 bool finalize = true) {
    if (finalize) launch_pool_merge(g, s);
    uint32_t status = 0;
    bingo_update_stats tmp;
    bingo_status st = read_stats(g, s, &tmp, &status);
    if (st != BINGO_OK) return st;
    // this call reports its device status through its return value; clear it so that it does not
    // surface again in a later bingo_check
    CK(cudaMemsetAsync((uint64_t*)g->d_ctl + CTL_STATUS, 0, 8, s), "status clear");
    if (stats) *stats = tmp;
    if (status & ST_INVALID) {
        set_error("invalid update record (id >= n, op > 2, or bias outside [1, 2^max_bits)); batch rejected");
        return BINGO_E_INVALID;
    }
    g->next_eid += tmp.inserted;
    g->m_live = g->m_live + tmp.inserted - tmp.deleted;
    (void)inserts_expected;
    if (status & ST_STATE) {
        g->broken = true;
        set_error("update found an inconsistent group structure; the graph is marked unusable");
        return BINGO_E_STATE;
    }
    if (status & ST_OOM) {
        set_error("device pool exhausted; batch rejected before any change");
        return BINGO_E_OOM;
    }
    if (status & ST_TIMEOUT) {
        set_error("a bounded device loop gave up");
        return BINGO_E_TIMEOUT;
    }
    return BINGO_OK;
}

__global__ void k_set_words(uint64_t* w, uint64_t count, uint64_t eid_base) {
    w[0] = count;
    w[1] = eid_base;
}

// Scratch sized for `count` records rounded up to a power of two (at least 1,024); reallocation
// invalidates the captured pipeline.
static bingo_status update_capacity(bingo_graph* g, uint64_t count) {
    uint64_t cap = 1024;
    while (cap < count) cap <<= 1;
    if (cap <= g->upd_cap) return BINGO_OK;
    if (g->upd_graph) cudaGraphExecDestroy(g->upd_graph);
    g->upd_graph = nullptr;
    cudaDeviceSynchronize();  // buffers may still be read by earlier work
    const uint64_t kc = 2 * cap;
    CK(ensure(g->s_in, 16 * cap), "update scratch");
    CK(ensure(g->s_rank, 16 * cap + 64), "update scratch");
    CK(ensure(g->s_keys, 8 * kc), "update scratch");
    CK(ensure(g->s_keys2, 8 * kc), "update scratch");
    CK(ensure(g->s_vals, 4 * kc), "update scratch");
    CK(ensure(g->s_vals2, 4 * kc), "update scratch");
    CK(ensure(g->s_seg, 8 * kc * 2 + 4 * (kc + 2) * 4 + 64), "update scratch");
    CK(ensure(g->s_aux, 4 * kc * 3 + 64), "update scratch");
    CK(ensure(g->s_best, 8 * kc + 64), "update scratch");
    CK(ensure(g->s_rec, 16 * kc), "update scratch");
    CK(ensure(g->s_seginfo, 16 * kc + 16), "update scratch");
    CK(ensure(g->s_gcand, 4ull * PRE_MULT * kc), "update scratch");
    CK(ensure(g->s_gcand_cnt, 16 * kc + 128), "update scratch");  // counts, segment list, chunk offsets and counts
    const uint64_t chunk_cap = std::min<uint64_t>((g->next_eid + kc) / PRE_CHUNK + kc + 64, 0xFFFFFFFFull);
    CK(ensure(g->s_chunkmap, 4 * chunk_cap), "update scratch");
    CK(ensure(g->s_tmp, std::max(radix_sort_tmp_bytes(kc), scan_tmp_bytes(kc))), "update scratch");
    if (!g->apply_blocks) {
        int per_sm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, g->G.fbits ? k_apply<true> : k_apply<false>,
                                                         APPLY_THREADS, 0),
           "apply occupancy");
        g->apply_blocks = (unsigned)std::max(1, per_sm) * (unsigned)g->num_sms;
    }
    g->upd_cap = cap;
    return BINGO_OK;
}

// The whole batch pipeline for a record capacity `cap`, with every size read on the device
// (record count, key count, segment count, edge-id base), so it can be captured once and replayed.
static bingo_status enqueue_updates(bingo_graph* g, uint64_t cap, cudaStream_t s) {
    uint64_t* ctl = (uint64_t*)g->d_ctl;
    const uint64_t kc = 2 * cap;
    CK(cudaMemsetAsync(ctl + CTL_STATUS, 0, 8, s), "status reset");
    CK(cudaMemsetAsync(ctl + CTL_STATS, 0, (CTL_SCR + 8 - CTL_STATS) * 8, s), "stats reset");
    BatchArgs A;
    A.ups = (const uint4*)g->s_in.p;
    A.count = cap;
    A.count_dev = ctl + CTL_SCR + 8;
    A.n = g->n;
    A.dst_n = g->G.dst_n;
    A.max_bits = g->G.base4 ? std::min<uint32_t>(g->cfg.max_bits, 2 * B4_POSITIONS) : g->cfg.max_bits;
    A.fbits = g->G.fbits;
    A.lambda = g->G.lambda;
    A.bn = bits_for(std::max(g->n, g->G.dst_n));  // one key width for the source and the destination
    A.keys = (uint64_t*)g->s_keys.p;
    A.vals = (uint32_t*)g->s_vals.p;
    A.packed = (uint64_t*)g->s_rank.p;
    A.pscan = A.packed + cap;
    A.status = (uint32_t*)(ctl + CTL_STATUS);
    A.perm = g->G.perm;
    uint64_t* total = (uint64_t*)(ctl + CTL_SCR + 4);  // low 32 bits: key count; high: insertions
    uint64_t* nkeys_dev = (uint64_t*)(ctl + CTL_SCR + 10);
    k_expand<<<grid_cap(g, cap, 256), 256, 0, s>>>(A);
    CK(scan_excl_u64(A.packed, A.pscan, cap, total, g->s_tmp, s, &g->launches), "update scan");
    k_make_keys<<<grid_cap(g, cap, 256), 256, 0, s>>>(A);
    k_key_count<<<1, 1, 0, s>>>(total, nkeys_dev);
    g->launches += 3;
    const uint32_t keybits = 2 * A.bn + 1;
    bool alt = false;
    CK(radix_sort_pairs(A.keys, A.vals, (uint64_t*)g->s_keys2.p, (uint32_t*)g->s_vals2.p, kc, keybits, g->s_tmp, s,
                        &alt, &g->launches, 0, nkeys_dev),
       "update sort");
    const uint64_t* skeys = alt ? (uint64_t*)g->s_keys2.p : A.keys;
    const uint32_t* svals = alt ? (uint32_t*)g->s_vals2.p : A.vals;
    uint64_t* flag = (uint64_t*)g->s_seg.p;
    uint64_t* segid = flag + kc;
    uint32_t* seg_start = (uint32_t*)(segid + kc);
    uint32_t* small_list = seg_start + kc + 2;
    uint32_t* big_list = small_list + kc + 2;
    uint32_t* dense_flag = big_list + kc + 2;
    uint64_t* nseg_dev = (uint64_t*)(ctl + CTL_SCR + 3);
    k_seg_flags<<<grid_cap(g, kc, 256), 256, 0, s>>>(skeys, svals, kc, nkeys_dev, A.bn, A.ups, A.pscan,
                                                     (const unsigned long long*)(ctl + CTL_SCR + 9), A.fbits,
                                                     A.lambda, g->G.base4, A.perm, flag, (uint4*)g->s_rec.p);
    CK(scan_excl_u64(flag, segid, kc, nseg_dev, g->s_tmp, s, &g->launches), "segment scan");
    k_seg_write<<<grid_cap(g, kc, 256), 256, 0, s>>>(flag, segid, kc, nkeys_dev, seg_start);
    g->launches += 2;
    unsigned long long* counts = (unsigned long long*)(ctl + CTL_SCR);  // small, big, pool bound
    CK(cudaMemsetAsync(counts, 0, 24, s), "counts reset");
    SegArgs S;
    memset(&S, 0, sizeof(S));
    S.B = A;
    S.sorted_keys = skeys;
    S.sorted_vals = svals;
    S.seg_start = seg_start;
    S.nseg_dev = nseg_dev;
    S.small_list = small_list;
    S.big_list = big_list;
    S.dense_flag = dense_flag;
    S.ndense = (unsigned long long*)(ctl + CTL_SCR + 14);
    CK(cudaMemsetAsync(S.ndense, 0, 16, s), "dense segment count reset");
    S.counts = counts;
    S.eid_base = 0;
    S.eid_base_dev = (const unsigned long long*)(ctl + CTL_SCR + 9);
    S.rec = (uint4*)g->s_rec.p;
    S.seginfo = (uint4*)g->s_seginfo.p;
    S.big_slots = g->cfg.update_chunk ? g->cfg.update_chunk : DEFAULT_UPDATE_CHUNK;
    S.gcand = (uint32_t*)g->s_gcand.p;
    S.gcand_cnt = (uint32_t*)g->s_gcand_cnt.p;
    S.huge_list = S.gcand_cnt + kc + 4;
    S.huge_coff = S.huge_list + kc + 4;
    S.huge_nch = S.huge_coff + kc + 4;
    S.chunk_seg = (uint32_t*)g->s_chunkmap.p;
    S.chunk_cap = (uint32_t)(g->s_chunkmap.bytes / 4);
    S.nhuge = (unsigned long long*)(ctl + CTL_SCR + 13);
    CK(cudaMemsetAsync(S.nhuge, 0, 8, s), "pre-pass count reset");
    S.holes = (uint32_t*)g->s_aux.p;
    S.surv = S.holes + kc;
    S.slot_scratch = S.surv + kc;
    S.best = (unsigned long long*)g->s_best.p;
    S.stats = (unsigned long long*)(ctl + CTL_STATS);
    k_seg_classify<<<grid_cap(g, kc, 256), 256, 0, s>>>(g->G, S);
    S.queue = (unsigned long long*)(ctl + CTL_SCR + 11);
    k_oom_check<<<1, 1, 0, s>>>(g->G, counts, S.queue);
    k_cand_plan<<<1, 1024, 0, s>>>(g->G, S);
    k_cand_scan<<<(unsigned)g->num_sms * 8, 256, 0, s>>>(g->G, S);
    if (g->G.fbits) {
        k_apply<true><<<g->apply_blocks, APPLY_THREADS, 0, s>>>(g->G, S);
    } else {
        k_apply<false><<<g->apply_blocks, APPLY_THREADS, 0, s>>>(g->G, S);
        k_apply_dense<<<g->apply_blocks, APPLY_THREADS, 0, s>>>(g->G, S);  // no dense-only segments on real biases
        g->launches++;
    }
    g->launches += 5;
    if (g->G.eh_mask) {
        k_eh_apply<<<grid_cap(g, kc, 256), 256, 0, s>>>(g->G, S, kc, nkeys_dev);
        g->launches++;
    }
    launch_pool_merge(g, s);
    CK(cudaGetLastError(), "update launch");
    return BINGO_OK;
}

extern "C" {

bingo_status bingo_apply_updates(bingo_graph* g, const bingo_update* ups, uint64_t count, void* stream,
                                 bingo_update_stats* stats) {
    if (!g) { set_error("NULL graph"); return BINGO_E_INVALID; }
    if (g->broken) { set_error("graph state is unusable after an earlier device failure"); return BINGO_E_STATE; }
    {
        const bingo_status ds = check_device(g, "apply_updates");
        if (ds != BINGO_OK) return ds;
    }
    if (count && !ups) { set_error("NULL update array"); return BINGO_E_INVALID; }
    if (count >= 0x3FFFFFFFull) { set_error("batch too large"); return BINGO_E_INVALID; }
    if (g->next_eid + count >= (1ull << 56)) { set_error("edge id space exhausted"); return BINGO_E_INVALID; }
    cudaStream_t s = (cudaStream_t)stream;
    if (count == 0) {
        if (stats) memset(stats, 0, sizeof(*stats));
        return BINGO_OK;
    }
    bingo_status st = update_capacity(g, count);
    if (st != BINGO_OK) return st;
    // the batch goes into the pipeline's fixed input buffer; count and edge-id base into device words
    CK(cudaMemcpyAsync(g->s_in.p, ups, count * 16, is_device_ptr(ups) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       s),
       "update upload");
    uint64_t* ctl = (uint64_t*)g->d_ctl;
    k_set_words<<<1, 1, 0, s>>>(ctl + CTL_SCR + 8, count, g->next_eid);
    g->launches++;
    const bool has_eh = g->G.eh_mask != 0;
    if (!g->upd_graph || g->upd_graph_eh != has_eh) {
        if (g->upd_graph) cudaGraphExecDestroy(g->upd_graph);
        g->upd_graph = nullptr;
        if (!g->cap_stream) CK(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking), "capture stream");
        const uint64_t l0 = g->launches;
        CK(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal), "update capture");
        const bingo_status est = enqueue_updates(g, g->upd_cap, g->cap_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(g->cap_stream, &graph);
        if (est != BINGO_OK) {
            if (graph) cudaGraphDestroy(graph);
            return est;
        }
        CK(ce, "update capture");
        cudaError_t ie = cudaGraphInstantiate(&g->upd_graph, graph, 0);
        cudaGraphDestroy(graph);
        CK(ie, "update graph instantiate");
        g->upd_graph_eh = has_eh;
        g->upd_graph_launches = g->launches - l0;
        g->launches = l0;
    }
    CK(cudaGraphLaunch(g->upd_graph, s), "update graph launch");
    g->launches += g->upd_graph_launches;
    bingo_update_stats local;
    if (!stats) stats = &local;
    st = finish_batch(g, s, stats, 0, false);
    if (st == BINGO_OK && g->G.eh_mask && stats && g->eh_distinct + stats->inserted > (g->G.eh_mask + 1) * 7 / 10) {
        g->eh_distinct += stats->inserted;
        st = edge_index_build(g, s);  // new edge-index pointers: the captured pipeline is re-captured
        if (g->upd_graph) cudaGraphExecDestroy(g->upd_graph);
        g->upd_graph = nullptr;
        if (st == BINGO_OK) CK(cudaStreamSynchronize(s), "edge index rebuild");
    } else if (st == BINGO_OK && stats) {
        g->eh_distinct += stats->inserted;
    }
    return st;
}

bingo_status bingo_stream_updates(bingo_graph* g, const bingo_update* ups, uint64_t count, void* stream,
                                  bingo_update_stats* stats) {
    if (!g) { set_error("NULL graph"); return BINGO_E_INVALID; }
    if (g->broken) { set_error("graph state is unusable after an earlier device failure"); return BINGO_E_STATE; }
    {
        const bingo_status ds = check_device(g, "stream_updates");
        if (ds != BINGO_OK) return ds;
    }
    if (count && !ups) { set_error("NULL update array"); return BINGO_E_INVALID; }
    if (count >= 0x7FFFFFFFull) { set_error("too many records"); return BINGO_E_INVALID; }
    if (g->next_eid + count >= (1ull << 56)) { set_error("edge id space exhausted"); return BINGO_E_INVALID; }
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* ctl = (uint64_t*)g->d_ctl;
    CK(cudaMemsetAsync(ctl + CTL_STATUS, 0, 8, s), "status reset");
    CK(cudaMemsetAsync(ctl + CTL_STATS, 0, (CTL_WORDS - CTL_STATS) * 8, s), "stats reset");
    if (count == 0) {
        if (stats) memset(stats, 0, sizeof(*stats));
        return BINGO_OK;
    }
    // The batch pipeline's captured graph holds pointers to these shared scratch buffers: if one must
    // grow, wait for earlier work, drop the graph and let the next batch size and capture it again.
    {
        auto grows = [](const Buf& b, size_t bytes) { return !(b.p && bytes <= b.bytes); };
        if ((!is_device_ptr(ups) && grows(g->s_in, count * 16)) || grows(g->s_rank, 16 * count + 64) ||
            grows(g->s_keys, 8 * count) || grows(g->s_keys2, 8 * count) || grows(g->s_vals, 4 * count) ||
            grows(g->s_vals2, 4 * count) || grows(g->s_seg, 8 * count * 2 + 4 * (count + 2) * 4 + 64)) {
            if (g->upd_graph) cudaGraphExecDestroy(g->upd_graph);
            g->upd_graph = nullptr;
            g->upd_cap = 0;
            cudaDeviceSynchronize();
        }
    }
    const uint4* dups = (const uint4*)ups;
    if (!is_device_ptr(ups)) {
        CK(ensure(g->s_in, count * 16), "update staging");
        CK(cudaMemcpyAsync(g->s_in.p, ups, count * 16, cudaMemcpyHostToDevice, s), "update upload");
        dups = (const uint4*)g->s_in.p;
    }
    CK(ensure(g->s_rank, 16 * count + 64), "stream scratch");
    CK(ensure(g->s_keys, 8 * count), "stream scratch");
    CK(ensure(g->s_keys2, 8 * count), "stream scratch");
    CK(ensure(g->s_vals, 4 * count), "stream scratch");
    CK(ensure(g->s_vals2, 4 * count), "stream scratch");
    CK(ensure(g->s_seg, 8 * count * 2 + 4 * (count + 2) * 4 + 64), "segment scratch");
    BatchArgs A;
    A.ups = dups;
    A.count = count;
    A.count_dev = nullptr;
    A.n = g->n;
    A.dst_n = g->G.dst_n;
    A.max_bits = g->G.base4 ? std::min<uint32_t>(g->cfg.max_bits, 2 * B4_POSITIONS) : g->cfg.max_bits;
    A.fbits = g->G.fbits;
    A.lambda = g->G.lambda;
    A.bn = bits_for(std::max(g->n, g->G.dst_n));  // one key width for the source and the destination
    A.keys = (uint64_t*)g->s_keys.p;
    A.vals = (uint32_t*)g->s_vals.p;
    A.packed = (uint64_t*)g->s_rank.p;
    A.pscan = A.packed + count;
    A.status = (uint32_t*)(ctl + CTL_STATUS);
    A.perm = g->G.perm;
    uint64_t* total = (uint64_t*)(ctl + CTL_SCR + 4);
    k_expand<<<grid_cap(g, count, 256), 256, 0, s>>>(A);  // validation + insertion flags
    CK(scan_excl_u64(A.packed, A.pscan, count, total, g->s_tmp, s, &g->launches), "stream scan");
    k_stream_keys<<<grid_cap(g, count, 256), 256, 0, s>>>(A);
    g->launches += 2;
    bool alt = false;
    CK(radix_sort_pairs(A.keys, A.vals, (uint64_t*)g->s_keys2.p, (uint32_t*)g->s_vals2.p, count, A.bn, g->s_tmp, s,
                        &alt, &g->launches, A.bn + 1),
       "stream sort");
    const uint64_t* skeys = alt ? (uint64_t*)g->s_keys2.p : A.keys;
    const uint32_t* svals = alt ? (uint32_t*)g->s_vals2.p : A.vals;
    uint64_t* flag = (uint64_t*)g->s_seg.p;
    uint64_t* segid = flag + count;
    uint32_t* seg_start = (uint32_t*)(segid + count);
    uint64_t* nseg_dev = (uint64_t*)(ctl + CTL_SCR + 3);
    k_seg_flags<<<grid_cap(g, count, 256), 256, 0, s>>>(skeys, svals, count, nullptr, A.bn, A.ups, A.pscan, nullptr,
                                                        0u, 0.0, 0u, nullptr, flag, nullptr);
    CK(scan_excl_u64(flag, segid, count, nseg_dev, g->s_tmp, s, &g->launches), "stream segments");
    k_seg_write<<<grid_cap(g, count, 256), 256, 0, s>>>(flag, segid, count, nullptr, seg_start);
    SegArgs S;
    memset(&S, 0, sizeof(S));
    S.B = A;
    S.sorted_keys = skeys;
    S.sorted_vals = svals;
    S.seg_start = seg_start;
    S.nseg_dev = nseg_dev;
    S.eid_base = g->next_eid;
    S.eid_base_dev = nullptr;
    S.stats = (unsigned long long*)(ctl + CTL_STATS);
    unsigned long long* reserved = (unsigned long long*)(ctl + CTL_SCR + 7);
    unsigned long long* nbig = (unsigned long long*)(ctl + CTL_SCR + 13);
    uint32_t* big_list = seg_start + count + 2;
    CK(cudaMemsetAsync(nbig, 0, 8, s), "stream big-vertex count");
    const unsigned blocks = grid_cap(g, count, STREAM_TEAMS, 8);
    const unsigned big_blocks = (unsigned)g->num_sms * 2;
    if (g->G.fbits) {
        k_stream_apply<true><<<blocks, STREAM_TEAMS * 32, 0, s>>>(g->G, S, reserved, big_list, nbig);
        k_stream_apply_big<true><<<big_blocks, STREAM_BIG_THREADS, 0, s>>>(g->G, S, reserved, big_list, nbig);
    } else {
        k_stream_apply<false><<<blocks, STREAM_TEAMS * 32, 0, s>>>(g->G, S, reserved, big_list, nbig);
        k_stream_apply_big<false><<<big_blocks, STREAM_BIG_THREADS, 0, s>>>(g->G, S, reserved, big_list, nbig);
    }
    g->launches += 4;
    CK(cudaGetLastError(), "stream launch");
    bingo_status st = finish_batch(g, s, stats, 0);
    if (st == BINGO_OK && g->G.eh_mask && g->eh_distinct + (stats ? stats->inserted : count) > (g->G.eh_mask + 1) * 7 / 10) {
        st = edge_index_build(g, s);
        if (st == BINGO_OK) CK(cudaStreamSynchronize(s), "edge index rebuild");
    } else if (st == BINGO_OK) {
        g->eh_distinct += stats ? stats->inserted : count;
    }
    return st;
}

bingo_status bingo_autotune_updates(bingo_graph* g, const bingo_update* ups, uint64_t count, void* stream,
                                    bingo_update_stats* stats, bingo_config* out_cfg) {
    if (!g || (count && !ups)) { set_error("autotune: bad arguments"); return BINGO_E_INVALID; }
    static const uint32_t cand[] = {1024, 2048, 4096, 8192, 16384};
    constexpr int NC = 5, ROUNDS = 2;
    cudaStream_t s = (cudaStream_t)stream;
    bingo_update_stats total;
    memset(&total, 0, sizeof(total));
    auto add = [&](const bingo_update_stats& x) {
        total.inserted += x.inserted;
        total.deleted += x.deleted;
        total.not_found += x.not_found;
        total.vertices_touched += x.vertices_touched;
        total.groups_rebuilt += x.groups_rebuilt;
        for (int a = 0; a < 5; a++)
            for (int b = 0; b < 5; b++) total.conversions[a][b] += x.conversions[a][b];
    };
    const uint64_t slice = count / (NC * ROUNDS);
    bingo_status st = BINGO_OK;
    if (slice == 0) {  // too few records to compare settings: apply them as one batch
        st = bingo_apply_updates(g, ups, count, stream, &total);
    } else {
        // the slices share one capacity (the largest slice), so only the setting changes between them
        if ((st = update_capacity(g, count - slice * (NC * ROUNDS - 1))) != BINGO_OK) return st;
        double per_rec[NC] = {0};
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const uint32_t saved = g->cfg.update_chunk;
        uint64_t off = 0;
        for (int r = 0; r < ROUNDS && st == BINGO_OK; r++) {
            for (int c = 0; c < NC && st == BINGO_OK; c++) {
                const bool last = r == ROUNDS - 1 && c == NC - 1;
                const uint64_t n = last ? count - off : slice;
                if (g->cfg.update_chunk != cand[c]) {
                    g->cfg.update_chunk = cand[c];
                    if (g->upd_graph) cudaGraphExecDestroy(g->upd_graph);  // the setting is baked into the graph
                    g->upd_graph = nullptr;
                }
                bingo_update_stats one;
                cudaEventRecord(e0, s);
                st = bingo_apply_updates(g, ups + off, n, stream, &one);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (st == BINGO_OK) {
                    add(one);
                    per_rec[c] += ms / (double)n;
                }
                off += n;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        int best = 0;
        for (int c = 1; c < NC; c++)
            if (per_rec[c] < per_rec[best]) best = c;
        g->cfg.update_chunk = st == BINGO_OK ? cand[best] : saved;
        if (g->upd_graph) cudaGraphExecDestroy(g->upd_graph);
        g->upd_graph = nullptr;
    }
    if (stats) *stats = total;
    if (out_cfg && st == BINGO_OK) st = bingo_get_config(g, out_cfg);
    return st;
}

}  // extern "C"
