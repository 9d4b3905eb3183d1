// Internal device structures and primitives of the radix-factorised sampler.
//
// Device state of a graph (all in HBM):
//   vh[v]   VHot, 64 bytes: one sector {adjacency block, degree d, nonempty-group mask, the
//           caller's id of v (path entries), the total weight outside the hot pairs, the hot pairs
//           a, b}, then copies of groups 2a, 2a+1, 2b, 2b+1 as {|G_k|, ref} (Eq. wpk: W(p_k) =
//           2^k |G_k|); ref = destination of the member of a one-element group, or the group block
//           of a regular/sparse group, else 0.  The hot pairs are the vertex's two heaviest pairs
//           (hot_summary): a walker step draws its group from this one line whenever the draw
//           falls in them.
//   vc[v]   VCold, 256 bytes: all 32 groups (the copy that updates read and write).
//   vu[v]   VUpd, 16 bytes: update-only fields (|S|, log2 capacities, sparse-list block).
//   pool    u32 words holding every variable-size block, in power-of-two sizes (offsets stored in
//           32-byte units):
//             adjacency   4*capA words: capA x {dst, bias} (8 B, AoS) then capA x u64 edge id
//             regular k   4*capA words: member destinations, member slots, inverted index (by slot), spare
//             sparse list 2*capA words: S = slots of edges in any sparse group [capA], then
//                         S_inv [capA] (by slot)
//             sparse k    4*capS words: member destinations, member positions in S, inverted index
//                         (by S position), spare
//             decimal     max(8, capA/4) words: capA bytes, the decimal part q of each adjacency
//                         slot (real-bias graphs only; referenced by group slot 31)
// A group's kind is never stored: it is the pure function of (|G_k|, d) given by Eq. group.
// Real-bias graphs (Section 4.3): slot k < 31 is the radix group of bit k of the integer parts,
// weighted 2^8 2^k |G_k| (units of 2^-8); slot 31 is the decimal group {Q_D = sum q, decimal
// block}, weighted Q_D, and is never given a kind.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "bingo.h"

namespace bingo {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t NONE32 = 0xFFFFFFFFu;
constexpr uint64_t DEAD_BIT = 1ull << 63;      // set in an adjacency edge id while its slot is being deleted
constexpr uint32_t MIN_CAPA = 4;               // smallest adjacency capacity of a vertex with edges
constexpr uint32_t MIN_CAPS = 4;
constexpr int NCLASS = 48;                     // pool size classes: block of 8 << c words
constexpr uint32_t MAX_POL = 16;

enum : uint32_t { K_EMPTY = 0, K_DENSE = 1, K_ONE = 2, K_SPARSE = 3, K_REGULAR = 4 };

// status bits accumulated on the device
enum : uint32_t {
    ST_INVALID = 1u,
    ST_OOM = 2u,
    ST_TIMEOUT = 4u,   // a bounded loop gave up (corrupt state or an impossible rejection)
    ST_STATE = 8u,
};

// Decoded vertex header (offsets in pool words); the stored form is VRec.
struct VHdr {
    uint64_t adj;   // word offset of the adjacency block (0 = none)
    uint32_t deg;   // live edges d
    uint32_t mask;  // bit k set iff |G_k| > 0
    uint64_t sref;  // word offset of the sparse-list block (0 = none)
    uint32_t nsp;   // |S|
    uint8_t lcapa;  // log2(capA) + 1, 0 = no adjacency block
    uint8_t lcaps;  // log2(capS) + 1, 0 = no sparse groups
    uint16_t pad;
    uint32_t word;  // the hot record's caller-id word as loaded (store_hdr leaves it alone)
};

// The hot line carries copies of the vertex's two heaviest group pairs (pairs a, b: groups 2a, 2a+1,
// 2b, 2b+1) and the total weight of every other group, so a draw that falls in those pairs needs no
// other access.  The cold record holds all 32 groups (the authoritative copy that updates read).
struct __align__(64) VHot {
    uint32_t adj;   // adjacency block, 32-byte units
    uint32_t deg;
    uint32_t mask;
    uint32_t word;  // the caller's id of this vertex (path entries of walks); top bit: the cold scan order (hot_summary)
    uint64_t wcold; // sum of the weights of the groups outside the hot pairs: with them, the vertex total
    uint32_t hp;    // the hot pairs: a = hp & 15 (scanned first), b = (hp >> 4) & 15
    uint32_t spare;
    uint2 g[4];     // copies of groups 2a, 2a+1, 2b, 2b+1
};
struct __align__(64) VCold {
    uint2 g[32];         // every group {|G_k|, ref}
};
// Fields that only updates read, in an array of their own.
struct __align__(16) VUpd {
    uint32_t nsp;
    uint8_t lcapa, lcaps;
    uint16_t pad;
    uint32_t sref;       // sparse-list block, 32-byte units
    uint32_t spare;
};
static_assert(sizeof(VHot) == 64, "VHot must be two sectors");
static_assert(offsetof(VHot, g) == 32, "hot copies fill the second sector");
static_assert(sizeof(VCold) == 256, "VCold must be four lines");
static_assert(sizeof(VUpd) == 16, "VUpd is 16 bytes");

constexpr uint64_t POOL_UNIT_WORDS = 8;  // offsets are stored in 32-byte units
constexpr uint64_t MAX_POOL_WORDS = (1ull << 32) * POOL_UNIT_WORDS;
__host__ __device__ __forceinline__ uint64_t words_of(uint64_t ref) { return ref * POOL_UNIT_WORDS; }
__host__ __device__ __forceinline__ uint32_t ref_of(uint64_t words) { return (uint32_t)(words / POOL_UNIT_WORDS); }

__host__ __device__ __forceinline__ uint32_t capa_of(const VHdr& h) { return h.lcapa ? (1u << (h.lcapa - 1)) : 0u; }
__host__ __device__ __forceinline__ uint32_t caps_of(const VHdr& h) { return h.lcaps ? (1u << (h.lcaps - 1)) : 0u; }

// alpha value that turns group adaption off: every nonempty group regular (the BS baseline of the
// group-adaption ablation, Section 6.2).
constexpr uint32_t ALL_REGULAR = 0xFFFFFFFFu;

// Eq. group (Section 5.1), in its printed order with strict percent comparisons.
__host__ __device__ __forceinline__ uint32_t kind_of(uint32_t c, uint32_t d, uint32_t alpha, uint32_t beta) {
    if (c == 0) return K_EMPTY;
    if (alpha == ALL_REGULAR) return K_REGULAR;
    const uint64_t c100 = 100ull * c;
    if (c100 > (uint64_t)alpha * d) return K_DENSE;
    if (c == 1) return K_ONE;
    if (c100 < (uint64_t)beta * d) return K_SPARSE;
    return K_REGULAR;
}
__host__ __device__ __forceinline__ bool is_list(uint32_t k) { return k == K_REGULAR || k == K_SPARSE; }

__host__ __device__ __forceinline__ uint32_t next_pow2_u32(uint32_t x) {
    if (x <= 1) return 1;
#ifdef __CUDA_ARCH__
    return 1u << (32 - __clz(x - 1));
#else
    return 1u << (32 - __builtin_clz(x - 1));
#endif
}
__host__ __device__ __forceinline__ uint32_t log2_u32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return 31 - __clz(x);
#else
    return 31 - __builtin_clz(x);
#endif
}
__host__ __device__ __forceinline__ uint32_t capa_for(uint32_t d) {
    if (d == 0) return 0;
    uint32_t c = next_pow2_u32(d);
    return c < MIN_CAPA ? MIN_CAPA : c;
}
__host__ __device__ __forceinline__ uint32_t caps_for(uint32_t s) {
    uint32_t c = next_pow2_u32(s);
    return c < MIN_CAPS ? MIN_CAPS : c;
}
// size class of a power-of-two block of `words` (>= 8) words
__host__ __device__ __forceinline__ uint32_t class_of(uint64_t words) {
    uint32_t c = 0;
    while ((8ull << c) < words) c++;
    return c;
}

// ---------------------------------------------------------------------------------------------- pool

struct Pool {
    uint32_t* base;                  // words
    uint64_t words;                  // capacity
    unsigned long long* top;         // device: bump pointer (words)
    long long* fcount;               // device [NCLASS]: free blocks available per class
    uint64_t* fstack;                // device [NCLASS][fcap]
    uint64_t fcap;                   // entries per class stack
    unsigned long long* npending;    // device: frees made during the current batch
    uint64_t* pending;               // device [pcap]: (offset << 8) | class
    uint64_t pcap;
    unsigned long long* leaked;      // device: words dropped because a free list was full
    uint32_t* status;                // device status word
};

#ifdef __CUDACC__
// Allocate a power-of-two block (words >= 8).  Free blocks of the class are
// popped first; otherwise the bump pointer advances.  Frees made in the same
// batch only become reusable at the batch's end, so pops never race pushes.
__device__ __forceinline__ uint64_t pool_alloc(const Pool& P, uint64_t words) {
    const uint32_t c = class_of(words);
    const uint64_t sz = 8ull << c;
    const long long i = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&P.fcount[c]), ~0ull) - 1;
    if (i >= 0 && (uint64_t)i < P.fcap) return P.fstack[(uint64_t)c * P.fcap + (uint64_t)i];
    unsigned long long off = atomicAdd(P.top, (unsigned long long)sz);
    if (off + sz > P.words) {
        atomicOr(P.status, ST_OOM);
        return 0;
    }
    return off;
}
__device__ __forceinline__ void pool_free(const Pool& P, uint64_t off, uint64_t words) {
    if (off == 0) return;
    const uint32_t c = class_of(words);
    unsigned long long i = atomicAdd(P.npending, 1ull);
    if (i < P.pcap) P.pending[i] = (off << 8) | c;
    else atomicAdd(P.leaked, (unsigned long long)(8ull << c));
}
#endif

// ---------------------------------------------------------------------------------------------- graph view

struct DevGraph {
    uint32_t n;
    uint32_t max_bits;
    uint32_t alpha, beta;
    uint32_t fbits;   // 0: integer biases; FRAC_BITS: real biases (slot 31 = decimal group)
    double lambda;    // real biases: amortisation factor
    uint32_t base4;   // 1: radix base 4, the stored bias word is the sub-group mask (b4_mask)
    // Internal vertex numbering: vertices are renumbered by descending out-degree (ties by id), so the
    // records of the vertices walks visit most sit together in HBM and L2.  order[i] = caller's id of
    // internal vertex i, perm[v] = internal id of the caller's vertex v; both null = identity.
    const uint32_t* order;
    const uint32_t* perm;
    // A partition graph holds the rows of the global vertices [base, base + n) as local vertices
    // 0 .. n-1; its destinations are global ids below dst_n.  A whole graph has base 0, dst_n = n.
    uint32_t base;
    uint32_t dst_n;

    VHot* vh;
    VCold* vc;
    VUpd* vu;
    Pool pool;
    // edge index (node2vec distance probe): open addressing over (src << 32 | dst) -> live copies
    unsigned long long* eh_key;  // EH_EMPTY = empty
    uint32_t* eh_cnt;
    uint64_t eh_mask;            // capacity - 1, 0 = absent
};
constexpr unsigned long long EH_EMPTY = 0xFFFFFFFFFFFFFFFFull;

// Partitioned walks (graphs split into vertex ranges, walkers moving between them): a walker between
// two partitions' launches is a record {walker id, current vertex, previous vertex (global ids), the
// step it is at}; the next launch of the current vertex's owner resumes it.
struct PartRec {
    uint64_t wid;
    uint32_t cur, prev, step, pad;
};
static_assert(sizeof(PartRec) == 24, "walker records are 24 bytes");
// One partition's node2vec edge index (keys: local source << 32 | global destination).
struct PartEH {
    const unsigned long long* key;
    const uint32_t* cnt;
    uint64_t mask;  // 0 = absent
};

#ifdef __CUDACC__
__device__ __forceinline__ VHdr load_hdr(const DevGraph& G, uint64_t v) {
    const VHot& a = G.vh[v];
    const VUpd& b = G.vu[v];
    VHdr h;
    h.adj = words_of(a.adj);
    h.deg = a.deg;
    h.mask = a.mask;
    h.sref = words_of(b.sref);
    h.nsp = b.nsp;
    h.lcapa = b.lcapa;
    h.lcaps = b.lcaps;
    h.pad = 0;
    h.word = a.word;
    return h;
}
__device__ __forceinline__ void store_hdr(const DevGraph& G, uint64_t v, const VHdr& h) {
    VHot& a = G.vh[v];
    VUpd& b = G.vu[v];
    a.adj = ref_of(h.adj);
    a.deg = h.deg;
    a.mask = h.mask;
    b.sref = ref_of(h.sref);  // the hot word (caller's id) is set once, at build
    b.nsp = h.nsp;
    b.lcapa = h.lcapa;
    b.lcaps = h.lcaps;
    b.pad = 0;
}

// ids at or above n pass through unchanged (callers reject them)
__device__ __forceinline__ uint32_t to_internal(const DevGraph& G, uint32_t v) {
    return (G.perm && v < G.n) ? __ldg(G.perm + v) : v;
}
__device__ __forceinline__ uint32_t to_caller(const DevGraph& G, uint32_t v) {
    return G.order ? __ldg(G.order + v) : v + G.base;
}

// {|G_k|, ref} of group k of vertex v
__device__ __forceinline__ uint2& grp(const DevGraph& G, uint64_t v, uint32_t k) {
    return G.vc[v].g[k];
}
__device__ __forceinline__ uint32_t& cnt_ref(const DevGraph& G, uint64_t v, uint32_t k) { return grp(G, v, k).x; }
__device__ __forceinline__ uint32_t& gref_ref(const DevGraph& G, uint64_t v, uint32_t k) { return grp(G, v, k).y; }

// ---- real biases (Section 4.3)
constexpr uint32_t FRAC_BITS = 8;
constexpr uint32_t DEC_SLOT = 31;
constexpr uint32_t REAL_MAX_DEG = 1u << 24;  // keeps Q_D < 2^32 and the vertex total < 2^64
// Words of the decimal block of an adjacency of capacity capa (one byte per slot).
__host__ __device__ __forceinline__ uint64_t dec_words(uint32_t capa) { return capa / 4 < 8 ? 8 : capa / 4; }
// Split a real bias (binary32 encoding) into the integer part I = floor(lambda b) and the decimal
// part q = floor((lambda b - I) 2^FRAC_BITS), with lambda b rounded once to binary64.  False if b is
// not finite or negative, lambda b >= 2^31, or the weight 2^FRAC_BITS I + q is zero.
__device__ __forceinline__ bool split_real_bias(uint32_t bits, double lambda, uint32_t& I, uint32_t& q) {
    const float b = __uint_as_float(bits);
    I = 0;
    q = 0;
    if (!isfinite(b) || b < 0.0f) return false;
    const double x = __dmul_rn(lambda, (double)b);
    if (!(x < 2147483648.0)) return false;
    const double ip = floor(x);
    I = (uint32_t)ip;
    q = (uint32_t)floor(__dmul_rn(__dsub_rn(x, ip), (double)(1u << FRAC_BITS)));
    return I != 0 || q != 0;
}
// The factorised part of an insertion's bias word: the integer bias, or the integer part of a real one.
__device__ __forceinline__ uint32_t int_part(const DevGraph& G, uint32_t bits) {
    if (!G.fbits) return bits;
    uint32_t I, q;
    split_real_bias(bits, G.lambda, I, q);
    return I;
}
// Sampling weight of group slot k with count c (Eq. wpk), in units of 2^-fbits.
__device__ __forceinline__ uint64_t slot_w(uint32_t c, uint32_t k, uint32_t fbits) {
    return (fbits && k == DEC_SLOT) ? (uint64_t)c : ((uint64_t)c << (k + fbits));
}
// Weight modes of the walker: integer base 2, real biases, integer base 4.
enum : int { WM_INT = 0, WM_REAL = 1, WM_B4 = 2 };
template <int WM>
__device__ __forceinline__ uint64_t slot_weight(uint32_t c, uint32_t k) {
    if constexpr (WM == WM_B4) return (uint64_t)c * ((uint64_t)(k % 3 + 1) << (2 * (k / 3)));
    else return slot_w(c, k, WM == WM_REAL ? FRAC_BITS : 0u);
}
// The graph's slot weight, its weight mode taken at run time (update and build kernels).
__device__ __forceinline__ uint64_t graph_slot_weight(const DevGraph& G, uint32_t c, uint32_t k) {
    return G.base4 ? slot_weight<WM_B4>(c, k) : slot_w(c, k, G.fbits);
}
// The hot pairs and the order in which a draw that falls beyond them scans the other (cold) pairs.
// The hot pairs a, b are the two pairs of largest weight W(p_2i) + W(p_2i+1), ranked by the weight's
// leading 21 bits (equal ranks: the lower pair; a vertex with one nonempty pair takes the lowest other
// pair as b).  The walker reads the cold pairs
// in batches whose loads are issued together, and reads a batch only when the draw lies beyond the
// earlier ones: upwards, the aligned batches [0, 4), [4, 8), [8, 12), [12, 16); downwards, windows
// of four consecutive pairs from the highest nonempty cold pair; hot pairs and batches without a
// nonempty pair are skipped.  Any fixed order gives the same law (Eq. group_prob).  The order is a
// pure function of the counts: downwards iff it reads fewer batches in expectation (each cold
// pair's weight times the number of batches read to reach it), ties upwards.  It is kept in the top
// bit of the hot record's caller-id word (vertex ids are below 2^31).
constexpr uint32_t WORD_DESC = 0x80000000u;
constexpr uint32_t WORD_ID = 0x7FFFFFFFu;
#ifdef __CUDACC__
// The hot pairs (hp), the total weight outside them (wcold, exact) and the cold scan order of a
// vertex from its 32 slot counts, computed by one whole warp (every lane calls it with its lane id and
// the count of slot `lane`): lane k weighs slot k, lane i < 16 pair i; the arg-maxima, batch and
// window ranks come from shuffles and ballots; the expected-batch comparison is a sum of weight x
// (upward rank - downward rank) in binary64, reduced in a fixed shuffle order, so the same counts
// always give the same result (build, update and the export's check all call this).
__device__ __forceinline__ void hot_summary(const DevGraph& G, uint32_t c, uint32_t lane, uint64_t& wcold,
                                            bool& desc, uint32_t& hp) {
    const uint64_t wk = graph_slot_weight(G, c, lane);
    uint64_t tot = wk;
#pragma unroll
    for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
    const uint32_t i = lane & 15;
    const uint64_t wp = __shfl_sync(0xFFFFFFFFu, wk, 2 * i) + __shfl_sync(0xFFFFFFFFu, wk, 2 * i + 1);
    const uint32_t cp = __shfl_sync(0xFFFFFFFFu, c, 2 * i) | __shfl_sync(0xFFFFFFFFu, c, 2 * i + 1);
    // pair ranks by a 32-bit key: the weight's bit length (7 bits) and the 20 bits below its leading
    // one, then 15 - i (so equal keys go to the lower pair); the heaviest, then the heaviest of the rest
    uint32_t key = 0;
    if (lane < 16) {
        const uint32_t e = 64u - (uint32_t)__clzll((long long)wp);  // 0 for an empty pair
        const uint32_t m = e > 21 ? (uint32_t)(wp >> (e - 21)) : (uint32_t)(wp << (21 - e));
        key = (e << 25) | ((m & 0xFFFFFu) << 5) | (15u - i);
    }
    const uint32_t a = 15u - (__reduce_max_sync(0xFFFFFFFFu, key) & 15u);
    const uint32_t b = 15u - (__reduce_max_sync(0xFFFFFFFFu, lane < 16 && i != a ? key : 0u) & 15u);
    hp = a | (b << 4);
    wcold = tot - __shfl_sync(0xFFFFFFFFu, wp, a) - __shfl_sync(0xFFFFFFFFu, wp, b);
    const bool ne = lane < 16 && i != a && i != b && cp != 0;
    const uint32_t M = __ballot_sync(0xFFFFFFFFu, ne);
    if (!M) { desc = false; return; }
    const uint32_t hi = 31 - __clz(M);
    const uint32_t bt = i / 4, w = (hi - i) / 4;  // meaningful where ne
    const uint32_t BM = __reduce_or_sync(0xFFFFFFFFu, ne ? 1u << bt : 0u);
    const uint32_t WMk = __reduce_or_sync(0xFFFFFFFFu, ne ? 1u << w : 0u);
    const int ra = __popc(BM & ((2u << bt) - 1u)), rd = __popc(WMk & ((2u << w) - 1u));
    double x = ne ? (double)wp * (double)(ra - rd) : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    desc = x > 0.0;
}
// Slot of the hot line that copies group k (0..3), or 4 if k is not in a hot pair.
__device__ __forceinline__ uint32_t hot_slot(uint32_t hp, uint32_t k) {
    const uint32_t p = k >> 1;
    return p == (hp & 15u) ? (k & 1u) : p == ((hp >> 4) & 15u) ? 2u + (k & 1u) : 4u;
}
// Write the hot line of v from the warp's slot counts and refs (lane k: group k), after the groups
// themselves: the copies of the hot pairs, the cold total, the hot pairs and the scan-order bit
// (word: the record's caller-id word as it stands).
__device__ __forceinline__ void write_hot(const DevGraph& G, uint64_t v, uint32_t lane, uint32_t c, uint32_t gref,
                                          uint32_t word) {
    uint64_t wc;
    bool desc;
    uint32_t hp;
    hot_summary(G, c, lane, wc, desc, hp);
    const uint32_t hs = hot_slot(hp, lane);
    if (hs < 4) G.vh[v].g[hs] = make_uint2(c, gref);
    if (lane == 0) {
        G.vh[v].wcold = wc;
        G.vh[v].hp = hp;
        G.vh[v].word = (word & WORD_ID) | (desc ? WORD_DESC : 0u);
    }
}
#endif
// ---- radix base 4 (Appendix): sub-group (digit position i, value v) is slot 3 i + v - 1.
constexpr uint32_t B4_POSITIONS = 10;  // biases below 4^10 = 2^20: slots 0..29
// Sub-group mask of a bias: bit 3 i + v - 1 for every nonzero base-4 digit v at position i.  Stored
// in place of the bias, so membership of slot k stays a bit test, as in base 2.
__host__ __device__ __forceinline__ uint32_t b4_mask(uint32_t w) {
    uint32_t m = 0;
    for (uint32_t i = 0; i < B4_POSITIONS; i++) {
        const uint32_t d = (w >> (2 * i)) & 3u;
        if (d) m |= 1u << (3 * i + d - 1);
    }
    return m;
}
// The bias a sub-group mask stands for.
__host__ __device__ __forceinline__ uint32_t b4_value(uint32_t m) {
    uint32_t w = 0;
    for (uint32_t k = 0; k < 3 * B4_POSITIONS; k++)
        if ((m >> k) & 1u) w += (k % 3 + 1) << (2 * (k / 3));
    return w;
}

// Kind of group slot k (Eq. group); the decimal slot of a real-bias graph has none.
__device__ __forceinline__ uint32_t slot_kind(const DevGraph& G, uint32_t c, uint32_t d, uint32_t k) {
    return (G.fbits && k == DEC_SLOT) ? (uint32_t)K_EMPTY : kind_of(c, d, G.alpha, G.beta);
}
__device__ __forceinline__ uint8_t* dec_bytes(const DevGraph& G, uint32_t ref) {
    return reinterpret_cast<uint8_t*>(G.pool.base + words_of(ref));
}

__device__ __forceinline__ uint2* adj_pairs(const DevGraph& G, uint64_t adj) { return reinterpret_cast<uint2*>(G.pool.base + adj); }
__device__ __forceinline__ uint64_t* adj_eids(const DevGraph& G, uint64_t adj, uint32_t capa) {
    return reinterpret_cast<uint64_t*>(G.pool.base + adj + 2ull * capa);
}

__device__ __forceinline__ uint64_t eh_hash(uint64_t key) {
    key ^= key >> 33;
    key *= 0xff51afd7ed558ccdull;
    key ^= key >> 33;
    key *= 0xc4ceb9fe1a85ec53ull;
    key ^= key >> 33;
    return key;
}
// live copies of (u, x) in an edge index; bounded probe
__device__ __forceinline__ uint32_t eh_lookup_in(const unsigned long long* keys, const uint32_t* cnts, uint64_t mask,
                                                 uint32_t u, uint32_t x) {
    const unsigned long long key = ((unsigned long long)u << 32) | x;
    uint64_t h = eh_hash(key) & mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
        unsigned long long k = __ldg(keys + h);
        if (k == key) return __ldg(cnts + h);
        if (k == EH_EMPTY) return 0;
        h = (h + 1) & mask;
    }
    return 0;
}
__device__ __forceinline__ uint32_t eh_lookup(const DevGraph& G, uint32_t u, uint32_t x) {
    return eh_lookup_in(G.eh_key, G.eh_cnt, G.eh_mask, u, x);
}

// ---------------------------------------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
// ten rounds of two 32x32 -> 64 multiplies with a Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Per walker-step stream: counter (walker lo, walker hi, step, j) with j = 0, 1, ...;
// the four outputs of each call are consumed in order.
struct StepRng {
    uint2 key;
    uint32_t c0, c1, step, j;
    uint4 buf;
    uint32_t left;
    __device__ __forceinline__ void init(uint2 k, uint64_t walker, uint32_t s) {
        key = k;
        c0 = (uint32_t)walker;
        c1 = (uint32_t)(walker >> 32);
        step = s;
        j = 0;
        left = 0;
    }
    __device__ __forceinline__ uint32_t next() {
        if (left == 0) {
            buf = philox4x32_10(make_uint4(c0, c1, step, j++), key);
            left = 4;
        }
        const uint32_t r = buf.x;
        buf.x = buf.y;
        buf.y = buf.z;
        buf.z = buf.w;
        left--;
        return r;
    }
};

// Exact uniform integer in [0, range), range >= 1: Lemire's multiply-shift with
// rejection ("Fast random integer generation in an interval", ACM TOMACS 2019).
// A draw is rejected iff the low word of x * range is below 2^32 mod range.
// The retry loop is bounded; running out (probability < 2^-60) flags ST_TIMEOUT.
__device__ __forceinline__ uint32_t below32(StepRng& R, uint32_t range, uint32_t* status) {
    uint32_t x = R.next();
    uint64_t m = (uint64_t)x * range;
    uint32_t l = (uint32_t)m;
    if (l < range) {
        const uint32_t t = (0u - range) % range;
        int guard = 0;
        while (l < t) {
            if (++guard > 64) { atomicOr(status, ST_TIMEOUT); break; }
            x = R.next();
            m = (uint64_t)x * range;
            l = (uint32_t)m;
        }
    }
    return (uint32_t)(m >> 32);
}
__device__ __forceinline__ uint64_t below64(StepRng& R, uint64_t range, uint32_t* status) {
    if (range <= 0xFFFFFFFFull) return below32(R, (uint32_t)range, status);
    uint64_t x = ((uint64_t)R.next() << 32) | R.next();
    uint64_t lo = x * range, hi = __umul64hi(x, range);
    if (lo < range) {
        const uint64_t t = (0ull - range) % range;
        int guard = 0;
        while (lo < t) {
            if (++guard > 64) { atomicOr(status, ST_TIMEOUT); break; }
            x = ((uint64_t)R.next() << 32) | R.next();
            lo = x * range;
            hi = __umul64hi(x, range);
        }
    }
    return hi;
}

// ---------------------------------------------------------------------------------------------- teams
// A team is the set of threads that cooperates on one vertex: a warp or a block.
// Every member must reach every team call (loops run a team-uniform trip count).

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

struct WarpTeam {
    __device__ __forceinline__ uint32_t size() const { return 32; }
    __device__ __forceinline__ uint32_t rank() const { return threadIdx.x & 31; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    // exclusive prefix count of a predicate, in rank order
    __device__ __forceinline__ uint32_t scan_pred(bool p, uint32_t& total) const {
        const uint32_t b = __ballot_sync(FULL, p);
        total = __popc(b);
        return __popc(b & lanemask_lt());
    }
    __device__ __forceinline__ uint32_t scan_excl(uint32_t x, uint32_t& total) const {
        uint32_t v = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, v, d);
            if ((threadIdx.x & 31) >= (uint32_t)d) v += y;
        }
        total = __shfl_sync(FULL, v, 31);
        return v - x;
    }
    __device__ __forceinline__ uint32_t sum(uint32_t x) const {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(FULL, x, d);
        return x;
    }
    __device__ __forceinline__ uint32_t max(uint32_t x) const {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) x = ::max(x, __shfl_xor_sync(FULL, x, d));
        return x;
    }
    __device__ __forceinline__ bool any(bool p) const { return __any_sync(FULL, p); }
    __device__ __forceinline__ uint32_t or_all(uint32_t x) const {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) x |= __shfl_xor_sync(FULL, x, d);
        return x;
    }
};

// Block-wide collectives over shared scratch `sm` (>= 40 words).  Out of line: a block team calls
// them from dozens of places, and inlining every copy made the update kernel's code far larger than
// the instruction cache.
static __device__ __noinline__ uint2 block_scan_excl(uint32_t* sm, uint32_t x) {  // {exclusive prefix, total}
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    uint32_t v = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, v, d);
        if (lane >= (uint32_t)d) v += y;
    }
    if (lane == 31) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < nw ? sm[lane] : 0, s = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, s, d);
            if (lane >= (uint32_t)d) s += y;
        }
        if (lane < nw) sm[lane] = s - t;
        if (lane == 31) sm[32] = s;
    }
    __syncthreads();
    const uint2 r = make_uint2(sm[w] + v - x, sm[32]);
    __syncthreads();
    return r;
}
static __device__ __noinline__ uint32_t block_max(uint32_t* sm, uint32_t x) {
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x = ::max(x, __shfl_xor_sync(FULL, x, d));
    if (lane == 0) sm[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < nw ? sm[lane] : 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) t = ::max(t, __shfl_xor_sync(FULL, t, d));
        if (lane == 0) sm[32] = t;
    }
    __syncthreads();
    const uint32_t r = sm[32];
    __syncthreads();
    return r;
}
static __device__ __noinline__ uint32_t block_or(uint32_t* sm, uint32_t x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x |= __shfl_xor_sync(FULL, x, d);
    if (threadIdx.x == 0) sm[33] = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicOr(&sm[33], x);
    __syncthreads();
    const uint32_t r = sm[33];
    __syncthreads();
    return r;
}

// Block team; needs `sm` = shared scratch of at least 40 words, private to the team.
struct BlockTeam {
    uint32_t* sm;
    __device__ __forceinline__ uint32_t size() const { return blockDim.x; }
    __device__ __forceinline__ uint32_t rank() const { return threadIdx.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ uint32_t scan_excl(uint32_t x, uint32_t& total) const {
        const uint2 r = block_scan_excl(sm, x);
        total = r.y;
        return r.x;
    }
    __device__ __forceinline__ uint32_t scan_pred(bool p, uint32_t& total) const { return scan_excl(p ? 1u : 0u, total); }
    __device__ __forceinline__ uint32_t sum(uint32_t x) const { return block_scan_excl(sm, x).y; }
    __device__ __forceinline__ uint32_t max(uint32_t x) const { return block_max(sm, x); }
    __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
    __device__ __forceinline__ uint32_t or_all(uint32_t x) const { return block_or(sm, x); }
};
#endif  // __CUDACC__

}  // namespace bingo
