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
constexpr int MAX_N2V_TRIES = 1 << 14;
constexpr uint32_t WF_PAD = 1u;  // pad path rows with 0xFFFFFFFF

struct WalkParams {
    uint64_t nwalkers;
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
    // stepwise state
    uint32_t* s_cur;
    uint32_t* s_prev;
};

// Identity of a walker: Philox key, local id (the counter's walker field) and policy.
struct WalkerId {
    uint2 key;
    uint64_t lid;
    uint32_t pid;
};

__device__ __forceinline__ WalkerId walker_id(const WalkParams& A, uint64_t wid) {
    WalkerId w;
    if (A.req_off) {
        uint32_t lo = 0, hi = A.nreq;  // last r with req_off[r] <= wid
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(A.req_off + mid) <= wid) lo = mid; else hi = mid;
        }
        const uint64_t k = __ldg(A.req_key + lo);
        w.key = make_uint2((uint32_t)k, (uint32_t)(k >> 32));
        w.lid = wid - __ldg(A.req_off + lo);
        w.pid = lo;
    } else {
        w.key = A.key;
        w.lid = wid;
        w.pid = A.pids ? __ldg(A.pids + wid) : 0u;
    }
    return w;
}

struct PolicyRegs {
    uint32_t kind, max_len, stop;
    uint64_t a0, a1, a2;
};
__device__ __forceinline__ PolicyRegs load_policy(const bingo_policy* p) {
    PolicyRegs r;
    r.kind = __ldg(&p->kind);
    r.max_len = __ldg(&p->max_len);
    r.stop = __ldg(&p->ppr_stop_u32);
    r.a0 = __ldg(reinterpret_cast<const unsigned long long*>(&p->n2v_accept[0]));
    r.a1 = __ldg(reinterpret_cast<const unsigned long long*>(&p->n2v_accept[1]));
    r.a2 = __ldg(reinterpret_cast<const unsigned long long*>(&p->n2v_accept[2]));
    return r;
}

__device__ __forceinline__ VHdr ld_hdr(const VHdr* p) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    const uint4 a = __ldg(q), b = __ldg(q + 1);
    VHdr h;
    h.adj = ((uint64_t)a.y << 32) | a.x;
    h.deg = a.z;
    h.mask = a.w;
    h.sref = ((uint64_t)b.y << 32) | b.x;
    h.nsp = b.z;
    h.lcapa = (uint8_t)(b.w & 0xFF);
    h.lcaps = (uint8_t)((b.w >> 8) & 0xFF);
    h.pad = 0;
    return h;
}

// --------------------------------------------------------------------------------- group selection
// All variants pick k* = min{k : sum_{j<=k} 2^j |G_j| > r} with r uniform in [0, sum_j 2^j |G_j|),
// i.e. group k with probability W(p_k) / sum W (Eq. group_prob); they differ only in how a team
// of T lanes shares the count line.

// T = 1: one lane per walker; the count line is read as 16-byte vectors, only where the mask has bits.
__device__ __forceinline__ void select_group_1(const DevGraph& G, uint32_t v, uint32_t mask, StepRng& R,
                                               uint32_t& ks, uint32_t& cs, uint32_t* status) {
    const uint4* line = reinterpret_cast<const uint4*>(G.cnt + (uint64_t)v * 32);
    uint64_t part[8];
    uint64_t tot = 0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        part[q] = 0;
        if ((mask >> (4 * q)) & 0xFu) {
            const uint4 x = __ldg(line + q);
            part[q] = ((uint64_t)x.x << (4 * q)) + ((uint64_t)x.y << (4 * q + 1)) + ((uint64_t)x.z << (4 * q + 2)) +
                      ((uint64_t)x.w << (4 * q + 3));
        }
        tot += part[q];
    }
    const uint64_t r = below64(R, tot, status);
    uint64_t acc = 0;
    int qs = 7;
    uint64_t base = 0;
    bool found = false;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const uint64_t nacc = acc + part[q];
        const bool hit = !found && r < nacc;
        qs = hit ? q : qs;
        base = hit ? acc : base;
        found |= hit;
        acc = nacc;
    }
    const uint4 x = __ldg(line + qs);
    const uint32_t c4[4] = {x.x, x.y, x.z, x.w};
    ks = 4 * qs + 3;
    cs = x.w;
    found = false;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        base += (uint64_t)c4[j] << (4 * qs + j);
        const bool hit = !found && r < base;
        ks = hit ? (uint32_t)(4 * qs + j) : ks;
        cs = hit ? c4[j] : cs;
        found |= hit;
    }
}

// T = 4: lane t of the team owns groups [8t, 8t+8) (one 32-byte sector of the line); a
// two-level shuffle prefix over the team, a ballot finds the lane holding k*.
__device__ __forceinline__ void select_group_4(const DevGraph& G, uint32_t v, uint32_t mask, StepRng& R,
                                               uint32_t& ks, uint32_t& cs, uint32_t* status, uint32_t tl,
                                               uint32_t team_mask, uint32_t team_base) {
    const uint4* line = reinterpret_cast<const uint4*>(G.cnt + (uint64_t)v * 32);
    uint32_t c[8];
    uint64_t s = 0;
    const uint32_t byte = (mask >> (8 * tl)) & 0xFFu;
    uint4 x0 = make_uint4(0, 0, 0, 0), x1 = make_uint4(0, 0, 0, 0);
    if (byte & 0x0Fu) x0 = __ldg(line + 2 * tl);
    if (byte & 0xF0u) x1 = __ldg(line + 2 * tl + 1);
    c[0] = x0.x; c[1] = x0.y; c[2] = x0.z; c[3] = x0.w;
    c[4] = x1.x; c[5] = x1.y; c[6] = x1.z; c[7] = x1.w;
#pragma unroll
    for (int j = 0; j < 8; j++) s += (uint64_t)c[j] << (8 * tl + j);
    uint64_t incl = s;
#pragma unroll
    for (int d = 1; d < 4; d <<= 1) {
        const uint64_t y = __shfl_up_sync(team_mask, incl, d, 4);
        if (tl >= (uint32_t)d) incl += y;
    }
    const uint64_t tot = __shfl_sync(team_mask, incl, team_base + 3);
    const uint64_t r = below64(R, tot, status);
    const uint64_t excl = incl - s;
    const bool mine = r < incl && r >= excl;
    const uint32_t b = __ballot_sync(team_mask, mine) & team_mask;
    const uint32_t owner = __ffs(b) - 1;
    uint32_t k_l = 8 * tl + 7, c_l = c[7];
    uint64_t acc = excl;
    bool found = false;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        acc += (uint64_t)c[j] << (8 * tl + j);
        const bool hit = !found && r < acc;
        k_l = hit ? 8 * tl + j : k_l;
        c_l = hit ? c[j] : c_l;
        found |= hit;
    }
    ks = __shfl_sync(team_mask, k_l, owner);
    cs = __shfl_sync(team_mask, c_l, owner);
}

// T = 32: lane k owns group k; a warp-wide shuffle prefix of W_k = 2^k |G_k| and a ballot of
// (prefix > r) give k* as the first set bit.
__device__ __forceinline__ void select_group_32(const DevGraph& G, uint32_t v, uint32_t mask, StepRng& R,
                                                uint32_t& ks, uint32_t& cs, uint32_t* status, uint32_t lane) {
    const uint32_t c = ((mask >> lane) & 1u) ? __ldg(G.cnt + (uint64_t)v * 32 + lane) : 0u;
    uint64_t incl = (uint64_t)c << lane;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(FULL, incl, d);
        if (lane >= (uint32_t)d) incl += y;
    }
    const uint64_t tot = __shfl_sync(FULL, incl, 31);
    const uint64_t r = below64(R, tot, status);
    const uint32_t b = __ballot_sync(FULL, r < incl);
    ks = __ffs(b) - 1;
    cs = __shfl_sync(FULL, c, ks);
}

// --------------------------------------------------------------------------------- intra-group pick
// Uniform member of G_k* (Eq. pvp): stored index (one-element), uniform position of the member list
// (regular), of the sparse group's list of sparse-list positions (sparse), or rejection over the whole
// neighbour list accepting a slot whose bias has bit k* (dense).  Returns the destination vertex.
__device__ __forceinline__ uint32_t pick_member(const DevGraph& G, const VHdr& h, uint32_t v, uint32_t ks,
                                                uint32_t cs, StepRng& R, uint32_t* status) {
    const uint32_t kd = kind_of(cs, h.deg, G.alpha, G.beta);
    const uint2* pairs = adj_pairs(G, h.adj);
    if (kd == K_DENSE) {
        for (int t = 0; t < MAX_DENSE_TRIES; t++) {
            const uint32_t j = below32(R, h.deg, status);
            const uint2 e = __ldg(pairs + j);
            if ((e.y >> ks) & 1u) return e.x;
        }
        atomicOr(status, ST_TIMEOUT);
        return NONE32;
    }
    const uint64_t gr = __ldg(G.gref + (uint64_t)v * 32 + ks);
    uint32_t slot;
    if (kd == K_ONE) {
        slot = (uint32_t)gr;
    } else {
        const uint32_t pos = below32(R, cs, status);
        slot = __ldg(G.pool.base + (gr & GOFF_MASK) + pos);
        if (kd == K_SPARSE) {
            if (slot >= h.nsp) { atomicOr(status, ST_STATE); return NONE32; }
            slot = __ldg(G.pool.base + h.sref + slot);
        }
    }
    if (slot >= h.deg) { atomicOr(status, ST_STATE); return NONE32; }  // state inconsistent: never index past d
    return __ldg(reinterpret_cast<const uint32_t*>(pairs + slot));
}

// One step of a walker at `cur`.  Returns false if the walk ends here (PPR stop, no out-edge, error).
template <int T>
__device__ __forceinline__ bool walk_step(const DevGraph& G, const WalkParams& A, const PolicyRegs& P, uint2 key,
                                          uint64_t lid, uint32_t step, uint32_t& cur, uint32_t& prev, uint32_t tl,
                                          uint32_t team_mask, uint32_t team_base, uint32_t lane) {
    StepRng R;
    R.init(key, lid, step);
    if (P.kind == BINGO_PPR && R.next() < P.stop) return false;
    const VHdr h = ld_hdr(G.hdr + cur);
    if (h.deg == 0) return false;
    for (int attempt = 0; attempt < MAX_N2V_TRIES; attempt++) {
        uint32_t ks, cs;
        if constexpr (T == 1) select_group_1(G, cur, h.mask, R, ks, cs, A.status);
        else if constexpr (T == 4) select_group_4(G, cur, h.mask, R, ks, cs, A.status, tl, team_mask, team_base);
        else select_group_32(G, cur, h.mask, R, ks, cs, A.status, lane);
        const uint32_t x = pick_member(G, h, cur, ks, cs, R, A.status);
        if (x >= G.n) {
            if (x != NONE32) atomicOr(A.status, ST_STATE);
            return false;
        }
        if (P.kind == BINGO_NODE2VEC && prev != NONE32) {
            const uint64_t u = R.next();
            bool acc;
            if (x == prev) {
                acc = u < P.a0;
            } else {
                const uint64_t a1 = P.a1, a2 = P.a2;
                const uint64_t lo = a1 < a2 ? a1 : a2, hi = a1 < a2 ? a2 : a1;
                if (u < lo) acc = true;        // accepted at either distance: no probe needed
                else if (u >= hi) acc = false; // rejected at either distance
                else acc = u < (eh_lookup(G, prev, x) ? a1 : a2);
            }
            if (!acc) continue;
        }
        prev = cur;
        cur = x;
        return true;
    }
    atomicOr(A.status, ST_TIMEOUT);
    return false;
}

__device__ __forceinline__ void finish_walker(const WalkParams& A, uint64_t wid, uint32_t steps, uint32_t tl,
                                              uint32_t T) {
    uint32_t* row = A.paths + wid * (uint64_t)A.stride;
    if (tl == 0) A.plen[wid] = steps + 1;
    if (A.flags & WF_PAD)
        for (uint32_t t = steps + 1 + tl; t < A.stride; t += T) row[t] = NONE32;
}

template <int T>
__global__ void __launch_bounds__(1024) k_walk_persistent(DevGraph G, WalkParams A) {
    const uint32_t lane = threadIdx.x & 31, tl = lane % T, team = lane / T;
    const uint32_t team_base = team * T;
    const uint32_t team_mask = (T == 32) ? FULL : (((1u << T) - 1u) << team_base);
    uint64_t wid = 0;
    WalkerId W;
    W.key = make_uint2(0, 0);
    W.lid = 0;
    W.pid = 0;
    PolicyRegs P;
    uint32_t cur = 0, prev = NONE32, step = 0, L = 0;
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
                if (!have && mine < A.nwalkers) {
                    wid = mine;
                    W = walker_id(A, wid);
                    if (W.pid >= A.npol) { W.pid = 0; atomicOr(A.status, ST_INVALID); }
                    P = load_policy(A.pols + W.pid);
                    cur = __ldg(A.starts + wid);
                    L = A.lengths ? __ldg(A.lengths + wid) : P.max_len;
                    if (L + 1 > A.stride) { L = A.stride - 1; atomicOr(A.status, ST_INVALID); }
                    if (cur >= G.n) { L = 0; atomicOr(A.status, ST_INVALID); }
                    prev = NONE32;
                    step = 0;
                    have = true;
                    if (tl == 0) A.paths[wid * (uint64_t)A.stride] = cur;
                    if (L == 0) {
                        finish_walker(A, wid, 0, tl, T);
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
            const bool took = walk_step<T>(G, A, P, W.key, W.lid, step, cur, prev, tl, team_mask, team_base, lane);
            if (took) {
                step++;
                if (tl == 0) A.paths[wid * (uint64_t)A.stride + step] = cur;
            }
            if (!took || step == L) {
                finish_walker(A, wid, step, tl, T);
                have = false;
            }
        }
    }
}

// The paper's step-by-step form (Section 6 (iii)): one launch per step, one thread per walker.
__global__ void k_walk_step(DevGraph G, WalkParams A, uint32_t s) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t wid = tid; wid < A.nwalkers; wid += nt) {
        WalkerId W = walker_id(A, wid);
        if (W.pid >= A.npol) W.pid = 0;
        const PolicyRegs P = load_policy(A.pols + W.pid);
        uint32_t L = A.lengths ? __ldg(A.lengths + wid) : P.max_len;
        if (L + 1 > A.stride) L = A.stride - 1;
        uint32_t cur, prev;
        if (s == 0) {
            cur = __ldg(A.starts + wid);
            prev = NONE32;
            if (cur >= G.n) { L = 0; atomicOr(A.status, ST_INVALID); }
            A.paths[wid * (uint64_t)A.stride] = cur;
            if (L == 0) {
                finish_walker(A, wid, 0, 0, 1);
                A.s_cur[wid] = NONE32;
                continue;
            }
        } else {
            cur = A.s_cur[wid];
            if (cur == NONE32) continue;
            prev = A.s_prev[wid];
        }
        const bool took = walk_step<1>(G, A, P, W.key, W.lid, s, cur, prev, 0, 0, 0, 0);
        if (took) A.paths[wid * (uint64_t)A.stride + s + 1] = cur;
        if (!took || s + 1 == L) {
            finish_walker(A, wid, took ? s + 1 : s, 0, 1);
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
        const VHdr h = G.hdr[v];
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

static int g_occ_cache[3][33];

static int walk_blocks_per_sm(int lanes, int wpb) {
    int li = lanes == 1 ? 0 : lanes == 4 ? 1 : 2;
    if (wpb < 1 || wpb > 32) return 1;
    if (g_occ_cache[li][wpb]) return g_occ_cache[li][wpb];
    int nb = 0;
    const int threads = wpb * 32;
    if (lanes == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_walk_persistent<1>, threads, 0);
    else if (lanes == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_walk_persistent<4>, threads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_walk_persistent<32>, threads, 0);
    if (nb < 1) nb = 1;
    g_occ_cache[li][wpb] = nb;
    return nb;
}

// Launch the walk on device buffers (all pointers device).  Pre: policies validated.
bingo_status walk_launch(bingo_graph* g, const WalkReq& q, cudaStream_t s) {
    WalkParams A;
    memset(&A, 0, sizeof(A));
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
    if (nwalkers == 0) return BINGO_OK;
    if (mode == BINGO_WALK_STEPWISE) {
        CK(ensure(g->s_walk, 8 * nwalkers), "walk state");
        A.s_cur = (uint32_t*)g->s_walk.p;
        A.s_prev = A.s_cur + nwalkers;
        const unsigned blocks = (unsigned)std::min<uint64_t>((nwalkers + 255) / 256, (uint64_t)g->num_sms * 8);
        for (uint32_t st = 0; st < (max_steps ? max_steps : 1); st++) {
            k_walk_step<<<blocks, 256, 0, s>>>(g->G, A, st);
            g->launches++;
        }
        CK(cudaGetLastError(), "stepwise walk launch");
        return BINGO_OK;
    }
    CK(cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), s), "walk queue reset");
    g->launches++;
    const int lanes = (int)g->tune.lanes, wpb = (int)g->tune.warps_per_block;
    int bps = (int)g->tune.blocks_per_sm;
    const int occ = walk_blocks_per_sm(lanes, wpb);
    if (bps <= 0 || bps > occ) bps = occ;
    uint64_t blocks = (uint64_t)g->num_sms * bps;
    const uint64_t walkers_per_block = (uint64_t)wpb * (32 / lanes);
    const uint64_t useful = (nwalkers + walkers_per_block - 1) / walkers_per_block;
    if (blocks > useful) blocks = useful;
    if (blocks == 0) blocks = 1;
    if (lanes == 1) k_walk_persistent<1><<<(unsigned)blocks, wpb * 32, 0, s>>>(g->G, A);
    else if (lanes == 4) k_walk_persistent<4><<<(unsigned)blocks, wpb * 32, 0, s>>>(g->G, A);
    else k_walk_persistent<32><<<(unsigned)blocks, wpb * 32, 0, s>>>(g->G, A);
    g->launches++;
    CK(cudaGetLastError(), "walk launch");
    return BINGO_OK;
}

}  // namespace bingo
