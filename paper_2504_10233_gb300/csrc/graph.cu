// Graph creation from CSR (Section 4.1, sampling space construction; Section 5.1,
// adaptive group representation), destruction, state export and reports.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bingo_host.h"
#include "groups.cuh"

using namespace bingo;

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

namespace bingo {
const char* last_error_cstr();
}

// ------------------------------------------------------------------------------------------- kernels

// Integer biases: 1 <= w < 2^max_bits.  Real biases (real = true) were checked by k_split_biases;
// their degree must stay below REAL_MAX_DEG.
__global__ void k_validate_csr(uint32_t n, uint32_t dst_n, uint64_t m, const uint64_t* __restrict__ rp,
                               const uint32_t* __restrict__ col, const uint32_t* __restrict__ bias, uint32_t max_bits,
                               bool real, uint32_t* status) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t j = tid; j < m; j += nt) {
        const uint32_t w = bias[j];
        bad |= col[j] >= dst_n || (!real && (w == 0 || (max_bits < 32 && (w >> max_bits) != 0)));
    }
    const uint64_t dlim = real ? REAL_MAX_DEG : 0xFFFFFFFFull;
    for (uint64_t v = tid; v < n; v += nt) {
        const uint64_t a = rp[v], b = rp[v + 1];
        bad |= b < a || b - a >= dlim;
    }
    if (tid == 0) bad |= rp[0] != 0 || rp[n] != m;
    if (bad) atomicOr(status, ST_INVALID);
}

// Real biases (Section 4.3): integer parts I[j] (factorised like integer biases) and decimal parts q[j].
__global__ void k_split_biases(const uint32_t* __restrict__ bits, uint64_t m, double lambda, uint32_t* __restrict__ I,
                               uint8_t* __restrict__ q, uint32_t* status) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t j = tid; j < m; j += nt) {
        uint32_t ii, qq;
        bad |= !split_real_bias(bits[j], lambda, ii, qq);
        I[j] = ii;
        q[j] = (uint8_t)qq;
    }
    if (bad) atomicOr(status, ST_INVALID);
}

// Radix base 4: every bias replaced by its sub-group mask (slot 3 i + v - 1 per nonzero digit).
__global__ void k_b4_masks(const uint32_t* __restrict__ w, uint64_t m, uint32_t* __restrict__ out) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = tid; j < m; j += nt) out[j] = b4_mask(w[j]);
}

// Per vertex: d, |G_k| (Eq. dwi / wpk by ballot over 32-edge chunks), mask, kinds (Eq. group),
// |S| and the words its blocks need.  One warp per vertex.
__global__ void k_build_count(DevGraph G, const uint64_t* __restrict__ rp, const uint32_t* __restrict__ bias,
                              uint64_t* __restrict__ words) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = warp; v < G.n; v += nwarps) {
        const uint32_t ov = G.order ? G.order[v] : (uint32_t)v;  // the caller's row of internal vertex v
        const uint64_t a = rp[ov];
        const uint32_t d = (uint32_t)(rp[ov + 1] - a);
        uint32_t c = 0;  // lane k: |G_k|
        for (uint32_t b = 0; b < d; b += 32) {
            const uint32_t w = (b + lane < d) ? bias[a + b + lane] : 0u;
#pragma unroll
            for (int k = 0; k < 32; k++) {
                const uint32_t bb = __ballot_sync(FULL, (w >> k) & 1u);
                if (lane == (uint32_t)k) c += __popc(bb);
            }
        }
        cnt_ref(G, v, lane) = c;
        gref_ref(G, v, lane) = 0;
        const uint32_t kd = kind_of(c, d, G.alpha, G.beta);
        const uint32_t mask = __ballot_sync(FULL, c > 0);
        const uint32_t regm = __ballot_sync(FULL, kd == K_REGULAR);
        const uint32_t spm = __ballot_sync(FULL, kd == K_SPARSE);
        uint32_t nsp = 0;
        if (spm) {
            for (uint32_t b = 0; b < d; b += 32) {
                const uint32_t w = (b + lane < d) ? bias[a + b + lane] : 0u;
                nsp += __popc(__ballot_sync(FULL, (w & spm) != 0u));
            }
        }
        if (lane == 0) {
            const uint32_t capa = capa_for(d);
            const uint32_t caps = spm ? caps_for(nsp) : 0;
            uint64_t wd = (uint64_t)4 * capa + (uint64_t)__popc(regm) * 4 * capa;
            if (G.fbits && capa) wd += dec_words(capa);
            if (spm) wd += 2ull * capa + (uint64_t)__popc(spm) * 4 * caps;
            words[v] = wd;
            VHdr h;
            h.adj = 0;
            h.deg = d;
            h.mask = mask;
            h.sref = 0;
            h.nsp = nsp;
            h.lcapa = capa ? (uint8_t)(log2_u32(capa) + 1) : 0;
            h.lcaps = caps ? (uint8_t)(log2_u32(caps) + 1) : 0;
            h.pad = 0;
            store_hdr(G, v, h);
            G.vh[v].word = G.order ? G.order[v] : G.base + (uint32_t)v;  // read by the walker for path entries
        }
    }
}

// Copy edges into the vertex's adjacency block and build its group structures.
__global__ void k_build_fill(DevGraph G, const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col,
                             const uint32_t* __restrict__ bias, const uint8_t* __restrict__ dec,
                             const uint64_t* __restrict__ offs, uint64_t base) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    WarpTeam t;
    for (uint64_t v = warp; v < G.n; v += nwarps) {
        VHdr h = load_hdr(G, v);
        const uint32_t d = h.deg, capa = capa_of(h), caps = caps_of(h);
        const uint64_t a = rp[G.order ? G.order[v] : (uint32_t)v];  // edge ids stay the caller's CSR positions
        uint64_t next = base + offs[v];
        const uint32_t c = cnt_ref(G, v, lane);
        const uint32_t kd = kind_of(c, d, G.alpha, G.beta);
        const uint32_t regm = __ballot_sync(FULL, kd == K_REGULAR);
        const uint32_t spm = __ballot_sync(FULL, kd == K_SPARSE);
        const uint32_t onem = __ballot_sync(FULL, kd == K_ONE);
        uint32_t gref = 0;
        if (d) {
            h.adj = next;
            uint2* pairs = adj_pairs(G, h.adj);
            uint64_t* eids = adj_eids(G, h.adj, capa);
            for (uint32_t j = lane; j < d; j += 32) {
                pairs[j] = make_uint2(G.perm ? G.perm[col[a + j]] : col[a + j], bias[a + j]);
                eids[j] = a + j;
            }
            next += 4ull * capa;
            if (G.fbits) {  // decimal block: q per slot; slot 31 = {Q_D, block}
                uint8_t* qb = reinterpret_cast<uint8_t*>(G.pool.base + next);
                uint32_t qs = 0;
                for (uint32_t j = lane; j < d; j += 32) {
                    qb[j] = dec[a + j];
                    qs += dec[a + j];
                }
                qs = __reduce_add_sync(FULL, qs);
                if (lane == DEC_SLOT) gref = ref_of(next);
                if (qs) h.mask |= 1u << DEC_SLOT;
                if (lane == 0) cnt_ref(G, v, DEC_SLOT) = qs;
                next += dec_words(capa);
            }
        }
        __syncwarp();
        for (uint32_t m = regm; m; m &= m - 1) {
            const uint32_t k = __ffs(m) - 1;
            build_regular(t, G, h.adj, d, k, next, capa);
            if (lane == k) gref = ref_of(next);
            next += 4ull * capa;
        }
        if (spm) {
            h.sref = next;
            const uint32_t ns = build_slist(t, G, h.adj, d, spm, h.sref, capa);
            next += 2ull * capa;
            __syncwarp();
            for (uint32_t m = spm; m; m &= m - 1) {
                const uint32_t k = __ffs(m) - 1;
                build_sparse(t, G, h.adj, h.sref, ns, k, next, caps);
                if (lane == k) gref = ref_of(next);
                next += 4ull * caps;
            }
        }
        for (uint32_t m = onem; m; m &= m - 1) {
            const uint32_t k = __ffs(m) - 1;
            const uint32_t s = find_one(t, G, h.adj, d, k);
            if (lane == k) gref = s < d ? adj_pairs(G, h.adj)[s].x : NONE32;  // the member's destination
        }
        gref_ref(G, v, lane) = gref;
        __syncwarp();
        // the hot line: copies of the hot pairs, the total outside them, the scan order (the decimal
        // slot's count was written above)
        write_hot(G, v, lane, cnt_ref(G, v, lane), gref, G.vh[v].word);
        if (lane == 0) store_hdr(G, v, h);
    }
}

// ---- internal numbering ----------------------------------------------------------------------------------

// BINGO_ORDER_AUTO renumbers every graph by degree (partition graphs keep the caller's ids): the
// most visited hot records then share lines and pages, which measured 15% faster walks on RMAT-26
// with uniform biases; the order table costs 4 bytes a vertex (walk starts and last vertices).
constexpr uint32_t ORDER_AUTO_MAX_N = 0x7FFFFFFFu;

// Sort keys of the degree numbering: a stable ascending sort of (2^32 - 1 - out-degree) orders the
// vertices by descending out-degree, ties by the caller's id.
__global__ void k_order_keys(uint32_t n, const uint64_t* __restrict__ rp, uint64_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = tid; v < n; v += nt) {
        const uint64_t d = rp[v + 1] - rp[v];
        keys[v] = 0xFFFFFFFFull - (d < 0xFFFFFFFFull ? d : 0xFFFFFFFFull);
        vals[v] = (uint32_t)v;
    }
}

__global__ void k_order_perm(uint32_t n, const uint32_t* __restrict__ order, uint32_t* __restrict__ perm) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = tid; i < n; i += nt) perm[order[i]] = (uint32_t)i;
}

// ---- export ----------------------------------------------------------------------------------------------

// Export row i is the caller's vertex ids[i] (ids null: vertex i), for i < count.
__global__ void k_export_sizes(DevGraph G, const uint32_t* __restrict__ ids, uint64_t count,
                               uint64_t* __restrict__ deg64, uint64_t* __restrict__ glen64,
                               uint64_t* __restrict__ nsp64) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < count; i += nwarps) {
        const uint64_t ve = ids ? ids[i] : i;  // the caller's id
        const uint64_t v = G.perm ? G.perm[ve] : ve;
        const VHdr h = load_hdr(G, v);
        const uint32_t c = cnt_ref(G, v, lane);
        const uint32_t kd = slot_kind(G, c, h.deg, lane);
        glen64[i * 32 + lane] = is_list(kd) ? c : 0;
        if (lane == 0) {
            deg64[i] = h.deg;
            nsp64[i] = h.sref ? h.nsp : 0;
        }
    }
}

__global__ void k_export_fill(DevGraph G, const uint32_t* __restrict__ ids, uint64_t count,
                              const uint64_t* __restrict__ eoff, const uint64_t* __restrict__ goff,
                              const uint64_t* __restrict__ soff, uint32_t* __restrict__ odst,
                              uint32_t* __restrict__ obias, uint64_t* __restrict__ oeid, uint8_t* __restrict__ okind,
                              uint32_t* __restrict__ oone, uint32_t* __restrict__ ocnt, uint32_t* __restrict__ omem,
                              uint32_t* __restrict__ ominv,
                              uint32_t* __restrict__ osp, uint32_t* __restrict__ ospinv,
                              unsigned long long* __restrict__ bad) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < count; i += nwarps) {
        const uint64_t ve = ids ? ids[i] : i;  // the caller's id
        const uint64_t v = G.perm ? G.perm[ve] : ve;
        const VHdr h = load_hdr(G, v);
        const uint32_t d = h.deg, capa = capa_of(h), caps = caps_of(h);
        if (d) {
            const uint2* pairs = adj_pairs(G, h.adj);
            const uint64_t* eids = adj_eids(G, h.adj, capa);
            for (uint32_t j = lane; j < d; j += 32) {
                const uint2 e = pairs[j];
                odst[eoff[i] + j] = G.order ? G.order[e.x] : e.x;
                obias[eoff[i] + j] = G.base4 ? b4_value(e.y) : e.y;
                oeid[eoff[i] + j] = eids[j];
            }
        }
        const uint32_t c = cnt_ref(G, v, lane);
        const uint32_t kd = slot_kind(G, c, d, lane);
        const uint32_t gr = gref_ref(G, v, lane);
        // the walker's hot line: copies of the hot pairs, the total outside them, the scan order and
        // the caller's id
        uint64_t wc;
        bool desc;
        uint32_t hp;
        hot_summary(G, c, lane, wc, desc, hp);
        const uint32_t hw = G.vh[v].word, hs = hot_slot(hp, lane);
        const bool copy_bad = hs < 4 && (G.vh[v].g[hs].x != c || G.vh[v].g[hs].y != gr);
        if (__any_sync(FULL, copy_bad) && lane == 0) atomicAdd(bad, 1ull);
        if (lane == 0 && (wc != G.vh[v].wcold || hp != G.vh[v].hp || (hw & WORD_ID) != G.base + (uint32_t)ve ||
                          ((hw & WORD_DESC) != 0) != desc))
            atomicAdd(bad, 1ull);
        okind[i * 32 + lane] = (uint8_t)kd;
        ocnt[i * 32 + lane] = c;
        uint32_t one_slot = NONE32;
        if (kd == K_ONE) {  // the stored reference is the destination; locate the member's slot
            const uint2* pairs = adj_pairs(G, h.adj);
            for (uint32_t j = 0; j < d; j++)
                if ((pairs[j].y >> lane) & 1u) { one_slot = j; break; }
            if (one_slot == NONE32 || pairs[one_slot].x != gr) atomicAdd(bad, 1ull);
        }
        oone[i * 32 + lane] = one_slot;
        const uint32_t listm = __ballot_sync(FULL, is_list(kd));
        for (uint32_t m = listm; m; m &= m - 1) {
            const uint32_t k = __ffs(m) - 1;
            const uint64_t g = words_of(__shfl_sync(FULL, gr, k));
            const uint32_t ck = __shfl_sync(FULL, c, k);
            const uint32_t kk = __shfl_sync(FULL, kd, k);
            const uint32_t icap = kk == K_REGULAR ? capa : caps;
            const uint32_t* mdst = G.pool.base + g;
            const uint32_t* mem = mdst + icap;
            const uint32_t* inv = mem + icap;
            const uint64_t o = goff[i * 32 + k];
            const uint2* pairs = adj_pairs(G, h.adj);
            const uint32_t* S = h.sref ? G.pool.base + h.sref : nullptr;
            for (uint32_t t = lane; t < ck; t += 32) {
                const uint32_t x = mem[t];
                omem[o + t] = x;
                ominv[o + t] = x < icap ? inv[x] : NONE32;
                // the stored destination must be the member's edge destination
                uint32_t slot = x;
                if (kk == K_SPARSE) slot = (S && x < h.nsp) ? S[x] : NONE32;
                if (slot >= d || pairs[slot].x != mdst[t]) atomicAdd(bad, 1ull);
            }
        }
        if (h.sref) {
            const uint32_t* S = G.pool.base + h.sref;
            const uint32_t* Sinv = S + capa;
            for (uint32_t t = lane; t < h.nsp; t += 32) {
                const uint32_t x = S[t];
                osp[soff[i] + t] = x;
                ospinv[soff[i] + t] = x < capa ? Sinv[x] : NONE32;
            }
        }
    }
}

// Decimal parts per edge in export order (real-bias graphs); counts slots whose Q_D disagrees.
__global__ void k_export_dec(DevGraph G, const uint64_t* __restrict__ eoff, uint8_t* __restrict__ oq,
                             unsigned long long* __restrict__ bad) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t ve = warp; ve < G.n; ve += nwarps) {
        const uint64_t v = G.perm ? G.perm[ve] : ve;
        const VHdr h = load_hdr(G, v);
        const uint32_t ref = gref_ref(G, v, DEC_SLOT);
        uint32_t qs = 0;
        if (h.deg && ref) {
            const uint8_t* qb = dec_bytes(G, ref);
            for (uint32_t j = lane; j < h.deg; j += 32) {
                oq[eoff[ve] + j] = qb[j];
                qs += qb[j];
            }
        }
        qs = __reduce_add_sync(FULL, qs);
        const bool flag = ((h.mask >> DEC_SLOT) & 1u) != (qs != 0);
        if (lane == 0 && (qs != cnt_ref(G, v, DEC_SLOT) || flag || (h.deg && !ref))) atomicAdd(bad, 1ull);
    }
}

// memory by structure: [0] adjacency words, [1] regular group words, [2] sparse words
__global__ void k_memory(DevGraph G, unsigned long long* out) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long a = 0, r = 0, s = 0;
    for (uint64_t v = warp; v < G.n; v += nwarps) {
        const VHdr h = load_hdr(G, v);
        const uint32_t capa = capa_of(h), caps = caps_of(h);
        const uint32_t kd = slot_kind(G, cnt_ref(G, v, lane), h.deg, lane);
        const uint32_t regm = __ballot_sync(FULL, kd == K_REGULAR), spm = __ballot_sync(FULL, kd == K_SPARSE);
        if (lane == 0) {
            a += 4ull * capa + (G.fbits && capa ? dec_words(capa) : 0ull);
            r += (unsigned long long)__popc(regm) * 4 * capa;
            if (h.sref) s += 2ull * capa + (unsigned long long)__popc(spm) * 4 * caps;
        }
    }
    if (lane == 0) {
        atomicAdd(out + 0, a);
        atomicAdd(out + 1, r);
        atomicAdd(out + 2, s);
    }
}

// ------------------------------------------------------------------------------------------- host

static unsigned grid_for(const bingo_graph* g, uint64_t work_items, unsigned block) {
    uint64_t b = (work_items + block - 1) / block;
    uint64_t cap = (uint64_t)g->num_sms * 16;
    if (b > cap) b = cap;
    if (b == 0) b = 1;
    return (unsigned)b;
}

static void free_graph(bingo_graph* g) {
    if (!g) return;
    if (g->upd_graph) cudaGraphExecDestroy(g->upd_graph);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    for (cudaStream_t c : g->io_copy)
        if (c) cudaStreamDestroy(c);
    for (cudaEvent_t e : g->io_done)
        if (e) cudaEventDestroy(e);
    if (g->io_kernel) cudaEventDestroy(g->io_kernel);
    if (g->io_flags) cudaFreeHost((void*)g->io_flags);
    void* ptrs[] = {g->d_hdr, g->d_cold, g->d_upd, g->d_order, g->d_perm, g->d_pool, g->d_ctl, g->d_fcount, g->d_fstack, g->d_pending, g->d_eh};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    Buf* bufs[] = {&g->s_in, &g->s_keys, &g->s_keys2, &g->s_vals, &g->s_vals2, &g->s_tmp, &g->s_seg,
                   &g->s_rank, &g->s_best, &g->s_aux, &g->s_walk, &g->s_stage, &g->s_rec, &g->s_seginfo, &g->s_gcand, &g->s_gcand_cnt, &g->s_chunkmap,
                   &g->w_starts, &g->w_len, &g->w_pid, &g->w_paths, &g->w_plen, &g->w_pols, &g->w_chunk_done,
                   &g->w_len64, &g->w_off, &g->w_packed};
    for (Buf* b : bufs) release(*b);
    delete g;
}

// stage a host or device array on the device; returns the device pointer (maybe the input)
static bingo_status stage_in(const void* src, size_t bytes, Buf& buf, cudaStream_t s, const void** out) {
    if (bytes == 0 || is_device_ptr(src)) {
        *out = src;
        return BINGO_OK;
    }
    CK(ensure(buf, bytes), "staging allocation");
    CK(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, s), "staging copy");
    *out = buf.p;
    return BINGO_OK;
}

extern "C" {

const char* bingo_version(void) { return "bingo-gb300 0.1 (sm_103a)"; }

const char* bingo_last_error(void) { return bingo::last_error_cstr(); }

void bingo_default_config(bingo_config* c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->alpha_pct = 40;
    c->beta_pct = 10;
    c->max_bits = 32;
}

bingo_status bingo_create(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* bias,
                          const bingo_config* cfg, void* stream, bingo_graph** out) {
    if (!out) { set_error("out is NULL"); return BINGO_E_INVALID; }
    *out = nullptr;
    if (n == 0 || n >= 0x80000000u || !row_ptr || (m && (!col || !bias))) {
        set_error("invalid graph arguments (n=%u, m=%llu)", n, (unsigned long long)m);
        return BINGO_E_INVALID;
    }
    bingo_config c;
    bingo_default_config(&c);
    if (cfg) c = *cfg;
    if (c.max_bits == 0 || c.max_bits > 32 || c.alpha_pct > 100 || c.beta_pct > 100) {
        set_error("invalid config (max_bits=%u alpha=%u beta=%u)", c.max_bits, c.alpha_pct, c.beta_pct);
        return BINGO_E_INVALID;
    }
    const bool real = c.bias_format == BINGO_BIAS_F32;
    if (c.bias_format > BINGO_BIAS_F32 || (real && !(c.lambda > 0.0 && c.lambda < 1e300))) {
        set_error("invalid bias format %u / lambda %g", c.bias_format, c.lambda);
        return BINGO_E_INVALID;
    }
    if (c.vertex_order > BINGO_ORDER_DEGREE) {
        set_error("invalid vertex order %u", c.vertex_order);
        return BINGO_E_INVALID;
    }
    const bool part = c.vertex_base != 0 || c.dst_space != 0;
    const uint32_t dst_n = c.dst_space ? c.dst_space : n;
    if (part && (dst_n >= 0x80000000u || (uint64_t)c.vertex_base + n > dst_n || c.vertex_order == BINGO_ORDER_DEGREE)) {
        set_error("invalid partition (base %u, %u rows, destination space %u; caller vertex order only)",
                  c.vertex_base, n, dst_n);
        return BINGO_E_INVALID;
    }
    if (part) c.vertex_order = BINGO_ORDER_CALLER;
    if (c.hot_l2_hint > BINGO_HOT_NORMAL) {
        set_error("invalid hot_l2_hint %u", c.hot_l2_hint);
        return BINGO_E_INVALID;
    }
    if (c.radix_base == 0) c.radix_base = 2;
    const bool base4 = c.radix_base == 4;
    if ((c.radix_base != 2 && !base4) || (base4 && real)) {
        set_error("invalid radix base %u (2, or 4 with integer biases)", c.radix_base);
        return BINGO_E_INVALID;
    }
    if (base4 && c.max_bits > 2 * B4_POSITIONS) c.max_bits = 2 * B4_POSITIONS;  // biases below 4^10
    cudaStream_t s = (cudaStream_t)stream;
    bingo_graph* g = new bingo_graph();
    g->cfg = c;
    g->n = n;
    cudaGetDevice(&g->device);
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    cudaDeviceGetAttribute(&g->l2_bytes, cudaDevAttrL2CacheSize, g->device);
    bingo_status st = BINGO_OK;
    auto fail = [&](bingo_status x) { free_graph(g); return x; };
    const uint64_t* rp = nullptr;
    const uint32_t *cl = nullptr, *bs = nullptr;
    Buf brp, bcl, bbs, bint, bdec;
    auto release_stage = [&]() { release(brp); release(bcl); release(bbs); release(bint); release(bdec); };
    if ((st = stage_in(row_ptr, sizeof(uint64_t) * ((size_t)n + 1), brp, s, (const void**)&rp)) != BINGO_OK) { release_stage(); return fail(st); }
    if ((st = stage_in(col, sizeof(uint32_t) * m, bcl, s, (const void**)&cl)) != BINGO_OK) { release_stage(); return fail(st); }
    if ((st = stage_in(bias, sizeof(uint32_t) * m, bbs, s, (const void**)&bs)) != BINGO_OK) { release_stage(); return fail(st); }

    auto cu = [&](cudaError_t e, const char* what) -> bool {
        if (e != cudaSuccess) { st = cuda_fail(e, what); return false; }
        return true;
    };
    if (!cu(cudaMalloc(&g->d_ctl, CTL_WORDS * sizeof(uint64_t)), "control words") ||
        !cu(cudaMemsetAsync(g->d_ctl, 0, CTL_WORDS * sizeof(uint64_t), s), "control init")) { release_stage(); return fail(st); }
    uint64_t* ctl = (uint64_t*)g->d_ctl;
    uint32_t* status = (uint32_t*)(ctl + CTL_STATUS);
    const uint8_t* dq = nullptr;
    if (real && m) {  // split every real bias; the integer parts are factorised from here on
        if (!cu(ensure(bint, sizeof(uint32_t) * m), "integer parts") || !cu(ensure(bdec, m), "decimal parts")) {
            release_stage(); return fail(st);
        }
        k_split_biases<<<grid_for(g, m, 256), 256, 0, s>>>(bs, m, c.lambda, (uint32_t*)bint.p, (uint8_t*)bdec.p, status);
        g->launches++;
        bs = (const uint32_t*)bint.p;
        dq = (const uint8_t*)bdec.p;
    }
    k_validate_csr<<<grid_for(g, (m > n ? m : n), 256), 256, 0, s>>>(n, dst_n, m, rp, cl, bs, c.max_bits, real, status);
    g->launches++;
    if (base4 && m) {  // factorise the sub-group masks from here on (validation saw the biases)
        if (!cu(ensure(bint, sizeof(uint32_t) * m), "sub-group masks")) { release_stage(); return fail(st); }
        k_b4_masks<<<grid_for(g, m, 256), 256, 0, s>>>(bs, m, (uint32_t*)bint.p);
        g->launches++;
        bs = (const uint32_t*)bint.p;
    }
    uint32_t hst = 0;
    if (!cu(cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, s), "status read") ||
        !cu(cudaStreamSynchronize(s), "validate")) { release_stage(); return fail(st); }
    if (hst & ST_INVALID) {
        set_error(real ? "invalid CSR: ids >= n, real biases not finite / negative / zero-weight / lambda*b >= 2^31, "
                         "degree >= 2^24, or malformed row_ptr"
                       : "invalid CSR: ids >= n, zero or too-wide biases, or malformed row_ptr");
        release_stage();
        return fail(BINGO_E_INVALID);
    }
    if (!cu(cudaMalloc(&g->d_hdr, sizeof(VHot) * (size_t)n), "vertex records (hot)") ||
        !cu(cudaMalloc(&g->d_cold, sizeof(VCold) * (size_t)n), "vertex records (cold)") ||
        !cu(cudaMalloc(&g->d_upd, sizeof(VUpd) * (size_t)n), "vertex records (update fields)")) { release_stage(); return fail(st); }
    DevGraph& G = g->G;
    G.n = n;
    G.base = c.vertex_base;
    G.dst_n = dst_n;
    g->part = part;
    G.max_bits = c.max_bits;
    G.alpha = c.all_regular ? ALL_REGULAR : c.alpha_pct;
    G.beta = c.all_regular ? 0u : c.beta_pct;
    G.fbits = real ? FRAC_BITS : 0;
    G.lambda = real ? c.lambda : 0.0;
    G.base4 = base4 ? 1u : 0u;
    G.vh = (VHot*)g->d_hdr;
    G.vc = (VCold*)g->d_cold;
    G.vu = (VUpd*)g->d_upd;
    G.pool.status = status;
    G.pool.top = (unsigned long long*)(ctl + CTL_TOP);
    G.pool.npending = (unsigned long long*)(ctl + CTL_NPENDING);
    G.pool.leaked = (unsigned long long*)(ctl + CTL_LEAKED);

    G.order = nullptr;
    G.perm = nullptr;
    Buf words, offs, tot;
    auto release_all = [&]() { release(words); release(offs); release(tot); release_stage(); };
    if (n >= 1 && (c.vertex_order == BINGO_ORDER_DEGREE ||
                   (c.vertex_order == BINGO_ORDER_AUTO && n >= 2 && n <= ORDER_AUTO_MAX_N))) {
        // internal numbering by descending out-degree (read from row_ptr, which validation accepted)
        Buf k1, k2, v2;
        auto release_sort = [&]() { release(k1); release(k2); release(v2); };
        if (!cu(cudaMalloc(&g->d_order, sizeof(uint32_t) * (size_t)n), "vertex order") ||
            !cu(cudaMalloc(&g->d_perm, sizeof(uint32_t) * (size_t)n), "vertex permutation") ||
            !cu(ensure(k1, sizeof(uint64_t) * n), "order keys") || !cu(ensure(k2, sizeof(uint64_t) * n), "order keys") ||
            !cu(ensure(v2, sizeof(uint32_t) * n), "order values")) { release_sort(); release_all(); return fail(st); }
        k_order_keys<<<grid_for(g, n, 256), 256, 0, s>>>(n, rp, (uint64_t*)k1.p, (uint32_t*)g->d_order);
        g->launches++;
        bool alt = false;
        if (!cu(radix_sort_pairs((uint64_t*)k1.p, (uint32_t*)g->d_order, (uint64_t*)k2.p, (uint32_t*)v2.p, n, 32,
                                 g->s_tmp, s, &alt, &g->launches), "vertex order sort") ||
            (alt && !cu(cudaMemcpyAsync(g->d_order, v2.p, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s),
                        "vertex order copy"))) { release_sort(); release_all(); return fail(st); }
        k_order_perm<<<grid_for(g, n, 256), 256, 0, s>>>(n, (const uint32_t*)g->d_order, (uint32_t*)g->d_perm);
        g->launches++;
        if (!cu(cudaStreamSynchronize(s), "vertex order")) { release_sort(); release_all(); return fail(st); }
        release_sort();
        G.order = (const uint32_t*)g->d_order;
        G.perm = (const uint32_t*)g->d_perm;
    }
    g->cfg.vertex_order = G.order ? BINGO_ORDER_DEGREE : BINGO_ORDER_CALLER;
    if (!cu(ensure(words, sizeof(uint64_t) * n), "build words") || !cu(ensure(offs, sizeof(uint64_t) * n), "build offsets") ||
        !cu(ensure(tot, 64), "build total")) { release_all(); return fail(st); }
    const unsigned wblocks = grid_for(g, (uint64_t)n * 32, 256);
    k_build_count<<<wblocks, 256, 0, s>>>(G, rp, bs, (uint64_t*)words.p);
    g->launches++;
    if (!cu(scan_excl_u64((uint64_t*)words.p, (uint64_t*)offs.p, n, (uint64_t*)tot.p, g->s_tmp, s, &g->launches), "build scan")) {
        release_all(); return fail(st);
    }
    uint64_t total = 0;
    if (!cu(cudaMemcpyAsync(&total, tot.p, 8, cudaMemcpyDeviceToHost, s), "total read") ||
        !cu(cudaStreamSynchronize(s), "build count")) { release_all(); return fail(st); }
    const uint64_t base = 8;  // word 0..7 reserved: offset 0 means "no block"
    uint64_t need = base + total;
    uint64_t pool_words = c.pool_words;
    size_t fr = 0, tt = 0;
    cudaMemGetInfo(&fr, &tt);
    if (pool_words == 0) {
        pool_words = 2 * need + (256ull << 20);  // room for growth and for the per-batch worst-case check
        const uint64_t avail = fr > (4ull << 30) ? (fr - (4ull << 30)) / 4 : 0;
        if (pool_words > avail) pool_words = std::max<uint64_t>(need + (need >> 4), avail);
    }
    pool_words = (pool_words + 7) & ~7ull;
    if (pool_words > MAX_POOL_WORDS) pool_words = MAX_POOL_WORDS;  // 32-bit offsets in 32-byte units
    if (pool_words < need) {
        set_error("pool too small: need %llu words, have %llu", (unsigned long long)need, (unsigned long long)pool_words);
        release_all();
        return fail(BINGO_E_OOM);
    }
    if (!cu(cudaMalloc(&g->d_pool, pool_words * 4), "pool")) { release_all(); return fail(st); }
    G.pool.base = (uint32_t*)g->d_pool;
    G.pool.words = pool_words;
    // free lists
    uint64_t fcap = pool_words / 256;
    fcap = std::max<uint64_t>(4096, std::min<uint64_t>(fcap, 1ull << 19));
    const uint64_t pcap = 1ull << 20;
    if (!cu(cudaMalloc(&g->d_fcount, sizeof(long long) * NCLASS), "free counts") ||
        !cu(cudaMalloc(&g->d_fstack, sizeof(uint64_t) * NCLASS * fcap), "free stacks") ||
        !cu(cudaMalloc(&g->d_pending, sizeof(uint64_t) * pcap), "pending frees") ||
        !cu(cudaMemsetAsync(g->d_fcount, 0, sizeof(long long) * NCLASS, s), "free init")) { release_all(); return fail(st); }
    G.pool.fcount = (long long*)g->d_fcount;
    G.pool.fstack = (uint64_t*)g->d_fstack;
    G.pool.fcap = fcap;
    G.pool.pending = (uint64_t*)g->d_pending;
    G.pool.pcap = pcap;
    G.eh_key = nullptr;
    G.eh_cnt = nullptr;
    G.eh_mask = 0;
    if (!cu(cudaMemcpyAsync(G.pool.top, &need, 8, cudaMemcpyHostToDevice, s), "pool top")) { release_all(); return fail(st); }
    k_build_fill<<<wblocks, 256, 0, s>>>(G, rp, cl, bs, dq, (uint64_t*)offs.p, base);
    g->launches++;
    if (!cu(cudaGetLastError(), "build fill") || !cu(cudaStreamSynchronize(s), "build fill")) { release_all(); return fail(st); }
    release_all();
    // load the walker kernels of this weight format and resolve the allocation-free walk's scratch
    // now, so that no later walk call triggers a lazy module load (which can allocate device memory)
    if (!cu(walk_preload(g, s), "walker kernels preload") || !cu(cudaStreamSynchronize(s), "walker kernels preload"))
        return fail(st);
    if ((st = noalloc_prepare()) != BINGO_OK) return fail(st);
    g->m_live = m;
    g->next_eid = m;
    g->tune.lanes = c.lanes_per_walker ? c.lanes_per_walker : 1;
    g->tune.warps_per_block = c.warps_per_block ? c.warps_per_block : 8;
    g->tune.blocks_per_sm = c.blocks_per_sm;
    g->tune.occ = c.reg_variant ? 1 : 0;
    *out = g;
    return BINGO_OK;
}

bingo_status bingo_destroy(bingo_graph* g) {
    if (!g) return BINGO_OK;
    cudaDeviceSynchronize();
    free_graph(g);
    return BINGO_OK;
}

uint64_t bingo_kernel_launches(bingo_graph* g) { return g ? g->launches : 0; }

bingo_status bingo_get_config(bingo_graph* g, bingo_config* out) {
    if (!g || !out) { set_error("NULL argument"); return BINGO_E_INVALID; }
    *out = g->cfg;
    out->lanes_per_walker = g->tune.lanes;
    out->warps_per_block = g->tune.warps_per_block;
    out->blocks_per_sm = g->tune.blocks_per_sm;
    out->reg_variant = g->tune.occ;
    out->pool_words = g->G.pool.words;
    return BINGO_OK;
}

bingo_status bingo_set_walk_config(bingo_graph* g, uint32_t lanes, uint32_t wpb, uint32_t bps, uint32_t regv) {
    if (!g) { set_error("NULL graph"); return BINGO_E_INVALID; }
    if (!(lanes == 1 || lanes == 4 || lanes == 32) || wpb == 0 || wpb > 24 || regv > 1 || (regv && wpb > 8)) {
        set_error("invalid walk config (lanes %u, warps/block %u, register variant %u)", lanes, wpb, regv);
        return BINGO_E_INVALID;
    }
    g->tune.lanes = lanes;
    g->tune.warps_per_block = wpb;
    g->tune.blocks_per_sm = bps;
    g->tune.occ = regv;
    return BINGO_OK;
}

struct ExportPlan {
    Buf deg64, eoff, glen, goff, nsp, soff, tot;
    void release_all() {
        release(deg64); release(eoff); release(glen); release(goff); release(nsp); release(soff); release(tot);
    }
};

// Sizes and offsets of the export rows: row i is the caller's vertex ids[i] (device array; null =
// every vertex in id order), i < n.
static bingo_status export_plan(bingo_graph* g, ExportPlan& P, uint64_t totals[3], const uint32_t* ids = nullptr,
                                uint64_t count = ~0ull) {
    const uint64_t n = ids ? count : g->n;
    CK(ensure(P.deg64, 8 * n), "export");
    CK(ensure(P.eoff, 8 * n), "export");
    CK(ensure(P.glen, 8 * 32 * n), "export");
    CK(ensure(P.goff, 8 * 32 * n), "export");
    CK(ensure(P.nsp, 8 * n), "export");
    CK(ensure(P.soff, 8 * n), "export");
    CK(ensure(P.tot, 64), "export");
    cudaStream_t s = 0;
    k_export_sizes<<<grid_for(g, n * 32, 256), 256, 0, s>>>(g->G, ids, n, (uint64_t*)P.deg64.p, (uint64_t*)P.glen.p,
                                                            (uint64_t*)P.nsp.p);
    uint64_t* tot = (uint64_t*)P.tot.p;
    CK(scan_excl_u64((uint64_t*)P.deg64.p, (uint64_t*)P.eoff.p, n, tot + 0, g->s_tmp, s, &g->launches), "export scan");
    CK(scan_excl_u64((uint64_t*)P.glen.p, (uint64_t*)P.goff.p, 32 * n, tot + 1, g->s_tmp, s, &g->launches), "export scan");
    CK(scan_excl_u64((uint64_t*)P.nsp.p, (uint64_t*)P.soff.p, n, tot + 2, g->s_tmp, s, &g->launches), "export scan");
    CK(cudaMemcpy(totals, tot, 24, cudaMemcpyDeviceToHost), "export totals");
    return BINGO_OK;
}

bingo_status bingo_state_sizes_get(bingo_graph* g, bingo_state_sizes* out) {
    if (!g || !out) { set_error("NULL argument"); return BINGO_E_INVALID; }
    CK(cudaDeviceSynchronize(), "sync");
    ExportPlan P;
    uint64_t t[3];
    bingo_status st = export_plan(g, P, t);
    P.release_all();
    if (st != BINGO_OK) return st;
    uint64_t top = 0;
    CK(cudaMemcpy(&top, g->G.pool.top, 8, cudaMemcpyDeviceToHost), "pool top");
    out->n = g->n;
    out->m = t[0];
    out->list_entries = t[1];
    out->sparse_entries = t[2];
    out->pool_words_used = top;
    out->pool_words_total = g->G.pool.words;
    out->next_edge_id = g->next_eid;
    return BINGO_OK;
}

bingo_status bingo_export_decimal(bingo_graph* g, uint8_t* q) {
    if (!g) { set_error("NULL graph"); return BINGO_E_INVALID; }
    if (!g->G.fbits) { set_error("not a real-bias graph"); return BINGO_E_STATE; }
    CK(cudaDeviceSynchronize(), "sync");
    ExportPlan P;
    uint64_t t[3];
    bingo_status st = export_plan(g, P, t);
    if (st != BINGO_OK) { P.release_all(); return st; }
    const uint64_t m = t[0];
    Buf o;
    cudaError_t e = ensure(o, m + 64);
    if (e != cudaSuccess) { P.release_all(); return cuda_fail(e, "export staging"); }
    unsigned long long* obad = (unsigned long long*)o.p;
    uint8_t* oq = (uint8_t*)o.p + 16;
    e = cudaMemset(obad, 0, 8);
    if (e == cudaSuccess) {
        k_export_dec<<<grid_for(g, (uint64_t)g->n * 32, 256), 256>>>(g->G, (uint64_t*)P.eoff.p, oq, obad);
        e = cudaDeviceSynchronize();
    }
    unsigned long long nbad = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&nbad, obad, 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && q && m) e = cudaMemcpy(q, oq, m, cudaMemcpyDeviceToHost);
    release(o);
    P.release_all();
    if (e != cudaSuccess) return cuda_fail(e, "export copy");
    if (nbad) {
        set_error("export: %llu vertices whose decimal total or flag disagrees with their decimal parts", nbad);
        return BINGO_E_STATE;
    }
    return BINGO_OK;
}

}  // extern "C"

// Export rows i < count of the caller's vertices ids[i] (device array; null = every vertex, count = n)
// to host buffers, each nullable.
static bingo_status export_rows(bingo_graph* g, const uint32_t* ids, uint64_t count, uint32_t* deg, uint32_t* dst,
                                uint32_t* bias, uint64_t* eid, uint32_t* cnt, uint8_t* kind, uint32_t* one_slot,
                                uint32_t* glen, uint32_t* members, uint32_t* member_inv, uint32_t* sp_len,
                                uint32_t* sp_list, uint32_t* sp_inv) {
    CK(cudaDeviceSynchronize(), "sync");
    ExportPlan P;
    uint64_t t[3];
    bingo_status st = export_plan(g, P, t, ids, count);
    if (st != BINGO_OK) { P.release_all(); return st; }
    const uint64_t n = ids ? count : g->n, m = t[0], L = t[1], S = t[2];
    Buf o;
    // device staging: dst, bias (u32 m each), eid (u64 m), kind (u8 32n), one and cnt (u32 32n each), mem/minv (L),
    // sp/spinv (S)
    const size_t bytes = 8 * m + 8 * m + 32 * n + 8 * 32 * n + 8 * L + 8 * S + 128;
    cudaError_t e = ensure(o, bytes);
    if (e != cudaSuccess) { P.release_all(); return cuda_fail(e, "export staging"); }
    char* p = (char*)o.p;
    uint64_t* oeid = (uint64_t*)p; p += 8 * m;
    uint32_t* odst = (uint32_t*)p; p += 4 * m;
    uint32_t* obias = (uint32_t*)p; p += 4 * m;
    uint32_t* oone = (uint32_t*)p; p += 4 * 32 * n;
    uint32_t* ocnt = (uint32_t*)p; p += 4 * 32 * n;
    uint32_t* omem = (uint32_t*)p; p += 4 * L;
    uint32_t* ominv = (uint32_t*)p; p += 4 * L;
    uint32_t* osp = (uint32_t*)p; p += 4 * S;
    uint32_t* ospinv = (uint32_t*)p; p += 4 * S;
    uint8_t* okind = (uint8_t*)p; p += 32 * n;
    unsigned long long* obad = (unsigned long long*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
    cudaMemset(obad, 0, 8);
    k_export_fill<<<grid_for(g, n * 32, 256), 256>>>(g->G, ids, n, (uint64_t*)P.eoff.p, (uint64_t*)P.goff.p,
                                                     (uint64_t*)P.soff.p, odst, obias, oeid, okind, oone, ocnt, omem,
                                                     ominv, osp, ospinv, obad);
    e = cudaDeviceSynchronize();
    unsigned long long nbad = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&nbad, obad, 8, cudaMemcpyDeviceToHost);
    std::vector<uint64_t> tmp;
    auto d2h32 = [&](uint32_t* dsth, const void* src, uint64_t cnt64) -> cudaError_t {
        if (!dsth || cnt64 == 0) return cudaSuccess;
        return cudaMemcpy(dsth, src, 4 * cnt64, cudaMemcpyDeviceToHost);
    };
    if (e == cudaSuccess && deg) {
        tmp.resize(n);
        e = cudaMemcpy(tmp.data(), P.deg64.p, 8 * n, cudaMemcpyDeviceToHost);
        for (uint64_t v = 0; v < n && e == cudaSuccess; v++) deg[v] = (uint32_t)tmp[v];
    }
    if (e == cudaSuccess && sp_len) {
        tmp.resize(n);
        e = cudaMemcpy(tmp.data(), P.nsp.p, 8 * n, cudaMemcpyDeviceToHost);
        for (uint64_t v = 0; v < n && e == cudaSuccess; v++) sp_len[v] = (uint32_t)tmp[v];
    }
    if (e == cudaSuccess && glen) {
        tmp.resize(32 * n);
        e = cudaMemcpy(tmp.data(), P.glen.p, 8 * 32 * n, cudaMemcpyDeviceToHost);
        for (uint64_t i = 0; i < 32 * n && e == cudaSuccess; i++) glen[i] = (uint32_t)tmp[i];
    }
    if (e == cudaSuccess) e = d2h32(dst, odst, m);
    if (e == cudaSuccess) e = d2h32(bias, obias, m);
    if (e == cudaSuccess && eid && m) e = cudaMemcpy(eid, oeid, 8 * m, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = d2h32(cnt, ocnt, 32 * n);
    if (e == cudaSuccess && kind) e = cudaMemcpy(kind, okind, 32 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = d2h32(one_slot, oone, 32 * n);
    if (e == cudaSuccess) e = d2h32(members, omem, L);
    if (e == cudaSuccess) e = d2h32(member_inv, ominv, L);
    if (e == cudaSuccess) e = d2h32(sp_list, osp, S);
    if (e == cudaSuccess) e = d2h32(sp_inv, ospinv, S);
    release(o);
    P.release_all();
    if (e != cudaSuccess) return cuda_fail(e, "export copy");
    if (nbad) {
        set_error("export: %llu stored member destinations disagree with the adjacency", nbad);
        return BINGO_E_STATE;
    }
    return BINGO_OK;
}

// Upload and validate a host or device list of the caller's vertex ids.
static bingo_status stage_ids(bingo_graph* g, const uint32_t* ids, uint64_t count, Buf& b, const uint32_t** out) {
    if (!ids || count == 0 || count > (1ull << 31)) { set_error("export_vertices: need 1..2^31 vertex ids"); return BINGO_E_INVALID; }
    std::vector<uint32_t> h;
    const uint32_t* hp = ids;
    if (is_device_ptr(ids)) {
        h.resize(count);
        CK(cudaMemcpy(h.data(), ids, 4 * count, cudaMemcpyDeviceToHost), "export_vertices ids");
        hp = h.data();
    }
    for (uint64_t i = 0; i < count; i++)
        if (hp[i] >= g->n) { set_error("export_vertices: id %u at %llu is >= n", hp[i], (unsigned long long)i); return BINGO_E_INVALID; }
    CK(ensure(b, 4 * count), "export_vertices ids");
    CK(cudaMemcpy(b.p, hp, 4 * count, cudaMemcpyHostToDevice), "export_vertices ids");
    *out = (const uint32_t*)b.p;
    return BINGO_OK;
}

extern "C" {

bingo_status bingo_export_state(bingo_graph* g, uint32_t* deg, uint32_t* dst, uint32_t* bias, uint64_t* eid,
                                uint32_t* cnt, uint8_t* kind, uint32_t* one_slot, uint32_t* glen, uint32_t* members,
                                uint32_t* member_inv, uint32_t* sp_len, uint32_t* sp_list, uint32_t* sp_inv) {
    if (!g) { set_error("NULL graph"); return BINGO_E_INVALID; }
    return export_rows(g, nullptr, g->n, deg, dst, bias, eid, cnt, kind, one_slot, glen, members, member_inv, sp_len,
                       sp_list, sp_inv);
}

bingo_status bingo_export_vertices_sizes(bingo_graph* g, const uint32_t* ids, uint64_t count, uint64_t sizes[3]) {
    if (!g || !sizes) { set_error("NULL argument"); return BINGO_E_INVALID; }
    CK(cudaDeviceSynchronize(), "sync");
    Buf b;
    const uint32_t* dids = nullptr;
    bingo_status st = stage_ids(g, ids, count, b, &dids);
    if (st == BINGO_OK) {
        ExportPlan P;
        st = export_plan(g, P, sizes, dids, count);
        P.release_all();
    }
    release(b);
    return st;
}

bingo_status bingo_export_vertices(bingo_graph* g, const uint32_t* ids, uint64_t count, uint32_t* deg, uint32_t* dst,
                                   uint32_t* bias, uint64_t* eid, uint32_t* cnt, uint8_t* kind, uint32_t* one_slot,
                                   uint32_t* glen, uint32_t* members, uint32_t* member_inv, uint32_t* sp_len,
                                   uint32_t* sp_list, uint32_t* sp_inv) {
    if (!g) { set_error("NULL graph"); return BINGO_E_INVALID; }
    CK(cudaDeviceSynchronize(), "sync");
    Buf b;
    const uint32_t* dids = nullptr;
    bingo_status st = stage_ids(g, ids, count, b, &dids);
    if (st == BINGO_OK)
        st = export_rows(g, dids, count, deg, dst, bias, eid, cnt, kind, one_slot, glen, members, member_inv, sp_len,
                         sp_list, sp_inv);
    release(b);
    return st;
}

bingo_status bingo_memory_report(bingo_graph* g, uint64_t out[6]) {
    if (!g || !out) { set_error("NULL argument"); return BINGO_E_INVALID; }
    Buf b;
    CK(ensure(b, 64), "memory report");
    cudaMemset(b.p, 0, 64);
    k_memory<<<grid_for(g, (uint64_t)g->n * 32, 256), 256>>>(g->G, (unsigned long long*)b.p);
    unsigned long long w[3];
    cudaError_t e = cudaMemcpy(w, b.p, 24, cudaMemcpyDeviceToHost);
    release(b);
    if (e != cudaSuccess) return cuda_fail(e, "memory report");
    out[0] = 4ull * w[0];
    out[1] = (uint64_t)g->n * (sizeof(VHot) + sizeof(VCold) + sizeof(VUpd));
    out[2] = 4ull * w[1];
    out[3] = 4ull * w[2];
    out[4] = g->G.eh_mask ? (g->G.eh_mask + 1) * 12 : 0;
    out[5] = 4ull * g->G.pool.words;
    return BINGO_OK;
}

}  // extern "C"
