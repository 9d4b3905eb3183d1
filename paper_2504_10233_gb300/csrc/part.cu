// 1-D partitioned graphs and walks with walker migration (the paper's supplement on dynamic graph
// support and partitioning: vertices split into ranges, each range's edges held by its own owner,
// walkers transferred to the owner of the vertex they reach).
//
// A partition set holds one partition graph per contiguous range of global vertex ids, each built
// with the kernels of a whole graph (its rows are local vertices, its destinations global ids).
// A walk runs in supersteps: every partition's launch resumes the walkers standing on its vertices
// and runs each until it ends or steps onto another partition's vertex, where it leaves a 24-byte
// record {walker, vertex, previous vertex, step}; an exchange routes the records to their owners
// for the next superstep, until no walker is left.  Walker w draws from Philox counters
// (w, step, j) wherever it runs, so the paths equal those of the same walk on the whole graph.
// Updates are routed to the owner of their source and applied there with the batch pipeline.
// In this library every partition lives on the calling thread's device; the records that cross
// between partitions are the data another transport would move between devices.
#include <string.h>

#include <algorithm>
#include <vector>

#include "bingo_host.h"

using namespace bingo;

#define CK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

namespace bingo {
bingo_status edge_index_build(bingo_graph* g, cudaStream_t s);
}

struct bingo_partset {
    uint32_t n = 0, P = 0;
    int device = 0;
    int num_sms = 0;
    std::vector<uint32_t> bounds;      // P + 1 boundaries: partition p holds [bounds[p], bounds[p+1])
    std::vector<bingo_graph*> parts;
    bingo::Buf d_bounds, d_peh, d_pols, rec_in, rec_out, d_ctl;  // d_ctl: u64 [0] outbox count, [1..P] counts, [P+1..2P] fills
    uint64_t supersteps = 0;           // of the last walk
};

namespace {

__device__ __forceinline__ uint32_t owner_of(const uint32_t* bounds, uint32_t P, uint32_t v) {
    uint32_t lo = 0, hi = P;  // last p with bounds[p] <= v
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (bounds[mid] <= v) lo = mid; else hi = mid;
    }
    return lo;
}

// Start records of every walker (invalid starts end at once: one-vertex path, the status flagged).
__global__ void k_part_start(uint64_t nwalkers, const uint32_t* __restrict__ starts, uint32_t n, uint32_t stride,
                             uint32_t pad, uint32_t* __restrict__ paths, uint32_t* __restrict__ plen,
                             PartRec* __restrict__ out, unsigned long long* __restrict__ nout,
                             uint32_t* __restrict__ status) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwalkers; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = starts[i];
        if (s >= n) {
            atomicOr(status, ST_INVALID);
            uint32_t* row = paths + i * (uint64_t)stride;
            row[0] = s;
            if (pad)
                for (uint32_t t = 1; t < stride; t++) row[t] = NONE32;
            plen[i] = 1;
            continue;
        }
        PartRec r;
        r.wid = i;
        r.cur = s;
        r.prev = NONE32;
        r.step = 0;
        r.pad = 0;
        out[atomicAdd(nout, 1ull)] = r;
    }
}

// Records per owner partition.
__global__ void k_part_count(const PartRec* __restrict__ rec, const unsigned long long* __restrict__ nrec,
                             const uint32_t* __restrict__ bounds, uint32_t P, unsigned long long* __restrict__ cnt) {
    const uint64_t n = *nrec;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + owner_of(bounds, P, rec[i].cur), 1ull);
}

// Every record to its owner's region of the inbox (regions at off[p], filled through fill[p]).
__global__ void k_part_scatter(const PartRec* __restrict__ rec, const unsigned long long* __restrict__ nrec,
                               const uint32_t* __restrict__ bounds, uint32_t P, const unsigned long long* __restrict__ off,
                               unsigned long long* __restrict__ fill, PartRec* __restrict__ inbox) {
    const uint64_t n = *nrec;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const PartRec r = rec[i];
        const uint32_t p = owner_of(bounds, P, r.cur);
        inbox[off[p] + atomicAdd(fill + p, 1ull)] = r;
    }
}

unsigned grid_of(const bingo_partset* ps, uint64_t items) {
    const uint64_t b = (items + 255) / 256;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, (uint64_t)ps->num_sms * 8));
}

void free_set(bingo_partset* ps) {
    for (bingo_graph* g : ps->parts)
        if (g) bingo_destroy(g);
    Buf* bs[] = {&ps->d_bounds, &ps->d_peh, &ps->d_pols, &ps->rec_in, &ps->rec_out, &ps->d_ctl};
    for (Buf* b : bs) release(*b);
    delete ps;
}

bingo_status check_set_device(const bingo_partset* ps, const char* who) {
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, who);
    if (dev != ps->device) {
        set_error("%s: the current device is %d but the partitions live on device %d", who, dev, ps->device);
        return BINGO_E_INVALID;
    }
    return BINGO_OK;
}

}  // namespace

extern "C" {

bingo_status bingo_part_create(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col,
                               const uint32_t* bias, const bingo_config* cfg, uint32_t nparts, const uint32_t* bounds,
                               void* stream, bingo_partset** out) {
    if (!out) { set_error("part_create: out is NULL"); return BINGO_E_INVALID; }
    *out = nullptr;
    if (n == 0 || n >= 0x80000000u || !row_ptr || (m && (!col || !bias)) || nparts == 0 || nparts > n || nparts > 1024) {
        set_error("part_create: invalid arguments (n=%u, parts=%u)", n, nparts);
        return BINGO_E_INVALID;
    }
    bingo_config c;
    bingo_default_config(&c);
    if (cfg) c = *cfg;
    if (c.bias_format != BINGO_BIAS_U32 || (c.radix_base != 0 && c.radix_base != 2)) {
        set_error("part_create: partitioned graphs take integer biases in radix base 2");
        return BINGO_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint64_t> rp(n + 1);
    if (is_device_ptr(row_ptr)) CK(cudaMemcpy(rp.data(), row_ptr, 8ull * (n + 1), cudaMemcpyDeviceToHost), "part_create row_ptr");
    else memcpy(rp.data(), row_ptr, 8ull * (n + 1));
    if (rp[0] != 0 || rp[n] != m) { set_error("part_create: row_ptr must run from 0 to m"); return BINGO_E_INVALID; }
    for (uint32_t v = 0; v < n; v++)
        if (rp[v + 1] < rp[v]) { set_error("part_create: row_ptr decreases at %u", v); return BINGO_E_INVALID; }
    bingo_partset* ps = new bingo_partset();
    ps->n = n;
    ps->P = nparts;
    cudaGetDevice(&ps->device);
    cudaDeviceGetAttribute(&ps->num_sms, cudaDevAttrMultiProcessorCount, ps->device);
    ps->bounds.resize(nparts + 1);
    if (bounds) {
        for (uint32_t p = 0; p <= nparts; p++) ps->bounds[p] = bounds[p];
    } else {  // contiguous ranges with (nearly) equal edge counts, each at least one vertex
        ps->bounds[0] = 0;
        for (uint32_t p = 1; p < nparts; p++) {
            const uint64_t target = m * p / nparts;
            uint32_t v = (uint32_t)(std::lower_bound(rp.begin(), rp.end(), target) - rp.begin());
            ps->bounds[p] = std::min<uint32_t>(std::max<uint32_t>(v, ps->bounds[p - 1] + 1), n - (nparts - p));
        }
    }
    ps->bounds[nparts] = n;
    for (uint32_t p = 0; p < nparts; p++)
        if (ps->bounds[p] >= ps->bounds[p + 1] || (p == 0 && ps->bounds[0] != 0)) {
            set_error("part_create: boundaries must increase strictly from 0 to n");
            free_set(ps);
            return BINGO_E_INVALID;
        }
    ps->parts.assign(nparts, nullptr);
    for (uint32_t p = 0; p < nparts; p++) {
        const uint32_t lo = ps->bounds[p], hi = ps->bounds[p + 1];
        std::vector<uint64_t> sub(hi - lo + 1);
        for (uint32_t v = lo; v <= hi; v++) sub[v - lo] = rp[v] - rp[lo];
        bingo_config cp = c;
        cp.vertex_base = lo;
        cp.dst_space = n;
        cp.vertex_order = BINGO_ORDER_CALLER;
        const bingo_status st = bingo_create(hi - lo, rp[hi] - rp[lo], sub.data(), col ? col + rp[lo] : nullptr,
                                             bias ? bias + rp[lo] : nullptr, &cp, stream, &ps->parts[p]);
        if (st != BINGO_OK) {
            free_set(ps);
            return st;
        }
    }
    cudaError_t e = ensure(ps->d_bounds, 4ull * (nparts + 1));
    if (e == cudaSuccess) e = cudaMemcpyAsync(ps->d_bounds.p, ps->bounds.data(), 4ull * (nparts + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = ensure(ps->d_ctl, 8ull * (2 * nparts + 2));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free_set(ps);
        return cuda_fail(e, "part_create");
    }
    *out = ps;
    return BINGO_OK;
}

bingo_status bingo_part_destroy(bingo_partset* ps) {
    if (!ps) return BINGO_OK;
    cudaDeviceSynchronize();
    free_set(ps);
    return BINGO_OK;
}

bingo_status bingo_part_info(bingo_partset* ps, uint32_t p, bingo_graph** graph, uint32_t* lo, uint32_t* hi) {
    if (!ps || p >= ps->P) { set_error("part_info: no partition %u", p); return BINGO_E_INVALID; }
    if (graph) *graph = ps->parts[p];
    if (lo) *lo = ps->bounds[p];
    if (hi) *hi = ps->bounds[p + 1];
    return BINGO_OK;
}

bingo_status bingo_part_apply_updates(bingo_partset* ps, const bingo_update* ups, uint64_t count, void* stream,
                                      bingo_update_stats* stats) {
    if (!ps) { set_error("NULL partition set"); return BINGO_E_INVALID; }
    bingo_status st = check_set_device(ps, "part_apply_updates");
    if (st != BINGO_OK) return st;
    if (count && !ups) { set_error("NULL update array"); return BINGO_E_INVALID; }
    if (stats) memset(stats, 0, sizeof(*stats));
    if (count == 0) return BINGO_OK;
    std::vector<bingo_update> h(count);
    if (is_device_ptr(ups)) CK(cudaMemcpy(h.data(), ups, sizeof(bingo_update) * count, cudaMemcpyDeviceToHost), "part_apply_updates");
    else memcpy(h.data(), ups, sizeof(bingo_update) * count);
    // the whole batch is validated before any partition changes (the partitions' own checks repeat it)
    const uint32_t mb = ps->parts[0]->cfg.max_bits;
    for (uint64_t i = 0; i < count; i++) {
        const bingo_update& u = h[i];
        const bool ins = u.op == BINGO_OP_INSERT || u.op == BINGO_OP_SET_BIAS;
        if (u.src >= ps->n || u.dst >= ps->n || u.op > 2 || (ins && (u.bias == 0 || (mb < 32 && (u.bias >> mb) != 0)))) {
            set_error("part_apply_updates: invalid record %llu (id >= n, op > 2, or bias outside [1, 2^max_bits)); batch rejected",
                      (unsigned long long)i);
            return BINGO_E_INVALID;
        }
    }
    // route each record to the owner of its source, local source id, batch order kept
    std::vector<std::vector<bingo_update>> per(ps->P);
    for (const bingo_update& u : h) {
        const uint32_t p = (uint32_t)(std::upper_bound(ps->bounds.begin(), ps->bounds.end(), u.src) - ps->bounds.begin()) - 1;
        bingo_update l = u;
        l.src -= ps->bounds[p];
        per[p].push_back(l);
    }
    for (uint32_t p = 0; p < ps->P; p++) {
        if (per[p].empty()) continue;
        bingo_update_stats sp;
        st = bingo_apply_updates(ps->parts[p], per[p].data(), per[p].size(), stream, &sp);
        if (st != BINGO_OK) return st;
        if (stats) {
            stats->inserted += sp.inserted;
            stats->deleted += sp.deleted;
            stats->not_found += sp.not_found;
            for (int a = 0; a < 5; a++)
                for (int b = 0; b < 5; b++) stats->conversions[a][b] += sp.conversions[a][b];
            stats->vertices_touched += sp.vertices_touched;
            stats->groups_rebuilt += sp.groups_rebuilt;
        }
    }
    return BINGO_OK;
}

bingo_status bingo_part_walk(bingo_partset* ps, uint64_t nwalkers, const uint32_t* starts, const uint32_t* lengths,
                             const uint8_t* policy_ids, const bingo_policy* policies, uint32_t npolicies, uint64_t seed,
                             uint32_t stride, uint32_t* paths, uint32_t* path_len, uint32_t mode, void* stream) {
    if (!ps) { set_error("NULL partition set"); return BINGO_E_INVALID; }
    bingo_status st = check_set_device(ps, "part_walk");
    if (st != BINGO_OK) return st;
    if ((mode & 0xFF) != BINGO_WALK_PERSISTENT || stride == 0) {
        set_error("part_walk: persistent form only, stride >= 1");
        return BINGO_E_INVALID;
    }
    bool need_n2v = false;
    uint32_t max_len = 0;
    st = check_policies(policies, npolicies, stride, lengths != nullptr, &need_n2v, &max_len);
    if (st != BINGO_OK) return st;
    ps->supersteps = 0;
    if (nwalkers == 0) return BINGO_OK;
    if (!starts || !paths || !path_len || !is_device_ptr(starts) || !is_device_ptr(paths) || !is_device_ptr(path_len) ||
        (lengths && !is_device_ptr(lengths)) || (policy_ids && !is_device_ptr(policy_ids))) {
        set_error("part_walk: starts, lengths, policy ids, paths and path_len must be device pointers");
        return BINGO_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t P = ps->P;
    if (need_n2v) {  // every partition's edge index, and a table of them for probes at the previous vertex's owner
        std::vector<PartEH> tab(P);
        for (uint32_t p = 0; p < P; p++) {
            bingo_graph* g = ps->parts[p];
            if (g->G.eh_mask == 0 && (st = edge_index_build(g, s)) != BINGO_OK) return st;
            tab[p].key = g->G.eh_key;
            tab[p].cnt = g->G.eh_cnt;
            tab[p].mask = g->G.eh_mask;
        }
        CK(ensure(ps->d_peh, sizeof(PartEH) * P), "part_walk probe table");
        CK(cudaMemcpyAsync(ps->d_peh.p, tab.data(), sizeof(PartEH) * P, cudaMemcpyHostToDevice, s), "part_walk probe table");
    }
    CK(ensure(ps->d_pols, sizeof(bingo_policy) * npolicies), "part_walk policies");
    CK(cudaMemcpyAsync(ps->d_pols.p, policies, sizeof(bingo_policy) * npolicies, cudaMemcpyHostToDevice, s), "part_walk policies");
    CK(ensure(ps->rec_in, sizeof(PartRec) * nwalkers), "part_walk records");
    CK(ensure(ps->rec_out, sizeof(PartRec) * nwalkers), "part_walk records");
    unsigned long long* ctl = (unsigned long long*)ps->d_ctl.p;  // [0] outbox count, [1..P] counts, [P+1..2P] fills
    PartRec* rin = (PartRec*)ps->rec_in.p;
    PartRec* rout = (PartRec*)ps->rec_out.p;
    const uint32_t* dbounds = (const uint32_t*)ps->d_bounds.p;
    const bool pad = !(mode & BINGO_WALK_NO_PAD);
    CK(cudaMemsetAsync(ctl, 0, 8ull * (2 * P + 1), s), "part_walk counters");
    k_part_start<<<grid_of(ps, nwalkers), 256, 0, s>>>(nwalkers, starts, ps->n, stride, pad ? 1u : 0u, paths, path_len,
                                                     rout, ctl, (uint32_t*)((uint64_t*)ps->parts[0]->d_ctl + CTL_STATUS));
    std::vector<unsigned long long> cnt(P), off(P + 1);
    for (;;) {
        // route the outbox to the owners: counts, then regions of the inbox
        CK(cudaMemsetAsync(ctl + 1, 0, 8ull * 2 * P, s), "part_walk counters");
        k_part_count<<<grid_of(ps, nwalkers), 256, 0, s>>>(rout, ctl, dbounds, P, ctl + 1);
        CK(cudaMemcpyAsync(cnt.data(), ctl + 1, 8ull * P, cudaMemcpyDeviceToHost, s), "part_walk counts");
        CK(cudaStreamSynchronize(s), "part_walk");
        off[0] = 0;
        for (uint32_t p = 0; p < P; p++) off[p + 1] = off[p] + cnt[p];
        if (off[P] == 0) break;
        if (ps->supersteps > (uint64_t)stride * (P + 1) + 4) {  // each superstep advances every walker by a step
            set_error("part_walk: walkers still moving after %llu supersteps", (unsigned long long)ps->supersteps);
            return BINGO_E_STATE;
        }
        CK(cudaMemcpyAsync(ctl + 1, off.data(), 8ull * P, cudaMemcpyHostToDevice, s), "part_walk offsets");
        k_part_scatter<<<grid_of(ps, off[P]), 256, 0, s>>>(rout, ctl, dbounds, P, ctl + 1, ctl + 1 + P, rin);
        CK(cudaMemsetAsync(ctl, 0, 8, s), "part_walk counters");
        // one superstep: every partition resumes its walkers until each ends or leaves
        for (uint32_t p = 0; p < P; p++) {
            if (!cnt[p]) continue;
            bingo_graph* g = ps->parts[p];
            WalkReq q;
            q.nwalkers = cnt[p];
            q.lengths = lengths;
            q.pids = policy_ids;
            q.dev_pols = (const bingo_policy*)ps->d_pols.p;
            q.npol = npolicies;
            q.seed = seed;
            q.stride = stride;
            q.paths = paths;
            q.plen = path_len;
            q.mode = BINGO_WALK_PERSISTENT;
            q.pad = pad;
            q.max_steps = lengths ? stride - 1 : max_len;
            q.queue = (unsigned long long*)((uint64_t*)g->d_ctl + CTL_QUEUE);
            q.resume = rin + off[p];
            q.outbox = rout;
            q.nout = ctl;
            q.peh = need_n2v ? (const PartEH*)ps->d_peh.p : nullptr;
            q.bounds = dbounds;
            q.npart = P;
            if ((st = walk_launch(g, q, s)) != BINGO_OK) return st;
        }
        ps->supersteps++;
    }
    return BINGO_OK;
}

bingo_status bingo_part_check(bingo_partset* ps, void* stream) {
    if (!ps) { set_error("NULL partition set"); return BINGO_E_INVALID; }
    bingo_status worst = BINGO_OK;
    for (bingo_graph* g : ps->parts) {
        const bingo_status st = bingo_check(g, stream);
        if (st != BINGO_OK && worst == BINGO_OK) worst = st;
    }
    return worst;
}

uint64_t bingo_part_supersteps(bingo_partset* ps) { return ps ? ps->supersteps : 0; }

}  // extern "C"
