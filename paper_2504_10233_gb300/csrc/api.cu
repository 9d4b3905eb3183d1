// C-ABI entry points for walks, the walker autotuner and device-status checks.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <thread>
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

bingo_status check_policies(const bingo_policy* pols, uint32_t npol, uint32_t stride, bool have_lengths,
                            bool* need_n2v, uint32_t* max_len) {
    if (!pols || npol == 0 || npol > MAX_POL) {
        set_error("policies: need 1..%u entries", MAX_POL);
        return BINGO_E_INVALID;
    }
    *need_n2v = false;
    *max_len = 0;
    for (uint32_t i = 0; i < npol; i++) {
        const bingo_policy& p = pols[i];
        if (p.kind > BINGO_NODE2VEC) { set_error("policy %u: unknown kind %u", i, p.kind); return BINGO_E_INVALID; }
        if (p.kind == BINGO_NODE2VEC) {
            *need_n2v = true;
            for (int d = 0; d < 3; d++)
                if (p.n2v_accept[d] > (1ull << 32)) { set_error("policy %u: n2v_accept > 2^32", i); return BINGO_E_INVALID; }
        }
        if (!have_lengths && (uint64_t)p.max_len + 1 > stride) {
            set_error("policy %u: max_len %u does not fit stride %u", i, p.max_len, stride);
            return BINGO_E_INVALID;
        }
        *max_len = std::max(*max_len, p.max_len);
    }
    return BINGO_OK;
}

bingo_status check_device(const bingo_graph* g, const char* who) {
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, who);
    if (dev != g->device) {
        set_error("%s: the current device is %d but the graph lives on device %d", who, dev, g->device);
        return BINGO_E_INVALID;
    }
    return BINGO_OK;
}

}  // namespace bingo

namespace {

// Host-output walk whose download overlaps the walk.  The one persistent launch counts finished
// walkers per id-ordered chunk (walkers are taken from the queue in id order, so chunks finish
// roughly in order), and the walker that completes a chunk writes this call's sequence number into
// the chunk's flag in host-mapped pinned memory.  This thread issues each chunk's download as soon
// as its flag shows, on WALK_IO_STREAMS copy streams in turn, so copies run while later chunks still
// walk.  Once the kernel has ended (its event completes; every loop in it is bounded) the remaining
// chunks are downloaded without looking at their flags, so the host never waits on a flag alone.
// The caller's stream waits for the last download.
bingo_status walk_host_io_overlap(bingo_graph* g, WalkReq q, uint32_t* paths, uint32_t* path_len,
                                  bool host_paths, bool host_plen, cudaStream_t s) {
    for (int k = 0; k < WALK_IO_STREAMS; k++) {
        if (!g->io_copy[k]) CK(cudaStreamCreateWithFlags(&g->io_copy[k], cudaStreamNonBlocking), "download stream");
        if (!g->io_done[k]) CK(cudaEventCreateWithFlags(&g->io_done[k], cudaEventDisableTiming), "walk event");
    }
    if (!g->io_kernel) CK(cudaEventCreateWithFlags(&g->io_kernel, cudaEventDisableTiming), "walk event");
    if (!g->io_flags) {
        void* h = nullptr;
        CK(cudaHostAlloc(&h, sizeof(uint32_t) * WALK_IO_MAX_CHUNKS, cudaHostAllocMapped), "chunk flags");
        memset(h, 0, sizeof(uint32_t) * WALK_IO_MAX_CHUNKS);
        void* d = nullptr;
        const cudaError_t e = cudaHostGetDevicePointer(&d, h, 0);
        if (e != cudaSuccess) { cudaFreeHost(h); return cuda_fail(e, "chunk flags"); }
        g->io_flags = (volatile uint32_t*)h;
        g->io_flags_dev = (uint32_t*)d;
    }
    const uint64_t n = q.nwalkers, stride = q.stride;
    uint32_t shift = WALK_IO_MIN_SHIFT;
    while (((n + (1ull << shift) - 1) >> shift) > WALK_IO_MAX_CHUNKS) shift++;
    const uint32_t nch = (uint32_t)((n + (1ull << shift) - 1) >> shift);
    CK(ensure(g->w_chunk_done, sizeof(uint32_t) * WALK_IO_MAX_CHUNKS), "chunk counters");
    CK(cudaMemsetAsync(g->w_chunk_done.p, 0, sizeof(uint32_t) * nch, s), "chunk counters");
    if (++g->io_seq == 0) g->io_seq = 1;  // flags hold earlier calls' numbers, never this one's
    q.chunk_done = (uint32_t*)g->w_chunk_done.p;
    q.host_flags = g->io_flags_dev;
    q.chunk_shift = shift;
    q.io_seq = g->io_seq;
    bingo_status st = walk_launch(g, q, s);
    if (st != BINGO_OK) return st;
    CK(cudaEventRecord(g->io_kernel, s), "walk event");
    // on a failed call below, wait for the copies already issued so that none lands after the return
    auto fail = [&](cudaError_t e, const char* what) {
        for (cudaStream_t c : g->io_copy) cudaStreamSynchronize(c);
        return cuda_fail(e, what);
    };
    // after the kernel: every copy stream orders its remaining downloads behind it
    auto after_kernel = [&]() {
        for (cudaStream_t c : g->io_copy) {
            const cudaError_t w = cudaStreamWaitEvent(c, g->io_kernel, 0);
            if (w != cudaSuccess) return w;
        }
        return cudaSuccess;
    };
    bool kernel_done = false;
    for (uint32_t c = 0; c < nch; c++) {
        while (!kernel_done && g->io_flags[c] != g->io_seq) {
            const cudaError_t e = cudaEventQuery(g->io_kernel);
            if (e == cudaSuccess) {
                kernel_done = true;
                const cudaError_t w = after_kernel();
                if (w != cudaSuccess) return fail(w, "walk event");
            } else if (e != cudaErrorNotReady) {
                return fail(e, "walk");
            } else {
                std::this_thread::yield();
            }
        }
        const uint64_t lo = (uint64_t)c << shift, cnt = std::min<uint64_t>(1ull << shift, n - lo);
        cudaStream_t cs = g->io_copy[c % WALK_IO_STREAMS];
        cudaError_t e = cudaSuccess;
        if (host_paths)
            e = cudaMemcpyAsync(paths + lo * stride, q.paths + lo * stride, 4 * cnt * stride, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && host_plen)
            e = cudaMemcpyAsync(path_len + lo, q.plen + lo, 4 * cnt, cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) return fail(e, "paths download");
    }
    if (!kernel_done) {
        const cudaError_t w = after_kernel();
        if (w != cudaSuccess) return fail(w, "walk event");
    }
    for (int k = 0; k < WALK_IO_STREAMS; k++) {
        CK(cudaEventRecord(g->io_done[k], g->io_copy[k]), "walk event");
        CK(cudaStreamWaitEvent(s, g->io_done[k], 0), "walk event");
    }
    return BINGO_OK;
}

// Philox4x32-10 of the walker on `count` (counter, key) tuples.
__global__ void k_philox_eval(uint64_t count, const uint4* ctr, const uint2* key, uint4* out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = philox4x32_10(ctr[i], key[i]);
}

// The draws one walker makes at one step, in the order the walker consumes them: its raw u32
// stream (range 0), or successive exact uniform integers in [0, range) (the bounded draws of group
// selection and member picks).
__global__ void k_walker_draws(uint2 key, uint64_t walker, uint32_t step, uint64_t range, uint32_t count,
                               uint64_t* out, uint32_t* status) {
    if (blockIdx.x || threadIdx.x) return;
    StepRng R;
    R.init(key, walker, step);
    for (uint32_t i = 0; i < count; i++) out[i] = range ? below64(R, range, status) : (uint64_t)R.next();
}

// Packed walk output: lengths widened for the scan, then every walker's row prefix copied to its
// offset (one thread per walker; each row is contiguous, and so is each packed path).
__global__ void k_len64(const uint32_t* __restrict__ plen, uint64_t n, uint64_t* __restrict__ out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = plen[i];
}
__global__ void k_pack_rows(const uint32_t* __restrict__ rows, uint32_t stride, const uint32_t* __restrict__ plen,
                            const uint64_t* __restrict__ off, uint64_t n, uint32_t* __restrict__ out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t L = plen[i] <= stride ? plen[i] : stride;
        const uint32_t* src = rows + i * (uint64_t)stride;
        uint32_t* dst = out + off[i];
        for (uint32_t j = 0; j < L; j++) dst[j] = src[j];
    }
}

}  // namespace

extern "C" {

bingo_status bingo_walk(bingo_graph* g, uint64_t nwalkers, const uint32_t* starts, const uint32_t* lengths,
                        const uint8_t* policy_ids, const bingo_policy* policies, uint32_t npolicies, uint64_t seed,
                        uint32_t stride, uint32_t* paths, uint32_t* path_len, uint32_t mode, void* stream) {
    if (!g) { set_error("NULL graph"); return BINGO_E_INVALID; }
    if (g->broken) { set_error("graph state is unusable after an earlier device failure"); return BINGO_E_STATE; }
    bingo_status st = check_device(g, "walk");
    if (st != BINGO_OK) return st;
    if (g->part) { set_error("walk: a partition graph walks only through bingo_part_walk"); return BINGO_E_STATE; }
    const uint32_t base_mode = mode & 0xFF;
    const bool pad = !(mode & 0x100);
    if (base_mode > BINGO_WALK_STEPWISE) { set_error("unknown walk mode %u", mode); return BINGO_E_INVALID; }
    if (nwalkers && (!starts || !paths || !path_len)) { set_error("NULL walk buffer"); return BINGO_E_INVALID; }
    if (stride == 0) { set_error("stride must be >= 1"); return BINGO_E_INVALID; }
    bool need_n2v = false;
    uint32_t max_len = 0;
    st = check_policies(policies, npolicies, stride, lengths != nullptr, &need_n2v, &max_len);
    if (st != BINGO_OK) return st;
    if (nwalkers == 0) return BINGO_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (need_n2v && g->G.eh_mask == 0) {
        st = edge_index_build(g, s);
        if (st != BINGO_OK) return st;
    }
    bool host_io = false;
    auto in = [&](const void* src, size_t bytes, Buf& b, const void** out) -> bingo_status {
        if (!src || is_device_ptr(src)) { *out = src; return BINGO_OK; }
        host_io = true;
        CK(ensure(b, bytes), "walk staging");
        CK(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, s), "walk upload");
        *out = b.p;
        return BINGO_OK;
    };
    const uint32_t *ds, *dl;
    const uint8_t* dp;
    if ((st = in(starts, 4 * nwalkers, g->w_starts, (const void**)&ds)) != BINGO_OK) return st;
    if ((st = in(lengths, 4 * nwalkers, g->w_len, (const void**)&dl)) != BINGO_OK) return st;
    if ((st = in(policy_ids, nwalkers, g->w_pid, (const void**)&dp)) != BINGO_OK) return st;
    uint32_t* dpaths = paths;
    uint32_t* dplen = path_len;
    const bool host_paths = !is_device_ptr(paths), host_plen = !is_device_ptr(path_len);
    if (host_paths) {
        CK(ensure(g->w_paths, 4ull * nwalkers * stride), "walk output staging");
        dpaths = (uint32_t*)g->w_paths.p;
        // without padding, entries past path_len must keep the caller's values through the round trip
        if (!pad)
            CK(cudaMemcpyAsync(dpaths, paths, 4ull * nwalkers * stride, cudaMemcpyHostToDevice, s), "paths upload");
    }
    if (host_plen) {
        CK(ensure(g->w_plen, 4ull * nwalkers), "walk output staging");
        dplen = (uint32_t*)g->w_plen.p;
    }
    CK(ensure(g->w_pols, sizeof(bingo_policy) * npolicies), "policy staging");
    CK(cudaMemcpyAsync(g->w_pols.p, policies, sizeof(bingo_policy) * npolicies, cudaMemcpyHostToDevice, s),
       "policy upload");
    WalkReq q;
    q.nwalkers = nwalkers;
    q.starts = ds;
    q.lengths = dl;
    q.pids = dp;
    q.dev_pols = (const bingo_policy*)g->w_pols.p;
    q.npol = npolicies;
    q.seed = seed;
    q.stride = stride;
    q.paths = dpaths;
    q.plen = dplen;
    q.mode = base_mode;
    q.pad = pad;
    q.max_steps = lengths ? stride - 1 : max_len;
    q.queue = (unsigned long long*)((uint64_t*)g->d_ctl + CTL_QUEUE);
    if ((host_paths || host_plen) && base_mode == BINGO_WALK_PERSISTENT && nwalkers >= WALK_IO_MIN) {
        st = walk_host_io_overlap(g, q, paths, path_len, host_paths, host_plen, s);
        if (st != BINGO_OK) return st;
    } else {
        st = walk_launch(g, q, s);
        if (st != BINGO_OK) return st;
        if (host_paths) CK(cudaMemcpyAsync(paths, dpaths, 4ull * nwalkers * stride, cudaMemcpyDeviceToHost, s), "paths download");
        if (host_plen) CK(cudaMemcpyAsync(path_len, dplen, 4ull * nwalkers, cudaMemcpyDeviceToHost, s), "lengths download");
    }
    if (host_io || host_paths || host_plen) {
        CK(cudaStreamSynchronize(s), "walk");
        uint32_t status = 0;
        CK(cudaMemcpy(&status, (uint64_t*)g->d_ctl + CTL_STATUS, 4, cudaMemcpyDeviceToHost), "status read");
        if (status & ST_STATE) { set_error("walk: inconsistent group structure"); return BINGO_E_STATE; }
        if (status & ST_INVALID) { set_error("walk: a start vertex >= n, a policy id >= npolicies or a length > stride-1"); return BINGO_E_INVALID; }
        if (status & ST_TIMEOUT) { set_error("walk: a bounded rejection loop gave up"); return BINGO_E_TIMEOUT; }
    }
    return BINGO_OK;
}

bingo_status bingo_walk_packed(bingo_graph* g, uint64_t nwalkers, const uint32_t* starts, const uint32_t* lengths,
                               const uint8_t* policy_ids, const bingo_policy* policies, uint32_t npolicies,
                               uint64_t seed, uint32_t max_steps, uint32_t* path_len, uint32_t* vertices,
                               uint64_t capacity, uint64_t* total, void* stream) {
    if (!g) { set_error("NULL graph"); return BINGO_E_INVALID; }
    if (g->broken) { set_error("graph state is unusable after an earlier device failure"); return BINGO_E_STATE; }
    bingo_status st = check_device(g, "walk_packed");
    if (st != BINGO_OK) return st;
    if (g->part) { set_error("walk_packed: a partition graph walks only through bingo_part_walk"); return BINGO_E_STATE; }
    if (nwalkers && (!starts || !path_len || (!vertices && capacity))) { set_error("walk_packed: NULL buffer"); return BINGO_E_INVALID; }
    if (max_steps >= 0xFFFFFFFFu) { set_error("walk_packed: max_steps too large"); return BINGO_E_INVALID; }
    const uint32_t stride = max_steps + 1;
    bool need_n2v = false;
    uint32_t max_len = 0;
    st = check_policies(policies, npolicies, stride, lengths != nullptr, &need_n2v, &max_len);
    if (st != BINGO_OK) return st;
    if (total) *total = 0;
    if (nwalkers == 0) return BINGO_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (need_n2v && g->G.eh_mask == 0) {
        st = edge_index_build(g, s);
        if (st != BINGO_OK) return st;
    }
    auto in = [&](const void* src, size_t bytes, Buf& b, const void** out) -> bingo_status {
        if (!src || is_device_ptr(src)) { *out = src; return BINGO_OK; }
        CK(ensure(b, bytes), "walk staging");
        CK(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, s), "walk upload");
        *out = b.p;
        return BINGO_OK;
    };
    const uint32_t *ds, *dl;
    const uint8_t* dp;
    if ((st = in(starts, 4 * nwalkers, g->w_starts, (const void**)&ds)) != BINGO_OK) return st;
    if ((st = in(lengths, 4 * nwalkers, g->w_len, (const void**)&dl)) != BINGO_OK) return st;
    if ((st = in(policy_ids, nwalkers, g->w_pid, (const void**)&dp)) != BINGO_OK) return st;
    const bool host_len = !is_device_ptr(path_len), host_vert = vertices && !is_device_ptr(vertices);
    CK(ensure(g->w_paths, 4ull * nwalkers * stride), "walk rows");
    uint32_t* dplen = path_len;
    if (host_len) {
        CK(ensure(g->w_plen, 4ull * nwalkers), "walk lengths");
        dplen = (uint32_t*)g->w_plen.p;
    }
    CK(ensure(g->w_pols, sizeof(bingo_policy) * npolicies), "policy staging");
    CK(cudaMemcpyAsync(g->w_pols.p, policies, sizeof(bingo_policy) * npolicies, cudaMemcpyHostToDevice, s),
       "policy upload");
    WalkReq q;
    q.nwalkers = nwalkers;
    q.starts = ds;
    q.lengths = dl;
    q.pids = dp;
    q.dev_pols = (const bingo_policy*)g->w_pols.p;
    q.npol = npolicies;
    q.seed = seed;
    q.stride = stride;
    q.paths = (uint32_t*)g->w_paths.p;
    q.plen = dplen;
    q.mode = BINGO_WALK_PERSISTENT;
    q.pad = false;
    q.max_steps = lengths ? max_steps : max_len;
    q.queue = (unsigned long long*)((uint64_t*)g->d_ctl + CTL_QUEUE);
    if ((st = walk_launch(g, q, s)) != BINGO_OK) return st;
    if (host_len) CK(cudaMemcpyAsync(path_len, dplen, 4ull * nwalkers, cudaMemcpyDeviceToHost, s), "lengths download");
    // offsets: exclusive scan of the lengths; off[nwalkers] = total
    CK(ensure(g->w_len64, 8ull * nwalkers), "walk offsets");
    CK(ensure(g->w_off, 8ull * (nwalkers + 1)), "walk offsets");
    uint64_t* off = (uint64_t*)g->w_off.p;
    const unsigned blocks = (unsigned)std::min<uint64_t>((nwalkers + 255) / 256, (uint64_t)g->num_sms * 16);
    k_len64<<<blocks, 256, 0, s>>>(dplen, nwalkers, (uint64_t*)g->w_len64.p);
    g->launches++;
    CK(scan_excl_u64((const uint64_t*)g->w_len64.p, off, nwalkers, off + nwalkers, g->s_tmp, s, &g->launches),
       "walk offsets");
    uint64_t tot = 0;
    CK(cudaMemcpyAsync(&tot, off + nwalkers, 8, cudaMemcpyDeviceToHost, s), "walk total");
    CK(cudaStreamSynchronize(s), "walk");
    uint32_t status = 0;
    CK(cudaMemcpy(&status, (uint64_t*)g->d_ctl + CTL_STATUS, 4, cudaMemcpyDeviceToHost), "status read");
    if (status & ST_STATE) { set_error("walk: inconsistent group structure"); return BINGO_E_STATE; }
    if (status & ST_INVALID) { set_error("walk: a start vertex >= n, a policy id >= npolicies or a length > max_steps"); return BINGO_E_INVALID; }
    if (status & ST_TIMEOUT) { set_error("walk: a bounded rejection loop gave up"); return BINGO_E_TIMEOUT; }
    if (total) *total = tot;
    if (tot > capacity) {
        set_error("walk_packed: the paths hold %llu vertices, more than the capacity %llu", (unsigned long long)tot,
                  (unsigned long long)capacity);
        return BINGO_E_INVALID;
    }
    uint32_t* dvert = vertices;
    if (host_vert) {
        CK(ensure(g->w_packed, 4ull * (tot ? tot : 1)), "packed paths");
        dvert = (uint32_t*)g->w_packed.p;
    }
    k_pack_rows<<<blocks, 256, 0, s>>>((const uint32_t*)g->w_paths.p, stride, dplen, off, nwalkers, dvert);
    g->launches++;
    CK(cudaGetLastError(), "pack paths");
    if (host_vert && tot) CK(cudaMemcpyAsync(vertices, dvert, 4ull * tot, cudaMemcpyDeviceToHost, s), "paths download");
    if (host_vert) CK(cudaStreamSynchronize(s), "paths download");
    return BINGO_OK;
}

// Synchronise `stream` and return (and clear) the device status latched by asynchronous calls.
bingo_status bingo_check(bingo_graph* g, void* stream) {
    if (!g) { set_error("NULL graph"); return BINGO_E_INVALID; }
    CK(cudaStreamSynchronize((cudaStream_t)stream), "sync");
    uint32_t status = 0;
    uint64_t* word = (uint64_t*)g->d_ctl + CTL_STATUS;
    CK(cudaMemcpy(&status, word, 4, cudaMemcpyDeviceToHost), "status read");
    CK(cudaMemset(word, 0, 8), "status clear");
    if (status & ST_STATE) { set_error("device found an inconsistent group structure"); return BINGO_E_STATE; }
    if (status & ST_INVALID) { set_error("device reported an invalid argument"); return BINGO_E_INVALID; }
    if (status & ST_OOM) { set_error("device pool exhausted"); return BINGO_E_OOM; }
    if (status & ST_TIMEOUT) { set_error("a bounded device loop gave up"); return BINGO_E_TIMEOUT; }
    return BINGO_OK;
}

bingo_status bingo_autotune(bingo_graph* g, uint64_t nwalkers, const uint32_t* starts, uint32_t length, void* stream,
                            bingo_config* out_cfg) {
    if (!g || !starts || nwalkers == 0 || length == 0) { set_error("autotune: bad arguments"); return BINGO_E_INVALID; }
    if (g->part) { set_error("autotune: a partition graph walks only through bingo_part_walk"); return BINGO_E_STATE; }
    cudaStream_t s = (cudaStream_t)stream;
    Buf dstarts, dpaths, dplen;
    const uint32_t* ds = starts;
    auto cleanup = [&]() { release(dstarts); release(dpaths); release(dplen); };
    if (!is_device_ptr(starts)) {
        cudaError_t e = ensure(dstarts, 4 * nwalkers);
        if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "autotune"); }
        cudaMemcpyAsync(dstarts.p, starts, 4 * nwalkers, cudaMemcpyHostToDevice, s);
        ds = (const uint32_t*)dstarts.p;
    }
    const uint32_t stride = length + 1;
    cudaError_t e = ensure(dpaths, 4ull * nwalkers * stride);
    if (e == cudaSuccess) e = ensure(dplen, 4ull * nwalkers);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "autotune"); }
    bingo_policy pol;
    memset(&pol, 0, sizeof(pol));
    pol.kind = BINGO_DEEPWALK;
    pol.max_len = length;
    e = ensure(g->w_pols, sizeof(bingo_policy));
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "autotune"); }
    cudaMemcpyAsync(g->w_pols.p, &pol, sizeof(pol), cudaMemcpyHostToDevice, s);
    WalkReq q;
    q.nwalkers = nwalkers;
    q.starts = ds;
    q.dev_pols = (const bingo_policy*)g->w_pols.p;
    q.npol = 1;
    q.stride = stride;
    q.paths = (uint32_t*)dpaths.p;
    q.plen = (uint32_t*)dplen.p;
    q.mode = BINGO_WALK_PERSISTENT;
    q.pad = false;
    q.max_steps = length;
    q.queue = (unsigned long long*)((uint64_t*)g->d_ctl + CTL_QUEUE);
    const WalkTune saved = g->tune;
    const uint32_t lanes_c[3] = {1, 4, 32};
    const uint32_t wpb_c[3] = {4, 8, 16};
    const uint32_t occ_c[2] = {0, 1};
    float best = 1e30f;
    WalkTune bestt = saved;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (uint32_t li = 0; li < 3; li++) {
        for (uint32_t wi = 0; wi < 6; wi++) {
            if (occ_c[wi / 3] && wpb_c[wi % 3] > 8) continue;
            g->tune.lanes = lanes_c[li];
            g->tune.warps_per_block = wpb_c[wi % 3];
            g->tune.occ = occ_c[wi / 3];
            g->tune.blocks_per_sm = 0;
            float tsum = 0;
            bool ok = true;
            for (int rep = 0; rep < 3 && ok; rep++) {
                cudaEventRecord(e0, s);
                q.seed = 1234 + rep;
                ok = walk_launch(g, q, s) == BINGO_OK;
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tsum += ms;
            }
            if (ok && tsum < best) {
                best = tsum;
                bestt = g->tune;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cleanup();
    g->tune = bestt;
    if (out_cfg) bingo_get_config(g, out_cfg);
    return best < 1e30f ? BINGO_OK : BINGO_E_CUDA;
}

// Group-adaption tuner: build the graph under each candidate (alpha, beta) of Eq. group, keep the
// candidates whose state fits the budget, time a trial walk on each and return the fastest.
bingo_status bingo_autotune_adaption(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col,
                                     const uint32_t* bias, const bingo_config* cfg, uint64_t state_budget_bytes,
                                     uint64_t nwalkers, const uint32_t* starts, uint32_t length, void* stream,
                                     bingo_graph** out, bingo_config* out_cfg) {
    if (!out || !starts || nwalkers == 0 || length == 0) { set_error("autotune_adaption: bad arguments"); return BINGO_E_INVALID; }
    *out = nullptr;
    bingo_config base;
    if (cfg) base = *cfg; else bingo_default_config(&base);
    if (base.all_regular) { set_error("autotune_adaption: all_regular graphs have no adaption to tune"); return BINGO_E_INVALID; }
    cudaStream_t s = (cudaStream_t)stream;
    // stage host inputs once for every candidate build and walk
    Buf brp, bcol, bbias, bst, bpaths, bplen;
    auto cleanup = [&]() { release(brp); release(bcol); release(bbias); release(bst); release(bpaths); release(bplen); };
    auto stage = [&](const void* src, size_t bytes, Buf& b, const void** dst) -> cudaError_t {
        if (!src || bytes == 0 || is_device_ptr(src)) { *dst = src; return cudaSuccess; }
        cudaError_t e = ensure(b, bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, s);
        *dst = b.p;
        return e;
    };
    const uint64_t* drp;
    const uint32_t *dcol, *dbias, *dst_;
    cudaError_t e = stage(row_ptr, 8ull * ((uint64_t)n + 1), brp, (const void**)&drp);
    if (e == cudaSuccess) e = stage(col, 4ull * m, bcol, (const void**)&dcol);
    if (e == cudaSuccess) e = stage(bias, 4ull * m, bbias, (const void**)&dbias);
    if (e == cudaSuccess) e = stage(starts, 4ull * nwalkers, bst, (const void**)&dst_);
    const uint32_t stride = length + 1;
    if (e == cudaSuccess) e = ensure(bpaths, 4ull * nwalkers * stride);
    if (e == cudaSuccess) e = ensure(bplen, 4ull * nwalkers);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "autotune_adaption staging"); }
    static const uint32_t alphas[] = {20, 40, 70, 100};  // 100: no group is ever dense
    static const uint32_t betas[] = {0, 10};             // 0: no group is ever sparse
    bingo_policy pol;
    memset(&pol, 0, sizeof(pol));
    pol.kind = BINGO_DEEPWALK;
    pol.max_len = length;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    bingo_graph* best = nullptr;
    float best_ms = 0.f;
    bingo_status st = BINGO_OK, last_fail = BINGO_OK;
    bool over_budget = false;
    for (uint32_t ai = 0; ai < 4 && st == BINGO_OK; ai++) {
        for (uint32_t bi = 0; bi < 2 && st == BINGO_OK; bi++) {
            bingo_config c = base;
            c.alpha_pct = alphas[ai];
            c.beta_pct = betas[bi];
            bingo_graph* g = nullptr;
            bingo_status cs = bingo_create(n, m, drp, dcol, dbias, &c, stream, &g);
            if (cs == BINGO_E_OOM) { last_fail = cs; continue; }  // this candidate does not fit the device
            if (cs != BINGO_OK) { st = cs; break; }
            uint64_t rep[6];
            cs = bingo_memory_report(g, rep);
            if (cs != BINGO_OK) { bingo_destroy(g); st = cs; break; }
            if (state_budget_bytes && rep[0] + rep[1] + rep[2] + rep[3] > state_budget_bytes) {
                over_budget = true;
                bingo_destroy(g);
                continue;
            }
            if ((e = ensure(g->w_pols, sizeof(bingo_policy))) != cudaSuccess ||
                (e = cudaMemcpyAsync(g->w_pols.p, &pol, sizeof(pol), cudaMemcpyHostToDevice, s)) != cudaSuccess) {
                bingo_destroy(g);
                st = cuda_fail(e, "autotune_adaption policy");
                break;
            }
            WalkReq q;
            q.nwalkers = nwalkers;
            q.starts = dst_;
            q.dev_pols = (const bingo_policy*)g->w_pols.p;
            q.npol = 1;
            q.stride = stride;
            q.paths = (uint32_t*)bpaths.p;
            q.plen = (uint32_t*)bplen.p;
            q.mode = BINGO_WALK_PERSISTENT;
            q.pad = false;
            q.max_steps = length;
            q.queue = (unsigned long long*)((uint64_t*)g->d_ctl + CTL_QUEUE);
            float tsum = 0.f;
            for (int rep_i = 0; rep_i < 3 && cs == BINGO_OK; rep_i++) {  // one warm-up, two timed
                q.seed = 4321 + rep_i;
                cudaEventRecord(e0, s);
                cs = walk_launch(g, q, s);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) cs = cuda_fail(cudaGetLastError(), "autotune_adaption walk");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep_i > 0) tsum += ms;
            }
            if (cs == BINGO_OK) cs = bingo_check(g, stream);
            if (cs != BINGO_OK) { bingo_destroy(g); st = cs; break; }
            if (!best || tsum < best_ms) {
                if (best) bingo_destroy(best);
                best = g;
                best_ms = tsum;
            } else {
                bingo_destroy(g);
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cleanup();
    if (st != BINGO_OK) {
        if (best) bingo_destroy(best);
        return st;
    }
    if (!best) {
        if (over_budget) set_error("autotune_adaption: no (alpha, beta) candidate fits %llu bytes of state",
                                   (unsigned long long)state_budget_bytes);
        else set_error("autotune_adaption: no candidate could be built (%d)", (int)last_fail);
        return BINGO_E_OOM;
    }
    *out = best;
    if (out_cfg) bingo_get_config(best, out_cfg);
    return BINGO_OK;
}

bingo_status bingo_policy_make(uint32_t kind, uint32_t max_len, double ppr_stop, double n2v_p, double n2v_q,
                               bingo_policy* out) {
    if (!out || kind > BINGO_NODE2VEC) { set_error("policy_make: bad kind or NULL output"); return BINGO_E_INVALID; }
    memset(out, 0, sizeof(*out));
    out->kind = kind;
    out->max_len = max_len;
    if (kind == BINGO_PPR) {
        if (!(ppr_stop >= 0.0 && ppr_stop <= 1.0)) { set_error("policy_make: PPR stop %g outside [0, 1]", ppr_stop); return BINGO_E_INVALID; }
        const double t = nearbyint(ppr_stop * 4294967296.0);
        out->ppr_stop_u32 = t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
    }
    if (kind == BINGO_NODE2VEC) {
        if (!(n2v_p > 0.0 && n2v_q > 0.0 && isfinite(n2v_p) && isfinite(n2v_q))) {
            set_error("policy_make: node2vec p = %g, q = %g must be positive and finite", n2v_p, n2v_q);
            return BINGO_E_INVALID;
        }
        // f(dist) of Eq. node2vec: 1/p at distance 0, 1 at distance 1, 1/q at distance 2
        const double f[3] = {1.0 / n2v_p, 1.0, 1.0 / n2v_q};
        const double mf = std::max(f[0], std::max(f[1], f[2]));
        for (int d = 0; d < 3; d++) {
            const double t = nearbyint(f[d] / mf * 4294967296.0);
            out->n2v_accept[d] = t >= 4294967296.0 ? (1ull << 32) : (uint64_t)t;
        }
    }
    return BINGO_OK;
}

bingo_status bingo_philox4x32_10(uint64_t count, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    if (count == 0) return BINGO_OK;
    if (!ctr || !key || !out || count > (1ull << 26)) { set_error("philox4x32_10: bad arguments"); return BINGO_E_INVALID; }
    Buf b;
    CK(ensure(b, 40 * count), "philox4x32_10 buffers");
    uint4* dc = (uint4*)b.p;
    uint4* dout = dc + count;
    uint2* dk = (uint2*)(dout + count);
    cudaError_t e = cudaMemcpy(dc, ctr, 16 * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, 8 * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_philox_eval<<<(unsigned)std::min<uint64_t>((count + 255) / 256, 1024), 256>>>(count, dc, dk, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 16 * count, cudaMemcpyDeviceToHost);
    release(b);
    return e == cudaSuccess ? BINGO_OK : cuda_fail(e, "philox4x32_10");
}

bingo_status bingo_walker_draws(uint64_t seed, uint64_t walker, uint32_t step, uint64_t range, uint32_t count,
                                uint64_t* out) {
    if (count == 0) return BINGO_OK;
    if (!out || count > (1u << 20)) { set_error("walker_draws: bad arguments"); return BINGO_E_INVALID; }
    Buf b;
    CK(ensure(b, 8ull * count + 8), "walker_draws buffers");
    uint32_t* dstatus = (uint32_t*)((uint64_t*)b.p + count);
    cudaError_t e = cudaMemset(dstatus, 0, 4);
    if (e == cudaSuccess) {
        k_walker_draws<<<1, 32>>>(make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), walker, step, range, count,
                                  (uint64_t*)b.p, dstatus);
        e = cudaGetLastError();
    }
    uint32_t status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(out, b.p, 8ull * count, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&status, dstatus, 4, cudaMemcpyDeviceToHost);
    release(b);
    if (e != cudaSuccess) return cuda_fail(e, "walker_draws");
    if (status) { set_error("walker_draws: a bounded draw ran out of retries"); return BINGO_E_TIMEOUT; }
    return BINGO_OK;
}

}  // extern "C"
