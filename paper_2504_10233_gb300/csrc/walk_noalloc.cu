// Allocation-free walk entry point.
//
// Some callers cannot allocate device memory at the moment they need a walk:
// code running inside a custom allocator or memory-pool callback, processes
// whose device memory is fully reserved up front by a framework, or
// real-time loops that forbid cudaMalloc/cudaFree because those calls can
// synchronise the device and stall other streams.  bingo_walk_noalloc serves
// them: it runs the same persistent walker as bingo_walk, but its only scratch
// (the walker work counter and the policy table) lives in a fixed array that
// the library reserves in device memory when it is loaded, so the call itself
// allocates nothing.
#include <mutex>

#include "bingo_host.h"

using namespace bingo;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 1024;    // counter (64 B slot) + up to MAX_POL policies
constexpr size_t NOALLOC_POLICY_OFFSET = 64;
static_assert(NOALLOC_POLICY_OFFSET + MAX_POL * sizeof(bingo_policy) <= NOALLOC_SCRATCH_BYTES, "scratch too small");

// The scratch array.  Every device that loads the library holds it until the process exits, and
// every call on a device shares it.  In host code this name is only a stand-in for the symbol: its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_walk_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[MAX_DEVICES] = {};

// Resolve the scratch address on the current device, once per device.
bingo_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "walk_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("walk_noalloc: device ordinal %d out of range", dev);
        return BINGO_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_walk_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "walk_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return BINGO_OK;
}

}  // namespace

extern "C" bingo_status bingo_walk_noalloc(bingo_graph* g, uint64_t nwalkers, const uint32_t* starts,
                                           const uint32_t* lengths, const uint8_t* policy_ids,
                                           const bingo_policy* policies, uint32_t npolicies, uint64_t seed,
                                           uint32_t stride, uint32_t* paths, uint32_t* path_len, uint32_t mode,
                                           void* stream) {
    if (!g) { set_error("walk_noalloc: NULL graph"); return BINGO_E_INVALID; }
    if (g->broken) { set_error("walk_noalloc: graph state is unusable"); return BINGO_E_STATE; }
    if (!policies || npolicies == 0 || npolicies > MAX_POL) {
        set_error("walk_noalloc: %u policies requested; the fixed scratch holds 1..%u", npolicies, MAX_POL);
        return BINGO_E_INVALID;
    }
    if ((mode & 0xFF) != BINGO_WALK_PERSISTENT) {
        set_error("walk_noalloc: only the persistent form runs without allocating (mode %u)", mode);
        return BINGO_E_INVALID;
    }
    if (stride == 0) { set_error("walk_noalloc: stride must be >= 1"); return BINGO_E_INVALID; }
    uint32_t max_len = 0;
    for (uint32_t i = 0; i < npolicies; i++) {
        const bingo_policy& p = policies[i];
        if (p.kind > BINGO_NODE2VEC) { set_error("walk_noalloc: policy %u has unknown kind %u", i, p.kind); return BINGO_E_INVALID; }
        if (p.kind == BINGO_NODE2VEC && g->G.eh_mask == 0) {
            set_error("walk_noalloc: node2vec needs the edge index, which only bingo_walk builds (it allocates)");
            return BINGO_E_STATE;
        }
        for (int d = 0; d < 3; d++)
            if (p.n2v_accept[d] > (1ull << 32)) { set_error("walk_noalloc: policy %u: n2v_accept > 2^32", i); return BINGO_E_INVALID; }
        if (!lengths && (uint64_t)p.max_len + 1 > stride) {
            set_error("walk_noalloc: policy %u max_len %u does not fit stride %u", i, p.max_len, stride);
            return BINGO_E_INVALID;
        }
        if (p.max_len > max_len) max_len = p.max_len;
    }
    if (nwalkers == 0) return BINGO_OK;
    if (!is_device_ptr(starts) || !is_device_ptr(paths) || !is_device_ptr(path_len) ||
        (lengths && !is_device_ptr(lengths)) || (policy_ids && !is_device_ptr(policy_ids))) {
        set_error("walk_noalloc: starts, lengths, policy ids, paths and path_len must be device pointers");
        return BINGO_E_INVALID;
    }
    void* scratch = nullptr;
    bingo_status st = scratch_address(&scratch);
    if (st != BINGO_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* queue = (unsigned long long*)scratch;
    bingo_policy* dev_pols = (bingo_policy*)((char*)scratch + NOALLOC_POLICY_OFFSET);
    cudaError_t e = cudaMemcpyAsync(dev_pols, policies, sizeof(bingo_policy) * npolicies, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "walk_noalloc: policy upload");
    WalkReq q;
    q.nwalkers = nwalkers;
    q.starts = starts;
    q.lengths = lengths;
    q.pids = policy_ids;
    q.dev_pols = dev_pols;
    q.npol = npolicies;
    q.seed = seed;
    q.stride = stride;
    q.paths = paths;
    q.plen = path_len;
    q.mode = BINGO_WALK_PERSISTENT;
    q.pad = !(mode & BINGO_WALK_NO_PAD);
    q.max_steps = lengths ? stride - 1 : max_len;
    q.queue = queue;  // walk_launch zeroes it on `s` before the kernel
    return walk_launch(g, q, s);
}
