// Allocation-free walk entry point.
//
// Some callers cannot allocate device memory at the moment they need a walk:
// code running inside a custom allocator or memory-pool callback, processes
// whose device memory is fully reserved up front by a framework, or
// real-time loops that forbid cudaMalloc/cudaFree because those calls can
// synchronise the device and stall other streams.  bingo_walk_noalloc serves
// them: it runs the same persistent walker as bingo_walk, but its only scratch
// (the walker work counter and the policy table) lives in a fixed
// file-scope device array, so the call itself allocates nothing.
//
// Under CUDA's lazy module loading a module is loaded (and its device memory,
// this array included, allocated) the first time one of its symbols or kernels
// is used.  bingo_create therefore resolves this array's address on the graph's
// device (noalloc_prepare) and loads every walker kernel instance of the graph's
// weight format (walk_preload), so the first bingo_walk_noalloc call on a graph
// finds everything loaded.
#include <mutex>

#include "bingo_host.h"

using namespace bingo;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 1024;    // counter (64 B slot) + up to MAX_POL policies
constexpr size_t NOALLOC_POLICY_OFFSET = 64;
static_assert(NOALLOC_POLICY_OFFSET + MAX_POL * sizeof(bingo_policy) <= NOALLOC_SCRATCH_BYTES, "scratch too small");
static_assert(MAX_POL == 16, "the header documents a 16-policy limit");

// The scratch array.  Every device that loads the library holds it until the process exits, and
// every call on a device shares it.  In host code this name is only a stand-in for the symbol: its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_walk_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[MAX_DEVICES] = {};

// The scratch address on device `dev`, once it has been resolved there (else null).
void* scratch_for(int dev) {
    if (dev < 0 || dev >= MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    return g_scratch_addr[dev];
}

}  // namespace

namespace bingo {

bingo_status noalloc_prepare(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "walk_noalloc setup: cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("walk_noalloc setup: device ordinal %d out of range", dev);
        return BINGO_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_walk_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "walk_noalloc setup: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    return BINGO_OK;
}

}  // namespace bingo

extern "C" bingo_status bingo_walk_noalloc(bingo_graph* g, uint64_t nwalkers, const uint32_t* starts,
                                           const uint32_t* lengths, const uint8_t* policy_ids,
                                           const bingo_policy* policies, uint32_t npolicies, uint64_t seed,
                                           uint32_t stride, uint32_t* paths, uint32_t* path_len, uint32_t mode,
                                           void* stream) {
    if (!g) { set_error("walk_noalloc: NULL graph"); return BINGO_E_INVALID; }
    if (g->broken) { set_error("walk_noalloc: graph state is unusable"); return BINGO_E_STATE; }
    bingo_status st = check_device(g, "walk_noalloc");
    if (st != BINGO_OK) return st;
    if (g->part) { set_error("walk_noalloc: a partition graph walks only through bingo_part_walk"); return BINGO_E_STATE; }
    if ((mode & 0xFF) != BINGO_WALK_PERSISTENT) {
        set_error("walk_noalloc: only the persistent form runs without allocating (mode %u)", mode);
        return BINGO_E_INVALID;
    }
    if (stride == 0) { set_error("walk_noalloc: stride must be >= 1"); return BINGO_E_INVALID; }
    bool need_n2v = false;
    uint32_t max_len = 0;
    st = check_policies(policies, npolicies, stride, lengths != nullptr, &need_n2v, &max_len);
    if (st != BINGO_OK) return st;
    if (need_n2v && g->G.eh_mask == 0) {
        set_error("walk_noalloc: node2vec needs the edge index, which only bingo_walk builds (it allocates)");
        return BINGO_E_STATE;
    }
    if (nwalkers == 0) return BINGO_OK;
    if (!is_device_ptr(starts) || !is_device_ptr(paths) || !is_device_ptr(path_len) ||
        (lengths && !is_device_ptr(lengths)) || (policy_ids && !is_device_ptr(policy_ids))) {
        set_error("walk_noalloc: starts, lengths, policy ids, paths and path_len must be device pointers");
        return BINGO_E_INVALID;
    }
    void* scratch = scratch_for(g->device);
    if (!scratch) {  // bingo_create resolves it; a graph whose set-up failed never reaches here
        set_error("walk_noalloc: scratch array not resolved on device %d", g->device);
        return BINGO_E_STATE;
    }
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
