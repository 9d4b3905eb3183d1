// Host-side graph object and helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "bingo_internal.cuh"

namespace bingo {

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

// grow-only device buffer
cudaError_t ensure(Buf& b, size_t bytes);
void release(Buf& b);

void set_error(const char* fmt, ...);
bingo_status cuda_fail(cudaError_t e, const char* what);
bool is_device_ptr(const void* p);

// device-wide exclusive scan of u64 values; *total_dev (device) receives the sum
cudaError_t scan_excl_u64(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* total_dev, Buf& tmp,
                          cudaStream_t s, uint64_t* launches);

// stable LSD radix sort of (key u64, value u32) pairs on the low `bits` key bits
// (sorts the key bits [lo_bit, lo_bit + bits)).  With n_dev, n is a capacity: grids are sized for n
// and the live length is read from *n_dev on the device (for graph capture).
cudaError_t radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, uint64_t n,
                             uint32_t bits, Buf& tmp, cudaStream_t s, bool* result_in_alt, uint64_t* launches,
                             uint32_t lo_bit = 0, const uint64_t* n_dev = nullptr);
size_t radix_sort_tmp_bytes(uint64_t n);
size_t scan_tmp_bytes(uint64_t n);

// One walk launch, all pointers on the device.
struct WalkReq {
    uint64_t nwalkers = 0;
    const uint32_t* starts = nullptr;
    const uint32_t* lengths = nullptr;   // nullable
    const uint8_t* pids = nullptr;       // nullable
    const bingo_policy* dev_pols = nullptr;
    uint32_t npol = 0;
    uint64_t seed = 0;
    uint32_t stride = 0;
    uint32_t* paths = nullptr;
    uint32_t* plen = nullptr;
    uint32_t mode = 0;                   // BINGO_WALK_PERSISTENT / STEPWISE
    bool pad = true;
    uint32_t max_steps = 0;              // step launches of the stepwise form
    unsigned long long* queue = nullptr; // device work counter of this launch
    const uint64_t* req_off = nullptr;   // request mode
    const uint64_t* req_key = nullptr;
    uint32_t nreq = 0;
    // completion notices for downloads that overlap the walk (all null/0 = off): walker w counts into
    // chunk_done[w >> chunk_shift]; the walker that completes a chunk writes io_seq to host_flags[chunk]
    uint32_t* chunk_done = nullptr;      // device counters, zeroed before the launch
    uint32_t* host_flags = nullptr;      // device view of host-mapped pinned memory
    uint32_t chunk_shift = 0;
    uint32_t io_seq = 0;
    // partitioned walks (see WalkParams in walk.cu); resume null = start mode
    const PartRec* resume = nullptr;
    PartRec* outbox = nullptr;
    unsigned long long* nout = nullptr;
    const PartEH* peh = nullptr;
    const uint32_t* bounds = nullptr;
    uint32_t npart = 0;
};

bingo_status walk_launch(bingo_graph* g, const WalkReq& q, cudaStream_t s);

// Validate a host array of walk policies (kinds, node2vec thresholds <= 2^32, max_len + 1 <= stride
// unless per-walker lengths are given); reports whether any is node2vec and the longest max_len.
// Shared by every walk entry point so that they accept exactly the same inputs.
bingo_status check_policies(const bingo_policy* pols, uint32_t npol, uint32_t stride, bool have_lengths,
                            bool* need_n2v, uint32_t* max_len);

// BINGO_E_INVALID unless the calling thread's current device is the graph's: every launch and every
// device pointer of a call belongs to the device that was current when the graph was created.
bingo_status check_device(const bingo_graph* g, const char* who);

// Launch every walker kernel instance of the graph's weight mode once, over zero walkers, on `s`:
// this loads each instance (lazy module loading would otherwise load it at its first real launch)
// and sizes the context's local-memory reservation for it, both of which can allocate device memory.
cudaError_t walk_preload(bingo_graph* g, cudaStream_t s);
// Resolve, on the current device, the address of the allocation-free walk's fixed scratch array
// (loading its module); later calls on that device reuse it.
bingo_status noalloc_prepare(void);

// Host-output walks of at least WALK_IO_MIN walkers download their rows in id-ordered chunks
// (at most WALK_IO_MAX_CHUNKS) while the walk runs.
constexpr uint64_t WALK_IO_MIN = 1ull << 17;
constexpr uint32_t WALK_IO_MAX_CHUNKS = 32;
constexpr uint32_t WALK_IO_MIN_SHIFT = 14;
// Chunk c is downloaded on copy stream c % WALK_IO_STREAMS.  One stream: device-to-pinned-host copies
// on GB300 measured 187 GB/s from one stream and 184 GB/s split over four.
constexpr int WALK_IO_STREAMS = 1;

struct WalkTune {
    uint32_t lanes = 1;         // lanes per walker: 1, 4, 32
    uint32_t warps_per_block = 8;
    uint32_t blocks_per_sm = 0; // 0 = occupancy maximum
    uint32_t occ = 0;           // register budget variant: 0 = 64 registers, 1 = 40 registers
};

}  // namespace bingo

struct bingo_graph {
    bingo_config cfg;
    int device = 0;
    int num_sms = 0;
    unsigned apply_blocks = 0;  // resident k_apply blocks (persistent grid)
    uint32_t n = 0;
    uint64_t m_live = 0;
    uint64_t next_eid = 0;
    bingo::DevGraph G{};
    // owned device allocations
    void* d_hdr = nullptr;      // VHot[n]
    int l2_bytes = 0;           // the device's L2 size (walker cache policy)
    void* d_cold = nullptr;     // VCold[n]
    void* d_upd = nullptr;      // VUpd[n]
    void* d_order = nullptr;    // internal -> caller vertex id [n] (degree numbering), else null
    void* d_perm = nullptr;     // caller -> internal vertex id [n]
    void* d_pool = nullptr;
    void* d_ctl = nullptr;      // control words: top, npending, leaked, status, queue, counters
    void* d_fcount = nullptr;
    void* d_fstack = nullptr;
    void* d_pending = nullptr;
    void* d_eh = nullptr;       // edge index keys + counts
    uint64_t eh_distinct = 0;   // keys ever placed in the edge index (tombstones included)
    // scratch
    bingo::Buf s_in, s_keys, s_keys2, s_vals, s_vals2, s_tmp, s_seg, s_rank, s_best, s_aux, s_walk, s_stage;
    bingo::Buf s_rec, s_seginfo;  // sorted insertion records, per-segment {v, first key, ni, nd}
    bingo::Buf s_gcand, s_gcand_cnt;  // deletion candidates of big segments from the pre-pass
    bingo::Buf s_chunkmap;            // pre-pass chunk -> listed segment
    bingo::Buf w_starts, w_len, w_pid, w_paths, w_plen, w_pols, w_chunk_done;
    bingo::Buf w_len64, w_off, w_packed;  // packed walks: lengths as u64, their exclusive scan, packed rows
    // host-buffer walks: download streams, events, host-mapped chunk flags (see walk_host_io_overlap)
    cudaStream_t io_copy[bingo::WALK_IO_STREAMS] = {};
    cudaEvent_t io_kernel = nullptr, io_done[bingo::WALK_IO_STREAMS] = {};
    volatile uint32_t* io_flags = nullptr;  // host view, WALK_IO_MAX_CHUNKS words
    uint32_t* io_flags_dev = nullptr;       // device view of the same memory
    uint32_t io_seq = 0;
    // walk tuning
    bingo::WalkTune tune;
    // captured update pipelines: one graph per record capacity (power of two)
    uint64_t upd_cap = 0;
    bool upd_graph_eh = false;
    cudaGraphExec_t upd_graph = nullptr;
    uint64_t upd_graph_launches = 0;   // kernels per replay
    cudaStream_t cap_stream = nullptr; // capture stream (the caller's may be the legacy stream)
    uint64_t launches = 0;
    bool broken = false;        // a device-side failure left the state unusable
    bool part = false;          // a partition graph (vertex range of a larger graph): walks only through bingo_part_walk
};

// control-word layout inside d_ctl (u64 words)
enum CtlSlot : int {
    CTL_TOP = 0,
    CTL_NPENDING = 1,
    CTL_LEAKED = 2,
    CTL_STATUS = 3,     // u32 in the low half
    CTL_QUEUE = 4,
    CTL_STATS = 8,      // 30 u64: inserted, deleted, not_found, touched, rebuilt, conv[5][5]
    CTL_SCR = 40,       // scratch words of the update pipeline
    CTL_WORDS = 64
};
