// Error reporting, host/device pointer detection, device-wide exclusive scan and
// a stable LSD radix sort of (u64 key, u32 value) pairs.
#include <stdarg.h>
#include <stdio.h>

#include "bingo_host.h"

namespace bingo {

static thread_local std::string g_last_error;

const char* last_error_cstr() { return g_last_error.c_str(); }

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

bingo_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return BINGO_E_OOM;
    return BINGO_E_CUDA;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaError_t ensure(Buf& b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    want = (want + (want >> 3) + 255) & ~(size_t)255;  // 12.5% headroom
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return e;
    }
    b.bytes = want;
    return cudaSuccess;
}

void release(Buf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// ------------------------------------------------------------------------------------------- scan

constexpr int SCAN_T = 512;
constexpr int SCAN_I = 8;
constexpr uint64_t SCAN_TILE = (uint64_t)SCAN_T * SCAN_I;

__device__ __forceinline__ uint64_t block_scan_excl_u64(uint64_t x, uint64_t* sm, uint64_t& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t v = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(FULL, v, d);
        if (lane >= d) v += y;
    }
    if (lane == 31) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        uint64_t t = lane < nw ? sm[lane] : 0, s = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t y = __shfl_up_sync(FULL, s, d);
            if (lane >= d) s += y;
        }
        if (lane < nw) sm[lane] = s - t;
        if (lane == 31) sm[32] = s;
    }
    __syncthreads();
    uint64_t r = sm[w] + v - x;
    total = sm[32];
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const uint64_t* __restrict__ in, uint64_t n, uint64_t* __restrict__ part) {
    __shared__ uint64_t sm[40];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; i++) {
        uint64_t j = base + (uint64_t)i * SCAN_T + threadIdx.x;
        if (j < n) s += in[j];
    }
    uint64_t tot;
    block_scan_excl_u64(s, sm, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_scan_parts(uint64_t* part, uint64_t nparts, uint64_t* total_dev) {
    __shared__ uint64_t sm[40];
    uint64_t carry = 0;
    for (uint64_t b = 0; b < nparts; b += blockDim.x) {
        uint64_t j = b + threadIdx.x;
        uint64_t x = j < nparts ? part[j] : 0, tot;
        uint64_t e = block_scan_excl_u64(x, sm, tot);
        if (j < nparts) part[j] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_dev) *total_dev = carry;
}

__global__ void k_scan_apply(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint64_t n,
                             const uint64_t* __restrict__ part) {
    __shared__ uint64_t sm[40];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    // each thread owns SCAN_I consecutive elements
    uint64_t v[SCAN_I], s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; i++) {
        uint64_t j = base + (uint64_t)threadIdx.x * SCAN_I + i;
        v[i] = j < n ? in[j] : 0;
        s += v[i];
    }
    uint64_t tot;
    uint64_t e = block_scan_excl_u64(s, sm, tot) + part[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_I; i++) {
        uint64_t j = base + (uint64_t)threadIdx.x * SCAN_I + i;
        if (j < n) out[j] = e;
        e += v[i];
    }
}

// Second pass for inputs of at most SCAN_FUSED_TILES tiles: each block adds up the partial sums of
// the tiles before it itself (no separate pass over the partials); block 0 also writes the total.
constexpr uint64_t SCAN_FUSED_TILES = 1024;
__global__ void k_scan_apply_fused(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint64_t n,
                                   const uint64_t* __restrict__ part, uint64_t nparts, uint64_t* total_dev) {
    __shared__ uint64_t sm[40];
    uint64_t before = 0, all = 0;
    for (uint64_t j = threadIdx.x; j < nparts; j += SCAN_T) {
        const uint64_t x = part[j];
        if (j < blockIdx.x) before += x;
        all += x;
    }
    uint64_t tot;
    block_scan_excl_u64(before, sm, tot);
    const uint64_t prefix = tot;
    if (blockIdx.x == 0) {
        block_scan_excl_u64(all, sm, tot);
        if (threadIdx.x == 0 && total_dev) *total_dev = tot;
    }
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    uint64_t v[SCAN_I], s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; i++) {
        uint64_t j = base + (uint64_t)threadIdx.x * SCAN_I + i;
        v[i] = j < n ? in[j] : 0;
        s += v[i];
    }
    uint64_t e = block_scan_excl_u64(s, sm, tot) + prefix;
#pragma unroll
    for (int i = 0; i < SCAN_I; i++) {
        uint64_t j = base + (uint64_t)threadIdx.x * SCAN_I + i;
        if (j < n) out[j] = e;
        e += v[i];
    }
}

cudaError_t scan_excl_u64(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* total_dev, Buf& tmp,
                          cudaStream_t s, uint64_t* launches) {
    if (n == 0) {
        if (total_dev) return cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), s);
        return cudaSuccess;
    }
    const uint64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    cudaError_t e = ensure(tmp, nb * sizeof(uint64_t));
    if (e != cudaSuccess) return e;
    uint64_t* part = (uint64_t*)tmp.p;
    k_scan_reduce<<<(unsigned)nb, SCAN_T, 0, s>>>(in, n, part);
    if (nb <= SCAN_FUSED_TILES) {
        k_scan_apply_fused<<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, n, part, nb, total_dev);
        if (launches) *launches += 2;
        return cudaGetLastError();
    }
    k_scan_parts<<<1, 1024, 0, s>>>(part, nb, total_dev);
    k_scan_apply<<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, n, part);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------- radix sort

constexpr int RS_T = 256;
constexpr int RS_I = 8;
constexpr uint32_t RS_TILE = RS_T * RS_I;
constexpr int RS_BINS = 256;

// Pass 1: digit histogram of each tile of RS_TILE keys, stored [digit][tile].  Tiles past the key
// count write zeros.
__global__ void k_rs_hist(const uint64_t* __restrict__ keys, uint64_t n_host, const uint64_t* __restrict__ n_dev,
                          uint32_t shift, uint64_t nblocks, uint64_t* __restrict__ hist) {
    __shared__ uint32_t h[RS_BINS];
    const uint64_t n = n_dev ? *n_dev : n_host;
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int i = 0; i < RS_I; i++) {
        uint64_t j = base + (uint64_t)i * RS_T + threadIdx.x;
        if (j < n) atomicAdd(&h[(keys[j] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Up to this many tiles the scatter kernel forms its digit bases from the histogram itself (a row
// sum per digit); beyond it a separate exclusive scan over [digit][tile] provides them.
constexpr uint64_t RS_FUSED_TILES = 256;

// Pass 2, stable scatter.  Digit bases: `offs` = the exclusive scan of the histogram in [digit][tile]
// order, or (fused) thread d adds up its digit's counts: all tiles of smaller digits (through a
// block scan of the digit totals) plus the earlier tiles of digit d.  Keys of the tile are then
// ranked in index order, round by round.
__global__ void k_rs_scatter(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t n_host,
                             const uint64_t* __restrict__ n_dev, uint32_t shift, uint64_t nblocks,
                             const uint64_t* __restrict__ offs, bool fused, uint64_t* __restrict__ okeys,
                             uint32_t* __restrict__ ovals) {
    const uint64_t n = n_dev ? *n_dev : n_host;
    const uint64_t tbase = (uint64_t)blockIdx.x * RS_TILE;
    if (tbase >= n) return;
    __shared__ uint64_t base[RS_BINS];
    __shared__ uint64_t ssm[40];
    __shared__ uint32_t wc[RS_T / 32][RS_BINS];
    const int w = threadIdx.x >> 5;
    if (fused) {
        const uint64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
        const uint64_t* row = offs + (uint64_t)threadIdx.x * nblocks;
        uint64_t before = 0, all = 0;
#pragma unroll 8
        for (uint64_t b = 0; b < ntiles; b++) {
            const uint64_t c = row[b];
            before += b < blockIdx.x ? c : 0;
            all += c;
        }
        uint64_t tot;
        base[threadIdx.x] = block_scan_excl_u64(all, ssm, tot) + before;
    } else {
        base[threadIdx.x] = offs[(uint64_t)threadIdx.x * nblocks + blockIdx.x];
    }
    for (int r = 0; r < RS_I; r++) {
#pragma unroll
        for (int ww = 0; ww < RS_T / 32; ww++) wc[ww][threadIdx.x] = 0;
        __syncthreads();
        const uint64_t j = tbase + (uint64_t)r * RS_T + threadIdx.x;
        const bool ok = j < n;
        uint64_t k = ok ? keys[j] : 0;
        uint32_t v = ok ? vals[j] : 0;
        const uint32_t d = ok ? (uint32_t)((k >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(FULL, d);
        const uint32_t rk = __popc(peers & lanemask_lt());
        if (ok && rk == 0) wc[w][d] = __popc(peers);
        __syncthreads();
        {   // exclusive prefix over warps, per digit; advance the digit base
            const uint32_t t = threadIdx.x;
            uint32_t acc = 0;
#pragma unroll
            for (int ww = 0; ww < RS_T / 32; ww++) {
                uint32_t c = wc[ww][t];
                wc[ww][t] = acc;
                acc += c;
            }
            __syncthreads();
            if (ok) {
                const uint64_t pos = base[d] + wc[w][d] + rk;
                okeys[pos] = k;
                ovals[pos] = v;
            }
            __syncthreads();
            base[t] += acc;
        }
        __syncthreads();
    }
}

size_t radix_sort_tmp_bytes(uint64_t n) {
    const uint64_t nb = (n + RS_TILE - 1) / RS_TILE;
    const uint64_t nh = nb * RS_BINS;
    const uint64_t nscan_parts = (nh + SCAN_TILE - 1) / SCAN_TILE;
    return (2 * nh + nscan_parts + 8) * sizeof(uint64_t);
}

size_t scan_tmp_bytes(uint64_t n) { return ((n + SCAN_TILE - 1) / SCAN_TILE + 8) * sizeof(uint64_t); }

// Stable LSD radix sort of (key, value) pairs on bits [lo_bit, lo_bit + bits), 8-bit digits: two
// launches per digit up to RS_FUSED_TILES tiles, else histogram + scan + scatter.  With n_dev the
// key count is read on the device (n = capacity).
cudaError_t radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, uint64_t n,
                             uint32_t bits, Buf& tmp, cudaStream_t s, bool* result_in_alt, uint64_t* launches,
                             uint32_t lo_bit, const uint64_t* n_dev) {
    *result_in_alt = false;
    if ((n <= 1 && !n_dev) || bits == 0) return cudaSuccess;
    const uint64_t nb = (n + RS_TILE - 1) / RS_TILE;
    const uint64_t nh = nb * RS_BINS;
    const uint64_t nscan_parts = (nh + SCAN_TILE - 1) / SCAN_TILE;
    // tmp layout: hist [nh] | offs [nh] | scan parts
    cudaError_t e = ensure(tmp, radix_sort_tmp_bytes(n));
    if (e != cudaSuccess) return e;
    uint64_t* hist = (uint64_t*)tmp.p;
    uint64_t* offs = hist + nh;
    Buf part;  // view into tmp
    part.p = offs + nh;
    part.bytes = (nscan_parts + 8) * sizeof(uint64_t);
    const bool fused = nb <= RS_FUSED_TILES;
    uint64_t *ik = keys, *ok = keys_alt;
    uint32_t *iv = vals, *ov = vals_alt;
    bool alt = false;
    for (uint32_t shift = lo_bit; shift < lo_bit + bits; shift += 8) {
        k_rs_hist<<<(unsigned)nb, RS_T, 0, s>>>(ik, n, n_dev, shift, nb, hist);
        if (!fused) {
            e = scan_excl_u64(hist, offs, nh, nullptr, part, s, launches);
            if (e != cudaSuccess) return e;
        }
        k_rs_scatter<<<(unsigned)nb, RS_T, 0, s>>>(ik, iv, n, n_dev, shift, nb, fused ? hist : offs, fused, ok, ov);
        if (launches) *launches += 2;
        uint64_t* tk = ik; ik = ok; ok = tk;
        uint32_t* tv = iv; iv = ov; ov = tv;
        alt = !alt;
    }
    *result_in_alt = alt;
    return cudaGetLastError();
}

}  // namespace bingo
