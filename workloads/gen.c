/*
 * Seeded synthetic workload generators (graphs, biases, update streams, walk
 * starts).  Both the CPU oracle tests and the CUDA path's tests and bench draw
 * their inputs from here, so both sides see the same bytes.  Nothing in this
 * file computes any part of the sampling method: it only produces inputs.
 *
 * Every random number is a pure function of (seed, stream, index), so the
 * output does not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- splitmix64 finaliser used as a counter hash -------------------------------- */
static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline uint64_t hash3(uint64_t seed, uint64_t stream, uint64_t i) {
    return mix64(mix64(mix64(seed) ^ (stream * 0xD6E8FEB86659FD93ull)) ^ i);
}

/* Uniform integer in [0, range) by multiply-shift on a 64-bit hash (inputs only). */
static inline uint64_t below(uint64_t h, uint64_t range) {
    return (uint64_t)(((__uint128_t)h * range) >> 64);
}

/* ---- Philox4x32-10 (Salmon et al., SC'11), used for walk start vertices --------- */
static inline void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void wl_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; r++) {
        philox_round(c, k);
        k[0] += 0x9E3779B9u;
        k[1] += 0xBB67AE85u;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Walk start i = floor(philox(i,0,0,0; seed).x * n / 2^32). */
void wl_walk_starts(uint32_t n, uint64_t count, uint64_t seed, uint32_t* out) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; i++) {
        uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0, 0}, o[4];
        wl_philox4x32_10(ctr, key, o);
        out[i] = (uint32_t)(((uint64_t)o[0] * n) >> 32);
    }
}

/* ---- graphs ------------------------------------------------------------------- */

/* Directed Erdos-Renyi multigraph: m edges with uniform endpoints, no self-loops. */
void wl_er(uint32_t n, uint64_t m, uint64_t seed, uint32_t* src, uint32_t* dst) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)m; e++) {
        uint32_t s = (uint32_t)below(hash3(seed, 1, (uint64_t)e), n);
        uint32_t d;
        uint64_t t = 0;
        do {
            d = (uint32_t)below(hash3(seed, 2, ((uint64_t)e << 8) ^ t), n);
            t++;
        } while (d == s && n > 1);
        src[e] = s;
        dst[e] = d;
    }
}

/* Bijective relabelling of [0, 2^bits) (bits <= 31): a balanced 4-round Feistel
 * network on 2*ceil(bits/2) bits, cycle-walked back into range for odd widths,
 * so vertex ids lose the RMAT locality. */
static inline uint32_t feistel_even(uint32_t x, uint32_t h, uint64_t seed) {
    uint32_t mask = (1u << h) - 1u;
    uint32_t L = x >> h, R = x & mask;
    for (int r = 0; r < 4; r++) {
        uint32_t f = (uint32_t)hash3(seed, 100 + r, R) & mask;
        uint32_t nL = R;
        R = L ^ f;
        L = nL;
    }
    return (L << h) | R;
}

uint32_t wl_relabel(uint32_t x, uint32_t bits, uint64_t seed) {
    if (bits == 0) return 0;
    uint32_t h = (bits + 1) / 2;
    uint32_t y = feistel_even(x, h, seed);
    while (y >= (1u << bits)) y = feistel_even(y, h, seed);
    return y;
}

/* RMAT (Chakrabarti et al.) with quadrant probabilities (a, b, c, 1-a-b-c), no
 * noise; self-loops and duplicates kept; vertex ids relabelled by a seeded
 * bijection of [0, 2^scale). */
void wl_rmat(uint32_t scale, uint64_t m, double a, double b, double c, uint64_t seed,
             uint32_t* src, uint32_t* dst) {
    const uint64_t two32 = 4294967296ull;
    uint32_t ta = (uint32_t)(a * (double)two32);
    uint32_t tb = (uint32_t)((a + b) * (double)two32);
    uint32_t tc = (uint32_t)((a + b + c) * (double)two32);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)m; e++) {
        uint64_t st = hash3(seed, 3, (uint64_t)e);
        uint32_t s = 0, d = 0;
        for (uint32_t l = 0; l < scale; l++) {
            st = mix64(st);
            uint32_t u = (uint32_t)(st >> 32);
            uint32_t sb, db;
            if (u < ta) { sb = 0; db = 0; }
            else if (u < tb) { sb = 0; db = 1; }
            else if (u < tc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        src[e] = wl_relabel(s, scale, seed ^ 0x5EEDull);
        dst[e] = wl_relabel(d, scale, seed ^ 0x5EEDull);
    }
}

/* Extra out-edges of hub vertices: for each of `nhubs` hubs (distinct vertices
 * chosen uniformly), `per_hub` edges to uniform destinations. */
void wl_hubs(uint32_t n, uint32_t nhubs, uint64_t per_hub, uint64_t seed,
             uint32_t* hub_ids, uint32_t* src, uint32_t* dst) {
    for (uint32_t h = 0; h < nhubs; h++) {
        uint64_t t = 0;
        for (;;) {
            uint32_t v = (uint32_t)below(hash3(seed, 7, ((uint64_t)h << 20) ^ t++), n);
            int dup = 0;
            for (uint32_t j = 0; j < h; j++) dup |= (hub_ids[j] == v);
            if (!dup) { hub_ids[h] = v; break; }
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)((uint64_t)nhubs * per_hub); i++) {
        src[i] = hub_ids[(uint64_t)i / per_hub];
        dst[i] = (uint32_t)below(hash3(seed, 8, (uint64_t)i), n);
    }
}

/* ---- biases ------------------------------------------------------------------- */

void wl_bias_uniform(uint64_t m, uint32_t lo, uint32_t hi_excl, uint64_t seed, uint32_t* w) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)m; e++)
        w[e] = lo + (uint32_t)below(hash3(seed, 4, (uint64_t)e), (uint64_t)(hi_excl - lo));
}

/* floor(Pareto(alpha = 1.5, xmin = 1)) clipped to `cap`, in exact integer
 * arithmetic: with U = (x+1)/2^32, w >= k  <=>  U^(-2/3) >= k  <=>
 * k^3 (x+1)^2 <= 2^64.  The largest such k is found by bisection. */
void wl_bias_pareto15(uint64_t m, uint32_t cap, uint64_t seed, uint32_t* w) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)m; e++) {
        uint64_t x1 = (uint64_t)(uint32_t)(hash3(seed, 5, (uint64_t)e) >> 32) + 1ull;
        __uint128_t rhs = (__uint128_t)1 << 64;
        __uint128_t x2 = (__uint128_t)x1 * x1;
        uint64_t lo = 1, hi = cap; /* invariant: lo satisfies (x1 <= 2^32 so k=1 ok) */
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo + 1) / 2;
            __uint128_t k3 = (__uint128_t)mid * mid * mid;
            /* k3 * x2 <= 2^64  without overflow: compare k3 <= floor(2^64 / x2) */
            if (k3 <= rhs / x2) lo = mid; else hi = mid - 1;
        }
        w[e] = (uint32_t)lo;
    }
}

/* Fixed-point biases for float weights in [lo/256, hi/256): integer w_fx uniform in [lo, hi). */
void wl_bias_fixed(uint64_t m, uint32_t lo, uint32_t hi_excl, uint64_t seed, uint32_t* w) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)m; e++)
        w[e] = lo + (uint32_t)below(hash3(seed, 6, (uint64_t)e), (uint64_t)(hi_excl - lo));
}

/* ---- CSR ---------------------------------------------------------------------- */

/* Stable counting sort of an edge list by source into CSR (edge order within a
 * source follows the input order). row_ptr has n+1 entries. */
void wl_to_csr(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
               const uint32_t* w, uint64_t* row_ptr, uint32_t* col, uint32_t* wout) {
    memset(row_ptr, 0, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint64_t e = 0; e < m; e++) row_ptr[src[e] + 1]++;
    for (uint32_t v = 0; v < n; v++) row_ptr[v + 1] += row_ptr[v];
    uint64_t* pos = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    memcpy(pos, row_ptr, sizeof(uint64_t) * (size_t)n);
    for (uint64_t e = 0; e < m; e++) {
        uint64_t p = pos[src[e]]++;
        col[p] = dst[e];
        wout[p] = w[e];
    }
    free(pos);
}

/* ---- update streams ------------------------------------------------------------ */

/*
 * Mixed update stream in the paper's protocol (Section 5.1, datasets): the
 * generated edges are split into an initial set A and a held-out set B; each
 * update is a delete of a uniformly chosen live edge of A, or an insert that
 * moves the next edge of B into A.  Here every batch holds exactly `ins_per_batch`
 * inserts and `del_per_batch` deletes in a seeded random order.
 *
 * in:  edges (src, dst, w)[m] in generation order.
 * out: keep[m] = 1 for edges of A (the initial graph), 0 for B;
 *      ups_* [nbatch * (ins+del)] update records (op 0 insert, 1 delete; deletes carry bias 0).
 * Requires m > nbatch*ins_per_batch.
 */
int wl_update_stream(uint64_t m, const uint32_t* src, const uint32_t* dst, const uint32_t* w,
                     uint32_t nbatch, uint64_t ins_per_batch, uint64_t del_per_batch, uint64_t seed,
                     uint8_t* keep, uint32_t* up_src, uint32_t* up_dst, uint32_t* up_w, uint32_t* up_op) {
    uint64_t nins = (uint64_t)nbatch * ins_per_batch;
    if (nins >= m) return -1;
    /* B = a uniformly random subset of size nins: partial Fisher-Yates on an index array. */
    uint64_t* idx = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)m);
    if (!idx) return -2;
    for (uint64_t i = 0; i < m; i++) idx[i] = i;
    for (uint64_t i = 0; i < nins; i++) {
        uint64_t j = i + below(hash3(seed, 20, i), m - i);
        uint64_t t = idx[i]; idx[i] = idx[j]; idx[j] = t;
    }
    memset(keep, 1, (size_t)m);
    for (uint64_t i = 0; i < nins; i++) keep[idx[i]] = 0;
    /* live edges of A, as edge numbers into the generated list */
    uint64_t nlive = m - nins, cap = m;
    uint64_t* live = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)cap);
    if (!live) { free(idx); return -2; }
    uint64_t L = 0;
    for (uint64_t e = 0; e < m; e++) if (keep[e]) live[L++] = e;
    (void)nlive;
    uint64_t per = ins_per_batch + del_per_batch, bnext = 0, out = 0;
    uint8_t* isdel = (uint8_t*)malloc((size_t)per);
    for (uint32_t b = 0; b < nbatch; b++) {
        /* exact counts, random order */
        for (uint64_t i = 0; i < per; i++) isdel[i] = (i >= ins_per_batch);
        for (uint64_t i = per; i > 1; i--) {
            uint64_t j = below(hash3(seed, 21, ((uint64_t)b << 32) ^ i), i);
            uint8_t t = isdel[i - 1]; isdel[i - 1] = isdel[j]; isdel[j] = t;
        }
        for (uint64_t i = 0; i < per; i++, out++) {
            if (!isdel[i] || L == 0) {
                uint64_t e = idx[bnext++];
                live[L++] = e;
                up_src[out] = src[e]; up_dst[out] = dst[e]; up_w[out] = w[e]; up_op[out] = 0;
            } else {
                uint64_t j = below(hash3(seed, 22, out), L);
                uint64_t e = live[j];
                live[j] = live[--L];
                up_src[out] = src[e]; up_dst[out] = dst[e]; up_w[out] = 0; up_op[out] = 1;
            }
        }
    }
    free(isdel); free(live); free(idx);
    return 0;
}

/*
 * Update batch over an existing CSR graph where inserts are fresh uniform edges
 * (no self-loops) with uniform biases in [wlo, whi), and deletes pick uniformly
 * among the live edges (without replacement within the batch).
 */
void wl_uniform_batch(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col,
                      uint64_t nins, uint64_t ndel, uint32_t wlo, uint32_t whi, uint64_t seed,
                      uint32_t* up_src, uint32_t* up_dst, uint32_t* up_w, uint32_t* up_op) {
    for (uint64_t i = 0; i < nins; i++) {
        uint32_t s = (uint32_t)below(hash3(seed, 30, i), n), d;
        uint64_t t = 0;
        do { d = (uint32_t)below(hash3(seed, 31, (i << 8) ^ t++), n); } while (d == s && n > 1);
        up_src[i] = s; up_dst[i] = d; up_op[i] = 0;
        up_w[i] = wlo + (uint32_t)below(hash3(seed, 32, i), (uint64_t)(whi - wlo));
    }
    /* deletes: partial Fisher-Yates over edge numbers, then map to (src, dst) */
    uint64_t* pick = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(ndel ? ndel : 1));
    /* sparse Fisher-Yates via a small open hash of swapped positions would be
     * overkill here: ndel is small relative to m, so draw with rejection of repeats. */
    uint64_t got = 0, t = 0;
    while (got < ndel && got < m) {
        uint64_t e = below(hash3(seed, 33, t++), m);
        int dup = 0;
        for (uint64_t j = 0; j < got; j++) if (pick[j] == e) { dup = 1; break; }
        if (!dup) pick[got++] = e;
    }
    for (uint64_t i = 0; i < got; i++) {
        uint64_t e = pick[i];
        /* binary search the source of edge number e */
        uint32_t lo = 0, hi = n;
        while (hi - lo > 1) { uint32_t mid = lo + (hi - lo) / 2; if (row_ptr[mid] <= e) lo = mid; else hi = mid; }
        up_src[nins + i] = lo; up_dst[nins + i] = col[e]; up_w[nins + i] = 0; up_op[nins + i] = 1;
    }
    free(pick);
}

/* Seeded shuffle of update records (mixes inserts and deletes inside a batch). */
void wl_shuffle_updates(uint64_t count, uint64_t seed, uint32_t* s, uint32_t* d, uint32_t* w, uint32_t* op) {
    for (uint64_t i = count; i > 1; i--) {
        uint64_t j = below(hash3(seed, 40, i), i);
        uint32_t t;
        t = s[i - 1]; s[i - 1] = s[j]; s[j] = t;
        t = d[i - 1]; d[i - 1] = d[j]; d[j] = t;
        t = w[i - 1]; w[i - 1] = w[j]; w[j] = t;
        t = op[i - 1]; op[i - 1] = op[j]; op[j] = t;
    }
}

/* Uniform doubles in [0,1) for host-side schedules (Poisson arrivals, request sizes). */
void wl_uniform01(uint64_t count, uint64_t seed, uint64_t stream, double* out) {
    for (uint64_t i = 0; i < count; i++)
        out[i] = (double)(hash3(seed, 50 + stream, i) >> 11) * (1.0 / 9007199254740992.0);
}
