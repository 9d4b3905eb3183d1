/*
 * bingo.h — C ABI of a GB300 (sm_103a) library for biased random walks on
 * dynamic graphs with radix-factorised sampling (Bingo, arXiv 2504.10233).
 *
 * Method (Section 4.1): each integer edge bias w is split into its binary
 * digits, D(w) = {2^k : w AND 2^k != 0} (Eq. dwi).  Every vertex keeps one
 * neighbour group G_k per bit position k, with total W(p_k) = 2^k |G_k|
 * (Eq. wpk).  Sampling picks a group with probability W(p_k) / sum_j W(p_j)
 * (Eq. group_prob), then a member uniformly (Eq. pvp), which draws neighbour i
 * with probability w_i / sum w (Theorem 1).  Groups are stored as dense,
 * one-element, sparse or regular by Eq. group (Section 5.1); edge insertions
 * and deletions update the groups in place, batched per source vertex with a
 * two-phase delete-and-swap (Section 5.2).
 *
 * Conventions for every entry point:
 *  - Pointer arguments may be device pointers or host pointers; the library
 *    detects which (cudaPointerGetAttributes).  Host inputs are copied to the
 *    device and host outputs are copied back before the call returns.  Device
 *    pointers are used in place, in stream order on `stream`.
 *  - The caller owns all inputs and outputs; the library owns bingo_graph and
 *    bingo_server and everything they allocate.
 *  - No call throws.  Every call returns a bingo_status; bingo_last_error()
 *    returns a thread-local message for the last failure on this thread.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.
 *  - Vertex ids are < n < 2^31.  Integer biases are 1 <= w < 2^max_bits
 *    (max_bits <= 32).  Graphs created with bias_format BINGO_BIAS_F32 take
 *    real biases instead (see bingo_config and bingo_create).
 *  - Calls on one graph must not run concurrently from several host threads.
 */
#ifndef BINGO_H
#define BINGO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bingo_graph bingo_graph;
typedef struct bingo_server bingo_server;

typedef enum {
    BINGO_OK = 0,
    BINGO_E_INVALID = 1, /* bad argument or malformed batch; state unchanged */
    BINGO_E_OOM = 2,     /* device memory or the graph's pool is exhausted; state unchanged */
    BINGO_E_CUDA = 3,    /* a CUDA call failed (message in bingo_last_error) */
    BINGO_E_TIMEOUT = 4, /* a bounded wait expired (device or host side) */
    BINGO_E_STATE = 5    /* call not valid in the object's current state */
} bingo_status;

/* Group kinds of Eq. group (Section 5.1). */
enum { BINGO_KIND_EMPTY = 0, BINGO_KIND_DENSE = 1, BINGO_KIND_ONE = 2, BINGO_KIND_SPARSE = 3, BINGO_KIND_REGULAR = 4 };

/* Walk applications (Section 2.2; Section 6.1 evaluation settings). */
enum { BINGO_DEEPWALK = 0, BINGO_PPR = 1, BINGO_NODE2VEC = 2 };

/* Update operations (Section 4.2): insertion, deletion, and a bias change
 * built from one insertion plus one deletion of the same (src, dst). */
enum { BINGO_OP_INSERT = 0, BINGO_OP_DELETE = 1, BINGO_OP_SET_BIAS = 2 };

/* Walk execution forms (low byte of `mode`), plus flags. */
enum {
    BINGO_WALK_PERSISTENT = 0, /* one persistent launch; warps pull walkers from a device queue */
    BINGO_WALK_STEPWISE = 1,   /* one launch per step over all walkers (the paper's step-by-step form, Section 6) */
    BINGO_WALK_NO_PAD = 0x100  /* flag: leave path entries beyond path_len untouched instead of writing 0xFFFFFFFF */
};

/* Bias formats (bingo_config.bias_format). */
enum {
    BINGO_BIAS_U32 = 0, /* integer biases, radix-factorised directly (Section 4.1) */
    BINGO_BIAS_F32 = 1  /* real biases with amortisation factor lambda (Section 4.3), see bingo_create */
};

/* Internal vertex numbering (bingo_config.vertex_order).  Not part of the paper's method: the graph
 * may renumber its vertices by descending out-degree (ties by id) so that the vertex records
 * walks visit most sit together in memory.  Ids are translated at every call and each vertex
 * keeps its adjacency in the caller's CSR order, so the graph (edges, edge ids, group contents)
 * is the same under either numbering, and so are walks on a freshly created graph or after
 * insertions and streaming updates.  A batch that deletes edges applies a vertex's deletions in
 * the order of their internal destination ids, which can leave the slots inside the vertex
 * ordered differently; walks are then equal in distribution, not draw for draw. */
enum { BINGO_ORDER_AUTO = 0, BINGO_ORDER_CALLER = 1, BINGO_ORDER_DEGREE = 2 };

typedef struct {
    uint32_t alpha_pct;        /* Eq. group alpha, percent (paper: 40) */
    uint32_t beta_pct;         /* Eq. group beta, percent (paper: 10) */
    uint32_t max_bits;         /* K: bias bits, 1..32; biases must be < 2^max_bits */
    uint32_t lanes_per_walker; /* group-selection team width: 1, 4 or 32; 0 = tuned default */
    uint32_t warps_per_block;  /* walker kernel block size in warps, 1..24 (1..8 with reg_variant 1); 0 = tuned default */
    uint32_t blocks_per_sm;    /* walker kernel persistent blocks per SM; 0 = tuned default */
    uint32_t update_chunk;     /* vertex segments above this many adjacency slots (or above 256 records) are applied
                                  by a whole 512-thread block instead of one warp; 0 = 4096 */
    uint32_t reg_variant;      /* walker register budget: 0 = up to 80 registers, 1 = 40 registers (more resident warps) */
    uint64_t pool_words;       /* device pool for adjacency and group blocks, in 4-byte words; 0 = auto */
    uint32_t bias_format;      /* BINGO_BIAS_U32 (default) or BINGO_BIAS_F32 */
    uint32_t all_regular;      /* 1: no group adaption, every nonempty group in regular format (the paper's
                                  BS baseline, Section 6.2); 0 (default): Eq. group */
    double lambda;             /* BINGO_BIAS_F32: amortisation factor lambda > 0 (Section 4.3) */
    uint32_t radix_base;       /* 2 (default; 0 means 2) or 4: one group per base-4 digit position, split into
                                  value sub-groups (Appendix, Fig. base4); base 4 needs integer biases < 2^20 */
    uint32_t vertex_order;     /* internal vertex numbering: BINGO_ORDER_AUTO (0; by degree),
                                  BINGO_ORDER_CALLER (the caller's ids) or BINGO_ORDER_DEGREE; every call still
                                  takes and returns the caller's ids (see BINGO_ORDER_*) */
    uint32_t vertex_base;      /* partition graphs (bingo_part_*): global id of local vertex 0; 0 otherwise */
    uint32_t dst_space;        /* partition graphs: destinations are global ids < dst_space; 0 = n (a whole graph) */
    uint32_t hot_l2_hint;      /* walker loads of the hot vertex records: BINGO_HOT_AUTO (0) or BINGO_HOT_EVICT_LAST
                                  (an L2 evict-last policy), BINGO_HOT_NORMAL (the default policy) */
} bingo_config;
enum { BINGO_HOT_AUTO = 0, BINGO_HOT_EVICT_LAST = 1, BINGO_HOT_NORMAL = 2 };

/* One update record, 16 bytes. */
typedef struct {
    uint32_t src, dst, bias; /* bias ignored for BINGO_OP_DELETE; binary32 encoding in BINGO_BIAS_F32 graphs */
    uint32_t op;             /* BINGO_OP_* */
} bingo_update;

typedef struct {
    uint64_t inserted;          /* insertion records applied (op 0 and op 2) */
    uint64_t deleted;           /* deletions that removed an edge (op 1 and op 2) */
    uint64_t not_found;         /* deletions whose (src, dst) had no live copy */
    uint64_t conversions[5][5]; /* [old kind][new kind] group-kind changes of touched vertices (Table trans) */
    uint64_t vertices_touched;
    uint64_t groups_rebuilt;    /* groups rebuilt from the adjacency after a kind change or a capacity change */
} bingo_update_stats;

typedef struct {
    uint32_t kind;           /* BINGO_DEEPWALK | BINGO_PPR | BINGO_NODE2VEC */
    uint32_t max_len;        /* steps; the path holds at most max_len + 1 vertices */
    uint32_t ppr_stop_u32;   /* PPR: before every step, stop iff a uniform u32 < ppr_stop_u32 */
    uint32_t reserved;
    uint64_t n2v_accept[3];  /* node2vec: accept a candidate at distance 0/1/2 from the previous vertex iff a
                                uniform u32 < n2v_accept[dist]; values in [0, 2^32] = f(dist) / max f * 2^32 */
} bingo_policy;

/*
 * Fill a walk policy (Section 2.2; Section 6.1 evaluation settings) from its
 * real-valued parameters, so that callers need not derive the u32 thresholds:
 *   PPR: ppr_stop_u32 = round(ppr_stop * 2^32), saturated at 2^32 - 1;
 *        ppr_stop in [0, 1].
 *   node2vec (Eq. node2vec): f(dist) = 1/p, 1, 1/q at distance 0, 1, 2;
 *        n2v_accept[d] = round(f(d) / max f * 2^32), so a candidate at
 *        distance d is accepted with probability f(d) / max f (exact when the
 *        ratios are dyadic, e.g. p = 2, q = 0.5 gives 2^30, 2^31, 2^32);
 *        p, q > 0 and finite.
 *   DeepWalk: no parameters (ppr_stop, p, q ignored).
 * Errors: BINGO_E_INVALID for an unknown kind, out-of-range parameters or a
 * NULL out.  Host only; no device work.
 */
bingo_status bingo_policy_make(uint32_t kind, uint32_t max_len, double ppr_stop, double n2v_p, double n2v_q,
                               bingo_policy* out);

/* Library and build info. */
const char* bingo_version(void);
/* Thread-local message describing the last non-OK status on this thread. */
const char* bingo_last_error(void);
/* Default configuration: alpha 40, beta 10 (Section 5.1), max_bits 32, everything else tuned. */
void bingo_default_config(bingo_config* cfg);

/*
 * Build the factorised sampling state from a CSR graph (Section 4.1, sampling
 * space construction; Section 5.1, adaptive group representation).
 *   n        number of vertices (< 2^31)
 *   m        number of edges
 *   row_ptr  uint64[n+1], row_ptr[0] = 0, row_ptr[n] = m
 *   col      uint32[m]  destination of each edge
 *   bias     uint32[m]  1 <= bias < 2^cfg->max_bits; or, with cfg->bias_format =
 *            BINGO_BIAS_F32, the IEEE-754 binary32 encoding of a real bias b
 *   cfg      nullable: defaults of bingo_default_config
 * Edge ids are assigned 0..m-1 in CSR order; later insertions continue the count.
 * Real biases (Section 4.3, steps (i)-(iv)): x = lambda * b is rounded once to
 * binary64 and split into its integer part I = floor(x), radix-factorised into
 * groups 0..30 exactly like an integer bias, and its decimal part, kept to 8
 * fractional bits as q = floor((x - I) * 256).  The decimal parts of a vertex
 * form one extra group whose total Q_D = sum q occupies group slot 31; the
 * sampler draws neighbour i with probability (256 I_i + q_i) / sum_j (256 I_j +
 * q_j), the decimal group's member by rejection on q / 256 over the neighbour
 * list (with an exact inverse-transform fallback).  Requirements: b finite and
 * >= 0, lambda b < 2^31, 256 I + q >= 1 (no zero weights), degree < 2^24.
 * max_bits is ignored for real biases.
 * Radix base 4 (cfg->radix_base = 4, Appendix "arbitrary radix bases"): the
 * bias w < 2^20 is split into base-4 digits; group 4^i is kept as value
 * sub-groups v = 1, 2, 3 (the edges whose digit i equals v, each carrying
 * v 4^i), stored in group slot 3 i + v - 1 (slots 0..29) with the same kinds
 * (Eq. group), member lists and updates as base-2 groups; the sampler draws
 * sub-group (i, v) with probability v 4^i |S_iv| / sum w (group, then
 * sub-group) and a member uniformly.  cnt[] of bingo_export_state is indexed
 * by slot; bias[] holds the biases.
 * Errors: BINGO_E_INVALID (bad ids or biases; nothing allocated), BINGO_E_OOM, BINGO_E_CUDA.
 * Synchronises `stream` before returning.  *out receives the new graph.
 */
bingo_status bingo_create(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col,
                          const uint32_t* bias, const bingo_config* cfg, void* stream, bingo_graph** out);

/* Free the graph and everything it owns.  NULL is allowed. */
bingo_status bingo_destroy(bingo_graph* g);

/*
 * Apply one batch of updates in place (Section 5.2, parallel batched graph
 * updates; Section 4.2 for single-edge insertion and deletion).
 *   ups    bingo_update[count]
 *   stats  nullable host pointer; filled when given
 * Semantics: all insertions of the batch in batch order (new edge ids continue
 * after the largest id ever assigned), then all deletions in batch order, each
 * removing the live copy of (src, dst) with the smallest edge id (the earliest
 * version of a duplicated edge).  A deletion of a missing edge is counted in
 * not_found and is not an error.  BINGO_OP_SET_BIAS is an insertion of
 * (src, dst, bias) plus a deletion of (src, dst) under these rules.  Group
 * kinds are re-evaluated for every touched vertex after the batch.
 * Errors: BINGO_E_INVALID if any record has src or dst >= n, op > 2, or an
 * inserted bias outside [1, 2^max_bits): the whole batch is rejected before any
 * change.  BINGO_E_OOM if the pool cannot hold the batch's growth: the batch
 * is rejected before any change.  Synchronises `stream` before returning.
 */
bingo_status bingo_apply_updates(bingo_graph* g, const bingo_update* ups, uint64_t count, void* stream,
                                 bingo_update_stats* stats);

/*
 * Streaming updates (Section 4.2): the result is that of applying the records
 * one at a time, in order, each as a batch of size one (so kinds are
 * re-evaluated after every record and a deletion sees every earlier
 * insertion).  Records of one source vertex are applied in record order by one
 * warp; records of different source vertices touch disjoint state and run
 * concurrently; edge ids follow record order.  Same validation and stats as
 * bingo_apply_updates (an invalid record rejects the whole call before any
 * change).  BINGO_E_OOM: a record whose worst-case growth no longer fits the
 * pool is not applied and processing stops; records already applied (of any
 * vertex) stay applied, each one complete.  Synchronises `stream`.
 */
bingo_status bingo_stream_updates(bingo_graph* g, const bingo_update* ups, uint64_t count, void* stream,
                                  bingo_update_stats* stats);

/*
 * Random walks (Section 2.2; sampling by Eqs. group_prob and pvp, dense groups
 * by rejection on the neighbour list, Section 5.1; node2vec by rejection
 * against f(prev, x) of Eq. node2vec, first step first-order).
 *   nwalkers    number of walkers; walker i starts at starts[i]
 *   starts      uint32[nwalkers]
 *   lengths     nullable uint32[nwalkers]: step limit per walker (default: its policy's max_len)
 *   policy_ids  nullable uint8[nwalkers]: index into policies (default 0)
 *   policies    host array of npolicies bingo_policy (npolicies 1..16)
 *   seed        Philox4x32-10 key; walker i draws from counters (i, 0, step, j)
 *   stride      row length of paths (>= longest step limit + 1)
 *   paths       uint32[nwalkers][stride]: vertex sequence including the start, padded with 0xFFFFFFFF
 *   path_len    uint32[nwalkers]: vertices written (steps taken + 1)
 *   mode        BINGO_WALK_PERSISTENT or BINGO_WALK_STEPWISE
 * A vertex without out-edges ends the walk.  Results depend only on (graph
 * state, seed, walker index) — not on the launch shape or the mode.
 * Asynchronous on `stream` when every pointer is a device pointer.  Any array
 * may instead be a host pointer: inputs are staged to the device and outputs
 * copied back, and the call synchronises `stream`.  With host outputs and at
 * least 2^17 walkers, the persistent form downloads the rows in id-ordered
 * chunks (at most 32) on a library-owned copy stream while the walk runs: the
 * walker that completes a chunk flags it in host-mapped memory, and the
 * calling thread starts that chunk's copy.  Results are the same either way.
 */
bingo_status bingo_walk(bingo_graph* g, uint64_t nwalkers, const uint32_t* starts, const uint32_t* lengths,
                        const uint8_t* policy_ids, const bingo_policy* policies, uint32_t npolicies, uint64_t seed,
                        uint32_t stride, uint32_t* paths, uint32_t* path_len, uint32_t mode, void* stream);

/*
 * bingo_walk with packed output: each walker's path without padding, walkers
 * concatenated in id order, so that only visited vertices cross to a host
 * buffer (short PPR walks in long rows are mostly padding).
 *   max_steps  every walker's step limit (its policy's max_len, or lengths[i])
 *              must be <= max_steps (BINGO_E_INVALID otherwise)
 *   path_len   uint32[nwalkers]: vertices of walker i's path (steps + 1)
 *   vertices   uint32[capacity]: the paths; walker i's starts at the exclusive
 *              prefix sum of path_len
 *   total      nullable host uint64: sum of path_len
 * The result equals bingo_walk's with stride = max_steps + 1 (same lengths; the
 * packed vertices are each row's first path_len entries).  If the total
 * exceeds capacity the call returns BINGO_E_INVALID after writing path_len and
 * *total, and vertices is not written.  Arrays may be host or device pointers
 * (host inputs staged, host outputs copied back).  Synchronises `stream` (the
 * total sizes the copy).  Other arguments and errors as bingo_walk.
 */
bingo_status bingo_walk_packed(bingo_graph* g, uint64_t nwalkers, const uint32_t* starts, const uint32_t* lengths,
                               const uint8_t* policy_ids, const bingo_policy* policies, uint32_t npolicies,
                               uint64_t seed, uint32_t max_steps, uint32_t* path_len, uint32_t* vertices,
                               uint64_t capacity, uint64_t* total, void* stream);

/*
 * Allocation-free variant of bingo_walk.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they
 * walk (code inside an allocator or memory-pool callback, frameworks that
 * reserve all device memory up front, real-time loops that forbid
 * cudaMalloc/cudaFree because they can synchronise the device).  It runs the
 * same persistent walker and gives bit-identical results to bingo_walk, and it
 * calls no cudaMalloc, cudaFree or other allocating routine.
 * Its scratch (work counter and policy table) is a fixed 1 KiB array that the
 * library reserves on every device that loads it, held until process exit.
 *  - Limits: npolicies 1..16 (the table's capacity); larger counts return
 *    BINGO_E_INVALID.  Only BINGO_WALK_PERSISTENT (optionally with
 *    BINGO_WALK_NO_PAD).  starts, lengths, policy_ids, paths and path_len must
 *    be device pointers (host pointers would need staging: BINGO_E_INVALID).
 *    node2vec needs the edge index that an earlier bingo_walk built
 *    (BINGO_E_STATE otherwise).
 *  - The first call on each device resolves the scratch array's address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call on a device shares the one array and the counter is reset at
 *    the start of each call, so calls whose work overlaps on the GPU (different
 *    streams, or host threads without ordering) race; serialise them on one
 *    stream.  Asynchronous on `stream`; device-side errors are latched as for
 *    bingo_walk and reported by bingo_check.
 */
bingo_status bingo_walk_noalloc(bingo_graph* g, uint64_t nwalkers, const uint32_t* starts, const uint32_t* lengths,
                                const uint8_t* policy_ids, const bingo_policy* policies, uint32_t npolicies,
                                uint64_t seed, uint32_t stride, uint32_t* paths, uint32_t* path_len, uint32_t mode,
                                void* stream);

/*
 * Synchronise `stream` and return the device status latched by earlier
 * asynchronous calls on this graph (BINGO_E_INVALID for a bad start vertex,
 * policy id or length; BINGO_E_TIMEOUT if a bounded rejection loop gave up),
 * then clear it.
 */
bingo_status bingo_check(bingo_graph* g, void* stream);

/*
 * The walker's random numbers, evaluated on the device by the same code the
 * walk kernels run, so that the generator can be checked against published
 * known-answer vectors and other implementations.  The paper does not fix a
 * generator; walks use Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11).
 *
 * bingo_philox4x32_10: out[4i..4i+3] = Philox4x32-10(counter ctr[4i..4i+3],
 *   key key[2i..2i+1]) for i < count (count <= 2^26).  Host pointers.
 * bingo_walker_draws: the draws of walker `walker` at step `step` of a walk
 *   with Philox key `seed` (key words: seed low, seed high), in the order the
 *   walker consumes them: the u32 outputs of counters (walker low, walker
 *   high, step, 0), (.., 1), ..., four words per counter in output order
 *   (range 0); or, with range >= 1, successive exact uniform integers in
 *   [0, range) drawn from that stream by Lemire's multiply-shift with
 *   rejection (32-bit draws for range < 2^32, else two words, high first).
 *   count <= 2^20; out is a host uint64[count].
 * Both allocate scratch device memory on the current device and synchronise
 * it.  Errors: BINGO_E_INVALID (bad sizes or NULL), BINGO_E_TIMEOUT (a
 * bounded draw ran out of retries, probability below 2^-60), BINGO_E_CUDA.
 */
bingo_status bingo_philox4x32_10(uint64_t count, const uint32_t* ctr, const uint32_t* key, uint32_t* out);
bingo_status bingo_walker_draws(uint64_t seed, uint64_t walker, uint32_t step, uint64_t range, uint32_t count,
                                uint64_t* out);

/* Sizes needed by bingo_export_state (host pointer). */
typedef struct {
    uint64_t n;            /* vertices */
    uint64_t m;            /* live edges */
    uint64_t list_entries; /* member entries of all regular and sparse groups */
    uint64_t sparse_entries; /* entries of all sparse neighbour lists */
    uint64_t pool_words_used;
    uint64_t pool_words_total;
    uint64_t next_edge_id;
} bingo_state_sizes;

bingo_status bingo_state_sizes_get(bingo_graph* g, bingo_state_sizes* out);

/*
 * Copy the whole sampling state to host buffers (checkpoint and parity checks).
 * All pointers are host pointers sized from bingo_state_sizes_get:
 *   deg[n]; dst[m], bias[m], eid[m]: adjacency of each vertex in slot order,
 *     vertices concatenated in id order (offsets = prefix sum of deg);
 *   cnt[32n]: |G_k|; kind[32n]: BINGO_KIND_*;
 *   one_slot[32n]: slot of the single member of one-element groups (else 0xFFFFFFFF);
 *   glen[32n]: stored member-list length of regular and sparse groups (else 0);
 *   members[list_entries]: member lists in (vertex, k) order — slots for
 *     regular groups, positions in the vertex's sparse list for sparse groups;
 *   member_inv[list_entries]: the group's inverted index read at each member
 *     (must equal the member's own position);
 *   sp_len[n]; sp_list[sparse_entries]: each vertex's sparse neighbour list (slots);
 *   sp_inv[sparse_entries]: the sparse list's inverted index read at each entry.
 * Synchronises the graph's internal stream.
 */
bingo_status bingo_export_state(bingo_graph* g, uint32_t* deg, uint32_t* dst, uint32_t* bias, uint64_t* eid,
                                uint32_t* cnt, uint8_t* kind, uint32_t* one_slot, uint32_t* glen, uint32_t* members,
                                uint32_t* member_inv, uint32_t* sp_len, uint32_t* sp_list, uint32_t* sp_inv);

/*
 * The same export restricted to a list of vertices, for checking the state of
 * graphs whose whole export does not fit host memory (parity on sampled
 * vertices; per-source batch semantics, Section 5.2, make a source's state
 * depend only on its own initial edges and records).
 *   ids    uint32[count] caller vertex ids (host or device), each < n;
 *          duplicates allowed; 1 <= count <= 2^31
 *   sizes  host uint64[3]: {edges, list entries, sparse-list entries} of the
 *          listed vertices (the sizes of dst/bias/eid, members/member_inv and
 *          sp_list/sp_inv below)
 * bingo_export_vertices fills the arrays of bingo_export_state with row i
 * describing vertex ids[i]: deg[count], cnt/kind/one_slot/glen[32 count],
 * sp_len[count], and the variable-length arrays concatenated in row order.
 * Every output is a nullable host pointer.  Errors: BINGO_E_INVALID (an id
 * >= n, count out of range), BINGO_E_STATE (an inconsistent stored
 * destination), BINGO_E_CUDA.  Synchronises the device.
 */
bingo_status bingo_export_vertices_sizes(bingo_graph* g, const uint32_t* ids, uint64_t count, uint64_t sizes[3]);
bingo_status bingo_export_vertices(bingo_graph* g, const uint32_t* ids, uint64_t count, uint32_t* deg, uint32_t* dst,
                                   uint32_t* bias, uint64_t* eid, uint32_t* cnt, uint8_t* kind, uint32_t* one_slot,
                                   uint32_t* glen, uint32_t* members, uint32_t* member_inv, uint32_t* sp_len,
                                   uint32_t* sp_list, uint32_t* sp_inv);

/*
 * Real-bias graphs (BINGO_BIAS_F32, Section 4.3): the decimal part q of every live
 * edge, in units of 2^-8, in the edge order of bingo_export_state (host pointer,
 * m bytes).  The integer parts are that call's bias[] and the decimal totals
 * Q_D its cnt[32 v + 31] (kind[32 v + 31] is BINGO_KIND_EMPTY: the decimal group
 * is not a radix group).  BINGO_E_STATE on an integer-bias graph.  Synchronises
 * the graph's internal stream.
 */
bingo_status bingo_export_decimal(bingo_graph* g, uint8_t* q);

/* Bytes of device state by structure: [0] adjacency (with decimal parts), [1] counts+headers+group refs,
 * [2] regular groups, [3] sparse groups + sparse lists, [4] edge index, [5] pool capacity. */
bingo_status bingo_memory_report(bingo_graph* g, uint64_t out[6]);

/*
 * Autotune the walker launch (lanes per walker, warps per block, register variant)
 * on this graph with a trial walk of `nwalkers` DeepWalk walkers of `length`
 * steps from the given device/host starts; the best setting is stored in the
 * graph's config.  out_cfg (nullable) receives it.  Synchronises `stream`.
 */
bingo_status bingo_autotune(bingo_graph* g, uint64_t nwalkers, const uint32_t* starts, uint32_t length, void* stream,
                            bingo_config* out_cfg);

/*
 * Autotune the update pipeline's update_chunk (the adjacency size above which a vertex's
 * segment is applied by a whole block rather than one warp) on the caller's own records,
 * which ARE applied: they are split into consecutive equal slices, one per candidate setting
 * and round, applied in order as separate batches (each slice's insertions before its
 * deletions, every slice seeing the earlier ones), and the setting with the least time per
 * record is kept in the graph's config.  ups: bingo_update[count], host or device.  stats
 * (nullable) receives the sums over all slices; out_cfg (nullable) the resulting config.
 * Errors as bingo_apply_updates; on an error the slices applied so far stay applied.
 * Synchronises `stream`.  The paper has no counterpart (it fixes its kernel shapes).
 */
bingo_status bingo_autotune_updates(bingo_graph* g, const bingo_update* ups, uint64_t count, void* stream,
                                    bingo_update_stats* stats, bingo_config* out_cfg);

/*
 * Choose the group-adaption thresholds of Eq. group (alpha, beta; Section 5.1)
 * for a graph.  The paper fixes alpha = 40, beta = 10 and reports the memory
 * and time of adaption against keeping every group regular (Section 6.2,
 * Fig. Moptimization); which point of that trade-off is best depends on the
 * graph and the hardware, so this call measures it.  The graph is built from
 * the CSR (arguments as bingo_create; host or device pointers) under every
 * candidate alpha in {20, 40, 70, 100} (100: no group is ever dense) x beta in
 * {0, 10} (0: no group is ever sparse), with cfg's other fields.  Candidates
 * whose state (bingo_memory_report [0] + [1] + [2] + [3]) exceeds
 * state_budget_bytes (0 = no limit) are dropped; on each of the others a trial
 * walk of `nwalkers` DeepWalk walkers of `length` steps from `starts` (host or
 * device) is timed (one warm-up, two timed launches), and the graph with the
 * least walk time is returned in *out; the others are destroyed.  Kinds stay a
 * pure function of (|G_k|, d, alpha, beta), so every candidate samples
 * exactly.  out_cfg (nullable) receives the chosen config (alpha_pct,
 * beta_pct).  Errors: as bingo_create; BINGO_E_OOM if no candidate fits the
 * budget or the device; BINGO_E_INVALID for cfg->all_regular (nothing to
 * tune).  Synchronises `stream`.
 */
bingo_status bingo_autotune_adaption(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col,
                                     const uint32_t* bias, const bingo_config* cfg, uint64_t state_budget_bytes,
                                     uint64_t nwalkers, const uint32_t* starts, uint32_t length, void* stream,
                                     bingo_graph** out, bingo_config* out_cfg);

/* Current configuration of the graph (host pointer). */
bingo_status bingo_get_config(bingo_graph* g, bingo_config* out);
bingo_status bingo_set_walk_config(bingo_graph* g, uint32_t lanes_per_walker, uint32_t warps_per_block,
                                   uint32_t blocks_per_sm, uint32_t reg_variant);

/* Kernel launches issued by this graph so far (walk, update and build kernels). */
uint64_t bingo_kernel_launches(bingo_graph* g);

/* ---------------------------------------------------------------------------------------------- serving
 * Continuous-batching request loop (the paper's "integrate all updates before
 * each walk", Section 6 (ii)): a host thread owns the graph; streaming updates
 * are queued and applied at epoch boundaries (immediately when no walk launch
 * is in flight; otherwise new admissions pause once the oldest queued update
 * has waited update_delay_us, the in-flight launches drain, and the epoch
 * advances); walk requests are admitted while device memory and walker slots
 * allow, merged into shared launches, and complete independently.  A request binds to the epoch current at admission,
 * and its paths depend only on (that epoch's state, its seed, walker index).
 */
typedef struct {
    uint64_t max_inflight_walkers; /* walker slots; 0 = 4M */
    uint64_t hbm_reserve_bytes;    /* admission keeps this much device memory free; 0 = 1 GiB */
    uint32_t max_update_batch;     /* updates applied per epoch at most; 0 = 65536 */
    uint32_t concurrent_launches;  /* walk launches in flight at once; 0 = 4 */
    uint32_t max_len_cap;          /* longest step limit a request may ask for; 0 = 128 */
    uint32_t flags;                /* BINGO_SERVER_NO_MERGE: one request per launch (the plain form) */
    uint32_t update_delay_us;      /* longest time a queued update waits while walks keep being admitted; 0 = 1000 */
    uint32_t reserved;
} bingo_server_config;

enum { BINGO_SERVER_NO_MERGE = 1 };

typedef struct {
    uint64_t requests_done, walkers_done, steps_done, updates_applied, epochs;
    double p50_ms, p99_ms, mean_ms; /* arrival to completion, completed requests */
} bingo_server_stats;

/* The server takes over the graph until bingo_server_destroy; no other call may use it meanwhile. */
bingo_status bingo_server_create(bingo_graph* g, const bingo_server_config* cfg, bingo_server** out);
bingo_status bingo_server_destroy(bingo_server* s);
/* Queue updates (host records, copied); *epoch (nullable) receives the epoch that will include them. */
bingo_status bingo_server_submit_updates(bingo_server* s, const bingo_update* ups, uint64_t n, uint64_t* epoch);
/* Queue a walk request (host starts, copied).  Returns a ticket. */
bingo_status bingo_server_submit_walk(bingo_server* s, const uint32_t* starts, uint64_t nwalkers,
                                      const bingo_policy* policy, uint64_t seed, uint64_t* ticket);
/* Wait up to timeout_ms for a request; copies paths ([nwalkers][policy max_len+1]) and lengths to host
 * buffers, and the epoch it ran at.  BINGO_E_TIMEOUT if not done in time (it stays queued). */
bingo_status bingo_server_wait(bingo_server* s, uint64_t ticket, uint32_t timeout_ms, uint32_t* paths,
                               uint32_t* path_len, uint64_t* epoch);
/* Admission control.  While paused (paused != 0) no request is admitted; queued requests keep their
 * place and updates are still applied at epoch boundaries.  Resuming (paused = 0) admits as usual. */
bingo_status bingo_server_pause(bingo_server* s, uint32_t paused);

/* One request's progress, for callers that track admission and latency: state 0 queued, 1 running,
 * 2 done (status then holds its bingo_status); the epoch it was admitted at; the times it was
 * submitted, admitted and completed, in ms since the server was created (-1 = not yet).  Valid
 * until bingo_server_wait returns the request.  Admission: a request is admitted while the walker
 * slots in flight plus its walkers stay within max_inflight_walkers (a lone request is always
 * admitted) and its launch buffers leave hbm_reserve_bytes of device memory free; otherwise it
 * waits in the queue, in order, until launches complete or memory frees. */
typedef struct {
    uint32_t state, status;
    uint64_t walkers;
    uint64_t epoch;
    double submit_ms, admit_ms, done_ms;
} bingo_server_request_info;
bingo_status bingo_server_request_get(bingo_server* s, uint64_t ticket, bingo_server_request_info* out);

/* Block until every queued update and request has been processed (bounded by timeout_ms). */
bingo_status bingo_server_drain(bingo_server* s, uint32_t timeout_ms);
bingo_status bingo_server_stats_get(bingo_server* s, bingo_server_stats* out);

/* ---------------------------------------------------------------------------------------------- partitions
 * 1-D partitioned graphs and walks with walker migration (Supplement, dynamic graph support and
 * partitioning).  The vertices are split into contiguous ranges; each range's out-edges, groups and
 * vertex records form one partition graph (created like a whole graph: rows are the range's
 * vertices, destinations global ids).  A walk runs in supersteps: each partition resumes the
 * walkers standing on its vertices and runs each until it ends or steps onto another partition's
 * vertex, leaving a 24-byte record {walker, vertex, previous vertex, step}; the records are routed
 * to their owners for the next superstep until no walker is left.  node2vec's distance probe reads
 * the edge index of the previous vertex's owner.  Walker w draws from Philox counters (w, step, j)
 * wherever it runs, so paths equal those of the same walk on the whole graph (created with
 * BINGO_ORDER_CALLER and given the same updates).  Updates go to the owner of their source.  All
 * partitions live on the device current at creation.  Edge ids are assigned per partition (each
 * partition numbers its own edges in its CSR order, then its insertions in batch order).
 */
typedef struct bingo_partset bingo_partset;

/* Build the partitions of a CSR graph (arguments as bingo_create; row_ptr host or device).  bounds:
 * nullable host uint32[nparts + 1], 0 = bounds[0] < bounds[1] < ... < bounds[nparts] = n; NULL =
 * contiguous ranges with nearly equal edge counts.  Integer biases, radix base 2.  Errors as
 * bingo_create, BINGO_E_INVALID for bad bounds.  Synchronises `stream`. */
bingo_status bingo_part_create(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col,
                               const uint32_t* bias, const bingo_config* cfg, uint32_t nparts, const uint32_t* bounds,
                               void* stream, bingo_partset** out);
bingo_status bingo_part_destroy(bingo_partset* ps);
/* Partition p's graph (for bingo_export_vertices with local ids 0 .. hi-lo-1) and its range [lo, hi). */
bingo_status bingo_part_info(bingo_partset* ps, uint32_t p, bingo_graph** graph, uint32_t* lo, uint32_t* hi);
/* One batch (host or device records, global ids), validated as a whole, then each record applied by
 * the owner of its source in batch order (Section 5.2 semantics per source).  stats: sums over the
 * partitions.  BINGO_E_OOM in a partition leaves the earlier partitions' records applied. */
bingo_status bingo_part_apply_updates(bingo_partset* ps, const bingo_update* ups, uint64_t count, void* stream,
                                      bingo_update_stats* stats);
/* bingo_walk over the partitions (persistent form; device buffers only; arguments and results as
 * bingo_walk).  Synchronises `stream` once per superstep; device-side errors are latched in the
 * partitions and reported by bingo_part_check. */
bingo_status bingo_part_walk(bingo_partset* ps, uint64_t nwalkers, const uint32_t* starts, const uint32_t* lengths,
                             const uint8_t* policy_ids, const bingo_policy* policies, uint32_t npolicies, uint64_t seed,
                             uint32_t stride, uint32_t* paths, uint32_t* path_len, uint32_t mode, void* stream);
/* bingo_check over every partition (the first non-OK status). */
bingo_status bingo_part_check(bingo_partset* ps, void* stream);
/* Supersteps the last bingo_part_walk took. */
uint64_t bingo_part_supersteps(bingo_partset* ps);

#ifdef __cplusplus
}
#endif
#endif /* BINGO_H */
