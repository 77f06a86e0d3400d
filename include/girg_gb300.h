/*
 * C ABI of the GB300 GIRG / HRG generator (arXiv 1905.06706, Bläsius et al.).
 *
 * One call generates one random graph on the device: weights and positions
 * (Sec. 2.1, Sec. 5.1 steps 1-2), the constant c for a target average degree
 * (Sec. 4.1, App. B.2), weight buckets and the Morton-sorted vertex array with
 * per-cell prefix sums (Sec. 3.1, Sec. 3.4, Lemma 1), the cell pairs of
 * Algorithm 1 (Sec. 3.3, App. B.1), all-pairs tests on neighbouring cells and
 * geometric jumps on distant cells (Sec. 3.2), and compaction of the edges
 * into the caller's buffer.  The HRG entry point runs the same path through the
 * mapping of Sec. 2.3 with the connection probability of Sec. 2.2.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers, others are host pointers.
 *   - `stream` is a cudaStream_t (passed as void*); all device work is ordered
 *     on it.  Calls return after the edge count has been copied to the host,
 *     i.e. they synchronise the stream once at the end (and once after the
 *     weight reductions).
 *   - Scratch memory comes from a memory pool the library owns (one per device,
 *     cudaMallocFromPoolAsync on `stream`) and goes back to it before return; the
 *     pool keeps freed memory for later calls (girg_scratch_pool_trim returns it
 *     to the driver).  The caller's pools are not touched; the caller owns every
 *     buffer it passes.
 *   - Edges are unordered pairs (u, v), u < v, of original vertex ids, stored
 *     as two uint32 (edge_bytes = 4) or two uint64 (edge_bytes = 8) per edge,
 *     in unspecified order.  No self loops, no multi-edges.
 *   - The edge set is a deterministic function of the parameters and seed, and
 *     equals the FP64 oracle's edge for edge in both precision modes (the oracle's
 *     default build evaluates ln and exp by the same fixed-point method).  Against
 *     an oracle built on the C library's log / exp / pow, at most 1e-9 of the
 *     decisions differ, each within a relative 1e-12 of its threshold.
 *   - Return value: a GIRG_* status.  On GIRG_E_CAPACITY *num_edges holds the
 *     number of edges the graph has and the buffer holds an unspecified subset.
 */
#ifndef GIRG_GB300_H
#define GIRG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GIRG_OK 0
#define GIRG_E_PARAM 1    /* parameter out of range (see each field) */
#define GIRG_E_CAPACITY 2 /* edge buffer too small; *num_edges = required */
#define GIRG_E_CUDA 3     /* a CUDA call failed */
#define GIRG_E_RANGE 4    /* largest / smallest weight >= 2^43 (no exact 128-bit sum) */
#define GIRG_E_INTERNAL 5 /* internal capacity or consistency check failed */

#define GIRG_PRECISION_FP32 0 /* FP32 decisions, FP64 recheck inside the error band */
#define GIRG_PRECISION_FP64 1 /* every decision in FP64 */

/* GIRG parameters (Sec. 2.1).
 *   n          number of vertices, 2 <= n < 2^31
 *   d          dimension of the torus, 1 <= d <= 8
 *   beta       power-law exponent of the weights, beta > 2
 *   T          temperature, 0 <= T < 1 (0: threshold variant)
 *   avg_deg    target expected average degree, used when c <= 0; 0 < avg_deg < n - 1
 *   c          the constant of Eq. 1; c <= 0 means "solve from avg_deg" (App. B.2)
 *   w_min      smallest weight, > 0
 *   seed       64-bit seed of every Philox stream
 *   edge_bytes 4 (uint32 endpoints), 8 (uint64 endpoints) or 0 (count-only: no edge
 *              is stored, d_edges may be NULL and capacity_edges is ignored; the
 *              edge count and the checksum of girg_last_stats are still produced, as
 *              the paper's benchmarks replace storage by a checksum, Sec. 5)
 *   precision  GIRG_PRECISION_FP32 or GIRG_PRECISION_FP64
 *   level_cap  deepest quadtree level to use; 0 = default: min(32/d, (bitlen(n)+4)/d)
 *              at T = 0, min(32/d, floor((2 bitlen(n) - 2 - d) / (2d))) at T > 0 (about
 *              2^(d/2) vertices per cell, which balances the all-pairs tests of
 *              neighbouring cells against the distant cells' jumps); a tuning knob:
 *              the sample is exact for any value >= 1, the graph drawn depends on it
 */
typedef struct {
    int64_t n;
    int32_t d;
    double beta;
    double T;
    double avg_deg;
    double c;
    double w_min;
    uint64_t seed;
    int32_t edge_bytes;
    int32_t precision;
    int32_t level_cap;
} girg_params;

/* HRG parameters (Sec. 2.2).
 *   alpha      radial dispersion, alpha > 1/2 (power-law exponent 2 alpha + 1)
 *   T          temperature, 0 <= T < 1
 *   avg_deg    target expected average degree, used when R <= 0 (0 < avg_deg < n - 1)
 *   R          disk radius R = 2 ln n + C (Sec. 2.2); R <= 0: solved from avg_deg
 *              by the search of hrg_solve_radius, with the quadrature's inner
 *              integrals evaluated on the device at T > 0 (same rule; the radius
 *              agrees with hrg_solve_radius to about 1e-12 relative)
 *   other fields as for girg_params.
 */
typedef struct {
    int64_t n;
    double alpha;
    double T;
    double avg_deg;
    double R;
    uint64_t seed;
    int32_t edge_bytes;
    int32_t precision;
    int32_t level_cap;
} hrg_params;

/* Generate one GIRG (Sec. 2.1) by the cell-pair sampler (Algorithm 1).
 *   d_edges        buffer of capacity_edges edges (layout above): device memory, or
 *                  page-locked host memory mapped into the device address space
 *                  (cudaHostAlloc), which the kernels then fill across the host link
 *                  with no separate copy; pageable host memory gives GIRG_E_PARAM
 *   num_edges      host out: number of edges of the graph
 *   c_used         host out (may be NULL): the c of Eq. 1 that was used
 * Errors: GIRG_E_PARAM, GIRG_E_CAPACITY, GIRG_E_CUDA, GIRG_E_RANGE, GIRG_E_INTERNAL. */
int girg_generate(const girg_params* params, void* d_edges, int64_t capacity_edges,
                  int64_t* num_edges, double* c_used, void* stream);

/* Generate one GIRG on caller-provided points (user-defined weights, Sec. 4.1):
 *   d_X   device, d x n uint32, coordinate k of vertex v at d_X[k * n + v]; the
 *         torus coordinate is d_X[k*n+v] * 2^-32
 *   d_w   device, n doubles > 0 (the smallest one is the bucket unit w_min)
 *   T, c  as in Eq. 1 (c > 0 required here)
 * Other arguments as for girg_generate. */
int girg_generate_from_points(int64_t n, int32_t d, const uint32_t* d_X, const double* d_w,
                              double T, double c, uint64_t seed, int32_t precision,
                              int32_t level_cap, int32_t edge_bytes, void* d_edges,
                              int64_t capacity_edges, int64_t* num_edges, void* stream);

/* Generate one HRG (Sec. 2.2) through the HRG -> GIRG mapping (Sec. 2.3).
 *   R_used   host out (may be NULL): the disk radius used (params->R, or the solved one)
 * Other arguments and errors as for girg_generate. */
int hrg_generate(const hrg_params* params, void* d_edges, int64_t capacity_edges,
                 int64_t* num_edges, double* R_used, void* stream);

/* Expected average degree of an HRG with n vertices, dispersion alpha, temperature T
 * and disk radius R (host computation, no GPU).  The paper gives no formula (Sec. 2.2:
 * R = 2 ln n + C, C sets the degree); this is (n - 1) P(edge) for two random vertices,
 * P(edge) = P(dist < R) at T = 0 and E[P(dist < t)] for t logistic with location R
 * and scale 2T at T > 0, by numerical quadrature (relative error about 1e-11).
 * Errors: GIRG_E_PARAM (n < 2, alpha <= 1/2, T outside [0, 1), R outside (0, 350]). */
int hrg_expected_avg_degree(int64_t n, double alpha, double T, double R, double* avg_deg);

/* The disk radius R whose expected average degree (hrg_expected_avg_degree) equals
 * avg_deg, to 1e-13 relative (host computation, no GPU).
 * Errors: GIRG_E_PARAM (as above, or avg_deg outside (0, n - 1) or unreachable). */
int hrg_solve_radius(int64_t n, double alpha, double T, double avg_deg, double* R);

/* The quadratic all-pairs generator (Table 1, "Pairwise") on the device: every
 * pair u < v is tested with the same per-pair coin as the type-I tests.  Inputs as
 * for girg_generate_from_points plus W = sum of the weights (must equal the exactly
 * rounded sum for parity with other paths).  Quadratic work: for validation and as
 * the plain-FP64 baseline. */
int girg_allpairs(int64_t n, int32_t d, const uint32_t* d_X, const double* d_w, double W,
                  double T, double c, uint64_t seed, int32_t precision, int32_t edge_bytes,
                  void* d_edges, int64_t capacity_edges, int64_t* num_edges, void* stream);

/* Largest n accepted by girg_allpairs_noalloc. */
#define GIRG_NOALLOC_MAX_N (1 << 20)

/* girg_allpairs without any device allocation.  The paper has no counterpart of this
 * entry point: it exists for callers that cannot allocate device memory, e.g. a
 * plug-in inside a host application that owns the whole device memory pool, or a
 * latency-critical loop where an allocation could block or fail under memory
 * pressure.  Arguments, results and errors are those of girg_allpairs, except that
 * n must not exceed GIRG_NOALLOC_MAX_N (larger n returns GIRG_E_PARAM before any
 * device work), and that d_X, d_w and d_edges are checked before any device work:
 * each must be device memory or page-locked host memory mapped into the device
 * (cudaHostAlloc); pageable host memory or a pointer CUDA does not know returns
 * GIRG_E_PARAM.  Its scratch (a per-vertex scale and the edge counters, about 4 MiB)
 * is a fixed device array of the library, held by every GPU that loads the library
 * until the process exits.  The first call on a device looks up that array's device
 * address (once per device, with the device current); make that first call before
 * any stream capture.  The address is kept for the life of the process, so
 * cudaDeviceReset is not supported while the library is loaded.  All calls share the
 * array, which keeps the last call's contents (the counters are cleared at the start
 * of every call): calls whose device work overlaps -- on different streams or host
 * threads -- race on it and must be serialised by the caller.  Like girg_allpairs,
 * the call synchronises `stream` before it returns (it reads the edge count back). */
int girg_allpairs_noalloc(int64_t n, int32_t d, const uint32_t* d_X, const double* d_w,
                          double W, double T, double c, uint64_t seed, int32_t precision,
                          int32_t edge_bytes, void* d_edges, int64_t capacity_edges,
                          int64_t* num_edges, void* stream);

/* Weights and positions of girg_generate (Sec. 2.1, Sec. 5.1 steps 1-2) into caller
 * buffers: d_w n doubles, d_X d x n uint32 (layout as above). */
int girg_points(int64_t n, int32_t d, double beta, double w_min, uint64_t seed, double* d_w,
                uint32_t* d_X, void* stream);

/* Radii and angular fixed-point coordinates of hrg_generate (Sec. 2.2): d_r n doubles,
 * d_X n uint32 (theta = 2 pi d_X[v] 2^-32). */
int hrg_points(int64_t n, double alpha, double R, uint64_t seed, double* d_r, uint32_t* d_X,
               void* stream);

/* The vertices of hrg_generate as GIRG points through the mapping of Sec. 2.3:
 * d_w n doubles, w_v = e^((R - r_v)/2); d_X n uint32, the 1-dimensional torus
 * coordinate theta_v / (2 pi) in fixed point (the same bits as hrg_points). */
int hrg_girg_points(int64_t n, double alpha, double R, uint64_t seed, double* d_w, uint32_t* d_X,
                    void* stream);

/* Expected average degree f(c) of App. B.2 for a GIRG with these parameters and
 * weights generated from params->seed (params->c is the c evaluated). */
int girg_expected_avg_degree(const girg_params* params, double* avg_deg, void* stream);

/* The scale K of Eq. 1 used by the last generate call on this host thread: Eq. 1 is
 * evaluated as p = min{1, (K q / r^d)^(1/T)}, q = w_u w_v / W, with K = c^T (T > 0),
 * and the threshold variant as r^d <= K q with K = c^d (T = 0).  K stays a moderate
 * number for every T, where c_used = K^(1/T) under- or overflows a double as T -> 0
 * (it is then reported as 0 or infinity). */
double girg_last_scale(void);

/* Resident point sets, for serving the same point set more than once.  With
 * max_bytes > 0, girg_generate keeps the layout of each graph it builds on the device:
 * the weight buckets and levels, the Morton-sorted vertex arrays with their cell
 * offsets (Sec. 3.1, 3.4, Lemma 1) and the bound tables of the distant cell pairs
 * (Sec. 3.2), keyed by n, d, beta, w_min, seed, T, c (or avg_deg when c <= 0) and
 * level_cap.  A later call with the same values skips the weights and positions, the
 * reductions, the search for c and the sort, and makes the same graph.  Least recently
 * used layouts are dropped beyond max_bytes (a layout larger than max_bytes is not
 * kept); an entry still in use by a call is freed when that call returns.  The memory
 * comes from the library's scratch pool and is not part of girg_scratch_bytes.
 * max_bytes = 0 (the default) turns the cache off and frees it.  Errors: GIRG_E_PARAM
 * (max_bytes < 0). */
int girg_point_cache(int64_t max_bytes);

/* Layouts kept, their bytes, and the cache hits and misses of girg_generate calls since
 * the cache was turned on.  Out pointers may be NULL. */
int girg_point_cache_stats(int64_t* entries, int64_t* bytes, int64_t* hits, int64_t* misses);

/* The library's scratch pool on the current device: bytes reserved from the driver,
 * bytes in use now, and the most bytes in use at once since the pool was created or
 * last reset (reset_high != 0 resets that mark after reading it).  Out pointers may be
 * NULL.  Errors: GIRG_E_CUDA. */
int girg_scratch_pool_usage(int64_t* reserved, int64_t* used, int64_t* used_high,
                            int32_t reset_high);

/* Return unused memory of the library's scratch pool on the current device to the
 * driver, keeping at most keep_bytes reserved.  Errors: GIRG_E_PARAM (keep_bytes < 0),
 * GIRG_E_CUDA. */
int girg_scratch_pool_trim(int64_t keep_bytes);

/* Expected number of edges of the graph girg_generate would make with these parameters
 * (n f / 2, f the expected average degree of App. B.2 for the generated weights; c > 0
 * is used as given, else the c solved for avg_deg), for sizing the edge buffer; the
 * realized count fluctuates around it.  Returns -1 on invalid parameters or a CUDA
 * error. */
int64_t girg_expected_edges(const girg_params* params, void* stream);

/* Counters of the last generate call on this host thread: [0] type-I pairs tested,
 * [1] coins drawn, [2] FP64 rechecks, [3] type-II items (non-empty cell pairs),
 * [4] jump draws, [5] type-II candidates, [6] rows, [7] type-I items, [8] chunks of
 * all type-II streams, [9] edges, [10] kernel launches, [11] vertex references of the type-I items
 * (sum of both side lengths), [12] type-I edges, [13] type-II streams, [14] edge
 * checksum: the sum mod 2^64 over the edges (u < v) of the splitmix64 finalizer of
 * u 2^32 + v (as an int64 bit pattern; independent of the edge order), [15] type-II
 * partner segments, [16] enumeration passes (rounds plus reruns after a work list
 * grew), [17] type-II work entries and [18] type-I work entries (rows times the
 * buckets they pair with).  Copies min(len, 19) values; returns the number copied. */
int girg_last_stats(int64_t* out, int32_t len);

/* Milliseconds spent in each phase of the last call on this host thread
 * (CUDA events): [0] points+reductions, [1] host work up to the layer partition
 * (search for c, levels), [2] keys+sort+gather, [3] cell-pair enumeration with the
 * scans of its lists, [4] the type-I kernel, [5] the type-II kernel, [6] total; host wall clock: [7] reduction readback, [8] search
 * for c, [9] table build (the type-II bound tables are built while the sort runs on
 * the device).  Copies
 * min(len, 10) values; returns the number copied. */
int girg_last_phase_ms(float* out, int32_t len);

/* Sorted vertex order of the bucket/Morton sort (Sec. 3.4) for the given points:
 * d_order (device, n int64) receives the original id at each sorted position.
 * Used to check the sort against the oracle. */
int girg_sorted_order(int64_t n, int32_t d, const uint32_t* d_X, const double* d_w, double T,
                      double c, int32_t level_cap, int64_t* d_order, void* stream);

/* The library's deterministic FP64 elementary functions, evaluated on the host (the
 * host builds the type-II bound tables with them; the device uses the same steps):
 * fn 0 ln x, 1 ln(1+x), 2 e^x, 3 x^y, 4 sin(pi x) for x in [0, 1/2], 5 acosh x,
 * 6 the GIRG probability of Eq. 1 at weights (x, y), r = 1/4, W = 1000, c = 1/2,
 * T = 3/4, d = 2, 7 the weight layer (Sec. 3.1) of weight x with minimum weight y as the
 * reduction and key kernels take it (from the bit fields, no division).  Returns NaN for
 * an unknown fn.  Diagnostic; no GPU needed. */
double girg_det_eval(int32_t fn, double x, double y);

/* Measured warp-instruction issue rate (the denominator of the pair kernels' issue
 * roofline).  One launch of a probe kernel that fills every SM (two 1024-thread
 * blocks per SM) with runs of one instruction kind over eight independent register
 * chains: kind 0 integer logic (lop3), 1 integer multiply-add (mad.lo.u32), 2 FP32
 * fused multiply-add.  iters in [1, 2^24] loop trips of 128 instructions per thread.
 * Writes the launch's CUDA-event time in *ms and the warp instructions the probe
 * issues by construction (blocks x 32 warps x iters x 128; the loop's own few
 * instructions per trip are not counted) in *warp_instructions.  Synchronises the
 * stream.  Errors: GIRG_E_PARAM (kind, iters or a null pointer), GIRG_E_CUDA.
 * Diagnostic: the paper has no counterpart. */
int girg_issue_probe(int32_t kind, int64_t iters, void* stream, float* ms,
                     int64_t* warp_instructions);

/* ------------------------------------------------------------------------
 * Continuous-batching server (many requests in flight on one GPU).
 * Worker threads each run girg_generate on their own CUDA stream, so the kernels
 * of concurrent requests overlap.  A request starts when a worker is free and its
 * estimated scratch (girg_scratch_bytes) fits memory_budget_bytes next to the
 * running ones (one request always may run); requests start in submission order,
 * except that up to 16 later requests that fit may pass one that does not.  Each
 * result equals that of a lone girg_generate call with the same parameters.  The
 * caller owns the edge buffers and must keep them alive until the result is polled.
 * The paper has no counterpart (its generator makes one graph per call). */
typedef struct girg_server girg_server;

typedef struct {
    int64_t request_id;  /* as submitted */
    int32_t status;      /* GIRG_* of the generation */
    int32_t pad;
    int64_t num_edges;
    double c_used;
    uint64_t checksum;   /* edge checksum, as girg_last_stats()[14] */
    double t_submit_us;  /* server clock (girg_server_clock_us) */
    double t_start_us;
    double t_done_us;
} girg_request_result;

/* Estimated peak device scratch of girg_generate for these parameters (bytes), or -1. */
int64_t girg_scratch_bytes(const girg_params* params);
/* Start `workers` worker threads on the current device.  Errors: GIRG_E_PARAM, GIRG_E_CUDA. */
int girg_server_create(int32_t workers, int64_t memory_budget_bytes, girg_server** out);
/* Queue one request (non-blocking; parameters are copied).  d_edges / capacity_edges as
 * for girg_generate (edge_bytes 0: count-only). */
int girg_server_submit(girg_server* server, const girg_params* params, void* d_edges,
                       int64_t capacity_edges, int64_t request_id);
/* Move up to max_results finished results into out (completion order); if wait_for > 0,
 * first block until min(wait_for, max_results) are available or nothing is queued or
 * running.  Returns the number written, or -GIRG_E_PARAM. */
int girg_server_poll(girg_server* server, girg_request_result* out, int32_t max_results,
                     int32_t wait_for);
/* Requests queued or running. */
int girg_server_pending(girg_server* server);
/* Microseconds since the server was created (the clock of the result timestamps). */
double girg_server_clock_us(girg_server* server);
/* Finish every queued request, stop the workers and free the server. */
int girg_server_destroy(girg_server* server);

/* Human-readable name of a status code (static storage). */
const char* girg_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* GIRG_GB300_H */
