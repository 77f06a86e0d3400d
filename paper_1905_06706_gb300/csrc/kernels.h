// Launchers of the device kernels (host-side declarations).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gg {

struct DevCfg;

// Copy the tables of det_log / det_exp to the current device for the kernels of
// gen.cu and pairs.cu (once per device; false if the copy failed).
bool det_tables_gen();
bool det_tables_pairs();

// Streaming multiprocessors of the current device (queried once per device); grids of
// grid-stride and persistent kernels are sized from it.
int device_sms();

// Kernel launches issued by the library on this host thread (for the benchmark's
// launch count).
extern thread_local unsigned long long g_launches;

// Results of the weight reduction pass.
struct Reduce {
    unsigned long long sum_lo, sum_hi;  // exact sum of the weights in units of 2^E0
    unsigned long long cnt[64];         // vertices per bucket
    unsigned long long wmax[64];        // largest weight per bucket (bits)
    unsigned long long rmin[64];        // HRG: smallest radius per bucket (bits)
    unsigned long long rmax[64];        // HRG: largest radius per bucket (bits)
    double s2;                          // sum w^2 (filled by the split threshold)
    unsigned int range_error;
    unsigned int blocks_done;           // blocks of the reduction finished
};

// The split threshold computed by the last block of the reduction (thr null: none).
struct ThresholdJob {
    int d;
    double T, target;
    double* thr;
};

void launch_girg_points(int64_t n, int d, double beta, double w_min, uint64_t seed, double* w,
                        uint32_t* X, cudaStream_t st);
void launch_hrg_points(int64_t n, double alpha, double R, uint64_t seed, double* r, double* w,
                       uint32_t* X, cudaStream_t st);
void launch_min_weight(int64_t n, const double* w, unsigned long long* out, cudaStream_t st);
// P(dist < t) of two random vertices of the hyperbolic disk (radius R, dispersion
// alpha) at each of the nt nodes d_ts: the double integral over the radii with the y
// rule (nodes a + (b - a) c[k], weights (b - a) w[k] on every smooth interval [a, b]),
// one block per node and interval, summed in a fixed order.  d_g (4 nt doubles)
// receives the parts of the node's at most four intervals; their sum in order is the CDF.
constexpr int kHrgYMax = 32;
struct HrgYRule {
    double c[kHrgYMax], w[kHrgYMax];
    int n;
};
void launch_hrg_dist_cdf(double alpha, double R, const HrgYRule& Y, const double* d_ts, int nt,
                         double* d_g, cudaStream_t st);
// Blocks of the reduction (one per-block partial each): a fixed partition of the
// vertices (a function of n alone, at least eight weights a thread up to 1216 blocks),
// independent of the device, so that the sums finished in block order round the same
// way on every GPU.
int reduce_blocks(int64_t n);
// part_s2 (reduce_blocks(n) doubles, or null): per-block sums of w^2.  With job (and
// part_s2), the last block also finishes red->s2 in block order and writes the split
// threshold of the degree model (App. B.2), estimated from the reduction, to job->thr.
void launch_reduce(int64_t n, const double* w, const double* r, double w_min, int E0,
                   double* part_s2, Reduce* out, cudaStream_t st,
                   const ThresholdJob* job = nullptr);
// The split of the weights for the degree model: one pass that gathers the weights
// above *thr into out (count[0] of them; copied to `sorted` in decreasing order when
// count[0] <= kTopSortMax, count[1] = 1) and sums over the rest: sums[0..3] = sum w,
// sum w^2, sum (w/thr)^(1/T), sum (w/thr)^(2/T) (finished in block order by the last
// block; count[2] counts the blocks and starts at 0).  part: 4 reduce_blocks(n)
// doubles; sorted: kTopSortMax doubles.
constexpr unsigned int kTopSortMax = 4096;  // ranked in 32 KB of static shared memory
void launch_split_weights(int64_t n, const double* w, const double* thr, double T, double* out,
                          unsigned int cap, unsigned int* count, double* part, double* sums,
                          double* sorted, cudaStream_t st);

// Sorting: keys (global cell index at the insertion level) with a histogram; val
// receives each vertex's arrival slot in its cell (slots) or its id (for the radix sort).
void launch_keys(int64_t n, int d, const double* w, const uint32_t* X, double w_min,
                 const int8_t* I, const uint32_t* layer_base, uint32_t* key, uint32_t* val,
                 uint32_t* cnt, bool slots, cudaStream_t st);
// Exclusive scan of n uint32 values in place (out may alias in); tmp >= scan_tmp_words(n).
size_t scan_tmp_words(int64_t n);
void launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t st);
// Exclusive scan of n uint32 counts into uint64 prefixes; tmp >= scan_tmp_words(n) uint64s.
void launch_scan_u32_to_u64(const uint32_t* in, unsigned long long* out, int64_t n,
                            unsigned long long* tmp, cudaStream_t st);
// The same with the length min(*n_dev, n_max) read on the device (tmp sized for n_max).
void launch_scan_u32_to_u64_dev(const uint32_t* in, unsigned long long* out,
                                const unsigned long long* n_dev, int64_t n_max,
                                unsigned long long* tmp, cudaStream_t st);
// Stable LSD radix sort of (key, val) on the low `bits` bits of key.
size_t radix_tmp_words(int64_t n);
void radix_sort_pairs(uint32_t* key, uint32_t* val, uint32_t* key_alt, uint32_t* val_alt,
                      int64_t n, int bits, uint32_t* tmp, cudaStream_t st, uint32_t** key_out,
                      uint32_t** val_out);
// n positive doubles in decreasing order (out must not alias in); words >=
// sort_desc_words(n) uint32 of scratch.
size_t sort_desc_words(int64_t n);
void sort_f64_desc(const double* in, int64_t n, double* out, uint32_t* words, cudaStream_t st);
// The same order by placement: key and slot from launch_keys (slots) and the scanned
// cell histogram offs; writes the sorted keys to skey and the sorted ids to sid (kt:
// scratch of n key-id pairs; skey and sid may reuse key and slot).  tmp >=
// place_tmp_words(n) words with tmp[0] zeroed.
size_t place_tmp_words(int64_t n);
void place_by_counts(const uint32_t* key, const uint32_t* slot, const uint32_t* offs, int64_t n,
                     uint2* kt, uint32_t* skey, uint32_t* sid, uint32_t* tmp, cudaStream_t st);
// Sorted per-vertex arrays.
// With rec (d <= 4): packed records instead of Xs and sv (see DevCfg::vrec).
void launch_gather_girg(int64_t n, int d, const uint32_t* perm, const uint32_t* X,
                        const double* w, double w_min, double log2W_half, float gamma,
                        float invd, uint32_t* Xs, double* ws, float* sv, uint8_t* slayer,
                        uint4* rec, cudaStream_t st);
void launch_gather_hrg(int64_t n, const uint32_t* perm, const uint32_t* X, const double* r,
                       const double* w, uint32_t* Xs, double* rs, float* E32, float* einv32,
                       float* sh32, uint8_t* slayer, uint4* hrec, cudaStream_t st);

// Pair sampling.
void launch_rows(const DevCfg& cfg, cudaStream_t st);
void launch_enumerate(const DevCfg& cfg, cudaStream_t st);
// After an enumeration, on the device: the list lengths clamped to their capacities
// plus one (lens[0] type-I items, lens[1] streams) for the scans, the zero sentinels
// past the lists, the work counters of the sampling kernels reset, and *ok = 1 iff
// no list overflowed (read by the sampling kernels through cfg.lists_ok).
void launch_prep_lists(const DevCfg& cfg, unsigned long long* lens, unsigned int* ok,
                       cudaStream_t st);
// Type I over the pair prefix cfg.t1_pre, type II over the chunk prefix cfg.chunk_pre.
void launch_type1(const DevCfg& cfg, cudaStream_t st);
void launch_type2(const DevCfg& cfg, cudaStream_t st);
void launch_allpairs(const DevCfg& cfg, const uint32_t* X, const double* w, const float* sv,
                     cudaStream_t st);
void launch_scale(int64_t n, const double* w, double log2W_half, float gamma, float invd,
                  float* sv, cudaStream_t st);

}  // namespace gg
