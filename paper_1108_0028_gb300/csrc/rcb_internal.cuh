// Internal declarations of the GB300 RCB tree library: the tree object, exact-arithmetic
// helpers shared by the build kernels, and the launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rcb.h"

namespace rcb {

typedef __int128 i128;
typedef unsigned __int128 u128;

constexpr int kMaxL = 28;           // deepest supported lowest level (node labels < 2^29)
constexpr int kTcta = 1024;        // largest cell whose subtree one CTA builds in shared memory (two CTAs per SM)
constexpr int kCtaThreads = 256;    // threads of that CTA
constexpr int kChunk = 2048;        // particles per chunk in the level passes over large cells
constexpr int kChunkThreads = 256;
constexpr int64_t kScanTileElems = 8192;  // elements per tile of the device-wide scans (build.cu)
// int64 words of scratch a scan over n elements needs (its per-tile sums and two spare words)
constexpr int64_t scan_tmp_words(int64_t n) { return (n + kScanTileElems - 1) / kScanTileElems + 2; }

// Device status words (int32), zeroed at the start of each build.
enum StatusWord {
    ST_ERR = 0,        // bitmask of ERRBIT_*
    ST_MAXNEAR = 1,    // largest near-list length seen by the walk
    ST_MAXFAR = 2,     // largest far-list length seen by the walk
    ST_FALLBACK = 3,   // walk decisions taken in FP64 after an inconclusive FP32 filter
    ST_NBIG = 4,       // number of large cells at the next level (level passes)
    ST_NROOTS = 5,     // subtree roots queued for the shared-memory builder
    ST_NCHUNKS = 6,    // chunks of the current level pass
    ST_NSINKS = 7,     // non-empty ll-cells
    ST_NBFALLBACK = 8, // neighbour decisions taken in FP64
    ST_NBLONG = 9,     // passes of sink particles with a neighbour row longer than its buffer slice
    ST_OUTSIDE = 10,   // particles outside their ll-cell (tree integrity check)
    ST_NWORDS = 16
};
enum ErrBits { ERRBIT_ARG = 1, ERRBIT_LIMIT = 2, ERRBIT_FIXED = 4, ERRBIT_STATE = 8, ERRBIT_NBTMP = 16 };

// ------------------------------------------------------------------------------------------
// Exact helpers.

// Order-preserving map of a float64 to int64 (valid for non-NaN values with -0 removed): lets
// comparisons, minima and maxima of coordinates run on the integer pipes.
__host__ __device__ inline int64_t dkey(double x) {
#ifdef __CUDA_ARCH__
    int64_t b = __double_as_longlong(x);
#else
    int64_t b;
    __builtin_memcpy(&b, &x, 8);
#endif
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__host__ __device__ inline double dkey_inv(int64_t k) {
    int64_t b = k ^ ((k >> 63) & 0x7fffffffffffffffLL);
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double x;
    __builtin_memcpy(&x, &b, 8);
    return x;
#endif
}

// v * 2^shift rounded to the nearest integer (ties to even), for |v| * 2^shift < 2^62, using
// integer operations on the IEEE-754 fields only (the value is exact before rounding).
__device__ inline int64_t fixed_point(double v, int shift) {
    uint64_t b = (uint64_t)__double_as_longlong(v);
    int e = (int)((b >> 52) & 0x7ff);
    uint64_t mant = b & ((1ull << 52) - 1);
    if (e == 0) {
        if (mant == 0) return 0;
        e = 1;  // subnormal
    } else {
        mant |= 1ull << 52;
    }
    int s = e - 1075 + shift;  // value = mant * 2^s
    uint64_t r;
    if (s >= 0) {
        r = mant << s;  // s <= 9 because the result is below 2^62
    } else {
        int rs = -s;
        if (rs > 63) {
            r = 0;
        } else {
            uint64_t q = mant >> rs;
            uint64_t rem = mant & ((1ull << rs) - 1);
            uint64_t half = 1ull << (rs - 1);
            if (rem > half || (rem == half && (q & 1ull))) ++q;
            r = q;
        }
    }
    return (b >> 63) ? -(int64_t)r : (int64_t)r;
}

__device__ inline double pow2i(int k) {  // exact 2^k for -1022 <= k <= 1023
    return __longlong_as_double((long long)(1023 + k) << 52);
}

// Nearest float64 (ties to even) of a signed 128-bit integer with |v| < 2^127.
__device__ inline double i128_to_double(i128 v) {
    bool neg = v < 0;
    u128 u = neg ? (u128)(-v) : (u128)v;
    uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    double d;
    if (hi == 0 && lo < (1ull << 53)) {
        d = __ull2double_rn(lo);
    } else {
        int p = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);  // top bit index
        int sh = p - 52;                                                            // >= 1
        u128 q = u >> sh;
        u128 rem = u & ((((u128)1) << sh) - 1);
        u128 half = ((u128)1) << (sh - 1);
        uint64_t m = (uint64_t)q;
        if (rem > half || (rem == half && (m & 1ull))) ++m;
        d = __dmul_rn(__ull2double_rn(m), pow2i(sh));
    }
    return neg ? -d : d;
}

// Centre-of-mass coordinate from the exact sums: RN(RN(S) 2^(E-62) / (RN(M) 2^(Em-62))).
// x 2^k rounded to nearest: a product with the exact power of two where that power is a normal
// double (the product then rounds exactly as scalbn does), scalbn otherwise.
__device__ inline double scale2(double x, int k) {
    return (k >= -1022 && k <= 1023) ? __dmul_rn(x, pow2i(k)) : scalbn(x, k);
}
// M = RN(RN(S_m) 2^(Em - 62)) and COM_d = RN(RN(RN(S_d) 2^(E_d - 62)) / M).
__device__ inline double mass_from_sum(i128 M, int Em) { return scale2(i128_to_double(M), Em - 62); }
__device__ inline double com_from_sums_m(i128 S, int E, double mass) {
    return __ddiv_rn(scale2(i128_to_double(S), E - 62), mass);
}

// |a - b|^2 rounded after every operation (no contraction).
__device__ inline double dist2_rn(double ax, double ay, double az, double bx, double by, double bz) {
    double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
    double s = __dmul_rn(dx, dx);
    s = __dadd_rn(s, __dmul_rn(dy, dy));
    s = __dadd_rn(s, __dmul_rn(dz, dz));
    return s;
}

__device__ inline i128 shfl_xor_i128(i128 v, int lane_mask) {
    u128 u = (u128)v;
    unsigned w0 = (unsigned)u, w1 = (unsigned)(u >> 32), w2 = (unsigned)(u >> 64), w3 = (unsigned)(u >> 96);
    w0 = __shfl_xor_sync(0xffffffffu, w0, lane_mask);
    w1 = __shfl_xor_sync(0xffffffffu, w1, lane_mask);
    w2 = __shfl_xor_sync(0xffffffffu, w2, lane_mask);
    w3 = __shfl_xor_sync(0xffffffffu, w3, lane_mask);
    return (i128)(((u128)w3 << 96) | ((u128)w2 << 64) | ((u128)w1 << 32) | (u128)w0);
}

// Double-float (hi + lo, both float32) representation of a float64.
__device__ inline float2 to_df(double v) {
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(__dsub_rn(v, (double)hi));
    return make_float2(hi, lo);
}

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
// Exclusive prefix sum of v across the warp.
__device__ inline int warp_excl_scan(int v) {
    const int lane = threadIdx.x & 31;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    return incl - v;
}

// Runs of positive length n_k (lane k) laid end to end from first[k] (exclusive prefix sums),
// lanes with n_k = 0 after the last run: the run holding position r0 + lane.  One OR-reduction
// marks the runs that start inside [r0, r0 + 32); a popcount does the rest.
__device__ inline int warp_run_of(int first, int n, int r0) {
    const int lane = threadIdx.x & 31;
    const int st = first - r0;
    const unsigned starts = __reduce_or_sync(0xffffffffu, (n > 0 && st >= 0 && st < 32) ? (1u << st) : 0u);
    const int before = __popc(__ballot_sync(0xffffffffu, n > 0 && st < 0));
    return before + __popc(starts & ((2u << lane) - 1u)) - 1;
}

__device__ inline void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Compensated accumulation of x into (s, c).
__device__ inline void comp_add(float &s, float &c, float x) {
    float t, e;
    two_sum(s, x, t, e);
    s = t;
    c = __fadd_rn(c, e);
}

}  // namespace rcb

// ------------------------------------------------------------------------------------------
// The tree object behind the opaque rcb_tree handle.
struct rcb_tree {
    // allocator and stream of the last build
    rcb_alloc_fn alloc;
    rcb_free_fn release;
    void *ctx;
    cudaStream_t stream;

    rcb_params params;
    int64_t N;
    int L;
    int64_t nn;       // 2^(L+1) node slots
    int64_t nleaves;  // 2^L
    int64_t cap_N;    // capacities of the current allocation
    int cap_L;

    // status
    int *d_status;  // [ST_NWORDS]
    int *h_status;  // pinned mirror ([ST_NWORDS + 16])
    int *h_status_dev;  // the same pinned buffer as the device sees it (written by kernels)
    int *d_E;       // [4] fixed-point exponents E_x, E_y, E_z, E_m
    int32_t *d_nbig;  // [kMaxL + 2] large cells per level of the level passes
    unsigned long long *d_maxbits;  // [4] bit patterns of max |m x_d| and max m

    // ping-pong particle records of the build (SoA)
    double *bx[2], *by[2], *bz[2];
    int64_t *bP[2];  // [4][cap_N]: m, m x, m y, m z fixed-point integers
    int32_t *bidx[2];

    // final particles in tree order
    double *px, *py, *pz, *pm, *ph;
    int32_t *pidx;
    float4 *p32;  // (x - com_leaf, m) in float32
    float *h32;

    // nodes, indexed by heap label
    int32_t *nfirst, *ncount, *naxis;
    double *nsplit;
    int64_t *nsplitkey;
    rcb::i128 *nS;          // [nn][4] exact sums
    int64_t *nbmin, *nbmax;  // [nn][3] keys of the tight box
    double *nmass, *ncom, *nrg, *nH, *nhint, *nhnode, *nQ;  // com, rg: [nn][3]; Q: [nn][6]
    float4 *w32;  // walk packs, two per node: [2n] (rg, hint), [2n + 1] (com, H) in float32; hint = -1: empty
    float4 *mq32a, *mq32b;   // (M, Qxx, Qxy, Qxz), (Qyy, Qyz, Qzz, 0) in float32
    float2 *ncomdf;          // [nn][3] double-float centre of mass
    float4 *nfar;            // [nn][4] far-field record: (COM hi, M), (COM lo, Qxx), (Qxy, Qxz, Qyy, Qyz), (Qzz)
    int32_t *narrive;        // bottom-up arrival counters

    // level passes over large cells
    int32_t *big_list[2];
    int32_t *roots;      // packed (node << 1 | parity)
    int4 *chunks;        // (cell node, start, count, chunk index within cell)
    int32_t *cell_chunk0;  // first chunk of each large cell (parallel to big_list)
    void *chunk_part;    // per-chunk partial reductions
    int64_t cap_chunks, cap_roots;

    // sinks and lists
    int32_t nsinks;
    int32_t *sinks;       // node labels of non-empty ll-cells, in label order
    int32_t *sink_of_leaf;  // [nleaves] sink index or -1
    int32_t cap_near, cap_far;
    int32_t *near_list, *far_list;  // [nsinks][cap]
    int32_t *near_nr, *near_nn, *far_n;  // per sink: reachable, non-reachable, far counts
    int64_t cap_lists_near, cap_lists_far;  // allocated entries

    // gravity / neighbours scratch
    double *coef;    // [nsinks][20] far-field Taylor coefficients
    float *coef32;   // their float32 values (mixed form)
    int64_t *nb_count;
    // neighbour rows staged by the fused near field or the standalone pass: a compact buffer of
    // sorted rows (original indices), each particle's row start in it (by original index), the
    // buffer's fill cursor, and the queue of passes whose rows did not fit
    int32_t *nb_tmp;
    int64_t cap_tmp;
    int64_t *nb_tstart;
    unsigned long long *nb_cursor;
    int2 *nb_long;
    int nb_nlong;   // queued passes (after the last count)
    int nb_tmp_ok;  // 1 if every row that fitted its slice is in nb_tmp
    void *scan_tmp;
    int64_t cap_scan;
    int64_t nb_total;
    int nb_valid;

    // backward
    int32_t *tnear_off, *tnear_sink, *tfar_off, *tfar_sink;
    int bwd_valid;
    // capacities of the backward scratch (kept across builds, grown when a build needs more):
    // entries of tnear_off, tfar_off, tnear_sink and tfar_sink, bytes of adj
    int64_t cap_bwd_off, cap_bwd_cur, cap_bwd_sink, cap_bwd_N, cap_bwd_adj;
    double *ones;     // unit weights for the centre-of-number split (cap_N)
    // median position split: per large cell of a level, a 256-bin digit histogram, the key prefix
    // chosen so far and the rank still sought (cap_N / (kTcta + 1) + 2 cells)
    int32_t *mps_hist;
    unsigned long long *mps_prefix;
    int32_t *mps_rank;
    // neighbour candidates of a MAC-only tree: reachable leaves per sink (front of the rows)
    int32_t *cand_list, *cand_far, *cand_n;  // cand_n: [3][nleaves] counts (front, back, far)
    int cap_cand;
    int64_t cap_lists_cand;
    float4 *dens_hl;  // density scratch: per particle (hi, m) and (lo, 1/h) in float32, original order
    int walk_pair;  // walk two sinks per thread (set when the last walk's longest far list exceeded 1024)
    double *adj;  // per-node adjoints

    int64_t stats_fallback;
    int64_t nroots_last;
    int64_t launches;        // kernel launches issued by the library for this tree
    int64_t near_pairs, cand_pairs;
    int64_t *d_pairs;        // [2] device counters of the two pair totals
    cudaEvent_t ev[2 * 16];  // start/stop per stage (RCB_FLAG_TIMING)
    bool ev_ready;
    bool ev_used[16];
};

namespace rcb {

// memory helpers (rcb_api.cu)
void *dev_alloc(rcb_tree *t, size_t bytes);
void dev_free(rcb_tree *t, void *p);

// build.cu
int64_t scan_tmp_bytes(int64_t n);
int scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total, void *tmp, cudaStream_t st);
int scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, void *tmp, cudaStream_t st);
int build_tree(rcb_tree *t, const double *x, const double *m, const double *h);
int refit_tree(rcb_tree *t, const double *x, const double *m);
// walk.cu
int walk_tree(rcb_tree *t);
int integrity_outside(rcb_tree *t, const double *x, int64_t *outside);  // build.cu
int gather_h(rcb_tree *t, const double *h);                             // build.cu
// nwords 32-bit words from src to dst by a kernel on st (no copy engine: small readbacks into the
// pinned status buffer and device copies do not queue behind the caller's large transfers)
int copy_words(void *dst, const void *src, int64_t nwords, cudaStream_t st);  // rcb_api.cu
int density(rcb_tree *t, const int64_t *offsets, const int32_t *idx, double *rho);  // density.cu
// neighbours.cu
int neighbour_counts(rcb_tree *t, int64_t *counts, int *status);  // count pass into caller memory
int neighbours(rcb_tree *t, int64_t *offsets, int32_t *idx, int64_t capacity, int64_t *needed);
int count_neighbours(rcb_tree *t);        // counts, offsets (nb_count) and staged rows unless valid
struct RowOut;
RowOut row_out(rcb_tree *t);              // where staged neighbour rows go (nb_rows.cuh)
int ensure_nb_tmp(rcb_tree *t);           // staging buffer of neighbour rows (grown from the last total)
int reset_nb_rows(rcb_tree *t);           // before a pass that stages rows: cursor, queue and flags
int scan_neighbour_counts(rcb_tree *t);   // nb_count: counts by original index -> offsets
int fetch_neighbour_total(rcb_tree *t);   // total and long-row count to the host; counts valid
// gravity.cu
int gravity(rcb_tree *t, double *acc, double *pot);
int gravity_neighbours(rcb_tree *t, double *acc, double *pot);  // mixed near field + neighbour counts/rows
// backward.cu
int gravity_backward(rcb_tree *t, const double *gacc, const double *gpot, double *gx, double *gm);

// Stage timing (RCB_FLAG_TIMING): events recorded on the tree's stream.
enum Stage {
    SG_INGEST = 0, SG_LEVELS = 1, SG_SUBTREE = 2, SG_LEAVES = 3, SG_WALK = 4, SG_BUILD = 5,
    SG_NB_COUNT = 6, SG_NB_FILL = 7, SG_NB_SORT = 8, SG_FAR = 9, SG_NEAR = 10, SG_BWD = 11
};
void stage_begin(rcb_tree *t, int stage);
void note_launch();  // counts kernel launches of the library (process-wide)
long long launch_count();
void stage_end(rcb_tree *t, int stage);

#define RCB_CUDA_TRY(expr)                          \
    do {                                            \
        cudaError_t _e = (expr);                    \
        if (_e != cudaSuccess) return RCB_ERR_CUDA; \
    } while (0)

}  // namespace rcb
