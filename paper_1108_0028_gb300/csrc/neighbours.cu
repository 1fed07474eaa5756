// Neighbour search (Sec. 2.3): the candidate (reachable) ll-cells of each sink are culled to
// the particles b != a with |r_a - r_b| < 2 h_a, and stored in one flat list with per-particle
// offsets (Sec. 2.3.2), rows in original order and sorted by original index.
//
// pass   one warp per sink stages its candidate particles in shared memory as float32 offsets
//        from the sink's centre of mass (the double-float cell-centre difference plus each
//        particle's float32 offset from its own cell's centre of mass), keeping only those within
//        2 H_A (1 + 2^-10) of the box of the sink's particles (H_A their largest h_a), since a
//        source farther out has r_ab > 2 h_a for every sink particle.
//        Lanes take (sink particle i, source stream j) pairs as the near field does: with P sink
//        particles, S = 32 / P streams, lane l holds particle l mod P and tests the source pairs
//        j, j + S, ... (j = l / P), two at a time with paired float32 instructions.  Three forms:
//          COUNT  counts only (by original index);
//          STAGE  counts, and rows gathered in shared memory (nb_rows.cuh), sorted and handed to a
//                 compact staging buffer -- the same rows the fused near-field kernel stages;
//          FILL   rows straight into the CSR once the offsets are known (the fallback for rows
//                 that did not fit the staging, and for a full staging buffer).
// scan   exclusive int64 scan over original indices gives the CSR offsets.
// copy   every staged row is copied to its offset in the caller's CSR.
// The float32 test decides by the sign of d^2 - (2h)^2 unless |d^2 - (2h)^2| <= B, B = 2^-19 F,
// F = (W + |d_a|_1)^2 + (2h)^2 with W the tile's largest |dCOM|_1 + |d_b|_1 + 2^-20 (|COM_A|_1 +
// |COM_B|_1): the three input roundings, the two float additions of the offsets, the double-float
// centre difference, the squares and sums, the subtraction and the rounding of (2h)^2 stay below
// 16 u F (u = 2^-24), so B covers them twice; the additive 1e-30 covers flushed subnormals.
// Inside the band the test is repeated in float64 on the original positions, rounded after every
// operation, which is the definition; the lists are therefore exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <climits>

#include "nb_rows.cuh"
#include "rcb_internal.cuh"

namespace rcb {
namespace {

constexpr int kNbWarps = 8;
constexpr int kNbTile = 256;  // staged source slots per warp (even)
constexpr unsigned kFull = 0xffffffffu;
enum NbMode { NB_COUNT = 0, NB_STAGE = 1, NB_FILL = 2 };

struct NbCtx {
    int nsinks;
    const int32_t *sinks, *near_list, *near_nr;
    int cap_near;
    const int32_t *nfirst, *ncount;
    const float2 *ncomdf;
    const double *px, *py, *pz, *ph;
    const int32_t *pidx;
    const float4 *p32;
    const float *h32;
    int64_t *counts;         // [N] by original index (COUNT, STAGE)
    const int64_t *offsets;  // [N+1] (FILL)
    int32_t *idx;            // (FILL)
    const int2 *items;       // FILL: (sink, first particle of the pass) to fill, or NULL for all
    int nitems;
    RowOut ro;               // STAGE
    int *status;
};

// Shared memory of one warp.  Per source pair k: A[k] = (-x_2k, -x_2k+1, -y_2k, -y_2k+1), B[k] =
// (-z_2k, -z_2k+1, sorted indices), C[k] = (original indices, unused).
template <int MODE>
struct NbSmem {
    static constexpr bool kRows = MODE != NB_COUNT;
    static constexpr int H = kNbTile / 2;
    static constexpr size_t bytes =
        (size_t)H * (kRows ? 3 : 2) * sizeof(float4) + (kRows ? kRowBuf * sizeof(int32_t) : 0) + 64 * sizeof(int);
    float4 *P;      // A[H], B[H], C[H] (STAGE, FILL)
    int32_t *rows;  // row buffer (STAGE, FILL)
    int *rowcnt;    // [32] entries of each row of the pass so far
    int *self;      // [32] slot of sink particle i of the pass in this tile, -1 if not staged
    __device__ NbSmem(unsigned char *p) {
        P = reinterpret_cast<float4 *>(p);
        rows = reinterpret_cast<int32_t *>(P + (kRows ? 3 : 2) * H);
        rowcnt = rows + (kRows ? kRowBuf : 0);
        self = rowcnt + 32;
    }
    __device__ __forceinline__ float4 a(int k) const { return P[k]; }
    __device__ __forceinline__ float4 b(int k) const { return P[k + H]; }
    __device__ __forceinline__ const int4 *D() const { return reinterpret_cast<const int4 *>(P + 2 * H); }
    __device__ __forceinline__ void put(int s, float dx, float dy, float dz, int sidx, int oidx) const {
        float *q = reinterpret_cast<float *>(P + (s >> 1));
        const int u = s & 1;
        q[u] = -dx;
        q[2 + u] = -dy;
        q[4 * H + u] = -dz;
        q[4 * H + 2 + u] = __int_as_float(sidx);
        if (kRows) reinterpret_cast<int *>(q)[8 * H + u] = oidx;
    }
};

// Where the next tile starts: candidate entry k0, of whose particles the first off0 are staged.
struct NbCursor {
    int k0, off0;
};

// Stage the next tile: one batch of up to 32 candidate cells, as many whole cells as fit in
// kNbTile - 2 slots (part of one cell if a single cell is larger).  Lanes describe the cells,
// every lane issues the gathers of all its slots before using any of them (two rounds of memory
// latency per tile), then sources farther than 2 H_A (1 + 2^-10) from the box of the sink's
// particles are dropped (r_ab > 2 h_a for every sink particle a) and the others stored.  Returns the number stored (padded to even with a far-away source); wmax gets the
// tile's largest w.
template <int MODE>
__device__ int stage_nb(const NbCtx &c, int s, int A, int fA, int a0, int P, int nr, NbCursor &cur,
                        const NbSmem<MODE> &sm, float3 blo, float3 bhi, float Xcut, float &wmax, bool &last) {
    constexpr int kCap = kNbTile - 2;
    constexpr int kU = (kCap + 31) / 32;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)s * c.cap_near;
    const float X2cut = Xcut * Xcut;
    sm.self[lane] = -1;
    wmax = 0.f;
    if (cur.k0 >= nr) {
        last = true;
        __syncwarp();
        return 0;
    }
    const int k0 = cur.k0;
    const int k = k0 + lane;
    int f = 0, n = 0;
    float ox = 0.f, oy = 0.f, oz = 0.f, ow = 0.f;
    if (k < nr) {
        const int B = c.near_list[base + k];
        const float2 a0f = c.ncomdf[3 * (int64_t)A], a1f = c.ncomdf[3 * (int64_t)A + 1],
                     a2f = c.ncomdf[3 * (int64_t)A + 2];
        f = c.nfirst[B];
        n = c.ncount[B];
        const float2 b0 = c.ncomdf[3 * (int64_t)B], b1 = c.ncomdf[3 * (int64_t)B + 1], b2 = c.ncomdf[3 * (int64_t)B + 2];
        ox = (b0.x - a0f.x) + (b0.y - a0f.y);
        oy = (b1.x - a1f.x) + (b1.y - a1f.y);
        oz = (b2.x - a2f.x) + (b2.y - a2f.y);
        ow = 0x1p-20f * ((fabsf(a0f.x) + fabsf(a1f.x) + fabsf(a2f.x)) + (fabsf(b0.x) + fabsf(b1.x) + fabsf(b2.x)));
        if (lane == 0) {  // the part of the first cell not staged yet
            f += cur.off0;
            n -= cur.off0;
        }
    }
    int excl = warp_excl_scan(n);
    const unsigned fit = __ballot_sync(kFull, k < nr && excl + n <= kCap);
    const int nfit = __popc(fit);
    int nslots;
    if (nfit > 0) {
        nslots = __shfl_sync(kFull, excl + n, nfit - 1);
        if (lane >= nfit) n = 0;
        cur.k0 = k0 + nfit;
        cur.off0 = 0;
    } else {
        nslots = kCap;
        if (lane > 0) n = 0;
        if (lane == 0) n = kCap;
        cur.off0 += kCap;
    }
    last = cur.k0 >= nr;
    excl = warp_excl_scan(n);
    int b[kU], cl[kU], ob[kU];
    float4 pb[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        const int r = 32 * u + lane;
        cl[u] = warp_run_of(excl, n, 32 * u);
        b[u] = __shfl_sync(kFull, f, cl[u]) + r - __shfl_sync(kFull, excl, cl[u]);
        pb[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        ob[u] = 0;
        if (r < nslots) {
            pb[u] = c.p32[b[u]];
            if (MODE != NB_COUNT) ob[u] = c.pidx[b[u]];
        }
    }
    __syncwarp();
    float wl = 0.f;
    int n_st = 0;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        const bool act = 32 * u + lane < nslots;
        const float cx = __shfl_sync(kFull, ox, cl[u]), cy = __shfl_sync(kFull, oy, cl[u]),
                    cz = __shfl_sync(kFull, oz, cl[u]), cw = __shfl_sync(kFull, ow, cl[u]);
        const float vx = cx + pb[u].x, vy = cy + pb[u].y, vz = cz + pb[u].z;
        // squared distance from the source to the sink particles' box
        const float gx = fmaxf(fmaxf(blo.x - vx, vx - bhi.x), 0.f), gy = fmaxf(fmaxf(blo.y - vy, vy - bhi.y), 0.f),
                    gz = fmaxf(fmaxf(blo.z - vz, vz - bhi.z), 0.f);
        const bool keep = act && !(fmaf(gz, gz, fmaf(gy, gy, gx * gx)) > X2cut);
        const unsigned mk = __ballot_sync(kFull, keep);
        if (keep) {
            const int at = n_st + __popc(mk & lt);
            sm.put(at, vx, vy, vz, b[u], ob[u]);
            wl = fmaxf(wl, (fabsf(cx) + fabsf(cy) + fabsf(cz)) + fabsf(pb[u].x) + fabsf(pb[u].y) + fabsf(pb[u].z) + cw);
            const int i = b[u] - fA - a0;  // a sink particle of this pass?
            if (i >= 0 && i < P) sm.self[i] = at;
        }
        n_st += __popc(mk);
    }
    if (n_st & 1) {
        if (lane == 0) sm.put(n_st, 1e18f, 1e18f, 1e18f, -1, -1);
        ++n_st;
    }
    for (int o = 16; o >= 1; o >>= 1) wl = fmaxf(wl, __shfl_xor_sync(kFull, wl, o));
    wmax = wl;
    __syncwarp();
    return n_st;
}

// The float64 definition for a pair inside the float32 band.
__device__ __noinline__ bool nb_exact(const double *px, const double *py, const double *pz, const double *ph, int a,
                                      int b) {
    if (b == a || b < 0) return false;
    const double s2 = __dmul_rn(2.0, ph[a]);
    return dist2_rn(px[a], py[a], pz[a], px[b], py[b], pz[b]) < __dmul_rn(s2, s2);
}

// One pass of P sink particles (from a0) of sink s against all its candidate tiles.  Each lane
// decides its pairs by the sign of d^2 - (2h)^2, exact outside the band |d^2 - (2h)^2| <= B; a
// block of loop steps in which some pair fell inside the band is gone through again with the
// float64 test deciding those pairs.  The pair of a particle with itself is skipped by its slot.
template <int MODE>
__device__ void nb_pass(const NbCtx &c, const NbSmem<MODE> &sm, int s, int a0, int &nfb) {
    const int lane = threadIdx.x & 31;
    const int A = c.sinks[s];
    const int fA = c.nfirst[A], nA = c.ncount[A];
    const int nr = c.near_nr[s];
    // the box of the sink cell's particles (float32 offsets from its centre of mass) and H_A
    float3 blo = make_float3(3e38f, 3e38f, 3e38f), bhi = make_float3(-3e38f, -3e38f, -3e38f);
    float HA = 0.f;
    for (int i = lane; i < nA; i += 32) {
        const float4 pa = c.p32[fA + i];
        blo = make_float3(fminf(blo.x, pa.x), fminf(blo.y, pa.y), fminf(blo.z, pa.z));
        bhi = make_float3(fmaxf(bhi.x, pa.x), fmaxf(bhi.y, pa.y), fmaxf(bhi.z, pa.z));
        HA = fmaxf(HA, c.h32[fA + i]);
    }
    for (int o = 16; o >= 1; o >>= 1) {
        blo.x = fminf(blo.x, __shfl_xor_sync(kFull, blo.x, o));
        blo.y = fminf(blo.y, __shfl_xor_sync(kFull, blo.y, o));
        blo.z = fminf(blo.z, __shfl_xor_sync(kFull, blo.z, o));
        bhi.x = fmaxf(bhi.x, __shfl_xor_sync(kFull, bhi.x, o));
        bhi.y = fmaxf(bhi.y, __shfl_xor_sync(kFull, bhi.y, o));
        bhi.z = fmaxf(bhi.z, __shfl_xor_sync(kFull, bhi.z, o));
        HA = fmaxf(HA, __shfl_xor_sync(kFull, HA, o));
    }
    const float Xcut = 2.0f * HA * (1.0f + 0x1p-10f);
    const int P = min(nb_pass_len(nA), nA - a0), S = 32 / P;
    const int i = lane % P, j = lane / P;
    const bool active = j < S;
    const int a = fA + a0 + i;
    const float4 pa = c.p32[a];
    const float h2f = 2.0f * c.h32[a];  // = float32(2 h) exactly
    const float h2 = h2f * h2f;
    const float2 xa = make_float2(pa.x, pa.x), ya = make_float2(pa.y, pa.y), za = make_float2(pa.z, pa.z);
    const float2 nh2 = make_float2(-h2, -h2);
    const float aabs1 = fabsf(pa.x) + fabsf(pa.y) + fabsf(pa.z);
    const int o_self = c.pidx[a];
    // rows: STAGE slices of rc entries; FILL rows of known length, in the buffer while they fit,
    // else straight into the CSR
    int rc = 0, exl = 0, lenl = -1;
    int32_t *rowp = sm.rows;
    int64_t goff = 0;
    bool inplace = false;
    if (MODE == NB_STAGE) {
        rc = kRowBuf / P;
        rowp = sm.rows + i * rc;
    } else if (MODE == NB_FILL) {
        goff = c.offsets[o_self];
        rc = (int)(c.offsets[o_self + 1] - goff);
        lenl = lane < P ? rc : 0;  // lane l < P holds row l
        exl = warp_excl_scan(lenl);
        inplace = __shfl_sync(kFull, exl + lenl, 31) > kRowBuf;
        rowp = inplace ? c.idx + goff : sm.rows + __shfl_sync(kFull, exl, i);
        if (lane >= P) lenl = -1;
    }
    if (lane < P) sm.rowcnt[lane] = 0;
    __syncwarp();
    NbCursor cur{0, 0};
    bool last = false;
    while (!last) {
        float wmax;
        const int ns = stage_nb<MODE>(c, s, A, fA, a0, P, nr, cur, sm, blo, bhi, Xcut, wmax, last);
        const float F = wmax + aabs1;
        const float B = fmaf(F, F, h2) * 0x1p-19f + 1e-30f;
        const int self = sm.self[i];
        const int np = ns >> 1;
        const int nsteps = (np + S - 1) / S;  // loop steps of the warp (stream 0 the longest)
        for (int t0 = 0; t0 < nsteps; t0 += 16) {
            const int kb = j + t0 * S;
            unsigned mask = 0;
            float bandmin = 3e38f;
            if (active) {
                int k = kb;
                for (int t = 0; t < 16 && k < np; ++t, k += S) {
                    const float4 a4 = sm.a(k), b4 = sm.b(k);
                    const float2 dx = __fadd2_rn(xa, make_float2(a4.x, a4.y));
                    const float2 dy = __fadd2_rn(ya, make_float2(a4.z, a4.w));
                    const float2 dz = __fadd2_rn(za, make_float2(b4.x, b4.y));
                    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                    const float2 e = __fadd2_rn(r2, nh2);  // d^2 - (2h)^2
                    const float ex = fabsf(e.x), ey = fabsf(e.y);
                    bandmin = fminf(bandmin, fminf(ex, ey));
                    // STAGE keeps the particle itself in its row (the copy into the CSR drops it)
                    mask |= (unsigned)(e.x < 0.f && ex > B && (MODE == NB_STAGE || 2 * k != self)) << (2 * t);
                    mask |= (unsigned)(e.y < 0.f && ey > B && (MODE == NB_STAGE || 2 * k + 1 != self)) << (2 * t + 1);
                }
            }
            // rare: a pair of these steps inside the band, the float64 test decides it
            if (__any_sync(kFull, bandmin <= B) && active) {
                int k = kb;
                for (int t = 0; t < 16 && k < np; ++t, k += S) {
                    const float4 a4 = sm.a(k), b4 = sm.b(k);
                    const float2 dx = __fadd2_rn(xa, make_float2(a4.x, a4.y));
                    const float2 dy = __fadd2_rn(ya, make_float2(a4.z, a4.w));
                    const float2 dz = __fadd2_rn(za, make_float2(b4.x, b4.y));
                    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                    const float2 e = __fadd2_rn(r2, nh2);
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (fabsf(u ? e.y : e.x) <= B) {
                            const int bb = __float_as_int(u ? b4.w : b4.z);
                            if ((MODE == NB_STAGE && bb == a) || nb_exact(c.px, c.py, c.pz, c.ph, a, bb))
                                mask |= 1u << (2 * t + u);
                            ++nfb;
                        }
                    }
                }
            }
            if (mask) {
                if constexpr (MODE == NB_COUNT) atomicAdd(sm.rowcnt + i, __popc(mask));
                else row_append(rowp, rc, sm.rowcnt + i, mask, kb, S, sm.D());
            }
        }
        __syncwarp();
    }
    const int run = lane < P ? sm.rowcnt[lane] : 0;  // lane l < P: the length of row l
    if constexpr (MODE == NB_COUNT) {
        if (lane < P) c.counts[c.pidx[fA + a0 + lane]] = run;
    } else if constexpr (MODE == NB_STAGE) {
        if (lane < P) c.counts[c.pidx[fA + a0 + lane]] = run - 1;  // the row holds the particle itself
        rows_finish(c.ro, sm.rows, rc, P, run, lane < P ? c.pidx[fA + a0 + lane] : 0, s, a0);
    } else {
        if (lane < P && run != rc) atomicOr(&c.status[ST_ERR], ERRBIT_STATE);
        __syncwarp();
        if (inplace) {
            for (int q = 0; q < P; ++q) {
                const int64_t o = __shfl_sync(kFull, goff, q);
                const int n = __shfl_sync(kFull, rc, q);
                warp_sort_inplace(c.idx + o, n);
            }
        } else {
            rows_sort_store(sm.rows, exl, lenl, goff, INT32_MAX, c.idx, P);  // these rows hold no self entry
        }
    }
    __syncwarp();
}

template <int MODE>
__global__ void __launch_bounds__(kNbWarps * 32, 2) k_nb(NbCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const NbSmem<MODE> sm(smem_raw + (size_t)w * NbSmem<MODE>::bytes);
    int nfb = 0;
    if (MODE == NB_FILL && c.items) {
        for (int q = blockIdx.x * kNbWarps + w; q < c.nitems; q += gridDim.x * kNbWarps) {
            const int2 it = c.items[q];
            nb_pass<MODE>(c, sm, it.x, it.y, nfb);
        }
    } else {
        for (int s = blockIdx.x * kNbWarps + w; s < c.nsinks; s += gridDim.x * kNbWarps) {
            const int nA = c.ncount[c.sinks[s]];
            for (int a0 = 0; a0 < nA; a0 += nb_pass_len(nA)) nb_pass<MODE>(c, sm, s, a0, nfb);
        }
    }
    for (int o = 16; o >= 1; o >>= 1) nfb += __shfl_xor_sync(kFull, nfb, o);
    if (lane == 0 && nfb && MODE != NB_FILL) atomicAdd(&c.status[ST_NBFALLBACK], nfb);
}

// Copy the staged rows to the CSR, sorting each by original index and leaving out the particle
// itself.  A warp takes 32 consecutive particles (original order) and their rows four at a time,
// one per group of 8 lanes, with the sorting networks of nb_rows.cuh (rows longer than 64 entries
// over the whole warp; beyond 128 in place in the staging buffer).  Rows that were not staged
// (tstart < 0) are left to the direct fill.
__global__ void __launch_bounds__(256, 4) k_nb_copy(const int64_t *tstart, const int64_t *offsets, int32_t *tmp,
                                                 int32_t *idx, int64_t N) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < N; base += nw * 32) {
        int64_t src = -1, dst = 0;
        int len = -1;
        if (base + lane < N) {
            src = tstart[base + lane];
            dst = offsets[base + lane];
            len = src >= 0 ? (int)(offsets[base + lane + 1] - dst) + 1 : -1;  // the staged row holds the particle
        }
        const int cnt = (int)(N - base < 32 ? N - base : 32);
        rows_sort_store(tmp, src, len, dst, (int32_t)(base + lane), idx, cnt);
    }
}

int sm_count_nb() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

NbCtx make_nbctx(rcb_tree *t) {
    NbCtx c;
    std::memset(&c, 0, sizeof(c));
    c.nsinks = t->nsinks;
    c.sinks = t->sinks;
    // candidates: the reachable leaves at the front of the near rows, or the candidate rows of a
    // MAC-only tree
    const bool mac_only = (t->params.flags & RCB_FLAG_MAC_ONLY) != 0;
    c.near_list = mac_only ? t->cand_list : t->near_list;
    c.near_nr = mac_only ? t->cand_n : t->near_nr;
    c.cap_near = mac_only ? t->cap_cand : t->cap_near;
    c.nfirst = t->nfirst;
    c.ncount = t->ncount;
    c.ncomdf = t->ncomdf;
    c.px = t->px;
    c.py = t->py;
    c.pz = t->pz;
    c.ph = t->ph;
    c.pidx = t->pidx;
    c.p32 = t->p32;
    c.h32 = t->h32;
    c.counts = t->nb_count;
    c.ro = row_out(t);
    c.status = t->d_status;
    return c;
}

template <int MODE>
int launch_nb(rcb_tree *t, const NbCtx &c, int nwork) {
    if (nwork == 0) return RCB_OK;
    const int nsm = sm_count_nb();
    const size_t smem = (size_t)kNbWarps * NbSmem<MODE>::bytes;
    RCB_CUDA_TRY(cudaFuncSetAttribute(k_nb<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int blocks = std::max(1, std::min((nwork + kNbWarps - 1) / kNbWarps, nsm * 16));
    k_nb<MODE><<<blocks, kNbWarps * 32, smem, t->stream>>>(c); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

}  // namespace

RowOut row_out(rcb_tree *t) {
    RowOut r;
    r.tmp = t->nb_tmp;
    r.cap_tmp = t->cap_tmp;
    r.cursor = t->nb_cursor;
    r.tstart = t->nb_tstart;
    r.long_q = t->nb_long;
    r.cap_long = (int)std::min<int64_t>(t->N, INT32_MAX);
    r.status = t->d_status;
    return r;
}

int ensure_nb_tmp(rcb_tree *t) {
    // entries for the last total and a margin, at least 64 per particle
    const int64_t want = std::max<int64_t>(64 * t->N, t->nb_total + t->nb_total / 8 + 1024);
    if (t->cap_tmp >= want && t->nb_tmp) return RCB_OK;
    dev_free(t, t->nb_tmp);
    t->nb_tmp = (int32_t *)dev_alloc(t, (size_t)want * sizeof(int32_t));
    if (!t->nb_tmp) {
        t->cap_tmp = 0;
        return RCB_ERR_ALLOC;
    }
    t->cap_tmp = want;
    return RCB_OK;
}

int reset_nb_rows(rcb_tree *t) {
    int rc = ensure_nb_tmp(t);
    if (rc) return rc;
    RCB_CUDA_TRY(cudaMemsetAsync(t->nb_cursor, 0, sizeof(unsigned long long), t->stream));
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_status + ST_NBFALLBACK, 0, 2 * sizeof(int), t->stream));
    return RCB_OK;
}

int neighbour_counts(rcb_tree *t, int64_t *counts, int *status) {
    NbCtx c = make_nbctx(t);
    c.counts = counts;
    c.status = status;
    return launch_nb<NB_COUNT>(t, c, t->nsinks);
}

int scan_neighbour_counts(rcb_tree *t) {
    return scan_i64(t->nb_count, t->nb_count, t->N, t->nb_count + t->N, t->scan_tmp, t->stream);
}

int fetch_neighbour_total(rcb_tree *t) {
    cudaStream_t st = t->stream;
    // the total (int64, 8-byte aligned slot of the pinned buffer), the error word and two status
    // words
    int rc = copy_words(t->h_status_dev + ST_NWORDS + 2, t->nb_count + t->N, 2, st);
    if (!rc) rc = copy_words(t->h_status_dev + ST_NBFALLBACK, t->d_status + ST_NBFALLBACK, 2, st);
    if (!rc) rc = copy_words(t->h_status_dev + ST_ERR, t->d_status + ST_ERR, 1, st);
    if (rc) return rc;
    RCB_CUDA_TRY(cudaStreamSynchronize(st));
    std::memcpy(&t->nb_total, t->h_status + ST_NWORDS + 2, sizeof(int64_t));
    t->nb_nlong = std::min<int>(t->h_status[ST_NBLONG], (int)std::min<int64_t>(t->N, INT32_MAX));
    t->nb_tmp_ok = (t->h_status[ST_ERR] & ERRBIT_NBTMP) ? 0 : 1;
    if (!t->nb_tmp_ok) {  // clear the bit; the next staging pass gets a larger buffer
        int zero = t->h_status[ST_ERR] & ~ERRBIT_NBTMP;
        RCB_CUDA_TRY(cudaMemcpyAsync(t->d_status + ST_ERR, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
        RCB_CUDA_TRY(cudaStreamSynchronize(st));
    }
    t->nb_valid = 1;
    return RCB_OK;
}

int count_neighbours(rcb_tree *t) {
    if (t->nb_valid) return RCB_OK;
    NbCtx c = make_nbctx(t);
    stage_begin(t, SG_NB_COUNT);
    int rc = reset_nb_rows(t);
    if (rc) return rc;
    c.ro = row_out(t);
    rc = launch_nb<NB_STAGE>(t, c, t->nsinks);
    if (rc) return rc;
    rc = scan_neighbour_counts(t);
    if (rc) return rc;
    stage_end(t, SG_NB_COUNT);
    return fetch_neighbour_total(t);
}

int neighbours(rcb_tree *t, int64_t *offsets, int32_t *idx, int64_t capacity, int64_t *needed) {
    cudaStream_t st = t->stream;
    int rc = count_neighbours(t);
    if (rc) return rc;
    rc = copy_words(offsets, t->nb_count, 2 * (t->N + 1), st);
    if (rc) return rc;
    *needed = t->nb_total;
    if (!idx) {
        RCB_CUDA_TRY(cudaStreamSynchronize(st));
        return RCB_OK;
    }
    if (capacity < t->nb_total) {
        RCB_CUDA_TRY(cudaStreamSynchronize(st));
        return RCB_ERR_CAPACITY;
    }
    NbCtx c = make_nbctx(t);
    c.offsets = t->nb_count;
    c.idx = idx;
    stage_begin(t, SG_NB_FILL);
    if (t->nb_tmp_ok) {
        const int nsm = sm_count_nb();
        k_nb_copy<<<std::max(1, nsm * 16), 256, 0, st>>>(t->nb_tstart, t->nb_count, t->nb_tmp, idx, t->N); note_launch();
        RCB_CUDA_TRY(cudaGetLastError());
        if (t->nb_nlong > 0) {  // passes with a row longer than its slice: filled directly
            c.items = t->nb_long;
            c.nitems = t->nb_nlong;
            rc = launch_nb<NB_FILL>(t, c, t->nb_nlong);
            if (rc) return rc;
        }
    } else {  // the staging buffer was full: every row filled directly (it grows for next time)
        rc = launch_nb<NB_FILL>(t, c, t->nsinks);
        if (rc) return rc;
    }
    stage_end(t, SG_NB_FILL);
    // the direct fill re-derives its rows; a row whose length differs from its count is an error
    rc = copy_words(t->h_status_dev, t->d_status, 1, st);
    if (rc) return rc;
    RCB_CUDA_TRY(cudaStreamSynchronize(st));
    if (t->h_status[ST_ERR] & ERRBIT_STATE) return RCB_ERR_STATE;
    return RCB_OK;
}

}  // namespace rcb
