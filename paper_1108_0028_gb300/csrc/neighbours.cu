// Neighbour search (Sec. 2.3): the candidate (reachable) ll-cells of each sink are culled to
// the particles b != a with |r_a - r_b| < 2 h_a, and stored in one flat list with per-particle
// offsets (Sec. 2.3.2), rows in original order and sorted by original index.
//
// count  one warp per sink stages its candidate particles in shared memory as float32 offsets
//        from the sink's centre of mass (the double-float cell-centre difference plus each
//        particle's float32 offset from its own cell's centre of mass), keeping only those within
//        (R_A + 2 H_A)(1 + 2^-10) of it: R_A is the largest |d_a| and H_A the largest h_a of the
//        sink's particles, so a source farther out has r_ab > 2 h_a for every sink particle.
//        Lanes take (sink particle i, source stream j) pairs as the near field does: with P sink
//        particles, S = 32 / P streams, lane l holds particle l mod P and tests the source pairs
//        j, j + S, ... (j = l / P), two at a time with paired float32 instructions.  A particle's
//        count goes to its original index.
// scan   exclusive int64 scan over original indices gives the CSR offsets.
// fill   the same pass once the offsets are known: each neighbour's original index is appended
//        to its row in shared memory (a shared-memory counter per row); once the sink is done the
//        rows are sorted in registers (a bitonic network of shuffles) and written at their
//        offsets.  Rows that do not fit the warp's row buffer are appended in place and sorted
//        there by the warp.
// The float32 test compares d^2 with (2h)^2 -+ B, B = 2^-19 F, F = (W + |d_a|_1)^2 + (2h)^2 with W
// the tile's largest |dCOM|_1 + |d_b|_1 + 2^-20 (|COM_A|_1 + |COM_B|_1): the three input
// roundings, the two float additions of the offsets, the double-float centre difference, the
// squares and sums, and the roundings of (2h)^2 and of (2h)^2 -+ B stay below 16 u F (u = 2^-24),
// so B covers them twice; the additive 1e-30 covers flushed subnormals.  Inside the band the
// test is repeated in float64 on the original positions, rounded after every operation, which is
// the definition; the lists are therefore exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <climits>

#include "rcb_internal.cuh"

namespace rcb {
namespace {

constexpr int kNbWarps = 8;
constexpr int kNbTile = 256;   // staged source slots per warp (even)
constexpr int kRowBuf = 1024;  // entries of the warp's shared-memory row buffer
constexpr unsigned kFull = 0xffffffffu;

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
    int64_t *counts;         // [N] by original index (count pass)
    const int64_t *offsets;  // [N+1] (fill pass)
    int32_t *idx;            // (fill pass)
    int *status;
};

// Shared memory of one warp.  Per source pair k: A[k] = (-x_2k, -x_2k+1, -y_2k, -y_2k+1), B[k] =
// (-z_2k, -z_2k+1, sorted indices), C[k] = (original indices, unused) for FILL.
template <bool FILL>
struct NbSmem {
    static constexpr size_t bytes =
        (size_t)(kNbTile / 2) * (FILL ? 3 : 2) * sizeof(float4) +
        (FILL ? 32 * sizeof(int64_t) + kRowBuf * sizeof(int32_t) + 96 * sizeof(int) : 0) + 32 * sizeof(int);
    float4 *A, *B;
    int4 *C;
    int64_t *goff;   // FILL: [32] offset of each row of the pass in the output
    int32_t *rows;   // FILL: row buffer
    int *rowpos;     // FILL: [32..64) row start in the buffer (-1: in place); [64..96) row length
    int *self;       // [32] slot of sink particle i of the pass in this tile, -1 if not staged
    __device__ NbSmem(unsigned char *p) {
        A = reinterpret_cast<float4 *>(p);
        B = A + kNbTile / 2;
        C = reinterpret_cast<int4 *>(B + kNbTile / 2);
        goff = reinterpret_cast<int64_t *>(C + (FILL ? kNbTile / 2 : 0));
        rows = reinterpret_cast<int32_t *>(goff + (FILL ? 32 : 0));
        rowpos = rows + (FILL ? kRowBuf : 0);
        self = rowpos + (FILL ? 96 : 0);
    }
    __device__ __forceinline__ void put(int s, float dx, float dy, float dz, int sidx, int oidx) const {
        float *a = reinterpret_cast<float *>(A + (s >> 1)), *b = reinterpret_cast<float *>(B + (s >> 1));
        const int u = s & 1;
        a[u] = -dx;
        a[2 + u] = -dy;
        b[u] = -dz;
        b[2 + u] = __int_as_float(sidx);
        if (FILL) reinterpret_cast<int *>(C + (s >> 1))[u] = oidx;
    }
};

struct NbCursor {
    int k0;
    int64_t pos, t0;
};

// Stage the next tile: candidate cells in list order, 32 at a time (lanes describe the cells,
// then take two slots each per round), sources beyond (R_A + 2 H_A)(1 + 2^-10) dropped.  Returns
// the number staged (padded to even with a far-away source); wmax gets the tile's largest w.
template <bool FILL>
__device__ int stage_nb(const NbCtx &c, int s, int A, int fA, int a0, int P, int nr, NbCursor &cur,
                        const NbSmem<FILL> &sm, float Rcut, float &wmax, bool &last) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)s * c.cap_near;
    const float2 a0f = c.ncomdf[3 * (int64_t)A], a1f = c.ncomdf[3 * (int64_t)A + 1], a2f = c.ncomdf[3 * (int64_t)A + 2];
    const float aabs = fabsf(a0f.x) + fabsf(a1f.x) + fabsf(a2f.x);
    const int64_t t0 = cur.t0, tend = t0 + (kNbTile - 2);
    const float R2cut = Rcut * Rcut;
    sm.self[lane] = -1;
    __syncwarp();
    float wl = 0.f;
    int n_st = 0;
    last = true;
    while (cur.k0 < nr) {
        const int k = cur.k0 + lane;
        int f = 0, n = 0;
        float ox = 0.f, oy = 0.f, oz = 0.f, ow = 0.f;
        if (k < nr) {
            const int B = c.near_list[base + k];
            f = c.nfirst[B];
            n = c.ncount[B];
            const float2 b0 = c.ncomdf[3 * (int64_t)B], b1 = c.ncomdf[3 * (int64_t)B + 1],
                         b2 = c.ncomdf[3 * (int64_t)B + 2];
            ox = (b0.x - a0f.x) + (b0.y - a0f.y);
            oy = (b1.x - a1f.x) + (b1.y - a1f.y);
            oz = (b2.x - a2f.x) + (b2.y - a2f.y);
            ow = 0x1p-20f * (aabs + (fabsf(b0.x) + fabsf(b1.x) + fabsf(b2.x)));
        }
        const int excl = warp_excl_scan(n);
        const int total = __shfl_sync(kFull, excl + n, 31);
        const int64_t pos = cur.pos;
        const int64_t hi = pos + total < tend ? pos + total : tend;
        for (int64_t j0 = pos > t0 ? pos : t0; j0 < hi; j0 += 64) {
            int b[2], cl[2];
            float cx[2], cy[2], cz[2], cw[2];
            bool act[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int rel = (int)(j0 + 32 * u + lane - pos);
                cl[u] = warp_run_of(excl, n, (int)(j0 + 32 * u - pos));
                b[u] = __shfl_sync(kFull, f, cl[u]) + rel - __shfl_sync(kFull, excl, cl[u]);
                cx[u] = __shfl_sync(kFull, ox, cl[u]);
                cy[u] = __shfl_sync(kFull, oy, cl[u]);
                cz[u] = __shfl_sync(kFull, oz, cl[u]);
                cw[u] = __shfl_sync(kFull, ow, cl[u]);
                act[u] = j0 + 32 * u + lane < hi;
            }
            float4 pb[2];
            int ob[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                pb[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                ob[u] = 0;
                if (act[u]) {
                    pb[u] = c.p32[b[u]];
                    if (FILL) ob[u] = c.pidx[b[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float vx = cx[u] + pb[u].x, vy = cy[u] + pb[u].y, vz = cz[u] + pb[u].z;
                const float d2 = fmaf(vz, vz, fmaf(vy, vy, vx * vx));
                const bool keep = act[u] && !(d2 > R2cut);
                const unsigned mk = __ballot_sync(kFull, keep);
                if (keep) {
                    const int at = n_st + __popc(mk & lt);
                    sm.put(at, vx, vy, vz, b[u], ob[u]);
                    wl = fmaxf(wl, (fabsf(cx[u]) + fabsf(cy[u]) + fabsf(cz[u])) + fabsf(pb[u].x) + fabsf(pb[u].y) +
                                       fabsf(pb[u].z) + cw[u]);
                    const int i = b[u] - fA - a0;  // a sink particle of this pass?
                    if (i >= 0 && i < P) sm.self[i] = at;
                }
                n_st += __popc(mk);
            }
        }
        if (pos + total > tend) {  // the tile is full: the next one continues inside this batch
            cur.t0 = tend;
            last = false;
            break;
        }
        cur.pos = pos + total;
        cur.k0 = min(cur.k0 + 32, nr);
    }
    if (last) cur.t0 = cur.pos;
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

// Sort 32 R keys, R per lane (element e = 32 r + lane), ascending in the same layout: a bitonic
// network whose comparators at distance >= 32 stay inside a lane and the others are shuffles.
template <int R>
__device__ inline void warp_sort(int32_t (&v)[R]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int p = r ^ (j >> 5);
                    if (p > r) {
                        const bool up = ((r * 32 + lane) & k) == 0;
                        const int32_t x = v[r], y = v[p];
                        v[r] = up ? min(x, y) : max(x, y);
                        v[p] = up ? max(x, y) : min(x, y);
                    }
                }
            } else {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int32_t y = __shfl_xor_sync(kFull, v[r], j);
                    const bool up = ((r * 32 + lane) & k) == 0;
                    v[r] = (lower == up) ? min(v[r], y) : max(v[r], y);
                }
            }
        }
    }
}

// The same network on each half-warp separately: 16 lanes x R keys per segment (shuffle
// distances below 16 stay inside a half-warp), so two rows of up to 16 R entries sort at once.
template <int R>
__device__ inline void halfwarp_sort(int32_t (&v)[R]) {
    const int hl = threadIdx.x & 15;
#pragma unroll
    for (int k = 2; k <= 16 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 16) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int p = r ^ (j >> 4);
                    if (p > r) {
                        const bool up = ((r * 16 + hl) & k) == 0;
                        const int32_t x = v[r], y = v[p];
                        v[r] = up ? min(x, y) : max(x, y);
                        v[p] = up ? max(x, y) : min(x, y);
                    }
                }
            } else {
                const bool lower = (hl & j) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int32_t y = __shfl_xor_sync(kFull, v[r], j);
                    const bool up = ((r * 16 + hl) & k) == 0;
                    v[r] = (lower == up) ? min(v[r], y) : max(v[r], y);
                }
            }
        }
    }
}

// In-place ascending sort of n keys at p (shared or global memory) by the whole warp: a bitonic
// network with every comparator ascending (a flip stage, then half-cleaners); positions >= n
// count as +infinity and are never touched.
__device__ void warp_sort_inplace(int32_t *p, int n) {
    const int lane = threadIdx.x & 31;
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    for (int k = 2; k <= p2; k <<= 1) {
        for (int i = lane; i < n; i += 32) {
            const int l = i ^ (k - 1);
            if (l > i && l < n) {
                const int32_t x = p[i], y = p[l];
                if (x > y) {
                    p[i] = y;
                    p[l] = x;
                }
            }
        }
        __syncwarp();
        for (int j = k >> 2; j > 0; j >>= 1) {
            for (int i = lane; i < n; i += 32) {
                const int l = i ^ j;
                if (l > i && l < n) {
                    const int32_t x = p[i], y = p[l];
                    if (x > y) {
                        p[i] = y;
                        p[l] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Write the rows of the pass (FILL): rows in the buffer are sorted in registers, two at a time on
// half-warps when both have at most 64 entries, and stored at their offsets; rows appended in
// place are sorted there.
__device__ void nb_write_rows(const NbCtx &c, const NbSmem<true> &sm, int P) {
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const int64_t *goff = sm.goff;
    const int *glen = sm.rowpos + 64;
    int i = 0;
    while (i < P) {
        const int n0 = glen[i], n1 = i + 1 < P ? glen[i + 1] : 0;
        const int rb0 = sm.rowpos[32 + i], rb1 = i + 1 < P ? sm.rowpos[32 + i + 1] : 0;
        if (i + 1 < P && n0 <= 64 && n1 <= 64 && rb0 >= 0 && rb1 >= 0) {
            const int n = half ? n1 : n0, rb = half ? rb1 : rb0;
            const int64_t o = half ? goff[i + 1] : goff[i];
            int32_t v[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int q = r * 16 + hl;
                v[r] = q < n ? sm.rows[rb + q] : INT32_MAX;
            }
            if (n0 <= 32 && n1 <= 32) {
                int32_t w2[2] = {v[0], v[1]};
                halfwarp_sort<2>(w2);
                if (hl < n) c.idx[o + hl] = w2[0];
                if (16 + hl < n) c.idx[o + 16 + hl] = w2[1];
            } else {
                halfwarp_sort<4>(v);
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (r * 16 + hl < n) c.idx[o + r * 16 + hl] = v[r];
            }
            i += 2;
            continue;
        }
        const int n = n0, rb = rb0;
        const int64_t o = goff[i];
        if (rb < 0) {
            warp_sort_inplace(c.idx + o, n);
        } else if (n <= 32) {
            int32_t v[1] = {lane < n ? sm.rows[rb + lane] : INT32_MAX};
            warp_sort<1>(v);
            if (lane < n) c.idx[o + lane] = v[0];
        } else if (n <= 64) {
            int32_t v[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) v[r] = r * 32 + lane < n ? sm.rows[rb + r * 32 + lane] : INT32_MAX;
            warp_sort<2>(v);
#pragma unroll
            for (int r = 0; r < 2; ++r)
                if (r * 32 + lane < n) c.idx[o + r * 32 + lane] = v[r];
        } else if (n <= 128) {
            int32_t v[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) v[r] = r * 32 + lane < n ? sm.rows[rb + r * 32 + lane] : INT32_MAX;
            warp_sort<4>(v);
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (r * 32 + lane < n) c.idx[o + r * 32 + lane] = v[r];
        } else {
            warp_sort_inplace(sm.rows + rb, n);
            for (int q = lane; q < n; q += 32) c.idx[o + q] = sm.rows[rb + q];
        }
        __syncwarp();
        i += 1;
    }
}

// Append the neighbours of one loop step to the rows (FILL): nb0 / nb1 flag the lane's two
// sources (original indices o0, o1); lanes of the same row (mask same) place their entries one
// after another by ballot, so every lane of the row keeps the same running length run.
__device__ __forceinline__ void nb_place(const NbCtx &c, const NbSmem<true> &sm, unsigned same, bool nb0, bool nb1,
                                         int o0, int o1, int rb, int64_t goff, int len, int &run) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned m0 = __ballot_sync(kFull, nb0) & same, m1 = __ballot_sync(kFull, nb1) & same;
    const int p0 = run + __popc(m0 & lt), p1 = run + __popc(m0) + __popc(m1 & lt);
    if (nb0 && p0 < len) {
        if (rb >= 0) sm.rows[rb + p0] = o0;
        else c.idx[goff + p0] = o0;
    }
    if (nb1 && p1 < len) {
        if (rb >= 0) sm.rows[rb + p1] = o1;
        else c.idx[goff + p1] = o1;
    }
    run += __popc(m0) + __popc(m1);
}

// Count pass (FILL = false) or fill pass (FILL = true, offsets known).  Each lane decides its
// pairs by the sign of d^2 - (2h)^2, exact outside the band |d^2 - (2h)^2| <= B; a block of loop
// steps in which some pair fell inside the band is gone through again with the float64 test
// deciding those pairs (counted, or placed by ballot as above).
template <bool FILL>
__global__ void __launch_bounds__(kNbWarps * 32) k_nb(NbCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const NbSmem<FILL> sm(smem_raw + (size_t)w * NbSmem<FILL>::bytes);
    int nfb = 0;
    for (int s = blockIdx.x * kNbWarps + w; s < c.nsinks; s += gridDim.x * kNbWarps) {
        const int A = c.sinks[s];
        const int fA = c.nfirst[A], nA = c.ncount[A];
        const int nr = c.near_nr[s];
        float RA, HA;
        {
            float R2 = 0.f, H = 0.f;
            for (int i = lane; i < nA; i += 32) {
                const float4 pa = c.p32[fA + i];
                R2 = fmaxf(R2, fmaf(pa.z, pa.z, fmaf(pa.y, pa.y, pa.x * pa.x)));
                H = fmaxf(H, c.h32[fA + i]);
            }
            for (int o = 16; o >= 1; o >>= 1) {
                R2 = fmaxf(R2, __shfl_xor_sync(kFull, R2, o));
                H = fmaxf(H, __shfl_xor_sync(kFull, H, o));
            }
            RA = sqrtf(R2) * (1.0f + 0x1p-10f);
            HA = H;
        }
        const float Rcut = (RA + 2.0f * HA) * (1.0f + 0x1p-10f);
        for (int a0 = 0; a0 < nA; a0 += 32) {
            const int P = min(32, nA - a0), S = 32 / P;
            const int i = lane % P, j = lane / P;
            const bool active = j < S;
            const int a = fA + a0 + i;
            const float4 pa = c.p32[a];
            const float h2f = 2.0f * c.h32[a];  // = float32(2 h) exactly
            const float h2 = h2f * h2f;
            const float2 xa = make_float2(pa.x, pa.x), ya = make_float2(pa.y, pa.y), za = make_float2(pa.z, pa.z);
            const float2 nh2 = make_float2(-h2, -h2);
            const float aabs1 = fabsf(pa.x) + fabsf(pa.y) + fabsf(pa.z);
            unsigned same = 0;  // lanes holding the same sink particle
            for (int jj = 0; jj < S; ++jj) same |= 1u << (i + jj * P);
            int cnt = 0, run = 0, rb = -1, len = 0;
            int64_t goff = 0;
            if (FILL) {
                int64_t goff_l = 0;
                int glen_l = 0;
                if (lane < P) {
                    const int o = c.pidx[fA + a0 + lane];
                    goff_l = c.offsets[o];
                    glen_l = (int)(c.offsets[o + 1] - goff_l);
                }
                const int ex = warp_excl_scan(glen_l);
                if (lane < P) {
                    sm.rowpos[32 + lane] = ex + glen_l <= kRowBuf ? ex : -1;
                    sm.rowpos[64 + lane] = glen_l;
                    sm.goff[lane] = goff_l;
                }
                __syncwarp();
                rb = sm.rowpos[32 + i];
                len = sm.rowpos[64 + i];
                goff = sm.goff[i];
            }
            NbCursor cur{0, 0, 0};
            bool last = false;
            while (!last) {
                float wmax;
                const int ns = stage_nb<FILL>(c, s, A, fA, a0, P, nr, cur, sm, Rcut, wmax, last);
                const float F = wmax + aabs1;
                const float B = fmaf(F, F, h2) * 0x1p-19f + 1e-30f;
                const int self = sm.self[i];
                const int np = ns >> 1;
                // the self pair counts below (once, in stream 0)
                if (!FILL && active && j == 0 && self >= 0 && B < h2) --cnt;
                const int nsteps = (np + S - 1) / S;  // loop steps of the warp (stream 0 the longest)
                for (int t0 = 0; t0 < nsteps; t0 += 16) {
                    const int t1 = min(nsteps, t0 + 16);
                    float bandmin = 3e38f;
                    for (int t = t0; t < t1; ++t) {
                        const int k = j + t * S;
                        const bool ok = active && k < np;
                        const int kk = ok ? k : 0;
                        const float4 a4 = sm.A[kk], b4 = sm.B[kk];
                        const float2 dx = __fadd2_rn(xa, make_float2(a4.x, a4.y));
                        const float2 dy = __fadd2_rn(ya, make_float2(a4.z, a4.w));
                        const float2 dz = __fadd2_rn(za, make_float2(b4.x, b4.y));
                        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                        const float2 e = __fadd2_rn(r2, nh2);  // d^2 - (2h)^2
                        const bool in0 = ok && fabsf(e.x) <= B, in1 = ok && fabsf(e.y) <= B;
                        if (ok) bandmin = fminf(bandmin, fminf(fabsf(e.x), fabsf(e.y)));
                        if constexpr (FILL) {
                            const int4 o4 = sm.C[kk];
                            const bool nb0 = ok && e.x < 0.f && !in0 && 2 * k != self;
                            const bool nb1 = ok && e.y < 0.f && !in1 && 2 * k + 1 != self;
                            nb_place(c, sm, same, nb0, nb1, o4.x, o4.y, rb, goff, len, run);
                        } else {
                            if (ok) cnt += (int)(__float_as_uint(e.x) >> 31) + (int)(__float_as_uint(e.y) >> 31);
                        }
                    }
                    // rare: a pair of these steps inside the band, the float64 test decides it
                    if (__any_sync(kFull, bandmin <= B)) {
                        for (int t = t0; t < t1; ++t) {
                            const int k = j + t * S;
                            const bool ok = active && k < np;
                            const int kk = ok ? k : 0;
                            const float4 a4 = sm.A[kk], b4 = sm.B[kk];
                            const float2 dx = __fadd2_rn(xa, make_float2(a4.x, a4.y));
                            const float2 dy = __fadd2_rn(ya, make_float2(a4.z, a4.w));
                            const float2 dz = __fadd2_rn(za, make_float2(b4.x, b4.y));
                            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                            const float2 e = __fadd2_rn(r2, nh2);
                            bool nb[2] = {false, false};
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                const float ev = u ? e.y : e.x;
                                if (ok && fabsf(ev) <= B) {
                                    nb[u] = nb_exact(c.px, c.py, c.pz, c.ph, a, __float_as_int(u ? b4.w : b4.z));
                                    if (!FILL) cnt += (int)nb[u] - (int)(__float_as_uint(ev) >> 31);
                                    ++nfb;
                                }
                            }
                            if constexpr (FILL) {
                                const int4 o4 = sm.C[kk];
                                nb_place(c, sm, same, nb[0], nb[1], o4.x, o4.y, rb, goff, len, run);
                            }
                        }
                    }
                }
                __syncwarp();
            }
            if constexpr (FILL) {
                // lane l < P holds row l in stream 0: its running length is the row's
                if (lane < P && run != sm.rowpos[64 + lane]) atomicOr(&c.status[ST_ERR], ERRBIT_STATE);
                __syncwarp();
                nb_write_rows(c, sm, P);
            } else {
                // sum the S streams of each sink particle through shared memory
                int *red = reinterpret_cast<int *>(sm.A);
                if (active) red[lane] = cnt;
                __syncwarp();
                if (lane < P) {
                    int tn = 0;
                    for (int jj = 0; jj < S; ++jj) tn += red[lane + jj * P];
                    c.counts[c.pidx[a]] = tn;
                }
            }
            __syncwarp();
        }
    }
    for (int o = 16; o >= 1; o >>= 1) nfb += __shfl_xor_sync(kFull, nfb, o);
    if (lane == 0 && nfb && !FILL) atomicAdd(&c.status[ST_NBFALLBACK], nfb);
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
    c.status = t->d_status;
    return c;
}

template <bool FILL>
int launch_nb(rcb_tree *t, const NbCtx &c) {
    if (t->nsinks == 0) return RCB_OK;
    const int nsm = sm_count_nb();
    const size_t smem = (size_t)kNbWarps * NbSmem<FILL>::bytes;
    RCB_CUDA_TRY(cudaFuncSetAttribute(k_nb<FILL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int blocks = std::max(1, std::min((t->nsinks + kNbWarps - 1) / kNbWarps, nsm * 16));
    k_nb<FILL><<<blocks, kNbWarps * 32, smem, t->stream>>>(c); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

}  // namespace

int neighbour_counts(rcb_tree *t, int64_t *counts, int *status) {
    NbCtx c = make_nbctx(t);
    c.counts = counts;
    c.status = status;
    return launch_nb<false>(t, c);
}

int scan_neighbour_counts(rcb_tree *t) {
    return scan_i64(t->nb_count, t->nb_count, t->N, t->nb_count + t->N, t->scan_tmp, t->stream);
}

int fetch_neighbour_total(rcb_tree *t) {
    cudaStream_t st = t->stream;
    // the total (int64, 8-byte aligned slot of the pinned buffer) and two status words
    int rc = copy_words(t->h_status_dev + ST_NWORDS + 2, t->nb_count + t->N, 2, st);
    if (!rc) rc = copy_words(t->h_status_dev + ST_NBFALLBACK, t->d_status + ST_NBFALLBACK, 2, st);
    if (rc) return rc;
    RCB_CUDA_TRY(cudaStreamSynchronize(st));
    std::memcpy(&t->nb_total, t->h_status + ST_NWORDS + 2, sizeof(int64_t));
    t->nb_valid = 1;
    return RCB_OK;
}

int count_neighbours(rcb_tree *t) {
    if (t->nb_valid) return RCB_OK;
    NbCtx c = make_nbctx(t);
    stage_begin(t, SG_NB_COUNT);
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_status + ST_NBFALLBACK, 0, 2 * sizeof(int), t->stream));
    int rc = launch_nb<false>(t, c);
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
    rc = launch_nb<true>(t, c);
    if (rc) return rc;
    stage_end(t, SG_NB_FILL);
    RCB_CUDA_TRY(cudaGetLastError());
    // the fill pass re-derives every row; a row whose length differs from its count is an error
    rc = copy_words(t->h_status_dev, t->d_status, 1, st);
    if (rc) return rc;
    RCB_CUDA_TRY(cudaStreamSynchronize(st));
    if (t->h_status[ST_ERR] & ERRBIT_STATE) return RCB_ERR_STATE;
    return RCB_OK;
}

}  // namespace rcb
