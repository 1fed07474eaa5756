// Gravity (Sec. 2.4): far field per sink by the cell-cell Taylor expansion (Eq. 5, Eq. 6) and
// near field by kernel-softened direct summation (Eqs. 9-10), in two forms.
//
// far    one warp per sink, lanes over its far nodes.  For a source B with mass M and traceless
//        quadrupole Q at x = r_A - r_B, with g = 1/|x|, v = Q x and s = x.v, the potential
//        Phi = -M g - s g^5 / 2 and its derivatives up to third order are
//          C0    = -M g - s g^5 / 2
//          C1_i  = a x_i - g^5 v_i,                             a = M g^3 + 5/2 s g^7
//          C2_ij = b x_i x_j + a d_ij - g^5 Q_ij + 5 g^7 (v_i x_j + v_j x_i),
//                                                               b = -3 M g^5 - 35/2 s g^9
//          C3_ijk = c x_i x_j x_k + b (d_ij x_k + d_ik x_j + d_jk x_i)
//                   + 5 g^7 (Q_ij x_k + Q_ik x_j + Q_jk x_i + v_i d_jk + v_j d_ik + v_k d_ij)
//                   - 35 g^9 (v_i x_j x_k + v_j x_i x_k + v_k x_i x_j),   c = 15 M g^7 + 315/2 s g^11
//        (1 + 3 + 6 + 10 = 20 coefficients per sink).  Mixed form: float32 tensor math on the
//        double-float difference of the two centres of mass, per-lane float32 partial sums, and
//        a compensated (TwoSum) reduce-scatter across the warp; each coefficient then becomes
//        one float64 (hi + lo).  FP64 form: everything in float64.
// near   one warp per sink; the particles of its near cells are staged in shared memory (mixed:
//        float32 offsets from the sink's centre of mass; FP64: absolute float64 positions), lanes
//        take sources, the sink's particles sit in registers.  Per pair
//          r^2, 1/r, q = 2 r / (h_a + h_b);  S/r = 1/r^3 and phi = -1/r for q >= 2, otherwise
//          the cubic-spline polynomials of Eq. 10 and their potential.
//        Mixed form accumulates in float32 per tile and folds each tile into a compensated
//        (sum, error) pair.  The epilogue reduces across lanes, evaluates the sink's third-order
//        Taylor polynomial at the particle (Eq. 6), adds both parts and scatters acc and pot to
//        original order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "far_math.cuh"
#include "rcb_internal.cuh"

namespace rcb {
namespace {

constexpr int kGWarps = 4;
constexpr int kGroupMixed = 8;  // sink particles per group (mixed near kernel)
constexpr int kGroupF64 = 4;
constexpr int kNearTileMixed = 1024;
constexpr int kNearTileF64 = 384;

struct GCtx {
    int nsinks;
    const int32_t *sinks, *near_list, *near_nr, *near_nn, *far_list, *far_n;
    int cap_near, cap_far;
    const int32_t *nfirst, *ncount;
    const double *ncom, *nmass, *nQ;
    const float2 *ncomdf;
    const float4 *mq32a, *mq32b;
    const float4 *nfar;
    const double *px, *py, *pz, *pm, *ph;
    const float4 *p32;
    const float *h32;
    const int32_t *pidx;
    double *coef;
    float *coef32;
    double *acc, *pot;
    // neighbour search fused into the mixed near field
    int64_t *nb_counts;  // [N] by original index
    int32_t *nb_rows;    // [N][kNbRowCap] by sorted index
    int2 *nb_long;
    int cap_long;
    int *status;
};

// ------------------------------------------------------------------------------------------ far
template <bool MIXED>
__global__ void __launch_bounds__(kGWarps * 32) k_far(GCtx c) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kGWarps + (threadIdx.x >> 5);
    for (int s = gw; s < c.nsinks; s += gridDim.x * kGWarps) {
        const int A = c.sinks[s];
        const int nf = c.far_n[s];
        const int64_t fb = (int64_t)s * c.cap_far;
        if (MIXED) {
            // two far nodes per lane and round (k and k + 32), paired float32 arithmetic
            float2 C2[20];
#pragma unroll
            for (int i = 0; i < 20; ++i) C2[i] = make_float2(0.f, 0.f);
            const float4 ah = c.nfar[4 * (int64_t)A], al = c.nfar[4 * (int64_t)A + 1];
            float4 p[2][4];
            auto fetch = [&](int k0) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int k = k0 + 32 * u;
                    if (k < nf) {
                        const float4 *r = c.nfar + 4 * (int64_t)c.far_list[fb + k];
                        p[u][0] = r[0];
                        p[u][1] = r[1];
                        p[u][2] = r[2];
                        p[u][3] = r[3];
                    } else {
                        // no node: zero mass and quadrupole (its offset is set to (1, 0, 0) below)
                        p[u][0] = make_float4(0.f, 0.f, 0.f, 0.f);
                        p[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                        p[u][2] = make_float4(0.f, 0.f, 0.f, 0.f);
                        p[u][3] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            };
            int k = lane;
            while (k < nf) {
                fetch(k);
                float4 q[2][4];
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int e = 0; e < 4; ++e) q[u][e] = p[u][e];
                const int kn = k + 64;
                const bool second = k + 32 < nf;
                const float2 x0 = make_float2((ah.x - q[0][0].x) + (al.x - q[0][1].x),
                                              second ? (ah.x - q[1][0].x) + (al.x - q[1][1].x) : 1.f);
                const float2 x1 = make_float2((ah.y - q[0][0].y) + (al.y - q[0][1].y),
                                              second ? (ah.y - q[1][0].y) + (al.y - q[1][1].y) : 0.f);
                const float2 x2 = make_float2((ah.z - q[0][0].z) + (al.z - q[0][1].z),
                                              second ? (ah.z - q[1][0].z) + (al.z - q[1][1].z) : 0.f);
                far_source2(x0, x1, x2, make_float2(q[0][0].w, q[1][0].w), make_float2(q[0][1].w, q[1][1].w),
                            make_float2(q[0][2].x, q[1][2].x), make_float2(q[0][2].y, q[1][2].y),
                            make_float2(q[0][2].z, q[1][2].z), make_float2(q[0][2].w, q[1][2].w),
                            make_float2(q[0][3].x, q[1][3].x), C2);
                k = kn;
            }
            float C[32];
#pragma unroll
            for (int i = 0; i < 20; ++i) C[i] = C2[i].x + C2[i].y;
#pragma unroll
            for (int i = 20; i < 32; ++i) C[i] = 0.f;
            float E[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) E[i] = 0.f;
            reduce_scatter_df<32>(C, E);
            if (lane < 20) {
                c.coef[(int64_t)s * 20 + lane] = __dadd_rn((double)C[0], (double)E[0]);
                c.coef32[(int64_t)s * 20 + lane] = __fadd_rn(C[0], E[0]);
            }
        } else {
            double C[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) C[i] = 0.0;
            const double ax = c.ncom[3 * (int64_t)A], ay = c.ncom[3 * (int64_t)A + 1], az = c.ncom[3 * (int64_t)A + 2];
            for (int k = lane; k < nf; k += 32) {
                const int B = c.far_list[fb + k];
                const double x[3] = {ax - c.ncom[3 * (int64_t)B], ay - c.ncom[3 * (int64_t)B + 1], az - c.ncom[3 * (int64_t)B + 2]};
                double Q6[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) Q6[q] = c.nQ[6 * (int64_t)B + q];
                far_source<double>(x, c.nmass[B], Q6, C);
            }
            reduce_scatter<32, double>(C);
            if (lane < 20) c.coef[(int64_t)s * 20 + lane] = C[0];
        }
    }
}

// near-list entry k of sink s (reachable cells first, then the rest from the back of the slot)
__device__ inline int near_entry(const GCtx &c, int64_t base, int nr, int k) {
    return k < nr ? c.near_list[base + k] : c.near_list[base + c.cap_near - 1 - (k - nr)];
}

// Stage sources [t0, t0 + tile) of the concatenated near cells.
template <bool MIXED>
__device__ int stage_near(const GCtx &c, int s, int A, int nlist, int nr, int64_t t0, int tile, void *smw) {
    const int lane = threadIdx.x & 31;
    const int64_t base = (int64_t)s * c.cap_near;
    int64_t pos = 0;
    int staged = 0;
    float2 cA[3];
    if (MIXED)
        for (int d = 0; d < 3; ++d) cA[d] = c.ncomdf[3 * (int64_t)A + d];
    for (int k0 = 0; k0 < nlist; k0 += 32) {
        const int k = k0 + lane;
        int f = 0, n = 0;
        float ox = 0.f, oy = 0.f, oz = 0.f;
        if (k < nlist) {
            const int B = near_entry(c, base, nr, k);
            f = c.nfirst[B];
            n = c.ncount[B];
            if (MIXED) {
                const float2 b0 = c.ncomdf[3 * (int64_t)B], b1 = c.ncomdf[3 * (int64_t)B + 1], b2 = c.ncomdf[3 * (int64_t)B + 2];
                ox = (b0.x - cA[0].x) + (b0.y - cA[0].y);
                oy = (b1.x - cA[1].x) + (b1.y - cA[1].y);
                oz = (b2.x - cA[2].x) + (b2.y - cA[2].y);
            }
        }
        int incl = n;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int group_total = __shfl_sync(0xffffffffu, incl, 31);
        const int64_t my0 = pos + incl - n;
        for (int j = 0; j < 32 && k0 + j < nlist; ++j) {
            const int64_t c0 = __shfl_sync(0xffffffffu, my0, j);
            const int cn = __shfl_sync(0xffffffffu, n, j);
            const int cf = __shfl_sync(0xffffffffu, f, j);
            const float bx = __shfl_sync(0xffffffffu, ox, j), by = __shfl_sync(0xffffffffu, oy, j),
                        bz = __shfl_sync(0xffffffffu, oz, j);
            const int64_t lo = c0 > t0 ? c0 : t0;
            const int64_t hi = c0 + cn < t0 + tile ? c0 + cn : t0 + tile;
            for (int64_t q = lo + lane; q < hi; q += 32) {
                const int b = cf + (int)(q - c0);
                const int slot = (int)(q - t0);
                if (MIXED) {
                    float4 *src = reinterpret_cast<float4 *>(smw);
                    float *hs = reinterpret_cast<float *>(src + kNearTileMixed);
                    int32_t *si = reinterpret_cast<int32_t *>(hs + kNearTileMixed);
                    const float4 pb = c.p32[b];
                    src[slot] = make_float4(bx + pb.x, by + pb.y, bz + pb.z, pb.w);
                    hs[slot] = c.h32[b];
                    si[slot] = b;
                } else {
                    double *X = reinterpret_cast<double *>(smw);
                    X[slot] = c.px[b];
                    X[kNearTileF64 + slot] = c.py[b];
                    X[2 * kNearTileF64 + slot] = c.pz[b];
                    X[3 * kNearTileF64 + slot] = c.pm[b];
                    X[4 * kNearTileF64 + slot] = c.ph[b];
                    reinterpret_cast<int32_t *>(X + 5 * kNearTileF64)[slot] = b;
                }
            }
            if (hi > lo) staged = max(staged, (int)(hi - t0));
        }
        pos += group_total;
        if (pos >= t0 + tile) break;
    }
    __syncwarp();
    return staged;
}


constexpr int kNearWarps = 8;     // warps per block of the mixed near kernel
constexpr int kNearTile = 512;    // staged sources per warp
constexpr int kNbChunks = kNearTile / 32;  // 32-source chunks of a tile
constexpr int kSuper = 3;                   // groups of sink particles sharing one staged tile

// Shared memory of one warp of the mixed near kernel.  With the neighbour search (NB) it also
// holds each source's sorted index (bitwise complement for sources of non-candidate cells) and
// each sink particle's float32 neighbour band.
template <bool NB>
struct NearSmem {
    static constexpr size_t bytes =
        kNearTile * (sizeof(float4) + sizeof(float)) + 2 * kGroupMixed * sizeof(float4) +
        kSuper * 32 * sizeof(float2) + (NB ? kSuper * kGroupMixed * sizeof(int) : 0) +
        (NB ? kNearTile * sizeof(int32_t) + kGroupMixed * sizeof(float2) + kGroupMixed * sizeof(float2) +
                  kNbChunks * kGroupMixed * sizeof(unsigned)
            : 0);
    float4 *src;    // (d_b relative to the sink's centre of mass, m_b)
    float *hs;      // h_b
    float4 *snk;    // (d_a, h_a) of the current group
    float4 *snk2;   // the same by pairs (i, i + 1): (x_i, x_i+1, y_i, y_i+1), (z_i, z_i+1, h_i, h_i+1)
    float2 *hi2;    // NB: upper band edges by pairs
    float2 *lo2;    // NB: lower band edges by pairs
    int32_t *sidx;  // NB
    float2 *band;   // NB: per sink particle (2h)^2 -+ B
    unsigned *mamb; // NB: [chunk][sink particle] sources inside the band (float64 decides)
    float2 *gacc;   // [group][lane] the lanes' compensated totals of the groups sharing a tile
    int *grun;      // NB: [group][sink particle] neighbours found so far
    __device__ NearSmem(unsigned char *p) {
        src = reinterpret_cast<float4 *>(p);
        hs = reinterpret_cast<float *>(src + kNearTile);
        snk = reinterpret_cast<float4 *>(hs + kNearTile);
        snk2 = snk + kGroupMixed;
        band = reinterpret_cast<float2 *>(snk2 + kGroupMixed);
        hi2 = band + (NB ? kGroupMixed : 0);
        lo2 = hi2 + (NB ? kGroupMixed / 2 : 0);
        sidx = reinterpret_cast<int32_t *>(lo2 + (NB ? kGroupMixed / 2 : 0));
        mamb = reinterpret_cast<unsigned *>(sidx + (NB ? kNearTile : 0));
        gacc = reinterpret_cast<float2 *>(mamb + (NB ? kNbChunks * kGroupMixed : 0));
        grun = reinterpret_cast<int *>(gacc + kSuper * 32);
    }
};

// Staged tile: the close sources at [0, nclose) of src/hs (and sidx), the far ones at
// [kNearTile - nfar, kNearTile) (see below).
struct NearTile {
    int nclose, nfar;
    int64_t S;  // all sources of the sink
};

// Stage sources [t0, t0 + kNearTile) of the sink's near cells.  For 32 cells at a time, lanes
// first describe the cells (first particle, count, centre-of-mass offset), then take one slot
// each (two slot chunks per round, so both gathers are in flight together), find the slot's
// cell, form the particle's float32 offset from the sink's centre of mass and store it with
// its mass and h, close sources from the front of the tile and far ones from the back.  The
// cell offset o is the double-float difference of the two centres of mass: it differs from the
// float64 difference by at most 2u |dCOM| + 3 2^-48 (|COM_A|_1 + |COM_B|_1) per component
// (u = 2^-24; the second term is the double-float representation).  With NB the sorted index is
// kept (bitwise complement for sources of non-candidate cells) and wmax gets the tile's largest
// w = |o|_1 + |d_b|_1 + 2^-20 (|COM_A|_1 + |COM_B|_1): the last term makes the representation
// error's share of the d^2 error at most 6 2^-28 F, well inside the neighbour band.
//
// Far sources: with R_A the largest |d_a| and H_A the largest h_a of the sink's particles, a
// source b with |d_b| > (R_A + X_b)(1 + 2^-10) has r_ab >= |d_b| - |d_a| > X_b for every sink
// particle a.  X_b = H_A + h_b puts all its pairs on the Newtonian branch of Eq. 10 (q >= 2);
// with NB, X_b = max(H_A + h_b, 2 H_A) also keeps it out of every sink particle's neighbour
// sphere (r < 2 h_a).  The 2^-10 margin is far above the float32 rounding of the test, of q and
// of the neighbour filter.
template <bool NB>
__device__ NearTile stage_near_mixed(const GCtx &c, int s, int A, int nlist, int nr, int64_t t0, const NearSmem<NB> &sm,
                                     float RA, float HA, float &wmax) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)s * c.cap_near;
    const float2 a0 = c.ncomdf[3 * (int64_t)A], a1 = c.ncomdf[3 * (int64_t)A + 1], a2 = c.ncomdf[3 * (int64_t)A + 2];
    const float aabs = fabsf(a0.x) + fabsf(a1.x) + fabsf(a2.x);
    int64_t pos = 0;
    float wl = 0.f;
    int nclose = 0, nfar = 0;
    for (int k0 = 0; k0 < nlist; k0 += 32) {
        const int k = k0 + lane;
        int f = 0, n = 0;
        float ox = 0.f, oy = 0.f, oz = 0.f, ow = 0.f;
        const bool inside = pos < t0 + kNearTile;  // cells beyond the tile are only counted
        if (k < nlist) {
            const int B = near_entry(c, base, nr, k);
            n = c.ncount[B];
        }
        if (k < nlist && inside) {
            const int B = near_entry(c, base, nr, k);
            f = c.nfirst[B];
            const float2 b0 = c.ncomdf[3 * (int64_t)B], b1 = c.ncomdf[3 * (int64_t)B + 1],
                         b2 = c.ncomdf[3 * (int64_t)B + 2];
            ox = (b0.x - a0.x) + (b0.y - a0.y);
            oy = (b1.x - a1.x) + (b1.y - a1.y);
            oz = (b2.x - a2.x) + (b2.y - a2.y);
            if (NB) ow = 0x1p-20f * (aabs + (fabsf(b0.x) + fabsf(b1.x) + fabsf(b2.x)));
        }
        const int excl = warp_excl_scan(n);
        const int total = __shfl_sync(0xffffffffu, excl + n, 31);
        const int64_t lo = pos > t0 ? pos : t0;
        const int64_t hi = pos + total < t0 + kNearTile ? pos + total : t0 + kNearTile;
        for (int64_t j0 = lo; j0 < hi; j0 += 64) {
            int b[2], cl[2];
            float cx[2], cy[2], cz[2], cw[2];
            bool act[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int rel = (int)(j0 + 32 * u + lane - pos);
                cl[u] = warp_run_of(excl, n, (int)(j0 + 32 * u - pos));
                b[u] = __shfl_sync(0xffffffffu, f, cl[u]) + rel - __shfl_sync(0xffffffffu, excl, cl[u]);
                cx[u] = __shfl_sync(0xffffffffu, ox, cl[u]);
                cy[u] = __shfl_sync(0xffffffffu, oy, cl[u]);
                cz[u] = __shfl_sync(0xffffffffu, oz, cl[u]);
                cw[u] = NB ? __shfl_sync(0xffffffffu, ow, cl[u]) : 0.f;
                act[u] = j0 + 32 * u + lane < hi;
            }
            float4 pb[2];
            float hb[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                pb[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                hb[u] = 0.f;
                if (act[u]) {
                    pb[u] = c.p32[b[u]];
                    hb[u] = c.h32[b[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float4 v = make_float4(cx[u] + pb[u].x, cy[u] + pb[u].y, cz[u] + pb[u].z, pb[u].w);
                const float d2 = fmaf(v.z, v.z, fmaf(v.y, v.y, v.x * v.x));
                const float X = NB ? fmaxf(HA + hb[u], HA + HA) : HA + hb[u];
                const float R = (RA + X) * (1.0f + 0x1p-10f);
                const bool far = d2 > R * R;
                const unsigned mc = __ballot_sync(0xffffffffu, act[u] && !far);
                const unsigned mf = __ballot_sync(0xffffffffu, act[u] && far);
                if (act[u]) {
                    const int at = far ? kNearTile - 1 - (nfar + __popc(mf & lt)) : nclose + __popc(mc & lt);
                    sm.src[at] = v;
                    sm.hs[at] = hb[u];
                    if (NB) {
                        sm.sidx[at] = k0 + cl[u] < nr ? b[u] : ~b[u];
                        wl = fmaxf(wl, (fabsf(cx[u]) + fabsf(cy[u]) + fabsf(cz[u])) + fabsf(pb[u].x) + fabsf(pb[u].y) +
                                           fabsf(pb[u].z) + cw[u]);
                    }
                }
                nclose += __popc(mc);
                nfar += __popc(mf);
            }
        }
        pos += total;
    }
    if (NB) {
        for (int o = 16; o >= 1; o >>= 1) wl = fmaxf(wl, __shfl_xor_sync(0xffffffffu, wl, o));
        wmax = wl;
    }
    __syncwarp();
    return NearTile{nclose, nfar, pos};
}

// Neighbour-search state of one group of sink particles.
struct NbGroup {
    int a0;                 // sorted index of the group's first sink particle
    int run[kGroupMixed];   // neighbours of sink particle i found so far (the same in every lane)
    int nfb;                // float64 decisions taken (per lane)
};

// Append the sources of mask m (bits = lanes of chunk k) to sink particle i's row: the lanes
// whose bit is set write consecutive slots.  The order inside a row is free (the compaction
// sorts each row).
__device__ __forceinline__ void nb_append(const GCtx &c, int a, int &run, unsigned m, int sb) {
    const int lane = threadIdx.x & 31;
    if ((m >> lane) & 1u) {
        const int p = run + __popc(m & ((1u << lane) - 1u));
        if (p < kNbRowCap) c.nb_rows[(int64_t)a * kNbRowCap + p] = sb;
    }
    run += __popc(m);
}

// Sources inside a sink particle's float32 band (mamb, recorded by the close loop per chunk and
// sink particle) are settled by the float64 test, every lane of the chunk at once, and appended.
template <int G>
__device__ inline void settle_band(const GCtx &c, const NearSmem<true> &sm, int nchunks, int na, NbGroup &g) {
    const int lane = threadIdx.x & 31;
    for (int e0 = 0; e0 < nchunks * G; e0 += 32) {
        const int e = e0 + lane;
        unsigned todo = __ballot_sync(0xffffffffu, e < nchunks * G && (e % G) < na && sm.mamb[e] != 0u);
        while (todo) {
            const int ee = e0 + __ffs(todo) - 1;
            todo &= todo - 1;
            const int k = ee / G, i = ee % G;
            const unsigned amb = sm.mamb[ee];
            const int a = g.a0 + i;
            const int sb = sm.sidx[32 * k + lane];
            bool nb = false;
            if (((amb >> lane) & 1u) && sb != a) {
                const double s2 = __dmul_rn(2.0, c.ph[a]);
                nb = dist2_rn(c.px[a], c.py[a], c.pz[a], c.px[sb], c.py[sb], c.pz[sb]) < __dmul_rn(s2, s2);
                ++g.nfb;
            }
            const unsigned m = __ballot_sync(0xffffffffu, nb);
#pragma unroll
            for (int q = 0; q < G; ++q)
                if (q == i) nb_append(c, a, g.run[q], m, sb);
        }
    }
}

// The pair loops of one staged tile for G sink particles (snk[0, G)), folded into the lane's
// compensated total (rs, rc) of value (lane mod 4 G) = 4 i + q.  With NB the close loop also
// tests every candidate pair (a, b) for |r_a - r_b| < 2 h_a (float32 d^2 against the band of
// sink particle i, one ballot per band edge) and records the masks from which emit_neighbours
// settles the in-band pairs in float64 and appends b's sorted index to a's row of slots.
template <int G, bool NB>
__device__ inline void near_tile(const GCtx &c, const NearSmem<NB> &sm, const NearTile &tl, int na, float &rs,
                                 float &rc, NbGroup &g) {
    const int nclose = tl.nclose;
    const int npair = (na + 1) >> 1;  // sink particle pairs holding a real particle (warp-uniform)
    static_assert(G % 2 == 0, "sink particles go by pairs");
    const int lane = threadIdx.x & 31;
    // In[q][p]: quantity q (a_x, a_y, a_z, phi) of sink particles 2p and 2p + 1.  Every pair
    // term below is computed for two sink particles at once with paired float32 instructions
    // (each half rounds exactly as the scalar operation would).
    float2 In[4][G / 2];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < G / 2; ++p) In[q][p] = make_float2(0.f, 0.f);
    // far sources: every pair outside its kernel support, Newtonian only
    for (int q0 = kNearTile - tl.nfar; q0 < kNearTile; q0 += 32) {
        const int j = q0 + lane;
        // padding lanes: a massless source far away (finite r, zero contribution)
        const float4 b = j < kNearTile ? sm.src[j] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
        const float2 nbx = make_float2(-b.x, -b.x), nby = make_float2(-b.y, -b.y), nbz = make_float2(-b.z, -b.z);
        const float2 nbm = make_float2(-b.w, -b.w);
#pragma unroll
        for (int p = 0; p < G / 2; ++p) {
            if (p > 0 && p >= npair) break;  // padding pairs of a short group
            const float4 sxy = sm.snk2[2 * p], szh = sm.snk2[2 * p + 1];
            const float2 dx = __fadd2_rn(make_float2(sxy.x, sxy.y), nbx);
            const float2 dy = __fadd2_rn(make_float2(sxy.z, sxy.w), nby);
            const float2 dz = __fadd2_rn(make_float2(szh.x, szh.y), nbz);
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            const float2 rinv = make_float2(rsqrtf(fmaxf(r2.x, 1e-30f)), rsqrtf(fmaxf(r2.y, 1e-30f)));
            const float2 nw = __fmul2_rn(nbm, __fmul2_rn(__fmul2_rn(rinv, rinv), rinv));  // -m_b / r^3
            In[0][p] = __ffma2_rn(nw, dx, In[0][p]);
            In[1][p] = __ffma2_rn(nw, dy, In[1][p]);
            In[2][p] = __ffma2_rn(nw, dz, In[2][p]);
            In[3][p] = __ffma2_rn(nbm, rinv, In[3][p]);
        }
    }
    // close sources: the full kernel-softened pair
    const float2 k05 = make_float2(0.5f, 0.5f), km12 = make_float2(-1.2f, -1.2f), k43 = make_float2(4.0f / 3.0f, 4.0f / 3.0f);
    const float2 k01 = make_float2(0.1f, 0.1f), km03 = make_float2(-0.3f, -0.3f), k23 = make_float2(2.0f / 3.0f, 2.0f / 3.0f);
    const float2 km14 = make_float2(-1.4f, -1.4f), km16 = make_float2(-1.0f / 6.0f, -1.0f / 6.0f);
    const float2 k12 = make_float2(1.2f, 1.2f), km3 = make_float2(-3.0f, -3.0f), k83 = make_float2(8.0f / 3.0f, 8.0f / 3.0f);
    const float2 km115 = make_float2(-1.0f / 15.0f, -1.0f / 15.0f), km130 = make_float2(-1.0f / 30.0f, -1.0f / 30.0f);
    const float2 k03 = make_float2(0.3f, 0.3f), km1 = make_float2(-1.0f, -1.0f), km16b = make_float2(-1.6f, -1.6f);
    const float2 k115 = make_float2(1.0f / 15.0f, 1.0f / 15.0f);
    for (int q0 = 0; q0 < nclose; q0 += 32) {
        const int j = q0 + lane;
        float4 b = make_float4(1e18f, 1e18f, 1e18f, 0.f);
        float hb = 1.f;
        int sb = -1;
        if (j < nclose) {
            b = sm.src[j];
            hb = sm.hs[j];
            if (NB) sb = sm.sidx[j];
        }
        const unsigned cand = NB ? __ballot_sync(0xffffffffu, sb >= 0) : 0u;  // candidate-cell sources
        const int kc = q0 >> 5;                                                  // chunk of the tile
        const bool own = NB && __any_sync(0xffffffffu, sb >= g.a0 && sb < g.a0 + G);  // holds group particles
        const float2 nbx = make_float2(-b.x, -b.x), nby = make_float2(-b.y, -b.y), nbz = make_float2(-b.z, -b.z);
        const float2 bm = make_float2(b.w, b.w), nbm = make_float2(-b.w, -b.w), hb2 = make_float2(hb, hb);
#pragma unroll
        for (int p = 0; p < G / 2; ++p) {
            if (p > 0 && p >= npair) break;  // padding pairs of a short group
            // sink particles 2p and 2p + 1 against this lane's source (the self pair has r = 0:
            // zero force; its potential m_a phi(0) is removed in the epilogue)
            const float4 sxy = sm.snk2[2 * p], szh = sm.snk2[2 * p + 1];
            const float2 dx = __fadd2_rn(make_float2(sxy.x, sxy.y), nbx);
            const float2 dy = __fadd2_rn(make_float2(sxy.z, sxy.w), nby);
            const float2 dz = __fadd2_rn(make_float2(szh.x, szh.y), nbz);
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            const float2 rinv = make_float2(rsqrtf(fmaxf(r2.x, 1e-30f)), rsqrtf(fmaxf(r2.y, 1e-30f)));
            const float2 r = __fmul2_rn(r2, rinv);
            const float2 hsum = __fadd2_rn(make_float2(szh.z, szh.w), hb2);
            const float2 hinv = make_float2(__fdividef(2.0f, hsum.x), __fdividef(2.0f, hsum.y));
            const float2 q = __fmul2_rn(r, hinv);
            const float2 q2 = __fmul2_rn(q, q);
            const float2 rinv3 = __fmul2_rn(__fmul2_rn(rinv, rinv), rinv);
            // Eq. 10 as S/r and its potential: q < 1, 1 <= q < 2, q >= 2
            const float2 h3 = __fmul2_rn(__fmul2_rn(hinv, hinv), hinv);
            const float2 s1 = __fmul2_rn(h3, __ffma2_rn(q2, __ffma2_rn(k05, q, km12), k43));
            const float2 p1 = __fmul2_rn(hinv, __ffma2_rn(q2, __ffma2_rn(q2, __ffma2_rn(k01, q, km03), k23), km14));
            const float2 s2v = __ffma2_rn(h3, __ffma2_rn(q, __ffma2_rn(q, __ffma2_rn(km16, q, k12), km3), k83),
                                          __fmul2_rn(km115, rinv3));
            const float2 p2v =
                __ffma2_rn(hinv, __ffma2_rn(q2, __ffma2_rn(q, __ffma2_rn(q, __ffma2_rn(km130, q, k03), km1), k43), km16b),
                           __fmul2_rn(k115, rinv));
            const float2 sr = make_float2(q.x < 1.0f ? s1.x : (q.x < 2.0f ? s2v.x : rinv3.x),
                                          q.y < 1.0f ? s1.y : (q.y < 2.0f ? s2v.y : rinv3.y));
            const float2 ph = make_float2(q.x < 1.0f ? p1.x : (q.x < 2.0f ? p2v.x : -rinv.x),
                                          q.y < 1.0f ? p1.y : (q.y < 2.0f ? p2v.y : -rinv.y));
            const float2 nw = __fmul2_rn(nbm, sr);
            In[0][p] = __ffma2_rn(nw, dx, In[0][p]);
            In[1][p] = __ffma2_rn(nw, dy, In[1][p]);
            In[2][p] = __ffma2_rn(nw, dz, In[2][p]);
            In[3][p] = __ffma2_rn(bm, ph, In[3][p]);
            if (NB) {
                // neighbour test of sink particles 2p and 2p + 1 against this chunk: sources below
                // the band are appended now, those inside it are recorded for settle_band; a
                // particle is not its own neighbour
                const float2 hi = sm.hi2[p], lo = sm.lo2[p];
                unsigned l0 = __ballot_sync(0xffffffffu, r2.x < lo.x) & cand;
                const unsigned h0 = __ballot_sync(0xffffffffu, r2.x <= hi.x) & cand;
                unsigned l1 = __ballot_sync(0xffffffffu, r2.y < lo.y) & cand;
                const unsigned h1 = __ballot_sync(0xffffffffu, r2.y <= hi.y) & cand;
                if (lane == 0) {
                    sm.mamb[kc * G + 2 * p] = h0 & ~l0;
                    sm.mamb[kc * G + 2 * p + 1] = h1 & ~l1;
                }
                if (own) {
                    l0 &= ~__ballot_sync(0xffffffffu, sb == g.a0 + 2 * p);
                    l1 &= ~__ballot_sync(0xffffffffu, sb == g.a0 + 2 * p + 1);
                }
                nb_append(c, g.a0 + 2 * p, g.run[2 * p], l0, sb);
                nb_append(c, g.a0 + 2 * p + 1, g.run[2 * p + 1], l1, sb);
            }
        }
    }
    if constexpr (NB) {
        __syncwarp();
        settle_band<G>(c, sm, (nclose + 31) >> 5, na, g);
    }
    // fold this tile: compensated reduce-scatter across lanes, then into (rs, rc)
    float Vs[4 * G], Vc[4 * G];
#pragma unroll
    for (int i = 0; i < G; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            Vs[4 * i + q] = (i & 1) ? In[q][i / 2].y : In[q][i / 2].x;
            Vc[4 * i + q] = 0.f;
        }
    reduce_scatter_df<4 * G>(Vs, Vc);
    float t, e;
    two_sum(rs, Vs[0], t, e);
    rs = t;
    rc = __fadd_rn(__fadd_rn(rc, Vc[0]), e);
}

// Mixed near field; with NB also the neighbour search of Sec. 2.3 on the same staged sources
// (counts to nb_counts by original index, rows of kNbRowCap slots to nb_rows, longer rows
// queued).  The float32 neighbour filter compares d^2 with (2h)^2 -+ B,
// B = 2^-19 ((W + |d_a|_1)^2 + (2h)^2) + 1e-30, W the tile's largest w (see stage_near_mixed):
// the input and offset roundings, the squares and sums and the roundings of (2h)^2 -+ B stay
// below 16 u F, half of B; inside the band the float64 test (the definition) decides.
template <bool NB>
__global__ void __launch_bounds__(kNearWarps * 32, 2) k_near_mixed(GCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const NearSmem<NB> sm(smem_raw + (size_t)w * NearSmem<NB>::bytes);
    NbGroup g;
    g.nfb = 0;
    for (int s = blockIdx.x * kNearWarps + w; s < c.nsinks; s += gridDim.x * kNearWarps) {
        const int A = c.sinks[s];
        const int fA = c.nfirst[A], nA = c.ncount[A];
        const int nr = c.near_nr[s], nlist = nr + c.near_nn[s];
        // R_A and H_A of the sink cell (float32 offsets from its centre of mass)
        float RA, HA;
        {
            float R2 = 0.f, H = 0.f;
            for (int i = lane; i < nA; i += 32) {
                const float4 pa = c.p32[fA + i];
                R2 = fmaxf(R2, fmaf(pa.z, pa.z, fmaf(pa.y, pa.y, pa.x * pa.x)));
                H = fmaxf(H, c.h32[fA + i]);
            }
            for (int o = 16; o >= 1; o >>= 1) {
                R2 = fmaxf(R2, __shfl_xor_sync(0xffffffffu, R2, o));
                H = fmaxf(H, __shfl_xor_sync(0xffffffffu, H, o));
            }
            RA = sqrtf(R2) * (1.0f + 0x1p-10f);
            HA = H;
        }
        // Up to kSuper groups of eight sink particles share each staged tile: the tile loop is
        // outside the group loop, and each group's lane totals and neighbour counts wait in
        // shared memory while another group runs.  Sinks with more particles take several
        // such passes.
        float wmax = 0.f;
        for (int A0 = 0; A0 < nA; A0 += kSuper * kGroupMixed) {
            const int ng = min(kSuper, (nA - A0 + kGroupMixed - 1) / kGroupMixed);
            for (int gi = 0; gi < ng; ++gi) {
                sm.gacc[gi * 32 + lane] = make_float2(0.f, 0.f);
                if (NB && lane < kGroupMixed) sm.grun[gi * kGroupMixed + lane] = 0;
            }
            __syncwarp();
            for (int64_t t0 = 0;; t0 += kNearTile) {
                const NearTile tl = stage_near_mixed<NB>(c, s, A, nlist, nr, t0, sm, RA, HA, wmax);
                for (int gi = 0; gi < ng; ++gi) {
                    const int a0 = A0 + gi * kGroupMixed;
                    const int na = min(kGroupMixed, nA - a0);
                    if (lane < kGroupMixed) {
                        const int i = min(lane, na - 1);
                        const float4 pa = c.p32[fA + a0 + i];
                        sm.snk[lane] = make_float4(pa.x, pa.y, pa.z, c.h32[fA + a0 + i]);
                    }
                    __syncwarp();
                    if (lane < kGroupMixed) {
                        const float4 u = sm.snk[lane & ~1], v = sm.snk[lane | 1];
                        sm.snk2[lane] = (lane & 1) ? make_float4(u.z, v.z, u.w, v.w) : make_float4(u.x, v.x, u.y, v.y);
                    }
                    if (NB) {
                        g.a0 = fA + a0;
#pragma unroll
                        for (int i = 0; i < kGroupMixed; ++i) g.run[i] = sm.grun[gi * kGroupMixed + i];
                        // neighbour band of each sink particle for this tile (-1: padding slot)
                        if (lane < kGroupMixed) {
                            float2 bd = make_float2(-1.f, -1.f);
                            if (lane < na) {
                                const float4 pa = c.p32[fA + a0 + lane];
                                const float h2f = 2.0f * c.h32[fA + a0 + lane];  // = float32(2 h) exactly
                                const float h2 = h2f * h2f;
                                const float F = wmax + (fabsf(pa.x) + fabsf(pa.y) + fabsf(pa.z));
                                const float B = fmaf(F, F, h2) * 0x1p-19f + 1e-30f;
                                bd = make_float2(h2 - B, h2 + B);
                            }
                            sm.band[lane] = bd;
                        }
                        __syncwarp();
                        if (lane < kGroupMixed / 2) {
                            sm.hi2[lane] = make_float2(sm.band[2 * lane].y, sm.band[2 * lane + 1].y);
                            sm.lo2[lane] = make_float2(sm.band[2 * lane].x, sm.band[2 * lane + 1].x);
                        }
                    }
                    __syncwarp();
                    const float2 st = sm.gacc[gi * 32 + lane];
                    float rs = st.x, rc = st.y;  // compensated total of value lane mod 4 G (= 4 i + q)
                    near_tile<kGroupMixed, NB>(c, sm, tl, na, rs, rc, g);
                    __syncwarp();
                    sm.gacc[gi * 32 + lane] = make_float2(rs, rc);
                    if (NB && lane < kGroupMixed) {
                        int n = g.run[0];
#pragma unroll
                        for (int i = 1; i < kGroupMixed; ++i)
                            if (lane == i) n = g.run[i];
                        sm.grun[gi * kGroupMixed + lane] = n;
                    }
                    __syncwarp();
                }
                if (t0 + kNearTile >= tl.S) break;
            }
            for (int gi = 0; gi < ng; ++gi) {
                const int a0 = A0 + gi * kGroupMixed;
                const int na = min(kGroupMixed, nA - a0);
                const float2 st = sm.gacc[gi * 32 + lane];
                const double tot = __dadd_rn((double)st.x, (double)st.y);  // lane l < 4 na: particle l/4, quantity l%4
                const double q0v = __shfl_sync(0xffffffffu, tot, (4 * lane) & 31);
                const double q1v = __shfl_sync(0xffffffffu, tot, (4 * lane + 1) & 31);
                const double q2v = __shfl_sync(0xffffffffu, tot, (4 * lane + 2) & 31);
                const double q3v = __shfl_sync(0xffffffffu, tot, (4 * lane + 3) & 31);
                if (lane < na) {
                    const int a = fA + a0 + lane;
                    const float4 pa = c.p32[a];
                    const float d[3] = {pa.x, pa.y, pa.z};
                    // the tile loop included the pair of a with itself: zero force, potential
                    // m_a phi(0) = m_a (-1.4) 2 / (h_a + h_a) computed exactly as the loop did
                    const float ha = c.h32[a];
                    const float self_pot = pa.w * (__fdividef(2.0f, ha + ha) * -1.4f);
                    float Cf[20];
#pragma unroll
                    for (int i = 0; i < 20; ++i) Cf[i] = c.coef32[(int64_t)s * 20 + i];
                    float phf, af[3];
                    taylor_eval<float>(Cf, d, phf, af);
                    const int o = c.pidx[a];
                    c.acc[3 * (int64_t)o] = q0v + (double)af[0];
                    c.acc[3 * (int64_t)o + 1] = q1v + (double)af[1];
                    c.acc[3 * (int64_t)o + 2] = q2v + (double)af[2];
                    if (c.pot) c.pot[o] = q3v + (double)phf - (double)self_pot;
                    if (NB) {
                        const int n = sm.grun[gi * kGroupMixed + lane];
                        c.nb_counts[o] = n;
                        if (n > kNbRowCap) {
                            const int q = atomicAdd(&c.status[ST_LONGROWS], 1);
                            if (q < c.cap_long) c.nb_long[q] = make_int2(a, s);
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
    if (NB) {
        int n = g.nfb;
        for (int o = 16; o >= 1; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
        if (lane == 0 && n) atomicAdd(&c.status[ST_NBFALLBACK], n);
    }
}

__global__ void __launch_bounds__(kGWarps * 32) k_near_f64(GCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char *smw = smem_raw + (size_t)w * kNearTileF64 * (5 * sizeof(double) + sizeof(int32_t));
    const double *X = reinterpret_cast<const double *>(smw);
    const int32_t *si = reinterpret_cast<const int32_t *>(X + 5 * kNearTileF64);
    for (int s = blockIdx.x * kGWarps + w; s < c.nsinks; s += gridDim.x * kGWarps) {
        const int A = c.sinks[s];
        const int fA = c.nfirst[A], nA = c.ncount[A];
        const int nr = c.near_nr[s], nlist = nr + c.near_nn[s];
        const int64_t base = (int64_t)s * c.cap_near;
        int64_t S = 0;
        for (int k = lane; k < nlist; k += 32) S += c.ncount[near_entry(c, base, nr, k)];
        for (int o = 16; o >= 1; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
        const double cA[3] = {c.ncom[3 * (int64_t)A], c.ncom[3 * (int64_t)A + 1], c.ncom[3 * (int64_t)A + 2]};
        bool staged_all = false;
        int ns_all = 0;
        for (int a0 = 0; a0 < nA; a0 += kGroupF64) {
            const int na = min(kGroupF64, nA - a0);
            double sx[kGroupF64], sy[kGroupF64], sz[kGroupF64], sh[kGroupF64];
            int sid[kGroupF64];
#pragma unroll
            for (int i = 0; i < kGroupF64; ++i) {
                const int a = fA + a0 + min(i, na - 1);
                sx[i] = c.px[a];
                sy[i] = c.py[a];
                sz[i] = c.pz[a];
                sh[i] = c.ph[a];
                sid[i] = i < na ? a : -1;
            }
            double V[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) V[i] = 0.0;
            for (int64_t t0 = 0; t0 < S; t0 += kNearTileF64) {
                int ns;
                if (staged_all) ns = ns_all;
                else {
                    ns = stage_near<false>(c, s, A, nlist, nr, t0, kNearTileF64, smw);
                    if (S <= kNearTileF64) {
                        staged_all = true;
                        ns_all = ns;
                    }
                }
                for (int q0 = 0; q0 < ns; q0 += 32) {
                    const int j = q0 + lane;
                    if (j >= ns) continue;
                    const double bx = X[j], by = X[kNearTileF64 + j], bz = X[2 * kNearTileF64 + j];
                    const double bm = X[3 * kNearTileF64 + j], bh = X[4 * kNearTileF64 + j];
                    const int bid = si[j];
#pragma unroll
                    for (int i = 0; i < kGroupF64; ++i) {
                        if (i < na && bid != sid[i]) {
                            double ax, ay, az, ph;
                            pair_force<double>(sx[i] - bx, sy[i] - by, sz[i] - bz, sh[i] + bh, bm, ax, ay, az, ph);
                            V[4 * i] += ax;
                            V[4 * i + 1] += ay;
                            V[4 * i + 2] += az;
                            V[4 * i + 3] += ph;
                        }
                    }
                }
                __syncwarp();
            }
            reduce_scatter<16, double>(V);  // lane l: particle (l%16)/4, quantity l%4
            const double tot = V[0];
            double q0v = __shfl_sync(0xffffffffu, tot, (4 * lane) & 15);
            double q1v = __shfl_sync(0xffffffffu, tot, (4 * lane + 1) & 15);
            double q2v = __shfl_sync(0xffffffffu, tot, (4 * lane + 2) & 15);
            double q3v = __shfl_sync(0xffffffffu, tot, (4 * lane + 3) & 15);
            if (lane < na) {
                const int a = fA + a0 + lane;
                double C[20];
#pragma unroll
                for (int i = 0; i < 20; ++i) C[i] = c.coef[(int64_t)s * 20 + i];
                const double d[3] = {c.px[a] - cA[0], c.py[a] - cA[1], c.pz[a] - cA[2]};
                double phf, af[3];
                taylor_eval<double>(C, d, phf, af);
                const int o = c.pidx[a];
                c.acc[3 * (int64_t)o] = q0v + af[0];
                c.acc[3 * (int64_t)o + 1] = q1v + af[1];
                c.acc[3 * (int64_t)o + 2] = q2v + af[2];
                if (c.pot) c.pot[o] = q3v + phf;
            }
        }
        __syncwarp();
    }
}

int sm_count_g() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

// FP64 Taylor coefficients of every sink into t->coef (used by the backward pass).
namespace {

GCtx make_gctx(rcb_tree *t, double *acc, double *pot) {
    GCtx c;
    std::memset(&c, 0, sizeof(c));
    c.nsinks = t->nsinks;
    c.sinks = t->sinks;
    c.near_list = t->near_list;
    c.near_nr = t->near_nr;
    c.near_nn = t->near_nn;
    c.far_list = t->far_list;
    c.far_n = t->far_n;
    c.cap_near = t->cap_near;
    c.cap_far = t->cap_far;
    c.nfirst = t->nfirst;
    c.ncount = t->ncount;
    c.ncom = t->ncom;
    c.nmass = t->nmass;
    c.nQ = t->nQ;
    c.ncomdf = t->ncomdf;
    c.mq32a = t->mq32a;
    c.mq32b = t->mq32b;
    c.nfar = t->nfar;
    c.px = t->px;
    c.py = t->py;
    c.pz = t->pz;
    c.pm = t->pm;
    c.ph = t->ph;
    c.p32 = t->p32;
    c.h32 = t->h32;
    c.pidx = t->pidx;
    c.coef = t->coef;
    c.coef32 = t->coef32;
    c.acc = acc;
    c.pot = pot;
    c.nb_counts = t->nb_count;
    c.nb_rows = t->nb_rows;
    c.nb_long = t->nb_long;
    c.cap_long = (int)t->N;
    c.status = t->d_status;
    return c;
}

}  // namespace

// Far-field coefficients alone, in the tree's precision (the backward pass differentiates the
// Taylor polynomial of the same coefficients the forward evaluated).
int far_coefficients(rcb_tree *t) {
    if (t->nsinks == 0) return RCB_OK;
    const GCtx c = make_gctx(t, nullptr, nullptr);
    const int nsm = sm_count_g();
    const int blocks = std::max(1, std::min((t->nsinks + kGWarps - 1) / kGWarps, nsm * 32));
    if (t->params.precision == RCB_MIXED) {
        k_far<true><<<blocks, kGWarps * 32, 0, t->stream>>>(c); note_launch();
    } else {
        k_far<false><<<blocks, kGWarps * 32, 0, t->stream>>>(c); note_launch();
    }
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

namespace {

template <bool NB>
int launch_near_mixed(rcb_tree *t, const GCtx &c) {
    const int nsm = sm_count_g();
    const size_t smem = (size_t)kNearWarps * NearSmem<NB>::bytes;
    RCB_CUDA_TRY(cudaFuncSetAttribute(k_near_mixed<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nb = std::max(1, std::min((t->nsinks + kNearWarps - 1) / kNearWarps, nsm * 2 * 16));
    k_near_mixed<NB><<<nb, kNearWarps * 32, smem, t->stream>>>(c); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

// Far field and near field; with NB (mixed form only) the near kernel also counts the
// neighbours and writes their slot rows.
int gravity_impl(rcb_tree *t, double *acc, double *pot, bool nb) {
    cudaStream_t st = t->stream;
    const GCtx c = make_gctx(t, acc, pot);
    if (t->nsinks == 0) return RCB_OK;
    const int nsm = sm_count_g();
    const int blocks = std::max(1, std::min((t->nsinks + kGWarps - 1) / kGWarps, nsm * 32));
    const bool mixed = t->params.precision == RCB_MIXED;
    if (mixed) {
        stage_begin(t, SG_FAR);
        k_far<true><<<blocks, kGWarps * 32, 0, st>>>(c); note_launch();
        stage_end(t, SG_FAR);
        stage_begin(t, SG_NEAR);
        const int rc = nb ? launch_near_mixed<true>(t, c) : launch_near_mixed<false>(t, c);
        if (rc) return rc;
    } else {
        stage_begin(t, SG_FAR);
        k_far<false><<<blocks, kGWarps * 32, 0, st>>>(c); note_launch();
        const size_t smem = (size_t)kGWarps * kNearTileF64 * (5 * sizeof(double) + sizeof(int32_t));
        RCB_CUDA_TRY(cudaFuncSetAttribute(k_near_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        stage_end(t, SG_FAR);
        stage_begin(t, SG_NEAR);
        k_near_f64<<<blocks, kGWarps * 32, smem, st>>>(c); note_launch();
    }
    stage_end(t, SG_NEAR);
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

}  // namespace

int gravity(rcb_tree *t, double *acc, double *pot) { return gravity_impl(t, acc, pot, false); }

int gravity_neighbours(rcb_tree *t, double *acc, double *pot) {
    if (t->params.precision != RCB_MIXED || (t->params.flags & RCB_FLAG_MAC_ONLY)) {
        // FP64 form, or MAC-only near lists that do not hold every candidate: two passes
        const int rc = gravity_impl(t, acc, pot, false);
        if (rc) return rc;
        return count_neighbours(t);
    }
    if (t->nb_valid) return gravity_impl(t, acc, pot, false);  // counts and rows are current
    int rc = ensure_nb_rows(t);
    if (rc) return rc;
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_status + ST_NBFALLBACK, 0, 2 * sizeof(int), t->stream));
    rc = gravity_impl(t, acc, pot, true);
    if (rc) return rc;
    stage_begin(t, SG_NB_COUNT);
    rc = scan_neighbour_counts(t);
    if (rc) return rc;
    stage_end(t, SG_NB_COUNT);
    return fetch_neighbour_total(t);
}

}  // namespace rcb
