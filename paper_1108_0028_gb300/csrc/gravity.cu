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
    const double *px, *py, *pz, *pm, *ph;
    const float4 *p32;
    const float *h32;
    const int32_t *pidx;
    double *coef;
    float *coef32;
    double *acc, *pot;
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
            float C[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) C[i] = 0.f;
            const float2 a0 = c.ncomdf[3 * (int64_t)A], a1 = c.ncomdf[3 * (int64_t)A + 1], a2 = c.ncomdf[3 * (int64_t)A + 2];
            for (int k = lane; k < nf; k += 32) {
                const int B = c.far_list[fb + k];
                const float2 b0 = c.ncomdf[3 * (int64_t)B], b1 = c.ncomdf[3 * (int64_t)B + 1], b2 = c.ncomdf[3 * (int64_t)B + 2];
                const float x[3] = {(a0.x - b0.x) + (a0.y - b0.y), (a1.x - b1.x) + (a1.y - b1.y),
                                    (a2.x - b2.x) + (a2.y - b2.y)};
                const float4 qa = c.mq32a[B], qb = c.mq32b[B];
                const float Q6[6] = {qa.y, qa.z, qa.w, qb.x, qb.y, qb.z};
                far_source<float>(x, qa.x, Q6, C);
            }
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
constexpr size_t kNearWarpBytes = kNearTile * (sizeof(float4) + sizeof(float) + sizeof(int32_t)) +
                                  kGroupMixed * (sizeof(float4) + sizeof(int32_t));

// Stage sources [t0, t0 + kNearTile) of the sink's near cells, one lane per cell: float32
// offsets from the sink's centre of mass (double-float difference of the two centres of mass
// plus the particle's float32 offset from its own cell's centre), mass, h, sorted index.
__device__ int stage_near_mixed(const GCtx &c, int s, int A, int nlist, int nr, int64_t t0, float4 *src, float *hs,
                                int32_t *si) {
    const int lane = threadIdx.x & 31;
    const int64_t base = (int64_t)s * c.cap_near;
    const float2 a0 = c.ncomdf[3 * (int64_t)A], a1 = c.ncomdf[3 * (int64_t)A + 1], a2 = c.ncomdf[3 * (int64_t)A + 2];
    int64_t pos = 0;
    for (int k0 = 0; k0 < nlist && pos < t0 + kNearTile; k0 += 32) {
        const int k = k0 + lane;
        int f = 0, n = 0;
        float ox = 0.f, oy = 0.f, oz = 0.f;
        if (k < nlist) {
            const int B = near_entry(c, base, nr, k);
            f = c.nfirst[B];
            n = c.ncount[B];
            const float2 b0 = c.ncomdf[3 * (int64_t)B], b1 = c.ncomdf[3 * (int64_t)B + 1], b2 = c.ncomdf[3 * (int64_t)B + 2];
            ox = (b0.x - a0.x) + (b0.y - a0.y);
            oy = (b1.x - a1.x) + (b1.y - a1.y);
            oz = (b2.x - a2.x) + (b2.y - a2.y);
        }
        int incl = n;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int64_t my0 = pos + incl - n;
        for (int q = 0; q < n; ++q) {
            const int64_t slot = my0 + q - t0;
            if (slot >= 0 && slot < kNearTile) {
                const float4 pb = c.p32[f + q];
                src[slot] = make_float4(ox + pb.x, oy + pb.y, oz + pb.z, pb.w);
                hs[slot] = c.h32[f + q];
                si[slot] = f + q;
            }
        }
        pos += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    const int64_t left = pos - t0;
    return (int)(left < kNearTile ? left : kNearTile);
}

__global__ void __launch_bounds__(kNearWarps * 32, 2) k_near_mixed(GCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char *smw = smem_raw + (size_t)w * kNearWarpBytes;
    float4 *src = reinterpret_cast<float4 *>(smw);
    float *hs = reinterpret_cast<float *>(src + kNearTile);
    int32_t *si = reinterpret_cast<int32_t *>(hs + kNearTile);
    float4 *snk = reinterpret_cast<float4 *>(si + kNearTile);  // (d_a, h_a) of the current group
    int32_t *sid = reinterpret_cast<int32_t *>(snk + kGroupMixed);
    for (int s = blockIdx.x * kNearWarps + w; s < c.nsinks; s += gridDim.x * kNearWarps) {
        const int A = c.sinks[s];
        const int fA = c.nfirst[A], nA = c.ncount[A];
        const int nr = c.near_nr[s], nlist = nr + c.near_nn[s];
        const int64_t base = (int64_t)s * c.cap_near;
        int64_t S = 0;
        for (int k = lane; k < nlist; k += 32) S += c.ncount[near_entry(c, base, nr, k)];
        for (int o = 16; o >= 1; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
        int ns_once = -1;  // staged tile count when all sources fit one tile
        for (int a0 = 0; a0 < nA; a0 += kGroupMixed) {
            const int na = min(kGroupMixed, nA - a0);
            if (lane < kGroupMixed) {
                const int i = min(lane, na - 1);
                const float4 pa = c.p32[fA + a0 + i];
                snk[lane] = make_float4(pa.x, pa.y, pa.z, c.h32[fA + a0 + i]);
                sid[lane] = lane < na ? fA + a0 + i : -1;
            }
            __syncwarp();
            float rs = 0.f, rc = 0.f;  // compensated total of value `lane` (= 4 i + q)
            for (int64_t t0 = 0; t0 < S; t0 += kNearTile) {
                int ns = ns_once;
                if (ns < 0) {
                    ns = stage_near_mixed(c, s, A, nlist, nr, t0, src, hs, si);
                    if (S <= kNearTile) ns_once = ns;
                }
                float In[4][kGroupMixed];
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int i = 0; i < kGroupMixed; ++i) In[q][i] = 0.f;
                for (int q0 = 0; q0 < ns; q0 += 32) {
                    const int j = q0 + lane;
                    float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
                    float hb = 1.f;
                    int bid = -2;
                    if (j < ns) {
                        b = src[j];
                        hb = hs[j];
                        bid = si[j];
                    }
#pragma unroll
                    for (int i = 0; i < kGroupMixed; ++i) {
                        if (i < na) {
                            const float4 sa = snk[i];
                            const float mb = bid == sid[i] ? 0.f : b.w;
                            float ax, ay, az, ph;
                            pair_force<float>(sa.x - b.x, sa.y - b.y, sa.z - b.z, sa.w + hb, mb, ax, ay, az, ph);
                            In[0][i] += ax;
                            In[1][i] += ay;
                            In[2][i] += az;
                            In[3][i] += ph;
                        }
                    }
                }
                // fold this tile: compensated reduce-scatter across lanes, then into (rs, rc)
                float Vs[32], Vc[32];
#pragma unroll
                for (int i = 0; i < kGroupMixed; ++i)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        Vs[4 * i + q] = In[q][i];
                        Vc[4 * i + q] = 0.f;
                    }
                reduce_scatter_df<32>(Vs, Vc);
                float t, e;
                two_sum(rs, Vs[0], t, e);
                rs = t;
                rc = __fadd_rn(__fadd_rn(rc, Vc[0]), e);
                __syncwarp();
            }
            const double tot = __dadd_rn((double)rs, (double)rc);  // lane l: particle l/4, quantity l%4
            const double q0v = __shfl_sync(0xffffffffu, tot, (4 * lane) & 31);
            const double q1v = __shfl_sync(0xffffffffu, tot, (4 * lane + 1) & 31);
            const double q2v = __shfl_sync(0xffffffffu, tot, (4 * lane + 2) & 31);
            const double q3v = __shfl_sync(0xffffffffu, tot, (4 * lane + 3) & 31);
            if (lane < na) {
                const int a = fA + a0 + lane;
                const float4 pa = c.p32[a];
                const float d[3] = {pa.x, pa.y, pa.z};
                float Cf[20];
#pragma unroll
                for (int i = 0; i < 20; ++i) Cf[i] = c.coef32[(int64_t)s * 20 + i];
                float phf, af[3];
                taylor_eval<float>(Cf, d, phf, af);
                const int o = c.pidx[a];
                c.acc[3 * (int64_t)o] = q0v + (double)af[0];
                c.acc[3 * (int64_t)o + 1] = q1v + (double)af[1];
                c.acc[3 * (int64_t)o + 2] = q2v + (double)af[2];
                if (c.pot) c.pot[o] = q3v + (double)phf;
            }
            __syncwarp();
        }
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
int far_coefficients_fp64(rcb_tree *t) {
    GCtx c;
    std::memset(&c, 0, sizeof(c));
    c.nsinks = t->nsinks;
    c.sinks = t->sinks;
    c.far_list = t->far_list;
    c.far_n = t->far_n;
    c.cap_far = t->cap_far;
    c.ncom = t->ncom;
    c.nmass = t->nmass;
    c.nQ = t->nQ;
    c.coef = t->coef;
    if (t->nsinks == 0) return RCB_OK;
    const int nsm = sm_count_g();
    const int blocks = std::max(1, std::min((t->nsinks + kGWarps - 1) / kGWarps, nsm * 32));
    k_far<false><<<blocks, kGWarps * 32, 0, t->stream>>>(c); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

int gravity(rcb_tree *t, double *acc, double *pot) {
    cudaStream_t st = t->stream;
    GCtx c;
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
    if (t->nsinks == 0) return RCB_OK;
    const int nsm = sm_count_g();
    const int blocks = std::max(1, std::min((t->nsinks + kGWarps - 1) / kGWarps, nsm * 32));
    const bool mixed = t->params.precision == RCB_MIXED;
    if (mixed) {
        stage_begin(t, SG_FAR);
        k_far<true><<<blocks, kGWarps * 32, 0, st>>>(c); note_launch();
        const size_t smem = (size_t)kNearWarps * kNearWarpBytes;
        RCB_CUDA_TRY(cudaFuncSetAttribute(k_near_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        stage_end(t, SG_FAR);
        stage_begin(t, SG_NEAR);
        const int nb = std::max(1, std::min((t->nsinks + kNearWarps - 1) / kNearWarps, nsm * 2 * 16));
        k_near_mixed<<<nb, kNearWarps * 32, smem, st>>>(c); note_launch();
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

}  // namespace rcb
