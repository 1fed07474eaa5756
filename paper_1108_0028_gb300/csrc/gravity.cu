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
#include "nb_rows.cuh"
#include "rcb_internal.cuh"

namespace rcb {
namespace {

constexpr int kGWarps = 4;
constexpr int kGroupF64 = 4;
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
    // neighbour rows fused into the mixed near field
    int64_t *nb_counts;  // [N] by original index
    RowOut ro;
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
            // the list entries of a round are loaded one round ahead (their latency overlaps the
            // arithmetic), the nodes' records at the start of their round
            int k = lane;
            int B[2] = {k < nf ? c.far_list[fb + k] : -1, k + 32 < nf ? c.far_list[fb + k + 32] : -1};
            while (k < nf) {
                float4 q[2][4];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (B[u] >= 0) {
                        const float4 *r = c.nfar + 4 * (int64_t)B[u];
                        q[u][0] = r[0];
                        q[u][1] = r[1];
                        q[u][2] = r[2];
                        q[u][3] = r[3];
                    } else {
                        // no node: zero mass and quadrupole (its offset is set to (1, 0, 0) below)
                        q[u][0] = make_float4(0.f, 0.f, 0.f, 0.f);
                        q[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                        q[u][2] = make_float4(0.f, 0.f, 0.f, 0.f);
                        q[u][3] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                const int kn = k + 64;
                B[0] = kn < nf ? c.far_list[fb + kn] : -1;
                B[1] = kn + 32 < nf ? c.far_list[fb + kn + 32] : -1;
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

// Stage sources [t0, t0 + tile) of the concatenated near cells (float64 near field).
__device__ int stage_near(const GCtx &c, int s, int A, int nlist, int nr, int64_t t0, int tile, void *smw) {
    const int lane = threadIdx.x & 31;
    const int64_t base = (int64_t)s * c.cap_near;
    int64_t pos = 0;
    int staged = 0;
    for (int k0 = 0; k0 < nlist; k0 += 32) {
        const int k = k0 + lane;
        int f = 0, n = 0;
        if (k < nlist) {
            const int B = near_entry(c, base, nr, k);
            f = c.nfirst[B];
            n = c.ncount[B];
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
            const int64_t lo = c0 > t0 ? c0 : t0;
            const int64_t hi = c0 + cn < t0 + tile ? c0 + cn : t0 + tile;
            for (int64_t q = lo + lane; q < hi; q += 32) {
                const int b = cf + (int)(q - c0);
                const int slot = (int)(q - t0);
                double *X = reinterpret_cast<double *>(smw);
                X[slot] = c.px[b];
                X[kNearTileF64 + slot] = c.py[b];
                X[2 * kNearTileF64 + slot] = c.pz[b];
                X[3 * kNearTileF64 + slot] = c.pm[b];
                X[4 * kNearTileF64 + slot] = c.ph[b];
                reinterpret_cast<int32_t *>(X + 5 * kNearTileF64)[slot] = b;
            }
            if (hi > lo) staged = max(staged, (int)(hi - t0));
        }
        pos += group_total;
        if (pos >= t0 + tile) break;
    }
    __syncwarp();
    return staged;
}

// ------------------------------------------------------------------------------ mixed near field
// One warp per sink.  The sources (the particles of the sink's near cells) are staged once per
// tile in shared memory; the warp's lanes then take (sink particle i, source stream j) pairs:
// with P sink particles in the pass, S = 32 / P streams, lane l holds particle i = l mod P and
// walks the source pairs k = j, j + S, ... (j = l / P).  Every lane evaluates two sources at once
// with paired float32 instructions (each half rounds as the scalar operation would) and keeps
// its own totals, so nothing crosses lanes until the sink is finished.  Sources are stored by
// pairs, positions and masses negated: (-x_2k, -x_2k+1, -y_2k, -y_2k+1), (-z.., -m..),
// (h.., original indices..) and, for the neighbour test, the sorted indices, so that every paired
// operand arrives from one shared-memory load.
constexpr int kNearWarps = 8;   // warps per block
constexpr int kNearMinBlocks = 2;
constexpr int kNearTile = 256;  // staged source slots per warp (even)
constexpr int kFoldIters = 16;  // source pairs summed in float32 before a compensated fold

// Shared memory of one warp: per source pair k, A[k], B[k], C[k] = (h_2k, h_2k+1, original
// indices); with the neighbour rows (NB) also D[k] = (sorted indices, unused), the row buffer
// (nb_rows.cuh) and per-lane counts; then the cell table of the tile being staged.
template <bool NB>
struct NearSmem {
    static constexpr int H = kNearTile / 2;  // source pairs per tile
    static constexpr size_t bytes = (size_t)H * (NB ? 4 : 3) * sizeof(float4) +
                                    (NB ? kRowBuf * sizeof(int32_t) + 64 * sizeof(int) : 0) + 32 * sizeof(float4);
    float4 *P;      // A[H], B[H], C[H], D[H] (NB)
    int32_t *rows;  // NB: row buffer
    int *rowcnt;    // NB: [32] per-lane counts when a pass is handed over, then [32] dummy words
    float4 *T;      // [32] cell table: offset of the cell's centre of mass, first particle - first slot
    __device__ NearSmem(unsigned char *p) {
        P = reinterpret_cast<float4 *>(p);
        rows = reinterpret_cast<int32_t *>(P + (NB ? 4 : 3) * H);
        rowcnt = rows + (NB ? kRowBuf : 0);
        T = reinterpret_cast<float4 *>(rowcnt + (NB ? 64 : 0));
    }
    __device__ __forceinline__ float4 a(int k) const { return P[k]; }
    __device__ __forceinline__ float4 b(int k) const { return P[k + H]; }
    __device__ __forceinline__ float4 c(int k) const { return P[k + 2 * H]; }
    __device__ __forceinline__ const int4 *D() const { return reinterpret_cast<const int4 *>(P + 3 * H); }
    // store source pair k: offsets v (from the sink's centre of mass), masses, h, original and
    // sorted indices of both sources; the offsets and masses negated
    __device__ __forceinline__ void put(int k, float3 v0, float3 v1, float m0, float m1, float h0, float h1, int o0,
                                        int o1, int i0, int i1) const {
        P[k] = make_float4(-v0.x, -v1.x, -v0.y, -v1.y);
        P[k + H] = make_float4(-v0.z, -v1.z, -m0, -m1);
        P[k + 2 * H] = make_float4(h0, h1, __int_as_float(o0), __int_as_float(o1));
        if (NB) *reinterpret_cast<int2 *>(P + 3 * H + k) = make_int2(i0, i1);
    }
};

// Where the next tile starts: list entry k0 of the sink's near list (the reachable cells come
// first, then the others), of whose particles the first off0 are already staged.
struct NearCursor {
    int k0, off0;
};

// One staged tile: close source pairs in pair slots [0, nclose / 2), of which the first ncc / 2
// come from neighbour candidates (reachable cells), far pairs in [H - nfar / 2, H); the counts
// are in sources (even).
struct NearTile {
    int nclose, ncc, nfar;
    bool last;  // no sources beyond this tile
};

// The cells of the next tile, loaded while the current tile is computed: the near-list entries
// wk + lane and wk + 32 + lane (bw0, bw1; -1 past the list) and, as loaded, first particle, count
// and double-float centre of mass of cell bw0 (the cell of entry wk + lane).  The loaded values
// are first used by the next staging, so that their latency overlaps the pair loops.
struct NearAhead {
    int wk, bw0, bw1;
    int f, n;
    float2 b0, b1, b2;
};

// Load the near-list window from entry k0 and the descriptors of the cells of its first half.
__device__ __forceinline__ void near_ahead_load(const GCtx &c, int64_t base, int nr, int nlist, int k0, int B0,
                                                bool have_b0, NearAhead &ah) {
    const int lane = threadIdx.x & 31;
    const int B = have_b0 ? B0 : (k0 + lane < nlist ? near_entry(c, base, nr, k0 + lane) : -1);
    ah.wk = k0;
    ah.bw0 = B;
    ah.bw1 = k0 + 32 + lane < nlist ? near_entry(c, base, nr, k0 + 32 + lane) : -1;
    ah.f = 0;
    ah.n = 0;
    ah.b0 = ah.b1 = ah.b2 = make_float2(0.f, 0.f);
    if (B >= 0) {
        ah.f = c.nfirst[B];
        ah.n = c.ncount[B];
        ah.b0 = c.ncomdf[3 * (int64_t)B];
        ah.b1 = c.ncomdf[3 * (int64_t)B + 1];
        ah.b2 = c.ncomdf[3 * (int64_t)B + 2];
    }
}

// Far test of one source at offset v with smoothing length hb (see stage_near_mixed).
template <bool NB>
__device__ __forceinline__ bool near_is_far(float3 v, float hb, float3 blo, float3 bhi, float HA) {
    const float gx = fmaxf(fmaxf(blo.x - v.x, v.x - bhi.x), 0.f), gy = fmaxf(fmaxf(blo.y - v.y, v.y - bhi.y), 0.f),
                gz = fmaxf(fmaxf(blo.z - v.z, v.z - bhi.z), 0.f);
    const float g2 = fmaf(gz, gz, fmaf(gy, gy, gx * gx));
    const float X = (NB ? fmaxf(HA + hb, HA + HA) : HA + hb) * (1.0f + 0x1p-10f);
    return g2 > X * X;
}

// Stage the next tile of sink s (cell A, sorted particles [fA, fA + nA), this pass the P
// particles from a0).  A tile is one batch of up to 32 near cells, all from the same part of the
// list (reachable or not), as many whole cells as fit in kNearTile slots (part of one cell if a
// single cell is larger).  The cells' descriptors (first particle, count, centre of mass) arrive
// with ah, loaded during the previous tile's pair loops; once the batch is known, the next tile's
// are loaded the same way.  The batch's cells go to a table in shared memory (offset of the
// centre of mass, first particle minus first slot).  Each lane then takes the slots 2r and
// 2r + 1 of pair slots r = lane + 32 u: it finds their cells from the cells' start bits, issues
// the gathers of half its pairs before using any of them (a tile costs two rounds of memory
// latency), forms each source's float32 offset from the sink's centre of mass and stores the
// pair, far pairs (both sources far; a missing second source counts as far and is padded with a
// massless source far away) from the back of the tile and the others from the front.  The cell
// offset o is the double-float difference of the two centres of mass: it differs from the float64
// difference by at most 2u |dCOM| + 3 2^-48 (|COM_A|_1 + |COM_B|_1) per component (u = 2^-24).
// With NB, wmax gets a bound on the tile's largest w = |o|_1 + |d_b|_1 + 2^-20 (|COM_A|_1 +
// |COM_B|_1) over candidate sources: the largest of the cell terms plus the largest |d_b|_1.  The
// last cell term makes the representation error's share of the d^2 error at most 6 2^-28 F, well
// inside the neighbour band.
//
// Far sources: with H_A the largest h_a of the sink's particles and the box [blo, bhi] of their
// float32 offsets d_a, a source b whose distance g from the box exceeds X_b (1 + 2^-10) has
// r_ab >= g > X_b for every sink particle a.  X_b = H_A + h_b puts all its pairs on the
// Newtonian branch of Eq. 10 (q >= 2); with NB, X_b = max(H_A + h_b, 2 H_A) also keeps it out of
// every sink particle's neighbour sphere (r < 2 h_a).  The 2^-10 margin is far above the float32
// rounding of the test, of q and of the neighbour filter.  A close pair may hold one far source:
// the close loop evaluates it on the Newtonian branch and never counts it as a neighbour.
template <bool NB>
__device__ NearTile stage_near_mixed(const GCtx &c, int s, int A, int fA, int a0, int P, int nlist, int nr,
                                     NearCursor &cur, NearAhead &ah, const NearSmem<NB> &sm, float3 blo,
                                     float3 bhi, float HA, float &wmax) {
    constexpr int kCap = kNearTile;
    constexpr int H = NearSmem<NB>::H;
    constexpr int kR = kNearTile / 64;  // rounds of 32 pair slots
    constexpr int kH = kR / 2;          // rounds per half
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)s * c.cap_near;
    if (cur.k0 >= nlist) {
        __syncwarp();
        return NearTile{0, 0, 0, true};
    }
    const int k0 = cur.k0, kend = k0 < nr ? nr : nlist;  // the tile stays within one part
    const bool cand = k0 < nr;
    const int k = k0 + lane;  // = ah.wk + lane
    int f = 0, n = 0;
    float ox = 0.f, oy = 0.f, oz = 0.f, ow = 0.f;
    if (k < kend) {
        const float2 a0f = c.ncomdf[3 * (int64_t)A], a1f = c.ncomdf[3 * (int64_t)A + 1],
                     a2f = c.ncomdf[3 * (int64_t)A + 2];
        f = ah.f;
        n = ah.n;
        const float2 b0 = ah.b0, b1 = ah.b1, b2 = ah.b2;
        ox = (b0.x - a0f.x) + (b0.y - a0f.y);
        oy = (b1.x - a1f.x) + (b1.y - a1f.y);
        oz = (b2.x - a2f.x) + (b2.y - a2f.y);
        if (NB) ow = 0x1p-20f * ((fabsf(a0f.x) + fabsf(a1f.x) + fabsf(a2f.x)) + (fabsf(b0.x) + fabsf(b1.x) + fabsf(b2.x)));
        if (lane == 0) {  // the part of the first cell not staged yet
            f += cur.off0;
            n -= cur.off0;
        }
    }
    int excl = warp_excl_scan(n);
    // whole cells that fit; if none, the first cell's next kCap particles
    const unsigned fit = __ballot_sync(0xffffffffu, k < kend && excl + n <= kCap);
    const int nfit = __popc(fit);  // cells fit from lane 0 on: fit = 2^nfit - 1
    int nslots;
    if (nfit > 0) {
        nslots = __shfl_sync(0xffffffffu, excl + n, nfit - 1);
        if (lane >= nfit) n = 0;
        cur.k0 = k0 + nfit;
        cur.off0 = 0;
    } else {
        nslots = kCap;
        if (lane > 0) n = 0;
        if (lane == 0) n = kCap;
        cur.off0 += kCap;
    }
    {  // the next tile's cells: entry cur.k0 + lane lies in the window (cur.k0 - k0 <= 32)
        const int d = cur.k0 - k0 + lane;
        const int e0 = __shfl_sync(0xffffffffu, ah.bw0, d & 31), e1 = __shfl_sync(0xffffffffu, ah.bw1, d & 31);
        near_ahead_load(c, base, nr, nlist, cur.k0, d < 32 ? e0 : e1, true, ah);
    }
    excl = warp_excl_scan(n);
    float wc = 0.f;  // NB: the cell term of w
    if (n > 0) {
        sm.T[lane] = make_float4(ox, oy, oz, __int_as_float(f - excl));
        if (NB) wc = ((fabsf(ox) + fabsf(oy)) + fabsf(oz)) + ow;
    }
    __syncwarp();
    float wl = 0.f;
    int nclose = 0, nfar = 0;  // pair slots
#pragma unroll 1
    for (int hh = 0; hh < 2; ++hh) {
        int cc0[kH], cc1[kH];
        float4 pb0[kH], pb1[kH];
        float hb0[kH], hb1[kH];
        int ob0[kH], ob1[kH], ib0[kH], ib1[kH];
#pragma unroll
        for (int u = 0; u < kH; ++u) {
            const int w0 = 64 * (hh * kH + u), sl = w0 + 2 * lane;  // the round's and the lane's first slot
            // the cells starting inside [w0, w0 + 64) as bits, and the number starting before it
            const int st = excl - w0;
            const bool in = n > 0 && st >= 0 && st < 64;
            const unsigned lo = __reduce_or_sync(0xffffffffu, in && st < 32 ? 1u << (st & 31) : 0u);
            const unsigned hi = __reduce_or_sync(0xffffffffu, in && st >= 32 ? 1u << (st & 31) : 0u);
            const int before = __popc(__ballot_sync(0xffffffffu, n > 0 && st < 0));
            const unsigned long long starts = ((unsigned long long)hi << 32) | lo;
            const int bit = 2 * lane;
            cc0[u] = min(31, max(0, before + __popcll(starts & ((2ull << bit) - 1ull)) - 1));
            cc1[u] = min(31, cc0[u] + (int)((starts >> (bit + 1)) & 1ull));
            pb0[u] = pb1[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            hb0[u] = hb1[u] = 1.f;
            ob0[u] = ob1[u] = ib0[u] = ib1[u] = -1;
            if (sl < nslots) {
                const int b = __float_as_int(sm.T[cc0[u]].w) + sl;
                pb0[u] = c.p32[b];
                hb0[u] = c.h32[b];
                if (NB) {
                    ib0[u] = b;
                    ob0[u] = c.pidx[b];
                }
            }
            if (sl + 1 < nslots) {
                const int b = __float_as_int(sm.T[cc1[u]].w) + sl + 1;
                pb1[u] = c.p32[b];
                hb1[u] = c.h32[b];
                if (NB) {
                    ib1[u] = b;
                    ob1[u] = c.pidx[b];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kH; ++u) {
            const int sl = 64 * (hh * kH + u) + 2 * lane;
            const bool act = sl < nslots, two = sl + 1 < nslots;
            const float4 t0 = sm.T[cc0[u]], t1 = sm.T[cc1[u]];
            const float3 v0 = make_float3(t0.x + pb0[u].x, t0.y + pb0[u].y, t0.z + pb0[u].z);
            float3 v1 = make_float3(t1.x + pb1[u].x, t1.y + pb1[u].y, t1.z + pb1[u].z);
            if (!two) v1 = make_float3(1e18f, 1e18f, 1e18f);
            const bool far = near_is_far<NB>(v0, hb0[u], blo, bhi, HA) &&
                             (!two || near_is_far<NB>(v1, hb1[u], blo, bhi, HA));
            const unsigned mc = __ballot_sync(0xffffffffu, act && !far);
            const unsigned mf = __ballot_sync(0xffffffffu, act && far);
            if (act) {
                const int at = far ? H - 1 - (nfar + __popc(mf & lt)) : nclose + __popc(mc & lt);
                sm.put(at, v0, v1, pb0[u].w, two ? pb1[u].w : 0.f, hb0[u], hb1[u], ob0[u], ob1[u], ib0[u], ib1[u]);
                if (NB && cand)
                    wl = fmaxf(wl, fmaxf((fabsf(pb0[u].x) + fabsf(pb0[u].y)) + fabsf(pb0[u].z),
                                         (fabsf(pb1[u].x) + fabsf(pb1[u].y)) + fabsf(pb1[u].z)));
            }
            nclose += __popc(mc);
            nfar += __popc(mf);
        }
    }
    if (NB) {
        for (int o = 16; o >= 1; o >>= 1) {
            wl = fmaxf(wl, __shfl_xor_sync(0xffffffffu, wl, o));
            wc = fmaxf(wc, __shfl_xor_sync(0xffffffffu, wc, o));
        }
        wmax = wc + wl;
    }
    __syncwarp();
    return NearTile{2 * nclose, cand ? 2 * nclose : 0, 2 * nfar, cur.k0 >= nlist};
}

// Lane state of the mixed near field: the lane's sink particle (float32 offset from the sink's
// centre of mass and h, each twice), its neighbour band, and its sums.  In[q] collects quantity q
// (a_x, a_y, a_z, phi) over two sources at a time; (sum, comp) is the compensated total.
struct NearLane {
    float2 xa, ya, za, ha;
    float h2, B;   // (2 h_a)^2 and the half width of the neighbour band
    float2 In[4];
    float sum[4], comp[4];
    int32_t *wp;     // NB: where the lane's next row entry goes (entry e of its part at part[e stride])
    int32_t *dummy;  // NB: the lane's scratch word for entries not kept
    int nsub, capsub, stride;
    int nfb;  // float64 neighbour decisions taken
};

__device__ __forceinline__ void near_fold(NearLane &L) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        comp_add(L.sum[q], L.comp[q], __fadd_rn(L.In[q].x, L.In[q].y));
        L.In[q] = make_float2(0.f, 0.f);
    }
}

__device__ __forceinline__ float2 near_r2(const NearLane &L, const float4 a, const float4 b, float2 &dx, float2 &dy,
                                         float2 &dz) {
    dx = __fadd2_rn(L.xa, make_float2(a.x, a.y));
    dy = __fadd2_rn(L.ya, make_float2(a.z, a.w));
    dz = __fadd2_rn(L.za, make_float2(b.x, b.y));
    return __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
}

// Far sources: every pair outside the kernel support, Newtonian only (r > 0 always).
__device__ __forceinline__ void near_pair_newton(NearLane &L, const float4 a, const float4 b) {
    float2 dx, dy, dz;
    const float2 r2 = near_r2(L, a, b, dx, dy, dz);
    const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 nm = make_float2(b.z, b.w);                                      // -m_b
    const float2 nw = __fmul2_rn(nm, __fmul2_rn(__fmul2_rn(rinv, rinv), rinv));  // -m_b / r^3
    L.In[0] = __ffma2_rn(nw, dx, L.In[0]);
    L.In[1] = __ffma2_rn(nw, dy, L.In[1]);
    L.In[2] = __ffma2_rn(nw, dz, L.In[2]);
    L.In[3] = __ffma2_rn(nm, rinv, L.In[3]);  // m_b phi, phi = -1/r
}

// Close sources: the full kernel-softened pair of Eq. 10 with its potential (branch-free, the
// branch of each half selected by its q); -phi is evaluated, so that the stored -m_b multiplies
// it.  Returns r^2 of both pairs.  The pair of a particle with itself has r = 0: zero force,
// potential m_a phi(0) (removed in the epilogue).
__device__ __forceinline__ float2 near_pair_close(NearLane &L, const float4 a, const float4 b, const float4 cc,
                                                  bool ok = true) {
    float2 dx, dy, dz;
    const float2 r2 = near_r2(L, a, b, dx, dy, dz);
    const float2 rinv = make_float2(rsqrtf(fmaxf(r2.x, 1e-30f)), rsqrtf(fmaxf(r2.y, 1e-30f)));
    const float2 r = __fmul2_rn(r2, rinv);
    const float2 hsum = __fadd2_rn(L.ha, make_float2(cc.x, cc.y));
    const float2 hinv = make_float2(__fdividef(2.0f, hsum.x), __fdividef(2.0f, hsum.y));
    const float2 q = __fmul2_rn(r, hinv);
    const float2 q2 = __fmul2_rn(q, q);
    const float2 rinv3 = __fmul2_rn(__fmul2_rn(rinv, rinv), rinv);
    const float2 h3 = __fmul2_rn(__fmul2_rn(hinv, hinv), hinv);
    // S/r:  q < 1:      h^-3 (4/3 - 6/5 q^2 + 1/2 q^3)
    //       1 <= q < 2: h^-3 (8/3 - 3 q + 6/5 q^2 - 1/6 q^3) - 1/(15 r^3)
    const float2 s1 = __fmul2_rn(h3, __ffma2_rn(q2, __ffma2_rn(make_float2(0.5f, 0.5f), q, make_float2(-1.2f, -1.2f)),
                                                make_float2(4.0f / 3.0f, 4.0f / 3.0f)));
    const float2 s2 = __ffma2_rn(
        h3,
        __ffma2_rn(q,
                   __ffma2_rn(q, __ffma2_rn(make_float2(-1.0f / 6.0f, -1.0f / 6.0f), q, make_float2(1.2f, 1.2f)),
                              make_float2(-3.0f, -3.0f)),
                   make_float2(8.0f / 3.0f, 8.0f / 3.0f)),
        __fmul2_rn(make_float2(-1.0f / 15.0f, -1.0f / 15.0f), rinv3));
    // -phi: q < 1:      h^-1 (7/5 - 2/3 q^2 + 3/10 q^4 - 1/10 q^5)
    //       1 <= q < 2: h^-1 (8/5 - 4/3 q^2 + q^3 - 3/10 q^4 + 1/30 q^5) - 1/(15 r)
    const float2 p1 = __fmul2_rn(
        hinv, __ffma2_rn(q2,
                         __ffma2_rn(q2, __ffma2_rn(make_float2(-0.1f, -0.1f), q, make_float2(0.3f, 0.3f)),
                                    make_float2(-2.0f / 3.0f, -2.0f / 3.0f)),
                         make_float2(1.4f, 1.4f)));
    const float2 p2 = __ffma2_rn(
        hinv,
        __ffma2_rn(q2,
                   __ffma2_rn(q,
                              __ffma2_rn(q, __ffma2_rn(make_float2(1.0f / 30.0f, 1.0f / 30.0f), q, make_float2(-0.3f, -0.3f)),
                                         make_float2(1.0f, 1.0f)),
                              make_float2(-4.0f / 3.0f, -4.0f / 3.0f)),
                   make_float2(1.6f, 1.6f)),
        __fmul2_rn(make_float2(-1.0f / 15.0f, -1.0f / 15.0f), rinv));
    const float2 sr = make_float2(q.x < 1.0f ? s1.x : (q.x < 2.0f ? s2.x : rinv3.x),
                                  q.y < 1.0f ? s1.y : (q.y < 2.0f ? s2.y : rinv3.y));
    const float2 np = make_float2(q.x < 1.0f ? p1.x : (q.x < 2.0f ? p2.x : rinv.x),
                                  q.y < 1.0f ? p1.y : (q.y < 2.0f ? p2.y : rinv.y));
    const float2 nm = ok ? make_float2(b.z, b.w) : make_float2(0.f, 0.f);  // -m_b
    const float2 nw = __fmul2_rn(nm, sr);
    L.In[0] = __ffma2_rn(nw, dx, L.In[0]);
    L.In[1] = __ffma2_rn(nw, dy, L.In[1]);
    L.In[2] = __ffma2_rn(nw, dz, L.In[2]);
    L.In[3] = __ffma2_rn(nm, np, L.In[3]);  // (-m_b)(-phi)
    return r2;
}

// The float64 definition of the neighbour test (b a sorted index, -1 for a padding slot).
__device__ __noinline__ int nb_settle(const double *px, const double *py, const double *pz, const double *ph, int a,
                                      int b) {
    if (b == a || b < 0) return 0;
    const double s2 = __dmul_rn(2.0, ph[a]);
    return dist2_rn(px[a], py[a], pz[a], px[b], py[b], pz[b]) < __dmul_rn(s2, s2) ? 1 : 0;
}

// Append original index o to the lane's part of its row (entries past its capacity are counted
// only: the row is then recomputed by the direct fill).
__device__ __forceinline__ void sub_push(NearLane &L, bool nb, int o) {
    const bool st = nb && L.nsub < L.capsub;
    *(st ? L.wp : L.dummy) = o;  // branch-free: a store to the lane's dummy word when not kept
    L.wp += st ? L.stride : 0;
    L.nsub += nb ? 1 : 0;
}

// The float64 decisions of one block of loop steps (pairs k0, k0 + S, ... below kend, at most
// kFoldIters) for the pairs inside the band |d^2 - (2h)^2| <= B, gone through again after the
// block when its smallest |d^2 - (2h)^2| fell inside (rare).  The pair of a particle with itself
// is kept, as the fast path keeps it (see k_near_mixed).
template <bool NB>
__device__ __forceinline__ void near_band(const GCtx &c, const NearSmem<NB> &sm, NearLane &L, int a, int k0, int kend,
                                       int S) {
    const float2 nh2 = make_float2(-L.h2, -L.h2);
    int k = k0;
    for (int t = 0; t < kFoldIters && k < kend; ++t, k += S) {
        float2 dx, dy, dz;
        const float2 e = __fadd2_rn(near_r2(L, sm.a(k), sm.b(k), dx, dy, dz), nh2);
        const float4 c4 = sm.c(k);
        const int4 d4 = sm.D()[k];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (fabsf(u ? e.y : e.x) <= L.B) {
                const int b = u ? d4.y : d4.x;
                const bool nb = b == a || nb_settle(c.px, c.py, c.pz, c.ph, a, b) != 0;
                sub_push(L, nb, __float_as_int(u ? c4.w : c4.z));
                ++L.nfb;
            }
        }
    }
}

// The pair loops of one staged tile for the lane's sink particle a (stream j of S).  Each loop
// runs in blocks of kFoldIters source pairs, folded into the compensated totals after each
// block.  With NB, in a tile of neighbour candidates (reachable cells) the close loop also tests
// every pair for |r_a - r_b| < 2 h_a: by the sign of d^2 - (2h)^2 where |d^2 - (2h)^2| > B (exact
// there), by the float64 test inside the band; each neighbour's original index goes to the lane's
// part of the row.
template <bool NB>
__device__ __forceinline__ void near_tile_lane(const GCtx &c, const NearSmem<NB> &sm, const NearTile &tl, int j, int S,
                                               int a, NearLane &L) {
    const int pc = tl.nclose >> 1;
    const bool nbtile = NB && tl.ncc > 0;  // a tile of neighbour candidates (the same for the whole warp)
    const float2 nh2 = make_float2(-L.h2, -L.h2);
    const float nB = -L.B;
    int k = j;
    while (k < pc) {
        const int kb = k;
        float bandmin = 3e38f;
#pragma unroll 1
        for (int t = 0; t < kFoldIters && k < pc; ++t, k += S) {
            const float4 c4 = sm.c(k);
            const float2 r2 = near_pair_close(L, sm.a(k), sm.b(k), c4);
            if (nbtile) {
                const float2 e = __fadd2_rn(r2, nh2);  // d^2 - (2h)^2
                sub_push(L, e.x < nB, __float_as_int(c4.z));
                sub_push(L, e.y < nB, __float_as_int(c4.w));
                bandmin = fminf(bandmin, fminf(fabsf(e.x), fabsf(e.y)));
            }
        }
        near_fold(L);
        if (nbtile && bandmin <= L.B) near_band<NB>(c, sm, L, a, kb, pc, S);
    }
    const int pf = kNearTile >> 1;
    k = ((kNearTile - tl.nfar) >> 1) + j;
    while (k < pf) {
#pragma unroll 2
        for (int t = 0; t < kFoldIters && k < pf; ++t, k += S) near_pair_newton(L, sm.a(k), sm.b(k));
        near_fold(L);
    }
}

// Mixed near field; with NB also the neighbour counts of Sec. 2.3 on the same staged sources
// (to nb_counts by original index).  The float32 neighbour filter compares d^2 with (2h)^2 -+ B,
// B = 2^-19 ((W + |d_a|_1)^2 + (2h)^2) + 1e-30, W the tile's largest w (see stage_near_mixed):
// the input and offset roundings, the squares and sums, the rounding of d^2 - (2h)^2 and of
// (2h)^2 stay below 16 u F, half of B; inside the band the float64 test (the definition) decides.
// The pair of a particle with itself (d^2 = 0) is kept in the staged row (below the band, or by
// index inside it): every staged row holds the particle itself once, which the copy into the
// CSR drops.
template <bool NB>
__global__ void __launch_bounds__(kNearWarps * 32, kNearMinBlocks) k_near_mixed(GCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const NearSmem<NB> sm(smem_raw + (size_t)w * NearSmem<NB>::bytes);
    int nfb_total = 0;
    for (int s = blockIdx.x * kNearWarps + w; s < c.nsinks; s += gridDim.x * kNearWarps) {
        const int A = c.sinks[s];
        const int fA = c.nfirst[A], nA = c.ncount[A];
        const int nr = c.near_nr[s], nlist = nr + c.near_nn[s];
        // the box of the sink cell's particles (float32 offsets from its centre of mass) and H_A
        float3 blo = make_float3(3e38f, 3e38f, 3e38f), bhi = make_float3(-3e38f, -3e38f, -3e38f);
        float HA = 0.f;
        // the first tile's cells, loaded alongside the sink's particles
        NearAhead ah;
        near_ahead_load(c, (int64_t)s * c.cap_near, nr, nlist, 0, 0, false, ah);
        for (int i = lane; i < nA; i += 32) {
            const float4 pa = c.p32[fA + i];
            blo = make_float3(fminf(blo.x, pa.x), fminf(blo.y, pa.y), fminf(blo.z, pa.z));
            bhi = make_float3(fmaxf(bhi.x, pa.x), fmaxf(bhi.y, pa.y), fmaxf(bhi.z, pa.z));
            HA = fmaxf(HA, c.h32[fA + i]);
        }
        for (int o = 16; o >= 1; o >>= 1) {
            blo.x = fminf(blo.x, __shfl_xor_sync(0xffffffffu, blo.x, o));
            blo.y = fminf(blo.y, __shfl_xor_sync(0xffffffffu, blo.y, o));
            blo.z = fminf(blo.z, __shfl_xor_sync(0xffffffffu, blo.z, o));
            bhi.x = fmaxf(bhi.x, __shfl_xor_sync(0xffffffffu, bhi.x, o));
            bhi.y = fmaxf(bhi.y, __shfl_xor_sync(0xffffffffu, bhi.y, o));
            bhi.z = fmaxf(bhi.z, __shfl_xor_sync(0xffffffffu, bhi.z, o));
            HA = fmaxf(HA, __shfl_xor_sync(0xffffffffu, HA, o));
        }
        // passes of up to 32 sink particles (one pass unless the cell holds more); with the
        // neighbour test the passes of nb_pass_len (at most 16 particles, two or more streams
        // per row), which the direct fill of a queued pass repeats
        const int Pp = NB ? nb_pass_len(nA) : 32;
        for (int a0 = 0; a0 < nA; a0 += Pp) {
            const int P = min(Pp, nA - a0), S = 32 / P;
            const int i = lane % P, j = lane / P;
            const bool active = j < S;
            const int a = fA + a0 + i;
            NearLane L;
            const float4 pa = c.p32[a];
            const float ha = c.h32[a];
            L.xa = make_float2(pa.x, pa.x);
            L.ya = make_float2(pa.y, pa.y);
            L.za = make_float2(pa.z, pa.z);
            L.ha = make_float2(ha, ha);
            {
                const float h2f = 2.0f * ha;  // = float32(2 h) exactly
                L.h2 = h2f * h2f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                L.In[q] = make_float2(0.f, 0.f);
                L.sum[q] = 0.f;
                L.comp[q] = 0.f;
            }
            L.nfb = 0;
            // NB: lane (i, j) keeps its part of row i as column g = i S + j of the row buffer seen as
            // rows of P S entries (simultaneous appends of different lanes fall in different banks)
            L.stride = P * S;
            L.capsub = NB ? kRowBuf / L.stride : 0;
            L.wp = sm.rows + (i * S + j);
            L.dummy = sm.rowcnt + 32 + lane;
            L.nsub = 0;
            NearCursor cur{0, 0};
            if (a0 > 0) near_ahead_load(c, (int64_t)s * c.cap_near, nr, nlist, 0, 0, false, ah);
            for (;;) {
                float wmax = 0.f;
                const NearTile tl =
                    stage_near_mixed<NB>(c, s, A, fA, a0, P, nlist, nr, cur, ah, sm, blo, bhi, HA, wmax);
                if (NB) {
                    const float F = wmax + (fabsf(pa.x) + fabsf(pa.y) + fabsf(pa.z));
                    L.B = fmaf(F, F, L.h2) * 0x1p-19f + 1e-30f;
                }
                if (active) near_tile_lane<NB>(c, sm, tl, j, S, a, L);
                __syncwarp();
                if (tl.last) break;
            }
            // sum the S streams of each sink particle (compensated), through shared memory
            float *red = reinterpret_cast<float *>(sm.P);
            if (active) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    red[lane * 9 + q] = L.sum[q];
                    red[lane * 9 + 4 + q] = L.comp[q];
                }
            }
            __syncwarp();
            if (lane < P) {
                float ts[4], tc[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ts[q] = 0.f;
                    tc[q] = 0.f;
                }
                for (int jj = 0; jj < S; ++jj) {
                    const float *r = red + (lane + jj * P) * 9;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float t, e;
                        two_sum(ts[q], r[q], t, e);
                        ts[q] = t;
                        tc[q] = __fadd_rn(__fadd_rn(tc[q], r[4 + q]), e);
                    }
                }
                // the tile loops included the pair of a with itself: zero force, potential
                // m_a phi(0) = -1.4 m_a 2 / (h_a + h_a), accumulated as (-m_a)(1.4 hinv)
                const float self_pot = -pa.w * (__fdividef(2.0f, ha + ha) * 1.4f);
                float Cf[20];
#pragma unroll
                for (int q = 0; q < 20; ++q) Cf[q] = c.coef32[(int64_t)s * 20 + q];
                const float d[3] = {pa.x, pa.y, pa.z};
                float phf, af[3];
                taylor_eval<float>(Cf, d, phf, af);
                const int o = c.pidx[a];
                c.acc[3 * (int64_t)o] = __dadd_rn((double)ts[0], (double)tc[0]) + (double)af[0];
                c.acc[3 * (int64_t)o + 1] = __dadd_rn((double)ts[1], (double)tc[1]) + (double)af[1];
                c.acc[3 * (int64_t)o + 2] = __dadd_rn((double)ts[2], (double)tc[2]) + (double)af[2];
                if (c.pot) c.pot[o] = __dadd_rn((double)ts[3], (double)tc[3]) + (double)phf - (double)self_pot;
            }
            nfb_total += L.nfb;
            __syncwarp();
            if (NB)
                rows_finish_parts(c.ro, c.nb_counts, sm.rows, sm.rowcnt, L.capsub, P, S, active ? L.nsub : 0,
                                  lane < P ? c.pidx[a] : 0, s, a0);
        }
    }
    if (NB) {
        for (int o = 16; o >= 1; o >>= 1) nfb_total += __shfl_xor_sync(0xffffffffu, nfb_total, o);
        if (lane == 0 && nfb_total) atomicAdd(&c.status[ST_NBFALLBACK], nfb_total);
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
                    ns = stage_near(c, s, A, nlist, nr, t0, kNearTileF64, smw);
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
    c.ro = row_out(t);
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
    const int nb = std::max(1, std::min((t->nsinks + kNearWarps - 1) / kNearWarps, nsm * kNearMinBlocks * 16));
    k_near_mixed<NB><<<nb, kNearWarps * 32, smem, t->stream>>>(c); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

// Far field and near field; with NB (mixed form only) the near kernel also counts the
// neighbours.
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
    if (t->nb_valid) return gravity_impl(t, acc, pot, false);  // the counts are current
    int rc = reset_nb_rows(t);
    if (rc) return rc;
    rc = gravity_impl(t, acc, pot, true);
    if (rc) return rc;
    stage_begin(t, SG_NB_COUNT);
    rc = scan_neighbour_counts(t);
    if (rc) return rc;
    stage_end(t, SG_NB_COUNT);
    return fetch_neighbour_total(t);
}

}  // namespace rcb
