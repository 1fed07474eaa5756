// Neighbour search (Sec. 2.3): the candidate (reachable) ll-cells of each sink are culled to
// the particles b != a with |r_a - r_b| < 2 h_a, and stored in one flat list with per-particle
// offsets (Sec. 2.3.2), rows in original order and sorted by original index.
//
// pass     one warp per sink stages its candidate particles in shared memory (one lane per cell)
//          as float32 offsets from the sink's centre of mass (the cell-centre difference formed
//          in float64, then each particle's float32 offset from its own cell's centre of mass).
//          Eight sink particles sit in registers; lanes take 32 sources at a time and every pair
//          test is one bit of a warp ballot.  A particle's count goes to its original index and
//          its neighbours' sorted indices to a row of kRowCap slots; longer rows are queued.
// scan     exclusive int64 scan over original indices gives the CSR offsets.
// compact  one warp per particle maps its slot row to original indices, sorts it (bitonic
//          network of shuffles) and writes it at its offset.
// long     queued rows are recomputed straight into place, one warp each, and sorted by one
//          block each.
// The float32 test compares d^2 with (2h)^2 -+ B, B = 2^-19 F, F = (W + |d_a|_1)^2 + (2h)^2 with W
// the tile's largest |dCOM|_1 + |d_b|_1: the three input roundings, the two float additions of
// the offsets, the squares and sums, and the roundings of (2h)^2 and of (2h)^2 -+ B stay below
// 13 u F (u = 2^-24), so B covers them more than twice; the additive 1e-30 covers flushed
// subnormals.  Inside the band the test is repeated in float64 on the original positions,
// rounded after every operation, which is the definition; the lists are therefore exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <climits>

#include "rcb_internal.cuh"

namespace rcb {
namespace {

constexpr int kNbWarps = 8;
constexpr int kNbTile = 512;      // staged sources per warp
constexpr int kNbGroup = 8;       // sink particles held in registers
constexpr int kMaxSinkPart = 64;  // sink particles whose running counts sit in shared memory
constexpr int kRowCap = kNbRowCap;  // slots of a particle's row before the compaction
constexpr unsigned kFull = 0xffffffffu;

struct NbCtx {
    int nsinks;
    const int32_t *sinks, *near_list, *near_nr;
    int cap_near;
    const int32_t *nfirst, *ncount;
    const double *ncom;
    const double *px, *py, *pz, *ph;
    const int32_t *pidx;
    const float4 *p32;
    const float *h32;
    int64_t *counts;         // [N] by original index
    const int64_t *offsets;  // [N+1]
    int32_t *idx;
    int32_t *rows;   // [N][kRowCap] by sorted index, entries sorted indices
    int2 *long_rows;  // (sorted particle, sink) of rows longer than kRowCap
    int cap_long;
    int *status;
};

struct NbSmem {
    float4 src[kNbWarps][kNbTile];    // (d_b relative to COM_A, |dCOM|_1 + |d_b|_1)
    int32_t sidx[kNbWarps][kNbTile];  // sorted index of the source
    int32_t oidx[kNbWarps][kNbTile];  // original index of the source
    int run[kNbWarps][kMaxSinkPart];  // neighbours found so far per sink particle
};

// Candidate sources of sink s: their number and the position of the sink's own cell among them
// (-1 when the cell is not among its own candidates, which needs h_int = 0).
struct SinkLayout {
    int64_t S, posA;
};

__device__ SinkLayout sink_layout(const NbCtx &c, int s, int A, int nr) {
    const int lane = threadIdx.x & 31;
    const int64_t base = (int64_t)s * c.cap_near;
    int64_t pos = 0, posA = -1;
    for (int k0 = 0; k0 < nr; k0 += 32) {
        const int k = k0 + lane;
        int n = 0;
        bool me = false;
        if (k < nr) {
            const int B = c.near_list[base + k];
            n = c.ncount[B];
            me = B == A;
        }
        const int excl = warp_excl_scan(n);
        const unsigned mm = __ballot_sync(kFull, me);
        const int before = __shfl_sync(kFull, excl, mm ? __ffs(mm) - 1 : 0);
        if (mm) posA = pos + before;
        pos += __shfl_sync(kFull, excl + n, 31);
    }
    return SinkLayout{pos, posA};
}

// Stage sources [t0, t0 + kNbTile): lanes first describe 32 candidate cells (first particle,
// count, centre-of-mass offset), then take one slot each, find its cell and copy the particle.
// Returns the staged count; wmax gets the largest w = |dCOM|_1 + |d_b|_1 of the tile.
template <bool ORIG>
__device__ int stage_tile(const NbCtx &c, int s, int A, int nr, int64_t t0, float4 *src, int32_t *sidx,
                          int32_t *oidx, float &wmax) {
    const int lane = threadIdx.x & 31;
    const int64_t base = (int64_t)s * c.cap_near;
    const double cAx = c.ncom[3 * (int64_t)A], cAy = c.ncom[3 * (int64_t)A + 1], cAz = c.ncom[3 * (int64_t)A + 2];
    int64_t pos = 0;
    float wl = 0.f;
    for (int k0 = 0; k0 < nr && pos < t0 + kNbTile; k0 += 32) {
        const int k = k0 + lane;
        int f = 0, n = 0;
        float dx = 0.f, dy = 0.f, dz = 0.f;
        if (k < nr) {
            const int B = c.near_list[base + k];
            f = c.nfirst[B];
            n = c.ncount[B];
            dx = __double2float_rn(__dsub_rn(c.ncom[3 * (int64_t)B], cAx));
            dy = __double2float_rn(__dsub_rn(c.ncom[3 * (int64_t)B + 1], cAy));
            dz = __double2float_rn(__dsub_rn(c.ncom[3 * (int64_t)B + 2], cAz));
        }
        const int excl = warp_excl_scan(n);
        const int total = __shfl_sync(kFull, excl + n, 31);
        const int64_t lo = pos > t0 ? pos : t0;
        const int64_t hi = pos + total < t0 + kNbTile ? pos + total : t0 + kNbTile;
        for (int64_t j0 = lo; j0 < hi; j0 += 32) {
            const int64_t j = j0 + lane;
            const int rel = (int)(j - pos);
            const int cl = warp_run_of(excl, n, (int)(j0 - pos));
            const int fc = __shfl_sync(kFull, f, cl), ec = __shfl_sync(kFull, excl, cl);
            const float cx = __shfl_sync(kFull, dx, cl), cy = __shfl_sync(kFull, dy, cl), cz = __shfl_sync(kFull, dz, cl);
            if (j < hi) {
                const int b = fc + rel - ec;
                const float4 pb = c.p32[b];
                const float wv = (fabsf(cx) + fabsf(cy) + fabsf(cz)) + fabsf(pb.x) + fabsf(pb.y) + fabsf(pb.z);
                src[j - t0] = make_float4(cx + pb.x, cy + pb.y, cz + pb.z, wv);
                sidx[j - t0] = b;
                if (ORIG) oidx[j - t0] = c.pidx[b];
                wl = fmaxf(wl, wv);
            }
        }
        pos += total;
    }
    for (int o = 16; o >= 1; o >>= 1) wl = fmaxf(wl, __shfl_xor_sync(kFull, wl, o));
    wmax = wl;
    __syncwarp();
    const int64_t left = pos - t0;
    return (int)(left < kNbTile ? left : kNbTile);
}

// Tests the staged sources [0, ns) against the sink particles a0 + i, i < na (sorted indices).
// Bit selfq_i = self0 + i (tile-relative slot of a0 + i itself) is cleared.  runs[i] holds the
// neighbours found so far; with EMIT, a neighbour's emit[j] goes to out[i * stride + run] while
// run < lim.
template <bool EMIT>
__device__ void test_group(const NbCtx &c, const float4 *src, const int32_t *sidx, const int32_t *emit, int ns,
                           float wmax, int a0, int na, int64_t self0, int *runs, int32_t *out, int64_t stride,
                           int64_t lim, int &nfb) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    float sx[kNbGroup], sy[kNbGroup], sz[kNbGroup], lo[kNbGroup], hi[kNbGroup];
    int run[kNbGroup], selfq[kNbGroup];
#pragma unroll
    for (int i = 0; i < kNbGroup; ++i) {
        const int a = a0 + (i < na ? i : 0);
        const float4 pa = c.p32[a];
        const float h2f = 2.0f * c.h32[a];  // = float32(2 h) exactly
        const float h2 = h2f * h2f;
        const float F = wmax + (fabsf(pa.x) + fabsf(pa.y) + fabsf(pa.z));
        const float B = fmaf(F, F, h2) * 0x1p-19f + 1e-30f;
        sx[i] = pa.x;
        sy[i] = pa.y;
        sz[i] = pa.z;
        lo[i] = h2 - B;
        hi[i] = h2 + B;
        run[i] = i < na ? runs[i] : 0;
        const int64_t q = self0 + i;
        selfq[i] = (q >= 0 && q < ns) ? (int)q : -1;
    }
    for (int q0 = 0; q0 < ns; q0 += 32) {
        const int j = q0 + lane;
        const bool valid = j < ns;
        const unsigned vm = __ballot_sync(kFull, valid);
        // padding lanes: a source far away (finite d^2, never below the bound)
        const float4 b = valid ? src[j] : make_float4(3e18f, 3e18f, 3e18f, 0.f);
#pragma unroll
        for (int i = 0; i < kNbGroup; ++i) {
            if (i < na) {
                const float dx = b.x - sx[i], dy = b.y - sy[i], dz = b.z - sz[i];
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                unsigned bh = __ballot_sync(kFull, r2 <= hi[i]);
                if (bh) {  // some lane may hold a neighbour (most chunks have none)
                    bh &= vm;
                    unsigned bl = __ballot_sync(kFull, r2 < lo[i]) & vm;
                    if (bl != bh) {
                        // inside the band: the float64 test decides
                        const unsigned amb = bh & ~bl;
                        bool nb = false;
                        if ((amb >> lane) & 1u) {
                            const int a = a0 + i, bs = sidx[j];
                            const double s2 = __dmul_rn(2.0, c.ph[a]);
                            nb = dist2_rn(c.px[a], c.py[a], c.pz[a], c.px[bs], c.py[bs], c.pz[bs]) < __dmul_rn(s2, s2);
                            ++nfb;
                        }
                        bl |= __ballot_sync(kFull, nb);
                    }
                    const int d = selfq[i] - q0;
                    if ((unsigned)d < 32u) bl &= ~(1u << d);
                    if (EMIT && ((bl >> lane) & 1u)) {
                        const int64_t p = (int64_t)run[i] + __popc(bl & lt);
                        if (p < lim) out[i * stride + p] = emit[j];
                    }
                    run[i] += __popc(bl);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kNbGroup; ++i)
        if (i < na && lane == 0) runs[i] = run[i];
    __syncwarp();
}

// Count pass; with EMIT also the slot rows and the queue of long rows.
template <bool EMIT>
__global__ void __launch_bounds__(kNbWarps * 32) k_nb_pass(NbCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NbSmem &sm = *reinterpret_cast<NbSmem *>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int nfb = 0;
    for (int s = blockIdx.x * kNbWarps + w; s < c.nsinks; s += gridDim.x * kNbWarps) {
        const int A = c.sinks[s];
        const int fA = c.nfirst[A], nA = c.ncount[A];
        const int nr = c.near_nr[s];
        const SinkLayout L = sink_layout(c, s, A, nr);
        for (int p0 = 0; p0 < nA; p0 += kMaxSinkPart) {
            const int np = min(kMaxSinkPart, nA - p0);
            for (int i = lane; i < np; i += 32) sm.run[w][i] = 0;
            __syncwarp();
            for (int64_t t0 = 0; t0 < L.S; t0 += kNbTile) {
                float wmax;
                const int ns = stage_tile<false>(c, s, A, nr, t0, sm.src[w], sm.sidx[w], sm.oidx[w], wmax);
                for (int g = 0; g < np; g += kNbGroup) {
                    const int a0 = fA + p0 + g;
                    const int64_t self0 = L.posA < 0 ? INT64_MIN / 2 : L.posA + p0 + g - t0;
                    test_group<EMIT>(c, sm.src[w], sm.sidx[w], sm.sidx[w], ns, wmax, a0, min(kNbGroup, np - g), self0,
                                     sm.run[w] + g, EMIT ? c.rows + (int64_t)a0 * kRowCap : nullptr, kRowCap, kRowCap,
                                     nfb);
                }
                __syncwarp();
            }
            for (int i = lane; i < np; i += 32) {
                const int a = fA + p0 + i;
                const int n = sm.run[w][i];
                c.counts[c.pidx[a]] = n;
                if (EMIT && n > kRowCap) {
                    const int q = atomicAdd(&c.status[ST_LONGROWS], 1);
                    if (q < c.cap_long) c.long_rows[q] = make_int2(a, s);
                }
            }
            __syncwarp();
        }
    }
    for (int o = 16; o >= 1; o >>= 1) nfb += __shfl_xor_sync(kFull, nfb, o);
    if (lane == 0 && nfb) atomicAdd(&c.status[ST_NBFALLBACK], nfb);
}

// Rows longer than kRowCap: one warp per row recomputes it straight into its place.
__global__ void __launch_bounds__(kNbWarps * 32) k_nb_long(NbCtx c, int nlong) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NbSmem &sm = *reinterpret_cast<NbSmem *>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int nfb = 0;
    for (int q = blockIdx.x * kNbWarps + w; q < nlong; q += gridDim.x * kNbWarps) {
        const int2 e = c.long_rows[q];
        const int a = e.x, s = e.y;
        const int A = c.sinks[s];
        const int fA = c.nfirst[A], nr = c.near_nr[s];
        const SinkLayout L = sink_layout(c, s, A, nr);
        const int64_t o = c.offsets[c.pidx[a]];
        if (lane == 0) sm.run[w][0] = 0;
        __syncwarp();
        for (int64_t t0 = 0; t0 < L.S; t0 += kNbTile) {
            float wmax;
            const int ns = stage_tile<true>(c, s, A, nr, t0, sm.src[w], sm.sidx[w], sm.oidx[w], wmax);
            const int64_t self0 = L.posA < 0 ? INT64_MIN / 2 : L.posA + (a - fA) - t0;
            test_group<true>(c, sm.src[w], sm.sidx[w], sm.oidx[w], ns, wmax, a, 1, self0, sm.run[w], c.idx + o, 0,
                             INT64_MAX, nfb);
            __syncwarp();
        }
    }
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

// A warp takes 32 consecutive particles (sorted indices): their permutation entries and offsets
// are loaded once, coalesced; then two rows at a time the slot entries are mapped to original
// indices, sorted in registers (one row per half-warp when both have at most 64 entries, else
// one row at a time over the warp) and written at the row's offset.  Rows longer than kRowCap
// are written by k_nb_long.
__device__ inline void load_row(const int32_t *rows, const int32_t *pidx, int64_t a, int n, int32_t v[4]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int q = r * 32 + lane;
        v[r] = (n <= kRowCap && q < n) ? pidx[rows[a * kRowCap + q]] : INT32_MAX;
    }
}

__global__ void __launch_bounds__(256) k_nb_compact(const int32_t *rows, const int32_t *pidx, const int64_t *offsets,
                                                    int32_t *idx, int64_t N) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < N; base += nw * 32) {
        int64_t ol = 0;
        int nl = 0;
        if (base + lane < N) {
            const int r = pidx[base + lane];
            ol = offsets[r];
            nl = (int)(offsets[r + 1] - ol);
        }
        const int cnt = (int)(N - base < 32 ? N - base : 32);
        const int half = lane >> 4, hl = lane & 15;
        for (int i = 0; i < cnt; i += 2) {
            const int n0 = __shfl_sync(0xffffffffu, nl, i);
            const int n1 = i + 1 < cnt ? __shfl_sync(0xffffffffu, nl, i + 1) : 0;
            const int64_t o0 = __shfl_sync(0xffffffffu, ol, i);
            const int64_t o1 = __shfl_sync(0xffffffffu, ol, min(i + 1, cnt - 1));
            if (n0 <= 64 && n1 <= 64) {
                // two rows at once, one per half-warp: up to 16 R entries each
                const int n = half ? n1 : n0;
                const int64_t a = base + i + half, o = half ? o1 : o0;
                int32_t v[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int q = r * 16 + hl;
                    v[r] = (q < n) ? pidx[rows[a * kRowCap + q]] : INT32_MAX;
                }
                if (n0 <= 32 && n1 <= 32) {
                    int32_t w2[2] = {v[0], v[1]};
                    halfwarp_sort<2>(w2);
                    if (hl < n) idx[o + hl] = w2[0];
                    if (16 + hl < n) idx[o + 16 + hl] = w2[1];
                } else {
                    halfwarp_sort<4>(v);
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (r * 16 + hl < n) idx[o + r * 16 + hl] = v[r];
                }
                continue;
            }
            // otherwise one row at a time over the whole warp
            for (int u = 0; u < 2 && i + u < cnt; ++u) {
                const int n = u ? n1 : n0;
                const int64_t o = u ? o1 : o0;
                int32_t cur[4];
                load_row(rows, pidx, base + i + u, n, cur);
                if (n <= 32) {
                    int32_t v[1] = {cur[0]};
                    warp_sort<1>(v);
                    if (lane < n) idx[o + lane] = v[0];
                } else if (n <= 64) {
                    int32_t v[2] = {cur[0], cur[1]};
                    warp_sort<2>(v);
                    idx[o + lane] = v[0];
                    if (lane + 32 < n) idx[o + lane + 32] = v[1];
                } else if (n <= kRowCap) {
                    warp_sort<4>(cur);
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (r * 32 + lane < n) idx[o + r * 32 + lane] = cur[r];
                }
            }
        }
    }
}

// Long rows: one block per row, a bitonic network in global memory with every comparator
// ascending (a flip stage, then half-cleaners); positions >= n count as +infinity and are never
// touched.
__global__ void k_sort_long(const int64_t *offsets, int32_t *idx, const int2 *long_rows, const int32_t *pidx,
                            int nlong) {
    for (int q = blockIdx.x; q < nlong; q += gridDim.x) {
        const int64_t r = pidx[long_rows[q].x];
        const int64_t o = offsets[r];
        const int64_t n = offsets[r + 1] - o;
        int64_t p2 = 1;
        while (p2 < n) p2 <<= 1;
        for (int64_t k = 2; k <= p2; k <<= 1) {
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
                const int64_t l = i ^ (k - 1);
                if (l > i && l < n) {
                    const int32_t x = idx[o + i], y = idx[o + l];
                    if (x > y) {
                        idx[o + i] = y;
                        idx[o + l] = x;
                    }
                }
            }
            __syncthreads();
            for (int64_t j = k >> 2; j > 0; j >>= 1) {
                for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
                    const int64_t l = i ^ j;
                    if (l > i && l < n) {
                        const int32_t x = idx[o + i], y = idx[o + l];
                        if (x > y) {
                            idx[o + i] = y;
                            idx[o + l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
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
    c.ncom = t->ncom;
    c.px = t->px;
    c.py = t->py;
    c.pz = t->pz;
    c.ph = t->ph;
    c.pidx = t->pidx;
    c.p32 = t->p32;
    c.h32 = t->h32;
    c.counts = t->nb_count;
    c.offsets = nullptr;
    c.idx = nullptr;
    c.rows = nullptr;
    c.long_rows = t->nb_long;
    c.cap_long = (int)t->N;
    c.status = t->d_status;
    return c;
}

template <bool EMIT>
int launch_pass(rcb_tree *t, const NbCtx &c) {
    const int nsm = sm_count_nb();
    const size_t smem = sizeof(NbSmem);
    const int blocks = std::max(1, std::min((t->nsinks + kNbWarps - 1) / kNbWarps, nsm * 8));
    RCB_CUDA_TRY(cudaFuncSetAttribute(k_nb_pass<EMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_nb_pass<EMIT><<<blocks, kNbWarps * 32, smem, t->stream>>>(c); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

}  // namespace

int neighbour_counts(rcb_tree *t, int64_t *counts, int *status) {
    NbCtx c = make_nbctx(t);
    c.counts = counts;
    c.status = status;
    return launch_pass<false>(t, c);
}

int ensure_nb_rows(rcb_tree *t) {
    if (t->cap_rows >= t->N) return RCB_OK;
    dev_free(t, t->nb_rows);
    t->nb_rows = (int32_t *)dev_alloc(t, (size_t)t->N * kRowCap * sizeof(int32_t));
    if (!t->nb_rows) {
        t->cap_rows = 0;
        return RCB_ERR_ALLOC;
    }
    t->cap_rows = t->N;
    return RCB_OK;
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
    t->nb_nlong = std::min(t->h_status[ST_LONGROWS], (int)t->N);
    t->nb_valid = 1;
    return RCB_OK;
}

int count_neighbours(rcb_tree *t) {
    if (t->nb_valid) return RCB_OK;
    NbCtx c = make_nbctx(t);
    stage_begin(t, SG_NB_COUNT);
    int rc = ensure_nb_rows(t);
    if (rc) return rc;
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_status + ST_NBFALLBACK, 0, 2 * sizeof(int), t->stream));
    c.rows = t->nb_rows;
    rc = launch_pass<true>(t, c);
    if (rc) return rc;
    rc = scan_neighbour_counts(t);
    if (rc) return rc;
    stage_end(t, SG_NB_COUNT);
    return fetch_neighbour_total(t);
}

int neighbours(rcb_tree *t, int64_t *offsets, int32_t *idx, int64_t capacity, int64_t *needed) {
    cudaStream_t st = t->stream;
    NbCtx c = make_nbctx(t);
    const int nsm = sm_count_nb();
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
    c.offsets = offsets;
    c.idx = idx;
    c.rows = t->nb_rows;
    stage_begin(t, SG_NB_FILL);
    k_nb_compact<<<std::max(1, nsm * 16), 256, 0, st>>>(t->nb_rows, t->pidx, offsets, idx, t->N); note_launch();
    stage_end(t, SG_NB_FILL);
    stage_begin(t, SG_NB_SORT);
    if (t->nb_nlong > 0) {
        const size_t smem = sizeof(NbSmem);
        RCB_CUDA_TRY(cudaFuncSetAttribute(k_nb_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int blocks = std::max(1, std::min((t->nb_nlong + kNbWarps - 1) / kNbWarps, nsm * 8));
        k_nb_long<<<blocks, kNbWarps * 32, smem, st>>>(c, t->nb_nlong); note_launch();
        k_sort_long<<<std::max(1, std::min(t->nb_nlong, nsm * 2)), 1024, 0, st>>>(offsets, idx, t->nb_long, t->pidx,
                                                                                 t->nb_nlong); note_launch();
    }
    stage_end(t, SG_NB_SORT);
    RCB_CUDA_TRY(cudaGetLastError());
    RCB_CUDA_TRY(cudaStreamSynchronize(st));
    return RCB_OK;
}

}  // namespace rcb
