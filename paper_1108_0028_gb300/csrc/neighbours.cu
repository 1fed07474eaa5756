// Neighbour search (Sec. 2.3): the candidate (reachable) ll-cells of each sink are culled to
// the particles b != a with |r_a - r_b| < 2 h_a, and stored in one flat list with per-particle
// offsets (Sec. 2.3.2), rows in original order and sorted by original index.
//
// count  one warp per sink stages the candidate cells' particles in shared memory as float32
//        offsets from the sink's centre of mass (cell-centre difference formed in float64,
//        then the particle's float32 offset from its own cell's centre of mass); lanes take
//        sources, the warp loops over the sink's particles; ballots count neighbours.
// scan   exclusive int64 scan over original indices gives the CSR offsets.
// fill   the same decisions write each neighbour's original index at its row position.
// sort   each row is sorted in shared memory (bitonic, one warp per row; one block per row
//        for rows longer than kRowWarp).
// The float32 test d^2 - (2h)^2 carries the bound B = 2^-19 F, F = (|dCOM|_1 + |d_b|_1 +
// |d_a|_1)^2 + (2h)^2: the three input roundings, the two float additions of the offsets, the
// squares, sums and final subtraction stay below 10 u F (u = 2^-24), so B covers them three
// times.  Inside the band the test is repeated in float64 on the original positions, rounded
// after every operation, which is the definition; the lists are therefore exact.
#include <cuda_runtime.h>

#include <algorithm>

#include "rcb_internal.cuh"

namespace rcb {
namespace {

constexpr int kNbWarps = 4;
constexpr int kNbTile = 1024;   // staged sources per warp
constexpr int kMaxSinkPart = 64;  // sink particles handled per pass of the staged tile
constexpr int kRowWarp = 1024;  // longest row sorted by one warp

struct NbCtx {
    int nsinks;
    const int32_t *sinks, *near_list, *near_nr;
    int cap_near;
    const int32_t *nfirst, *ncount;
    const double *ncom;
    const double *px, *py, *pz, *ph;
    const int32_t *pidx;
    const float4 *p32;
    int64_t *counts;          // [N] by original index
    const int64_t *offsets;   // [N+1]
    int32_t *idx;
    int *status;
};

struct NbSmem {
    float4 src[kNbWarps][kNbTile];   // (x, y, z relative to COM_A, bound term |dCOM|_1 + |d_b|_1)
    int32_t sidx[kNbWarps][kNbTile]; // sorted index of the source
    float4 snk[kNbWarps][kMaxSinkPart];  // (d_a, |d_a|_1)
    float h2[kNbWarps][kMaxSinkPart];    // (2 h_a)^2 in float32
    int cnt[kNbWarps][kMaxSinkPart];
};

// Stage sources [t0, t0 + kNbTile) of the concatenated candidate cells; returns how many.
__device__ int stage_tile(const NbCtx &c, int s, int A, int nr, int64_t t0, float4 *src, int32_t *sidx) {
    const int lane = threadIdx.x & 31;
    const int64_t base = (int64_t)s * c.cap_near;
    const double cAx = c.ncom[3 * (int64_t)A], cAy = c.ncom[3 * (int64_t)A + 1], cAz = c.ncom[3 * (int64_t)A + 2];
    int64_t pos = 0;  // running source index over the cells
    int staged = 0;
    for (int k0 = 0; k0 < nr; k0 += 32) {
        const int k = k0 + lane;
        int B = 0, f = 0, n = 0;
        float dx = 0.f, dy = 0.f, dz = 0.f, sd = 0.f;
        if (k < nr) {
            B = c.near_list[base + k];
            f = c.nfirst[B];
            n = c.ncount[B];
            double ddx = __dsub_rn(c.ncom[3 * (int64_t)B], cAx);
            double ddy = __dsub_rn(c.ncom[3 * (int64_t)B + 1], cAy);
            double ddz = __dsub_rn(c.ncom[3 * (int64_t)B + 2], cAz);
            dx = __double2float_rn(ddx);
            dy = __double2float_rn(ddy);
            dz = __double2float_rn(ddz);
            sd = fabsf(dx) + fabsf(dy) + fabsf(dz);
        }
        int incl = n;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int group_total = __shfl_sync(0xffffffffu, incl, 31);
        const int64_t my0 = pos + incl - n;  // this cell's first source index
        // copy the part of each cell that falls inside the tile
        for (int j = 0; j < 32 && k0 + j < nr; ++j) {
            const int64_t c0 = __shfl_sync(0xffffffffu, my0, j);
            const int cn = __shfl_sync(0xffffffffu, n, j);
            const int cf = __shfl_sync(0xffffffffu, f, j);
            const float ox = __shfl_sync(0xffffffffu, dx, j), oy = __shfl_sync(0xffffffffu, dy, j),
                        oz = __shfl_sync(0xffffffffu, dz, j), os = __shfl_sync(0xffffffffu, sd, j);
            const int64_t lo = c0 > t0 ? c0 : t0;
            const int64_t hi = c0 + cn < t0 + (int64_t)kNbTile ? c0 + cn : t0 + (int64_t)kNbTile;
            for (int64_t q = lo + lane; q < hi; q += 32) {
                const int b = cf + (int)(q - c0);
                const float4 pb = c.p32[b];
                const float x = ox + pb.x, y = oy + pb.y, z = oz + pb.z;
                src[q - t0] = make_float4(x, y, z, os + fabsf(pb.x) + fabsf(pb.y) + fabsf(pb.z));
                sidx[q - t0] = b;
            }
            if (hi > lo) staged = max(staged, (int)(hi - t0));
        }
        pos += group_total;
        if (pos >= t0 + kNbTile) break;
    }
    __syncwarp();
    return staged;
}

__device__ inline bool is_neighbour(const NbCtx &c, float4 sa, float h2, int a, float4 sb, int b, int &nfb) {
    if (a == b) return false;
    const float dx = sb.x - sa.x, dy = sb.y - sa.y, dz = sb.z - sa.z;
    const float f = dx * dx + dy * dy + dz * dz - h2;
    const float Fm = sb.w + sa.w;
    const float B = (Fm * Fm + h2) * 0x1p-19f + 1e-30f;
    if (f < -B) return true;
    if (f > B) return false;
    ++nfb;
    const double s2 = __dmul_rn(2.0, c.ph[a]);
    return dist2_rn(c.px[a], c.py[a], c.pz[a], c.px[b], c.py[b], c.pz[b]) < __dmul_rn(s2, s2);
}

template <bool FILL>
__global__ void __launch_bounds__(kNbWarps * 32) k_neighbours(NbCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NbSmem &sm = *reinterpret_cast<NbSmem *>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int nfb = 0;
    for (int s = blockIdx.x * kNbWarps + w; s < c.nsinks; s += gridDim.x * kNbWarps) {
        const int A = c.sinks[s];
        const int fA = c.nfirst[A], nA = c.ncount[A];
        const int nr = c.near_nr[s];
        // total sources
        int64_t S = 0;
        for (int k = lane; k < nr; k += 32) S += c.ncount[c.near_list[(int64_t)s * c.cap_near + k]];
        for (int o = 16; o >= 1; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
        for (int a0 = 0; a0 < nA; a0 += kMaxSinkPart) {
            const int na = min(kMaxSinkPart, nA - a0);
            for (int i = lane; i < na; i += 32) {
                const int a = fA + a0 + i;
                const float4 pa = c.p32[a];
                const float h2 = __double2float_rn(__dmul_rn(2.0, c.ph[a]));
                sm.snk[w][i] = make_float4(pa.x, pa.y, pa.z, fabsf(pa.x) + fabsf(pa.y) + fabsf(pa.z));
                sm.h2[w][i] = h2 * h2;
                sm.cnt[w][i] = 0;
            }
            __syncwarp();
            for (int64_t t0 = 0; t0 < S; t0 += kNbTile) {
                const int ns = stage_tile(c, s, A, nr, t0, sm.src[w], sm.sidx[w]);
                for (int i = 0; i < na; ++i) {
                    const int a = fA + a0 + i;
                    const float4 sa = sm.snk[w][i];
                    const float h2 = sm.h2[w][i];
                    int run = sm.cnt[w][i];
                    int64_t row0 = 0;
                    if (FILL) row0 = c.offsets[c.pidx[a]];
                    for (int q0 = 0; q0 < ns; q0 += 32) {
                        const int q = q0 + lane;
                        bool nb = false;
                        int b = -1;
                        if (q < ns) {
                            b = sm.sidx[w][q];
                            nb = is_neighbour(c, sa, h2, a, sm.src[w][q], b, nfb);
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, nb);
                        if (FILL && nb) c.idx[row0 + run + __popc(bal & lt)] = c.pidx[b];
                        run += __popc(bal);
                    }
                    if (lane == 0) sm.cnt[w][i] = run;
                    __syncwarp();
                }
            }
            if (!FILL)
                for (int i = lane; i < na; i += 32) c.counts[c.pidx[fA + a0 + i]] = sm.cnt[w][i];
            __syncwarp();
        }
    }
    for (int o = 16; o >= 1; o >>= 1) nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
    if (lane == 0 && nfb) atomicAdd(&c.status[ST_NBFALLBACK], nfb);
}

// Sort rows (one warp per row) in shared memory; longer rows are queued for k_sort_long.
__global__ void __launch_bounds__(kNbWarps * 32) k_sort_rows(const int64_t *offsets, int64_t N, int32_t *idx,
                                                              int32_t *long_rows, int *status, int cap_long) {
    __shared__ int32_t buf[kNbWarps][kRowWarp];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t r = (int64_t)blockIdx.x * kNbWarps + w; r < N; r += (int64_t)gridDim.x * kNbWarps) {
        const int64_t o = offsets[r];
        const int n = (int)(offsets[r + 1] - o);
        if (n <= 1) continue;
        if (n > kRowWarp) {
            if (lane == 0) {
                int slot = atomicAdd(&status[ST_LONGROWS], 1);
                if (slot < cap_long) long_rows[slot] = (int32_t)r;
            }
            continue;
        }
        int p2 = 1;
        while (p2 < n) p2 <<= 1;
        for (int i = lane; i < p2; i += 32) buf[w][i] = i < n ? idx[o + i] : INT32_MAX;
        __syncwarp();
        // bitonic network with every comparator ascending: a flip stage (i vs i ^ (k-1)) then
        // half-cleaners (i vs i ^ j); padding at the end never has to move
        for (int k = 2; k <= p2; k <<= 1) {
            for (int i = lane; i < p2; i += 32) {
                const int l = i ^ (k - 1);
                if (l > i) {
                    const int32_t x = buf[w][i], y = buf[w][l];
                    if (x > y) {
                        buf[w][i] = y;
                        buf[w][l] = x;
                    }
                }
            }
            __syncwarp();
            for (int j = k >> 2; j > 0; j >>= 1) {
                for (int i = lane; i < p2; i += 32) {
                    const int l = i ^ j;
                    if (l > i) {
                        const int32_t x = buf[w][i], y = buf[w][l];
                        if (x > y) {
                            buf[w][i] = y;
                            buf[w][l] = x;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (int i = lane; i < n; i += 32) idx[o + i] = buf[w][i];
        __syncwarp();
    }
}

// Rows longer than one warp's buffer: one block per row, bitonic sort in global memory.
__global__ void k_sort_long(const int64_t *offsets, int32_t *idx, const int32_t *long_rows, const int *nlong_ptr,
                            int cap_long) {
    const int nlong = min(*nlong_ptr, cap_long);
    for (int q = blockIdx.x; q < nlong; q += gridDim.x) {
        const int64_t r = long_rows[q];
        const int64_t o = offsets[r];
        const int64_t n = offsets[r + 1] - o;
        int64_t p2 = 1;
        while (p2 < n) p2 <<= 1;
        // the same all-ascending network; positions >= n are +infinity and never compared
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

}  // namespace

int neighbour_counts(rcb_tree *t, int64_t *counts, int *status) {
    NbCtx c;
    c.nsinks = t->nsinks;
    c.sinks = t->sinks;
    c.near_list = t->near_list;
    c.near_nr = t->near_nr;
    c.cap_near = t->cap_near;
    c.nfirst = t->nfirst;
    c.ncount = t->ncount;
    c.ncom = t->ncom;
    c.px = t->px;
    c.py = t->py;
    c.pz = t->pz;
    c.ph = t->ph;
    c.pidx = t->pidx;
    c.p32 = t->p32;
    c.counts = counts;
    c.offsets = nullptr;
    c.idx = nullptr;
    c.status = status;
    const int nsm = sm_count_nb();
    const size_t smem = sizeof(NbSmem);
    const int blocks = std::max(1, std::min((t->nsinks + kNbWarps - 1) / kNbWarps, nsm * 16));
    RCB_CUDA_TRY(cudaFuncSetAttribute(k_neighbours<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_neighbours<false><<<blocks, kNbWarps * 32, smem, t->stream>>>(c); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

int neighbours(rcb_tree *t, int64_t *offsets, int32_t *idx, int64_t capacity, int64_t *needed) {
    cudaStream_t st = t->stream;
    NbCtx c;
    c.nsinks = t->nsinks;
    c.sinks = t->sinks;
    c.near_list = t->near_list;
    c.near_nr = t->near_nr;
    c.cap_near = t->cap_near;
    c.nfirst = t->nfirst;
    c.ncount = t->ncount;
    c.ncom = t->ncom;
    c.px = t->px;
    c.py = t->py;
    c.pz = t->pz;
    c.ph = t->ph;
    c.pidx = t->pidx;
    c.p32 = t->p32;
    c.counts = t->nb_count;
    c.offsets = offsets;
    c.idx = idx;
    c.status = t->d_status;
    const int nsm = sm_count_nb();
    const size_t smem = sizeof(NbSmem);
    const int blocks = std::max(1, std::min((t->nsinks + kNbWarps - 1) / kNbWarps, nsm * 16));
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_status + ST_NBFALLBACK, 0, 2 * sizeof(int), st));
    if (!t->nb_valid) {
        stage_begin(t, SG_NB_COUNT);
        RCB_CUDA_TRY(cudaFuncSetAttribute(k_neighbours<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_neighbours<false><<<blocks, kNbWarps * 32, smem, st>>>(c); note_launch();
        RCB_CUDA_TRY(cudaGetLastError());
        int rc = scan_i64(t->nb_count, t->nb_count, t->N, t->nb_count + t->N, t->scan_tmp, st);
        if (rc) return rc;
        stage_end(t, SG_NB_COUNT);
        RCB_CUDA_TRY(cudaMemcpyAsync(&t->nb_total, t->nb_count + t->N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        RCB_CUDA_TRY(cudaStreamSynchronize(st));
        t->nb_valid = 1;
    }
    RCB_CUDA_TRY(cudaMemcpyAsync(offsets, t->nb_count, (t->N + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    *needed = t->nb_total;
    if (!idx) {
        RCB_CUDA_TRY(cudaStreamSynchronize(st));
        return RCB_OK;
    }
    if (capacity < t->nb_total) {
        RCB_CUDA_TRY(cudaStreamSynchronize(st));
        return RCB_ERR_CAPACITY;
    }
    RCB_CUDA_TRY(cudaFuncSetAttribute(k_neighbours<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    stage_begin(t, SG_NB_FILL);
    k_neighbours<true><<<blocks, kNbWarps * 32, smem, st>>>(c); note_launch();
    const int rb = (int)std::min<int64_t>((t->N + kNbWarps - 1) / kNbWarps, (int64_t)nsm * 16);
    int32_t *lr = t->nb_long;
    const int cap_long = (int)t->N;
    stage_end(t, SG_NB_FILL);
    stage_begin(t, SG_NB_SORT);
    k_sort_rows<<<std::max(rb, 1), kNbWarps * 32, 0, st>>>(offsets, t->N, idx, lr, t->d_status, cap_long); note_launch();
    k_sort_long<<<std::max(1, nsm * 2), 1024, 0, st>>>(offsets, idx, lr, t->d_status + ST_LONGROWS, cap_long); note_launch();
    stage_end(t, SG_NB_SORT);
    RCB_CUDA_TRY(cudaGetLastError());
    RCB_CUDA_TRY(cudaStreamSynchronize(st));
    return RCB_OK;
}

}  // namespace rcb
