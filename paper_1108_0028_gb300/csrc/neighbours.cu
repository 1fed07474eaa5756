// Neighbour search (Sec. 2.3): the candidate (reachable) ll-cells of each sink are culled to
// the particles b != a with |r_a - r_b| < 2 h_a, and stored in one flat list with per-particle
// offsets (Sec. 2.3.2), rows in original order and sorted by original index.
//
// sizes  per sink: particles of its candidate cells (S) and the words of its ballot masks
//        (n_A x ceil(S/32)); a scan places every sink's masks.
// count  one warp per sink stages the candidate particles in shared memory (one lane per cell)
//        as float32 offsets from the sink's centre of mass (the cell-centre difference formed
//        in float64, then each particle's float32 offset from its own cell's centre of mass);
//        lanes take 32 sources, the warp loops over the sink's particles; each 32-source
//        ballot is the neighbour mask of that chunk.  Counts go to the particle's original
//        index; masks to global memory.
// scan   exclusive int64 scan over original indices gives the CSR offsets.
// fill   per sink, a prefix table of its candidate cells maps a source number to a particle;
//        each particle's row is expanded from its masks into shared memory, sorted (bitonic)
//        and written in one coalesced run.  Rows longer than kRowWarp are written unsorted and
//        sorted afterwards by one block each.
// The float32 test d^2 - (2h)^2 carries the bound B = 2^-19 F, F = (|dCOM|_1 + |d_b|_1 +
// |d_a|_1)^2 + (2h)^2: the three input roundings, the two float additions of the offsets, the
// squares, sums and final subtraction stay below 10 u F (u = 2^-24), so B covers them three
// times; the additive 1e-30 covers flushed subnormals.  Inside the band the test is repeated in
// float64 on the original positions, rounded after every operation, which is the definition;
// the lists are therefore exact.
#include <cuda_runtime.h>

#include <algorithm>

#include "rcb_internal.cuh"

namespace rcb {
namespace {

constexpr int kNbWarps = 8;
constexpr int kNbTile = 512;      // staged sources per warp (count pass)
constexpr int kMaxSinkPart = 64;  // sink particles kept in shared memory per pass
constexpr int kRowWarp = 1024;    // longest row sorted by one warp

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
    const int64_t *mask_off;  // [nsinks + 1] word offsets of each sink's masks (or null)
    uint32_t *masks;
    int32_t *long_rows;
    int cap_long;
};

struct NbSmem {
    float4 src[kNbWarps][kNbTile];        // (x, y, z relative to COM_A, |dCOM|_1 + |d_b|_1)
    int32_t sidx[kNbWarps][kNbTile];      // sorted index of the source
    float4 snk[kNbWarps][kMaxSinkPart];   // (d_a, |d_a|_1)
    float h2[kNbWarps][kMaxSinkPart];     // (2 h_a)^2 in float32
    int cnt[kNbWarps][kMaxSinkPart];
};

__device__ inline int64_t sources_of(const NbCtx &c, int s, int nr) {
    const int lane = threadIdx.x & 31;
    int64_t S = 0;
    for (int k = lane; k < nr; k += 32) S += c.ncount[c.near_list[(int64_t)s * c.cap_near + k]];
    for (int o = 16; o >= 1; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
    return S;
}

__global__ void k_nb_sizes(NbCtx c, int64_t *words) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = gw; s < c.nsinks; s += nw) {
        const int64_t S = sources_of(c, s, c.near_nr[s]);
        if (lane == 0) words[s] = (int64_t)c.ncount[c.sinks[s]] * ((S + 31) / 32);
    }
}

// Stage sources [t0, t0 + kNbTile): one lane per candidate cell copies that cell's particles.
__device__ int stage_tile(const NbCtx &c, int s, int A, int nr, int64_t t0, float4 *src, int32_t *sidx) {
    const int lane = threadIdx.x & 31;
    const int64_t base = (int64_t)s * c.cap_near;
    const double cAx = c.ncom[3 * (int64_t)A], cAy = c.ncom[3 * (int64_t)A + 1], cAz = c.ncom[3 * (int64_t)A + 2];
    int64_t pos = 0;
    for (int k0 = 0; k0 < nr && pos < t0 + kNbTile; k0 += 32) {
        const int k = k0 + lane;
        int f = 0, n = 0;
        float dx = 0.f, dy = 0.f, dz = 0.f, sd = 0.f;
        if (k < nr) {
            const int B = c.near_list[base + k];
            f = c.nfirst[B];
            n = c.ncount[B];
            dx = __double2float_rn(__dsub_rn(c.ncom[3 * (int64_t)B], cAx));
            dy = __double2float_rn(__dsub_rn(c.ncom[3 * (int64_t)B + 1], cAy));
            dz = __double2float_rn(__dsub_rn(c.ncom[3 * (int64_t)B + 2], cAz));
            sd = fabsf(dx) + fabsf(dy) + fabsf(dz);
        }
        int incl = n;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int64_t my0 = pos + incl - n;
        for (int q = 0; q < n; ++q) {
            const int64_t slot = my0 + q - t0;
            if (slot >= 0 && slot < kNbTile) {
                const float4 pb = c.p32[f + q];
                src[slot] = make_float4(dx + pb.x, dy + pb.y, dz + pb.z, sd + fabsf(pb.x) + fabsf(pb.y) + fabsf(pb.z));
                sidx[slot] = f + q;
            }
        }
        pos += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    const int64_t left = pos - t0;
    return (int)(left < kNbTile ? left : kNbTile);
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

// Count pass (and, when masks are given, the per-chunk neighbour masks).
__global__ void __launch_bounds__(kNbWarps * 32) k_nb_count(NbCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NbSmem &sm = *reinterpret_cast<NbSmem *>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int nfb = 0;
    for (int s = blockIdx.x * kNbWarps + w; s < c.nsinks; s += gridDim.x * kNbWarps) {
        const int A = c.sinks[s];
        const int fA = c.nfirst[A], nA = c.ncount[A];
        const int nr = c.near_nr[s];
        const int64_t S = sources_of(c, s, nr);
        const int nch = (int)((S + 31) / 32);
        uint32_t *mrow = c.masks ? c.masks + c.mask_off[s] : nullptr;
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
                const int c0 = (int)(t0 / 32);
                for (int i = 0; i < na; ++i) {
                    const int a = fA + a0 + i;
                    const float4 sa = sm.snk[w][i];
                    const float h2 = sm.h2[w][i];
                    int run = 0;
                    uint32_t mine = 0;
                    for (int q0 = 0; q0 < ns; q0 += 32) {
                        const int q = q0 + lane;
                        bool nb = false;
                        if (q < ns) nb = is_neighbour(c, sa, h2, a, sm.src[w][q], sm.sidx[w][q], nfb);
                        const unsigned bal = __ballot_sync(0xffffffffu, nb);
                        run += __popc(bal);
                        if (lane == (q0 >> 5)) mine = bal;
                    }
                    if (mrow) {
                        const int nct = (ns + 31) >> 5;  // chunks of this tile (<= 16)
                        if (lane < nct) mrow[(int64_t)(a0 + i) * nch + c0 + lane] = mine;
                    }
                    if (lane == 0) sm.cnt[w][i] += run;
                    __syncwarp();
                }
            }
            for (int i = lane; i < na; i += 32) c.counts[c.pidx[fA + a0 + i]] = sm.cnt[w][i];
            __syncwarp();
        }
    }
    for (int o = 16; o >= 1; o >>= 1) nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
    if (lane == 0 && nfb) atomicAdd(&c.status[ST_NBFALLBACK], nfb);
}

// Fill pass: expand the masks into rows, sort each row, write it.  Shared memory per warp: the
// prefix table of the sink's candidate cells (first source number, first particle) and one row.
__global__ void __launch_bounds__(kNbWarps * 32) k_nb_fill(NbCtx c, int table_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *tab = reinterpret_cast<int32_t *>(smem_raw) + (size_t)w * (2 * table_cap + kRowWarp);
    int32_t *tpos = tab, *tfirst = tab + table_cap;
    int32_t *row = tab + 2 * table_cap;
    for (int s = blockIdx.x * (blockDim.x >> 5) + w; s < c.nsinks; s += gridDim.x * (blockDim.x >> 5)) {
        const int A = c.sinks[s];
        const int fA = c.nfirst[A], nA = c.ncount[A];
        const int nr = c.near_nr[s];
        const int64_t base = (int64_t)s * c.cap_near;
        int pos = 0;
        for (int k0 = 0; k0 < nr; k0 += 32) {
            const int k = k0 + lane;
            int n = 0, f = 0;
            if (k < nr) {
                const int B = c.near_list[base + k];
                n = c.ncount[B];
                f = c.nfirst[B];
            }
            int incl = n;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (k < nr) {
                tpos[k] = pos + incl - n;
                tfirst[k] = f;
            }
            pos += __shfl_sync(0xffffffffu, incl, 31);
        }
        __syncwarp();
        const int S = pos;
        const int nch = (S + 31) / 32;
        const uint32_t *mrow = c.masks + c.mask_off[s];
        for (int i = 0; i < nA; ++i) {
            const int a = fA + i;
            const int64_t o = c.offsets[c.pidx[a]];
            const int n = (int)(c.offsets[c.pidx[a] + 1] - o);
            if (n == 0) continue;
            const bool fits = n <= kRowWarp;
            int run = 0;
            for (int ch0 = 0; ch0 < nch; ch0 += 32) {
                const int ch = ch0 + lane;
                uint32_t m = ch < nch ? mrow[(int64_t)i * nch + ch] : 0u;
                const int pc = __popc(m);
                int incl = pc;
                for (int o2 = 1; o2 < 32; o2 <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, o2);
                    if (lane >= o2) incl += t;
                }
                int p = run + incl - pc;
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    const int j = ch * 32 + bit;  // source number
                    int lo = 0, hi = nr - 1;      // last cell with tpos <= j
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (tpos[mid] <= j) lo = mid;
                        else hi = mid - 1;
                    }
                    const int32_t orig = c.pidx[tfirst[lo] + (j - tpos[lo])];
                    if (fits) row[p] = orig;
                    else c.idx[o + p] = orig;
                    ++p;
                }
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
            __syncwarp();
            if (!fits) {
                if (lane == 0) {
                    const int slot = atomicAdd(&c.status[ST_LONGROWS], 1);
                    if (slot < c.cap_long) c.long_rows[slot] = c.pidx[a];
                }
                continue;
            }
            int p2 = 1;
            while (p2 < n) p2 <<= 1;
            for (int q = n + lane; q < p2; q += 32) row[q] = INT32_MAX;
            __syncwarp();
            // bitonic network with every comparator ascending: a flip stage (i vs i ^ (k-1)) then
            // half-cleaners (i vs i ^ j); padding at the end never has to move
            for (int k = 2; k <= p2; k <<= 1) {
                for (int q = lane; q < p2; q += 32) {
                    const int l = q ^ (k - 1);
                    if (l > q) {
                        const int32_t x = row[q], y = row[l];
                        if (x > y) {
                            row[q] = y;
                            row[l] = x;
                        }
                    }
                }
                __syncwarp();
                for (int j = k >> 2; j > 0; j >>= 1) {
                    for (int q = lane; q < p2; q += 32) {
                        const int l = q ^ j;
                        if (l > q) {
                            const int32_t x = row[q], y = row[l];
                            if (x > y) {
                                row[q] = y;
                                row[l] = x;
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            for (int q = lane; q < n; q += 32) c.idx[o + q] = row[q];
            __syncwarp();
        }
    }
}

// Rows longer than one warp's buffer: one block per row, the same network in global memory;
// positions >= n are +infinity and never compared.
__global__ void k_sort_long(const int64_t *offsets, int32_t *idx, const int32_t *long_rows, const int *nlong_ptr,
                            int cap_long) {
    const int nlong = min(*nlong_ptr, cap_long);
    for (int q = blockIdx.x; q < nlong; q += gridDim.x) {
        const int64_t r = long_rows[q];
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
    c.offsets = nullptr;
    c.idx = nullptr;
    c.status = t->d_status;
    c.mask_off = nullptr;
    c.masks = nullptr;
    c.long_rows = t->nb_long;
    c.cap_long = (int)t->N;
    return c;
}

int launch_count(rcb_tree *t, const NbCtx &c) {
    const int nsm = sm_count_nb();
    const size_t smem = sizeof(NbSmem);
    const int blocks = std::max(1, std::min((t->nsinks + kNbWarps - 1) / kNbWarps, nsm * 8));
    RCB_CUDA_TRY(cudaFuncSetAttribute(k_nb_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_nb_count<<<blocks, kNbWarps * 32, smem, t->stream>>>(c); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

}  // namespace

int neighbour_counts(rcb_tree *t, int64_t *counts, int *status) {
    NbCtx c = make_nbctx(t);
    c.counts = counts;
    c.status = status;
    return launch_count(t, c);
}

int neighbours(rcb_tree *t, int64_t *offsets, int32_t *idx, int64_t capacity, int64_t *needed) {
    cudaStream_t st = t->stream;
    NbCtx c = make_nbctx(t);
    const int nsm = sm_count_nb();
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_status + ST_NBFALLBACK, 0, 2 * sizeof(int), st));
    if (!t->nb_valid) {
        stage_begin(t, SG_NB_COUNT);
        // per-sink mask sizes and offsets; (re)allocate the mask buffer when it is too small
        int64_t *words = t->nb_count;  // scratch until the count pass overwrites it
        const int gw = std::max(1, std::min((t->nsinks + 7) / 8, nsm * 16));
        k_nb_sizes<<<gw, 256, 0, st>>>(c, words); note_launch();
        int rc = scan_i64(words, t->nb_maskoff, t->nsinks, t->nb_maskoff + t->nsinks, t->scan_tmp, st);
        if (rc) return rc;
        int64_t total_words = 0;
        RCB_CUDA_TRY(cudaMemcpyAsync(&total_words, t->nb_maskoff + t->nsinks, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        RCB_CUDA_TRY(cudaStreamSynchronize(st));
        if (total_words > t->cap_masks) {
            dev_free(t, t->nb_masks);
            const int64_t cap = total_words + total_words / 8 + 1024;
            t->nb_masks = (uint32_t *)dev_alloc(t, cap * sizeof(uint32_t));
            if (!t->nb_masks) {
                t->cap_masks = 0;
                return RCB_ERR_ALLOC;
            }
            t->cap_masks = cap;
        }
        c.mask_off = t->nb_maskoff;
        c.masks = t->nb_masks;
        rc = launch_count(t, c);
        if (rc) return rc;
        rc = scan_i64(t->nb_count, t->nb_count, t->N, t->nb_count + t->N, t->scan_tmp, st);
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
    c.offsets = offsets;
    c.idx = idx;
    c.mask_off = t->nb_maskoff;
    c.masks = t->nb_masks;
    stage_begin(t, SG_NB_FILL);
    // warps per block such that every warp's cell table (cap_near cells) and row fit
    const size_t per_warp = (2 * (size_t)t->cap_near + kRowWarp) * sizeof(int32_t);
    int warps = kNbWarps;
    while (warps > 1 && per_warp * warps > 200 * 1024) warps >>= 1;
    if (per_warp * warps > 227 * 1024) return RCB_ERR_LIMIT;
    const size_t smem = per_warp * warps;
    RCB_CUDA_TRY(cudaFuncSetAttribute(k_nb_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int blocks = std::max(1, std::min((t->nsinks + warps - 1) / warps, nsm * 8));
    k_nb_fill<<<blocks, warps * 32, smem, st>>>(c, t->cap_near); note_launch();
    stage_end(t, SG_NB_FILL);
    stage_begin(t, SG_NB_SORT);
    k_sort_long<<<std::max(1, nsm * 2), 1024, 0, st>>>(offsets, idx, t->nb_long, t->d_status + ST_LONGROWS,
                                                        (int)t->N); note_launch();
    stage_end(t, SG_NB_SORT);
    RCB_CUDA_TRY(cudaGetLastError());
    RCB_CUDA_TRY(cudaStreamSynchronize(st));
    return RCB_OK;
}

}  // namespace rcb
