// Tree build (Sec. 2.1) on the GPU.
//
// Data flow (all in device memory, one stream):
//   ingest      validate inputs; per-axis fixed-point exponents; SoA records (x, y, z, the four
//               62-bit fixed-point integers of m and m x, original index) in buffer 0; root sums
//   level pass  for every cell larger than kTcta particles: per-chunk counts and partial sums of
//               the left part (reduce), per-cell chunk offsets and both children's exact sums,
//               boxes, centres of mass and splits (finalize), then a stable scatter of the
//               chunk's records into the other buffer (scatter).  Cells that become small are
//               queued as subtree roots.
//   subtree     one CTA per queued root loads its <= kTcta records into shared memory and
//               splits them level by level down to L (flags, block scan, stable move, exact
//               children reductions), then writes the particles in tree order.
//   median      (median position split only) before a level pass, the key of rank floor(n/2)
//               along each large cell's axis by an exact radix selection, and in the subtree
//               kernel by counting ranks in shared memory; it replaces the centre-of-mass split
//   leaves      per non-empty ll-cell: Eq. 1 quadrupole, radii h_node_int and h_node, float32
//               cell-relative copies; then an arrival-counter climb computes every parent by
//               Eq. 2 as soon as both of its children are done.
// Every comparison of coordinates runs on order-preserving int64 keys; centre-of-mass sums are
// exact 128-bit integer sums, so the particle sets of all cells are a pure function of the
// input (Sec. 2.1.3-2.1.4 with the exact centre of mass).
#include <cuda_runtime.h>

#include <algorithm>

#include "rcb_internal.cuh"

namespace rcb {
namespace {

struct Red {  // exact reduction of a particle set
    i128 S[4];
    int64_t lo[3], hi[3];
    int32_t n;
};

__device__ inline void red_init(Red &r) {
    for (int k = 0; k < 4; ++k) r.S[k] = 0;
    for (int d = 0; d < 3; ++d) { r.lo[d] = INT64_MAX; r.hi[d] = INT64_MIN; }
    r.n = 0;
}

__device__ inline void red_add_particle(Red &r, const int64_t P[4], const int64_t key[3]) {
    for (int k = 0; k < 4; ++k) r.S[k] += (i128)P[k];
    for (int d = 0; d < 3; ++d) {
        r.lo[d] = min(r.lo[d], key[d]);
        r.hi[d] = max(r.hi[d], key[d]);
    }
    r.n += 1;
}

__device__ inline void red_merge(Red &a, const Red &b) {
    for (int k = 0; k < 4; ++k) a.S[k] += b.S[k];
    for (int d = 0; d < 3; ++d) {
        a.lo[d] = min(a.lo[d], b.lo[d]);
        a.hi[d] = max(a.hi[d], b.hi[d]);
    }
    a.n += b.n;
}

__device__ inline int64_t shfl_xor_ll(int64_t v, int m) {
    return (int64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, m);
}
__device__ inline int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ inline int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ inline void red_warp_allreduce(Red &r) {
    for (int m = 16; m >= 1; m >>= 1) {
        Red o;
        for (int k = 0; k < 4; ++k) o.S[k] = shfl_xor_i128(r.S[k], m);
        for (int d = 0; d < 3; ++d) {
            o.lo[d] = shfl_xor_ll(r.lo[d], m);
            o.hi[d] = shfl_xor_ll(r.hi[d], m);
        }
        o.n = __shfl_xor_sync(0xffffffffu, r.n, m);
        red_merge(r, o);
    }
}

// Block-wide reduction; every thread gets the result.  `scratch` holds blockDim/32 Reds.
__device__ void red_block(Red &r, Red *scratch) {
    red_warp_allreduce(r);
    int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) scratch[w] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        Red t = scratch[0];
        for (int i = 1; i < nw; ++i) red_merge(t, scratch[i]);
        scratch[0] = t;
    }
    __syncthreads();
    r = scratch[0];
    __syncthreads();
}

struct Ctx {  // device-side view of the tree arrays used by the build kernels
    int L;
    int mps;  // median position split instead of the centre-of-mass split
    int64_t capN;
    int64_t cap_big, cap_roots;
    int *status;
    const int *E;
    int32_t *nfirst, *ncount, *naxis;
    double *nsplit;
    int64_t *nsplitkey;
    i128 *nS;
    int64_t *nbmin, *nbmax;
    double *nmass, *ncom, *nrg, *nH;
};

// Write a cell created at `level` from its exact reduction: sums, box, centre of mass,
// geometric centre, size and (above the lowest level) the split of Sec. 2.1.3.
__device__ void write_cell(const Ctx &c, int node, int level, int first, const Red &r) {
    c.nfirst[node] = first;
    c.ncount[node] = r.n;
    if (r.n == 0) return;
    for (int k = 0; k < 4; ++k) c.nS[4 * (int64_t)node + k] = r.S[k];
    double ext[3];
    double H = 0.0;
    const double mass = mass_from_sum(r.S[0], c.E[3]);
    for (int d = 0; d < 3; ++d) {
        c.nbmin[3 * (int64_t)node + d] = r.lo[d];
        c.nbmax[3 * (int64_t)node + d] = r.hi[d];
        double lo = dkey_inv(r.lo[d]), hi = dkey_inv(r.hi[d]);
        c.ncom[3 * (int64_t)node + d] = com_from_sums_m(r.S[1 + d], c.E[d], mass);
        c.nrg[3 * (int64_t)node + d] = __dmul_rn(0.5, __dadd_rn(lo, hi));
        ext[d] = __dsub_rn(hi, lo);
        H = fmax(H, ext[d]);
    }
    c.nmass[node] = mass;
    c.nH[node] = H;
    if (level < c.L) {
        int ax = 0;
        double best = -1.0;
        for (int d = 0; d < 3; ++d)
            if (ext[d] > best) { best = ext[d]; ax = d; }  // ties -> lowest axis
        double s = c.ncom[3 * (int64_t)node + ax];
        c.naxis[node] = ax;
        c.nsplit[node] = s;
        c.nsplitkey[node] = dkey(s);
    }
}

// ------------------------------------------------------------------------------------------
// Ingest.

__global__ void k_ingest_scan(const double *__restrict__ x, const double *__restrict__ m,
                              const double *__restrict__ h, int64_t N, int *status,
                              unsigned long long *maxbits) {
    unsigned long long mx[4] = {0, 0, 0, 0};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double mi = m[i], hi = h[i];
        if (!isfinite(mi) || !(mi > 0.0) || !isfinite(hi) || !(hi > 0.0)) bad = true;
        for (int d = 0; d < 3; ++d) {
            double xi = x[3 * i + d];
            if (!isfinite(xi)) bad = true;
            double p = fabs(__dmul_rn(mi, __dadd_rn(xi, 0.0)));
            unsigned long long b = (unsigned long long)__double_as_longlong(p);
            if (isfinite(p) && b > mx[d]) mx[d] = b;
        }
        unsigned long long bm = (unsigned long long)__double_as_longlong(mi);
        if (mi > 0.0 && isfinite(mi) && bm > mx[3]) mx[3] = bm;
    }
    for (int k = 0; k < 4; ++k) {
        unsigned long long v = mx[k];
        for (int o = 16; o >= 1; o >>= 1) {
            unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
        if ((threadIdx.x & 31) == 0 && v) atomicMax(&maxbits[k], v);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&status[ST_ERR], ERRBIT_ARG);
}

__global__ void k_exponents(const unsigned long long *maxbits, int *E) {
    if (threadIdx.x < 4) {
        double v = __longlong_as_double((long long)maxbits[threadIdx.x]);
        int e = 0;
        if (v != 0.0) (void)frexp(v, &e);
        E[threadIdx.x] = e;
    }
}

__global__ void k_ingest_write(const double *__restrict__ x, const double *__restrict__ m, int64_t N, int64_t capN,
                               const int *E, double *__restrict__ bx, double *__restrict__ by,
                               double *__restrict__ bz, int64_t *__restrict__ bP, int32_t *__restrict__ bidx,
                               Red *partials, int *status) {
    __shared__ Red scratch[32];
    Red r;
    red_init(r);
    int sh[4] = {62 - E[0], 62 - E[1], 62 - E[2], 62 - E[3]};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double mi = m[i];
        double xc[3];
        int64_t P[4], key[3];
        for (int d = 0; d < 3; ++d) {
            xc[d] = __dadd_rn(x[3 * i + d], 0.0);  // -0 -> +0
            key[d] = dkey(xc[d]);
            P[1 + d] = fixed_point(__dmul_rn(mi, xc[d]), sh[d]);
        }
        P[0] = fixed_point(mi, sh[3]);
        if (P[0] < 1) bad = true;
        bx[i] = xc[0];
        by[i] = xc[1];
        bz[i] = xc[2];
        for (int k = 0; k < 4; ++k) bP[k * capN + i] = P[k];
        bidx[i] = (int32_t)i;
        red_add_particle(r, P, key);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&status[ST_ERR], ERRBIT_FIXED);
    red_block(r, scratch);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

// Root cell (level 0) from the ingest partials; queue it as a large cell or a subtree root.
__global__ void k_root_finalize(Ctx c, const Red *partials, int nparts, int32_t *big_list, int32_t *roots,
                                int32_t *nbig_lvl) {
    __shared__ Red scratch[32];
    Red r;
    red_init(r);
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) red_merge(r, partials[i]);
    red_block(r, scratch);
    if (threadIdx.x == 0) {
        write_cell(c, 1, 0, 0, r);
        if (r.n > kTcta && c.L > 0) {
            big_list[0] = 1;
            c.status[ST_NBIG] = 1;
            nbig_lvl[0] = 1;
        } else {
            roots[0] = (1 << 1) | 0;
            c.status[ST_NROOTS] = 1;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Level passes over large cells.

struct ChunkPart {
    i128 SL[4];
    int64_t loL[3], hiL[3], loR[3], hiR[3];
    int32_t nL;
    int32_t leftoff;
};

// Chunk list of the large cells of one level (single block).
__global__ void k_chunk_plan(const int32_t *big, const int32_t *nbig_ptr, const int32_t *nfirst, const int32_t *ncount,
                             int32_t *cell_chunk0, int4 *chunks, int *status) {
    const int nbig = *nbig_ptr;
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nbig; base += blockDim.x) {
        int i = base + threadIdx.x;
        int nch = 0;
        if (i < nbig) nch = (ncount[big[i]] + kChunk - 1) / kChunk;
        // block exclusive scan of nch
        int v = nch;
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) warp_tot[w] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                int t = warp_tot[k];
                warp_tot[k] = s;
                s += t;
            }
        }
        __syncthreads();
        int excl = carry + warp_tot[w] + v - nch;
        if (i < nbig) {
            int node = big[i];
            int f = nfirst[node], cnt = ncount[node];
            cell_chunk0[i] = excl;
            for (int k = 0; k < nch; ++k) {
                int st = f + k * kChunk;
                chunks[excl + k] = make_int4(node, st, min(kChunk, f + cnt - st), i);
            }
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + nch;
        __syncthreads();
    }
    if (threadIdx.x == 0) status[ST_NCHUNKS] = carry;
}

// Per chunk: number of particles left of the split, their exact sums, and both sides' boxes.
__global__ void __launch_bounds__(kChunkThreads)
    k_level_reduce(Ctx c, const int4 *chunks, const int *nchunks_ptr, const double *__restrict__ bx,
                   const double *__restrict__ by, const double *__restrict__ bz, const int64_t *__restrict__ bP,
                   ChunkPart *parts) {
    __shared__ Red scratch[kChunkThreads / 32];
    int nchunks = *nchunks_ptr;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        int4 cd = chunks[ch];
        int node = cd.x, start = cd.y, cnt = cd.z;
        int ax = c.naxis[node];
        int64_t sk = c.nsplitkey[node];
        Red rl, rr;
        red_init(rl);
        red_init(rr);
        // the chunk's elements, kChunk / kChunkThreads per thread, in batches of four whose loads
        // are all issued before their arithmetic
        constexpr int kPer = kChunk / kChunkThreads, kBatch = 4;
#pragma unroll
        for (int j0 = 0; j0 < kPer; j0 += kBatch) {
            double vx[kBatch], vy[kBatch], vz[kBatch];
            int64_t vP[kBatch][4];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int i = threadIdx.x + (j0 + u) * kChunkThreads;
                if (i < cnt) {
                    const int64_t e = start + i;
                    vx[u] = bx[e];
                    vy[u] = by[e];
                    vz[u] = bz[e];
#pragma unroll
                    for (int k = 0; k < 4; ++k) vP[u][k] = bP[k * c.capN + e];
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int i = threadIdx.x + (j0 + u) * kChunkThreads;
                if (i < cnt) {
                    int64_t key[3] = {dkey(vx[u]), dkey(vy[u]), dkey(vz[u])};
                    if (key[ax] < sk) red_add_particle(rl, vP[u], key);
                    else {
                        for (int d = 0; d < 3; ++d) {
                            rr.lo[d] = min(rr.lo[d], key[d]);
                            rr.hi[d] = max(rr.hi[d], key[d]);
                        }
                    }
                }
            }
        }
        red_block(rl, scratch);
        // right side: only the box is needed (its sums are parent minus left)
        for (int m = 16; m >= 1; m >>= 1)
            for (int d = 0; d < 3; ++d) {
                rr.lo[d] = min64(rr.lo[d], shfl_xor_ll(rr.lo[d], m));
                rr.hi[d] = max64(rr.hi[d], shfl_xor_ll(rr.hi[d], m));
            }
        __shared__ int64_t boxR[kChunkThreads / 32][6];
        int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0)
            for (int d = 0; d < 3; ++d) { boxR[w][d] = rr.lo[d]; boxR[w][3 + d] = rr.hi[d]; }
        __syncthreads();
        if (threadIdx.x == 0) {
            ChunkPart p;
            for (int k = 0; k < 4; ++k) p.SL[k] = rl.S[k];
            for (int d = 0; d < 3; ++d) {
                p.loL[d] = rl.lo[d];
                p.hiL[d] = rl.hi[d];
                int64_t lo = INT64_MAX, hi = INT64_MIN;
                for (int k = 0; k < kChunkThreads / 32; ++k) {
                    lo = min(lo, boxR[k][d]);
                    hi = max(hi, boxR[k][3 + d]);
                }
                p.loR[d] = lo;
                p.hiR[d] = hi;
            }
            p.nL = rl.n;
            p.leftoff = 0;
            parts[ch] = p;
        }
        __syncthreads();
    }
}

// Per large cell (one warp each): chunk offsets, both children, and their classification.
__global__ void k_level_finalize(Ctx c, int level, const int32_t *big, const int32_t *nbig_ptr,
                                 const int32_t *cell_chunk0, const int *nchunks_ptr, ChunkPart *parts,
                                 int32_t *big_next, int32_t *nbig_next, int32_t *roots, int parity_next) {
    const int nbig = *nbig_ptr;
    int lane = threadIdx.x & 31;
    int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nw = (gridDim.x * blockDim.x) >> 5;
    int nchunks = *nchunks_ptr;
    for (int i = gw; i < nbig; i += nw) {
        int node = big[i];
        int f = c.nfirst[node], cnt = c.ncount[node];
        int c0 = cell_chunk0[i];
        int nch = (cnt + kChunk - 1) / kChunk;
        if (c0 + nch > nchunks) {  // inconsistent plan: report, do not touch memory
            if (lane == 0) atomicOr(&c.status[ST_ERR], ERRBIT_STATE);
            continue;
        }
        Red L;
        red_init(L);
        int64_t loR[3], hiR[3];
        for (int d = 0; d < 3; ++d) { loR[d] = INT64_MAX; hiR[d] = INT64_MIN; }
        int run = 0;  // left particles before the current group of 32 chunks
        for (int base = 0; base < nch; base += 32) {
            int k = base + lane;
            int nl = 0;
            if (k < nch) {
                const ChunkPart &p = parts[c0 + k];
                nl = p.nL;
                Red t;
                for (int q = 0; q < 4; ++q) t.S[q] = p.SL[q];
                for (int d = 0; d < 3; ++d) {
                    t.lo[d] = p.loL[d];
                    t.hi[d] = p.hiL[d];
                    loR[d] = min(loR[d], p.loR[d]);
                    hiR[d] = max(hiR[d], p.hiR[d]);
                }
                t.n = nl;
                red_merge(L, t);
            }
            int v = nl;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            if (k < nch) parts[c0 + k].leftoff = run + v - nl;
            run += __shfl_sync(0xffffffffu, v, 31);
        }
        red_warp_allreduce(L);
        for (int m = 16; m >= 1; m >>= 1)
            for (int d = 0; d < 3; ++d) {
                loR[d] = min64(loR[d], shfl_xor_ll(loR[d], m));
                hiR[d] = max64(hiR[d], shfl_xor_ll(hiR[d], m));
            }
        // both children at once (lanes 0 and 1): the float64 work of write_cell costs the same
        // per warp instruction with one active lane as with two
        if (lane < 2) {
            Red X = L;  // lane 0: the left child; lane 1: the right child
            if (lane == 1) {
                for (int q = 0; q < 4; ++q) X.S[q] = c.nS[4 * (int64_t)node + q] - L.S[q];
                for (int d = 0; d < 3; ++d) { X.lo[d] = loR[d]; X.hi[d] = hiR[d]; }
                X.n = cnt - L.n;
            }
            write_cell(c, 2 * node + lane, level + 1, lane == 0 ? f : f + L.n, X);
        }
        if (lane == 0) {
            int kids[2] = {2 * node, 2 * node + 1};
            int kn[2] = {L.n, cnt - L.n};
            for (int s = 0; s < 2; ++s) {
                if (kn[s] == 0) continue;
                if (kn[s] > kTcta && level + 1 < c.L) {
                    int slot = atomicAdd(nbig_next, 1);
                    if (slot < c.cap_big) big_next[slot] = kids[s];
                    else atomicOr(&c.status[ST_ERR], ERRBIT_STATE);
                } else {
                    int slot = atomicAdd(&c.status[ST_NROOTS], 1);
                    if (slot < c.cap_roots) roots[slot] = (kids[s] << 1) | parity_next;
                    else atomicOr(&c.status[ST_ERR], ERRBIT_STATE);
                }
            }
        }
    }
}

// Stable scatter of each chunk's records to their children's ranges in the other buffer.
__global__ void __launch_bounds__(kChunkThreads)
    k_level_scatter(Ctx c, const int4 *chunks, const int *nchunks_ptr, const ChunkPart *parts,
                    const double *__restrict__ bx, const double *__restrict__ by, const double *__restrict__ bz,
                    const int64_t *__restrict__ bP, const int32_t *__restrict__ bidx, double *__restrict__ ox,
                    double *__restrict__ oy, double *__restrict__ oz, int64_t *__restrict__ oP,
                    int32_t *__restrict__ oidx) {
    __shared__ int wsum[kChunkThreads / 32];
    int nchunks = *nchunks_ptr;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int kPer = kChunk / kChunkThreads;  // elements per thread (8)
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        int4 cd = chunks[ch];
        int node = cd.x, start = cd.y, cnt = cd.z;
        int ax = c.naxis[node];
        int64_t sk = c.nsplitkey[node];
        int f = c.nfirst[node];
        int nLcell = c.ncount[2 * node];
        int leftoff = parts[ch].leftoff;
        int rightoff = (start - f) - leftoff;
        // element order: warp w owns [w*256, w*256+256), group j = 32 consecutive elements
        unsigned masks[kPer];
        int wcount = 0;
        for (int j = 0; j < kPer; ++j) {
            int i = w * 32 * kPer + j * 32 + lane;
            bool left = false;
            if (i < cnt) {
                int64_t e = start + i;
                double v = ax == 0 ? bx[e] : (ax == 1 ? by[e] : bz[e]);
                left = dkey(v) < sk;
            }
            masks[j] = __ballot_sync(0xffffffffu, left);
            wcount += __popc(masks[j]);
        }
        if (lane == 0) wsum[w] = wcount;
        __syncthreads();
        int before = 0;
        for (int k = 0; k < w; ++k) before += wsum[k];
        __syncthreads();
        unsigned lt = (1u << lane) - 1u;
        int run = before;
        // two batches of four elements: every field load of a batch is issued before its stores
        constexpr int kBatch = 4;
#pragma unroll
        for (int j0 = 0; j0 < kPer; j0 += kBatch) {
            double vx[kBatch], vy[kBatch], vz[kBatch];
            int64_t vP[kBatch][4];
            int32_t vi[kBatch];
            int64_t dst[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int j = j0 + u;
                const int i = w * 32 * kPer + j * 32 + lane;
                const bool left = (masks[j] >> lane) & 1u;
                const int lrank = run + __popc(masks[j] & lt);
                run += __popc(masks[j]);
                dst[u] = left ? (int64_t)f + leftoff + lrank : (int64_t)f + nLcell + rightoff + (i - lrank);
                if (i < cnt) {
                    const int64_t e = start + i;
                    vx[u] = bx[e];
                    vy[u] = by[e];
                    vz[u] = bz[e];
#pragma unroll
                    for (int k = 0; k < 4; ++k) vP[u][k] = bP[k * c.capN + e];
                    vi[u] = bidx[e];
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int i = w * 32 * kPer + (j0 + u) * 32 + lane;
                if (i < cnt) {
                    ox[dst[u]] = vx[u];
                    oy[dst[u]] = vy[u];
                    oz[dst[u]] = vz[u];
#pragma unroll
                    for (int k = 0; k < 4; ++k) oP[k * c.capN + dst[u]] = vP[u][k];
                    oidx[dst[u]] = vi[u];
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Median position split of the large cells of one level (Sec. 2.1.3 variant).  The split key is
// the order statistic of rank floor(n/2) of the cell's keys along its axis, found by an exact
// radix selection: eight rounds of one 8-bit digit each, from the most significant.  In a round
// every chunk histograms the digit of those keys that match the prefix chosen so far (k_mps_hist),
// then one warp per cell finds the digit whose bin holds the rank still sought (k_mps_pick).
// Keys are dkey with the sign bit flipped, so that unsigned order is coordinate order.

constexpr int kMpsBins = 256;

__device__ inline unsigned long long mps_ukey(double v) {
    return (unsigned long long)dkey(v) ^ 0x8000000000000000ull;
}

__global__ void __launch_bounds__(kChunkThreads)
    k_mps_hist(Ctx c, const int4 *chunks, const int *nchunks_ptr, const double *__restrict__ bx,
               const double *__restrict__ by, const double *__restrict__ bz, const unsigned long long *prefix,
               int shift, int32_t *hist) {
    __shared__ int32_t h[kMpsBins];
    const int nchunks = *nchunks_ptr;
    const bool first_round = shift >= 56;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        for (int i = threadIdx.x; i < kMpsBins; i += blockDim.x) h[i] = 0;
        __syncthreads();
        const int4 cd = chunks[ch];
        const int node = cd.x, start = cd.y, cnt = cd.z, cell = cd.w;
        const int ax = c.naxis[node];
        const double *b = ax == 0 ? bx : (ax == 1 ? by : bz);
        const unsigned long long high = first_round ? 0ull : prefix[cell] >> (shift + 8);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const unsigned long long u = mps_ukey(b[start + i]);
            if (first_round || (u >> (shift + 8)) == high) atomicAdd(&h[(u >> shift) & (kMpsBins - 1)], 1);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kMpsBins; i += blockDim.x)
            if (h[i]) atomicAdd(&hist[(int64_t)cell * kMpsBins + i], h[i]);
        __syncthreads();
    }
}

// One warp per large cell: the digit holding the sought rank; clears the cell's bins for the next
// round.  After the last round the prefix is the split key.
__global__ void k_mps_pick(Ctx c, const int32_t *big, const int32_t *nbig_ptr, int shift, int32_t *hist,
                           unsigned long long *prefix, int32_t *rank) {
    const int nbig = *nbig_ptr;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < nbig; i += nw) {
        const int node = big[i];
        int r = shift >= 56 ? c.ncount[node] / 2 : rank[i];
        unsigned long long pre = shift >= 56 ? 0ull : prefix[i];
        int32_t *hc = hist + (int64_t)i * kMpsBins;
        int v[kMpsBins / 32];
        int tot = 0;
#pragma unroll
        for (int k = 0; k < kMpsBins / 32; ++k) {
            v[k] = hc[(kMpsBins / 32) * lane + k];
            hc[(kMpsBins / 32) * lane + k] = 0;
            tot += v[k];
        }
        int incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int excl = incl - tot;
        const bool mine = r >= excl && r < incl;
        const unsigned ball = __ballot_sync(0xffffffffu, mine);
        if (ball == 0u) {  // the histogram does not hold the rank: inconsistent state, report
            if (lane == 0) atomicOr(&c.status[ST_ERR], ERRBIT_STATE);
            continue;
        }
        int digit = 0, before = 0;
        if (mine) {
            int acc = excl;
#pragma unroll
            for (int k = 0; k < kMpsBins / 32; ++k) {
                if (r < acc + v[k]) {
                    digit = (kMpsBins / 32) * lane + k;
                    before = acc;
                    break;
                }
                acc += v[k];
            }
        }
        const int src = __ffs(ball) - 1;
        digit = __shfl_sync(0xffffffffu, digit, src);
        before = __shfl_sync(0xffffffffu, before, src);
        r -= before;
        pre |= (unsigned long long)digit << shift;
        if (lane == 0) {
            rank[i] = r;
            prefix[i] = pre;
            if (shift == 0) {
                const int64_t key = (int64_t)(pre ^ 0x8000000000000000ull);
                c.nsplitkey[node] = key;
                c.nsplit[node] = dkey_inv(key);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Subtrees in shared memory.

struct SubtreeSmem {
    double x[kTcta], y[kTcta], z[kTcta];
    int64_t P[4][kTcta];
    int32_t idx[kTcta];
    uint16_t perm[2][kTcta];
    uint16_t cellOf[2][kTcta];
    uint16_t scan[kTcta + 1];
    int32_t cnode[2][kTcta];
    uint16_t cfirst[2][kTcta], ccount[2][kTcta];
    int64_t csplit[kTcta];
    int8_t caxis[kTcta];
    union {
        struct {
            uint16_t newidx[2 * kTcta];
            // reductions of the children larger than 32 particles (at most kTcta / 33 of them),
            // written out together by one warp
            Red bred[32];
        };
        // median split: every particle's key along its cell's axis, by position (newidx and
        // bred are dead whenever subtree_median runs)
        int64_t mkey[kTcta];
    };
    int bci[32];
    int nbred;
    int warp_tot[33];
    int nkids;
};

// Block exclusive scan of per-thread value v; returns this thread's exclusive prefix and writes
// the block total to *total.  warp_tot holds 33 ints.
__device__ int block_excl_scan(int v, int *warp_tot, int *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            int t = warp_tot[k];
            warp_tot[k] = s;
            s += t;
        }
        warp_tot[32] = s;
    }
    __syncthreads();
    int excl = warp_tot[w] + incl - v;
    *total = warp_tot[32];
    __syncthreads();
    return excl;
}

__device__ inline void load_particle(const SubtreeSmem &s, int home, int64_t P[4], int64_t key[3]) {
    for (int k = 0; k < 4; ++k) P[k] = s.P[k][home];
    key[0] = dkey(s.x[home]);
    key[1] = dkey(s.y[home]);
    key[2] = dkey(s.z[home]);
}

struct Bufs {
    const double *x[2], *y[2], *z[2];
    const int64_t *P[2];
    const int32_t *idx[2];
};

// Median position split of every cell of order `cur` (all of them internal): each particle's rank
// along its cell's axis, ties broken by position; the particle of rank floor(n/2) writes its key
// as the cell's split (exactly one per cell).
__device__ void subtree_median(const Ctx &c, SubtreeSmem &s, int cur, int n) {
    // the keys first, in position order, so that the rank count reads one key per comparison
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int ax = s.caxis[s.cellOf[cur][p]];
        const double *coord = ax == 0 ? s.x : (ax == 1 ? s.y : s.z);
        s.mkey[p] = dkey(coord[s.perm[cur][p]]);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int ci = s.cellOf[cur][p];
        const int f = s.cfirst[cur][ci], cn = s.ccount[cur][ci];
        const int64_t kp = s.mkey[p];
        int below = 0;
        for (int q = f; q < f + cn; ++q) {
            const int64_t kq = s.mkey[q];
            below += (kq < kp) || (kq == kp && q < p);
        }
        if (below == cn / 2) {
            const int node = s.cnode[cur][ci];
            s.csplit[ci] = kp;
            c.nsplitkey[node] = kp;
            c.nsplit[node] = dkey_inv(kp);
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kCtaThreads, 2)
    k_subtree(Ctx c, const int32_t *roots, const int *nroots_ptr, Bufs B, const double *__restrict__ m_in,
              const double *__restrict__ h_in, double *__restrict__ px, double *__restrict__ py,
              double *__restrict__ pz, double *__restrict__ pm, double *__restrict__ ph,
              int32_t *__restrict__ pidx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SubtreeSmem &s = *reinterpret_cast<SubtreeSmem *>(smem_raw);
    const int nroots = *nroots_ptr;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    for (int ri = blockIdx.x; ri < nroots; ri += gridDim.x) {
        int packed = roots[ri];
        int root = packed >> 1, parity = packed & 1;
        int k0 = 31 - __clz(root);
        int gfirst = c.nfirst[root], n = c.ncount[root];
        const double *bx = B.x[parity], *by = B.y[parity], *bz = B.z[parity];
        const int64_t *bP = B.P[parity];
        const int32_t *bidx = B.idx[parity];
        if (k0 >= c.L || n > kTcta) {
            // an ll-cell: its particles only need to reach the output arrays
            for (int i = tid; i < n; i += nt) {
                int64_t e = gfirst + i;
                int32_t o = bidx[e];
                px[e] = bx[e];
                py[e] = by[e];
                pz[e] = bz[e];
                pidx[e] = o;
                pm[e] = m_in[o];
                ph[e] = h_in[o];
            }
            continue;
        }
        for (int i = tid; i < n; i += nt) {
            int64_t e = gfirst + i;
            s.x[i] = bx[e];
            s.y[i] = by[e];
            s.z[i] = bz[e];
            for (int k = 0; k < 4; ++k) s.P[k][i] = bP[k * c.capN + e];
            s.idx[i] = bidx[e];
            s.perm[0][i] = (uint16_t)i;
            s.cellOf[0][i] = 0;
        }
        if (tid == 0) {
            s.cnode[0][0] = root;
            s.cfirst[0][0] = 0;
            s.ccount[0][0] = (uint16_t)n;
            s.caxis[0] = (int8_t)c.naxis[root];
            s.csplit[0] = c.nsplitkey[root];
            s.nkids = 1;
        }
        __syncthreads();
        if (c.mps) subtree_median(c, s, 0, n);
        int cur = 0;
        int K = 1;
        for (int level = k0; level < c.L; ++level) {
            const int nxt = cur ^ 1;
            // 1. flags of the positions this thread owns (4 consecutive), block scan
            constexpr int kPer = kTcta / kCtaThreads;
            bool fl[kPer];
            int cntl = 0;
            for (int j = 0; j < kPer; ++j) {
                int p = tid * kPer + j;
                bool left = false;
                if (p < n) {
                    int ci = s.cellOf[cur][p];
                    int home = s.perm[cur][p];
                    int ax = s.caxis[ci];
                    double v = ax == 0 ? s.x[home] : (ax == 1 ? s.y[home] : s.z[home]);
                    left = dkey(v) < s.csplit[ci];
                }
                fl[j] = left;
                cntl += left;
            }
            int total;
            int excl = block_excl_scan(cntl, s.warp_tot, &total);
            for (int j = 0; j < kPer; ++j) {
                int p = tid * kPer + j;
                if (p < n) s.scan[p] = (uint16_t)excl;
                excl += fl[j];
            }
            if (tid == 0) s.scan[n] = (uint16_t)total;
            __syncthreads();
            // 2. children of every active cell; compact the non-empty ones
            int nonempty_local = 0;
            constexpr int kCellPer = 2 * kTcta / kCtaThreads;  // 8 child slots per thread
            uint16_t cl[kCellPer];
            for (int j = 0; j < kCellPer; ++j) {
                int slot = tid * kCellPer + j;  // child slot = 2 * cell + side
                uint16_t cc = 0;
                if (slot < 2 * K) {
                    int ci = slot >> 1;
                    int f = s.cfirst[cur][ci], cn = s.ccount[cur][ci];
                    int nl = s.scan[f + cn] - s.scan[f];
                    cc = (slot & 1) ? (uint16_t)(cn - nl) : (uint16_t)nl;
                }
                cl[j] = cc;
                nonempty_local += cc > 0;
            }
            int kexcl = block_excl_scan(nonempty_local, s.warp_tot, &total);
            for (int j = 0; j < kCellPer; ++j) {
                int slot = tid * kCellPer + j;
                if (slot < 2 * K) {
                    int ci = slot >> 1;
                    if (cl[j] > 0) {
                        int f = s.cfirst[cur][ci];
                        int nl = s.scan[f + s.ccount[cur][ci]] - s.scan[f];
                        s.newidx[slot] = (uint16_t)kexcl;
                        s.cnode[nxt][kexcl] = 2 * s.cnode[cur][ci] + (slot & 1);
                        s.cfirst[nxt][kexcl] = (uint16_t)((slot & 1) ? f + nl : f);
                        s.ccount[nxt][kexcl] = cl[j];
                        ++kexcl;
                    } else {
                        // an empty child: record its placement only
                        int node = 2 * s.cnode[cur][ci] + (slot & 1);
                        int f = s.cfirst[cur][ci];
                        int nl = s.scan[f + s.ccount[cur][ci]] - s.scan[f];
                        c.nfirst[node] = gfirst + ((slot & 1) ? f + nl : f);
                    }
                }
            }
            const int K2 = total;
            __syncthreads();
            // 3. stable move into the next order
            for (int j = 0; j < kPer; ++j) {
                int p = tid * kPer + j;
                if (p < n) {
                    int ci = s.cellOf[cur][p];
                    int f = s.cfirst[cur][ci], cn = s.ccount[cur][ci];
                    int base = s.scan[f];
                    int nl = s.scan[f + cn] - base;
                    int r = s.scan[p] - base;
                    int np = fl[j] ? f + r : f + nl + (p - f - r);
                    s.perm[nxt][np] = s.perm[cur][p];
                    s.cellOf[nxt][np] = s.newidx[2 * ci + (fl[j] ? 0 : 1)];
                }
            }
            __syncthreads();
            // 4. exact reductions of the children: a warp for large ones (kept in shared memory),
            // a thread for small ones; then the cells, one thread each: the float64 arithmetic of
            // write_cell costs the same per warp instruction however few lanes are active, so the
            // large cells' are written together by the last warp
            if (tid == 0) s.nbred = 0;
            __syncthreads();
            for (int ci = warp; ci < K2; ci += nwarps) {
                int cn = s.ccount[nxt][ci];
                if (cn <= 32) continue;
                int f = s.cfirst[nxt][ci];
                Red r;
                red_init(r);
                for (int q = lane; q < cn; q += 32) {
                    int64_t P[4], key[3];
                    load_particle(s, s.perm[nxt][f + q], P, key);
                    red_add_particle(r, P, key);
                }
                red_warp_allreduce(r);
                if (lane == 0) {
                    const int slot = atomicAdd(&s.nbred, 1);  // < 32: every such cell holds > 32 of <= kTcta
                    s.bred[slot] = r;
                    s.bci[slot] = ci;
                }
            }
            __syncthreads();
            if (tid >= nt - 32 && tid - (nt - 32) < s.nbred) {
                const int slot = tid - (nt - 32), ci = s.bci[slot];
                const int node = s.cnode[nxt][ci];
                write_cell(c, node, level + 1, gfirst + s.cfirst[nxt][ci], s.bred[slot]);
                if (level + 1 < c.L) {
                    s.caxis[ci] = (int8_t)c.naxis[node];
                    s.csplit[ci] = c.nsplitkey[node];
                }
            }
            for (int ci = tid; ci < K2; ci += nt) {
                int cn = s.ccount[nxt][ci];
                if (cn > 32) continue;
                int f = s.cfirst[nxt][ci];
                Red r;
                red_init(r);
                for (int q = 0; q < cn; ++q) {
                    int64_t P[4], key[3];
                    load_particle(s, s.perm[nxt][f + q], P, key);
                    red_add_particle(r, P, key);
                }
                int node = s.cnode[nxt][ci];
                write_cell(c, node, level + 1, gfirst + f, r);
                if (level + 1 < c.L) {
                    s.caxis[ci] = (int8_t)c.naxis[node];
                    s.csplit[ci] = c.nsplitkey[node];
                }
            }
            __syncthreads();
            cur = nxt;
            K = K2;
            if (c.mps && level + 1 < c.L) subtree_median(c, s, cur, n);
        }
        // write the particles in tree order
        for (int p = tid; p < n; p += nt) {
            int home = s.perm[cur][p];
            int64_t e = gfirst + p;
            int32_t o = s.idx[home];
            px[e] = s.x[home];
            py[e] = s.y[home];
            pz[e] = s.z[home];
            pidx[e] = o;
            pm[e] = m_in[o];
            ph[e] = h_in[o];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// Sinks, leaf moments and the bottom-up pass.

__global__ void k_count_sinks(const int32_t *ncount, int64_t leaf0, int64_t nleaves, int32_t *flags) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nleaves; j += (int64_t)gridDim.x * blockDim.x)
        flags[j] = ncount[leaf0 + j] > 0;
}

__global__ void k_write_sinks(const int32_t *flags, const int32_t *pos, int64_t leaf0, int64_t nleaves,
                              int32_t *sinks, int32_t *sink_of_leaf) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nleaves; j += (int64_t)gridDim.x * blockDim.x) {
        if (flags[j]) {
            sinks[pos[j]] = (int32_t)(leaf0 + j);
            sink_of_leaf[j] = pos[j];
        } else {
            sink_of_leaf[j] = -1;
        }
    }
}

struct LeafCtx {
    int32_t *nfirst, *ncount;
    double *nmass, *ncom, *nrg, *nH, *nhint, *nhnode, *nQ;
    int32_t *narrive;
    const double *px, *py, *pz, *pm, *ph;
    float4 *p32;
    float *h32;
};

// Eq. 2 and the parent's enclosing radius from its non-empty children.
__device__ void parent_moments(const LeafCtx &c, int P) {
    double Q[6] = {0, 0, 0, 0, 0, 0};
    double hint = 0.0;
    double cp[3] = {__ldcg(&c.ncom[3 * (int64_t)P]), __ldcg(&c.ncom[3 * (int64_t)P + 1]), __ldcg(&c.ncom[3 * (int64_t)P + 2])};
    double gp[3] = {__ldcg(&c.nrg[3 * (int64_t)P]), __ldcg(&c.nrg[3 * (int64_t)P + 1]), __ldcg(&c.nrg[3 * (int64_t)P + 2])};
    for (int C = 2 * P; C <= 2 * P + 1; ++C) {
        if (__ldcg(&c.ncount[C]) == 0) continue;
        double dx[3];
        for (int d = 0; d < 3; ++d) dx[d] = __dsub_rn(__ldcg(&c.ncom[3 * (int64_t)C + d]), cp[d]);
        double dr2 = __dadd_rn(__dadd_rn(__dmul_rn(dx[0], dx[0]), __dmul_rn(dx[1], dx[1])), __dmul_rn(dx[2], dx[2]));
        double MC = __ldcg(&c.nmass[C]);
        double tM = __dmul_rn(3.0, MC);
        int k = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = i; j < 3; ++j, ++k) {
                double v = __ldcg(&c.nQ[6 * (int64_t)C + k]) + tM * dx[i] * dx[j];
                if (i == j) v -= MC * dr2;
                Q[k] += v;
            }
        double r = __dsqrt_rn(dist2_rn(gp[0], gp[1], gp[2], __ldcg(&c.nrg[3 * (int64_t)C]), __ldcg(&c.nrg[3 * (int64_t)C + 1]),
                                       __ldcg(&c.nrg[3 * (int64_t)C + 2])));
        r = __dadd_rn(r, __ldcg(&c.nhint[C]));
        hint = fmax(hint, r);
    }
    for (int k = 0; k < 6; ++k) c.nQ[6 * (int64_t)P + k] = Q[k];
    c.nhint[P] = hint;
    c.nhnode[P] = 0.0;
}

// One thread per sink: Eq. 1, radii, float32 copies.  FP64 runs at 1/66 of FP32 on this GPU, so
// the float64 work per particle is kept small: the quadrupole accumulates with fused
// multiply-adds (it is compared within a tolerance, not bit for bit), and the two radii are
// exact maxima found from float32 estimates: every distance estimate has relative error below
// 2^-21, so when the runner-up estimate is more than 2^-18 below the leader the exact maximum is
// the leader's (only it is evaluated in float64); otherwise every particle is.
//   h_int  = max_a |r_a - r_g|          (a correctly rounded square root is monotonic, so the
//                                        exact maximum of the squares gives the same double)
//   h_node = max_a (|r_a - r_g| + 2 h_a)
__global__ void k_leaves_up(LeafCtx c, const int32_t *sinks, int nsinks) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsinks) return;
    int n = sinks[s];
    int f = c.nfirst[n], cnt = c.ncount[n];
    // the particle arrays are read-only here and never alias the float32 copies written below
    const double *__restrict__ px = c.px, *__restrict__ py = c.py, *__restrict__ pz = c.pz;
    const double *__restrict__ pm = c.pm, *__restrict__ ph = c.ph;
    float4 *__restrict__ p32 = c.p32;
    float *__restrict__ h32 = c.h32;
    double com[3] = {c.ncom[3 * (int64_t)n], c.ncom[3 * (int64_t)n + 1], c.ncom[3 * (int64_t)n + 2]};
    double rg[3] = {c.nrg[3 * (int64_t)n], c.nrg[3 * (int64_t)n + 1], c.nrg[3 * (int64_t)n + 2]};
    // Eq. 1 as Q = 3 S - tr(S) I with S = sum m d d^T: one multiply per axis and six fused
    // multiply-adds per particle
    double S[6] = {0, 0, 0, 0, 0, 0};
    float i1 = -1.f, i2 = -1.f, e1 = -1.f, e2 = -1.f;  // largest and second largest estimates
    int ai = f, a1 = f;
    for (int a = f; a < f + cnt; ++a) {
        const double x = px[a], y = py[a], z = pz[a], m = pm[a], h = ph[a];
        const double dx = __dsub_rn(x, com[0]), dy = __dsub_rn(y, com[1]), dz = __dsub_rn(z, com[2]);
        const double mx = m * dx, my = m * dy, mz = m * dz;
        S[0] = fma(mx, dx, S[0]);
        S[1] = fma(mx, dy, S[1]);
        S[2] = fma(mx, dz, S[2]);
        S[3] = fma(my, dy, S[3]);
        S[4] = fma(my, dz, S[4]);
        S[5] = fma(mz, dz, S[5]);
        // r_a - r_g in float64, rounded once to float32 per component (relative error 2^-24 each),
        // so the float32 distance has relative error below 2^-21
        const float gx = __double2float_rn(__dsub_rn(x, rg[0])), gy = __double2float_rn(__dsub_rn(y, rg[1])),
                    gz = __double2float_rn(__dsub_rn(z, rg[2]));
        const float dg = __fsqrt_rn(fmaf(gz, gz, fmaf(gy, gy, gx * gx)));
        const float hf = __double2float_rn(h);
        const float est = __fadd_rn(dg, 2.0f * hf);  // 2 RN(h) = RN(2 h) exactly
        if (dg > i1) {
            i2 = i1;
            i1 = dg;
            ai = a;
        } else if (dg > i2) {
            i2 = dg;
        }
        if (est > e1) {
            e2 = e1;
            e1 = est;
            a1 = a;
        } else if (est > e2) {
            e2 = est;
        }
        p32[a] = make_float4(__double2float_rn(dx), __double2float_rn(dy), __double2float_rn(dz), __double2float_rn(m));
        h32[a] = hf;
    }
    const double tr = S[0] + S[3] + S[5];
    const double Q[6] = {3.0 * S[0] - tr, 3.0 * S[1], 3.0 * S[2], 3.0 * S[3] - tr, 3.0 * S[4], 3.0 * S[5] - tr};
    double d2max = 0.0;
    const bool clear_i = i2 < __fmul_rn(i1, 1.0f - 0x1p-18f);
    for (int a = clear_i ? ai : f; a < (clear_i ? ai + 1 : f + cnt); ++a)
        d2max = fmax(d2max, dist2_rn(px[a], py[a], pz[a], rg[0], rg[1], rg[2]));
    const double hint = __dsqrt_rn(d2max);
    double hnode = 0.0;
    const bool clear = e2 < __fmul_rn(e1, 1.0f - 0x1p-18f);
    for (int a = clear ? a1 : f; a < (clear ? a1 + 1 : f + cnt); ++a)
        hnode = fmax(hnode, __dadd_rn(__dsqrt_rn(dist2_rn(px[a], py[a], pz[a], rg[0], rg[1], rg[2])),
                                      __dmul_rn(2.0, ph[a])));
    for (int k = 0; k < 6; ++k) c.nQ[6 * (int64_t)n + k] = Q[k];
    c.nhint[n] = hint;
    c.nhnode[n] = hnode;
}

// Eq. 2 for every non-empty node of one level from its children (one launch per level, from
// the level above the ll-cells up to the root).
__global__ void k_level_up(LeafCtx c, int level) {
    const int64_t first = (int64_t)1 << level, count = first;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int P = (int)(first + i);
        if (c.ncount[P] > 0) parent_moments(c, P);
    }
}

struct PackCtx {
    const int32_t *ncount;
    const double *nmass, *ncom, *nrg, *nH, *nhint, *nQ;
    float4 *w32, *mq32a, *mq32b;
    float2 *ncomdf;
    float4 *nfar;
};

__global__ void k_pack_nodes(PackCtx c, int64_t nn) {
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nn; n += (int64_t)gridDim.x * blockDim.x) {
        if (n == 0 || c.ncount[n] == 0) {
            c.w32[2 * n] = make_float4(0.f, 0.f, 0.f, -1.f);
            c.w32[2 * n + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            c.mq32a[n] = make_float4(0.f, 0.f, 0.f, 0.f);
            c.mq32b[n] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int d = 0; d < 3; ++d) c.ncomdf[3 * n + d] = make_float2(0.f, 0.f);
            for (int k = 0; k < 4; ++k) c.nfar[4 * n + k] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        c.w32[2 * n] = make_float4(__double2float_rn(c.nrg[3 * n]), __double2float_rn(c.nrg[3 * n + 1]),
                                __double2float_rn(c.nrg[3 * n + 2]), __double2float_rn(c.nhint[n]));
        c.w32[2 * n + 1] = make_float4(__double2float_rn(c.ncom[3 * n]), __double2float_rn(c.ncom[3 * n + 1]),
                                __double2float_rn(c.ncom[3 * n + 2]), __double2float_rn(c.nH[n]));
        c.mq32a[n] = make_float4(__double2float_rn(c.nmass[n]), __double2float_rn(c.nQ[6 * n]),
                                 __double2float_rn(c.nQ[6 * n + 1]), __double2float_rn(c.nQ[6 * n + 2]));
        c.mq32b[n] = make_float4(__double2float_rn(c.nQ[6 * n + 3]), __double2float_rn(c.nQ[6 * n + 4]),
                                 __double2float_rn(c.nQ[6 * n + 5]), 0.f);
        float2 df[3];
        for (int d = 0; d < 3; ++d) {
            df[d] = to_df(c.ncom[3 * n + d]);
            c.ncomdf[3 * n + d] = df[d];
        }
        const float4 qa = c.mq32a[n], qb = c.mq32b[n];
        c.nfar[4 * n] = make_float4(df[0].x, df[1].x, df[2].x, qa.x);
        c.nfar[4 * n + 1] = make_float4(df[0].y, df[1].y, df[2].y, qa.y);
        c.nfar[4 * n + 2] = make_float4(qa.z, qa.w, qb.x, qb.y);
        c.nfar[4 * n + 3] = make_float4(qb.z, 0.f, 0.f, 0.f);
    }
}


// ------------------------------------------------------------------------------------------
// Three-phase device-wide exclusive scans (int32 -> int32 and int64 -> int64).
constexpr int kScanThreads = 1024, kScanPer = 8, kScanTile = kScanThreads * kScanPer;
static_assert(kScanTile == kScanTileElems, "the scan's scratch size is derived from kScanTileElems");

template <typename T>
__device__ T block_scan_excl_t(T v, T *warp_tot, T *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        T s = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            T t = warp_tot[k];
            warp_tot[k] = s;
            s += t;
        }
        warp_tot[32] = s;
    }
    __syncthreads();
    T excl = warp_tot[w] + incl - v;
    *total = warp_tot[32];
    __syncthreads();
    return excl;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const TI *in, int64_t n, TO *tile_sums) {
    __shared__ TO wt[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    TO v = 0;
    for (int j = 0; j < kScanPer; ++j)
        if (base + j < n) v += (TO)in[base + j];
    TO tot;
    block_scan_excl_t<TO>(v, wt, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

template <typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(TO *tile_sums, int64_t ntiles, TO *total_out) {
    __shared__ TO wt[33];
    __shared__ TO carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < ntiles; b += kScanThreads) {
        int64_t i = b + threadIdx.x;
        TO v = i < ntiles ? tile_sums[i] : (TO)0;
        TO tot;
        TO ex = block_scan_excl_t<TO>(v, wt, &tot);
        if (i < ntiles) tile_sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const TI *in, int64_t n, const TO *tile_sums, TO *out) {
    __shared__ TO wt[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    TO loc[kScanPer];
    TO v = 0;
    for (int j = 0; j < kScanPer; ++j) {
        loc[j] = base + j < n ? (TO)in[base + j] : (TO)0;
        v += loc[j];
    }
    TO tot;
    TO ex = block_scan_excl_t<TO>(v, wt, &tot) + tile_sums[blockIdx.x];
    for (int j = 0; j < kScanPer; ++j) {
        if (base + j < n) out[base + j] = ex;
        ex += loc[j];
    }
}

// ------------------------------------------------------------------------------------------
// Refit (Sec. 2.1.8): same particle sets, new positions and masses.

__global__ void k_refit_scan(const double *__restrict__ x, const double *__restrict__ m, int64_t N, int *status,
                             unsigned long long *maxbits) {
    unsigned long long mx[4] = {0, 0, 0, 0};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double mi = m[i];
        if (!isfinite(mi) || !(mi > 0.0)) bad = true;
        for (int d = 0; d < 3; ++d) {
            const double xi = x[3 * i + d];
            if (!isfinite(xi)) bad = true;
            const double p = fabs(__dmul_rn(mi, __dadd_rn(xi, 0.0)));
            const unsigned long long b = (unsigned long long)__double_as_longlong(p);
            if (isfinite(p) && b > mx[d]) mx[d] = b;
        }
        const unsigned long long bm = (unsigned long long)__double_as_longlong(mi);
        if (mi > 0.0 && isfinite(mi) && bm > mx[3]) mx[3] = bm;
    }
    for (int k = 0; k < 4; ++k) {
        unsigned long long v = mx[k];
        for (int o = 16; o >= 1; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
        if ((threadIdx.x & 31) == 0 && v) atomicMax(&maxbits[k], v);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&status[ST_ERR], ERRBIT_ARG);
}

__global__ void k_refit_gather(const double *__restrict__ x, const double *__restrict__ m, int64_t N,
                               const int32_t *pidx, double *px, double *py, double *pz, double *pm) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = pidx[p];
        px[p] = __dadd_rn(x[3 * o], 0.0);
        py[p] = __dadd_rn(x[3 * o + 1], 0.0);
        pz[p] = __dadd_rn(x[3 * o + 2], 0.0);
        pm[p] = m[o];
    }
}

__device__ inline i128 ldcg_i128(const i128 *p) {
    const long long *q = reinterpret_cast<const long long *>(p);
    const unsigned long long lo = (unsigned long long)__ldcg(q);
    const long long hi = __ldcg(q + 1);
    return (i128)(((u128)(unsigned long long)hi << 64) | (u128)lo);
}
__device__ inline int64_t ldcg_i64(const int64_t *p) { return (int64_t)__ldcg(reinterpret_cast<const long long *>(p)); }

// One thread per sink: exact sums and box of the ll-cell from its particles, then every parent
// (once both children are done) from its children's sums and boxes.  Splits are kept.
__global__ void k_refit_cells(Ctx c, const int32_t *sinks, int nsinks, const double *px, const double *py,
                              const double *pz, const double *pm, int32_t *narrive) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsinks) return;
    int n = sinks[s];
    const int sh[4] = {62 - c.E[0], 62 - c.E[1], 62 - c.E[2], 62 - c.E[3]};
    Red r;
    red_init(r);
    const int f = c.nfirst[n], cnt = c.ncount[n];
    bool bad = false;
    for (int a = f; a < f + cnt; ++a) {
        const double xs[3] = {px[a], py[a], pz[a]};
        int64_t P[4], key[3];
        for (int d = 0; d < 3; ++d) {
            key[d] = dkey(xs[d]);
            P[1 + d] = fixed_point(__dmul_rn(pm[a], xs[d]), sh[d]);
        }
        P[0] = fixed_point(pm[a], sh[3]);
        if (P[0] < 1) bad = true;
        red_add_particle(r, P, key);
    }
    if (bad) atomicOr(&c.status[ST_ERR], ERRBIT_FIXED);
    write_cell(c, n, c.L, f, r);
    while (n > 1) {
        const int sib = n ^ 1, P = n >> 1;
        __threadfence();
        if (__ldcg(&c.ncount[sib]) > 0) {
            if (atomicAdd(&narrive[P], 1) == 0) return;
            __threadfence();
        }
        Red q;
        red_init(q);
        for (int C = 2 * P; C <= 2 * P + 1; ++C) {
            const int cc = __ldcg(&c.ncount[C]);
            if (cc == 0) continue;
            Red t;
            for (int k = 0; k < 4; ++k) t.S[k] = ldcg_i128(&c.nS[4 * (int64_t)C + k]);
            for (int d = 0; d < 3; ++d) {
                t.lo[d] = ldcg_i64(&c.nbmin[3 * (int64_t)C + d]);
                t.hi[d] = ldcg_i64(&c.nbmax[3 * (int64_t)C + d]);
            }
            t.n = cc;
            red_merge(q, t);
        }
        write_cell(c, P, c.L, c.nfirst[P], q);  // level L: keep the build's split
        n = P;
    }
}

Ctx make_ctx(rcb_tree *t) {
    Ctx c;
    c.L = t->L;
    c.mps = (t->params.flags & RCB_FLAG_MEDIAN_SPLIT) ? 1 : 0;
    c.capN = t->cap_N;
    c.cap_big = t->cap_N / (kTcta + 1) + 2;
    c.cap_roots = t->cap_roots;
    c.status = t->d_status;
    c.E = t->d_E;
    c.nfirst = t->nfirst;
    c.ncount = t->ncount;
    c.naxis = t->naxis;
    c.nsplit = t->nsplit;
    c.nsplitkey = t->nsplitkey;
    c.nS = t->nS;
    c.nbmin = t->nbmin;
    c.nbmax = t->nbmax;
    c.nmass = t->nmass;
    c.ncom = t->ncom;
    c.nrg = t->nrg;
    c.nH = t->nH;
    return c;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

int read_status(rcb_tree *t) {
    const int rc = copy_words(t->h_status_dev, t->d_status, ST_NWORDS, t->stream);
    if (rc) return rc;
    RCB_CUDA_TRY(cudaStreamSynchronize(t->stream));
    return RCB_OK;
}

}  // namespace


size_t subtree_smem_bytes() { return sizeof(SubtreeSmem); }

size_t chunk_part_bytes(int64_t cap_chunks) {
    return std::max<size_t>((size_t)cap_chunks * sizeof(ChunkPart), (size_t)4096 * sizeof(Red));
}

int64_t scan_tmp_bytes(int64_t n) { return scan_tmp_words(n) * (int64_t)sizeof(int64_t); }

int scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total, void *tmp, cudaStream_t st) {
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    int32_t *sums = reinterpret_cast<int32_t *>(tmp);
    if (ntiles == 0) return cudaMemsetAsync(total, 0, sizeof(int32_t), st) == cudaSuccess ? RCB_OK : RCB_ERR_CUDA;
    k_scan_tiles<int32_t, int32_t><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, sums); note_launch();
    k_scan_sums<int32_t><<<1, kScanThreads, 0, st>>>(sums, ntiles, total); note_launch();
    k_scan_apply<int32_t, int32_t><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, sums, out); note_launch();
    return cudaGetLastError() == cudaSuccess ? RCB_OK : RCB_ERR_CUDA;
}

int scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, void *tmp, cudaStream_t st) {
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    int64_t *sums = reinterpret_cast<int64_t *>(tmp);
    if (ntiles == 0) return cudaMemsetAsync(total, 0, sizeof(int64_t), st) == cudaSuccess ? RCB_OK : RCB_ERR_CUDA;
    k_scan_tiles<int64_t, int64_t><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, sums); note_launch();
    k_scan_sums<int64_t><<<1, kScanThreads, 0, st>>>(sums, ntiles, total); note_launch();
    k_scan_apply<int64_t, int64_t><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, sums, out); note_launch();
    return cudaGetLastError() == cudaSuccess ? RCB_OK : RCB_ERR_CUDA;
}

// Eq. 2 level by level, from the level above the ll-cells up to the root.
static void launch_levels_up(const LeafCtx &lc, int L, int nsm, cudaStream_t st) {
    for (int level = L - 1; level >= 0; --level) {
        const int64_t nodes = (int64_t)1 << level;
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((nodes + 255) / 256, (int64_t)nsm * 8));
        k_level_up<<<g, 256, 0, st>>>(lc, level); note_launch();
    }
}

int build_tree(rcb_tree *t, const double *x, const double *m, const double *h) {
    cudaStream_t st = t->stream;
    const int64_t N = t->N;
    const int nsm = sm_count();
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_status, 0, ST_NWORDS * sizeof(int), st));
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_maxbits, 0, 4 * sizeof(unsigned long long), st));
    RCB_CUDA_TRY(cudaMemsetAsync(t->ncount, 0, t->nn * sizeof(int32_t), st));
    RCB_CUDA_TRY(cudaMemsetAsync(t->narrive, 0, t->nn * sizeof(int32_t), st));

    int grid = (int)std::min<int64_t>((N + 255) / 256, (int64_t)nsm * 8);
    if (grid < 1) grid = 1;
    stage_begin(t, SG_INGEST);
    k_ingest_scan<<<grid, 256, 0, st>>>(x, m, h, N, t->d_status, t->d_maxbits); note_launch();
    k_exponents<<<1, 32, 0, st>>>(t->d_maxbits, t->d_E); note_launch();
    Red *partials = reinterpret_cast<Red *>(t->chunk_part);  // reused: grid <= cap_chunks
    k_ingest_write<<<grid, 256, 0, st>>>(x, m, N, t->cap_N, t->d_E, t->bx[0], t->by[0], t->bz[0], t->bP[0],
                                         t->bidx[0], partials, t->d_status); note_launch();
    Ctx c = make_ctx(t);
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_nbig, 0, (kMaxL + 2) * sizeof(int32_t), st));
    k_root_finalize<<<1, 256, 0, st>>>(c, partials, grid, t->big_list[0], t->roots, t->d_nbig); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    stage_end(t, SG_INGEST);
    int rc = read_status(t);
    if (rc) return rc;
    if (t->h_status[ST_ERR] & (ERRBIT_ARG | ERRBIT_FIXED)) return RCB_ERR_ARG;
    stage_begin(t, SG_LEVELS);

    // level passes while large cells remain.  The number of large cells of every level lives on
    // the device (d_nbig[level]); kernels read it and do nothing when it is zero, so the host
    // launches levels in batches with upper-bound grids and synchronises once per batch.
    int nbig = t->h_status[ST_NBIG];
    int level = 0;
    if (c.mps) {
        if (!t->mps_hist || !t->mps_prefix || !t->mps_rank) return RCB_ERR_STATE;
        RCB_CUDA_TRY(cudaMemsetAsync(t->mps_hist, 0, (size_t)c.cap_big * kMpsBins * sizeof(int32_t), st));
    }
    ChunkPart *parts = reinterpret_cast<ChunkPart *>(t->chunk_part);
    const int64_t big_cap = N / (kTcta + 1) + 2;
    constexpr int kBatch = 4;
    while (nbig > 0) {
        int64_t nbig_bound = nbig;
        for (int b = 0; b < kBatch && level < t->L; ++b, ++level) {
            const int cur = level & 1;
            const int64_t bound = (N + kChunk - 1) / kChunk + nbig_bound + 1;
            if (bound > t->cap_chunks) return RCB_ERR_LIMIT;
            k_chunk_plan<<<1, 1024, 0, st>>>(t->big_list[cur], t->d_nbig + level, t->nfirst, t->ncount,
                                             t->cell_chunk0, t->chunks, t->d_status); note_launch();
            const int g = (int)std::min<int64_t>(bound, (int64_t)nsm * 8);
            if (c.mps) {
                const int gp = (int)std::max<int64_t>(1, (nbig_bound * 32 + 255) / 256);
                for (int shift = 56; shift >= 0; shift -= 8) {
                    k_mps_hist<<<g, kChunkThreads, 0, st>>>(c, t->chunks, t->d_status + ST_NCHUNKS, t->bx[cur],
                                                            t->by[cur], t->bz[cur], t->mps_prefix, shift,
                                                            t->mps_hist); note_launch();
                    k_mps_pick<<<gp, 256, 0, st>>>(c, t->big_list[cur], t->d_nbig + level, shift, t->mps_hist,
                                                   t->mps_prefix, t->mps_rank); note_launch();
                }
            }
            k_level_reduce<<<g, kChunkThreads, 0, st>>>(c, t->chunks, t->d_status + ST_NCHUNKS, t->bx[cur],
                                                        t->by[cur], t->bz[cur], t->bP[cur], parts); note_launch();
            const int gf = (int)std::max<int64_t>(1, (nbig_bound * 32 + 255) / 256);
            k_level_finalize<<<gf, 256, 0, st>>>(c, level, t->big_list[cur], t->d_nbig + level, t->cell_chunk0,
                                                 t->d_status + ST_NCHUNKS, parts, t->big_list[cur ^ 1],
                                                 t->d_nbig + level + 1, t->roots, (level + 1) & 1); note_launch();
            k_level_scatter<<<g, kChunkThreads, 0, st>>>(c, t->chunks, t->d_status + ST_NCHUNKS, parts, t->bx[cur],
                                                         t->by[cur], t->bz[cur], t->bP[cur], t->bidx[cur],
                                                         t->bx[cur ^ 1], t->by[cur ^ 1], t->bz[cur ^ 1],
                                                         t->bP[cur ^ 1], t->bidx[cur ^ 1]); note_launch();
            nbig_bound = std::min<int64_t>(2 * nbig_bound, big_cap);
        }
        RCB_CUDA_TRY(cudaGetLastError());
        rc = copy_words(t->h_status_dev + ST_NWORDS, t->d_nbig + level, 1, st);
        if (rc) return rc;
        rc = read_status(t);
        if (rc) return rc;
        if (t->h_status[ST_ERR] & ERRBIT_STATE) return RCB_ERR_LIMIT;
        nbig = level < t->L ? t->h_status[ST_NWORDS] : 0;
    }
    stage_end(t, SG_LEVELS);
    int nroots = t->h_status[ST_NROOTS];
    if (nroots > t->cap_roots || (t->h_status[ST_ERR] & ERRBIT_STATE)) return RCB_ERR_LIMIT;
    t->nroots_last = nroots;

    // subtrees in shared memory
    {
        Bufs B;
        for (int q = 0; q < 2; ++q) {
            B.x[q] = t->bx[q];
            B.y[q] = t->by[q];
            B.z[q] = t->bz[q];
            B.P[q] = t->bP[q];
            B.idx[q] = t->bidx[q];
        }
        stage_begin(t, SG_SUBTREE);
        size_t smem = sizeof(SubtreeSmem);
        RCB_CUDA_TRY(cudaFuncSetAttribute(k_subtree, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int g = std::max(1, std::min(nroots, 2 * nsm));
        k_subtree<<<g, kCtaThreads, smem, st>>>(c, t->roots, t->d_status + ST_NROOTS, B, m, h, t->px, t->py, t->pz,
                                                t->pm, t->ph, t->pidx); note_launch();
        RCB_CUDA_TRY(cudaGetLastError());
        stage_end(t, SG_SUBTREE);
    }

    // sinks: non-empty ll-cells in label order
    stage_begin(t, SG_LEAVES);
    {
        int32_t *flags = reinterpret_cast<int32_t *>(t->near_nr);  // scratch: >= nleaves entries
        int32_t *pos = t->sink_of_leaf;
        int64_t leaf0 = t->nleaves;
        int g = (int)std::min<int64_t>((t->nleaves + 255) / 256, (int64_t)nsm * 8);
        k_count_sinks<<<g, 256, 0, st>>>(t->ncount, leaf0, t->nleaves, flags); note_launch();
        rc = scan_i32(flags, pos, t->nleaves, t->d_status + ST_NSINKS, t->scan_tmp, st);
        if (rc) return rc;
        k_write_sinks<<<g, 256, 0, st>>>(flags, pos, leaf0, t->nleaves, t->sinks, t->sink_of_leaf); note_launch();
        RCB_CUDA_TRY(cudaGetLastError());
        rc = read_status(t);
        if (rc) return rc;
        t->nsinks = t->h_status[ST_NSINKS];
    }

    // leaf moments and bottom-up
    {
        LeafCtx lc;
        lc.nfirst = t->nfirst;
        lc.ncount = t->ncount;
        lc.nmass = t->nmass;
        lc.ncom = t->ncom;
        lc.nrg = t->nrg;
        lc.nH = t->nH;
        lc.nhint = t->nhint;
        lc.nhnode = t->nhnode;
        lc.nQ = t->nQ;
        lc.narrive = t->narrive;
        lc.px = t->px;
        lc.py = t->py;
        lc.pz = t->pz;
        lc.pm = t->pm;
        lc.ph = t->ph;
        lc.p32 = t->p32;
        lc.h32 = t->h32;
        if (t->nsinks > 0) k_leaves_up<<<(t->nsinks + 127) / 128, 128, 0, st>>>(lc, t->sinks, t->nsinks); note_launch();
        launch_levels_up(lc, t->L, nsm, st);
        PackCtx pc;
        pc.ncount = t->ncount;
        pc.nmass = t->nmass;
        pc.ncom = t->ncom;
        pc.nrg = t->nrg;
        pc.nH = t->nH;
        pc.nhint = t->nhint;
        pc.nQ = t->nQ;
        pc.w32 = t->w32;
        pc.mq32a = t->mq32a;
        pc.mq32b = t->mq32b;
        pc.ncomdf = t->ncomdf;
    pc.nfar = t->nfar;
        int g = (int)std::min<int64_t>((t->nn + 255) / 256, (int64_t)nsm * 8);
        k_pack_nodes<<<g, 256, 0, st>>>(pc, t->nn); note_launch();
        RCB_CUDA_TRY(cudaGetLastError());
    }
    stage_end(t, SG_LEAVES);
    return RCB_OK;
}

// ------------------------------------------------------------------------------------------
// Tree integrity check (Sec. 2.1.8).  A particle stays in its ll-cell when, at its new position,
// it lies on the side of every ancestor's split plane that it was sorted to: x_axis < split for a
// left child, not less for a right child.  Only planes with particles on both sides count (a
// cell whose other child is empty separates nothing; a one-particle cell is split through that
// particle).  The ancestors' planes of one sink make a box,
// lo <= x < hi per axis (lo the largest split among right turns, hi the smallest among left
// turns; unbounded otherwise); one warp per sink builds it and tests the sink's particles
// against it.  Non-finite coordinates count as outside.

__global__ void k_integrity(const int32_t *sinks, int nsinks, const int32_t *nfirst, const int32_t *ncount,
                            const int32_t *naxis, const double *nsplit, const int32_t *pidx, const double *x,
                            int *outside) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    int nout = 0;
    for (int s = gw; s < nsinks; s += nw) {
        const int A = sinks[s];
        double lo0 = -INFINITY, lo1 = -INFINITY, lo2 = -INFINITY, hi0 = INFINITY, hi1 = INFINITY, hi2 = INFINITY;
        for (int n = A; n > 1; n >>= 1) {
            if (ncount[n ^ 1] == 0) continue;
            const int p = n >> 1, ax = naxis[p];
            const double sp = nsplit[p];
            if (n & 1) {  // right child: x_axis >= split
                if (ax == 0) lo0 = fmax(lo0, sp);
                else if (ax == 1) lo1 = fmax(lo1, sp);
                else lo2 = fmax(lo2, sp);
            } else {      // left child: x_axis < split
                if (ax == 0) hi0 = fmin(hi0, sp);
                else if (ax == 1) hi1 = fmin(hi1, sp);
                else hi2 = fmin(hi2, sp);
            }
        }
        const int f = nfirst[A], cnt = ncount[A];
        for (int a = f + lane; a < f + cnt; a += 32) {
            const int64_t o = pidx[a];
            const double v0 = x[3 * o], v1 = x[3 * o + 1], v2 = x[3 * o + 2];
            const bool in = v0 >= lo0 && v0 < hi0 && v1 >= lo1 && v1 < hi1 && v2 >= lo2 && v2 < hi2;
            nout += in ? 0 : 1;
        }
    }
    for (int o = 16; o >= 1; o >>= 1) nout += __shfl_xor_sync(0xffffffffu, nout, o);
    if (lane == 0 && nout) atomicAdd(outside, nout);
}

__global__ void k_gather_h(const double *h, int64_t N, const int32_t *pidx, double *ph, int *status) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        const double v = h[pidx[p]];
        if (!isfinite(v) || !(v > 0.0)) atomicOr(&status[ST_ERR], ERRBIT_ARG);
        ph[p] = v;
    }
}

int integrity_outside(rcb_tree *t, const double *x, int64_t *outside) {
    if (t->nsinks <= 0) return RCB_ERR_STATE;
    cudaStream_t st = t->stream;
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_status, 0, ST_NWORDS * sizeof(int), st));
    const int nsm = sm_count();
    const int grid = std::max(1, std::min((t->nsinks + 7) / 8, nsm * 8));
    k_integrity<<<grid, 256, 0, st>>>(t->sinks, t->nsinks, t->nfirst, t->ncount, t->naxis, t->nsplit, t->pidx, x,
                                      t->d_status + ST_OUTSIDE); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    const int rc = read_status(t);
    if (rc) return rc;
    *outside = t->h_status[ST_OUTSIDE];
    return RCB_OK;
}

// New smoothing lengths (original order) into tree order; the leaf pass derives the float32
// copies and the radii from them.
int gather_h(rcb_tree *t, const double *h) {
    cudaStream_t st = t->stream;
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_status, 0, sizeof(int), st));
    const int nsm = sm_count();
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((t->N + 255) / 256, (int64_t)nsm * 8));
    k_gather_h<<<grid, 256, 0, st>>>(h, t->N, t->pidx, t->ph, t->d_status); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    const int rc = read_status(t);
    if (rc) return rc;
    if (t->h_status[ST_ERR] & ERRBIT_ARG) return RCB_ERR_ARG;
    return RCB_OK;
}

int refit_tree(rcb_tree *t, const double *x, const double *m) {
    if (t->nsinks <= 0) return RCB_ERR_STATE;
    cudaStream_t st = t->stream;
    const int64_t N = t->N;
    const int nsm = sm_count();
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_status, 0, sizeof(int), st));
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_maxbits, 0, 4 * sizeof(unsigned long long), st));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, (int64_t)nsm * 8));
    k_refit_scan<<<grid, 256, 0, st>>>(x, m, N, t->d_status, t->d_maxbits); note_launch();
    k_exponents<<<1, 32, 0, st>>>(t->d_maxbits, t->d_E); note_launch();
    k_refit_gather<<<grid, 256, 0, st>>>(x, m, N, t->pidx, t->px, t->py, t->pz, t->pm); note_launch();
    RCB_CUDA_TRY(cudaMemsetAsync(t->narrive, 0, t->nn * sizeof(int32_t), st));
    Ctx c = make_ctx(t);
    k_refit_cells<<<(t->nsinks + 127) / 128, 128, 0, st>>>(c, t->sinks, t->nsinks, t->px, t->py, t->pz, t->pm,
                                                          t->narrive); note_launch();
    RCB_CUDA_TRY(cudaMemsetAsync(t->narrive, 0, t->nn * sizeof(int32_t), st));
    LeafCtx lc;
    lc.nfirst = t->nfirst;
    lc.ncount = t->ncount;
    lc.nmass = t->nmass;
    lc.ncom = t->ncom;
    lc.nrg = t->nrg;
    lc.nH = t->nH;
    lc.nhint = t->nhint;
    lc.nhnode = t->nhnode;
    lc.nQ = t->nQ;
    lc.narrive = t->narrive;
    lc.px = t->px;
    lc.py = t->py;
    lc.pz = t->pz;
    lc.pm = t->pm;
    lc.ph = t->ph;
    lc.p32 = t->p32;
    lc.h32 = t->h32;
    k_leaves_up<<<(t->nsinks + 127) / 128, 128, 0, st>>>(lc, t->sinks, t->nsinks); note_launch();
    launch_levels_up(lc, t->L, sm_count(), st);
    PackCtx pc;
    pc.ncount = t->ncount;
    pc.nmass = t->nmass;
    pc.ncom = t->ncom;
    pc.nrg = t->nrg;
    pc.nH = t->nH;
    pc.nhint = t->nhint;
    pc.nQ = t->nQ;
    pc.w32 = t->w32;
    pc.mq32a = t->mq32a;
    pc.mq32b = t->mq32b;
    pc.ncomdf = t->ncomdf;
    pc.nfar = t->nfar;
    const int g = (int)std::min<int64_t>((t->nn + 255) / 256, (int64_t)nsm * 8);
    k_pack_nodes<<<g, 256, 0, st>>>(pc, t->nn); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    const int rc = read_status(t);
    if (rc) return rc;
    if (t->h_status[ST_ERR] & (ERRBIT_ARG | ERRBIT_FIXED)) return RCB_ERR_ARG;
    t->nb_valid = 0;  // neighbour counts depend on the positions (candidate lists stay frozen)
    return RCB_OK;
}

}  // namespace rcb
