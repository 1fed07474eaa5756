// Neighbour rows in a warp's shared memory (Sec. 2.3 lists, built by the fused near-field kernel
// and by the standalone neighbour pass): placement of the entries found in a loop step, the
// sorting networks that order a row by original index, and the hand-off of a finished pass of
// rows to the compact staging buffer from which rcb_neighbours copies them into the caller's CSR.
//
// A staged row holds the particle's neighbours and the particle itself (once, in any order); the
// copy into the CSR sorts the row by original index and drops the particle itself.  The row
// buffer of a pass has kRowBuf entries, split into equal slices (one per row, or one per lane
// holding a part of a row).  Entries beyond a slice are counted but not stored; such a row is
// "long" and its pass is queued for the direct fill (which recomputes it straight into the CSR).
#pragma once

#include <climits>

#include "rcb_internal.cuh"

namespace rcb {

constexpr int kRowBuf = 1280;  // entries of a warp's shared-memory row buffer

// Sink particles per pass of the neighbour test: at most 16, as even as possible
// (ceil(nA / ceil(nA / 16)), the last pass shorter), so that every particle of a pass has at
// least two source streams and its row is spread over two or more parts of the row buffer (in
// the fused kernel, or at least 80 entries of it in the standalone one).  A pass is (sink,
// first particle a0); every kernel that runs or re-runs a pass takes its length from here.
__host__ __device__ inline int nb_pass_len(int nA) {
    const int np = (nA + 15) >> 4;
    return np > 0 ? (nA + np - 1) / np : 1;
}

// Where finished rows go.
struct RowOut {
    int32_t *tmp;                    // compact staging buffer of rows (original indices)
    int64_t cap_tmp;
    unsigned long long *cursor;      // entries of tmp taken so far
    int64_t *tstart;                 // [N] by original index: row start in tmp, -1 if not there
    int2 *long_q;                    // (sink, first particle of the pass) of passes with long rows
    int cap_long;
    int *status;
};

// Append the neighbours a lane found in one block of loop steps: bit 2t + u of mask flags source
// u of the lane's pair in step t, pair index k0 + t S, whose original indices are D[k].x, D[k].y.
// The entries take consecutive places of the row from a shared-memory counter (one atomic per
// block); the order inside a row is free, since every row is sorted when it is finished.
__device__ __forceinline__ void row_append(int32_t *row, int rc, int *rowcnt, unsigned mask, int k0, int S,
                                           const int4 *D) {
    int p = atomicAdd(rowcnt, __popc(mask));
    while (mask) {
        const int bit = __ffs(mask) - 1;
        mask &= mask - 1;
        const int4 d = D[k0 + (bit >> 1) * S];
        if (p < rc) row[p] = (bit & 1) ? d.y : d.x;
        ++p;
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
                    const int32_t y = __shfl_xor_sync(0xffffffffu, v[r], j);
                    const bool up = ((r * 32 + lane) & k) == 0;
                    v[r] = (lower == up) ? min(v[r], y) : max(v[r], y);
                }
            }
        }
    }
}

// The same network on each group of 8 lanes: 8 lanes x R keys per segment, so four rows of up to
// 8 R entries sort at once.
template <int R>
__device__ inline void seg8_sort(int32_t (&v)[R]) {
    const int gl = threadIdx.x & 7;
#pragma unroll
    for (int k = 2; k <= 8 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 8) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int p = r ^ (j >> 3);
                    if (p > r) {
                        const bool up = ((r * 8 + gl) & k) == 0;
                        const int32_t x = v[r], y = v[p];
                        v[r] = up ? min(x, y) : max(x, y);
                        v[p] = up ? max(x, y) : min(x, y);
                    }
                }
            } else {
                const bool lower = (gl & j) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int32_t y = __shfl_xor_sync(0xffffffffu, v[r], j);
                    const bool up = ((r * 8 + gl) & k) == 0;
                    v[r] = (lower == up) ? min(v[r], y) : max(v[r], y);
                }
            }
        }
    }
}

// In-place ascending sort of n keys at p (shared or global memory) by the whole warp: a bitonic
// network with every comparator ascending (a flip stage, then half-cleaners); positions >= n
// count as +infinity and are never touched.
__device__ inline void warp_sort_inplace(int32_t *p, int n) {
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

// Sort rows src[rs[i] .. rs[i] + len[i]) (shared or global memory) and store each at dst + off[i],
// for the rows i < P with len[i] >= 0 (negative: skip); every entry equal to self[i] is left out
// (a staged row holds its own particle once, so the stored row is one shorter).  Four rows of
// at most 64 entries at a time, one per group of 8 lanes; longer rows over the whole warp (in
// place in src beyond 128 entries).  rs, len, off and self are read with a shuffle from lane i.
__device__ __forceinline__ void store_dropping(int32_t *dst, int64_t o, int e, int n, int32_t v, int32_t self) {
    if (e < n && v != self) dst[o + e - (v > self ? 1 : 0)] = v;
}

__device__ inline void rows_sort_store(int32_t *src, int64_t rs_l, int len_l, int64_t off_l, int32_t self_l, int32_t *dst,
                                       int P) {
    const int lane = threadIdx.x & 31, g = lane >> 3, gl = lane & 7;
    int i = 0;
    while (i < P) {
        // four rows at once, one per group of 8 lanes (a skipped or missing row is empty here)
        const int r = min(i + g, P - 1);
        const int nr0 = __shfl_sync(0xffffffffu, len_l, r);  // every lane takes part in the shuffle
        const int nr = i + g < P ? nr0 : -1;
        const int64_t rs = __shfl_sync(0xffffffffu, rs_l, r);
        const int64_t o = __shfl_sync(0xffffffffu, off_l, r);
        const int32_t sf = __shfl_sync(0xffffffffu, self_l, r);
        const int nmax = __reduce_max_sync(0xffffffffu, nr);
        if (nmax <= 64) {
            const int n = max(nr, 0);
            if (nmax <= 16) {
                int32_t v[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) v[q] = q * 8 + gl < n ? src[rs + q * 8 + gl] : INT32_MAX;
                seg8_sort<2>(v);
#pragma unroll
                for (int q = 0; q < 2; ++q) store_dropping(dst, o, q * 8 + gl, n, v[q], sf);
            } else if (nmax <= 32) {
                int32_t v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = q * 8 + gl < n ? src[rs + q * 8 + gl] : INT32_MAX;
                seg8_sort<4>(v);
#pragma unroll
                for (int q = 0; q < 4; ++q) store_dropping(dst, o, q * 8 + gl, n, v[q], sf);
            } else {
                int32_t v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = q * 8 + gl < n ? src[rs + q * 8 + gl] : INT32_MAX;
                seg8_sort<8>(v);
#pragma unroll
                for (int q = 0; q < 8; ++q) store_dropping(dst, o, q * 8 + gl, n, v[q], sf);
            }
            i += 4;
            continue;
        }
        // otherwise one row at a time over the whole warp
        const int n = __shfl_sync(0xffffffffu, len_l, i);
        const int64_t r0 = __shfl_sync(0xffffffffu, rs_l, i);
        const int64_t o0 = __shfl_sync(0xffffffffu, off_l, i);
        const int32_t s0 = __shfl_sync(0xffffffffu, self_l, i);
        if (n > 0) {
            if (n <= 128) {
                int32_t v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = q * 32 + lane < n ? src[r0 + q * 32 + lane] : INT32_MAX;
                warp_sort<4>(v);
#pragma unroll
                for (int q = 0; q < 4; ++q) store_dropping(dst, o0, q * 32 + lane, n, v[q], s0);
            } else {
                warp_sort_inplace(src + r0, n);
                __syncwarp();
                for (int q = lane; q < n; q += 32) store_dropping(dst, o0, q, n, src[r0 + q], s0);
            }
        }
        __syncwarp();
        i += 1;
    }
}

// Hand a finished pass over: lane l < P holds row l's length run (its entries in rows[l rc ..],
// in any order), original index o.  Rows that fit their slice are copied as they are to the
// staging buffer, one reservation per pass (the copy into the CSR sorts them); a row longer than
// its slice gets tstart = -1 and the pass is queued for the direct fill.  If the staging buffer is
// full, every row of the pass gets tstart = -1 and an error bit tells the host to fill directly
// instead.
__device__ inline void rows_finish(const RowOut &ro, int32_t *rows, int rc, int P, int run, int o, int s, int a0) {
    const int lane = threadIdx.x & 31;
    const bool lng = lane < P && run > rc;
    const int keep = lane < P && !lng ? run : 0;
    const int ex = warp_excl_scan(keep);
    const int tot = __shfl_sync(0xffffffffu, ex + keep, 31);
    unsigned long long base = 0;
    if (lane == 0 && tot > 0) base = atomicAdd(ro.cursor, (unsigned long long)tot);
    base = __shfl_sync(0xffffffffu, base, 0);
    const bool fits = tot == 0 || base + (unsigned long long)tot <= (unsigned long long)ro.cap_tmp;
    if (!fits && lane == 0) atomicOr(&ro.status[ST_ERR], ERRBIT_NBTMP);
    if (lane < P) ro.tstart[o] = (lng || !fits) ? -1 : (int64_t)base + ex;
    if (__any_sync(0xffffffffu, lng) && lane == 0) {
        const int q = atomicAdd(&ro.status[ST_NBLONG], 1);
        if (q < ro.cap_long) ro.long_q[q] = make_int2(s, a0);
    }
    if (fits) {
        for (int q = 0; q < P; ++q) {
            const int n = __shfl_sync(0xffffffffu, keep, q);
            const int64_t d = (int64_t)base + __shfl_sync(0xffffffffu, ex, q);
            for (int e = lane; e < n; e += 32) ro.tmp[d + e] = rows[q * rc + e];
        }
    }
    __syncwarp();
}

// Hand a finished pass over when every lane (i, j) of the P S lanes holding a sink particle kept
// its part of row i as column g = i S + j of the row buffer seen as rows of P S entries, cap
// entries at most (nsub of them counted): part lengths go
// through cnt (shared memory, 32 entries); lane l < P holds row l's particle (original index o).
// The parts of every row that fits are copied in order to the staging buffer (one reservation
// per pass); counts[o] receives the row length less the particle itself.
static __device__ __noinline__ void rows_finish_parts(const RowOut &ro, int64_t *counts, const int32_t *rows, int *cnt, int cap,
                                         int P, int S, int nsub, int o, int s, int a0) {
    const int lane = threadIdx.x & 31;
    const int i = lane % P, j = lane / P;
    const int PS = P * S;
    if (j < S) cnt[i * S + j] = nsub;
    __syncwarp();
    int tot = 0;
    bool over = false;
    if (lane < P)
        for (int jj = 0; jj < S; ++jj) {
            const int v = cnt[lane * S + jj];
            tot += v;
            over = over || v > cap;
        }
    // the parts, in slice order g = lane
    const bool gover = __shfl_sync(0xffffffffu, (int)over, min(lane / S, 31)) != 0;
    const int seglen = lane < PS && !gover ? cnt[lane] : 0;
    const int exg = warp_excl_scan(seglen);
    const int T = __shfl_sync(0xffffffffu, exg + seglen, 31);
    unsigned long long base = 0;
    if (lane == 0 && T > 0) base = atomicAdd(ro.cursor, (unsigned long long)T);
    base = __shfl_sync(0xffffffffu, base, 0);
    const bool fits = T == 0 || base + (unsigned long long)T <= (unsigned long long)ro.cap_tmp;
    if (!fits && lane == 0) atomicOr(&ro.status[ST_ERR], ERRBIT_NBTMP);
    const int rstart = __shfl_sync(0xffffffffu, exg, min(lane * S, 31));
    if (lane < P) {
        ro.tstart[o] = (over || !fits) ? -1 : (int64_t)base + rstart;
        counts[o] = tot - 1;
    }
    if (__any_sync(0xffffffffu, over) && lane == 0) {
        const int q = atomicAdd(&ro.status[ST_NBLONG], 1);
        if (q < ro.cap_long) ro.long_q[q] = make_int2(s, a0);
    }
    if (fits)
        for (int g = 0; g < PS; ++g) {  // part g, lanes over its entries
            const int ng = __shfl_sync(0xffffffffu, seglen, g);
            const int64_t d = (int64_t)base + __shfl_sync(0xffffffffu, exg, g);
            for (int e = lane; e < ng; e += 32) ro.tmp[d + e] = rows[e * PS + g];
        }
    __syncwarp();
}

}  // namespace rcb
