// Per-sink tree walk (Sec. 2.2, Sec. 2.3.1, Sec. 2.4.1) emitting near and far lists.
//
// One thread walks for one sink (non-empty ll-cells in label order, so the 32 sinks of a warp
// are spatial neighbours and share most of the nodes they load).  The walk is the stackless
// depth-first order of Sec. 2.2 on heap labels, starting at node 2: after a node that is not
// opened, climb while the node is a right child, then step to the next label.
//
// Decisions (in this order, Sec. 2.4.1):
//   reachable   |r_gA - r_gB|^2 < (h_node(A) + h_node_int(B))^2   -> ll-cell: near + candidate
//                                                                    internal: open
//   MAC         H_B^2 < theta^2 R_AB^2                            -> far
//   otherwise   ll-cell: near; internal: open
// Each test is first evaluated in float32 with a forward error bound B = 2^-20 F, where F is
// the same expression evaluated on magnitudes (input rounding, ~7 roundings and the final
// subtraction stay below 8u F with u = 2^-24, so B is twice the worst case).  Only when
// |value| <= B is the test repeated in float64, rounded after every operation exactly as the
// definition is written; the lists are therefore identical to an all-float64 walk.
#include <cuda_runtime.h>

#include <algorithm>

#include "rcb_internal.cuh"

namespace rcb {
namespace {

constexpr int kWalkWarps = 4;

struct WalkCtx {
    int L;
    int64_t nn;
    double theta2;
    float theta2f;
    const float4 *w32;  // [2n] (r_g, h_int), [2n + 1] (COM, H); h_int = -1 marks an empty node
    const double *nrg, *nhint, *ncom, *nH, *nhnode;
    const int32_t *sinks;
    int nsinks;
    int cap_near, cap_far;
    int32_t *near_list, *far_list, *near_nr, *near_nn, *far_n;
    int *status;
};

__device__ inline float sq(float v) { return v * v; }

// MODE 0: the walk above.  MODE 1: MAC-only near lists (the variant of Sec. 2.5 without the
// reachability override): MAC -> far, otherwise leaf -> near (from the back), internal -> open.
// MODE 2: neighbour candidates only: reachable leaves -> near (from the front), reachable
// internal nodes opened, the rest skipped; no far list.
template <int MODE>
__global__ void __launch_bounds__(kWalkWarps * 32) k_walk(WalkCtx c) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = s < c.nsinks;
    int nr = 0, nnr = 0, nf = 0, nfallback = 0;
    bool limit = false;
    if (valid) {
        const int A = c.sinks[s];
        const float4 a32 = c.w32[2 * A], b32 = c.w32[2 * A + 1];
        const float3 rgA = make_float3(a32.x, a32.y, a32.z);
        const float3 comA = make_float3(b32.x, b32.y, b32.z);
        const float hA = __double2float_rn(c.nhnode[A]);
        const float3 rgAabs = make_float3(fabsf(rgA.x), fabsf(rgA.y), fabsf(rgA.z));
        const float3 comAabs = make_float3(fabsf(comA.x), fabsf(comA.y), fabsf(comA.z));
        const int64_t near_base = (int64_t)s * c.cap_near;
        const int64_t far_base = (int64_t)s * c.cap_far;
        const int leaf0 = 1 << c.L;
        int n = 2;
        int64_t iter = 0;
        const int64_t max_iter = 2 * c.nn + 8;
        while (true) {
            if (++iter > max_iter) {
                limit = true;
                break;
            }
            bool open = false;
            // both halves of the node's 32-byte pack at once (one sector, one round of latency)
            const float4 na = c.w32[2 * n], nb = c.w32[2 * n + 1];
            if (na.w >= 0.f) {  // non-empty
                const bool is_leaf = n >= leaf0;
                // reachability
                const float dx = rgA.x - na.x, dy = rgA.y - na.y, dz = rgA.z - na.z;
                const float d2 = dx * dx + dy * dy + dz * dz;
                const float rr = hA + na.w;
                const float f = d2 - rr * rr;
                const float F = sq(rgAabs.x + fabsf(na.x)) + sq(rgAabs.y + fabsf(na.y)) + sq(rgAabs.z + fabsf(na.z)) + rr * rr;
                const float B = F * 0x1p-20f + 1e-30f;
                bool reach;
                if (MODE == 1) reach = false;
                else if (f < -B) reach = true;
                else if (f > B) reach = false;
                else {
                    ++nfallback;
                    const double e2 = dist2_rn(c.nrg[3 * (int64_t)A], c.nrg[3 * (int64_t)A + 1], c.nrg[3 * (int64_t)A + 2],
                                               c.nrg[3 * (int64_t)n], c.nrg[3 * (int64_t)n + 1], c.nrg[3 * (int64_t)n + 2]);
                    const double r = __dadd_rn(c.nhnode[A], c.nhint[n]);
                    reach = e2 < __dmul_rn(r, r);
                }
                if (reach) {
                    if (is_leaf) {
                        if (nr + nnr < c.cap_near) c.near_list[near_base + nr] = n;
                        ++nr;
                    } else {
                        open = true;
                    }
                } else if (MODE != 2) {
                    const float ex = comA.x - nb.x, ey = comA.y - nb.y, ez = comA.z - nb.z;
                    const float R2 = ex * ex + ey * ey + ez * ez;
                    const float fm = nb.w * nb.w - c.theta2f * R2;
                    const float Fm = nb.w * nb.w +
                                     c.theta2f * (sq(comAabs.x + fabsf(nb.x)) + sq(comAabs.y + fabsf(nb.y)) + sq(comAabs.z + fabsf(nb.z)));
                    const float Bm = Fm * 0x1p-20f + 1e-30f;
                    bool mac;
                    if (fm < -Bm) mac = true;
                    else if (fm > Bm) mac = false;
                    else {
                        ++nfallback;
                        const double R2d = dist2_rn(c.ncom[3 * (int64_t)A], c.ncom[3 * (int64_t)A + 1], c.ncom[3 * (int64_t)A + 2],
                                                    c.ncom[3 * (int64_t)n], c.ncom[3 * (int64_t)n + 1], c.ncom[3 * (int64_t)n + 2]);
                        const double H = c.nH[n];
                        mac = __dmul_rn(H, H) < __dmul_rn(c.theta2, R2d);
                    }
                    if (mac) {
                        if (nf < c.cap_far) c.far_list[far_base + nf] = n;
                        ++nf;
                    } else if (is_leaf) {
                        if (nr + nnr < c.cap_near) c.near_list[near_base + c.cap_near - 1 - nnr] = n;
                        ++nnr;
                    } else {
                        open = true;
                    }
                }
            }
            if (open) {
                n = 2 * n;
                continue;
            }
            // next node in depth-first order: drop the trailing one bits, then step right
            n = (n >> (__ffs(~n) - 1)) + 1;
            if (n == 1) break;
        }
        c.near_nr[s] = nr;
        c.near_nn[s] = nnr;
        c.far_n[s] = nf;
    }
    int mn = nr + nnr, mf = nf;
    for (int o = 16; o >= 1; o >>= 1) {
        mn = max(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mf = max(mf, __shfl_xor_sync(0xffffffffu, mf, o));
        nfallback += __shfl_xor_sync(0xffffffffu, nfallback, o);
    }
    const bool anylimit = __any_sync(0xffffffffu, limit);
    if (lane == 0) {
        atomicMax(&c.status[ST_MAXNEAR], mn);
        atomicMax(&c.status[ST_MAXFAR], mf);
        if (nfallback) atomicAdd(&c.status[ST_FALLBACK], nfallback);
        if (anylimit) atomicOr(&c.status[ST_ERR], ERRBIT_LIMIT);
    }
}

// The same walk for two consecutive sinks at once (siblings in label order, whose walks share
// most nodes): one thread follows the union of the two depth-first walks and loads every node
// once.  A sink that did not open a node the other opened sits out the node's subtree (skip =
// that node) and rejoins when the walk leaves it.  Each sink still meets its own nodes in
// depth-first order, so its lists are the ones its own walk writes.
struct WSink {
    int A;
    float3 rgA, comA, rgAabs, comAabs;
    float hA;
    int64_t near_base, far_base;
    int nr, nnr, nf;
};

__device__ inline void wsink_init(const WalkCtx &c, int s, WSink &k) {
    k.A = c.sinks[s];
    const float4 a32 = c.w32[2 * k.A], b32 = c.w32[2 * k.A + 1];
    k.rgA = make_float3(a32.x, a32.y, a32.z);
    k.comA = make_float3(b32.x, b32.y, b32.z);
    k.hA = __double2float_rn(c.nhnode[k.A]);
    k.rgAabs = make_float3(fabsf(k.rgA.x), fabsf(k.rgA.y), fabsf(k.rgA.z));
    k.comAabs = make_float3(fabsf(k.comA.x), fabsf(k.comA.y), fabsf(k.comA.z));
    k.near_base = (int64_t)s * c.cap_near;
    k.far_base = (int64_t)s * c.cap_far;
    k.nr = k.nnr = k.nf = 0;
}

// The decision for one non-empty node (as in k_walk): 1 near from the front, 2 near from the
// back, 3 far, 4 open.  The entry is written here.
__device__ __forceinline__ int wsink_visit(const WalkCtx &c, WSink &k, int n, const float4 &na, const float4 &nb,
                                           bool is_leaf, int &nfallback) {
    const float dx = k.rgA.x - na.x, dy = k.rgA.y - na.y, dz = k.rgA.z - na.z;
    const float d2 = dx * dx + dy * dy + dz * dz;
    const float rr = k.hA + na.w;
    const float f = d2 - rr * rr;
    const float F = sq(k.rgAabs.x + fabsf(na.x)) + sq(k.rgAabs.y + fabsf(na.y)) + sq(k.rgAabs.z + fabsf(na.z)) + rr * rr;
    const float B = F * 0x1p-20f + 1e-30f;
    bool reach;
    if (f < -B) reach = true;
    else if (f > B) reach = false;
    else {
        ++nfallback;
        const double e2 = dist2_rn(c.nrg[3 * (int64_t)k.A], c.nrg[3 * (int64_t)k.A + 1], c.nrg[3 * (int64_t)k.A + 2],
                                   c.nrg[3 * (int64_t)n], c.nrg[3 * (int64_t)n + 1], c.nrg[3 * (int64_t)n + 2]);
        const double r = __dadd_rn(c.nhnode[k.A], c.nhint[n]);
        reach = e2 < __dmul_rn(r, r);
    }
    if (reach) {
        if (!is_leaf) return 4;
        if (k.nr + k.nnr < c.cap_near) c.near_list[k.near_base + k.nr] = n;
        ++k.nr;
        return 1;
    }
    const float ex = k.comA.x - nb.x, ey = k.comA.y - nb.y, ez = k.comA.z - nb.z;
    const float R2 = ex * ex + ey * ey + ez * ez;
    const float fm = nb.w * nb.w - c.theta2f * R2;
    const float Fm = nb.w * nb.w +
                     c.theta2f * (sq(k.comAabs.x + fabsf(nb.x)) + sq(k.comAabs.y + fabsf(nb.y)) + sq(k.comAabs.z + fabsf(nb.z)));
    const float Bm = Fm * 0x1p-20f + 1e-30f;
    bool mac;
    if (fm < -Bm) mac = true;
    else if (fm > Bm) mac = false;
    else {
        ++nfallback;
        const double R2d = dist2_rn(c.ncom[3 * (int64_t)k.A], c.ncom[3 * (int64_t)k.A + 1], c.ncom[3 * (int64_t)k.A + 2],
                                    c.ncom[3 * (int64_t)n], c.ncom[3 * (int64_t)n + 1], c.ncom[3 * (int64_t)n + 2]);
        const double H = c.nH[n];
        mac = __dmul_rn(H, H) < __dmul_rn(c.theta2, R2d);
    }
    if (mac) {
        if (k.nf < c.cap_far) c.far_list[k.far_base + k.nf] = n;
        ++k.nf;
        return 3;
    }
    if (!is_leaf) return 4;
    if (k.nr + k.nnr < c.cap_near) c.near_list[k.near_base + c.cap_near - 1 - k.nnr] = n;
    ++k.nnr;
    return 2;
}

// m lies in the subtree of a (heap labels)
__device__ inline bool in_subtree(int m, int a) {
    const int d = (31 - __clz(m)) - (31 - __clz(a));
    return d >= 0 && (m >> d) == a;
}

__global__ void __launch_bounds__(kWalkWarps * 32) k_walk_pair(WalkCtx c) {
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int s0 = 2 * t, s1 = 2 * t + 1;
    const bool v0 = s0 < c.nsinks, v1 = s1 < c.nsinks;
    WSink k0, k1;
    int nfallback = 0;
    bool limit = false;
    if (v0) wsink_init(c, s0, k0);
    if (v1) wsink_init(c, s1, k1);
    if (v0) {
        int skip0 = 0, skip1 = v1 ? 0 : 1;  // 1: the whole tree (no second sink)
        const int leaf0 = 1 << c.L;
        int n = 2;
        int64_t iter = 0;
        const int64_t max_iter = 2 * c.nn + 8;
        while (true) {
            if (++iter > max_iter) {
                limit = true;
                break;
            }
            if (skip0 && !in_subtree(n, skip0)) skip0 = 0;
            if (skip1 && !in_subtree(n, skip1)) skip1 = 0;
            // both halves of the node's 32-byte pack at once (one sector, one round of latency)
            const float4 na = c.w32[2 * n], nb = c.w32[2 * n + 1];
            if (na.w >= 0.f) {  // non-empty
                const bool is_leaf = n >= leaf0;
                const int a0 = skip0 ? 0 : wsink_visit(c, k0, n, na, nb, is_leaf, nfallback);
                const int a1 = skip1 ? 0 : wsink_visit(c, k1, n, na, nb, is_leaf, nfallback);
                if (a0 == 4 || a1 == 4) {
                    if (!skip0 && a0 != 4) skip0 = n;
                    if (!skip1 && a1 != 4) skip1 = n;
                    n = 2 * n;
                    continue;
                }
            }
            // next node in depth-first order: drop the trailing one bits, then step right
            n = (n >> (__ffs(~n) - 1)) + 1;
            if (n == 1) break;
        }
        c.near_nr[s0] = k0.nr;
        c.near_nn[s0] = k0.nnr;
        c.far_n[s0] = k0.nf;
        if (v1) {
            c.near_nr[s1] = k1.nr;
            c.near_nn[s1] = k1.nnr;
            c.far_n[s1] = k1.nf;
        }
    }
    int mn = v0 ? k0.nr + k0.nnr : 0, mf = v0 ? k0.nf : 0;
    if (v1) {
        mn = max(mn, k1.nr + k1.nnr);
        mf = max(mf, k1.nf);
    }
    for (int o = 16; o >= 1; o >>= 1) {
        mn = max(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mf = max(mf, __shfl_xor_sync(0xffffffffu, mf, o));
        nfallback += __shfl_xor_sync(0xffffffffu, nfallback, o);
    }
    const bool anylimit = __any_sync(0xffffffffu, limit);
    if (lane == 0) {
        atomicMax(&c.status[ST_MAXNEAR], mn);
        atomicMax(&c.status[ST_MAXFAR], mf);
        if (nfallback) atomicAdd(&c.status[ST_FALLBACK], nfallback);
        if (anylimit) atomicOr(&c.status[ST_ERR], ERRBIT_LIMIT);
    }
}

// Per sink: (sink particles) x (particles of all near cells) and x (of reachable cells).
__global__ void k_pair_counts(const int32_t *sinks, int nsinks, const int32_t *ncount, const int32_t *near_list,
                              const int32_t *near_nr, const int32_t *near_nn, int cap_near,
                              unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long all = 0, reach = 0;
    for (int s = gw; s < nsinks; s += nw) {
        const int nA = ncount[sinks[s]];
        const int nr = near_nr[s], nn = near_nn[s];
        const int64_t base = (int64_t)s * cap_near;
        for (int k = lane; k < nr + nn; k += 32) {
            const int B = k < nr ? near_list[base + k] : near_list[base + cap_near - 1 - (k - nr)];
            const unsigned long long p = (unsigned long long)nA * ncount[B];
            all += p;
            if (k < nr) reach += p;
        }
    }
    for (int o = 16; o >= 1; o >>= 1) {
        all += __shfl_xor_sync(0xffffffffu, all, o);
        reach += __shfl_xor_sync(0xffffffffu, reach, o);
    }
    if (lane == 0) {
        atomicAdd(&out[0], all);
        atomicAdd(&out[1], reach);
    }
}

}  // namespace

int count_pairs(rcb_tree *t) {
    cudaStream_t st = t->stream;
    RCB_CUDA_TRY(cudaMemsetAsync(t->d_pairs, 0, 2 * sizeof(int64_t), st));
    int blocks = std::max(1, std::min((t->nsinks + 7) / 8, 152 * 8));
    k_pair_counts<<<blocks, 256, 0, st>>>(t->sinks, t->nsinks, t->ncount, t->near_list, t->near_nr, t->near_nn,
                                          t->cap_near, (unsigned long long *)t->d_pairs); note_launch();
    int64_t h[2];
    RCB_CUDA_TRY(cudaMemcpyAsync(h, t->d_pairs, sizeof(h), cudaMemcpyDeviceToHost, st));
    RCB_CUDA_TRY(cudaStreamSynchronize(st));
    t->near_pairs = h[0];
    t->cand_pairs = h[1];
    return RCB_OK;
}

// The walk into one set of per-sink lists, growing their capacities until every sink fits.
static int walk_into(rcb_tree *t, int mode, int32_t *&near_list, int32_t *&far_list, int32_t *near_nr,
                     int32_t *near_nn, int32_t *far_n, int &cap_near, int &cap_far, int64_t &cap_lists_near,
                     int64_t &cap_lists_far) {
    cudaStream_t st = t->stream;
    WalkCtx c;
    c.L = t->L;
    c.nn = t->nn;
    c.theta2 = t->params.theta * t->params.theta;
    c.theta2f = (float)c.theta2;
    c.w32 = t->w32;
    c.nrg = t->nrg;
    c.nhint = t->nhint;
    c.ncom = t->ncom;
    c.nH = t->nH;
    c.nhnode = t->nhnode;
    c.sinks = t->sinks;
    c.nsinks = t->nsinks;
    c.status = t->d_status;
    for (int attempt = 0; attempt < 3; ++attempt) {
        c.cap_near = cap_near;
        c.cap_far = cap_far;
        c.near_list = near_list;
        c.far_list = far_list;
        c.near_nr = near_nr;
        c.near_nn = near_nn;
        c.far_n = far_n;
        RCB_CUDA_TRY(cudaMemsetAsync(t->d_status + ST_MAXNEAR, 0, 3 * sizeof(int), st));
        const int blocks = (t->nsinks + kWalkWarps * 32 - 1) / (kWalkWarps * 32);
        if (mode == 0 && t->walk_pair) {
            // Long walks (concentrated inputs) share node loads between sibling sinks; short ones
            // keep one sink per thread for more parallelism.  Both write the same lists.
            const int nthreads = (t->nsinks + 1) / 2;
            const int bp = (nthreads + kWalkWarps * 32 - 1) / (kWalkWarps * 32);
            if (bp > 0) k_walk_pair<<<bp, kWalkWarps * 32, 0, st>>>(c); note_launch();
        } else if (blocks > 0) {
            if (mode == 0) k_walk<0><<<blocks, kWalkWarps * 32, 0, st>>>(c);
            else if (mode == 1) k_walk<1><<<blocks, kWalkWarps * 32, 0, st>>>(c);
            else k_walk<2><<<blocks, kWalkWarps * 32, 0, st>>>(c);
            note_launch();
        }
        RCB_CUDA_TRY(cudaGetLastError());
        {
            const int rc = copy_words(t->h_status_dev, t->d_status, ST_NWORDS, st);
            if (rc) return rc;
        }
        RCB_CUDA_TRY(cudaStreamSynchronize(st));
        if (t->h_status[ST_ERR] & ERRBIT_LIMIT) return RCB_ERR_LIMIT;
        int need_near = t->h_status[ST_MAXNEAR], need_far = t->h_status[ST_MAXFAR];
        if (mode != 2) t->stats_fallback = t->h_status[ST_FALLBACK];
        if (mode == 0) t->walk_pair = need_far > 1024;
        if (need_near <= cap_near && need_far <= cap_far) return RCB_OK;
        // grow the per-sink list capacities and walk again
        int cn = std::max(cap_near, ((need_near + 31) / 32) * 32 + 32);
        int cf = std::max(cap_far, ((need_far + 31) / 32) * 32 + 32);
        dev_free(t, near_list);
        dev_free(t, far_list);
        near_list = (int32_t *)dev_alloc(t, (size_t)t->nsinks * cn * sizeof(int32_t) + 16);
        far_list = (int32_t *)dev_alloc(t, (size_t)t->nsinks * cf * sizeof(int32_t) + 16);
        if (!near_list || !far_list) return RCB_ERR_ALLOC;
        cap_near = cn;
        cap_far = cf;
        cap_lists_near = (int64_t)t->nsinks * cn;
        cap_lists_far = (int64_t)t->nsinks * cf;
    }
    return RCB_ERR_LIMIT;
}

// The walks of a build or update: the lists gravity uses (standard, or MAC-only with
// RCB_FLAG_MAC_ONLY) and, for MAC-only lists, the neighbour candidates from a walk of their own.
int walk_tree(rcb_tree *t) {
    if (!(t->params.flags & RCB_FLAG_MAC_ONLY))
        return walk_into(t, 0, t->near_list, t->far_list, t->near_nr, t->near_nn, t->far_n, t->cap_near, t->cap_far,
                         t->cap_lists_near, t->cap_lists_far);
    int rc = walk_into(t, 1, t->near_list, t->far_list, t->near_nr, t->near_nn, t->far_n, t->cap_near, t->cap_far,
                       t->cap_lists_near, t->cap_lists_far);
    if (rc) return rc;
    if (!t->cand_n) {
        t->cand_n = (int32_t *)dev_alloc(t, 3 * (size_t)std::max<int64_t>(t->nleaves, 1) * sizeof(int32_t));
        if (!t->cand_n) return RCB_ERR_ALLOC;
        t->cap_cand = 0;
    }
    if (!t->cand_list) {
        t->cap_cand = 64;
        t->cap_lists_cand = (int64_t)t->nsinks * t->cap_cand;
        t->cand_list = (int32_t *)dev_alloc(t, (size_t)t->cap_lists_cand * sizeof(int32_t) + 16);
        t->cand_far = (int32_t *)dev_alloc(t, 16);
        if (!t->cand_list || !t->cand_far) return RCB_ERR_ALLOC;
    } else if ((int64_t)t->nsinks * t->cap_cand > t->cap_lists_cand) {
        dev_free(t, t->cand_list);
        t->cap_lists_cand = (int64_t)t->nsinks * t->cap_cand;
        t->cand_list = (int32_t *)dev_alloc(t, (size_t)t->cap_lists_cand * sizeof(int32_t) + 16);
        if (!t->cand_list) return RCB_ERR_ALLOC;
    }
    int cap_far0 = 0;
    int64_t far_lists0 = 0;
    return walk_into(t, 2, t->cand_list, t->cand_far, t->cand_n, t->cand_n + t->nleaves, t->cand_n + 2 * t->nleaves,
                     t->cap_cand, cap_far0, t->cap_lists_cand, far_lists0);
}

}  // namespace rcb
