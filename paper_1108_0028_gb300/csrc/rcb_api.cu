// C ABI entry points (include/rcb.h): argument checks, memory management and orchestration.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "rcb_internal.cuh"

namespace rcb {

void *dev_alloc(rcb_tree *t, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (t->alloc) {
        p = t->alloc(bytes, t->ctx, (void *)t->stream);
    } else {
        if (cudaMallocAsync(&p, bytes, t->stream) != cudaSuccess) p = nullptr;
    }
    return p;
}

void dev_free(rcb_tree *t, void *p) {
    if (!p) return;
    if (t->release) t->release(p, t->ctx, (void *)t->stream);
    else cudaFreeAsync(p, t->stream);
}

size_t chunk_part_bytes(int64_t cap_chunks);  // build.cu
int count_pairs(rcb_tree *t);                  // walk.cu

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

void stage_begin(rcb_tree *t, int stage) {
    if (!(t->params.flags & RCB_FLAG_TIMING)) return;
    if (!t->ev_ready) {
        for (int i = 0; i < 32; ++i) cudaEventCreate(&t->ev[i]);
        t->ev_ready = true;
    }
    cudaEventRecord(t->ev[2 * stage], t->stream);
    t->ev_used[stage] = true;
}

void stage_end(rcb_tree *t, int stage) {
    if (!(t->params.flags & RCB_FLAG_TIMING) || !t->ev_ready) return;
    cudaEventRecord(t->ev[2 * stage + 1], t->stream);
}

namespace {

int depth_rule(int64_t N, int32_t n_ll) {
    int L = 1;
    while (!(N < ((int64_t)n_ll << L))) {
        ++L;
        if (L > 40) break;
    }
    return L;
}

// Every device array of the tree, for allocation and release in one place.
template <typename F>
void for_each_array(rcb_tree *t, F f) {
    f((void **)&t->d_status);
    f((void **)&t->d_E);
    f((void **)&t->d_nbig);
    f((void **)&t->d_maxbits);
    f((void **)&t->d_pairs);
    for (int b = 0; b < 2; ++b) {
        f((void **)&t->bx[b]);
        f((void **)&t->by[b]);
        f((void **)&t->bz[b]);
        f((void **)&t->bP[b]);
        f((void **)&t->bidx[b]);
        f((void **)&t->big_list[b]);
    }
    void **p[] = {(void **)&t->px, (void **)&t->py, (void **)&t->pz, (void **)&t->pm, (void **)&t->ph,
                  (void **)&t->pidx, (void **)&t->p32, (void **)&t->h32, (void **)&t->nfirst, (void **)&t->ncount,
                  (void **)&t->naxis, (void **)&t->nsplit, (void **)&t->nsplitkey, (void **)&t->nS,
                  (void **)&t->nbmin, (void **)&t->nbmax, (void **)&t->nmass, (void **)&t->ncom, (void **)&t->nrg,
                  (void **)&t->nH, (void **)&t->nhint, (void **)&t->nhnode, (void **)&t->nQ, (void **)&t->w32,
                  (void **)&t->mq32a, (void **)&t->mq32b, (void **)&t->ncomdf, (void **)&t->nfar,
                  (void **)&t->narrive, (void **)&t->roots, (void **)&t->chunks, (void **)&t->cell_chunk0,
                  (void **)&t->chunk_part, (void **)&t->sinks, (void **)&t->sink_of_leaf, (void **)&t->near_nr,
                  (void **)&t->near_nn, (void **)&t->far_n, (void **)&t->near_list, (void **)&t->far_list,
                  (void **)&t->coef, (void **)&t->coef32, (void **)&t->nb_count, (void **)&t->nb_tmp, (void **)&t->nb_tstart, (void **)&t->nb_cursor, (void **)&t->nb_long, (void **)&t->scan_tmp, (void **)&t->tnear_off,
                  (void **)&t->tnear_sink, (void **)&t->tfar_off, (void **)&t->tfar_sink, (void **)&t->adj,
                  (void **)&t->dens_hl, (void **)&t->ones, (void **)&t->cand_list, (void **)&t->cand_far,
                  (void **)&t->cand_n, (void **)&t->mps_hist, (void **)&t->mps_prefix, (void **)&t->mps_rank};
    for (void **q : p) f(q);
}

void release_arrays(rcb_tree *t) {
    for_each_array(t, [&](void **q) {
        dev_free(t, *q);
        *q = nullptr;
    });
    t->cap_N = 0;
    t->cap_L = 0;
    t->cap_near = t->cap_far = 0;
    t->cap_lists_near = t->cap_lists_far = 0;
    t->cap_tmp = 0;
    t->cap_bwd_off = t->cap_bwd_cur = t->cap_bwd_sink = t->cap_bwd_N = t->cap_bwd_adj = 0;
}

int allocate_arrays(rcb_tree *t, int64_t N, int L) {
    const int64_t capN = N;
    const int64_t nn = (int64_t)2 << L, nl = (int64_t)1 << L;
    const int64_t cap_big = N / (kTcta + 1) + 2;
    const int64_t cap_chunks = std::max<int64_t>(N / kChunk + cap_big + 2, 4096);
    const int64_t cap_roots = 2 * (int64_t)(L + 1) * cap_big + 2;
    bool ok = true;
    auto A = [&](void **q, size_t bytes) {
        *q = dev_alloc(t, bytes);
        ok = ok && *q;
    };
    A((void **)&t->d_status, ST_NWORDS * sizeof(int));
    A((void **)&t->d_E, 4 * sizeof(int));
    A((void **)&t->d_nbig, (kMaxL + 2) * sizeof(int32_t));
    A((void **)&t->d_maxbits, 4 * sizeof(unsigned long long));
    A((void **)&t->d_pairs, 2 * sizeof(int64_t));
    for (int b = 0; b < 2; ++b) {
        A((void **)&t->bx[b], capN * sizeof(double));
        A((void **)&t->by[b], capN * sizeof(double));
        A((void **)&t->bz[b], capN * sizeof(double));
        A((void **)&t->bP[b], 4 * capN * sizeof(int64_t));
        A((void **)&t->bidx[b], capN * sizeof(int32_t));
        A((void **)&t->big_list[b], cap_big * sizeof(int32_t));
    }
    A((void **)&t->px, capN * sizeof(double));
    A((void **)&t->py, capN * sizeof(double));
    A((void **)&t->pz, capN * sizeof(double));
    A((void **)&t->pm, capN * sizeof(double));
    A((void **)&t->ph, capN * sizeof(double));
    A((void **)&t->pidx, capN * sizeof(int32_t));
    A((void **)&t->p32, capN * sizeof(float4));
    A((void **)&t->h32, capN * sizeof(float));
    A((void **)&t->nfirst, nn * sizeof(int32_t));
    A((void **)&t->ncount, nn * sizeof(int32_t));
    A((void **)&t->naxis, nn * sizeof(int32_t));
    A((void **)&t->nsplit, nn * sizeof(double));
    A((void **)&t->nsplitkey, nn * sizeof(int64_t));
    A((void **)&t->nS, 4 * nn * sizeof(i128));
    A((void **)&t->nbmin, 3 * nn * sizeof(int64_t));
    A((void **)&t->nbmax, 3 * nn * sizeof(int64_t));
    A((void **)&t->nmass, nn * sizeof(double));
    A((void **)&t->ncom, 3 * nn * sizeof(double));
    A((void **)&t->nrg, 3 * nn * sizeof(double));
    A((void **)&t->nH, nn * sizeof(double));
    A((void **)&t->nhint, nn * sizeof(double));
    A((void **)&t->nhnode, nn * sizeof(double));
    A((void **)&t->nQ, 6 * nn * sizeof(double));
    A((void **)&t->w32, 2 * nn * sizeof(float4));
    A((void **)&t->mq32a, nn * sizeof(float4));
    A((void **)&t->mq32b, nn * sizeof(float4));
    A((void **)&t->ncomdf, 3 * nn * sizeof(float2));
    A((void **)&t->nfar, 4 * nn * sizeof(float4));
    A((void **)&t->narrive, nn * sizeof(int32_t));
    A((void **)&t->roots, cap_roots * sizeof(int32_t));
    A((void **)&t->chunks, cap_chunks * sizeof(int4));
    A((void **)&t->cell_chunk0, cap_big * sizeof(int32_t));
    A((void **)&t->chunk_part, chunk_part_bytes(cap_chunks));
    A((void **)&t->sinks, nl * sizeof(int32_t));
    A((void **)&t->sink_of_leaf, nl * sizeof(int32_t));
    A((void **)&t->near_nr, nl * sizeof(int32_t));
    A((void **)&t->near_nn, nl * sizeof(int32_t));
    A((void **)&t->far_n, nl * sizeof(int32_t));
    A((void **)&t->coef, 20 * nl * sizeof(double));
    A((void **)&t->coef32, 20 * nl * sizeof(float));
    A((void **)&t->nb_count, (capN + 1) * sizeof(int64_t));
    A((void **)&t->nb_tstart, capN * sizeof(int64_t));
    A((void **)&t->nb_cursor, sizeof(unsigned long long));
    A((void **)&t->nb_long, capN * sizeof(int2));
    A((void **)&t->scan_tmp, (size_t)scan_tmp_bytes(std::max<int64_t>(capN + 1, nl)) + 256);
    if (!ok) return RCB_ERR_ALLOC;
    t->cap_N = capN;
    t->cap_L = L;
    t->cap_chunks = cap_chunks;
    t->cap_roots = cap_roots;
    return RCB_OK;
}

int ensure_lists(rcb_tree *t) {
    int64_t need_near = (int64_t)std::max(t->nsinks, 1) * std::max(t->cap_near, 32);
    int64_t need_far = (int64_t)std::max(t->nsinks, 1) * std::max(t->cap_far, 32);
    if (t->cap_near == 0) {
        t->cap_near = 96;
        t->cap_far = 224;
        need_near = (int64_t)std::max(t->nsinks, 1) * t->cap_near;
        need_far = (int64_t)std::max(t->nsinks, 1) * t->cap_far;
    }
    if (need_near > t->cap_lists_near) {
        dev_free(t, t->near_list);
        t->near_list = (int32_t *)dev_alloc(t, need_near * sizeof(int32_t));
        if (!t->near_list) return RCB_ERR_ALLOC;
        t->cap_lists_near = need_near;
    }
    if (need_far > t->cap_lists_far) {
        dev_free(t, t->far_list);
        t->far_list = (int32_t *)dev_alloc(t, need_far * sizeof(int32_t));
        if (!t->far_list) return RCB_ERR_ALLOC;
        t->cap_lists_far = need_far;
    }
    return RCB_OK;
}

}  // namespace
__global__ void k_copy_words(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

int copy_words(void *dst, const void *src, int64_t nwords, cudaStream_t st) {
    if (nwords <= 0) return RCB_OK;
    const int grid = (int)std::min<int64_t>((nwords + 255) / 256, 4096);
    k_copy_words<<<grid, 256, 0, st>>>((const uint32_t *)src, (uint32_t *)dst, nwords); note_launch();
    return cudaGetLastError() == cudaSuccess ? RCB_OK : RCB_ERR_CUDA;
}

__global__ void k_fill_ones(double *v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) v[i] = 1.0;
}

// unit weights for the centre-of-number split
int fill_ones(double *v, int64_t n, cudaStream_t st) {
    k_fill_ones<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(v, n); note_launch();
    return cudaGetLastError() == cudaSuccess ? RCB_OK : RCB_ERR_CUDA;
}

}  // namespace rcb

using namespace rcb;

extern "C" {

const char *rcb_strerror(int status) {
    switch (status) {
        case RCB_OK: return "ok";
        case RCB_ERR_ARG: return "invalid argument";
        case RCB_ERR_ALLOC: return "device allocation failed";
        case RCB_ERR_CAPACITY: return "output capacity too small";
        case RCB_ERR_CUDA: return "CUDA error";
        case RCB_ERR_LIMIT: return "bounded device loop gave up";
        case RCB_ERR_STATE: return "tree state does not allow this call";
        default: return "unknown status";
    }
}

int rcb_build(const double *x, const double *m, const double *h, int64_t N, const rcb_params *params,
              rcb_alloc_fn alloc, rcb_free_fn release, void *ctx, void *stream, rcb_tree **tree) {
    if (!tree || !params || !x || !m || !h) return RCB_ERR_ARG;
    if (N < 1 || N >= ((int64_t)1 << 31)) return RCB_ERR_ARG;
    if (params->n_ll < 1 || !(params->theta >= 0.0) || !std::isfinite(params->theta)) return RCB_ERR_ARG;
    if (params->precision != RCB_FP64 && params->precision != RCB_MIXED) return RCB_ERR_ARG;
    if ((params->flags & ~(RCB_FLAG_TIMING | RCB_FLAG_CENTRE_OF_NUMBER | RCB_FLAG_MAC_ONLY | RCB_FLAG_MEDIAN_SPLIT)) != 0)
        return RCB_ERR_ARG;
    if ((params->flags & RCB_FLAG_CENTRE_OF_NUMBER) && (params->flags & RCB_FLAG_MEDIAN_SPLIT)) return RCB_ERR_ARG;
    if ((alloc == nullptr) != (release == nullptr)) return RCB_ERR_ARG;
    const int L = depth_rule(N, params->n_ll);
    if (L > kMaxL) return RCB_ERR_ARG;

    rcb_tree *t = *tree;
    const bool created = t == nullptr;
    if (created) {
        t = new (std::nothrow) rcb_tree;
        if (!t) return RCB_ERR_ALLOC;
        std::memset((void *)t, 0, sizeof(rcb_tree));
        if (cudaMallocHost((void **)&t->h_status, 2 * ST_NWORDS * sizeof(int)) != cudaSuccess) {
            delete t;
            return RCB_ERR_CUDA;
        }
        if (cudaHostGetDevicePointer((void **)&t->h_status_dev, t->h_status, 0) != cudaSuccess) {
            cudaFreeHost(t->h_status);
            delete t;
            return RCB_ERR_CUDA;
        }
    }
    const bool new_alloc = t->alloc != alloc || t->release != release || t->ctx != ctx;
    if (!created && (new_alloc || N > t->cap_N || L > t->cap_L)) release_arrays(t);
    t->alloc = alloc;
    t->release = release;
    t->ctx = ctx;
    t->stream = (cudaStream_t)stream;
    t->params = *params;
    t->N = N;
    t->L = L;
    t->nn = (int64_t)2 << L;
    t->nleaves = (int64_t)1 << L;
    t->nb_valid = 0;
    t->bwd_valid = 0;
    t->near_pairs = t->cand_pairs = -1;
    int rc = RCB_OK;
    if (t->cap_N == 0) rc = allocate_arrays(t, N, L);
    stage_begin(t, SG_BUILD);
    if (rc == RCB_OK) {
        if (params->flags & RCB_FLAG_CENTRE_OF_NUMBER) {
            // every cell cut through its centre of number: the partition of unit weights, then the
            // nodes' mass-weighted moments by a refit (which keeps the splits)
            if (!t->ones) {
                t->ones = (double *)dev_alloc(t, (size_t)t->cap_N * sizeof(double));
                if (!t->ones) rc = RCB_ERR_ALLOC;
                else rc = fill_ones(t->ones, t->cap_N, t->stream);
            }
            if (rc == RCB_OK) rc = build_tree(t, x, t->ones, h);
            if (rc == RCB_OK) rc = refit_tree(t, x, m);
        } else {
            if ((params->flags & RCB_FLAG_MEDIAN_SPLIT) && !t->mps_hist) {
                const int64_t cap_big = t->cap_N / (kTcta + 1) + 2;
                t->mps_hist = (int32_t *)dev_alloc(t, (size_t)cap_big * 256 * sizeof(int32_t));
                t->mps_prefix = (unsigned long long *)dev_alloc(t, (size_t)cap_big * sizeof(unsigned long long));
                t->mps_rank = (int32_t *)dev_alloc(t, (size_t)cap_big * sizeof(int32_t));
                if (!t->mps_hist || !t->mps_prefix || !t->mps_rank) rc = RCB_ERR_ALLOC;
            }
            if (rc == RCB_OK) rc = build_tree(t, x, m, h);
        }
    }
    if (rc == RCB_OK) rc = ensure_lists(t);
    if (rc == RCB_OK) {
        stage_begin(t, SG_WALK);
        rc = walk_tree(t);
        stage_end(t, SG_WALK);
    }
    stage_end(t, SG_BUILD);
    if (rc != RCB_OK) {
        if (created) {
            rcb_free(t);
        }
        return rc;
    }
    *tree = t;
    return RCB_OK;
}

int rcb_neighbours(rcb_tree *tree, int64_t *offsets, int32_t *idx, int64_t capacity, int64_t *needed, void *stream) {
    if (!tree || !offsets || !needed) return RCB_ERR_ARG;
    tree->stream = (cudaStream_t)stream;
    return neighbours(tree, offsets, idx, capacity, needed);
}

int rcb_gravity(rcb_tree *tree, double *acc, double *pot, void *stream) {
    if (!tree || !acc) return RCB_ERR_ARG;
    tree->stream = (cudaStream_t)stream;
    return gravity(tree, acc, pot);
}

int rcb_gravity_neighbours(rcb_tree *tree, double *acc, double *pot, int64_t *offsets, int64_t *needed,
                           void *stream) {
    if (!tree || !acc || !offsets || !needed) return RCB_ERR_ARG;
    tree->stream = (cudaStream_t)stream;
    int rc = gravity_neighbours(tree, acc, pot);
    if (rc) return rc;
    return neighbours(tree, offsets, nullptr, 0, needed);
}

int rcb_gravity_backward(rcb_tree *tree, const double *g_acc, const double *g_pot, double *g_x, double *g_m,
                         void *stream) {
    if (!tree || !g_acc || !g_x || !g_m) return RCB_ERR_ARG;
    tree->stream = (cudaStream_t)stream;
    return gravity_backward(tree, g_acc, g_pot, g_x, g_m);
}

int rcb_refit(rcb_tree *tree, const double *x, const double *m, void *stream) {
    if (!tree || !x || !m) return RCB_ERR_ARG;
    tree->stream = (cudaStream_t)stream;
    return refit_tree(tree, x, m);
}

int rcb_update(rcb_tree *tree, const double *x, const double *m, const double *h, int32_t *rebuilt, void *stream) {
    if (!tree || !x || !m || !h) return RCB_ERR_ARG;
    tree->stream = (cudaStream_t)stream;
    int64_t outside = 0;
    int rc = rcb::integrity_outside(tree, x, &outside);
    if (rc) return rc;
    if (outside == 0) {
        // every particle is still in its ll-cell: new h, refit bottom-up, new lists
        if ((rc = rcb::gather_h(tree, h)) != RCB_OK) return rc;
        if ((rc = rcb::refit_tree(tree, x, m)) != RCB_OK) return rc;
        if ((rc = rcb::walk_tree(tree)) != RCB_OK) return rc;
        tree->nb_valid = 0;
        tree->bwd_valid = 0;
        tree->near_pairs = tree->cand_pairs = -1;
        if (rebuilt) *rebuilt = 0;
        return RCB_OK;
    }
    rcb_tree *t = tree;
    const rcb_params params = tree->params;
    rc = rcb_build(x, m, h, tree->N, &params, tree->alloc, tree->release, tree->ctx, stream, &t);
    if (rebuilt) *rebuilt = 1;
    return rc;
}

int rcb_density(rcb_tree *tree, const int64_t *offsets, const int32_t *idx, double *rho, void *stream) {
    if (!tree || !offsets || !idx || !rho) return RCB_ERR_ARG;
    tree->stream = (cudaStream_t)stream;
    return rcb::density(tree, offsets, idx, rho);
}

int rcb_set_precision(rcb_tree *tree, int32_t precision) {
    if (!tree || (precision != RCB_FP64 && precision != RCB_MIXED)) return RCB_ERR_ARG;
    tree->params.precision = precision;
    return RCB_OK;
}

int rcb_tree_info(const rcb_tree *t, int64_t *info) {
    if (!t || !info) return RCB_ERR_ARG;
    std::memset(info, 0, 16 * sizeof(int64_t));
    info[0] = t->N;
    info[1] = t->L;
    info[2] = t->nn;
    info[3] = t->nleaves;
    info[4] = t->nsinks;
    info[5] = t->cap_near;
    info[6] = t->cap_far;
    // list totals need the per-sink counts on the host
    if (t->nsinks > 0 && t->near_nr) {
        std::vector<int32_t> a(t->nsinks), b(t->nsinks), c(t->nsinks);
        if (cudaMemcpyAsync(a.data(), t->near_nr, t->nsinks * sizeof(int32_t), cudaMemcpyDeviceToHost, t->stream) ||
            cudaMemcpyAsync(b.data(), t->near_nn, t->nsinks * sizeof(int32_t), cudaMemcpyDeviceToHost, t->stream) ||
            cudaMemcpyAsync(c.data(), t->far_n, t->nsinks * sizeof(int32_t), cudaMemcpyDeviceToHost, t->stream) ||
            cudaStreamSynchronize(t->stream))
            return RCB_ERR_CUDA;
        int64_t sn = 0, sf = 0, sr = 0;
        for (int i = 0; i < t->nsinks; ++i) {
            sn += a[i] + b[i];
            sr += a[i];
            sf += c[i];
        }
        info[7] = sn;
        info[8] = sf;
        info[9] = sr;
    }
    info[10] = t->stats_fallback;
    info[11] = t->nroots_last;
    info[12] = t->params.precision;
    if (t->near_pairs < 0 && t->nsinks > 0) {
        if (count_pairs(const_cast<rcb_tree *>(t)) != RCB_OK) return RCB_ERR_CUDA;
    }
    info[13] = t->near_pairs;
    info[14] = t->cand_pairs;
    info[15] = launch_count();
    return RCB_OK;
}

int rcb_stage_times(rcb_tree *t, double *ms, void *stream) {
    if (!t || !ms) return RCB_ERR_ARG;
    for (int i = 0; i < 16; ++i) ms[i] = 0.0;
    if (!t->ev_ready) return RCB_OK;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return RCB_ERR_CUDA;
    if (cudaStreamSynchronize(t->stream) != cudaSuccess) return RCB_ERR_CUDA;
    for (int i = 0; i < 16; ++i) {
        if (!t->ev_used[i]) continue;
        float v = 0.f;
        if (cudaEventElapsedTime(&v, t->ev[2 * i], t->ev[2 * i + 1]) == cudaSuccess) ms[i] = v;
    }
    return RCB_OK;
}

int rcb_export_topology(rcb_tree *t, int32_t *leaf_of, int32_t *perm, int64_t *first, int64_t *count, int32_t *axis,
                        double *split, int64_t *sums, double *mass, double *com, double *bmin, double *bmax,
                        double *rg, double *H, double *hint, double *hnode, double *Q, void *stream) {
    if (!t) return RCB_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nn = t->nn, N = t->N;
    std::vector<int32_t> f32(nn), c32(nn), ax32(nn), pidx(N);
    std::vector<int64_t> kmin(3 * nn), kmax(3 * nn);
    std::vector<double> sp(nn), ms(nn), cm(3 * nn), g(3 * nn), hh(nn), hi(nn), hn(nn), q(6 * nn);
    std::vector<i128> S(4 * nn);
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
    };
    if (cp(f32.data(), t->nfirst, nn * 4) || cp(c32.data(), t->ncount, nn * 4) || cp(ax32.data(), t->naxis, nn * 4) ||
        cp(pidx.data(), t->pidx, N * 4) || cp(kmin.data(), t->nbmin, 3 * nn * 8) ||
        cp(kmax.data(), t->nbmax, 3 * nn * 8) || cp(sp.data(), t->nsplit, nn * 8) || cp(ms.data(), t->nmass, nn * 8) ||
        cp(cm.data(), t->ncom, 3 * nn * 8) || cp(g.data(), t->nrg, 3 * nn * 8) || cp(hh.data(), t->nH, nn * 8) ||
        cp(hi.data(), t->nhint, nn * 8) || cp(hn.data(), t->nhnode, nn * 8) || cp(q.data(), t->nQ, 6 * nn * 8) ||
        cp(S.data(), t->nS, 4 * nn * sizeof(i128)) || cudaStreamSynchronize(st))
        return RCB_ERR_CUDA;
    const int64_t leaf0 = t->nleaves;
    for (int64_t n = 0; n < nn; ++n) {
        const bool live = n > 0 && c32[n] > 0;
        const bool internal = n < leaf0;
        if (first) first[n] = live ? f32[n] : 0;
        if (count) count[n] = n > 0 ? c32[n] : 0;
        if (axis) axis[n] = live && internal ? ax32[n] : 0;
        if (split) split[n] = live && internal ? sp[n] : 0.0;
        if (sums)
            for (int k = 0; k < 4; ++k) {
                i128 v = live ? S[4 * n + k] : 0;
                sums[8 * n + 2 * k] = (int64_t)(uint64_t)(u128)v;
                sums[8 * n + 2 * k + 1] = (int64_t)(v >> 64);
            }
        if (mass) mass[n] = live ? ms[n] : 0.0;
        for (int d = 0; d < 3; ++d) {
            if (com) com[3 * n + d] = live ? cm[3 * n + d] : 0.0;
            if (bmin) bmin[3 * n + d] = live ? dkey_inv(kmin[3 * n + d]) : 0.0;
            if (bmax) bmax[3 * n + d] = live ? dkey_inv(kmax[3 * n + d]) : 0.0;
            if (rg) rg[3 * n + d] = live ? g[3 * n + d] : 0.0;
        }
        if (H) H[n] = live ? hh[n] : 0.0;
        if (hint) hint[n] = live ? hi[n] : 0.0;
        if (hnode) hnode[n] = live && !internal ? hn[n] : 0.0;
        if (Q)
            for (int k = 0; k < 6; ++k) Q[6 * n + k] = live ? q[6 * n + k] : 0.0;
    }
    if (perm) std::memcpy(perm, pidx.data(), N * sizeof(int32_t));
    if (leaf_of) {
        for (int64_t j = 0; j < t->nleaves; ++j) {
            int64_t n = leaf0 + j;
            if (c32[n] <= 0) continue;
            for (int64_t p = f32[n]; p < f32[n] + c32[n]; ++p) leaf_of[pidx[p]] = (int32_t)j;
        }
    }
    return RCB_OK;
}

int rcb_export_lists(rcb_tree *t, int64_t *near_off, int32_t *near_ids, uint8_t *near_reach, int64_t cap_near,
                     int64_t *far_off, int32_t *far_ids, int64_t cap_far, void *stream) {
    if (!t || !near_off || !near_ids || !near_reach || !far_off || !far_ids) return RCB_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int ns = t->nsinks;
    std::vector<int32_t> sinks(ns), nr(ns), nnr(ns), nf(ns);
    std::vector<int32_t> nl((size_t)ns * t->cap_near), fl((size_t)ns * t->cap_far);
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
    };
    if (ns > 0 && (cp(sinks.data(), t->sinks, ns * 4) || cp(nr.data(), t->near_nr, ns * 4) ||
                   cp(nnr.data(), t->near_nn, ns * 4) || cp(nf.data(), t->far_n, ns * 4) ||
                   cp(nl.data(), t->near_list, nl.size() * 4) || cp(fl.data(), t->far_list, fl.size() * 4)))
        return RCB_ERR_CUDA;
    if (cudaStreamSynchronize(st)) return RCB_ERR_CUDA;
    int64_t tn = 0, tf = 0;
    for (int i = 0; i < ns; ++i) {
        tn += nr[i] + nnr[i];
        tf += nf[i];
    }
    if (tn > cap_near || tf > cap_far) return RCB_ERR_CAPACITY;
    const int64_t leaf0 = t->nleaves;
    std::vector<int32_t> sink_of(t->nleaves, -1);
    for (int i = 0; i < ns; ++i) sink_of[sinks[i] - leaf0] = i;
    int64_t pn = 0, pf = 0;
    near_off[0] = 0;
    far_off[0] = 0;
    for (int64_t j = 0; j < t->nleaves; ++j) {
        int s = sink_of[j];
        if (s >= 0) {
            const int32_t *row = nl.data() + (size_t)s * t->cap_near;
            for (int k = 0; k < nr[s]; ++k) {
                near_ids[pn] = row[k];
                near_reach[pn++] = 1;
            }
            for (int k = 0; k < nnr[s]; ++k) {
                near_ids[pn] = row[t->cap_near - 1 - k];
                near_reach[pn++] = 0;
            }
            const int32_t *frow = fl.data() + (size_t)s * t->cap_far;
            for (int k = 0; k < nf[s]; ++k) far_ids[pf++] = frow[k];
        }
        near_off[j + 1] = pn;
        far_off[j + 1] = pf;
    }
    return RCB_OK;
}

void rcb_free(rcb_tree *tree) {
    if (!tree) return;
    release_arrays(tree);
    if (tree->ev_ready)
        for (int i = 0; i < 32; ++i) cudaEventDestroy(tree->ev[i]);
    if (tree->h_status) cudaFreeHost(tree->h_status);
    tree->h_status = nullptr;
    delete tree;
}

}  // extern "C"
