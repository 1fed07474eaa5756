// SPH density by summation over the neighbour lists (Sec. 2.3: smoothed quantities are sums of
// kernel-weighted properties of the neighbours), the first consumer of rcb_neighbours' CSR:
//   rho_a = (m_a w(0) + sum_{b in nb(a)} m_b w(r_ab / h_a)) / (pi h_a^3),
//   w(q) = 1 - 3/2 q^2 + 3/4 q^3 (q < 1), (2 - q)^3 / 4 (1 <= q < 2), 0 beyond,
// the cubic spline the paper uses (support 2h).  The positions are split once per particle into
// float32 pairs (hi, lo) with x = hi + lo to about 2^-48 |x|, so the pair offsets
// (hi_a - hi_b) + (lo_a - lo_b) keep float32 relative accuracy at any distance; w and the sum run
// in float32 (one warp per particle), the result is stored in float64.
#include <cuda_runtime.h>

#include <algorithm>

#include "rcb_internal.cuh"

namespace rcb {
namespace {

// Per particle, original order: (hi x, hi y, hi z, m) and (lo x, lo y, lo z, 1 / h).
__global__ void k_density_split(const double *px, const double *py, const double *pz, const double *pm,
                                const double *ph, const int32_t *pidx, int64_t N, float4 *hl) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        const double x = px[p], y = py[p], z = pz[p];
        const float hx = __double2float_rn(x), hy = __double2float_rn(y), hz = __double2float_rn(z);
        const int64_t o = pidx[p];
        hl[2 * o] = make_float4(hx, hy, hz, __double2float_rn(pm[p]));
        hl[2 * o + 1] = make_float4(__double2float_rn(x - (double)hx), __double2float_rn(y - (double)hy),
                                    __double2float_rn(z - (double)hz), __double2float_rn(1.0 / ph[p]));
    }
}

__device__ inline float spline_w(float q) {
    if (q < 1.f) return fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.f);
    if (q < 2.f) {
        const float t = 2.f - q;
        return 0.25f * t * t * t;
    }
    return 0.f;
}

__global__ void k_density(const float4 *hl, int64_t N, const int64_t *off, const int32_t *idx, double *rho) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = gw; a < N; a += nw) {
        const float4 ha = hl[2 * a], la = hl[2 * a + 1];
        const float hinv = la.w;
        float s = 0.f;
        for (int64_t k = off[a] + lane; k < off[a + 1]; k += 32) {
            const int64_t b = idx[k];
            const float4 hb = hl[2 * b], lb = hl[2 * b + 1];
            const float dx = (ha.x - hb.x) + (la.x - lb.x), dy = (ha.y - hb.y) + (la.y - lb.y),
                        dz = (ha.z - hb.z) + (la.z - lb.z);
            const float r = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
            s = fmaf(hb.w, spline_w(r * hinv), s);
        }
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const double hi = (double)hinv;
            rho[a] = ((double)s + (double)ha.w) * (hi * hi * hi) * 0.31830988618379067;  // 1 / pi
        }
    }
}

int sm_count_d() {
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

int density(rcb_tree *t, const int64_t *offsets, const int32_t *idx, double *rho) {
    if (t->N <= 0) return RCB_ERR_STATE;
    cudaStream_t st = t->stream;
    if (!t->dens_hl) {
        t->dens_hl = (float4 *)dev_alloc(t, (size_t)t->cap_N * 2 * sizeof(float4));
        if (!t->dens_hl) return RCB_ERR_ALLOC;
    }
    const int nsm = sm_count_d();
    const int gp = (int)std::max<int64_t>(1, std::min<int64_t>((t->N + 255) / 256, (int64_t)nsm * 8));
    k_density_split<<<gp, 256, 0, st>>>(t->px, t->py, t->pz, t->pm, t->ph, t->pidx, t->N, t->dens_hl); note_launch();
    const int gw = (int)std::max<int64_t>(1, std::min<int64_t>((t->N + 7) / 8, (int64_t)nsm * 16));
    k_density<<<gw, 256, 0, st>>>(t->dens_hl, t->N, offsets, idx, rho); note_launch();
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

}  // namespace rcb
