// Backward pass of gravity: vector-Jacobian product of (acc, pot) with respect to positions
// and masses, with the tree's particle sets and interaction lists held fixed (no counterpart
// in the paper; the forward it differentiates is Sec. 2.4).  Smoothing lengths are constants.
//
// Given v_a = dL/da_a and w_a = dL/dPhi_a (sorted order after a gather):
//   taylor   per sink: the coefficients C (Eq. 6) are recomputed in FP64; for every particle
//            dL/dd_a = w grad P(d_a) - Hess P(d_a) v_a goes to x_a and, negated, to the sink's
//            centre of mass; dL/dC = sum_a (w dP/dC - v . d(grad P)/dC) per sink.
//   far      per (sink A, far node B): the 20 coefficients are functions of x = COM_A - COM_B,
//            M_B and Q_B (Eq. 5).  dL/dx comes from the same coefficient code run on dual
//            numbers (value + 3 partials); dL/dM and dL/dQ from its linearity in M and Q.
//            dL/dx is added to COM_A's adjoint and subtracted from COM_B's; M_B and Q_B adjoints
//            accumulate per node (atomic adds).
//   near     pair terms are recomputed (never stored): the sink side pulls over its near list;
//            the source side pulls over a transposed near list (sinks that list the cell).
//   nodes    every particle climbs its ancestors and adds the moment adjoints of each node:
//            M = sum m_b, COM = sum m_b x_b / M, Q = sum m_b (3 d d - d^2 I), d = x_b - COM
//            (Eq. 1; Eq. 2 reproduces it exactly); Q has no derivative through the COM
//            because sum m_b d_b = 0.
#include <cuda_runtime.h>

#include <algorithm>

#include "far_math.cuh"
#include "rcb_internal.cuh"

namespace rcb {

// Forward-mode dual number with K partial derivatives (FP64).
template <int K>
struct Dual {
    double v;
    double d[K];
    __device__ Dual() {}
    __device__ Dual(double x) : v(x) {
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] = 0.0;
    }
};
template <int K>
__device__ inline Dual<K> operator+(const Dual<K> &a, const Dual<K> &b) {
    Dual<K> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <int K>
__device__ inline Dual<K> operator-(const Dual<K> &a, const Dual<K> &b) {
    Dual<K> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <int K>
__device__ inline Dual<K> operator-(const Dual<K> &a) {
    Dual<K> r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
    return r;
}
template <int K>
__device__ inline Dual<K> operator*(const Dual<K> &a, const Dual<K> &b) {
    Dual<K> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.v * b.d[k] + b.v * a.d[k];
    return r;
}
template <int K>
__device__ inline Dual<K> &operator+=(Dual<K> &a, const Dual<K> &b) {
    a = a + b;
    return a;
}
template <int K>
__device__ inline Dual<K> rsqrt(const Dual<K> &a) {
    Dual<K> r;
    r.v = ::rsqrt(a.v);
    const double f = -0.5 * r.v * r.v * r.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = f * a.d[k];
    return r;
}

namespace {

constexpr int kBW = 4;          // warps per block
constexpr int kBTile = 384;     // staged particles per warp
constexpr int kBGroup = 4;      // particles held in registers per pass

struct BCtx {
    int nsinks;
    int64_t nleaves;
    const int32_t *sinks, *sink_of_leaf, *near_list, *near_nr, *near_nn, *far_list, *far_n;
    int cap_near, cap_far;
    const int32_t *nfirst, *ncount;
    const double *ncom, *nmass, *nQ;
    const double *px, *py, *pz, *pm, *ph;
    const int32_t *pidx;
    const double *coef;     // [nsinks][20] FP64 coefficients (recomputed)
    double *cbar;           // [nsinks][20] dL/dC
    const double *gA, *gP;  // sorted order: [3N], [N]
    double *gxs, *gms;      // sorted-order accumulators
    double *adj;            // [nn][10]: M, COM x/y/z, Q (6 slots)
    const int32_t *tnear_off, *tnear_sink;  // transposed near list per leaf
    const int32_t *pleaf;
    const double *gacc, *gpot;
    double *gx, *gm;
    int64_t N;
    int L;
};

__global__ void k_bwd_gather(BCtx c) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.N; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = c.pidx[p];
        double *gA = const_cast<double *>(c.gA), *gP = const_cast<double *>(c.gP);
        gA[3 * p] = c.gacc[3 * o];
        gA[3 * p + 1] = c.gacc[3 * o + 1];
        gA[3 * p + 2] = c.gacc[3 * o + 2];
        gP[p] = c.gpot ? c.gpot[o] : 0.0;
    }
}

__global__ void k_bwd_pleaf(BCtx c) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = gw; s < c.nsinks; s += nw) {
        const int A = c.sinks[s];
        for (int p = c.nfirst[A] + lane; p < c.nfirst[A] + c.ncount[A]; p += 32) const_cast<int32_t *>(c.pleaf)[p] = A;
    }
}

// Taylor part: per sink (warp), lanes over its particles.
__global__ void __launch_bounds__(kBW * 32) k_bwd_taylor(BCtx c) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = gw; s < c.nsinks; s += nw) {
        const int A = c.sinks[s];
        const int f = c.nfirst[A], n = c.ncount[A];
        double C[20];
#pragma unroll
        for (int i = 0; i < 20; ++i) C[i] = c.coef[(int64_t)s * 20 + i];
        const double cA[3] = {c.ncom[3 * (int64_t)A], c.ncom[3 * (int64_t)A + 1], c.ncom[3 * (int64_t)A + 2]};
        double cb[20];
#pragma unroll
        for (int i = 0; i < 20; ++i) cb[i] = 0.0;
        double comb[3] = {0.0, 0.0, 0.0};
        for (int a0 = 0; a0 < n; a0 += 32) {
            const int a = f + a0 + lane;
            if (a0 + lane < n) {
                const double d[3] = {c.px[a] - cA[0], c.py[a] - cA[1], c.pz[a] - cA[2]};
                const double v[3] = {c.gA[3 * (int64_t)a], c.gA[3 * (int64_t)a + 1], c.gA[3 * (int64_t)a + 2]};
                const double w = c.gP[a];
                double g[3], H[6];
                taylor_grad_hess<double>(C, d[0], d[1], d[2], g, H);
                // dL/dd_k = w grad_k - sum_i v_i Hess_ik
                const double gd[3] = {w * g[0] - (v[0] * H[0] + v[1] * H[1] + v[2] * H[2]),
                                      w * g[1] - (v[0] * H[1] + v[1] * H[3] + v[2] * H[4]),
                                      w * g[2] - (v[0] * H[2] + v[1] * H[4] + v[2] * H[5])};
                c.gxs[3 * (int64_t)a] = gd[0];
                c.gxs[3 * (int64_t)a + 1] = gd[1];
                c.gxs[3 * (int64_t)a + 2] = gd[2];
                c.gms[a] = 0.0;
                comb[0] -= gd[0];
                comb[1] -= gd[1];
                comb[2] -= gd[2];
                taylor_cbar<double>(d[0], d[1], d[2], v[0], v[1], v[2], w, cb);
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
            for (int i = 0; i < 20; ++i) cb[i] += __shfl_xor_sync(0xffffffffu, cb[i], o);
#pragma unroll
            for (int k = 0; k < 3; ++k) comb[k] += __shfl_xor_sync(0xffffffffu, comb[k], o);
        }
        if (lane < 20) {
            double val = cb[0];
#pragma unroll
            for (int i = 1; i < 20; ++i)
                if (lane == i) val = cb[i];
            c.cbar[(int64_t)s * 20 + lane] = val;
        }
        if (lane < 3) {
            const double val = lane == 0 ? comb[0] : (lane == 1 ? comb[1] : comb[2]);
            atomicAdd(&c.adj[10 * (int64_t)A + 1 + lane], val);
        }
    }
}

// Far interactions: per sink (warp), lanes over its far nodes.
__global__ void __launch_bounds__(kBW * 32) k_bwd_far(BCtx c) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = gw; s < c.nsinks; s += nw) {
        const int A = c.sinks[s];
        const int nf = c.far_n[s];
        double cb[20];
#pragma unroll
        for (int i = 0; i < 20; ++i) cb[i] = c.cbar[(int64_t)s * 20 + i];
        const double cA[3] = {c.ncom[3 * (int64_t)A], c.ncom[3 * (int64_t)A + 1], c.ncom[3 * (int64_t)A + 2]};
        double RA[3] = {0.0, 0.0, 0.0};
        for (int k = lane; k < nf; k += 32) {
            const int B = c.far_list[(int64_t)s * c.cap_far + k];
            const double x[3] = {cA[0] - c.ncom[3 * (int64_t)B], cA[1] - c.ncom[3 * (int64_t)B + 1],
                                 cA[2] - c.ncom[3 * (int64_t)B + 2]};
            double q6[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) q6[q] = c.nQ[6 * (int64_t)B + q];
            const double M = c.nmass[B];
            // dL/dx by dual numbers
            Dual<3> xd[3], Qd[6], Cd[20];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                xd[i] = Dual<3>(x[i]);
                xd[i].d[i] = 1.0;
            }
#pragma unroll
            for (int q = 0; q < 6; ++q) Qd[q] = Dual<3>(q6[q]);
#pragma unroll
            for (int i = 0; i < 20; ++i) Cd[i] = Dual<3>(0.0);
            far_source<Dual<3>>(xd, Dual<3>(M), Qd, Cd);
            double Rb[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int i = 0; i < 20; ++i)
#pragma unroll
                for (int k2 = 0; k2 < 3; ++k2) Rb[k2] += cb[i] * Cd[i].d[k2];
            // dL/dM and dL/dQ: the coefficients are linear in M and in the stored Q slots
            double basis[20];
            const double zero6[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int i = 0; i < 20; ++i) basis[i] = 0.0;
            far_source<double>(x, 1.0, zero6, basis);
            double Mb = 0.0;
#pragma unroll
            for (int i = 0; i < 20; ++i) Mb += cb[i] * basis[i];
            atomicAdd(&c.adj[10 * (int64_t)B], Mb);
#pragma unroll 1
            for (int q = 0; q < 6; ++q) {
                double e6[6] = {0, 0, 0, 0, 0, 0};
                e6[q] = 1.0;
#pragma unroll
                for (int i = 0; i < 20; ++i) basis[i] = 0.0;
                far_source<double>(x, 0.0, e6, basis);
                double Qb = 0.0;
#pragma unroll
                for (int i = 0; i < 20; ++i) Qb += cb[i] * basis[i];
                atomicAdd(&c.adj[10 * (int64_t)B + 4 + q], Qb);
            }
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) {
                RA[k2] += Rb[k2];
                atomicAdd(&c.adj[10 * (int64_t)B + 1 + k2], -Rb[k2]);
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) RA[k2] += __shfl_xor_sync(0xffffffffu, RA[k2], o);
        if (lane < 3) {
            const double val = lane == 0 ? RA[0] : (lane == 1 ? RA[1] : RA[2]);
            atomicAdd(&c.adj[10 * (int64_t)A + 1 + lane], val);
        }
    }
}

// Stage particles [t0, t0 + kBTile) of a list of cells (cell ids given by a functor).
template <typename CellAt>
__device__ int stage_cells(const BCtx &c, int ncells, CellAt cell_at, int64_t t0, double *X, int32_t *I) {
    const int lane = threadIdx.x & 31;
    int64_t pos = 0;
    int staged = 0;
    for (int k0 = 0; k0 < ncells; k0 += 32) {
        const int k = k0 + lane;
        int f = 0, n = 0;
        if (k < ncells) {
            const int B = cell_at(k);
            f = c.nfirst[B];
            n = c.ncount[B];
        }
        int incl = n;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int64_t my0 = pos + incl - n;
        for (int j = 0; j < 32 && k0 + j < ncells; ++j) {
            const int64_t c0 = __shfl_sync(0xffffffffu, my0, j);
            const int cn = __shfl_sync(0xffffffffu, n, j);
            const int cf = __shfl_sync(0xffffffffu, f, j);
            const int64_t lo = c0 > t0 ? c0 : t0;
            const int64_t hi = c0 + cn < t0 + kBTile ? c0 + cn : t0 + kBTile;
            for (int64_t q = lo + lane; q < hi; q += 32) {
                const int b = cf + (int)(q - c0);
                const int slot = (int)(q - t0);
                X[slot] = c.px[b];
                X[kBTile + slot] = c.py[b];
                X[2 * kBTile + slot] = c.pz[b];
                X[3 * kBTile + slot] = c.pm[b];
                X[4 * kBTile + slot] = c.ph[b];
                X[5 * kBTile + slot] = c.gA[3 * (int64_t)b];
                X[6 * kBTile + slot] = c.gA[3 * (int64_t)b + 1];
                X[7 * kBTile + slot] = c.gA[3 * (int64_t)b + 2];
                X[8 * kBTile + slot] = c.gP[b];
                I[slot] = b;
            }
            if (hi > lo) staged = max(staged, (int)(hi - t0));
        }
        pos += total;
        if (pos >= t0 + kBTile) break;
    }
    __syncwarp();
    return staged;
}

constexpr size_t kBSmemPerWarp = kBTile * (9 * sizeof(double) + sizeof(int32_t));

// SIDE 0: sink side, a in the sink, b over the near cells: gxs[a] += g.
// SIDE 1: source side, b in a cell, a over the sinks listing it: gxs[b] -= g, gms[b] += gm.
template <int SIDE>
__global__ void __launch_bounds__(kBW * 32) k_bwd_near(BCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double *X = reinterpret_cast<double *>(smem_raw + (size_t)w * kBSmemPerWarp);
    int32_t *I = reinterpret_cast<int32_t *>(X + 9 * kBTile);
    const int nunits = SIDE == 0 ? c.nsinks : (int)c.nleaves;
    for (int u = blockIdx.x * kBW + w; u < nunits; u += gridDim.x * kBW) {
        int own, ncells = 0;
        int64_t list0 = 0;
        int nr = 0;
        if (SIDE == 0) {
            own = c.sinks[u];
            nr = c.near_nr[u];
            ncells = nr + c.near_nn[u];
            list0 = (int64_t)u * c.cap_near;
        } else {
            own = (int)c.nleaves + u;
            if (c.ncount[own] == 0) continue;
            list0 = c.tnear_off[u];
            ncells = c.tnear_off[u + 1] - c.tnear_off[u];
        }
        auto cell_at = [&](int k) -> int {
            if (SIDE == 0) return k < nr ? c.near_list[list0 + k] : c.near_list[list0 + c.cap_near - 1 - (k - nr)];
            return c.sinks[c.tnear_sink[list0 + k]];
        };
        int64_t S = 0;
        for (int k = lane; k < ncells; k += 32) S += c.ncount[cell_at(k)];
        for (int o = 16; o >= 1; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
        const int f = c.nfirst[own], n = c.ncount[own];
        for (int p0 = 0; p0 < n; p0 += kBGroup) {
            const int np = min(kBGroup, n - p0);
            double ox[kBGroup], oy[kBGroup], oz[kBGroup], oh[kBGroup], om[kBGroup], ovx[kBGroup], ovy[kBGroup],
                ovz[kBGroup], ow[kBGroup];
            int oid[kBGroup];
#pragma unroll
            for (int i = 0; i < kBGroup; ++i) {
                const int p = f + p0 + min(i, np - 1);
                ox[i] = c.px[p];
                oy[i] = c.py[p];
                oz[i] = c.pz[p];
                oh[i] = c.ph[p];
                om[i] = c.pm[p];
                ovx[i] = c.gA[3 * (int64_t)p];
                ovy[i] = c.gA[3 * (int64_t)p + 1];
                ovz[i] = c.gA[3 * (int64_t)p + 2];
                ow[i] = c.gP[p];
                oid[i] = i < np ? p : -1;
            }
            double acc[4][kBGroup];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int i = 0; i < kBGroup; ++i) acc[q][i] = 0.0;
            for (int64_t t0 = 0; t0 < S; t0 += kBTile) {
                const int ns = stage_cells(c, ncells, cell_at, t0, X, I);
                for (int q0 = 0; q0 < ns; q0 += 32) {
                    const int j = q0 + lane;
                    if (j >= ns) continue;
                    const double jx = X[j], jy = X[kBTile + j], jz = X[2 * kBTile + j], jm = X[3 * kBTile + j],
                                 jh = X[4 * kBTile + j];
                    const double jvx = X[5 * kBTile + j], jvy = X[6 * kBTile + j], jvz = X[7 * kBTile + j],
                                 jw = X[8 * kBTile + j];
                    const int jid = I[j];
#pragma unroll
                    for (int i = 0; i < kBGroup; ++i) {
                        if (i < np && jid != oid[i]) {
                            double gx, gy, gz, gmv;
                            if (SIDE == 0) {  // a = own particle, b = staged
                                pair_grad<double>(ox[i] - jx, oy[i] - jy, oz[i] - jz, oh[i] + jh, jm, ovx[i], ovy[i],
                                                  ovz[i], ow[i], gx, gy, gz, gmv);
                                acc[0][i] += gx;
                                acc[1][i] += gy;
                                acc[2][i] += gz;
                            } else {  // a = staged, b = own particle
                                pair_grad<double>(jx - ox[i], jy - oy[i], jz - oz[i], jh + oh[i], om[i], jvx, jvy, jvz,
                                                  jw, gx, gy, gz, gmv);
                                acc[0][i] -= gx;
                                acc[1][i] -= gy;
                                acc[2][i] -= gz;
                                acc[3][i] += gmv;
                            }
                        }
                    }
                }
                __syncwarp();
            }
            double V[16];
#pragma unroll
            for (int i = 0; i < kBGroup; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) V[4 * i + q] = acc[q][i];
            reduce_scatter<16, double>(V);
            const double tot = V[0];
            const double q0v = __shfl_sync(0xffffffffu, tot, (4 * lane) & 15);
            const double q1v = __shfl_sync(0xffffffffu, tot, (4 * lane + 1) & 15);
            const double q2v = __shfl_sync(0xffffffffu, tot, (4 * lane + 2) & 15);
            const double q3v = __shfl_sync(0xffffffffu, tot, (4 * lane + 3) & 15);
            if (lane < np) {
                const int p = f + p0 + lane;
                c.gxs[3 * (int64_t)p] += q0v;
                c.gxs[3 * (int64_t)p + 1] += q1v;
                c.gxs[3 * (int64_t)p + 2] += q2v;
                if (SIDE == 1) c.gms[p] += q3v;
            }
        }
        __syncwarp();
    }
}

// Transposed near list: for every ll-cell B, the sinks whose near list holds B.
__global__ void k_tnear_count(BCtx c, int32_t *cnt) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = gw; s < c.nsinks; s += nw) {
        const int nr = c.near_nr[s], nl = nr + c.near_nn[s];
        const int64_t base = (int64_t)s * c.cap_near;
        for (int k = lane; k < nl; k += 32) {
            const int B = k < nr ? c.near_list[base + k] : c.near_list[base + c.cap_near - 1 - (k - nr)];
            atomicAdd(&cnt[B - c.nleaves], 1);
        }
    }
}

__global__ void k_tnear_fill(BCtx c, int32_t *cursor, int32_t *out) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = gw; s < c.nsinks; s += nw) {
        const int nr = c.near_nr[s], nl = nr + c.near_nn[s];
        const int64_t base = (int64_t)s * c.cap_near;
        for (int k = lane; k < nl; k += 32) {
            const int B = k < nr ? c.near_list[base + k] : c.near_list[base + c.cap_near - 1 - (k - nr)];
            const int slot = atomicAdd(&cursor[B - c.nleaves], 1);
            out[slot] = s;
        }
    }
}

// Sort each transposed row (insertion sort by one thread: rows are short) for a fixed order.
__global__ void k_tnear_sort(const int32_t *off, int64_t nleaves, int32_t *rows) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nleaves; j += (int64_t)gridDim.x * blockDim.x) {
        const int a = off[j], b = off[j + 1];
        for (int i = a + 1; i < b; ++i) {
            const int v = rows[i];
            int k = i - 1;
            while (k >= a && rows[k] > v) {
                rows[k + 1] = rows[k];
                --k;
            }
            rows[k + 1] = v;
        }
    }
}

// Node adjoints to particles (climb), then scatter to original order.
__global__ void k_bwd_nodes(BCtx c) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.N; p += (int64_t)gridDim.x * blockDim.x) {
        const double x[3] = {c.px[p], c.py[p], c.pz[p]};
        const double mb = c.pm[p];
        double gx[3] = {c.gxs[3 * p], c.gxs[3 * p + 1], c.gxs[3 * p + 2]};
        double gm = c.gms[p];
        for (int n = c.pleaf[p]; n >= 1; n >>= 1) {
            const double *a = c.adj + 10 * (int64_t)n;
            const double Mb = a[0];
            const double Cb[3] = {a[1], a[2], a[3]};
            const double Qb[6] = {a[4], a[5], a[6], a[7], a[8], a[9]};
            bool nz = Mb != 0.0 || Cb[0] != 0.0 || Cb[1] != 0.0 || Cb[2] != 0.0;
#pragma unroll
            for (int q = 0; q < 6; ++q) nz = nz || Qb[q] != 0.0;
            if (!nz) continue;
            const double M = c.nmass[n];
            double d[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) d[k] = x[k] - c.ncom[3 * (int64_t)n + k];
            const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            gm += Mb + (Cb[0] * d[0] + Cb[1] * d[1] + Cb[2] * d[2]) / M;
            // slots xx, xy, xz, yy, yz, zz of Q = sum m (3 d d - d^2 I):
            //   dQ_ij/dm = 3 d_i d_j - d^2 d_ij
            //   dQ_ij/dx_k = m (3 (d_ik d_j + d_i d_jk) - 2 d_k d_ij)
            gm += Qb[0] * (3.0 * d[0] * d[0] - d2) + Qb[1] * 3.0 * d[0] * d[1] + Qb[2] * 3.0 * d[0] * d[2] +
                  Qb[3] * (3.0 * d[1] * d[1] - d2) + Qb[4] * 3.0 * d[1] * d[2] + Qb[5] * (3.0 * d[2] * d[2] - d2);
            const double tr = Qb[0] + Qb[3] + Qb[5];
            gx[0] += mb * (6.0 * Qb[0] * d[0] + 3.0 * Qb[1] * d[1] + 3.0 * Qb[2] * d[2] - 2.0 * tr * d[0]);
            gx[1] += mb * (3.0 * Qb[1] * d[0] + 6.0 * Qb[3] * d[1] + 3.0 * Qb[4] * d[2] - 2.0 * tr * d[1]);
            gx[2] += mb * (3.0 * Qb[2] * d[0] + 3.0 * Qb[4] * d[1] + 6.0 * Qb[5] * d[2] - 2.0 * tr * d[2]);
#pragma unroll
            for (int k = 0; k < 3; ++k) gx[k] += Cb[k] * mb / M;
        }
        const int64_t o = c.pidx[p];
        c.gx[3 * o] = gx[0];
        c.gx[3 * o + 1] = gx[1];
        c.gx[3 * o + 2] = gx[2];
        c.gm[o] = gm;
    }
}

int sm_count_b() {
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

int far_coefficients_fp64(rcb_tree *t);  // gravity.cu

int gravity_backward(rcb_tree *t, const double *gacc, const double *gpot, double *gx, double *gm) {
    cudaStream_t st = t->stream;
    const int64_t N = t->N, nn = t->nn, nl = t->nleaves;
    if (t->nsinks == 0) return RCB_OK;
    // scratch, allocated on the first backward after a build (through the tree's allocator)
    if (!t->bwd_valid) {
        dev_free(t, t->tnear_off);
        dev_free(t, t->tnear_sink);
        dev_free(t, t->tfar_off);
        dev_free(t, t->tfar_sink);
        dev_free(t, t->adj);
        int64_t total = 0;
        {
            // total near entries
            int64_t info[16];
            if (rcb_tree_info(t, info) != RCB_OK) return RCB_ERR_CUDA;
            total = info[7];
        }
        t->tnear_off = (int32_t *)dev_alloc(t, (nl + 1) * sizeof(int32_t));
        t->tnear_sink = (int32_t *)dev_alloc(t, std::max<int64_t>(total, 1) * sizeof(int32_t));
        t->tfar_off = (int32_t *)dev_alloc(t, std::max<int64_t>(nl, 1) * sizeof(int32_t));   // cursor scratch
        t->tfar_sink = (int32_t *)dev_alloc(t, N * sizeof(int32_t));                          // leaf of each particle
        t->adj = (double *)dev_alloc(t, (size_t)nn * 10 * sizeof(double) + (size_t)N * 8 * sizeof(double) +
                                            (size_t)t->nsinks * 20 * sizeof(double));
        if (!t->tnear_off || !t->tnear_sink || !t->tfar_off || !t->tfar_sink || !t->adj) return RCB_ERR_ALLOC;
    }
    double *adj = t->adj;
    double *gxs = adj + nn * 10;
    double *gms = gxs + 3 * N;
    double *gA = gms + N;
    double *gP = gA + 3 * N;
    double *cbar = gP + N;
    BCtx c;
    c.nsinks = t->nsinks;
    c.nleaves = nl;
    c.sinks = t->sinks;
    c.sink_of_leaf = t->sink_of_leaf;
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
    c.px = t->px;
    c.py = t->py;
    c.pz = t->pz;
    c.pm = t->pm;
    c.ph = t->ph;
    c.pidx = t->pidx;
    c.coef = t->coef;
    c.cbar = cbar;
    c.gA = gA;
    c.gP = gP;
    c.gxs = gxs;
    c.gms = gms;
    c.adj = adj;
    c.tnear_off = t->tnear_off;
    c.tnear_sink = t->tnear_sink;
    c.pleaf = t->tfar_sink;
    c.gacc = gacc;
    c.gpot = gpot;
    c.gx = gx;
    c.gm = gm;
    c.N = N;
    c.L = t->L;
    const int nsm = sm_count_b();
    const int gridp = (int)std::min<int64_t>((N + 255) / 256, (int64_t)nsm * 8);
    const int gridw = std::max(1, std::min((t->nsinks + kBW - 1) / kBW, nsm * 16));
    stage_begin(t, SG_BWD);
    if (!t->bwd_valid) {
        int32_t *cnt = t->tfar_off;
        RCB_CUDA_TRY(cudaMemsetAsync(cnt, 0, nl * sizeof(int32_t), st));
        k_tnear_count<<<gridw, kBW * 32, 0, st>>>(c, cnt); note_launch();
        int rc = scan_i32(cnt, t->tnear_off, nl, t->tnear_off + nl, t->scan_tmp, st);
        if (rc) return rc;
        RCB_CUDA_TRY(cudaMemcpyAsync(cnt, t->tnear_off, nl * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        k_tnear_fill<<<gridw, kBW * 32, 0, st>>>(c, cnt, t->tnear_sink); note_launch();
        k_tnear_sort<<<(int)std::min<int64_t>((nl + 255) / 256, (int64_t)nsm * 8), 256, 0, st>>>(t->tnear_off, nl,
                                                                                            t->tnear_sink); note_launch();
        k_bwd_pleaf<<<gridw, kBW * 32, 0, st>>>(c); note_launch();
        RCB_CUDA_TRY(cudaGetLastError());
        t->bwd_valid = 1;
    }
    int rc = far_coefficients_fp64(t);
    if (rc) return rc;
    RCB_CUDA_TRY(cudaMemsetAsync(adj, 0, (size_t)nn * 10 * sizeof(double), st));
    k_bwd_gather<<<gridp, 256, 0, st>>>(c); note_launch();
    k_bwd_taylor<<<gridw, kBW * 32, 0, st>>>(c); note_launch();
    k_bwd_far<<<gridw, kBW * 32, 0, st>>>(c); note_launch();
    const size_t smem = kBW * kBSmemPerWarp;
    RCB_CUDA_TRY(cudaFuncSetAttribute(k_bwd_near<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RCB_CUDA_TRY(cudaFuncSetAttribute(k_bwd_near<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_bwd_near<0><<<gridw, kBW * 32, smem, st>>>(c); note_launch();
    const int gridl = (int)std::max<int64_t>(1, std::min<int64_t>((nl + kBW - 1) / kBW, (int64_t)nsm * 16));
    k_bwd_near<1><<<gridl, kBW * 32, smem, st>>>(c); note_launch();
    k_bwd_nodes<<<gridp, 256, 0, st>>>(c); note_launch();
    stage_end(t, SG_BWD);
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

}  // namespace rcb
