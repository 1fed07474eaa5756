// Backward pass of gravity: vector-Jacobian product of (acc, pot) with respect to positions
// and masses, with the tree's particle sets and interaction lists held fixed (no counterpart
// in the paper; the forward it differentiates is Sec. 2.4).  Smoothing lengths are constants.
//
// Given v_a = dL/da_a and w_a = dL/dPhi_a (sorted order after a gather):
//   taylor   per sink: the coefficients C (Eq. 6) are recomputed; for every particle
//            dL/dd_a = w grad P(d_a) - Hess P(d_a) v_a goes to x_a and, negated, to the sink's
//            centre of mass; dL/dC = sum_a (w dP/dC - v . d(grad P)/dC) per sink.
//   far      per (sink A, far node B): the 20 coefficients are functions of x = COM_A - COM_B,
//            M_B and Q_B (Eq. 5); one hand-written reverse of that formula gives dL/dx, dL/dM
//            and dL/dQ.  dL/dx is added to COM_A's adjoint and subtracted from COM_B's; M_B and
//            Q_B adjoints accumulate per node (atomic adds).
//   near     pair terms are recomputed (never stored): the sink side pulls over its near list;
//            the source side pulls over a transposed near list (sinks that list the cell).
//   nodes    a node's adjoints reach the particles below it through a quadratic polynomial of
//            the particle's position (from M = sum m_b, COM = sum m_b x_b / M,
//            Q = sum m_b (3 d d - d^2 I), Eq. 1); the polynomials of all ancestors are summed
//            top-down, re-centred on each node's centre of mass, and evaluated once per particle.
// The FP64 form runs every step in FP64.  The mixed form takes the float32 coefficients of the
// mixed forward and runs the Taylor, far and near parts in float32 (compensated per-tile sums in
// the near part); node adjoints and the polynomials stay FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "far_math.cuh"
#include "nb_rows.cuh"
#include "rcb_internal.cuh"

namespace rcb {

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
    const float4 *nfar;     // mixed form: per node (COM hi, M), (COM lo, Qxx), (Qxy, Qxz, Qyy, Qyz), (Qzz)
    const float2 *ncomdf;   // mixed form: double-float centres of mass
    const float4 *p32;      // mixed form: (x - COM of the particle's leaf, m)
    const float *h32;
    const int32_t *pidx;
    const double *coef;     // [nsinks][20] coefficients in the tree's precision (recomputed)
    double *cbar;           // [nsinks][20] dL/dC
    float *cbar32;          // mixed form: the same in float32
    float4 *gv32;           // mixed form: (dL/da, dL/dPhi) per particle in float32, sorted order
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
        if (c.gv32)
            c.gv32[p] = make_float4((float)gA[3 * p], (float)gA[3 * p + 1], (float)gA[3 * p + 2], (float)gP[p]);
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

// Taylor part, mixed form: the same in float32 from the float coefficients and the particle
// offsets from the sink's centre of mass.
__global__ void __launch_bounds__(kBW * 32) k_bwd_taylor_mixed(BCtx c, const float *coef32) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = gw; s < c.nsinks; s += nw) {
        const int A = c.sinks[s];
        const int f = c.nfirst[A], n = c.ncount[A];
        float C[20];
#pragma unroll
        for (int i = 0; i < 20; ++i) C[i] = coef32[(int64_t)s * 20 + i];
        float cb[20];
#pragma unroll
        for (int i = 0; i < 20; ++i) cb[i] = 0.f;
        float comb[3] = {0.f, 0.f, 0.f};
        for (int a0 = 0; a0 < n; a0 += 32) {
            const int a = f + a0 + lane;
            if (a0 + lane < n) {
                const float4 pa = c.p32[a];
                const float4 gv = c.gv32[a];
                const float v[3] = {gv.x, gv.y, gv.z};
                const float w = gv.w;
                float g[3], H[6];
                taylor_grad_hess<float>(C, pa.x, pa.y, pa.z, g, H);
                const float gd[3] = {w * g[0] - (v[0] * H[0] + v[1] * H[1] + v[2] * H[2]),
                                     w * g[1] - (v[0] * H[1] + v[1] * H[3] + v[2] * H[4]),
                                     w * g[2] - (v[0] * H[2] + v[1] * H[4] + v[2] * H[5])};
                c.gxs[3 * (int64_t)a] = gd[0];
                c.gxs[3 * (int64_t)a + 1] = gd[1];
                c.gxs[3 * (int64_t)a + 2] = gd[2];
                c.gms[a] = 0.0;
                comb[0] -= gd[0];
                comb[1] -= gd[1];
                comb[2] -= gd[2];
                taylor_cbar<float>(pa.x, pa.y, pa.z, v[0], v[1], v[2], w, cb);
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
            float val = cb[0];
#pragma unroll
            for (int i = 1; i < 20; ++i)
                if (lane == i) val = cb[i];
            c.cbar32[(int64_t)s * 20 + lane] = val;
        }
        if (lane < 3) atomicAdd(&c.adj[10 * (int64_t)A + 1 + lane], (double)(lane == 0 ? comb[0] : (lane == 1 ? comb[1] : comb[2])));
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

// Far interactions: per sink (warp), lanes over its far nodes, by a hand-written reverse of the
// coefficient formula (far_source).  With P1, P2, P3 the coefficient adjoints spread over the full
// symmetric tensors (a slot's adjoint divided by its multiplicity), t3_k = P3_iik, T = P3 x,
// u = T x, v = Q x, s = x.v and the scalars of far_source (a, b, c; d = -105 M g^9 - 3465/2 s g^13
// continues the sequence),
//   L = sum cbar.C = M mu + sigma s + nu.v + Q:K,
//   alpha = P1.x + tr P2,  beta = x.P2 x + 3 t3.x,  gamma = u.x,
//   mu    = g^3 alpha - 3 g^5 beta + 15 g^7 gamma - cbar_0 g                      (= dL/dM)
//   sigma = 5/2 g^7 alpha - 35/2 g^9 beta + 315/2 g^11 gamma - cbar_0 g^5 / 2
//   nu    = -g^5 P1 + 10 g^7 P2 x - 105 g^9 u + 15 g^7 t3,   K = -g^5 P2 + 15 g^7 T,
//   dL/dQ_ij = sigma x_i x_j + nu_i x_j + K_ij (summed over (i, j) and (j, i) for off-diagonal slots),
//   dL/dx = x S + a P1 + b (2 P2 x + 3 t3) + 3 c u + 2 sigma v + Q nu + 10 g^7 P2 v - 210 g^9 T v
//           + 15 g^7 W,   W_k = Q_ij P3_ijk,
//   S = cbar_0 a + alpha b + beta c + gamma d + 5 g^7 (P1.v + Q:P2) - 70 g^9 v.P2 x
//       - 105 g^9 (t3.v + Q:T) + 945 g^11 u.v.
// dL/dx is added to COM_A's adjoint and subtracted from COM_B's; M_B and Q_B adjoints accumulate
// per node (FP64 atomic adds).  The mixed form reads the offsets from the double-float node
// records as the forward does and computes in float32.
template <typename T>
struct FarCbar {
    T cb0, P1[3], p2xx, p2xy, p2xz, p2yy, p2yz, p2zz, p3[10], t3[3], trP2;
    template <typename S>
    __device__ explicit FarCbar(const S *cbs) {
        cb0 = (T)cbs[0];
        P1[0] = (T)cbs[1];
        P1[1] = (T)cbs[2];
        P1[2] = (T)cbs[3];
        // slots xx, xy, xz, yy, yz, zz
        p2xx = (T)cbs[4];
        p2xy = T(0.5) * (T)cbs[5];
        p2xz = T(0.5) * (T)cbs[6];
        p2yy = (T)cbs[7];
        p2yz = T(0.5) * (T)cbs[8];
        p2zz = (T)cbs[9];
        // slots xxx, xxy, xxz, xyy, xyz, xzz, yyy, yyz, yzz, zzz (multiplicities 1 3 3 3 6 3 1 3 3 1)
        const T mult[10] = {T(1), T(3), T(3), T(3), T(6), T(3), T(1), T(3), T(3), T(1)};
#pragma unroll
        for (int i = 0; i < 10; ++i) p3[i] = (T)cbs[10 + i] / mult[i];
        t3[0] = p3[0] + p3[3] + p3[5];
        t3[1] = p3[1] + p3[6] + p3[8];
        t3[2] = p3[2] + p3[7] + p3[9];
        trP2 = p2xx + p2yy + p2zz;
    }
};

template <typename T>
__device__ inline T rsqrt_t(T x);
template <>
__device__ inline float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ inline double rsqrt_t<double>(double x) { return rsqrt(x); }

// Adjoints of one (sink, far node) pair: mu = dL/dM, q = dL/dQ slots, gx = dL/dx.
template <typename T>
__device__ inline void far_adjoint(const FarCbar<T> &P, T x0, T x1, T x2, T M, T Qxx, T Qxy, T Qxz, T Qyy, T Qyz,
                                   T Qzz, T &mu, T q[6], T gx[3]) {
    const T rr = x0 * x0 + x1 * x1 + x2 * x2;
    const T g = rsqrt_t(rr), g2 = g * g, g3 = g * g2, g5 = g3 * g2, g7 = g5 * g2, g9 = g7 * g2, g11 = g9 * g2;
    const T v0 = Qxx * x0 + Qxy * x1 + Qxz * x2, v1 = Qxy * x0 + Qyy * x1 + Qyz * x2,
            v2 = Qxz * x0 + Qyz * x1 + Qzz * x2;
    const T sv = x0 * v0 + x1 * v1 + x2 * v2;
    const T gs = sv * g2;  // s g^2 keeps s g^13 = (s g^2) g^11 in range
    const T *p3 = P.p3;
    // T = P3 x (symmetric), u = T x, gamma = u.x
    const T Txx = p3[0] * x0 + p3[1] * x1 + p3[2] * x2, Txy = p3[1] * x0 + p3[3] * x1 + p3[4] * x2,
            Txz = p3[2] * x0 + p3[4] * x1 + p3[5] * x2, Tyy = p3[3] * x0 + p3[6] * x1 + p3[7] * x2,
            Tyz = p3[4] * x0 + p3[7] * x1 + p3[8] * x2, Tzz = p3[5] * x0 + p3[8] * x1 + p3[9] * x2;
    const T u0 = Txx * x0 + Txy * x1 + Txz * x2, u1 = Txy * x0 + Tyy * x1 + Tyz * x2,
            u2 = Txz * x0 + Tyz * x1 + Tzz * x2;
    const T gam = u0 * x0 + u1 * x1 + u2 * x2;
    const T w0 = P.p2xx * x0 + P.p2xy * x1 + P.p2xz * x2, w1 = P.p2xy * x0 + P.p2yy * x1 + P.p2yz * x2,
            w2 = P.p2xz * x0 + P.p2yz * x1 + P.p2zz * x2;  // P2 x
    const T alpha = P.P1[0] * x0 + P.P1[1] * x1 + P.P1[2] * x2 + P.trP2;
    const T beta = w0 * x0 + w1 * x1 + w2 * x2 + T(3) * (P.t3[0] * x0 + P.t3[1] * x1 + P.t3[2] * x2);
    const T a = M * g3 + T(2.5) * gs * g5, b = T(-3) * M * g5 - T(17.5) * gs * g7,
            cc = T(15) * M * g7 + T(157.5) * gs * g9, d = T(-105) * M * g9 - T(1732.5) * gs * g11;
    mu = g3 * alpha - T(3) * g5 * beta + T(15) * g7 * gam - P.cb0 * g;
    const T sig = T(2.5) * g7 * alpha - T(17.5) * g9 * beta + T(157.5) * g11 * gam - T(0.5) * P.cb0 * g5;
    const T e7 = T(15) * g7, e9 = T(-105) * g9, e7b = T(10) * g7;
    const T n0 = -g5 * P.P1[0] + e7b * w0 + e9 * u0 + e7 * P.t3[0];
    const T n1 = -g5 * P.P1[1] + e7b * w1 + e9 * u1 + e7 * P.t3[1];
    const T n2 = -g5 * P.P1[2] + e7b * w2 + e9 * u2 + e7 * P.t3[2];
    const T Kxx = -g5 * P.p2xx + e7 * Txx, Kxy = -g5 * P.p2xy + e7 * Txy, Kxz = -g5 * P.p2xz + e7 * Txz,
            Kyy = -g5 * P.p2yy + e7 * Tyy, Kyz = -g5 * P.p2yz + e7 * Tyz, Kzz = -g5 * P.p2zz + e7 * Tzz;
    q[0] = sig * x0 * x0 + n0 * x0 + Kxx;
    q[1] = T(2) * sig * x0 * x1 + n0 * x1 + n1 * x0 + T(2) * Kxy;
    q[2] = T(2) * sig * x0 * x2 + n0 * x2 + n2 * x0 + T(2) * Kxz;
    q[3] = sig * x1 * x1 + n1 * x1 + Kyy;
    q[4] = T(2) * sig * x1 * x2 + n1 * x2 + n2 * x1 + T(2) * Kyz;
    q[5] = sig * x2 * x2 + n2 * x2 + Kzz;
    const T QP2 = Qxx * P.p2xx + Qyy * P.p2yy + Qzz * P.p2zz + T(2) * (Qxy * P.p2xy + Qxz * P.p2xz + Qyz * P.p2yz);
    const T QT = Qxx * Txx + Qyy * Tyy + Qzz * Tzz + T(2) * (Qxy * Txy + Qxz * Txz + Qyz * Tyz);
    const T P1v = P.P1[0] * v0 + P.P1[1] * v1 + P.P1[2] * v2;
    const T vw = v0 * w0 + v1 * w1 + v2 * w2;
    const T t3v = P.t3[0] * v0 + P.t3[1] * v1 + P.t3[2] * v2;
    const T uv = u0 * v0 + u1 * v1 + u2 * v2;
    const T S = P.cb0 * a + alpha * b + beta * cc + gam * d + T(5) * g7 * (P1v + QP2) - T(70) * g9 * vw +
                e9 * (t3v + QT) + T(945) * g11 * uv;
    const T W0 = Qxx * p3[0] + Qyy * p3[3] + Qzz * p3[5] + T(2) * (Qxy * p3[1] + Qxz * p3[2] + Qyz * p3[4]);
    const T W1 = Qxx * p3[1] + Qyy * p3[6] + Qzz * p3[8] + T(2) * (Qxy * p3[3] + Qxz * p3[4] + Qyz * p3[7]);
    const T W2 = Qxx * p3[2] + Qyy * p3[7] + Qzz * p3[9] + T(2) * (Qxy * p3[4] + Qxz * p3[5] + Qyz * p3[8]);
    const T P2v0 = P.p2xx * v0 + P.p2xy * v1 + P.p2xz * v2, P2v1 = P.p2xy * v0 + P.p2yy * v1 + P.p2yz * v2,
            P2v2 = P.p2xz * v0 + P.p2yz * v1 + P.p2zz * v2;
    const T Tv0 = Txx * v0 + Txy * v1 + Txz * v2, Tv1 = Txy * v0 + Tyy * v1 + Tyz * v2,
            Tv2 = Txz * v0 + Tyz * v1 + Tzz * v2;
    const T Qn0 = Qxx * n0 + Qxy * n1 + Qxz * n2, Qn1 = Qxy * n0 + Qyy * n1 + Qyz * n2,
            Qn2 = Qxz * n0 + Qyz * n1 + Qzz * n2;
    const T c3 = T(3) * cc, s2 = T(2) * sig, f10 = T(10) * g7, f210 = T(-210) * g9;
    gx[0] = x0 * S + a * P.P1[0] + b * (T(2) * w0 + T(3) * P.t3[0]) + c3 * u0 + s2 * v0 + Qn0 + f10 * P2v0 +
            f210 * Tv0 + e7 * W0;
    gx[1] = x1 * S + a * P.P1[1] + b * (T(2) * w1 + T(3) * P.t3[1]) + c3 * u1 + s2 * v1 + Qn1 + f10 * P2v1 +
            f210 * Tv1 + e7 * W1;
    gx[2] = x2 * S + a * P.P1[2] + b * (T(2) * w2 + T(3) * P.t3[2]) + c3 * u2 + s2 * v2 + Qn2 + f10 * P2v2 +
            f210 * Tv2 + e7 * W2;
}

template <bool MIXED>
__global__ void __launch_bounds__(kBW * 32) k_bwd_far(BCtx c) {
    using T = typename std::conditional<MIXED, float, double>::type;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = gw; s < c.nsinks; s += nw) {
        const int A = c.sinks[s];
        const int nf = c.far_n[s];
        const FarCbar<T> P(c.cbar + (int64_t)s * 20);
        float4 ah = make_float4(0.f, 0.f, 0.f, 0.f), al = ah;
        double cA[3] = {0.0, 0.0, 0.0};
        if (MIXED) {
            ah = c.nfar[4 * (int64_t)A];
            al = c.nfar[4 * (int64_t)A + 1];
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) cA[k] = c.ncom[3 * (int64_t)A + k];
        }
        T RA[3] = {T(0), T(0), T(0)};
        for (int k = lane; k < nf; k += 32) {
            const int B = c.far_list[(int64_t)s * c.cap_far + k];
            T x0, x1, x2, M, Q[6];
            if (MIXED) {
                const float4 r0 = c.nfar[4 * (int64_t)B], r1 = c.nfar[4 * (int64_t)B + 1],
                             r2 = c.nfar[4 * (int64_t)B + 2], r3 = c.nfar[4 * (int64_t)B + 3];
                x0 = (ah.x - r0.x) + (al.x - r1.x);
                x1 = (ah.y - r0.y) + (al.y - r1.y);
                x2 = (ah.z - r0.z) + (al.z - r1.z);
                M = r0.w;
                Q[0] = r1.w;
                Q[1] = r2.x;
                Q[2] = r2.y;
                Q[3] = r2.z;
                Q[4] = r2.w;
                Q[5] = r3.x;
            } else {
                x0 = cA[0] - c.ncom[3 * (int64_t)B];
                x1 = cA[1] - c.ncom[3 * (int64_t)B + 1];
                x2 = cA[2] - c.ncom[3 * (int64_t)B + 2];
                M = c.nmass[B];
#pragma unroll
                for (int qq = 0; qq < 6; ++qq) Q[qq] = c.nQ[6 * (int64_t)B + qq];
            }
            T mu, qa[6], gx[3];
            far_adjoint<T>(P, x0, x1, x2, M, Q[0], Q[1], Q[2], Q[3], Q[4], Q[5], mu, qa, gx);
            RA[0] += gx[0];
            RA[1] += gx[1];
            RA[2] += gx[2];
            double *aB = c.adj + 10 * (int64_t)B;
            atomicAdd(aB, (double)mu);
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) atomicAdd(aB + 1 + k2, -(double)gx[k2]);
#pragma unroll
            for (int qq = 0; qq < 6; ++qq) atomicAdd(aB + 4 + qq, (double)qa[qq]);
        }
        double R[3] = {RA[0], RA[1], RA[2]};
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) R[k2] += __shfl_xor_sync(0xffffffffu, R[k2], o);
        if (lane < 3) atomicAdd(&c.adj[10 * (int64_t)A + 1 + lane], lane == 0 ? R[0] : (lane == 1 ? R[1] : R[2]));
    }
}

// Mixed form of the far interactions with the node adjoints merged per CTA before they reach
// global memory: a CTA takes kFGroup consecutive sinks (siblings and cousins in tree order, whose
// far lists share most nodes), adds each pair's ten node adjoints into a shared-memory hash table
// keyed by node (float32; at most one term per sink and node), then flushes every entry once with
// FP64 atomic adds.  A node that finds no slot within kFProbe probes goes straight to global
// memory.
constexpr int kFWarps = 8;
constexpr int kFGroup = 16;
constexpr int kFHash = 2048;
constexpr int kFProbe = 32;

struct FarHash {
    int32_t key[kFHash];
    float val[10][kFHash];
    static constexpr size_t bytes = (size_t)kFHash * (sizeof(int32_t) + 10 * sizeof(float));
};

__device__ inline int far_hash_slot(FarHash &hs, int B) {
    unsigned h = ((unsigned)B * 2654435761u) >> 21;  // 11 bits: kFHash = 2048
    volatile int32_t *key = hs.key;
    for (int probe = 0; probe < kFProbe; ++probe) {
        const int k = key[h];
        if (k == B) return (int)h;
        if (k == -1) {
            const int old = atomicCAS(&hs.key[h], -1, B);
            if (old == -1 || old == B) return (int)h;
        }
        h = (h + 1) & (kFHash - 1);
    }
    return -1;
}

__global__ void __launch_bounds__(kFWarps * 32) k_bwd_far_mixed(BCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FarHash &hs = *reinterpret_cast<FarHash *>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kFHash; i += blockDim.x) {
        hs.key[i] = -1;
#pragma unroll
        for (int q = 0; q < 10; ++q) hs.val[q][i] = 0.f;
    }
    __syncthreads();
    for (int g0 = blockIdx.x * kFGroup; g0 < c.nsinks; g0 += gridDim.x * kFGroup) {
        const int g1 = min(g0 + kFGroup, c.nsinks);
        for (int s = g0 + w; s < g1; s += kFWarps) {
            const int A = c.sinks[s];
            const int nf = c.far_n[s];
            const FarCbar<float> P(c.cbar32 + (int64_t)s * 20);
            const float4 ah = c.nfar[4 * (int64_t)A], al = c.nfar[4 * (int64_t)A + 1];
            float RA[3] = {0.f, 0.f, 0.f};
            for (int k = lane; k < nf; k += 32) {
                const int B = c.far_list[(int64_t)s * c.cap_far + k];
                const float4 r0 = c.nfar[4 * (int64_t)B], r1 = c.nfar[4 * (int64_t)B + 1],
                             r2 = c.nfar[4 * (int64_t)B + 2], r3 = c.nfar[4 * (int64_t)B + 3];
                const float x0 = (ah.x - r0.x) + (al.x - r1.x), x1 = (ah.y - r0.y) + (al.y - r1.y),
                            x2 = (ah.z - r0.z) + (al.z - r1.z);
                float mu, qa[6], gx[3];
                far_adjoint<float>(P, x0, x1, x2, r0.w, r1.w, r2.x, r2.y, r2.z, r2.w, r3.x, mu, qa, gx);
                RA[0] += gx[0];
                RA[1] += gx[1];
                RA[2] += gx[2];
                const float vals[10] = {mu, -gx[0], -gx[1], -gx[2], qa[0], qa[1], qa[2], qa[3], qa[4], qa[5]};
                const int slot = far_hash_slot(hs, B);
                if (slot >= 0) {
#pragma unroll
                    for (int q = 0; q < 10; ++q) atomicAdd(&hs.val[q][slot], vals[q]);
                } else {
                    double *aB = c.adj + 10 * (int64_t)B;
#pragma unroll
                    for (int q = 0; q < 10; ++q) atomicAdd(aB + q, (double)vals[q]);
                }
            }
            double R[3] = {RA[0], RA[1], RA[2]};
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
                for (int k2 = 0; k2 < 3; ++k2) R[k2] += __shfl_xor_sync(0xffffffffu, R[k2], o);
            if (lane < 3) atomicAdd(&c.adj[10 * (int64_t)A + 1 + lane], lane == 0 ? R[0] : (lane == 1 ? R[1] : R[2]));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kFHash; i += blockDim.x) {
            const int B = hs.key[i];
            if (B >= 0) {
                double *aB = c.adj + 10 * (int64_t)B;
#pragma unroll
                for (int q = 0; q < 10; ++q) {
                    atomicAdd(aB + q, (double)hs.val[q][i]);
                    hs.val[q][i] = 0.f;
                }
                hs.key[i] = -1;
            }
        }
        __syncthreads();
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

// ------------------------------------------------------------------------------ near (mixed)
// The pair gradient of pair_grad in float32.  q = 2 r / (h_a + h_b) < 2 is tested as
// r < h_a + h_b, so the reciprocal 2 / (h_a + h_b) (fast division) is taken only for softened
// pairs; 3 / q = 3/2 (h_a + h_b) / r; 1 / r by rsqrtf.
__device__ inline void pair_grad32(float dx, float dy, float dz, float hsum, float mb, float vx, float vy, float vz,
                                   float w, float &gx, float &gy, float &gz, float &gm) {
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
    const float r = r2 * rinv;
    const float rinv2 = rinv * rinv;
    float sr = rinv * rinv2;
    float dsr = -3.f * sr * rinv2;
    float p = -rinv;
    if (r < hsum) {
        const float hinv = __fdividef(2.0f, hsum);
        const float q = r * hinv;
        const float h2 = hinv * hinv, h3 = h2 * hinv, h5 = h3 * h2;
        const float q2 = q * q;
        if (q < 1.f) {
            sr = h3 * (4.0f / 3.0f + q2 * (-1.2f + 0.5f * q));
            dsr = h5 * (-2.4f + 1.5f * q);
            p = hinv * (q2 * (2.0f / 3.0f + q2 * (-0.3f + 0.1f * q)) - 1.4f);
        } else {
            const float r3 = sr;
            sr = h3 * (8.0f / 3.0f + q * (-3.f + q * (1.2f - q * (1.0f / 6.0f)))) - (1.0f / 15.0f) * r3;
            dsr = h5 * (-1.5f * hsum * rinv + 2.4f - 0.5f * q) + 0.2f * r3 * rinv2;
            p = hinv * (q2 * (4.0f / 3.0f + q * (-1.f + q * (0.3f - q * (1.0f / 30.0f)))) - 1.6f) +
                (1.0f / 15.0f) * rinv;
        }
    }
    const float rv = dx * vx + dy * vy + dz * vz;
    const float k1 = mb * sr, k2 = mb * dsr * rv, k3 = w * mb * sr;
    gx = k3 * dx - (k1 * vx + k2 * dx);
    gy = k3 * dy - (k1 * vy + k2 * dy);
    gz = k3 * dz - (k1 * vz + k2 * dz);
    gm = w * p - sr * rv;
}

constexpr int kMTile = 384;   // staged particles per warp (mixed)
constexpr int kMGroup = 8;    // own particles per pass (mixed)
constexpr int kMSuper = 3;    // groups of own particles sharing one staged tile

// Per-warp staging.  SIDE 0 (sources b): a = (x, y, z, m_b), hb = h_b.  SIDE 1 (sink particles a):
// a = (x, y, z, h_a), v = (dL/da_a, dL/dPhi_a).  Positions relative to the own cell's centre of mass.
struct BNearSmem {
    float4 a[kMTile];
    float4 v[kMTile];
    float hb[kMTile];
    int32_t id[kMTile];
    float2 gacc[kMSuper][32];  // the groups' compensated lane totals while another group runs
    static constexpr size_t bytes =
        (size_t)kMTile * (2 * sizeof(float4) + sizeof(float) + sizeof(int32_t)) + kMSuper * 32 * sizeof(float2);
};

// Stage slots [t0, t0 + kMTile) of the concatenated cells; one lane per slot.
template <int SIDE, typename CellAt>
__device__ int stage_cells_mixed(const BCtx &c, int ncells, CellAt cell_at, int64_t t0, float2 cO[3],
                                 BNearSmem &sm) {
    const int lane = threadIdx.x & 31;
    int64_t pos = 0;
    int staged = 0;
    for (int k0 = 0; k0 < ncells; k0 += 32) {
        const int k = k0 + lane;
        int f = 0, n = 0;
        float ox = 0.f, oy = 0.f, oz = 0.f;
        if (k < ncells) {
            const int B = cell_at(k);
            f = c.nfirst[B];
            n = c.ncount[B];
            const float2 b0 = c.ncomdf[3 * (int64_t)B], b1 = c.ncomdf[3 * (int64_t)B + 1],
                         b2 = c.ncomdf[3 * (int64_t)B + 2];
            ox = (b0.x - cO[0].x) + (b0.y - cO[0].y);
            oy = (b1.x - cO[1].x) + (b1.y - cO[1].y);
            oz = (b2.x - cO[2].x) + (b2.y - cO[2].y);
        }
        const int excl = warp_excl_scan(n);
        const int total = __shfl_sync(0xffffffffu, excl + n, 31);
        const int64_t lo = pos > t0 ? pos : t0;
        const int64_t hi = pos + total < t0 + kMTile ? pos + total : t0 + kMTile;
        for (int64_t r0 = lo; r0 < hi; r0 += 32) {
            const int j = warp_run_of(excl, n, (int)(r0 - pos));
            const int jf = __shfl_sync(0xffffffffu, f, j & 31), je = __shfl_sync(0xffffffffu, excl, j & 31);
            const float bx = __shfl_sync(0xffffffffu, ox, j & 31), by = __shfl_sync(0xffffffffu, oy, j & 31),
                        bz = __shfl_sync(0xffffffffu, oz, j & 31);
            const int64_t q = r0 + lane;
            if (q < hi) {
                const int b = jf + (int)(q - pos) - je;
                const int slot = (int)(q - t0);
                const float4 pb = c.p32[b];
                if (SIDE == 0) {
                    sm.a[slot] = make_float4(pb.x + bx, pb.y + by, pb.z + bz, pb.w);
                    sm.hb[slot] = c.h32[b];
                } else {
                    sm.a[slot] = make_float4(pb.x + bx, pb.y + by, pb.z + bz, c.h32[b]);
                    sm.v[slot] = c.gv32[b];
                }
                sm.id[slot] = b;
            }
        }
        if (hi > lo) staged = (int)(hi - t0);
        pos += total;
        if (pos >= t0 + kMTile) break;
    }
    __syncwarp();
    return staged;
}

// SIDE 0: sink side, a in the sink, b over the near cells: gxs[a] += g.
// SIDE 1: source side, b in a leaf, a over the sink particles listing it: gxs[b] -= g, gms[b] += gm.
// Up to kMSuper groups of own particles share each staged tile (the tile loop runs outside the
// group loop).  Per tile and group the float32 sums are reduce-scattered across lanes with
// compensation and folded into the group's (sum, error) pair per lane, which waits in shared
// memory while another group runs.
template <int SIDE>
__global__ void __launch_bounds__(kBW * 32, 3) k_bwd_near_mixed(BCtx c) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    BNearSmem &sm = *reinterpret_cast<BNearSmem *>(smem_raw + (size_t)w * BNearSmem::bytes);
    constexpr int NQ = SIDE == 0 ? 3 : 4;
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
        float2 cO[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) cO[d] = c.ncomdf[3 * (int64_t)own + d];
        int64_t S = 0;
        for (int k = lane; k < ncells; k += 32) S += c.ncount[cell_at(k)];
        for (int o = 16; o >= 1; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
        const int f = c.nfirst[own], n = c.ncount[own];
        for (int P0 = 0; P0 < n; P0 += kMSuper * kMGroup) {
            const int ng = min(kMSuper, (n - P0 + kMGroup - 1) / kMGroup);
            for (int gi = 0; gi < ng; ++gi) sm.gacc[gi][lane] = make_float2(0.f, 0.f);
            for (int64_t t0 = 0; t0 < S; t0 += kMTile) {
                const int ns = stage_cells_mixed<SIDE>(c, ncells, cell_at, t0, cO, sm);
                for (int gi = 0; gi < ng; ++gi) {
                    const int p0 = P0 + gi * kMGroup;
                    const int np = min(kMGroup, n - p0);
                    float ox[kMGroup], oy[kMGroup], oz[kMGroup], oh[kMGroup], om[kMGroup], ovx[kMGroup], ovy[kMGroup],
                        ovz[kMGroup], ow[kMGroup];
                    int oid[kMGroup];
#pragma unroll
                    for (int i = 0; i < kMGroup; ++i) {
                        const int p = f + p0 + min(i, np - 1);
                        const float4 pp = c.p32[p];
                        ox[i] = pp.x;
                        oy[i] = pp.y;
                        oz[i] = pp.z;
                        om[i] = pp.w;
                        oh[i] = c.h32[p];
                        if (SIDE == 0) {
                            const float4 gv = c.gv32[p];
                            ovx[i] = gv.x;
                            ovy[i] = gv.y;
                            ovz[i] = gv.z;
                            ow[i] = gv.w;
                        }
                        oid[i] = i < np ? p : -1;
                    }
                    float acc[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) acc[i] = 0.f;
                    for (int j = lane; j < ns; j += 32) {
                        const float4 ja = sm.a[j];
                        const int jid = sm.id[j];
                        if (SIDE == 0) {
                            const float jh = sm.hb[j];
#pragma unroll
                            for (int i = 0; i < kMGroup; ++i) {
                                if (i > 0 && i >= np) break;  // padding of a short group (warp-uniform)
                                float gx, gy, gz, gmv;
                                pair_grad32(ox[i] - ja.x, oy[i] - ja.y, oz[i] - ja.z, oh[i] + jh, ja.w, ovx[i], ovy[i],
                                            ovz[i], ow[i], gx, gy, gz, gmv);
                                if (jid != oid[i]) {
                                    acc[NQ * i] += gx;
                                    acc[NQ * i + 1] += gy;
                                    acc[NQ * i + 2] += gz;
                                }
                            }
                        } else {
                            const float4 jv = sm.v[j];
#pragma unroll
                            for (int i = 0; i < kMGroup; ++i) {
                                if (i > 0 && i >= np) break;  // padding of a short group (warp-uniform)
                                float gx, gy, gz, gmv;
                                pair_grad32(ja.x - ox[i], ja.y - oy[i], ja.z - oz[i], ja.w + oh[i], om[i], jv.x, jv.y, jv.z,
                                            jv.w, gx, gy, gz, gmv);
                                if (jid != oid[i]) {
                                    acc[NQ * i] -= gx;
                                    acc[NQ * i + 1] -= gy;
                                    acc[NQ * i + 2] -= gz;
                                    acc[NQ * i + 3] += gmv;
                                }
                            }
                        }
                    }
                    // lane l ends with quantity l (of NQ * kMGroup <= 32) of this tile, then folds it in
                    float E[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) E[i] = 0.f;
                    reduce_scatter_df<32>(acc, E);
                    float2 st = sm.gacc[gi][lane];
                    float t, e;
                    two_sum(st.x, acc[0], t, e);
                    st.x = t;
                    st.y = __fadd_rn(__fadd_rn(st.y, E[0]), e);
                    sm.gacc[gi][lane] = st;
                }
                __syncwarp();
            }
            for (int gi = 0; gi < ng; ++gi) {
                const int p0 = P0 + gi * kMGroup;
                const int np = min(kMGroup, n - p0);
                const float2 st = sm.gacc[gi][lane];
                const double tot = (double)st.x + (double)st.y;
                if (lane < NQ * np) {
                    const int i = lane / NQ, qq = lane - NQ * i;
                    const int p = f + p0 + i;
                    if (qq < 3)
                        c.gxs[3 * (int64_t)p + qq] += tot;
                    else
                        c.gms[p] += tot;
                }
            }
            __syncwarp();
        }
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

// Sort each transposed row, for a fixed order: a warp takes 32 rows and sorts them in registers,
// four at a time on groups of 8 lanes (longer rows over the whole warp; beyond 128 entries in
// place), with the sorting networks of the neighbour rows.
__global__ void __launch_bounds__(256, 4) k_tnear_sort(const int32_t *off, int64_t nleaves, int32_t *rows) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < nleaves; base += nw * 32) {
        int64_t a = 0;
        int n = -1;
        if (base + lane < nleaves) {
            a = off[base + lane];
            n = (int)(off[base + lane + 1] - a);
        }
        const int cnt = (int)(nleaves - base < 32 ? nleaves - base : 32);
        rows_sort_store(rows, a, n, a, INT32_MAX, rows, cnt);
    }
}

// Node adjoints to particles.  Node n's adjoints (M, COM, Q) reach a particle b below it as
//   dL/dm_b += phi_n(x_b),  dL/dx_b += m_b grad phi_n(x_b),
//   phi_n(x) = Mbar + COMbar.d / M + Qbar:(3 d d - d^2 I),  d = x - COM_n
// (M = sum m_b, COM = sum m_b x_b / M, Q = sum m_b (3 d d - d^2 I), Eq. 1; Q has no derivative
// through the COM because sum m_b d_b = 0).  phi_n is a quadratic polynomial, so the sum over a
// particle's ancestors is one quadratic Phi per node, built top-down a level at a time:
// Phi_n = phi_n + Phi_parent re-centred on COM_n.  adj[10 n] is overwritten with Phi_n as
// (c0, c1[3], C2 slots xx, xy, xz, yy, yz, zz) with Phi(x) = c0 + c1.d + d.C2 d.
__global__ void k_bwd_phi_level(BCtx c, int level) {
    const int64_t n0 = (int64_t)1 << level, n1 = n0 << 1;
    for (int64_t n = n0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < n1; n += (int64_t)gridDim.x * blockDim.x) {
        double *a = c.adj + 10 * n;
        if (c.ncount[n] == 0) {
#pragma unroll
            for (int q = 0; q < 10; ++q) a[q] = 0.0;
            continue;
        }
        const double M = c.nmass[n];
        const double tr = a[4] + a[7] + a[9];
        double P[10] = {a[0],          a[1] / M,      a[2] / M,      a[3] / M,      3.0 * a[4] - tr,
                        1.5 * a[5],    1.5 * a[6],    3.0 * a[7] - tr, 1.5 * a[8],  3.0 * a[9] - tr};
        if (level > 0) {
            const int64_t p = n >> 1;
            const double *q = c.adj + 10 * p;
            const double e[3] = {c.ncom[3 * n] - c.ncom[3 * p], c.ncom[3 * n + 1] - c.ncom[3 * p + 1],
                                 c.ncom[3 * n + 2] - c.ncom[3 * p + 2]};
            const double Ce[3] = {q[4] * e[0] + q[5] * e[1] + q[6] * e[2], q[5] * e[0] + q[7] * e[1] + q[8] * e[2],
                                  q[6] * e[0] + q[8] * e[1] + q[9] * e[2]};
            P[0] += q[0] + q[1] * e[0] + q[2] * e[1] + q[3] * e[2] + (Ce[0] * e[0] + Ce[1] * e[1] + Ce[2] * e[2]);
            P[1] += q[1] + 2.0 * Ce[0];
            P[2] += q[2] + 2.0 * Ce[1];
            P[3] += q[3] + 2.0 * Ce[2];
#pragma unroll
            for (int k = 4; k < 10; ++k) P[k] += q[k];
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) a[q] = P[q];
    }
}

// Evaluate the sink's Phi at every particle, add the particle's own terms and scatter to
// original order.
__global__ void k_bwd_particles(BCtx c) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.N; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = c.pleaf[p];
        const double *q = c.adj + 10 * n;
        const double d[3] = {c.px[p] - c.ncom[3 * n], c.py[p] - c.ncom[3 * n + 1], c.pz[p] - c.ncom[3 * n + 2]};
        const double Cd[3] = {q[4] * d[0] + q[5] * d[1] + q[6] * d[2], q[5] * d[0] + q[7] * d[1] + q[8] * d[2],
                              q[6] * d[0] + q[8] * d[1] + q[9] * d[2]};
        const double mb = c.pm[p];
        const double gm = c.gms[p] + (q[0] + q[1] * d[0] + q[2] * d[1] + q[3] * d[2] +
                                      (Cd[0] * d[0] + Cd[1] * d[1] + Cd[2] * d[2]));
        const int64_t o = c.pidx[p];
        c.gx[3 * o] = c.gxs[3 * p] + mb * (q[1] + 2.0 * Cd[0]);
        c.gx[3 * o + 1] = c.gxs[3 * p + 1] + mb * (q[2] + 2.0 * Cd[1]);
        c.gx[3 * o + 2] = c.gxs[3 * p + 2] + mb * (q[3] + 2.0 * Cd[2]);
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

int far_coefficients(rcb_tree *t);  // gravity.cu

int gravity_backward(rcb_tree *t, const double *gacc, const double *gpot, double *gx, double *gm) {
    cudaStream_t st = t->stream;
    const int64_t N = t->N, nn = t->nn, nl = t->nleaves;
    if (t->nsinks == 0) return RCB_OK;
    // scratch, through the tree's allocator: kept across builds and grown when a build needs more
    // (the transposed near list's entries are known only after its count, below)
    const size_t adj_bytes = (size_t)nn * 10 * sizeof(double) + (size_t)N * 8 * sizeof(double) +
                             (size_t)t->nsinks * 20 * sizeof(double) + (size_t)N * sizeof(float4) +
                             (size_t)t->nsinks * 20 * sizeof(float);
    auto grow = [&](void **q, int64_t &cap, int64_t need, size_t elem) {
        if (*q && cap >= need) return true;
        dev_free(t, *q);
        *q = dev_alloc(t, (size_t)std::max<int64_t>(need, 1) * elem);
        cap = *q ? need : 0;
        return *q != nullptr;
    };
    if (!t->bwd_valid) {
        if (!grow((void **)&t->tnear_off, t->cap_bwd_off, nl + 1, sizeof(int32_t)) ||
            !grow((void **)&t->tfar_off, t->cap_bwd_cur, nl + 1, sizeof(int32_t)) ||
            !grow((void **)&t->tfar_sink, t->cap_bwd_N, N, sizeof(int32_t)) ||
            !grow((void **)&t->adj, t->cap_bwd_adj, (int64_t)adj_bytes, 1))
            return RCB_ERR_ALLOC;
    }
    double *adj = t->adj;
    double *gxs = adj + nn * 10;
    double *gms = gxs + 3 * N;
    double *gA = gms + N;
    double *gP = gA + 3 * N;
    double *cbar = gP + N;
    float4 *gv32 = reinterpret_cast<float4 *>(cbar + (size_t)t->nsinks * 20);
    float *cbar32 = reinterpret_cast<float *>(gv32 + N);
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
    c.nfar = t->nfar;
    c.ncomdf = t->ncomdf;
    c.p32 = t->p32;
    c.h32 = t->h32;
    c.pidx = t->pidx;
    c.coef = t->coef;
    c.cbar = cbar;
    c.cbar32 = cbar32;
    c.gv32 = t->params.precision == RCB_MIXED ? gv32 : nullptr;
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
        // the number of entries, through the mapped status words (no pageable copy)
        rc = copy_words(t->h_status_dev + ST_NWORDS + 4, t->tnear_off + nl, 1, st);
        if (rc) return rc;
        RCB_CUDA_TRY(cudaStreamSynchronize(st));
        const int64_t total = t->h_status[ST_NWORDS + 4];
        if (!grow((void **)&t->tnear_sink, t->cap_bwd_sink, total, sizeof(int32_t))) return RCB_ERR_ALLOC;
        c.tnear_sink = t->tnear_sink;
        RCB_CUDA_TRY(cudaMemcpyAsync(cnt, t->tnear_off, nl * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        k_tnear_fill<<<gridw, kBW * 32, 0, st>>>(c, cnt, t->tnear_sink); note_launch();
        k_tnear_sort<<<(int)std::max<int64_t>(1, std::min<int64_t>((nl + 255) / 256, (int64_t)nsm * 16)), 256, 0, st>>>(
            t->tnear_off, nl, t->tnear_sink); note_launch();
        k_bwd_pleaf<<<gridw, kBW * 32, 0, st>>>(c); note_launch();
        RCB_CUDA_TRY(cudaGetLastError());
        t->bwd_valid = 1;
    }
    int rc = far_coefficients(t);
    if (rc) return rc;
    RCB_CUDA_TRY(cudaMemsetAsync(adj, 0, (size_t)nn * 10 * sizeof(double), st));
    k_bwd_gather<<<gridp, 256, 0, st>>>(c); note_launch();
    if (t->params.precision == RCB_MIXED) {
        k_bwd_taylor_mixed<<<gridw, kBW * 32, 0, st>>>(c, t->coef32); note_launch();
    } else {
        k_bwd_taylor<<<gridw, kBW * 32, 0, st>>>(c); note_launch();
    }
    const int gridl = (int)std::max<int64_t>(1, std::min<int64_t>((nl + kBW - 1) / kBW, (int64_t)nsm * 16));
    if (t->params.precision == RCB_MIXED) {
        RCB_CUDA_TRY(cudaFuncSetAttribute(k_bwd_far_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FarHash::bytes));
        const int gridf = std::max(1, std::min((t->nsinks + kFGroup - 1) / kFGroup, nsm * 2));
        k_bwd_far_mixed<<<gridf, kFWarps * 32, FarHash::bytes, st>>>(c); note_launch();
        const size_t smem = kBW * BNearSmem::bytes;
        RCB_CUDA_TRY(cudaFuncSetAttribute(k_bwd_near_mixed<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RCB_CUDA_TRY(cudaFuncSetAttribute(k_bwd_near_mixed<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_bwd_near_mixed<0><<<gridw, kBW * 32, smem, st>>>(c); note_launch();
        k_bwd_near_mixed<1><<<gridl, kBW * 32, smem, st>>>(c); note_launch();
    } else {
        k_bwd_far<false><<<gridw, kBW * 32, 0, st>>>(c); note_launch();
        const size_t smem = kBW * kBSmemPerWarp;
        RCB_CUDA_TRY(cudaFuncSetAttribute(k_bwd_near<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RCB_CUDA_TRY(cudaFuncSetAttribute(k_bwd_near<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_bwd_near<0><<<gridw, kBW * 32, smem, st>>>(c); note_launch();
        k_bwd_near<1><<<gridl, kBW * 32, smem, st>>>(c); note_launch();
    }
    for (int l = 0; l <= t->L; ++l) {
        const int64_t cnt = (int64_t)1 << l;
        k_bwd_phi_level<<<(int)std::min<int64_t>((cnt + 255) / 256, (int64_t)nsm * 8), 256, 0, st>>>(c, l); note_launch();
    }
    k_bwd_particles<<<gridp, 256, 0, st>>>(c); note_launch();
    stage_end(t, SG_BWD);
    RCB_CUDA_TRY(cudaGetLastError());
    return RCB_OK;
}

}  // namespace rcb
