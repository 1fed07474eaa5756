// Far- and near-field arithmetic shared by the gravity kernels and their backward pass:
// symmetric-tensor slots, the monopole + quadrupole Taylor coefficients of one far source
// (Eq. 5 expanded to third order), the sink's Taylor polynomial (Eq. 6), warp reduce-scatters,
// and the kernel-softened pair force (Eqs. 9-10) with its gradient.
#pragma once

#include <cuda_runtime.h>

#include "rcb_internal.cuh"

namespace rcb {

// Coefficients of one far source, accumulated into C.  x = r_A - r_B, g = 1/|x|, v = Q x,
// s = x.v, and
//   C0     = -M g - s g^5 / 2
//   C1_i   = a x_i - g^5 v_i                                       a = M g^3 + 5/2 s g^7
//   C2_ij  = b x_i x_j + a d_ij - g^5 Q_ij + 5 g^7 (v_i x_j + v_j x_i)
//                                                                  b = -3 M g^5 - 35/2 s g^9
//   C3_ijk = c x_i x_j x_k + b (d_ij x_k + d_ik x_j + d_jk x_i)
//            + 5 g^7 (Q_ij x_k + Q_ik x_j + Q_jk x_i + v_i d_jk + v_j d_ik + v_k d_ij)
//            - 35 g^9 (v_i x_j x_k + v_j x_i x_k + v_k x_i x_j)      c = 15 M g^7 + 315/2 s g^11
// Slots: C[0]; C[1..3] = x, y, z; C[4..9] = xx, xy, xz, yy, yz, zz; C[10..19] = xxx, xxy, xxz,
// xyy, xyz, xzz, yyy, yyz, yzz, zzz.  Every slot is written out so that all indices are
// compile-time constants.
template <typename T>
__device__ inline T c3_slot(T c, T b, T f7, T f9, T xi, T xj, T xk, T Qij, T Qik, T Qjk, T vi, T vj, T vk, T dsum,
                            T vsum) {
    return c * xi * xj * xk + f7 * (Qij * xk + Qik * xj + Qjk * xi) - f9 * (vi * xj * xk + vj * xi * xk + vk * xi * xj) +
           b * dsum + f7 * vsum;
}

template <typename T>
__device__ inline void far_source(const T x[3], T M, const T Q6[6], T C[20]) {
    const T x0 = x[0], x1 = x[1], x2 = x[2];
    const T r2 = x0 * x0 + x1 * x1 + x2 * x2;
    const T g = rsqrt(r2);
    const T g2 = g * g, g3 = g * g2, g5 = g3 * g2, g7 = g5 * g2, g9 = g7 * g2, g11 = g9 * g2;
    const T Qxx = Q6[0], Qxy = Q6[1], Qxz = Q6[2], Qyy = Q6[3], Qyz = Q6[4], Qzz = Q6[5];
    const T v0 = Qxx * x0 + Qxy * x1 + Qxz * x2;
    const T v1 = Qxy * x0 + Qyy * x1 + Qyz * x2;
    const T v2 = Qxz * x0 + Qyz * x1 + Qzz * x2;
    const T s = x0 * v0 + x1 * v1 + x2 * v2;
    const T a = M * g3 + T(2.5) * s * g7;
    const T b = T(-3) * M * g5 - T(17.5) * s * g9;
    const T c = T(15) * M * g7 + T(157.5) * s * g11;
    const T f7 = T(5) * g7, f9 = T(35) * g9;
    const T zero = T(0);
    C[0] += -M * g - T(0.5) * s * g5;
    C[1] += a * x0 - g5 * v0;
    C[2] += a * x1 - g5 * v1;
    C[3] += a * x2 - g5 * v2;
    C[4] += b * x0 * x0 - g5 * Qxx + f7 * (v0 * x0 + v0 * x0) + a;
    C[5] += b * x0 * x1 - g5 * Qxy + f7 * (v0 * x1 + v1 * x0);
    C[6] += b * x0 * x2 - g5 * Qxz + f7 * (v0 * x2 + v2 * x0);
    C[7] += b * x1 * x1 - g5 * Qyy + f7 * (v1 * x1 + v1 * x1) + a;
    C[8] += b * x1 * x2 - g5 * Qyz + f7 * (v1 * x2 + v2 * x1);
    C[9] += b * x2 * x2 - g5 * Qzz + f7 * (v2 * x2 + v2 * x2) + a;
    const T t3 = T(3);
    C[10] += c3_slot(c, b, f7, f9, x0, x0, x0, Qxx, Qxx, Qxx, v0, v0, v0, t3 * x0, t3 * v0);
    C[11] += c3_slot(c, b, f7, f9, x0, x0, x1, Qxx, Qxy, Qxy, v0, v0, v1, x1, v1);
    C[12] += c3_slot(c, b, f7, f9, x0, x0, x2, Qxx, Qxz, Qxz, v0, v0, v2, x2, v2);
    C[13] += c3_slot(c, b, f7, f9, x0, x1, x1, Qxy, Qxy, Qyy, v0, v1, v1, x0, v0);
    C[14] += c3_slot(c, b, f7, f9, x0, x1, x2, Qxy, Qxz, Qyz, v0, v1, v2, zero, zero);
    C[15] += c3_slot(c, b, f7, f9, x0, x2, x2, Qxz, Qxz, Qzz, v0, v2, v2, x0, v0);
    C[16] += c3_slot(c, b, f7, f9, x1, x1, x1, Qyy, Qyy, Qyy, v1, v1, v1, t3 * x1, t3 * v1);
    C[17] += c3_slot(c, b, f7, f9, x1, x1, x2, Qyy, Qyz, Qyz, v1, v1, v2, x2, v2);
    C[18] += c3_slot(c, b, f7, f9, x1, x2, x2, Qyz, Qyz, Qzz, v1, v2, v2, x1, v1);
    C[19] += c3_slot(c, b, f7, f9, x2, x2, x2, Qzz, Qzz, Qzz, v2, v2, v2, t3 * x2, t3 * v2);
}

// far_source for two far sources at once, (.x, .y) halves, with paired float32 instructions;
// the products are grouped as in far_source and every accumulation is a fused multiply-add
// into C.
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 c3_slot2(float2 C, float2 cx, float2 b, float2 f7, float2 nf9, float2 xi, float2 xj,
                                           float2 xk, float2 Qij, float2 Qik, float2 Qjk, float2 vi, float2 vj,
                                           float2 vk, float2 dsum, float2 vsum) {
    // c x_i x_j x_k + f7 (Q_ij x_k + Q_ik x_j + Q_jk x_i + vsum) - f9 (v_i x_j x_k + v_j x_i x_k + v_k x_i x_j)
    // + b dsum, with cx = c x_i
    const float2 xjk = __fmul2_rn(xj, xk);
    const float2 t = __ffma2_rn(Qjk, xi, __ffma2_rn(Qik, xj, __fmul2_rn(Qij, xk)));
    const float2 u = __ffma2_rn(vk, __fmul2_rn(xi, xj), __ffma2_rn(vj, __fmul2_rn(xi, xk), __fmul2_rn(vi, xjk)));
    return __ffma2_rn(cx, xjk, __ffma2_rn(f7, __fadd2_rn(t, vsum), __ffma2_rn(nf9, u, __ffma2_rn(b, dsum, C))));
}

__device__ inline void far_source2(float2 x0, float2 x1, float2 x2, float2 M, float2 Qxx, float2 Qxy, float2 Qxz,
                                   float2 Qyy, float2 Qyz, float2 Qzz, float2 C[20]) {
    const float2 r2 = __ffma2_rn(x2, x2, __ffma2_rn(x1, x1, __fmul2_rn(x0, x0)));
    const float2 g = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 g2 = __fmul2_rn(g, g), g3 = __fmul2_rn(g, g2), g5 = __fmul2_rn(g3, g2), g7 = __fmul2_rn(g5, g2);
    const float2 g9 = __fmul2_rn(g7, g2), g11 = __fmul2_rn(g9, g2);
    const float2 v0 = __ffma2_rn(Qxz, x2, __ffma2_rn(Qxy, x1, __fmul2_rn(Qxx, x0)));
    const float2 v1 = __ffma2_rn(Qyz, x2, __ffma2_rn(Qyy, x1, __fmul2_rn(Qxy, x0)));
    const float2 v2 = __ffma2_rn(Qzz, x2, __ffma2_rn(Qyz, x1, __fmul2_rn(Qxz, x0)));
    const float2 s = __ffma2_rn(x2, v2, __ffma2_rn(x1, v1, __fmul2_rn(x0, v0)));
    const float2 a = __ffma2_rn(M, g3, __fmul2_rn(f2s(2.5f), __fmul2_rn(s, g7)));
    const float2 b = __ffma2_rn(__fmul2_rn(f2s(-3.0f), M), g5, __fmul2_rn(f2s(-17.5f), __fmul2_rn(s, g9)));
    const float2 c = __ffma2_rn(__fmul2_rn(f2s(15.0f), M), g7, __fmul2_rn(f2s(157.5f), __fmul2_rn(s, g11)));
    const float2 f7 = __fmul2_rn(f2s(5.0f), g7), nf9 = __fmul2_rn(f2s(-35.0f), g9);
    const float2 ng5 = f2neg(g5), two = f2s(2.0f), three = f2s(3.0f), zero = f2s(0.0f);
    C[0] = __ffma2_rn(f2neg(M), g, __ffma2_rn(f2s(-0.5f), __fmul2_rn(s, g5), C[0]));
    C[1] = __ffma2_rn(a, x0, __ffma2_rn(ng5, v0, C[1]));
    C[2] = __ffma2_rn(a, x1, __ffma2_rn(ng5, v1, C[2]));
    C[3] = __ffma2_rn(a, x2, __ffma2_rn(ng5, v2, C[3]));
    const float2 bx0 = __fmul2_rn(b, x0), bx1 = __fmul2_rn(b, x1), bx2 = __fmul2_rn(b, x2);
    C[4] = __ffma2_rn(bx0, x0, __ffma2_rn(ng5, Qxx, __ffma2_rn(f7, __fmul2_rn(two, __fmul2_rn(v0, x0)), __fadd2_rn(a, C[4]))));
    C[5] = __ffma2_rn(bx0, x1, __ffma2_rn(ng5, Qxy, __ffma2_rn(f7, __ffma2_rn(v0, x1, __fmul2_rn(v1, x0)), C[5])));
    C[6] = __ffma2_rn(bx0, x2, __ffma2_rn(ng5, Qxz, __ffma2_rn(f7, __ffma2_rn(v0, x2, __fmul2_rn(v2, x0)), C[6])));
    C[7] = __ffma2_rn(bx1, x1, __ffma2_rn(ng5, Qyy, __ffma2_rn(f7, __fmul2_rn(two, __fmul2_rn(v1, x1)), __fadd2_rn(a, C[7]))));
    C[8] = __ffma2_rn(bx1, x2, __ffma2_rn(ng5, Qyz, __ffma2_rn(f7, __ffma2_rn(v1, x2, __fmul2_rn(v2, x1)), C[8])));
    C[9] = __ffma2_rn(bx2, x2, __ffma2_rn(ng5, Qzz, __ffma2_rn(f7, __fmul2_rn(two, __fmul2_rn(v2, x2)), __fadd2_rn(a, C[9]))));
    const float2 cx0 = __fmul2_rn(c, x0), cx1 = __fmul2_rn(c, x1), cx2 = __fmul2_rn(c, x2);
    C[10] = c3_slot2(C[10], cx0, b, f7, nf9, x0, x0, x0, Qxx, Qxx, Qxx, v0, v0, v0, __fmul2_rn(three, x0), __fmul2_rn(three, v0));
    C[11] = c3_slot2(C[11], cx0, b, f7, nf9, x0, x0, x1, Qxx, Qxy, Qxy, v0, v0, v1, x1, v1);
    C[12] = c3_slot2(C[12], cx0, b, f7, nf9, x0, x0, x2, Qxx, Qxz, Qxz, v0, v0, v2, x2, v2);
    C[13] = c3_slot2(C[13], cx0, b, f7, nf9, x0, x1, x1, Qxy, Qxy, Qyy, v0, v1, v1, x0, v0);
    C[14] = c3_slot2(C[14], cx0, b, f7, nf9, x0, x1, x2, Qxy, Qxz, Qyz, v0, v1, v2, zero, zero);
    C[15] = c3_slot2(C[15], cx0, b, f7, nf9, x0, x2, x2, Qxz, Qxz, Qzz, v0, v2, v2, x0, v0);
    C[16] = c3_slot2(C[16], cx1, b, f7, nf9, x1, x1, x1, Qyy, Qyy, Qyy, v1, v1, v1, __fmul2_rn(three, x1), __fmul2_rn(three, v1));
    C[17] = c3_slot2(C[17], cx1, b, f7, nf9, x1, x1, x2, Qyy, Qyz, Qyz, v1, v1, v2, x2, v2);
    C[18] = c3_slot2(C[18], cx1, b, f7, nf9, x1, x2, x2, Qyz, Qyz, Qzz, v1, v2, v2, x1, v1);
    C[19] = c3_slot2(C[19], cx2, b, f7, nf9, x2, x2, x2, Qzz, Qzz, Qzz, v2, v2, v2, __fmul2_rn(three, x2), __fmul2_rn(three, v2));
}

// Gradient and Hessian of the sink's third-order Taylor polynomial P at offset d (Eq. 6).
template <typename T>
__device__ inline void taylor_grad_hess(const T C[20], T d0, T d1, T d2, T g[3], T H[6]) {
    const T M00 = C[4], M01 = C[5], M02 = C[6], M11 = C[7], M12 = C[8], M22 = C[9];
    const T T000 = C[10], T001 = C[11], T002 = C[12], T011 = C[13], T012 = C[14], T022 = C[15], T111 = C[16],
            T112 = C[17], T122 = C[18], T222 = C[19];
    H[0] = M00 + T000 * d0 + T001 * d1 + T002 * d2;
    H[1] = M01 + T001 * d0 + T011 * d1 + T012 * d2;
    H[2] = M02 + T002 * d0 + T012 * d1 + T022 * d2;
    H[3] = M11 + T011 * d0 + T111 * d1 + T112 * d2;
    H[4] = M12 + T012 * d0 + T112 * d1 + T122 * d2;
    H[5] = M22 + T022 * d0 + T122 * d1 + T222 * d2;
    // grad_i = C1_i + M_ij d_j + 1/2 T_ijk d_j d_k = C1_i + 1/2 (M_ij + H_ij) d_j
    const T h = T(0.5);
    g[0] = C[1] + h * ((M00 + H[0]) * d0 + (M01 + H[1]) * d1 + (M02 + H[2]) * d2);
    g[1] = C[2] + h * ((M01 + H[1]) * d0 + (M11 + H[3]) * d1 + (M12 + H[4]) * d2);
    g[2] = C[3] + h * ((M02 + H[2]) * d0 + (M12 + H[4]) * d1 + (M22 + H[5]) * d2);
}

// Third-order Taylor polynomial of the sink (Eq. 6): phi and a = -grad phi at offset d.
template <typename T>
__device__ inline void taylor_eval(const T C[20], const T d[3], T &phi, T acc[3]) {
    const T d0 = d[0], d1 = d[1], d2 = d[2];
    T g[3], H[6];
    taylor_grad_hess(C, d0, d1, d2, g, H);
    // Phi = C0 + d.(C1 + 1/2 M d + 1/6 T d d) = C0 + d.(C1 + (g - C1) / ... ) written out:
    const T q2 = T(0.5) * (C[4] * d0 * d0 + C[7] * d1 * d1 + C[9] * d2 * d2) + C[5] * d0 * d1 + C[6] * d0 * d2 +
                 C[8] * d1 * d2;
    const T q3 = (C[10] * d0 * d0 * d0 + C[16] * d1 * d1 * d1 + C[19] * d2 * d2 * d2) * T(1.0 / 6.0) +
                 T(0.5) * (C[11] * d0 * d0 * d1 + C[12] * d0 * d0 * d2 + C[13] * d0 * d1 * d1 + C[15] * d0 * d2 * d2 +
                           C[17] * d1 * d1 * d2 + C[18] * d1 * d2 * d2) +
                 C[14] * d0 * d1 * d2;
    phi = C[0] + C[1] * d0 + C[2] * d1 + C[3] * d2 + q2 + q3;
    acc[0] = -g[0];
    acc[1] = -g[1];
    acc[2] = -g[2];
}

// dL/dC of one particle for a = -grad P(d), Phi = P(d), given v = dL/da and w = dL/dPhi
// (accumulated into cb).
template <typename T>
__device__ inline void taylor_cbar(T d0, T d1, T d2, T v0, T v1, T v2, T w, T cb[20]) {
    const T h = T(0.5), s6 = T(1.0 / 6.0);
    cb[0] += w;
    cb[1] += w * d0 - v0;
    cb[2] += w * d1 - v1;
    cb[3] += w * d2 - v2;
    cb[4] += w * h * d0 * d0 - v0 * d0;
    cb[5] += w * d0 * d1 - (v0 * d1 + v1 * d0);
    cb[6] += w * d0 * d2 - (v0 * d2 + v2 * d0);
    cb[7] += w * h * d1 * d1 - v1 * d1;
    cb[8] += w * d1 * d2 - (v1 * d2 + v2 * d1);
    cb[9] += w * h * d2 * d2 - v2 * d2;
    cb[10] += w * s6 * d0 * d0 * d0 - v0 * h * d0 * d0;
    cb[11] += w * h * d0 * d0 * d1 - (v0 * d0 * d1 + v1 * h * d0 * d0);
    cb[12] += w * h * d0 * d0 * d2 - (v0 * d0 * d2 + v2 * h * d0 * d0);
    cb[13] += w * h * d0 * d1 * d1 - (v0 * h * d1 * d1 + v1 * d0 * d1);
    cb[14] += w * d0 * d1 * d2 - (v0 * d1 * d2 + v1 * d0 * d2 + v2 * d0 * d1);
    cb[15] += w * h * d0 * d2 * d2 - (v0 * h * d2 * d2 + v2 * d0 * d2);
    cb[16] += w * s6 * d1 * d1 * d1 - v1 * h * d1 * d1;
    cb[17] += w * h * d1 * d1 * d2 - (v1 * d1 * d2 + v2 * h * d1 * d1);
    cb[18] += w * h * d1 * d2 * d2 - (v1 * h * d2 * d2 + v2 * d1 * d2);
    cb[19] += w * s6 * d2 * d2 * d2 - v2 * h * d2 * d2;
}

// Butterfly reduce-scatter of V values (power of two, <= 32) across the warp: afterwards lane l
// holds the warp total of value (l mod V) in v[0].  Plain arithmetic.
template <int V, typename T>
__device__ inline void reduce_scatter(T (&v)[V]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (o >= V) {
#pragma unroll
            for (int i = 0; i < V; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
        } else {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < o; ++i) {
                const T send = up ? v[i] : v[i + o];
                const T keep = up ? v[i + o] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
}

// The same with compensated float pairs (s[i] + c[i]).
template <int V>
__device__ inline void reduce_scatter_df(float (&s)[V], float (&c)[V]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (o >= V) {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const float rs = __shfl_xor_sync(0xffffffffu, s[i], o), rc = __shfl_xor_sync(0xffffffffu, c[i], o);
                float t, e;
                two_sum(s[i], rs, t, e);
                s[i] = t;
                c[i] = __fadd_rn(__fadd_rn(c[i], rc), e);
            }
        } else {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < o; ++i) {
                const float ss = up ? s[i] : s[i + o], sc = up ? c[i] : c[i + o];
                const float ks = up ? s[i + o] : s[i], kc = up ? c[i + o] : c[i];
                const float rs = __shfl_xor_sync(0xffffffffu, ss, o), rc = __shfl_xor_sync(0xffffffffu, sc, o);
                float t, e;
                two_sum(ks, rs, t, e);
                s[i] = t;
                c[i] = __fadd_rn(__fadd_rn(kc, rc), e);
            }
        }
    }
}

template <typename T>
__device__ inline void pair_force(T dx, T dy, T dz, T hsum, T mb, T &ax, T &ay, T &az, T &ph);

template <>
__device__ inline void pair_force<float>(float dx, float dy, float dz, float hsum, float mb, float &ax, float &ay,
                                         float &az, float &ph) {
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
    const float r = r2 * rinv;
    const float hinv = __fdividef(2.0f, hsum);
    const float q = r * hinv;
    float sr = rinv * rinv * rinv;  // S/r for q >= 2
    float p = -rinv;
    if (q < 2.0f) {
        const float h3 = hinv * hinv * hinv;
        const float q2 = q * q;
        if (q < 1.0f) {
            sr = h3 * (4.0f / 3.0f + q2 * (-1.2f + 0.5f * q));
            p = hinv * (q2 * (2.0f / 3.0f + q2 * (-0.3f + 0.1f * q)) - 1.4f);
        } else {
            sr = h3 * (8.0f / 3.0f + q * (-3.0f + q * (1.2f - q * (1.0f / 6.0f)))) - (1.0f / 15.0f) * sr;
            p = hinv * (q2 * (4.0f / 3.0f + q * (-1.0f + q * (0.3f - q * (1.0f / 30.0f)))) - 1.6f) + (1.0f / 15.0f) * rinv;
        }
    }
    const float w = mb * sr;
    ax = -w * dx;
    ay = -w * dy;
    az = -w * dz;
    ph = mb * p;
}

template <>
__device__ inline void pair_force<double>(double dx, double dy, double dz, double hsum, double mb, double &ax,
                                          double &ay, double &az, double &ph) {
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double rinv = r2 > 0.0 ? rsqrt(r2) : 0.0;
    const double r = r2 * rinv;
    const double hinv = 2.0 / hsum;
    const double q = r * hinv;
    double sr = rinv * rinv * rinv;
    double p = -rinv;
    if (q < 2.0) {
        const double h3 = hinv * hinv * hinv;
        const double q2 = q * q;
        if (q < 1.0) {
            sr = h3 * (4.0 / 3.0 + q2 * (-1.2 + 0.5 * q));
            p = hinv * (q2 * (2.0 / 3.0 + q2 * (-0.3 + 0.1 * q)) - 1.4);
        } else {
            sr = h3 * (8.0 / 3.0 + q * (-3.0 + q * (1.2 - q * (1.0 / 6.0)))) - (1.0 / 15.0) * sr;
            p = hinv * (q2 * (4.0 / 3.0 + q * (-1.0 + q * (0.3 - q * (1.0 / 30.0)))) - 1.6) + (1.0 / 15.0) * rinv;
        }
    }
    const double w = mb * sr;
    ax = -w * dx;
    ay = -w * dy;
    az = -w * dz;
    ph = mb * p;
}


// Gradient of one pair term.  With r = x_a - x_b, F(r) = (S/r) r and phi(r):
//   a_a = -m_b F,  Phi_a = m_b phi,  dF/dr = (S/r) I + ((S/r)'/r) r r^T,  dphi/dr = (S/r) r.
// For v = dL/da_a and w = dL/dPhi_a this returns g = dL/dr (to add to x_a and subtract from x_b)
// and gm = dL/dm_b.
template <typename T>
__device__ inline void pair_grad(T dx, T dy, T dz, T hsum, T mb, T vx, T vy, T vz, T w, T &gx, T &gy, T &gz,
                                 T &gm) {
    const T r2 = dx * dx + dy * dy + dz * dz;
    const T rinv = r2 > T(0) ? rsqrt(r2) : T(0);
    const T r = r2 * rinv;
    const T hinv = T(2) / hsum;
    const T q = r * hinv;
    const T rinv2 = rinv * rinv;
    T sr = rinv * rinv2;            // S/r
    T dsr = T(-3) * sr * rinv2;     // (S/r)'/r
    T p = -rinv;
    if (q < T(2)) {
        const T h2 = hinv * hinv, h3 = h2 * hinv, h5 = h3 * h2;
        const T q2 = q * q;
        if (q < T(1)) {
            sr = h3 * (T(4.0 / 3.0) + q2 * (T(-1.2) + T(0.5) * q));
            dsr = h5 * (T(-2.4) + T(1.5) * q);
            p = hinv * (q2 * (T(2.0 / 3.0) + q2 * (T(-0.3) + T(0.1) * q)) - T(1.4));
        } else {
            const T r3 = sr;
            sr = h3 * (T(8.0 / 3.0) + q * (T(-3) + q * (T(1.2) - q * T(1.0 / 6.0)))) - T(1.0 / 15.0) * r3;
            dsr = h5 * (T(-3) / q + T(2.4) - T(0.5) * q) + T(0.2) * r3 * rinv2;
            p = hinv * (q2 * (T(4.0 / 3.0) + q * (T(-1) + q * (T(0.3) - q * T(1.0 / 30.0)))) - T(1.6)) +
                T(1.0 / 15.0) * rinv;
        }
    }
    const T rv = dx * vx + dy * vy + dz * vz;
    const T k1 = mb * sr, k2 = mb * dsr * rv, k3 = w * mb * sr;
    gx = -(k1 * vx + k2 * dx) + k3 * dx;
    gy = -(k1 * vy + k2 * dy) + k3 * dy;
    gz = -(k1 * vz + k2 * dz) + k3 * dz;
    gm = -sr * rv + w * p;
}

}  // namespace rcb
