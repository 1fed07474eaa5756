// Far- and near-field arithmetic shared by the gravity kernels and their backward pass:
// symmetric-tensor slots, the monopole + quadrupole Taylor coefficients of one far source
// (Eq. 5 expanded to third order), the sink's Taylor polynomial (Eq. 6), warp reduce-scatters,
// and the kernel-softened pair force (Eqs. 9-10) with its gradient.
#pragma once

#include <cuda_runtime.h>

#include "rcb_internal.cuh"

namespace rcb {

// symmetric slot of an index pair / triple (orders 2 and 3, lexicographic sorted tuples)
__host__ __device__ constexpr int s2(int i, int j) {
    return i > j ? s2(j, i) : (i == 0 ? j : (i == 1 ? 2 + j : 5));
}
__host__ __device__ constexpr int sort3_slot(int a, int b, int c) {
    // a <= b <= c
    return a == 0 ? (b == 0 ? c : (b == 1 ? 2 + c : 5)) : (a == 1 ? (b == 1 ? 5 + c : 8) : 9);
}
__host__ __device__ constexpr int s3(int i, int j, int k) {
    return (i <= j && j <= k)   ? sort3_slot(i, j, k)
           : (i <= k && k <= j) ? sort3_slot(i, k, j)
           : (j <= i && i <= k) ? sort3_slot(j, i, k)
           : (j <= k && k <= i) ? sort3_slot(j, k, i)
           : (k <= i && i <= j) ? sort3_slot(k, i, j)
                                : sort3_slot(k, j, i);
}

// Coefficients of one far source (see the file header); C is accumulated into.
template <typename T>
__device__ inline void far_source(const T x[3], T M, const T Q6[6], T C[20]) {
    const T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    const T g = rsqrt(r2);
    const T g2 = g * g, g3 = g * g2, g5 = g3 * g2, g7 = g5 * g2, g9 = g7 * g2, g11 = g9 * g2;
    T Q[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q[i][j] = Q6[s2(i, j)];
    T v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = Q[i][0] * x[0] + Q[i][1] * x[1] + Q[i][2] * x[2];
    const T s = x[0] * v[0] + x[1] * v[1] + x[2] * v[2];
    const T a = M * g3 + T(2.5) * s * g7;
    const T b = T(-3) * M * g5 - T(17.5) * s * g9;
    const T c = T(15) * M * g7 + T(157.5) * s * g11;
    const T f7 = T(5) * g7, f9 = T(35) * g9;
    C[0] += -M * g - T(0.5) * s * g5;
#pragma unroll
    for (int i = 0; i < 3; ++i) C[1 + i] += a * x[i] - g5 * v[i];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            T t = b * x[i] * x[j] - g5 * Q[i][j] + f7 * (v[i] * x[j] + v[j] * x[i]);
            if (i == j) t += a;
            C[4 + s2(i, j)] += t;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
#pragma unroll
            for (int k = j; k < 3; ++k) {
                T t = c * x[i] * x[j] * x[k] + f7 * (Q[i][j] * x[k] + Q[i][k] * x[j] + Q[j][k] * x[i]) -
                      f9 * (v[i] * x[j] * x[k] + v[j] * x[i] * x[k] + v[k] * x[i] * x[j]);
                T dsum = T(0), vsum = T(0);
                if (i == j) { dsum += x[k]; vsum += v[k]; }
                if (i == k) { dsum += x[j]; vsum += v[j]; }
                if (j == k) { dsum += x[i]; vsum += v[i]; }
                t += b * dsum + f7 * vsum;
                C[10 + s3(i, j, k)] += t;
            }
}

// Third-order Taylor polynomial of the sink (Eq. 6): phi and a = -grad phi at offset d.
template <typename T>
__device__ inline void taylor_eval(const T C[20], const T d[3], T &phi, T acc[3]) {
    T g[3];
    T p = C[0];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        g[i] = C[1 + i];
        p += C[1 + i] * d[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const T c2 = C[4 + s2(i, j)];
            g[i] += c2 * d[j];
            p += T(0.5) * c2 * d[i] * d[j];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T c3 = C[10 + s3(i, j, k)];
                g[i] += T(0.5) * c3 * d[j] * d[k];
                p += c3 * d[i] * d[j] * d[k] * T(1.0 / 6.0);
            }
        }
    phi = p;
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[i] = -g[i];
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
