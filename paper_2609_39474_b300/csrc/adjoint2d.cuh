// Discrete adjoint of one converged D2Q9 physical step: implicit differentiation of the accepted
// fixed point f = T(f; h) (Eqs. fixed-point-problem, sweep) at the operating point.
//
// With m = R(f) (Eq. macro-reconstruct) the operating-point collision depends on f only through m
// (Eq. collision-operating), so dT/df = S K P with K = D_m / (1 + a/2), D_m = dC/dm per site (the
// source s = h - a m carried along, Eqs. source-moments, source-distribution).  The adjoint system
// (I - dT/df)^T lambda = P^T mu / (1 + a/2) therefore has its solution in range(P^T): lambda = P^T
// theta with the three-field fixed point
//     theta = c + A theta,   c = mu / (1 + a/2),   (A theta)(x) = K(x)^T v(x),
//     v_k(x) = theta_0(x + c_k) + c_k . theta_u(x + c_k)              (pull-transpose of streaming),
// solved by the transposed shadow correction (P E = I makes it act on theta directly):
//     rho = c + A theta - theta,   theta <- theta + rho + F^{-1} chi (H(k)^H)^{-1} F rho.
// Then dL/dh = K_h^T v + mu / (2 (1 + a/2)) with K_h = D_m / (2 (1 + a/2)) + G_s, G_s = dC/ds, and
// the BDF history h = c1 m^n - c2 m^{n-1} + (0, F) passes it to m^n, m^{n-1} and the force.
//
// Per site, with S0 = sum w v, S1 = sum w v c, T = sum w v c c (weighted moments of v):
//   (D_m^T v)_p = (1 - a/2) S0
//   (D_m^T v)_b = (3 - 1.5a) S1_b + (9 - 4.5a) (T u)_b + 4.5 (T s)_b - ((3 - 1.5a) u_b + 1.5 s_b) S0
//   (G_s^T v)_0 = S0 / 2,   (G_s^T v)_b = 1.5 S1_b - 1.5 u_b S0 + 4.5 (T u)_b
// (derivatives of C_k = w_k [p + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u] + w_k [s0 + 3 (c.s - u.s) +
// 9 (c.u)(c.s)] / 2 with s0 = h0 - a p, s_u = h_u - a u).
#pragma once

#include "common.cuh"
#include "march.cuh"

namespace msc {

struct AdjArgs {
    const double* m;     // m^{n+1}, 3 fields
    const double* heff;  // h^n + (0, F), 3 fields (formed by k_adj_prepare)
    const double* mu;    // dL/dm^{n+1}, 3 fields
    double* abar_cur;    // dL/dm^n (accumulated)
    double* abar_prev;   // dL/dm^{n-1} (accumulated; unused when c2 = 0)
    double* dforce;      // dL/dF (accumulated, 2 values)
    double a, inv, c1, c2;
    int n;
    double* partial;     // per-block partial sums (grid x 2)
    unsigned int* counter;
    double* out;         // reduction results
};

// fixed-order sum of up to two values over the grid: per-block partials, the last block adds them
__device__ inline void grid_sum2(double v0, double v1, double* partial, unsigned int* counter, double* out,
                                 bool accumulate) {
    __shared__ double s0[32], s1[32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    if (lane == 0) { s0[warp] = v0; s1[warp] = v1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b0 = 0.0, b1 = 0.0;
        for (int w = 0; w < nw; ++w) { b0 += s0[w]; b1 += s1[w]; }
        partial[2 * blockIdx.x] = b0;
        partial[2 * blockIdx.x + 1] = b1;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double t0 = 0.0, t1 = 0.0;
    for (unsigned int b = 0; b < gridDim.x; ++b) {
        t0 += __ldcg(partial + 2 * b);
        t1 += __ldcg(partial + 2 * b + 1);
    }
    *counter = 0u;
    if (accumulate) { out[0] += t0; out[1] += t1; }
    else { out[0] = t0; out[1] = t1; }
}

// h_eff = c1 m^n - c2 m^{n-1} + (0, F) (the forward's formula), theta = c = mu / (1 + a/2), |c|^2
template <typename T>
__global__ void __launch_bounds__(kFieldThreads) k_adj_prepare(AdjArgs A, const double* __restrict__ m_cur,
                                                               const double* __restrict__ m_prev, double f0,
                                                               double f1, double* __restrict__ heff,
                                                               T* __restrict__ theta) {
    const size_t sites = (size_t)A.n * A.n;
    const double fc[3] = {0.0, f0, f1};
    double cc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sites; i += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t o = c * sites + i;
            heff[o] = fma(A.c1, m_cur[o], fma(-A.c2, m_prev[o], fc[c]));
            const double cv = A.mu[o] * A.inv;
            theta[o] = (T)cv;
            cc += cv * cv;
        }
    }
    grid_sum2(cc, 0.0, A.partial, A.counter, A.out, false);
}

// One application of the reduced adjoint map.  FINAL = false: rho = c + A theta - theta and |rho|^2.
// FINAL = true: nu = dL/dh (see the header), accumulated into abar_cur (+c1 nu), abar_prev (-c2 nu)
// and dforce (the velocity parts of nu summed over sites).
template <typename T, bool FINAL>
__global__ void __launch_bounds__(kFieldThreads) k_adj_sweep(AdjArgs A, const T* __restrict__ theta,
                                                             T* __restrict__ rho) {
    using L = D2Q9;
    const int n = A.n, nm = n - 1;
    const size_t sites = (size_t)n * n;
    const double a = A.a, inv = A.inv;
    double r0 = 0.0, r1 = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sites; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i & nm), y = (int)(i >> (__ffs(n) - 1));
        // v_k(x) = (P^T theta)_k (x + c_k)
        double S0 = 0.0, S1x = 0.0, S1y = 0.0, Txx = 0.0, Txy = 0.0, Tyy = 0.0;
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const size_t j = (size_t)((y + L::cy(k)) & nm) * n + ((x + L::cx(k)) & nm);
            double v = (double)theta[j];
            if (L::cx(k)) v += L::cx(k) * (double)theta[sites + j];
            if (L::cy(k)) v += L::cy(k) * (double)theta[2 * sites + j];
            const double wv = L::w(k) * v;
            S0 += wv;
            if (L::cx(k)) { S1x += L::cx(k) * wv; Txx += wv; }
            if (L::cy(k)) { S1y += L::cy(k) * wv; Tyy += wv; }
            if (L::cx(k) && L::cy(k)) Txy += L::cx(k) * L::cy(k) * wv;
        }
        const double p = A.m[i], ux = A.m[sites + i], uy = A.m[2 * sites + i];
        const double sx = A.heff[sites + i] - a * ux, sy = A.heff[2 * sites + i] - a * uy;
        (void)p;
        const double Tux = Txx * ux + Txy * uy, Tuy = Txy * ux + Tyy * uy;
        const double Tsx = Txx * sx + Txy * sy, Tsy = Txy * sx + Tyy * sy;
        const double k3 = 3.0 - 1.5 * a, k9 = 9.0 - 4.5 * a;
        const double A0 = inv * (1.0 - 0.5 * a) * S0;
        const double Ax = inv * (k3 * S1x + k9 * Tux + 4.5 * Tsx - (k3 * ux + 1.5 * sx) * S0);
        const double Ay = inv * (k3 * S1y + k9 * Tuy + 4.5 * Tsy - (k3 * uy + 1.5 * sy) * S0);
        const double c0 = A.mu[i] * inv, cx = A.mu[sites + i] * inv, cy = A.mu[2 * sites + i] * inv;
        if (!FINAL) {
            const double q0 = c0 + A0 - (double)theta[i];
            const double qx = cx + Ax - (double)theta[sites + i];
            const double qy = cy + Ay - (double)theta[2 * sites + i];
            rho[i] = (T)q0;
            rho[sites + i] = (T)qx;
            rho[2 * sites + i] = (T)qy;
            r0 += q0 * q0 + qx * qx + qy * qy;
        } else {
            const double g0 = 0.5 * S0;
            const double gx = 1.5 * S1x - 1.5 * ux * S0 + 4.5 * Tux;
            const double gy = 1.5 * S1y - 1.5 * uy * S0 + 4.5 * Tuy;
            const double nu0 = 0.5 * A0 + g0 + 0.5 * c0;
            const double nux = 0.5 * Ax + gx + 0.5 * cx;
            const double nuy = 0.5 * Ay + gy + 0.5 * cy;
            A.abar_cur[i] += A.c1 * nu0;
            A.abar_cur[sites + i] += A.c1 * nux;
            A.abar_cur[2 * sites + i] += A.c1 * nuy;
            if (A.c2 != 0.0) {
                A.abar_prev[i] -= A.c2 * nu0;
                A.abar_prev[sites + i] -= A.c2 * nux;
                A.abar_prev[2 * sites + i] -= A.c2 * nuy;
            }
            r0 += nux;
            r1 += nuy;
        }
    }
    if (!FINAL) grid_sum2(r0, 0.0, A.partial, A.counter, A.out, false);
    else grid_sum2(r0, r1, A.partial, A.counter, A.dforce, true);
}

// theta += rho + delta (delta = the transposed shadow correction of rho)
template <typename T>
__global__ void __launch_bounds__(kFieldThreads) k_adj_update(T* __restrict__ theta, const T* __restrict__ rho,
                                                              const T* __restrict__ delta, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        theta[i] = theta[i] + rho[i] + delta[i];
}

}  // namespace msc
