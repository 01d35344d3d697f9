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

// Arguments of one adjoint step.  A run of steps has its argument blocks in device memory (one
// host-to-device copy per run) and the graph of the transposed solve picks the block of the current
// step through AdjCtl::slot, so that one instantiated graph serves every step unchanged.
struct AdjArgs {
    const double* m;       // m^{n+1}, 3 fields
    const double* m_cur;   // m^n
    const double* m_prev;  // m^{n-1} (m^n when c2 = 0)
    const double* mu;      // dL/dm^{n+1}, 3 fields
    double* heff;          // h^n + (0, F), 3 fields (formed by k_adj_prepare)
    double* abar_cur;      // dL/dm^n (accumulated)
    double* abar_prev;     // dL/dm^{n-1} (accumulated; unused when c2 = 0)
    double* dforce;        // dL/dF (accumulated, 2 values)
    double* partial;       // per-block partial sums (grid x 2)
    unsigned int* counter;
    double a, inv, c1, c2;  // BDF reaction a, 1 / (1 + a/2), history weights
    double f0, f1;          // body force
    double eps;             // relative residual bound of the transposed solve
    int kmax;               // iteration limit
    int n;
    int warm;               // start from c + (theta - c) of the last converged step (else theta = c)
};

// Outcome of one step's transposed solve (read back once per run of steps).
struct AdjStat {
    double cnorm;  // RMS of c = mu / (1 + a/2)
    double rel;    // last relative residual RMS(rho) / RMS(c)
    int it;        // corrections applied
    int status;    // MSC_OK, MSC_ERR_NONFINITE, MSC_ERR_NONCONVERGED; MSC_ERR_STATE: not run
};

// Position in a run of steps: the current step, and whether an earlier step failed (the rest of
// the run then does nothing).  Advanced by k_adj_advance, the last node of each step's graph.
struct AdjCtl {
    int slot;
    int abort;
};

// Fixed-order sum of two values over the grid: per-block partials; the last block to finish adds
// them with all its threads (a strided pass in block order, then the fixed warp and block trees),
// so the totals do not depend on which block finishes last.  Returns true on the one thread (of the
// last block) that holds the totals.
__device__ inline bool grid_sum2(double v0, double v1, double* partial, unsigned int* counter, double& t0,
                                 double& t1) {
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
    if (!last) return false;  // uniform over the block
    __threadfence();
    double a0 = 0.0, a1 = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        a0 += __ldcg(partial + 2 * b);
        a1 += __ldcg(partial + 2 * b + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    if (lane == 0) { s0[warp] = a0; s1[warp] = a1; }  // thread 0 finished reading s0, s1 above
    __syncthreads();
    if (threadIdx.x != 0) return false;
    t0 = 0.0;
    t1 = 0.0;
    for (int w = 0; w < nw; ++w) { t0 += s0[w]; t1 += s1[w]; }
    *counter = 0u;
    return true;
}

// h_eff = c1 m^n - c2 m^{n-1} + (0, F) (the forward's formula), c = mu / (1 + a/2), |c|^2, and the
// start theta = c, or theta = c + w with w = theta - c of the last converged step (warm start: the
// transposed maps of neighbouring steps differ little, so their propagated parts A theta do too);
// the last block opens the loop of the transposed solve when c is finite and nonzero.
template <typename T>
__global__ void __launch_bounds__(kFieldThreads) k_adj_prepare(const AdjArgs* __restrict__ args,
                                                               AdjStat* stats, const AdjCtl* ctl,
                                                               T* __restrict__ theta, const T* __restrict__ warm,
                                                               cudaGraphConditionalHandle h_loop, int cond) {
    const int slot = ctl->slot;
    AdjStat* st = stats + slot;
    if (ctl->abort) {  // an earlier step of the run failed
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->cnorm = 0.0;
            st->rel = 0.0;
            st->it = 0;
            st->status = MSC_ERR_STATE;
            if (cond) cudaGraphSetConditional(h_loop, 0u);
        }
        return;
    }
    const AdjArgs* __restrict__ P = args + slot;
    const size_t sites = (size_t)P->n * P->n;
    const double c1 = P->c1, c2 = P->c2, inv = P->inv;
    const double* __restrict__ m_cur = P->m_cur;
    const double* __restrict__ m_prev = P->m_prev;
    const double* __restrict__ mu = P->mu;
    double* __restrict__ heff = P->heff;
    const double fc[3] = {0.0, P->f0, P->f1};
    const bool use_warm = P->warm != 0;
    double cc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sites; i += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t o = c * sites + i;
            heff[o] = fma(c1, m_cur[o], fma(-c2, m_prev[o], fc[c]));
            const double cv = mu[o] * inv;
            theta[o] = use_warm ? (T)cv + warm[o] : (T)cv;
            cc += cv * cv;
        }
    }
    double t0, t1;
    if (grid_sum2(cc, 0.0, P->partial, P->counter, t0, t1)) {
        const double cnorm = sqrt(t0 / (3.0 * (double)sites));
        st->cnorm = cnorm;
        st->rel = 0.0;
        st->it = 0;
        st->status = isfinite(cnorm) ? MSC_OK : MSC_ERR_NONFINITE;
        if (cond) cudaGraphSetConditional(h_loop, isfinite(cnorm) && cnorm > 0.0 ? 1u : 0u);
    }
}

// One application of the reduced adjoint map.  FINAL = false: rho = c + A theta - theta and |rho|^2;
// the last block takes the acceptance decision of the iteration (relative residual below eps:
// stop; not finite or the limit reached: stop with that status; else one more correction).
// FINAL = true (only after a converged solve): nu = dL/dh (see the header), accumulated into
// abar_cur (+c1 nu), abar_prev (-c2 nu) and dforce (the velocity parts of nu summed over sites).
// The per-site arithmetic runs in the working type T (as the forward sweep does for FP32
// storage); the accumulators and the grid sums stay FP64.
template <typename T, bool FINAL>
__global__ void __launch_bounds__(kFieldThreads) k_adj_sweep(const AdjArgs* __restrict__ args,
                                                             AdjStat* stats, const AdjCtl* ctl,
                                                             const T* __restrict__ theta, T* __restrict__ rho,
                                                             T* __restrict__ warm,
                                                             cudaGraphConditionalHandle h_loop,
                                                             cudaGraphConditionalHandle h_corr, int cond) {
    using L = D2Q9;
    using R = T;
    const int slot = ctl->slot;
    AdjStat* st = stats + slot;
    if (FINAL && st->status != MSC_OK) return;
    const AdjArgs* __restrict__ P = args + slot;
    const int n = P->n, nm = n - 1;
    const size_t sites = (size_t)n * n;
    const R a = (R)P->a, inv = (R)P->inv;
    const R k3 = (R)(3.0 - 1.5 * P->a), k9 = (R)(9.0 - 4.5 * P->a), k1 = (R)(P->inv * (1.0 - 0.5 * P->a));
    const double* __restrict__ m = P->m;
    const double* __restrict__ heff = P->heff;
    const double* __restrict__ mu = P->mu;
    R r0 = R(0), r1 = R(0);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sites; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i & nm), y = (int)(i >> (__ffs(n) - 1));
        // v_k(x) = (P^T theta)_k (x + c_k)
        R S0 = R(0), S1x = R(0), S1y = R(0), Txx = R(0), Txy = R(0), Tyy = R(0);
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const size_t j = (size_t)((y + L::cy(k)) & nm) * n + ((x + L::cx(k)) & nm);
            R v = theta[j];
            if (L::cx(k)) v += R(L::cx(k)) * theta[sites + j];
            if (L::cy(k)) v += R(L::cy(k)) * theta[2 * sites + j];
            const R wv = R(L::w(k)) * v;
            S0 += wv;
            if (L::cx(k)) { S1x += R(L::cx(k)) * wv; Txx += wv; }
            if (L::cy(k)) { S1y += R(L::cy(k)) * wv; Tyy += wv; }
            if (L::cx(k) && L::cy(k)) Txy += R(L::cx(k) * L::cy(k)) * wv;
        }
        const R ux = (R)m[sites + i], uy = (R)m[2 * sites + i];
        const R sx = (R)(heff[sites + i] - P->a * m[sites + i]), sy = (R)(heff[2 * sites + i] - P->a * m[2 * sites + i]);
        const R Tux = Txx * ux + Txy * uy, Tuy = Txy * ux + Tyy * uy;
        const R Tsx = Txx * sx + Txy * sy, Tsy = Txy * sx + Tyy * sy;
        const R A0 = k1 * S0;
        const R Ax = inv * (k3 * S1x + k9 * Tux + R(4.5) * Tsx - (k3 * ux + R(1.5) * sx) * S0);
        const R Ay = inv * (k3 * S1y + k9 * Tuy + R(4.5) * Tsy - (k3 * uy + R(1.5) * sy) * S0);
        const R c0 = (R)mu[i] * inv, cx = (R)mu[sites + i] * inv, cy = (R)mu[2 * sites + i] * inv;
        if (!FINAL) {
            const R q0 = c0 + A0 - theta[i];
            const R qx = cx + Ax - theta[sites + i];
            const R qy = cy + Ay - theta[2 * sites + i];
            rho[i] = q0;
            rho[sites + i] = qx;
            rho[2 * sites + i] = qy;
            r0 += q0 * q0 + qx * qx + qy * qy;
        } else {
            const double c1 = P->c1, c2 = P->c2;
            double* __restrict__ ac = P->abar_cur;
            const R g0 = R(0.5) * S0;
            const R gx = R(1.5) * S1x - R(1.5) * ux * S0 + R(4.5) * Tux;
            const R gy = R(1.5) * S1y - R(1.5) * uy * S0 + R(4.5) * Tuy;
            const double nu0 = (double)(R(0.5) * A0 + g0 + R(0.5) * c0);
            const double nux = (double)(R(0.5) * Ax + gx + R(0.5) * cx);
            const double nuy = (double)(R(0.5) * Ay + gy + R(0.5) * cy);
            ac[i] += c1 * nu0;
            ac[sites + i] += c1 * nux;
            ac[2 * sites + i] += c1 * nuy;
            if (c2 != 0.0) {
                double* __restrict__ ap = P->abar_prev;
                ap[i] -= c2 * nu0;
                ap[sites + i] -= c2 * nux;
                ap[2 * sites + i] -= c2 * nuy;
            }
            r0 += (R)nux;
            r1 += (R)nuy;
            // the next step's warm start: w = theta - c
            warm[i] = theta[i] - c0;
            warm[sites + i] = theta[sites + i] - cx;
            warm[2 * sites + i] = theta[2 * sites + i] - cy;
        }
    }
    double t0, t1;
    if (!grid_sum2((double)r0, (double)r1, P->partial, P->counter, t0, t1)) return;
    if (FINAL) {
        P->dforce[0] += t0;
        P->dforce[1] += t1;
        return;
    }
    const double rel = sqrt(t0 / (3.0 * (double)sites)) / st->cnorm;
    st->rel = rel;
    unsigned int go = 0u;
    if (!isfinite(rel)) st->status = MSC_ERR_NONFINITE;
    else if (rel < P->eps) st->status = MSC_OK;
    else if (st->it >= P->kmax) st->status = MSC_ERR_NONCONVERGED;
    else { st->it += 1; go = 1u; }
    if (cond) {  // graph mode; a host-driven run reads the decision from the outcome block
        cudaGraphSetConditional(h_loop, go);
        cudaGraphSetConditional(h_corr, go);
    }
}

// end of a step: record a failure (the rest of the run is skipped) and move to the next slot
__global__ void k_adj_advance(const AdjStat* stats, AdjCtl* ctl) {
    const int slot = ctl->slot;
    if (stats[slot].status != MSC_OK) ctl->abort = 1;
    ctl->slot = slot + 1;
}

}  // namespace msc
