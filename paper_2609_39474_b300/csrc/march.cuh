// Physical-step kernels of the device-resident march (Sections 2.3, 3.1; Algorithm 1):
// equilibrium initialisation, moments, BDF history term and population warm start, the
// reconstruction of m^{n+1} at acceptance, and the single-thread control kernels that rotate
// the histories and drive the CUDA-graph conditional nodes.  Field kernels are grid-stride
// loops over sites with SoA (coalesced) access; lattices enter through L::Q, L::D, L::c*, L::w.
#pragma once

#include "common.cuh"

namespace msc {

constexpr int kFieldThreads = 256;

template <class L>
__device__ __forceinline__ double cdotu(int k, const double* u) {
    double s = 0.0;
    if (L::cx(k)) s += L::cx(k) * u[0];
    if (L::cy(k)) s += L::cy(k) * u[1];
    if (L::D == 3 && L::cz(k)) s += L::cz(k) * u[2];
    return s;
}

// f = f_eq(p_hat, u)   (Eq. feq); p and u are double fields, f in the storage type
template <class L, typename T>
__global__ void k_equilibrium(const double* __restrict__ p, const double* __restrict__ u,
                              T* __restrict__ f, size_t sites) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sites;
         i += (size_t)gridDim.x * blockDim.x) {
        double uv[3] = {0.0, 0.0, 0.0};
        double uu = 0.0;
#pragma unroll
        for (int al = 0; al < L::D; ++al) {
            uv[al] = u[al * sites + i];
            uu += uv[al] * uv[al];
        }
        const double ph = p[i];
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const double cu = cdotu<L>(k, uv);
            f[k * sites + i] = (T)(L::w(k) * (ph + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
        }
    }
}

// m = P f in double (Eq. moments); optionally a second copy
template <class L, typename T>
__global__ void k_moments(const T* __restrict__ f, double* __restrict__ m, double* __restrict__ m2,
                          size_t sites) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sites;
         i += (size_t)gridDim.x * blockDim.x) {
        double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const double v = (double)f[k * sites + i];
            r += v;
            if (L::cx(k)) jx += L::cx(k) * v;
            if (L::cy(k)) jy += L::cy(k) * v;
            if (L::D == 3 && L::cz(k)) jz += L::cz(k) * v;
        }
        m[i] = r;
        m[sites + i] = jx;
        m[2 * sites + i] = jy;
        if (L::D == 3) m[3 * sites + i] = jz;
        if (m2) {
            m2[i] = r;
            m2[sites + i] = jx;
            m2[2 * sites + i] = jy;
            if (L::D == 3) m2[3 * sites + i] = jz;
        }
    }
}

// Start of a physical step: h_q from the accepted moment histories (Eq. bdf2) and the trial
// populations from the population-history extrapolation (Section 3.1) into the working slot.
template <class L, typename T>
__global__ void k_step_begin(const DevState* __restrict__ st, T* __restrict__ fbase, size_t fstride,
                             const double* __restrict__ mbuf, T* __restrict__ h, size_t sites) {
    const volatile DevState* vs = st;
    const int q = vs->q;
    const double dt = vs->dt;
    const int nav = vs->n_avail;
    const size_t mstride = (size_t)(L::D + 1) * sites;
    const double* mn = mbuf + (size_t)vs->m_cur * mstride;
    const double* mnm1 = mbuf + (size_t)vs->m_prev * mstride;
    const T* f0 = fbase + (size_t)vs->slot_fn[0] * fstride;
    const T* f1 = fbase + (size_t)vs->slot_fn[1] * fstride;
    const T* f2 = fbase + (size_t)vs->slot_fn[2] * fstride;
    T* ft = fbase + (size_t)vs->slot_cur * fstride;
    const double c1 = q == 1 ? 1.0 / dt : 4.0 / (2.0 * dt);
    const double c2 = q == 1 ? 0.0 : 1.0 / (2.0 * dt);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sites;
         i += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c <= L::D; ++c) {
            const size_t o = c * sites + i;
            h[o] = (T)(c1 * mn[o] - c2 * mnm1[o]);
        }
        if (nav == 1) {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) ft[k * sites + i] = f0[k * sites + i];
        } else if (nav == 2) {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) {
                const size_t o = k * sites + i;
                ft[o] = T(2) * f0[o] - f1[o];
            }
        } else {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) {
                const size_t o = k * sites + i;
                ft[o] = T(3) * (f0[o] - f1[o]) + f2[o];
            }
        }
    }
}

// Acceptance: m^{n+1} = R_{q,h}(f^{n+1}) with the unrotated histories (Eq. macro-reconstruct),
// evaluated in FP64 and written into the m^{n-1} slot (rotated by k_step_finish).
template <class L, typename T>
__global__ void k_step_end(const DevState* __restrict__ st, const T* __restrict__ fbase, size_t fstride,
                           double* __restrict__ mbuf, size_t sites) {
    const volatile DevState* vs = st;
    if (!vs->accepted) return;
    const int q = vs->q;
    const double dt = vs->dt;
    const double a = vs->a;
    const double inv = 1.0 / (1.0 + a / 2.0);
    const size_t mstride = (size_t)(L::D + 1) * sites;
    const double* mn = mbuf + (size_t)vs->m_cur * mstride;
    double* mnm1 = mbuf + (size_t)vs->m_prev * mstride;
    const T* ft = fbase + (size_t)vs->slot_cur * fstride;
    const double c1 = q == 1 ? 1.0 / dt : 4.0 / (2.0 * dt);
    const double c2 = q == 1 ? 0.0 : 1.0 / (2.0 * dt);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sites;
         i += (size_t)gridDim.x * blockDim.x) {
        double mom[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const double v = (double)ft[k * sites + i];
            mom[0] += v;
            if (L::cx(k)) mom[1] += L::cx(k) * v;
            if (L::cy(k)) mom[2] += L::cy(k) * v;
            if (L::D == 3 && L::cz(k)) mom[3] += L::cz(k) * v;
        }
#pragma unroll
        for (int c = 0; c <= L::D; ++c) {
            const size_t o = c * sites + i;
            const double hc = c1 * mn[o] - c2 * mnm1[o];
            mnm1[o] = (mom[c] + 0.5 * hc) * inv;
        }
    }
}

// ---- single-thread control kernels ------------------------------------------------------------

__global__ void k_set_params(DevState* st, msc_params p) {
    st->nu = p.nu;
    st->dt = p.dt;
    st->eps = p.eps;
    st->kmax = p.kmax;
    st->nmin = p.nmin;
    st->corrector = p.corrector;
    st->replay = p.replay;
    st->params_ok = 1;
}

__global__ void k_reset_history(DevState* st) {
    st->steps_done = 0;
    st->n_avail = 1;
    st->slot_fn[0] = 0;
    st->slot_fn[1] = 1;
    st->slot_fn[2] = 2;
    st->slot_cur = 3;
    st->slot_nxt = 4;
    st->m_cur = 0;
    st->m_prev = 1;
    st->status = MSC_OK;
    st->steps_in_call = 0;
    st->inner_total = 0;
    st->hist_pos = 0;
    st->last_iters = 0;
    st->last_q = 0;
    st->R_last = 0.0;
}

__global__ void k_set_target(DevState* st, int n_steps) {
    st->steps_target = n_steps;
    st->steps_in_call = 0;
    st->inner_total = 0;
    st->hist_pos = 0;
    st->status = MSC_OK;
}

__global__ void k_arm(DevState* st, cudaGraphConditionalHandle h_step) {
    const bool go = st->steps_target > 0 && st->params_ok && st->status == MSC_OK;
    if (!st->params_ok) st->status = MSC_ERR_STATE;
    cudaGraphSetConditional(h_step, go ? 1u : 0u);
}

__device__ inline bool slot_in_history(const DevState* st, int s) {
    for (int i = 0; i < st->n_avail; ++i)
        if (st->slot_fn[i] == s) return true;
    return false;
}

__global__ void k_step_setup(DevState* st, cudaGraphConditionalHandle h_iter) {
    st->q = st->steps_done == 0 ? 1 : 2;
    st->a = st->q == 1 ? 1.0 / st->dt : 3.0 / (2.0 * st->dt);
    st->iter = 0;
    st->accepted = 0;
    st->lift = 0;
    int picked = 0;
    for (int s = 0; s < kNumFBuf && picked < 2; ++s) {
        if (slot_in_history(st, s)) continue;
        if (picked == 0) st->slot_cur = s; else st->slot_nxt = s;
        ++picked;
    }
    cudaGraphSetConditional(h_iter, 1u);
}

__global__ void k_step_finish(DevState* st, int* iters_out, int max_steps,
                              cudaGraphConditionalHandle h_step) {
    unsigned int go = 0u;
    if (st->accepted && st->status == MSC_OK) {
        const int k = st->steps_in_call;
        if (k < max_steps) iters_out[k] = st->iter;
        st->slot_fn[2] = st->slot_fn[1];
        st->slot_fn[1] = st->slot_fn[0];
        st->slot_fn[0] = st->slot_cur;
        if (st->n_avail < 3) st->n_avail += 1;
        const int t = st->m_cur;  // m^{n+1} was written into the m^{n-1} slot
        st->m_cur = st->m_prev;
        st->m_prev = t;
        st->steps_done += 1;
        st->steps_in_call = k + 1;
        st->steps_target -= 1;
        st->last_iters = st->iter;
        st->last_q = st->q;
        go = st->steps_target > 0 ? 1u : 0u;
    }
    cudaGraphSetConditional(h_step, go);
}

// m^n = P f^n of the accepted slot into both moment slots (after an explicit march)
template <class L, typename T>
__global__ void k_moments_state(const DevState* __restrict__ st, const T* __restrict__ fbase, size_t fstride,
                                double* __restrict__ mbuf, size_t sites) {
    const volatile DevState* vs = st;
    const T* f = fbase + (size_t)vs->slot_fn[0] * fstride;
    const size_t mstride = (size_t)(L::D + 1) * sites;
    double* m0 = mbuf + (size_t)vs->m_cur * mstride;
    double* m1 = mbuf + (size_t)vs->m_prev * mstride;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sites;
         i += (size_t)gridDim.x * blockDim.x) {
        double mom[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const double v = (double)f[k * sites + i];
            mom[0] += v;
            if (L::cx(k)) mom[1] += L::cx(k) * v;
            if (L::cy(k)) mom[2] += L::cy(k) * v;
            if (L::D == 3 && L::cz(k)) mom[3] += L::cz(k) * v;
        }
#pragma unroll
        for (int c = 0; c <= L::D; ++c) {
            m0[c * sites + i] = mom[c];
            m1[c * sites + i] = mom[c];
        }
    }
}

// explicit march bookkeeping: ping-pong between the accepted slot and one free slot
__global__ void k_ex_setup(DevState* st, int pairs) {
    st->ex_a = st->slot_fn[0];
    st->ex_b = (st->slot_fn[0] + 1) % kNumFBuf;
    st->ex_pairs_left = pairs;
}

__global__ void k_ex_arm(DevState* st, cudaGraphConditionalHandle h_ex) {
    cudaGraphSetConditional(h_ex, st->ex_pairs_left > 0 ? 1u : 0u);
}

__global__ void k_ex_finish(DevState* st, int odd) {
    st->slot_fn[0] = odd ? st->ex_b : st->ex_a;
    int s1 = (st->slot_fn[0] + 1) % kNumFBuf;
    int s2 = (st->slot_fn[0] + 2) % kNumFBuf;
    st->slot_fn[1] = s1;
    st->slot_fn[2] = s2;
    st->n_avail = 1;
    st->steps_done = 0;
    st->m_cur = 0;
    st->m_prev = 1;
}

}  // namespace msc
