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

// The BDF history term h = c1 m_a - c2 m_b + f_c (Eq. bdf2 plus the body force), written to
// h[o] in the working-field type.  FP64 storage evaluates and stores it in FP64.
//
// FP32 / FP16 storage stores h as a binary32 pair, hi at h[o] and lo at h[o + lo_off], with
// hi + lo = h to ~2^-48 relative.  The sweep subtracts a m (m ~ the moments, a = a_q) from h with a
// fused multiply-add on hi and then adds lo, so the source s = h - a m, a small difference of two
// large terms, keeps its own relative accuracy; a single binary32 h would carry a rounding error of
// 2^-24 |h| into s at every site, which the long-wave shadow solve amplifies by 1/(a + nu|k|^2) and
// the march accumulates over its steps.  The pair is formed from the FP64 history with binary32
// error-free transformations only (B300's FP64 pipe runs at ~1/58 of the FP32 rate):
//   h = a_f g,  g = m_a + (m_a - m_b) c2/a   (c1 = a + c2 for BDF1 and BDF2)
// with a_f the binary32 a_q that the sweep uses for that step, so that the step's fixed point
// balances a_f m against h without a relative bias from rounded constants (with m_a = m_b = m, h is
// a_f m to ~2^-48).  m_a, m_b are split exactly into binary32 pairs (split_f64), m_a - m_b and its
// product with c2/a = 1/3 (BDF2, weight split into hi + lo) or 0 (BDF1) are formed in binary32
// (relative error 2^-23 of a term of size |m_a - m_b|), g as a two-sum pair, a_f g with the exact
// product error from an FMA; the force joins the low part and a final two-sum renormalises.  Both
// step kernels use this one routine, so a march resumed from a saved state repeats the
// uninterrupted march bit for bit.
template <typename T>
__device__ __forceinline__ void bdf_history(double c1, double ma, double c2, double mb, double fc, float af, int q,
                                            T* __restrict__ h, size_t o, size_t lo_off) {
    if constexpr (std::is_same<T, float>::value) {
        (void)c1;
        (void)c2;
        float ah, al, bh, bl;
        split_f64(ma, ah, al);
        split_f64(mb, bh, bl);
        float t = 0.0f;
        if (q == 2) {
            const float d = (ah - bh) + (al - bl);
            const float r_hi = (float)(1.0 / 3.0);
            const float r_lo = (float)(1.0 / 3.0 - (double)r_hi);
            t = fmaf(d, r_hi, d * r_lo);
        }
        float gh, ge;
        two_sum(ah, t, gh, ge);
        const float gl = ge + al;
        const float ph = af * gh;
        const float pl = fmaf(af, gl, fmaf(af, gh, -ph)) + narrow_f64(fc);
        float hi, lo;
        two_sum(ph, pl, hi, lo);
        h[o] = hi;
        h[o + lo_off] = lo;
    } else {
        (void)af;
        (void)q;
        (void)lo_off;
        h[o] = (T)fma(c1, ma, fma(-c2, mb, fc));
    }
}

// elements of the working field h: a binary32 pair per value for FP32 / FP16 storage (hi fields,
// then lo fields), one FP64 value otherwise
template <typename T>
__host__ __device__ constexpr int h_parts() {
    return std::is_same<T, float>::value ? 2 : 1;
}

// storage scale of the populations: from the state when there is one, else 1
__device__ __forceinline__ double pop_scale(const DevState* st) {
    return st ? st->fscale : 1.0;
}

// f = f_eq(p_hat, u)   (Eq. feq); p and u are double fields, f in the storage type S
template <class L, typename S>
__global__ void k_equilibrium(const double* __restrict__ p, const double* __restrict__ u,
                              S* __restrict__ f, size_t sites, const DevState* st = nullptr) {
    const double isig = st ? st->isig : 1.0;
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
            st_pop<double, S>(f, k * sites + i, L::w(k) * (ph + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu), isig);
        }
    }
}

// max |f_eq(p_hat, u)| over sites and directions into st->fmax_bits (FP16 storage scale)
template <class L>
__global__ void k_feq_absmax(const double* __restrict__ p, const double* __restrict__ u, size_t sites,
                             DevState* st) {
    double mx = 0.0;
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
            mx = fmax(mx, fabs(L::w(k) * (ph + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)));
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0 && mx > 0.0)
        atomicMax(&st->fmax_bits, (unsigned long long)__double_as_longlong(mx));
}

// sigma = the power of two just above max |f^0| (1 for a zero field): stored values |f| / sigma < 1
__global__ void k_set_scale(DevState* st) {
    const double mx = __longlong_as_double((long long)st->fmax_bits);
    double sig = 1.0;
    if (mx > 0.0 && isfinite(mx)) {
        int e;
        frexp(mx, &e);  // mx = m 2^e with 0.5 <= m < 1
        sig = ldexp(1.0, e);
    }
    st->fscale = sig;
    st->isig = 1.0 / sig;
}

// m = P f in double (Eq. moments); optionally a second copy
template <class L, typename S>
__global__ void k_moments(const S* __restrict__ f, double* __restrict__ m, double* __restrict__ m2,
                          size_t sites, const DevState* st = nullptr) {
    const double sig = pop_scale(st);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sites;
         i += (size_t)gridDim.x * blockDim.x) {
        double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const double v = ld_pop<double, S>(f, k * sites + i, sig);
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

// P of one site's trial populations into the P f field of its ring slot (D3Q19: the halo-free sweep
// reads the moments of its input from there)
template <class L, typename T, typename S>
__device__ __forceinline__ void store_trial_moments(S* __restrict__ pf, size_t sites, size_t i, const T* tv) {
    T q[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        q[0] += tv[k];
        if (L::cx(k)) q[1] += T(L::cx(k)) * tv[k];
        if (L::cy(k)) q[2] += T(L::cy(k)) * tv[k];
        if (L::D == 3 && L::cz(k)) q[3] += T(L::cz(k)) * tv[k];
    }
#pragma unroll
    for (int c = 0; c <= L::D; ++c) pf[c * sites + i] = (S)q[c];
}

// Start of a physical step: h_q from the accepted moment histories (Eq. bdf2) and the trial
// populations from the population-history extrapolation (Section 3.1) into the working slot
// (and, with pfbase, their moments P f into the slot's P f field).
template <class L, typename T, typename S = T>
__device__ __forceinline__ void step_begin_range(const DevState* __restrict__ st, S* __restrict__ fbase,
                                                 size_t fstride, const double* __restrict__ mbuf,
                                                 T* __restrict__ h, size_t sites, size_t i0, size_t istride,
                                                 S* __restrict__ pfbase = nullptr, size_t pfstride = 0) {
    const DevState* vs = st;
    if (vs->prepared) return;  // formed by the previous step's k_step_end
    if (!vs->params_ok || vs->steps_target <= 0 || vs->status != MSC_OK) return;  // no step runs
    const int q = vs->q;
    const double dt = vs->dt;
    const int nav = vs->n_avail < vs->warm_order ? vs->n_avail : vs->warm_order;
    const size_t mstride = (size_t)(L::D + 1) * sites;
    const double* mn = mbuf + (size_t)vs->m_cur * mstride;
    const double* mnm1 = mbuf + (size_t)vs->m_prev * mstride;
    const S* f0 = fbase + (size_t)vs->slot_fn[0] * fstride;
    const S* f1 = fbase + (size_t)vs->slot_fn[1] * fstride;
    const S* f2 = fbase + (size_t)vs->slot_fn[2] * fstride;
    S* ft = fbase + (size_t)vs->slot_cur * fstride;
    S* pft = pfbase ? pfbase + (size_t)vs->slot_cur * pfstride : nullptr;
    const double c1 = vs->c1, c2 = vs->c2;
    const float af = narrow_f64(vs->a);  // the sweep's binary32 a_q
    const size_t lo_off = (size_t)(L::D + 1) * sites;
    (void)dt;
    const T sig = from_f64<T>(vs->fscale), isig = from_f64<T>(vs->isig);
    const double fc[4] = {0.0, vs->force[0], vs->force[1], vs->force[2]};
    for (size_t i = i0; i < sites; i += istride) {
#pragma unroll
        for (int c = 0; c <= L::D; ++c) {  // h = c1 m^n - c2 m^{n-1} + (0, F), as k_step_end forms it
            const size_t o = c * sites + i;
            bdf_history<T>(c1, mn[o], c2, mnm1[o], fc[c], af, q, h, o, lo_off);
        }
        if constexpr (L::D == 3) {
            if (pft) {  // the trial in the storage type and its moments
                T tv[L::Q];
#pragma unroll
                for (int k = 0; k < L::Q; ++k) {
                    const size_t o = k * sites + i;
                    const T v0 = ld_pop<T, S>(f0, o, sig);
                    tv[k] = nav == 1 ? v0
                                     : (nav == 2 ? T(2) * v0 - ld_pop<T, S>(f1, o, sig)
                                                 : T(3) * (v0 - ld_pop<T, S>(f1, o, sig)) + ld_pop<T, S>(f2, o, sig));
                    st_pop<T, S>(ft, o, tv[k], isig);
                }
                store_trial_moments<L, T, S>(pft, sites, i, tv);
                continue;
            }
        }
        if (nav == 1) {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) ft[k * sites + i] = f0[k * sites + i];
        } else if (nav == 2) {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) {
                const size_t o = k * sites + i;
                st_pop<T, S>(ft, o, T(2) * ld_pop<T, S>(f0, o, sig) - ld_pop<T, S>(f1, o, sig), isig);
            }
        } else {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) {
                const size_t o = k * sites + i;
                st_pop<T, S>(ft, o, T(3) * (ld_pop<T, S>(f0, o, sig) - ld_pop<T, S>(f1, o, sig)) +
                                        ld_pop<T, S>(f2, o, sig), isig);
            }
        }
    }
}

template <class L, typename T, typename S = T>
__global__ void k_step_begin(const DevState* __restrict__ st, S* __restrict__ fbase, size_t fstride,
                             const double* __restrict__ mbuf, T* __restrict__ h, size_t sites,
                             S* __restrict__ pfbase, size_t pfstride) {
    step_begin_range<L, T, S>(st, fbase, fstride, mbuf, h, sites, blockIdx.x * (size_t)blockDim.x + threadIdx.x,
                           (size_t)gridDim.x * blockDim.x, pfbase, pfstride);
}

// Acceptance: m^{n+1} = R_{q,h}(f^{n+1}) with the unrotated histories (Eq. macro-reconstruct),
// evaluated in FP64 (P f accumulated in the storage type) and written into the m^{n-1} slot
// (rotated by k_step_finish).  When another step of this march follows, the same pass also forms
// that step's BDF2 history term h = (4 m^{n+1} - m^n)/(2 dt) and its population warm start
// (2 f^{n+1} - f^n, or 3 f^{n+1} - 3 f^n + f^{n-1}; Section 3.1) into the free working slot, so
// that the next k_step_begin has nothing to do.
template <class L, typename T, typename S = T, bool FORCE = true>
__device__ __forceinline__ void step_end_range(const DevState* __restrict__ st, S* __restrict__ fbase,
                                               size_t fstride, double* __restrict__ mbuf, T* __restrict__ h,
                                               size_t sites, size_t i0, size_t istride, S* __restrict__ pfbase = nullptr,
                                               size_t pfstride = 0) {
    const DevState* vs = st;
    if (!vs->accepted || vs->steps_target <= 0) return;  // no accepted step of this march to finish
    const double inv = vs->inv_a;
    const size_t mstride = (size_t)(L::D + 1) * sites;
    const bool next = vs->status == MSC_OK && vs->steps_target > 1;
    int nav = vs->n_avail + 1 < 3 ? vs->n_avail + 1 : 3;  // accepted states after rotation
    if (nav > vs->warm_order) nav = vs->warm_order;
    if (!next) nav = 0;
    // the ring slots, the moment slots and h never overlap: no store below aliases a load
    const double* __restrict__ mn = mbuf + (size_t)vs->m_cur * mstride;
    double* __restrict__ mnm1 = mbuf + (size_t)vs->m_prev * mstride;
    const S* __restrict__ ft = fbase + (size_t)vs->slot_cur * fstride;
    const S* __restrict__ f0 = fbase + (size_t)vs->slot_fn[0] * fstride;
    const S* __restrict__ f1 = fbase + (size_t)vs->slot_fn[1] * fstride;
    S* __restrict__ trial = fbase + (size_t)vs->slot_nxt * fstride;
    S* __restrict__ ptrial = pfbase ? pfbase + (size_t)vs->slot_nxt * pfstride : nullptr;
    const T sig = from_f64<T>(vs->fscale), isig = from_f64<T>(vs->isig);
    const double n1 = vs->n1, n2 = vs->n2;  // BDF2 for the next step
    const float an = narrow_f64(vs->qa[1]);  // the next step's binary32 a_2, as its sweep will use it
    const size_t lo_off = (size_t)(L::D + 1) * sites;
    const double k1 = vs->k1, k2 = vs->k2;  // formed once per step (FP64 products are slow on B300)
    // body force: (0, F) joins h in the reconstruction and in the next step's h (FORCE = false: F = 0)
    const double fc[4] = {0.0, FORCE ? vs->force[0] : 0.0, FORCE ? vs->force[1] : 0.0, FORCE ? vs->force[2] : 0.0};
    const double kf[4] = {0.0, 0.5 * inv * fc[1], 0.5 * inv * fc[2], 0.5 * inv * fc[3]};
#pragma unroll 2
    for (size_t i = i0; i < sites; i += istride) {
        // every load of the site is issued before any arithmetic or store (one memory latency per site)
        T fv[L::Q], g0[L::Q], g1[L::Q];
        double mcv[L::D + 1], mpv[L::D + 1];
#pragma unroll
        for (int k = 0; k < L::Q; ++k) fv[k] = ld_pop<T, S>(ft, k * sites + i, sig);
        if (nav >= 2) {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) g0[k] = ld_pop<T, S>(f0, k * sites + i, sig);
        }
        if (nav == 3) {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) g1[k] = ld_pop<T, S>(f1, k * sites + i, sig);
        }
#pragma unroll
        for (int c = 0; c <= L::D; ++c) {
            mcv[c] = mn[c * sites + i];
            mpv[c] = mnm1[c * sites + i];
        }
        T mom[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const T v = fv[k];
            mom[0] += v;
            if (L::cx(k)) mom[1] += T(L::cx(k)) * v;
            if (L::cy(k)) mom[2] += T(L::cy(k)) * v;
            if (L::D == 3 && L::cz(k)) mom[3] += T(L::cz(k)) * v;
        }
#pragma unroll
        for (int c = 0; c <= L::D; ++c) {
            // m^{n+1} = (P f + h/2) inv with h = c1 m^n - c2 m^{n-1} + (0, F), constants folded (FP64)
            const size_t o = c * sites + i;
            const double mc = mcv[c];
            const double md = to_f64<T>(mom[c]);
            const double mnew = FORCE ? fma(k1, mc, fma(-k2, mpv[c], fma(inv, md, kf[c])))
                                      : fma(k1, mc, fma(-k2, mpv[c], inv * md));
            mnm1[o] = mnew;
            if (next) bdf_history<T>(n1, mnew, n2, mc, fc[c], an, 2, h, o, lo_off);
        }
        if constexpr (L::D == 3) {
            if (ptrial && nav >= 1) {
                T tv[L::Q];
#pragma unroll
                for (int k = 0; k < L::Q; ++k) {
                    tv[k] = nav == 1 ? fv[k] : (nav == 2 ? T(2) * fv[k] - g0[k] : T(3) * (fv[k] - g0[k]) + g1[k]);
                    st_pop<T, S>(trial, k * sites + i, tv[k], isig);
                }
                store_trial_moments<L, T, S>(ptrial, sites, i, tv);
                continue;
            }
        }
        if (nav == 1) {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) st_pop<T, S>(trial, k * sites + i, fv[k], isig);
        } else if (nav == 2) {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) st_pop<T, S>(trial, k * sites + i, T(2) * fv[k] - g0[k], isig);
        } else if (nav == 3) {
#pragma unroll
            for (int k = 0; k < L::Q; ++k) st_pop<T, S>(trial, k * sites + i, T(3) * (fv[k] - g0[k]) + g1[k], isig);
        }
    }
}

// FP32 storage: six blocks per SM (the FP64 history update keeps the FP64 pipe busy only with
// enough warps resident)
template <class L, typename T, typename S = T, bool FORCE = true>
__global__ void __launch_bounds__(kFieldThreads)
    k_step_end(const DevState* __restrict__ st, S* __restrict__ fbase, size_t fstride, double* __restrict__ mbuf,
               T* __restrict__ h, size_t sites, S* __restrict__ pfbase, size_t pfstride) {
    step_end_range<L, T, S, FORCE>(st, fbase, fstride, mbuf, h, sites, blockIdx.x * (size_t)blockDim.x + threadIdx.x,
                                   (size_t)gridDim.x * blockDim.x, pfbase, pfstride);
}

// FP64 coefficients of the closed-form Schur solve (Eq. schur) at every masked wavevector, for
// BDF1 (a = 1/dt) and BDF2 (a = 3/(2 dt)).  With dv = a + nu|k|^2 and D = a + cs^2 |k|^2 / dv the
// solve is dp = A rp - i B (k.rm), du = Dv rm - i Cc k dp, and the table stores
// (A, B, Cc, Dv) = (s/D, s/(D dv), cs^2/dv, s/dv) with s = 1/N_Omega folded in.  Mode index:
// 2D jx + (n/4+1) jyk, 3D jx + (n/4+1)(jyk + (n/2+1) jzk), with jyk = j_y + n/4, jzk = j_z + n/4.
__host__ __device__ inline size_t solve_modes(int dim, int n) {
    const size_t a = n / 4 + 1, b = n / 2 + 1;
    return dim == 2 ? a * b : a * b * b;
}

__device__ inline void solve_coefficients(double a, double nu, double k2, double scale, double* out) {
    const double cs2 = 1.0 / 3.0;
    const double dv = a + nu * k2;
    const double idv = 1.0 / dv;
    const double iD = 1.0 / (a + cs2 * k2 * idv);
    out[0] = iD * scale;
    out[1] = iD * idv * scale;
    out[2] = cs2 * idv;
    out[3] = idv * scale;
}

__global__ void k_solve_tables(double* coef, int dim, int n, double dt, double nu) {
    const size_t nm = solve_modes(dim, n);
    const int nx4 = n / 4 + 1, ny = n / 2 + 1;
    const double tpn = 6.283185307179586476925286766559 / (double)n;
    const double scale = dim == 2 ? 1.0 / ((double)n * n) : 1.0 / ((double)n * n * n);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < 2 * nm; t += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / nm) + 1;
        const size_t m = t - (size_t)(q - 1) * nm;
        const int jx = (int)(m % nx4);
        const size_t r = m / nx4;
        const int jy = (int)(r % ny) - n / 4;
        const int jz = dim == 3 ? (int)(r / ny) - n / 4 : 0;
        const double kx = tpn * jx, ky = tpn * jy, kz = tpn * jz;
        const double a = q == 1 ? 1.0 / dt : 3.0 / (2.0 * dt);
        solve_coefficients(a, nu, kx * kx + ky * ky + kz * kz, scale, coef + 4 * t);
    }
}

// m^n (the moment buffer the state names) into out, count = (d+1) sites values
__global__ void __launch_bounds__(kFieldThreads) k_copy_fields(const DevState* st, const double* mbuf,
                                                               double* __restrict__ out, size_t count) {
    const double* __restrict__ m = mbuf + (size_t)st->m_cur * count;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = m[i];
}

// ---- single-thread control kernels ------------------------------------------------------------

// the step constants of BDF order q = 1, 2 (Eq. bdf2), formed once per dt by tabulate_step_constants:
// a single-thread control kernel would otherwise run five FP64 divisions on every physical step
__device__ inline void tabulate_step_constants(DevState* st) {
    const double dt = st->dt;
    st->qa[0] = 1.0 / dt;
    st->qa[1] = 3.0 / (2.0 * dt);
    for (int i = 0; i < 2; ++i) st->qinv[i] = 1.0 / (1.0 + st->qa[i] / 2.0);
    st->qc1[0] = 1.0 / dt;
    st->qc1[1] = 4.0 / (2.0 * dt);
    st->qc2[0] = 0.0;
    st->qc2[1] = 1.0 / (2.0 * dt);
}

__device__ inline void set_step_constants(DevState* st) {
    const int i = st->q == 1 ? 0 : 1;
    st->a = st->qa[i];
    st->inv_a = st->qinv[i];
    st->c1 = st->qc1[i];
    st->c2 = st->qc2[i];
    st->k1 = 0.5 * st->c1 * st->inv_a;
    st->k2 = 0.5 * st->c2 * st->inv_a;
}

__global__ void k_set_params(DevState* st, msc_params p) {
    st->nu = p.nu;
    st->dt = p.dt;
    tabulate_step_constants(st);
    st->n1 = 4.0 / (2.0 * p.dt);
    st->n2 = 1.0 / (2.0 * p.dt);
    st->eps = p.eps;
    st->kmax = p.kmax;
    st->nmin = p.nmin;
    st->corrector = p.corrector;
    st->replay = p.replay;
    st->warm_order = p.warm_order;
    st->count_multiple = p.count_multiple;
    st->force[0] = p.force[0];
    st->force[1] = p.force[1];
    st->force[2] = p.force[2];
    st->omega_p = p.omega[0] > 0.0 ? p.omega[0] : 1.0;
    st->omega_m = p.omega[1] > 0.0 ? p.omega[1] : 1.0;
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
    st->prepared = 0;
    st->fscale = 1.0;
    st->isig = 1.0;
    st->fmax_bits = 0ull;
}

__device__ inline void set_target(DevState* st, int n_steps) {
    st->prepared = 0;
    st->steps_target = n_steps;
    st->steps_in_call = 0;
    st->inner_total = 0;
    st->hist_pos = 0;
    st->status = MSC_OK;
}

__global__ void k_set_target(DevState* st, int n_steps) { set_target(st, n_steps); }

// a march may run: parameters set (else MSC_ERR_STATE), steps left and no error recorded
__device__ inline bool arm_state(DevState* st) {
    if (!st->params_ok) {
        if (st->steps_target > 0) st->status = MSC_ERR_STATE;
        return false;
    }
    return st->steps_target > 0 && st->status == MSC_OK;
}

__device__ inline bool slot_in_history(const DevState* st, int s) {
    for (int i = 0; i < st->n_avail; ++i)
        if (st->slot_fn[i] == s) return true;
    return false;
}

// start of a physical step (BDF order, a_q, working slots) unless k_step_finish already did it
__device__ inline void step_setup(DevState* st) {
    if (st->prepared) return;
    st->q = st->steps_done == 0 ? 1 : 2;
    set_step_constants(st);
    st->iter = 0;
    st->accepted = 0;
    st->lift = 0;
    int picked = 0;
    for (int s = 0; s < kNumFBuf && picked < 2; ++s) {
        if (slot_in_history(st, s)) continue;
        if (picked == 0) st->slot_cur = s; else st->slot_nxt = s;
        ++picked;
    }
}

__global__ void k_step_setup(DevState* st, cudaGraphConditionalHandle h_iter, int cond) {
    step_setup(st);
    if (cond) cudaGraphSetConditional(h_iter, 1u);
}

// End of an accepted step: rotate the population and moment histories, count the step and, when
// another step of this call follows, set that step up (its h and trial were formed by k_step_end).
// Returns whether another step follows.
__device__ inline unsigned int step_finish(DevState* st, int* iters_out, int max_steps) {
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
    // the next step's trial was written into the old slot_nxt by k_step_end
    const int trial = st->slot_nxt;
    if (go) {
        st->q = 2;
        set_step_constants(st);
        st->iter = 0;
        st->accepted = 0;
        st->lift = 0;
        st->slot_cur = trial;
        for (int s = 0; s < kNumFBuf; ++s) {
            if (s == trial || slot_in_history(st, s)) continue;
            st->slot_nxt = s;
            break;
        }
        st->prepared = 1;
    } else {
        st->prepared = 0;
    }
    return go;
}

// the march graph's prologue: arm the step loop and set up its first step (k_step_begin follows)
__global__ void k_arm_setup(DevState* st, cudaGraphConditionalHandle h_step) {
    const bool go = arm_state(st);
    if (go) step_setup(st);
    cudaGraphSetConditional(h_step, go ? 1u : 0u);
}

__global__ void k_step_finish(DevState* st, int* iters_out, int max_steps,
                              cudaGraphConditionalHandle h_step, int cond) {
    const unsigned int go = step_finish(st, iters_out, max_steps);
    if (cond) cudaGraphSetConditional(h_step, go);
}

// the march graph's step end: the step loop's condition.  The second step of the graph's unrolled
// pair finds no live step when the first was the march's last, and leaves the condition as that
// step set it.
__global__ void k_step_finish_graph(DevState* st, int* iters_out, int max_steps, cudaGraphConditionalHandle h_step) {
    wait_for_predecessor();
    if (st->steps_target <= 0) return;
    const unsigned int go = step_finish(st, iters_out, max_steps);
    cudaGraphSetConditional(h_step, go);
}

// m^n = P f^n of the accepted slot into both moment slots (after an explicit march)
template <class L, typename T, typename S = T>
__device__ __forceinline__ void moments_state_range(const DevState* __restrict__ st, const S* __restrict__ fbase,
                                                    size_t fstride, double* __restrict__ mbuf, size_t sites,
                                                    size_t i0, size_t istride) {
    const DevState* vs = st;
    const S* f = fbase + (size_t)vs->slot_fn[0] * fstride;
    const size_t mstride = (size_t)(L::D + 1) * sites;
    const double sig = vs->fscale;
    double* m0 = mbuf + (size_t)vs->m_cur * mstride;
    double* m1 = mbuf + (size_t)vs->m_prev * mstride;
    for (size_t i = i0; i < sites; i += istride) {
        double mom[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
            const double v = ld_pop<double, S>(f, k * sites + i, sig);
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

template <class L, typename T, typename S = T>
__global__ void k_moments_state(const DevState* __restrict__ st, const S* __restrict__ fbase, size_t fstride,
                                double* __restrict__ mbuf, size_t sites) {
    moments_state_range<L, T, S>(st, fbase, fstride, mbuf, sites, blockIdx.x * (size_t)blockDim.x + threadIdx.x,
                              (size_t)gridDim.x * blockDim.x);
}

// explicit march bookkeeping: ping-pong between the accepted slot and one free slot; the
// counter holds the remaining iterations of the graph's unrolled loop body
__global__ void k_ex_setup(DevState* st, int loop_iters) {
    st->ex_a = st->slot_fn[0];
    st->ex_b = (st->slot_fn[0] + 1) % kNumFBuf;
    st->ex_loops_left = loop_iters;
}

__global__ void k_ex_arm(DevState* st, cudaGraphConditionalHandle h_ex) {
    cudaGraphSetConditional(h_ex, st->ex_loops_left > 0 ? 1u : 0u);
}

__device__ inline void ex_finish(DevState* st, int odd) {
    st->slot_fn[0] = odd ? st->ex_b : st->ex_a;
    int s1 = (st->slot_fn[0] + 1) % kNumFBuf;
    int s2 = (st->slot_fn[0] + 2) % kNumFBuf;
    st->slot_fn[1] = s1;
    st->slot_fn[2] = s2;
    st->n_avail = 1;
    st->steps_done = 0;
    st->m_cur = 0;
    st->m_prev = 1;
    st->prepared = 0;
}

__global__ void k_ex_finish(DevState* st, int odd) { ex_finish(st, odd); }

}  // namespace msc
