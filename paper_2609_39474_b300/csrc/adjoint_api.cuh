// C ABI of the discrete adjoint (kernels in adjoint2d.cuh) and of device-resident state blobs.
// Included at the end of msclbm.cu (it uses that file's context internals).
#pragma once

#include "adjoint2d.cuh"

namespace {

int adjoint_grid(size_t sites) {
    size_t b = (sites + kFieldThreads - 1) / kFieldThreads;
    if (b > 148 * 8) b = 148 * 8;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
int run_adjoint_step(msc_ctx* c, int q, const double* m_new, const double* m_cur, const double* m_prev,
                     const double* abar_new, double* abar_cur, double* abar_prev, double* dforce, double eps,
                     int kmax, msc_adjoint_stats* out) {
    using C = typename Cplx<T>::type;
    const int n = c->desc.n;
    const size_t sites = c->sites;
    const double dt = c->params.dt;
    AdjArgs A;
    memset(&A, 0, sizeof(A));
    A.m = m_new;
    A.mu = abar_new;
    A.abar_cur = abar_cur;
    A.abar_prev = abar_prev;
    A.dforce = dforce;
    A.a = q == 1 ? 1.0 / dt : 3.0 / (2.0 * dt);
    A.inv = 1.0 / (1.0 + A.a / 2.0);
    A.c1 = q == 1 ? 1.0 / dt : 4.0 / (2.0 * dt);
    A.c2 = q == 1 ? 0.0 : 1.0 / (2.0 * dt);
    A.n = n;
    // scratch: the context's working arrays (the forward state is reloaded before the next march)
    double* heff = at<double>(c, c->lay.mbuf);
    A.heff = heff;
    A.partial = heff + 3 * sites;
    A.counter = at<unsigned int>(c, c->lay.counter);
    A.out = reinterpret_cast<double*>(c->ws + c->lay.counter + 64);
    T* theta = at<T>(c, c->lay.h);
    T* rho = at<T>(c, c->lay.pr);
    T* delta = at<T>(c, c->lay.dm);
    const int grid = adjoint_grid(sites);
    int rc = set_smem_limits<T>(2, n);
    if (rc) return rc;
    const RowGeom rg = row_geometry(n, 3, n);
    Spec2Args<T> S;
    memset(&S, 0, sizeof(S));
    S.pr = rho;
    S.spec = at<C>(c, c->lay.spec);
    S.dm = delta;
    S.tw = at<C>(c, c->lay.tw);
    S.n = n;
    S.logn = c->logn;
    S.P = rg.P;
    S.G = 1;
    S.nf = 3;
    S.rows = n;
    S.a = A.a;
    S.nu = c->params.nu;
    S.kunit = 6.283185307179586476925286766559 / (double)n;
    S.nscale = 1.0 / ((double)n * n);
    k_adj_prepare<T><<<grid, kFieldThreads, 0, c->stream>>>(A, m_cur, m_prev ? m_prev : m_cur, c->params.force[0],
                                                             c->params.force[1], heff, theta);
    CK(cudaGetLastError());
    double host[2];
    CK(cudaMemcpyAsync(host, A.out, 16, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double cnorm = sqrt(host[0] / (3.0 * (double)sites));
    int it = 0, status = MSC_OK;
    double rel = 0.0;
    if (cnorm > 0.0) {
        for (;;) {
            k_adj_sweep<T, false><<<grid, kFieldThreads, 0, c->stream>>>(A, theta, rho);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(host, A.out, 16, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            rel = sqrt(host[0] / (3.0 * (double)sites)) / cnorm;
            if (!std::isfinite(rel)) { status = MSC_ERR_NONFINITE; break; }
            if (rel < eps) break;
            if (it >= kmax) { status = MSC_ERR_NONCONVERGED; break; }
            ++it;
            k_rowfft_fwd<T><<<rg.blocks, rg.threads, spec_row_smem<T>(n, rg.P), c->stream>>>(S);
            k_colsolve_adjoint<T><<<n / 4 + 1, spec2_col_threads(n), spec2_col_smem<T>(n), c->stream>>>(S);
            k_rowfft_inv<T><<<rg.blocks, rg.threads, spec_row_smem<T>(n, rg.P), c->stream>>>(S);
            k_adj_update<T><<<grid, kFieldThreads, 0, c->stream>>>(theta, rho, delta, 3 * sites);
            CK(cudaGetLastError());
        }
    }
    if (status == MSC_OK) {
        k_adj_sweep<T, true><<<grid, kFieldThreads, 0, c->stream>>>(A, theta, rho);
        CK(cudaGetLastError());
    }
    if (out) {
        out->iters = it;
        out->status = status;
        out->residual = rel;
    }
    return status == MSC_OK ? MSC_OK : status;
}

}  // namespace

extern "C" {

int msc_adjoint_step(msc_ctx* c, int q, const double* m_new, const double* m_cur, const double* m_prev,
                     const double* abar_new, double* abar_cur, double* abar_prev, double* dforce, double eps,
                     int kmax, msc_adjoint_stats* out) {
    if (!c || (q != 1 && q != 2) || !m_new || !m_cur || !abar_new || !abar_cur || !dforce || !(eps > 0.0) ||
        kmax < 0)
        return MSC_ERR_ARG;
    if (q == 2 && (!m_prev || !abar_prev)) return MSC_ERR_ARG;
    if (c->desc.dim != 2) return MSC_ERR_ARG;
    if (!c->params_set) return MSC_ERR_STATE;
    if (ctx_trt(c)) return MSC_ERR_ARG;  // the adjoint differentiates the operating-point collision
    if (c->desc.precision == MSC_FP64)
        return run_adjoint_step<double>(c, q, m_new, m_cur, m_prev, abar_new, abar_cur, abar_prev, dforce, eps,
                                        kmax, out);
    return run_adjoint_step<float>(c, q, m_new, m_cur, m_prev, abar_new, abar_cur, abar_prev, dforce, eps, kmax,
                                   out);
}

// device-resident state blobs: the layout of msc_save_state, in device memory
int msc_save_state_device(msc_ctx* c, void* blob, size_t* bytes) {
    if (!c || !bytes) return MSC_ERR_ARG;
    DevState s;
    int rc = read_state(c, &s);
    if (rc) return rc;
    const size_t F = c->desc.dim + 1;
    const size_t need = 32 + (size_t)s.n_avail * c->lay.fstride + 2 * F * c->sites * 8;
    if (!blob) {
        *bytes = need;
        return MSC_OK;
    }
    if (*bytes < need) return MSC_ERR_ARG;
    int sig_exp = 0;
    frexp(s.fscale > 0.0 ? s.fscale : 1.0, &sig_exp);
    int32_t hdr[6] = {0x4d53434c, c->desc.dim, c->desc.n, c->desc.precision, s.n_avail, sig_exp - 1};
    unsigned char h[32];
    memcpy(h, hdr, 24);
    int64_t sd = s.steps_done;
    memcpy(h + 24, &sd, 8);
    unsigned char* b = (unsigned char*)blob;
    CK(cudaMemcpyAsync(b, h, 32, cudaMemcpyHostToDevice, c->stream));
    size_t o = 32;
    for (int i = 0; i < s.n_avail; ++i) {
        CK(cudaMemcpyAsync(b + o, c->ws + c->lay.fbuf + (size_t)s.slot_fn[i] * c->lay.fstride, c->lay.fstride,
                           cudaMemcpyDeviceToDevice, c->stream));
        o += c->lay.fstride;
    }
    const double* mb = at<double>(c, c->lay.mbuf);
    CK(cudaMemcpyAsync(b + o, mb + (size_t)s.m_cur * F * c->sites, F * c->sites * 8, cudaMemcpyDeviceToDevice,
                       c->stream));
    o += F * c->sites * 8;
    CK(cudaMemcpyAsync(b + o, mb + (size_t)s.m_prev * F * c->sites, F * c->sites * 8, cudaMemcpyDeviceToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));  // the header staging buffer is on the host stack
    *bytes = need;
    return MSC_OK;
}

int msc_load_state_device(msc_ctx* c, const void* blob, size_t bytes) {
    if (!c || !blob || bytes < 32) return MSC_ERR_ARG;
    const unsigned char* b = (const unsigned char*)blob;
    unsigned char h[32];
    CK(cudaMemcpyAsync(h, b, 32, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int32_t hdr[6];
    memcpy(hdr, h, 24);
    if (hdr[0] != 0x4d53434c || hdr[1] != c->desc.dim || hdr[2] != c->desc.n || hdr[3] != c->desc.precision ||
        hdr[4] < 1 || hdr[4] > 3 || hdr[5] < -1000 || hdr[5] > 1000)
        return MSC_ERR_ARG;
    int64_t sd;
    memcpy(&sd, h + 24, 8);
    const size_t F = c->desc.dim + 1;
    const size_t need = 32 + (size_t)hdr[4] * c->lay.fstride + 2 * F * c->sites * 8;
    if (bytes < need) return MSC_ERR_ARG;
    DevState s;
    int rc = read_state(c, &s);
    if (rc) return rc;
    size_t o = 32;
    for (int i = 0; i < hdr[4]; ++i) {
        CK(cudaMemcpyAsync(c->ws + c->lay.fbuf + (size_t)i * c->lay.fstride, b + o, c->lay.fstride,
                           cudaMemcpyDeviceToDevice, c->stream));
        o += c->lay.fstride;
    }
    double* mb = at<double>(c, c->lay.mbuf);
    CK(cudaMemcpyAsync(mb, b + o, F * c->sites * 8, cudaMemcpyDeviceToDevice, c->stream));
    o += F * c->sites * 8;
    CK(cudaMemcpyAsync(mb + F * c->sites, b + o, F * c->sites * 8, cudaMemcpyDeviceToDevice, c->stream));
    s.n_avail = hdr[4];
    s.slot_fn[0] = 0;
    s.slot_fn[1] = 1;
    s.slot_fn[2] = 2;
    s.m_cur = 0;
    s.m_prev = 1;
    s.steps_done = sd;
    s.status = MSC_OK;
    s.prepared = 0;
    s.fscale = ldexp(1.0, hdr[5]);
    s.isig = 1.0 / s.fscale;
    CK(cudaMemcpyAsync(c->ws + c->lay.state, &s, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->fields_set = true;
    return MSC_OK;
}

}  // extern "C"

// ---- self-check of the integer-pipe format conversions against the hardware conversions ---------
namespace {
__device__ unsigned int conv_mix(unsigned long long& s) {  // splitmix64 step, high half
    s += 0x9e3779b97f4a7c15ull;
    unsigned long long z = s;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (unsigned int)((z ^ (z >> 31)) >> 32);
}
__global__ void k_conversion_check(unsigned long long seed, int per_thread, unsigned int* bad) {
    unsigned long long s = seed ^ (0x5851f42d4c957f2dull * (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x));
    unsigned int nbad = 0;
    for (int i = 0; i < per_thread; ++i) {
        // random binary32 patterns (every exponent) and random binary64 patterns near the binary32 range
        const unsigned int fb = conv_mix(s);
        const float f = __uint_as_float(fb);
        const double w = widen_f32(f), wr = (double)f;
        if (!(w == wr || (w != w && wr != wr)) || (w == wr && __double_as_longlong(w) != __double_as_longlong(wr))) ++nbad;
        const unsigned long long hi = conv_mix(s), lo = conv_mix(s);
        unsigned long long db = (hi << 32) | lo;
        const unsigned long long ex = 880ull + (hi % 290ull);  // exponents 880 .. 1169 around the range
        db = (db & 0x800fffffffffffffull) | (ex << 52);
        if ((i & 7) == 0) db = (db & ~0x1fffffffull) | ((i & 8) ? 0x10000000ull : 0x0fffffffull);  // ties, near ties
        const double d = __longlong_as_double((long long)db);
        const float n = narrow_f64(d), nr = __double2float_rn(d);
        if (__float_as_uint(n) != __float_as_uint(nr)) ++nbad;
    }
    if (nbad) atomicAdd(bad, nbad);
}
}  // namespace

extern "C" int msc_selftest_conversions(int blocks, int per_thread, unsigned long long seed, int* mismatches) {
    if (blocks < 1 || per_thread < 1 || !mismatches) return MSC_ERR_ARG;
    unsigned int* d = nullptr;
    CK(cudaMalloc(&d, sizeof(unsigned int)));
    unsigned int h = 0;
    if (cudaMemset(d, 0, sizeof(unsigned int)) != cudaSuccess) { cudaFree(d); return MSC_ERR_CUDA; }
    k_conversion_check<<<blocks, 256>>>(seed, per_thread, d);
    const bool ok = cudaGetLastError() == cudaSuccess &&
                    cudaMemcpy(&h, d, sizeof(unsigned int), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(d);
    if (!ok) return MSC_ERR_CUDA;
    *mismatches = (int)h;
    return MSC_OK;
}
