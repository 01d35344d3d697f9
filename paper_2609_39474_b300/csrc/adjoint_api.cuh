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

static_assert(sizeof(AdjArgs) <= kAdjArgBytes && sizeof(AdjStat) <= kAdjStatBytes && sizeof(AdjCtl) <= kAdjCtlBytes,
              "adjoint blocks fit their workspace slots");

AdjCtl* adj_ctl(msc_ctx* c) { return at<AdjCtl>(c, c->lay.adj); }
AdjArgs* adj_args(msc_ctx* c) { return at<AdjArgs>(c, c->lay.adj + kAdjCtlBytes); }
AdjStat* adj_stats(msc_ctx* c) { return at<AdjStat>(c, c->lay.adj + kAdjCtlBytes + MSC_ADJOINT_CHUNK * kAdjArgBytes); }

// argument block of the shadow-correction passes of the transposed solve (BDF order q)
template <typename T>
Spec2Args<T> adjoint_spec_args(msc_ctx* c, int q) {
    using C = typename Cplx<T>::type;
    const int n = c->desc.n;
    Spec2Args<T> S;
    memset(&S, 0, sizeof(S));
    S.pr = at<T>(c, c->lay.pr);
    S.spec = at<C>(c, c->lay.spec);
    S.dm = at<T>(c, c->lay.h);  // the inverse row pass adds rho and the correction to theta
    S.tw = at<C>(c, c->lay.tw);
    S.n = n;
    S.logn = c->logn;
    S.P = row_geometry(n, 3, n).P;
    S.G = 1;
    S.nf = 3;
    S.rows = n;
    S.kunit = 6.283185307179586476925286766559 / (double)n;
    S.nscale = 1.0 / ((double)n * n);
    S.st = nullptr;  // the table of this BDF order, computed for the context's dt and nu
    S.coef = at<double>(c, c->lay.coef) + (size_t)(q - 1) * 4 * solve_modes(2, n);
    return S;
}

// The transposed solve of one step as a graph with conditional nodes, so that its iteration runs
// without the host:
//   prepare (h_eff, theta = c, |c|)  ->  WHILE { sweep (rho, |rho|, decision) -> IF { forward row
//   FFTs, transposed column solve, inverse row FFTs with theta += rho + correction } }  ->  final
//   sweep (dL/dh)  ->  advance to the next step of the run.
// The arguments of the step come from the device-resident block AdjCtl::slot names, so one
// instantiated graph per BDF order serves every step and a run of steps needs no host round trip.
template <typename T>
int build_adjoint_graph(msc_ctx* c, int q, cudaGraphExec_t* out) {
    const int n = c->desc.n;
    const size_t sites = c->sites;
    cudaError_t err = cudaSuccess;
    const AdjArgs* args = adj_args(c);
    AdjStat* stats = adj_stats(c);
    AdjCtl* ctl = adj_ctl(c);
    T* theta = at<T>(c, c->lay.h);
    T* rho = at<T>(c, c->lay.pr);
    const int grid = adjoint_grid(sites);
    const RowGeom rg = row_geometry(n, 3, n);
    Spec2Args<T> S = adjoint_spec_args<T>(c, q);

    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h_loop, h_corr;
    if (cudaGraphConditionalHandleCreate(&h_loop, g, 0, 0) != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    int cond = 1;
    T* warm = at<T>(c, c->lay.adjw);
    void* a_prep[] = {(void*)&args, &stats, (void*)&ctl, &theta, &warm, &h_loop, &cond};
    cudaGraphNode_t prep = add_kernel(g, {}, (const void*)k_adj_prepare<T>, dim3(grid), dim3(kFieldThreads), 0, a_prep,
                                      &err);
    cudaGraph_t body;
    cudaGraphNode_t loop = add_cond(g, {prep}, h_loop, cudaGraphCondTypeWhile, &body, &err);
    if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    if (cudaGraphConditionalHandleCreate(&h_corr, body, 0, 0) != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    void* a_sw[] = {(void*)&args, &stats, (void*)&ctl, &theta, &rho, &warm, &h_loop, &h_corr, &cond};
    cudaGraphNode_t sw = add_kernel(body, {}, (const void*)k_adj_sweep<T, false>, dim3(grid), dim3(kFieldThreads), 0,
                                    a_sw, &err);
    cudaGraph_t corr;
    add_cond(body, {sw}, h_corr, cudaGraphCondTypeIf, &corr, &err);
    if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    void* a_sp[] = {&S};
    cudaGraphNode_t f1 = add_kernel(corr, {}, (const void*)k_rowfft_fwd<T>, dim3(rg.blocks), dim3(rg.threads),
                                    spec_row_smem<T>(n, rg.P), a_sp, &err);
    cudaGraphNode_t f2 = add_kernel(corr, {f1}, (const void*)k_colsolve_adjoint<T>, dim3(n / 4 + 1),
                                    dim3(spec2_col_threads(n)), spec2_col_smem<T>(n), a_sp, &err);
    add_kernel(corr, {f2}, (const void*)k_rowfft_inv_acc<T>, dim3(rg.blocks), dim3(rg.threads),
               spec_row_smem<T>(n, rg.P), a_sp, &err);
    void* a_fin[] = {(void*)&args, &stats, (void*)&ctl, &theta, &rho, &warm, &h_loop, &h_corr, &cond};
    cudaGraphNode_t fin = add_kernel(g, {loop}, (const void*)k_adj_sweep<T, true>, dim3(grid), dim3(kFieldThreads), 0,
                                     a_fin, &err);
    void* a_adv[] = {&stats, &ctl};
    add_kernel(g, {fin}, (const void*)k_adj_advance, dim3(1), dim3(1), 0, a_adv, &err);
    if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    cudaGraphExec_t x = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return MSC_ERR_CUDA;
    *out = x;
    return MSC_OK;
}

// the argument blocks of a run of at most MSC_ADJOINT_CHUNK steps, and the position reset to its
// first step, in one host-to-device copy
int upload_adjoint_run(msc_ctx* c, int count, const msc_adjoint_io* io, double* dforce, double eps, int kmax) {
    const size_t sites = c->sites;
    const double dt = c->params.dt;
    struct Upload {
        AdjCtl ctl;
        unsigned char pad[kAdjCtlBytes - sizeof(AdjCtl)];
        AdjArgs args[MSC_ADJOINT_CHUNK];
    } up;
    static_assert(offsetof(Upload, args) == kAdjCtlBytes, "upload image matches the workspace");
    memset(&up, 0, sizeof(up));
    for (int i = 0; i < count; ++i) {
        const int q = io[i].q;
        AdjArgs& A = up.args[i];
        A.m = io[i].m_new;
        A.m_cur = io[i].m_cur;
        A.m_prev = q == 2 ? io[i].m_prev : io[i].m_cur;
        A.mu = io[i].abar_new;
        // scratch: the context's working arrays (the forward state is reloaded before the next march)
        A.heff = at<double>(c, c->lay.mbuf);
        A.partial = A.heff + 3 * sites;
        A.counter = at<unsigned int>(c, c->lay.counter);
        A.abar_cur = io[i].abar_cur;
        A.abar_prev = q == 2 ? io[i].abar_prev : nullptr;
        A.dforce = dforce;
        A.a = q == 1 ? 1.0 / dt : 3.0 / (2.0 * dt);
        A.inv = 1.0 / (1.0 + A.a / 2.0);
        A.c1 = q == 1 ? 1.0 / dt : 4.0 / (2.0 * dt);
        A.c2 = q == 1 ? 0.0 : 1.0 / (2.0 * dt);
        A.f0 = c->params.force[0];
        A.f1 = c->params.force[1];
        A.eps = eps;
        A.kmax = kmax;
        A.n = c->desc.n;
        A.warm = io[i].warm ? 1 : 0;
    }
    // the image ends right after the last used argument block; a pageable source: the call
    // returns once the image is staged, so the stack copy may go
    const size_t bytes = kAdjCtlBytes + (size_t)count * sizeof(AdjArgs);
    CK(cudaMemcpyAsync(c->ws + c->lay.adj, &up, bytes, cudaMemcpyHostToDevice, c->stream));
    return MSC_OK;
}

// one run of at most MSC_ADJOINT_CHUNK steps: one upload, one graph launch per step, one read-back
template <typename T>
int run_adjoint_chunk(msc_ctx* c, int count, const msc_adjoint_io* io, double* dforce, double eps, int kmax,
                      AdjStat* hs) {
    int rc = upload_adjoint_run(c, count, io, dforce, eps, kmax);
    if (rc) return rc;
    for (int i = 0; i < count; ++i) CK(cudaGraphLaunch(c->x_adj[io[i].q - 1], c->stream));
    CK(cudaMemcpyAsync(hs, adj_stats(c), (size_t)count * sizeof(AdjStat), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MSC_OK;
}

// The same run with every kernel launched from the host and the loop decided on the host from the
// outcome block (one synchronisation per iteration): the kernels and their order are those of the
// graph, so the results are identical.  For profilers, which do not descend into conditional nodes.
template <typename T>
int run_adjoint_chunk_stepwise(msc_ctx* c, int count, const msc_adjoint_io* io, double* dforce, double eps,
                               int kmax, AdjStat* hs) {
    int rc = upload_adjoint_run(c, count, io, dforce, eps, kmax);
    if (rc) return rc;
    const int n = c->desc.n;
    const AdjArgs* args = adj_args(c);
    AdjStat* stats = adj_stats(c);
    AdjCtl* ctl = adj_ctl(c);
    T* theta = at<T>(c, c->lay.h);
    T* rho = at<T>(c, c->lay.pr);
    T* warm = at<T>(c, c->lay.adjw);
    const int grid = adjoint_grid(c->sites);
    const RowGeom rg = row_geometry(n, 3, n);
    const cudaGraphConditionalHandle none = 0;
    cudaStream_t s = c->stream;
    for (int i = 0; i < count; ++i) {
        const Spec2Args<T> S = adjoint_spec_args<T>(c, io[i].q);
        AdjStat h;
        k_adj_prepare<T><<<grid, kFieldThreads, 0, s>>>(args, stats, ctl, theta, warm, none, 0);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&h, stats + i, sizeof(AdjStat), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        bool more = h.status == MSC_OK && h.cnorm > 0.0;
        int it = 0;
        while (more) {
            k_adj_sweep<T, false><<<grid, kFieldThreads, 0, s>>>(args, stats, ctl, theta, rho, warm, none, none, 0);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(&h, stats + i, sizeof(AdjStat), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (h.it == it) break;  // converged, failed or at the limit: no correction
            it = h.it;
            k_rowfft_fwd<T><<<rg.blocks, rg.threads, spec_row_smem<T>(n, rg.P), s>>>(S);
            k_colsolve_adjoint<T><<<n / 4 + 1, spec2_col_threads(n), spec2_col_smem<T>(n), s>>>(S);
            k_rowfft_inv_acc<T><<<rg.blocks, rg.threads, spec_row_smem<T>(n, rg.P), s>>>(S);
            CK(cudaGetLastError());
        }
        k_adj_sweep<T, true><<<grid, kFieldThreads, 0, s>>>(args, stats, ctl, theta, rho, warm, none, none, 0);
        k_adj_advance<<<1, 1, 0, s>>>(stats, ctl);
        CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(hs, stats, (size_t)count * sizeof(AdjStat), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return MSC_OK;
}

template <typename T>
int run_adjoint_steps(msc_ctx* c, int count, const msc_adjoint_io* io, double* dforce, double eps, int kmax,
                      msc_adjoint_stats* out, bool stepwise) {
    int rc = set_smem_limits<T>(2, c->desc.n);
    if (rc) return rc;
    CK(cudaFuncSetAttribute(k_colsolve_adjoint<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)spec2_col_smem<T>(c->desc.n)));
    CK(cudaFuncSetAttribute(k_rowfft_inv_acc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)spec_row_smem<T>(c->desc.n, row_geometry(c->desc.n, 3, c->desc.n).P)));
    rc = refresh_tables(c);
    if (rc) return rc;
    for (int q = 1; q <= 2; ++q) {
        bool used = false;
        for (int i = 0; i < count; ++i) used |= io[i].q == q;
        if (used && !stepwise && !c->x_adj[q - 1]) {
            rc = build_adjoint_graph<T>(c, q, &c->x_adj[q - 1]);
            if (rc) return rc;
        }
    }
    int first_fail = MSC_OK;
    AdjStat hs[MSC_ADJOINT_CHUNK];
    for (int i0 = 0; i0 < count; i0 += MSC_ADJOINT_CHUNK) {
        const int m = count - i0 < MSC_ADJOINT_CHUNK ? count - i0 : MSC_ADJOINT_CHUNK;
        if (first_fail == MSC_OK) {
            rc = stepwise ? run_adjoint_chunk_stepwise<T>(c, m, io + i0, dforce, eps, kmax, hs)
                          : run_adjoint_chunk<T>(c, m, io + i0, dforce, eps, kmax, hs);
            if (rc) return rc;
        } else {
            for (int i = 0; i < m; ++i) hs[i] = AdjStat{0.0, 0.0, 0, MSC_ERR_STATE};
        }
        for (int i = 0; i < m; ++i) {
            if (first_fail == MSC_OK && hs[i].status != MSC_OK) first_fail = hs[i].status;
            if (out) {
                out[i0 + i].iters = hs[i].it;
                out[i0 + i].status = hs[i].status;
                out[i0 + i].residual = hs[i].rel;
            }
        }
    }
    return first_fail;
}

}  // namespace

extern "C" {

static int adjoint_steps_entry(msc_ctx* c, int count, const msc_adjoint_io* io, double* dforce, double eps, int kmax,
                               msc_adjoint_stats* out, bool stepwise) {
    if (!c || count < 0 || (count > 0 && !io) || !dforce || !(eps > 0.0) || kmax < 0) return MSC_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        const msc_adjoint_io& s = io[i];
        if ((s.q != 1 && s.q != 2) || !s.m_new || !s.m_cur || !s.abar_new || !s.abar_cur) return MSC_ERR_ARG;
        if (s.q == 2 && (!s.m_prev || !s.abar_prev)) return MSC_ERR_ARG;
    }
    if (c->desc.dim != 2) return MSC_ERR_ARG;
    if (!c->params_set) return MSC_ERR_STATE;
    if (ctx_trt(c)) return MSC_ERR_ARG;  // the adjoint differentiates the operating-point collision
    if (count == 0) return MSC_OK;
    if (c->desc.precision == MSC_FP64) return run_adjoint_steps<double>(c, count, io, dforce, eps, kmax, out, stepwise);
    return run_adjoint_steps<float>(c, count, io, dforce, eps, kmax, out, stepwise);
}

int msc_adjoint_steps(msc_ctx* c, int count, const msc_adjoint_io* io, double* dforce, double eps, int kmax,
                      msc_adjoint_stats* out) {
    return adjoint_steps_entry(c, count, io, dforce, eps, kmax, out, false);
}

int msc_adjoint_steps_stepwise(msc_ctx* c, int count, const msc_adjoint_io* io, double* dforce, double eps,
                               int kmax, msc_adjoint_stats* out) {
    return adjoint_steps_entry(c, count, io, dforce, eps, kmax, out, true);
}

int msc_adjoint_step(msc_ctx* c, int q, const double* m_new, const double* m_cur, const double* m_prev,
                     const double* abar_new, double* abar_cur, double* abar_prev, double* dforce, double eps,
                     int kmax, msc_adjoint_stats* out) {
    const msc_adjoint_io s = {q, m_new, m_cur, m_prev, abar_new, abar_cur, abar_prev, 0};
    return msc_adjoint_steps(c, 1, &s, dforce, eps, kmax, out);
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
