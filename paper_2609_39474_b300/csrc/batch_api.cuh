// C ABI of the batched D2Q9 march (kernels in batch2d.cuh): batch construction, tiling, the
// batch graphs and the autotuner.  Included at the end of msclbm.cu (it uses that file's context
// internals and graph helpers).
#pragma once

#include <algorithm>

#include "batch2d.cuh"

struct msc_batch {
    int n_inst, precision;
    msc_ctx* ctx[kBatchMax];  // batch order: n descending, caller order within one n
    int perm[kBatchMax];      // batch index -> caller index
    int cls[kBatchMax];       // batch index -> size class
    cudaStream_t stream;
    unsigned char* ws;
    size_t off_inst, off_map, off_act, off_upart, off_ucount, off_tsum;
    msc_batch_tuning tun;
    // launch geometry derived from the tiling; fld_grid: the field kernels' strided grid (at most one
    // resident wave, and no more blocks than the whole batch has field blocks)
    int sweep_grid, row_blocks, row_threads, col_blocks, col_threads, fld_blocks;
    int fld_grid;
    size_t row_smem, col_smem;
    BMap map;  // host copy of the uploaded prefix tables
    bool graph_force;  // the march graph's step end carries the body-force terms
    cudaGraph_t g_march;
    cudaGraphExec_t x_march;
    cudaGraph_t g_ex;
    cudaGraphExec_t x_ex;
};

namespace {

constexpr int kBatchExUnroll = 8;  // explicit steps per round of the batched explicit graph (even)
constexpr int kHbChoices[] = {4, 8, 16, 32, 64};

size_t binst_bytes() { return std::max(sizeof(BInst<double>), sizeof(BInst<float>)); }

int max_units(int n) { return ((n + kStripOut - 1) / kStripOut) * (n / 4); }  // sweep_rows = 4

bool batch_list_ok(msc_ctx* const* ctxs, int n_inst, int* n_classes) {
    if (!ctxs || n_inst < 1 || n_inst > kBatchMax) return false;
    int sizes[kBatchMax];
    int ns = 0;
    for (int i = 0; i < n_inst; ++i) {
        const msc_ctx* c = ctxs[i];
        if (!c || c->desc.dim != 2 || c->desc.precision != ctxs[0]->desc.precision) return false;
        if (c->desc.precision == MSC_FP16) return false;  // batches hold FP32 or FP64 storage
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return false;  // one context once
        bool seen = false;
        for (int k = 0; k < ns; ++k) seen |= sizes[k] == c->desc.n;
        if (!seen) sizes[ns++] = c->desc.n;
    }
    if (ns > MSC_BATCH_CLASSES) return false;
    if (n_classes) *n_classes = ns;
    return true;
}

struct BatchOffsets {
    size_t inst, map, act, upart, ucount, tsum, total;
};

BatchOffsets batch_offsets(msc_ctx* const* ctxs, int n_inst) {
    BatchOffsets o;
    size_t p = 0;
    auto take = [&](size_t bytes) {
        const size_t r = p;
        p = align_up(p + bytes, 256);
        return r;
    };
    size_t units = 0;
    for (int i = 0; i < n_inst; ++i) units += max_units(ctxs[i]->desc.n);
    o.inst = take((size_t)n_inst * binst_bytes());
    o.map = take(sizeof(BMap));
    o.act = take(sizeof(BAct));
    o.upart = take(units * sizeof(double));
    o.ucount = take((size_t)n_inst * 32);
    o.tsum = take((size_t)n_inst * sizeof(double));
    o.total = p;
    return o;
}

int col_thread_cap(int precision) { return precision == MSC_FP64 ? 384 : 768; }

// points per thread of a transform line: 16 in the radix-16 form, 4 in the radix-4 form that the
// single-lattice correction uses at n <= kSpec2Radix4Max (the batch follows it, so that its results
// stay those of the single march bit for bit)
int fft_pts(int n) { return spec2_radix4(n) ? 4 : 16; }

bool tuning_ok(const msc_batch* b, const msc_batch_tuning* t) {
    if (t->n_classes != b->tun.n_classes) return false;
    if (t->sweep_ctas_per_sm < 1 || t->sweep_ctas_per_sm > 16) return false;
    for (int c = 0; c < t->n_classes; ++c) {
        const int n = b->tun.n[c];
        if (t->n[c] != n) return false;
        const int hb = t->sweep_rows[c], P = t->fft_rows[c], G = t->col_lines[c];
        bool hb_ok = false;
        for (int h : kHbChoices) hb_ok |= h == hb;
        if (!hb_ok || hb > n) return false;
        if (!is_pow2(P) || P > n / 2 || P * n / fft_pts(n) > kFftThreads) return false;
        if (!is_pow2(G) || G > 64 || 3 * G * n / fft_pts(n) > col_thread_cap(b->precision)) return false;
    }
    return true;
}

// default tiling: the single-context geometry of each size
void default_tuning(msc_batch* b) {
    msc_batch_tuning& t = b->tun;
    for (int c = 0; c < t.n_classes; ++c) {
        const int n = t.n[c];
        t.sweep_rows[c] = sweep2_geometry(n, 4).hb;  // the batch's unit tables assume >= 4 rows per unit
        t.fft_rows[c] = spec2_radix4(n) ? row_geometry_n4(n).P : row_geometry(n, 3, n).P;
        t.col_lines[c] = 1;
    }
    t.sweep_ctas_per_sm = 4;
    t.sweep_us = t.rowfft_us = t.colsolve_us = 0.f;
}

template <typename T>
BInst<T> make_inst(msc_batch* b, int i, double* upart, unsigned int* ucount, double* tsum) {
    msc_ctx* c = b->ctx[i];
    using C = typename Cplx<T>::type;
    const int cl = b->cls[i];
    const int n = c->desc.n;
    BInst<T> B;
    memset(&B, 0, sizeof(B));
    B.sw = sweep2_args_graph<T>(c);
    B.sw.hb = b->tun.sweep_rows[cl];
    B.sw.nrowblk = n / B.sw.hb;
    B.sw.a = c->params_set ? 3.0 / (2.0 * c->params.dt) : 1.0;
    B.sw.inv = 1.0 / (1.0 + B.sw.a / 2.0);
    B.sp = spec3_args<T>(n, c->logn, B.sw.a, c->params_set ? c->params.nu : 1.0 / 6.0, at<T>(c, c->lay.pr),
                         at<C>(c, c->lay.spec), at<T>(c, c->lay.dm), at<C>(c, c->lay.tw), at<DevState>(c, c->lay.state),
                         at<double>(c, c->lay.coef));
    B.sp.nf = 3;
    B.sp.rows = n;
    B.sp.nscale = 1.0 / ((double)n * n);
    B.sp.P = b->tun.fft_rows[cl];
    B.sp.G = b->tun.col_lines[cl];
    B.st = at<DevState>(c, c->lay.state);
    B.fbase = at<T>(c, c->lay.fbuf);
    B.fstride = c->lay.fstride / sizeof(T);
    B.mbuf = at<double>(c, c->lay.mbuf);
    B.h = at<T>(c, c->lay.h);
    B.sites = c->sites;
    B.iters = at<int>(c, c->lay.iters);
    B.max_steps = c->desc.max_steps;
    B.units = B.sw.nstrips * B.sw.nrowblk;
    B.upart = upart;
    B.ucount = ucount;
    B.t_sumsq = tsum;
    return B;
}

// Derive the launch geometry from the tiling and upload the per-instance arguments and prefix
// tables.  t_slots (optional): per instance the (input, output) ring slots of the tuning sweep.
template <typename T>
int upload_batch(msc_batch* b, const int (*t_slots)[2] = nullptr) {
    using C = typename Cplx<T>::type;
    BInst<T> I[kBatchMax];
    BMap& M = b->map;
    memset(&M, 0, sizeof(M));
    M.n_inst = b->n_inst;
    double* upart = reinterpret_cast<double*>(b->ws + b->off_upart);
    int rth = 32, cth = 32;
    size_t rsm = 0, csm = 0;
    for (int i = 0; i < b->n_inst; ++i) {
        msc_ctx* c = b->ctx[i];
        const int n = c->desc.n, cl = b->cls[i];
        I[i] = make_inst<T>(b, i, upart, reinterpret_cast<unsigned int*>(b->ws + b->off_ucount + 32 * i),
                            reinterpret_cast<double*>(b->ws + b->off_tsum) + i);
        upart += max_units(n);
        if (t_slots) {
            I[i].t_fin = I[i].fbase + (size_t)t_slots[i][0] * I[i].fstride;
            I[i].t_fout = I[i].fbase + (size_t)t_slots[i][1] * I[i].fstride;
        }
        const int P = b->tun.fft_rows[cl], G = b->tun.col_lines[cl];
        const int nx4 = n / 4 + 1;
        M.unit_off[i + 1] = M.unit_off[i] + I[i].units;
        M.row_off[i + 1] = M.row_off[i] + 3 * (n / 2) / P;
        M.col_off[i + 1] = M.col_off[i] + (nx4 + G - 1) / G;
        size_t fb = (c->sites + 4 * kFieldThreads - 1) / (4 * kFieldThreads);
        M.fld_off[i + 1] = M.fld_off[i] + (int)(fb < 1 ? 1 : fb);
        M.col_g[i] = G;
        M.st[i] = I[i].st;
        M.iters[i] = I[i].iters;
        M.max_steps[i] = I[i].max_steps;
        rth = std::max(rth, (P * n / fft_pts(n) + 31) / 32 * 32);
        cth = std::max(cth, (3 * G * n / fft_pts(n) + 31) / 32 * 32);
        rsm = std::max(rsm, (size_t)P * padded_len(n) * sizeof(C));
        csm = std::max(csm, (size_t)3 * G * padded_len(n) * sizeof(C));
    }
    b->row_blocks = M.row_off[b->n_inst];
    b->col_blocks = M.col_off[b->n_inst];
    b->fld_blocks = M.fld_off[b->n_inst];
    b->row_threads = rth;
    b->col_threads = cth;
    b->row_smem = rsm;
    b->col_smem = csm;
    const int units = M.unit_off[b->n_inst];
    int grid = 148 * b->tun.sweep_ctas_per_sm;
    const int need = (units + kSweepWarps - 1) / kSweepWarps;
    b->sweep_grid = grid < need ? grid : need;
    CK(cudaFuncSetAttribute(k_browfft<T, false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    CK(cudaFuncSetAttribute(k_browfft<T, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    CK(cudaFuncSetAttribute(k_browfft<T, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    CK(cudaFuncSetAttribute(k_browfft<T, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    CK(cudaFuncSetAttribute(k_bcolsolve<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
    CK(cudaFuncSetAttribute(k_bcolsolve<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
    {  // the field kernels' strided grid: one resident wave (the march's rounds walk the compacted list)
        int occ = 0, dev = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bstep_end<T, false>, kFieldThreads, 0) !=
                cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return MSC_ERR_CUDA;
        const int cap = (occ < 1 ? 1 : occ) * sms;
        b->fld_grid = b->fld_blocks < cap ? b->fld_blocks : cap;
    }
    CK(cudaMemcpyAsync(b->ws + b->off_inst, I, (size_t)b->n_inst * sizeof(BInst<T>), cudaMemcpyHostToDevice,
                       b->stream));
    CK(cudaMemcpyAsync(b->ws + b->off_map, &M, sizeof(BMap), cudaMemcpyHostToDevice, b->stream));
    // the sources are host stack memory: finish the copies before they go out of scope
    CK(cudaStreamSynchronize(b->stream));
    return MSC_OK;
}

void drop_batch_graphs(msc_batch* b) {
    if (b->x_march) cudaGraphExecDestroy(b->x_march);
    if (b->g_march) cudaGraphDestroy(b->g_march);
    if (b->x_ex) cudaGraphExecDestroy(b->x_ex);
    if (b->g_ex) cudaGraphDestroy(b->g_ex);
    b->x_march = nullptr;
    b->g_march = nullptr;
    b->x_ex = nullptr;
    b->g_ex = nullptr;
}

template <typename T>
int build_batch_march_graph(msc_batch* b) {
    cudaError_t err = cudaSuccess;
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    const BInst<T>* I = reinterpret_cast<const BInst<T>*>(b->ws + b->off_inst);
    const BMap* M = reinterpret_cast<const BMap*>(b->ws + b->off_map);
    BAct* W = reinterpret_cast<BAct*>(b->ws + b->off_act);
    int zero = 0;
    cudaGraphConditionalHandle h_round;
    CK(cudaGraphConditionalHandleCreate(&h_round, g, 0, 0));
    void* a_setup[] = {&M, &W, &h_round};
    cudaGraphNode_t setup = add_kernel(g, {}, (const void*)k_bsetup, dim3(1), dim3(kBatchMax), 0, a_setup, &err);
    void* a_fld[] = {&I, &M, &W};
    cudaGraphNode_t begin = add_kernel(g, {setup}, (const void*)k_bstep_begin<T>, dim3(b->fld_grid),
                                       dim3(kFieldThreads), 0, a_fld, &err);
    cudaGraph_t body;
    add_cond(g, {begin}, h_round, cudaGraphCondTypeWhile, &body, &err);
    if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    void* a_sw[] = {&I, &M, &W, &zero};
    cudaGraphNode_t sw = add_kernel(body, {}, (const void*)k_bsweep2<T, 0>, dim3(b->sweep_grid),
                                    dim3(kSweepWarps * 32), 0, a_sw, &err);
    void* a_sp[] = {&I, &M, &W};
    cudaGraphNode_t r1 = add_kernel(body, {sw}, (const void*)k_browfft<T, false, 0>, dim3(b->row_blocks),
                                    dim3(b->row_threads), b->row_smem, a_sp, &err);
    cudaGraphNode_t cs = add_kernel(body, {r1}, (const void*)k_bcolsolve<T, 0>, dim3(b->col_blocks),
                                    dim3(b->col_threads), b->col_smem, a_sp, &err);
    cudaGraphNode_t r2 = add_kernel(body, {cs}, (const void*)k_browfft<T, true, 0>, dim3(b->row_blocks),
                                    dim3(b->row_threads), b->row_smem, a_sp, &err);
    const void* fn_end = b->graph_force ? (const void*)k_bstep_end<T, true> : (const void*)k_bstep_end<T, false>;
    cudaGraphNode_t en = add_kernel(body, {r2}, fn_end, dim3(b->fld_grid),
                                    dim3(kFieldThreads), 0, a_fld, &err);
    void* a_fin[] = {&M, &W, &h_round};
    add_kernel(body, {en}, (const void*)k_bfinish, dim3(1), dim3(kBatchMax), 0, a_fin, &err);
    if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    cudaGraphExec_t x;
    if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    b->g_march = g;
    b->x_march = x;
    return MSC_OK;
}

template <typename T>
int build_batch_explicit_graph(msc_batch* b) {
    cudaError_t err = cudaSuccess;
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    const BInst<T>* I = reinterpret_cast<const BInst<T>*>(b->ws + b->off_inst);
    const BMap* M = reinterpret_cast<const BMap*>(b->ws + b->off_map);
    cudaGraphConditionalHandle h_ex;
    CK(cudaGraphConditionalHandleCreate(&h_ex, g, 0, 0));
    int zero = 0, unroll = kBatchExUnroll;
    void* a_arm[] = {&M, &zero, &h_ex};  // a count of 0 only evaluates the condition
    cudaGraphNode_t arm = add_kernel(g, {}, (const void*)k_bex_count, dim3(1), dim3(kBatchMax), 0, a_arm, &err);
    cudaGraph_t body;
    add_cond(g, {arm}, h_ex, cudaGraphCondTypeWhile, &body, &err);
    if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    int nodes[kBatchExUnroll];
    const BAct* no_list = nullptr;  // the explicit march walks every instance
    cudaGraphNode_t prev = nullptr;
    for (int i = 0; i < kBatchExUnroll; ++i) {
        nodes[i] = i;
        void* a_sw[] = {&I, &M, &no_list, &nodes[i]};
        std::vector<cudaGraphNode_t> deps;
        if (prev) deps.push_back(prev);
        prev = prev && kExplicitProgrammatic
                   ? add_kernel_after(body, prev, (const void*)k_bsweep2<T, 2>, dim3(b->sweep_grid),
                                      dim3(kSweepWarps * 32), 0, a_sw, &err)
                   : add_kernel(body, deps, (const void*)k_bsweep2<T, 2>, dim3(b->sweep_grid), dim3(kSweepWarps * 32),
                                0, a_sw, &err);
    }
    void* a_cnt[] = {&M, &unroll, &h_ex};
    add_kernel(body, {prev}, (const void*)k_bex_count, dim3(1), dim3(kBatchMax), 0, a_cnt, &err);
    if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    cudaGraphExec_t x;
    if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    b->g_ex = g;
    b->x_ex = x;
    return MSC_OK;
}

int batch_upload(msc_batch* b, const int (*t_slots)[2] = nullptr) {
    return b->precision == MSC_FP64 ? upload_batch<double>(b, t_slots) : upload_batch<float>(b, t_slots);
}

// ---- autotuner ---------------------------------------------------------------------------------

struct BatchTimer {
    cudaEvent_t e0, e1;
    bool ok;
    BatchTimer() : ok(cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {}
    ~BatchTimer() {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
};

// best of `reps` launches of one tuning-mode kernel family (0 sweep, 1 row pair, 2 column solve), us
template <typename T>
float time_batch_kernel(msc_batch* b, BatchTimer& tm, int which, int reps) {
    const BInst<T>* I = reinterpret_cast<const BInst<T>*>(b->ws + b->off_inst);
    const BMap* M = reinterpret_cast<const BMap*>(b->ws + b->off_map);
    float best = 1e30f;
    for (int r = 0; r < reps + 1; ++r) {  // the first launch warms up
        if (cudaEventRecord(tm.e0, b->stream) != cudaSuccess) return -1.f;
        if (which == 0) {
            k_bsweep2<T, 1><<<b->sweep_grid, kSweepWarps * 32, 0, b->stream>>>(I, M, nullptr, 0);
        } else if (which == 1) {
            k_browfft<T, false, 1><<<b->row_blocks, b->row_threads, b->row_smem, b->stream>>>(I, M, nullptr);
            k_browfft<T, true, 1><<<b->row_blocks, b->row_threads, b->row_smem, b->stream>>>(I, M, nullptr);
        } else {
            k_bcolsolve<T, 1><<<b->col_blocks, b->col_threads, b->col_smem, b->stream>>>(I, M, nullptr);
        }
        if (cudaGetLastError() != cudaSuccess) return -1.f;
        if (cudaEventRecord(tm.e1, b->stream) != cudaSuccess || cudaEventSynchronize(tm.e1) != cudaSuccess)
            return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, tm.e0, tm.e1);
        if (r > 0 && ms * 1000.f < best) best = ms * 1000.f;
    }
    return best;
}

// per instance the (input, output) ring slots of a stateless sweep: the accepted populations and
// a slot outside the history
int tuning_slots(msc_batch* b, int (*slots)[2]) {
    for (int i = 0; i < b->n_inst; ++i) {
        DevState hs;
        int rc = read_state(b->ctx[i], &hs);
        if (rc) return rc;
        slots[i][0] = hs.slot_fn[0];
        slots[i][1] = -1;
        for (int s = 0; s < kNumFBuf && slots[i][1] < 0; ++s) {
            bool used = false;
            for (int k = 0; k < hs.n_avail && k < 3; ++k) used |= hs.slot_fn[k] == s;
            if (!used && s != hs.slot_fn[0]) slots[i][1] = s;
        }
        if (slots[i][0] < 0 || slots[i][0] >= kNumFBuf || slots[i][1] < 0) return MSC_ERR_STATE;
    }
    return MSC_OK;
}

template <typename T>
int autotune_batch(msc_batch* b, int reps) {
    // tuning sweeps read each instance's accepted populations and write a free ring slot
    int slots[kBatchMax][2];
    int rc0 = tuning_slots(b, slots);
    if (rc0) return rc0;
    BatchTimer tm;
    if (!tm.ok) return MSC_ERR_CUDA;
    msc_batch_tuning& t = b->tun;
    int rc;
    auto measure = [&](int which, float* us) -> int {
        int r = batch_upload(b, slots);
        if (r) return r;
        *us = time_batch_kernel<T>(b, tm, which, reps);
        return *us < 0.f ? MSC_ERR_CUDA : MSC_OK;
    };
    float cur;
    // sweep: rows per warp unit, one size class at a time, then the persistent grid
    for (int c = 0; c < t.n_classes; ++c) {
        int best_hb = t.sweep_rows[c];
        float best = 1e30f;
        for (int hb : kHbChoices) {
            if (hb > t.n[c]) continue;
            t.sweep_rows[c] = hb;
            if ((rc = measure(0, &cur))) return rc;
            if (cur < best) { best = cur; best_hb = hb; }
        }
        t.sweep_rows[c] = best_hb;
    }
    {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bsweep2<T, 0>, kSweepWarps * 32, 0) != cudaSuccess)
            return MSC_ERR_CUDA;
        int best_k = t.sweep_ctas_per_sm;
        float best = 1e30f;
        for (int k = 1; k <= occ && k <= 16; ++k) {
            t.sweep_ctas_per_sm = k;
            if ((rc = measure(0, &cur))) return rc;
            if (cur < best) { best = cur; best_k = k; }
        }
        t.sweep_ctas_per_sm = best_k;
        t.sweep_us = best;
    }
    // row transforms (forward + inverse together)
    for (int c = 0; c < t.n_classes; ++c) {
        const int n = t.n[c];
        int best_p = t.fft_rows[c];
        float best = 1e30f;
        for (int P = 1; P <= n / 2 && P * n / fft_pts(n) <= kFftThreads; P <<= 1) {
            t.fft_rows[c] = P;
            if ((rc = measure(1, &cur))) return rc;
            if (cur < best) { best = cur; best_p = P; }
        }
        t.fft_rows[c] = best_p;
        t.rowfft_us = best;
    }
    // column solve
    for (int c = 0; c < t.n_classes; ++c) {
        const int n = t.n[c];
        int best_g = t.col_lines[c];
        float best = 1e30f;
        for (int G = 1; G <= 64 && 3 * G * n / fft_pts(n) <= col_thread_cap(b->precision); G <<= 1) {
            t.col_lines[c] = G;
            if ((rc = measure(2, &cur))) return rc;
            if (cur < best) { best = cur; best_g = G; }
        }
        t.col_lines[c] = best_g;
        t.colsolve_us = best;
    }
    return MSC_OK;
}

}  // namespace

extern "C" {

size_t msc_batch_workspace_bytes(msc_ctx* const* ctxs, int n_inst) {
    if (!batch_list_ok(ctxs, n_inst, nullptr)) return 0;
    return batch_offsets(ctxs, n_inst).total;
}

int msc_batch_create(msc_batch** out, msc_ctx* const* ctxs, int n_inst, void* ws, size_t bytes, void* stream) {
    if (!out) return MSC_ERR_ARG;
    *out = nullptr;
    int ncl = 0;
    if (!batch_list_ok(ctxs, n_inst, &ncl) || !ws || reinterpret_cast<uintptr_t>(ws) % 256) return MSC_ERR_ARG;
    const BatchOffsets o = batch_offsets(ctxs, n_inst);
    if (bytes < o.total) return MSC_ERR_ARG;
    for (int i = 0; i < n_inst; ++i)
        if (ctxs[i]->stream != (cudaStream_t)stream) return MSC_ERR_ARG;
    msc_batch* b = (msc_batch*)calloc(1, sizeof(msc_batch));
    if (!b) return MSC_ERR_ARG;
    b->n_inst = n_inst;
    b->precision = ctxs[0]->desc.precision;
    b->stream = (cudaStream_t)stream;
    b->ws = (unsigned char*)ws;
    b->off_inst = o.inst;
    b->off_map = o.map;
    b->off_act = o.act;
    b->off_upart = o.upart;
    b->off_ucount = o.ucount;
    b->off_tsum = o.tsum;
    // batch order: larger lattices first (their work units are handed out first), stable
    int idx[kBatchMax];
    for (int i = 0; i < n_inst; ++i) idx[i] = i;
    std::stable_sort(idx, idx + n_inst, [&](int x, int y) { return ctxs[x]->desc.n > ctxs[y]->desc.n; });
    b->tun.n_classes = 0;
    for (int k = 0; k < n_inst; ++k) {
        b->ctx[k] = ctxs[idx[k]];
        b->perm[k] = idx[k];
        const int n = b->ctx[k]->desc.n;
        int cl = -1;
        for (int c = 0; c < b->tun.n_classes; ++c)
            if (b->tun.n[c] == n) cl = c;
        if (cl < 0) {
            cl = b->tun.n_classes++;
            b->tun.n[cl] = n;
        }
        b->cls[k] = cl;
    }
    (void)ncl;
    default_tuning(b);
    if (cudaMemsetAsync(b->ws + o.ucount, 0, (size_t)n_inst * 32, b->stream) != cudaSuccess ||
        batch_upload(b) != MSC_OK) {
        free(b);
        return MSC_ERR_CUDA;
    }
    *out = b;
    return MSC_OK;
}

void msc_batch_destroy(msc_batch* b) {
    if (!b) return;
    drop_batch_graphs(b);
    free(b);
}

int msc_batch_march(msc_batch* b, const int* n_steps) {
    if (!b || !n_steps) return MSC_ERR_ARG;
    BSteps s;
    memset(&s, 0, sizeof(s));
    for (int i = 0; i < b->n_inst; ++i) {
        const int k = n_steps[b->perm[i]];
        msc_ctx* c = b->ctx[i];
        if (k < 0) return MSC_ERR_ARG;
        if (k > 0 && (!c->params_set || !c->fields_set)) return MSC_ERR_STATE;
        if (k > 0 && ctx_trt(c)) return MSC_ERR_ARG;  // the batched sweep is the operating-point kernel
        if (k > 0 && c->params.replay && k > c->desc.max_steps) return MSC_ERR_ARG;
        s.n[i] = k;
    }
    bool force = false;
    for (int i = 0; i < b->n_inst; ++i) {
        if (s.n[i] == 0) continue;
        int rc = refresh_tables(b->ctx[i]);
        if (rc) return rc;
        force |= params_force(b->ctx[i]->params);
    }
    if (b->x_march && force != b->graph_force) {  // the step-end kernel depends on whether a force acts
        cudaGraphExecDestroy(b->x_march);
        cudaGraphDestroy(b->g_march);
        b->x_march = nullptr;
        b->g_march = nullptr;
    }
    b->graph_force = force;
    if (!b->x_march) {
        int rc = b->precision == MSC_FP64 ? build_batch_march_graph<double>(b) : build_batch_march_graph<float>(b);
        if (rc) return rc;
    }
    const BMap* M = reinterpret_cast<const BMap*>(b->ws + b->off_map);
    k_btargets<<<1, kBatchMax, 0, b->stream>>>(M, s);
    CK(cudaGetLastError());
    CK(cudaGraphLaunch(b->x_march, b->stream));
    return MSC_OK;
}

int msc_batch_explicit_march(msc_batch* b, const int* n_steps) {
    if (!b || !n_steps) return MSC_ERR_ARG;
    BSteps s;
    memset(&s, 0, sizeof(s));
    bool any = false;
    for (int i = 0; i < b->n_inst; ++i) {
        const int k = n_steps[b->perm[i]];
        if (k < 0) return MSC_ERR_ARG;
        if (k > 0 && !b->ctx[i]->fields_set) return MSC_ERR_STATE;
        s.n[i] = k;
        any |= k > 0;
    }
    if (!any) return MSC_OK;
    if (!b->x_ex) {
        int rc = b->precision == MSC_FP64 ? build_batch_explicit_graph<double>(b)
                                          : build_batch_explicit_graph<float>(b);
        if (rc) return rc;
    }
    const BMap* M = reinterpret_cast<const BMap*>(b->ws + b->off_map);
    k_bex_setup<<<1, kBatchMax, 0, b->stream>>>(M, s);
    CK(cudaGetLastError());
    CK(cudaGraphLaunch(b->x_ex, b->stream));
    k_bex_finish<<<1, kBatchMax, 0, b->stream>>>(M, s);
    CK(cudaGetLastError());
    if (b->precision == MSC_FP64)
        k_bmoments_state<double><<<b->fld_grid, kFieldThreads, 0, b->stream>>>(
            reinterpret_cast<const BInst<double>*>(b->ws + b->off_inst), M, s);
    else
        k_bmoments_state<float><<<b->fld_grid, kFieldThreads, 0, b->stream>>>(
            reinterpret_cast<const BInst<float>*>(b->ws + b->off_inst), M, s);
    CK(cudaGetLastError());
    return MSC_OK;
}

int msc_batch_get_tuning(msc_batch* b, msc_batch_tuning* out) {
    if (!b || !out) return MSC_ERR_ARG;
    *out = b->tun;
    return MSC_OK;
}

int msc_batch_set_tuning(msc_batch* b, const msc_batch_tuning* t) {
    if (!b || !t || !tuning_ok(b, t)) return MSC_ERR_ARG;
    b->tun = *t;
    drop_batch_graphs(b);
    return batch_upload(b);
}

int msc_batch_time_stage(msc_batch* b, int which, int reps, float* us) {
    if (!b || !us || reps < 1 || which < 0 || which > 2) return MSC_ERR_ARG;
    int slots[kBatchMax][2];
    int rc = tuning_slots(b, slots);
    if (rc) return rc;
    rc = batch_upload(b, slots);
    if (rc) return rc;
    BatchTimer tm;
    if (!tm.ok) return MSC_ERR_CUDA;
    *us = b->precision == MSC_FP64 ? time_batch_kernel<double>(b, tm, which, reps)
                                   : time_batch_kernel<float>(b, tm, which, reps);
    return *us < 0.f ? MSC_ERR_CUDA : MSC_OK;
}

int msc_batch_autotune(msc_batch* b, int reps, msc_batch_tuning* out) {
    if (!b || reps < 1) return MSC_ERR_ARG;
    drop_batch_graphs(b);
    int rc = b->precision == MSC_FP64 ? autotune_batch<double>(b, reps) : autotune_batch<float>(b, reps);
    int rc2 = batch_upload(b);  // the chosen tiling, march mode
    if (rc) return rc;
    if (rc2) return rc2;
    if (out) *out = b->tun;
    return MSC_OK;
}

}  // extern "C"
