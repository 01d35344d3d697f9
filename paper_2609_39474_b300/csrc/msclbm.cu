// C ABI of the MSC-LBM library: contexts, the device-resident march (CUDA graph with nested
// conditional WHILE nodes, so that the acceptance test of Algorithm 1 never leaves the device),
// the explicit LBM baseline and the stage entry points.  See include/msclbm.h.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "march.cuh"
#include "spectral2d.cuh"
#include "spectral3d.cuh"
#include "sweep2d.cuh"
#include "sweep3d.cuh"
#include "sweep3p.cuh"

using namespace msc;

// explicit LBM steps per iteration of the conditional loop of the explicit-march graph (even)
constexpr int kExplicitUnroll = 8;

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return MSC_ERR_CUDA; \
    } while (0)

struct msc_ctx {
    msc_lattice_desc desc;
    int Q, logn;
    size_t sites;
    size_t elem;  // bytes per stored population / field element
    Layout lay;
    unsigned char* ws;
    cudaStream_t stream;
    bool params_set, fields_set;
    bool coef_dirty;  // solve coefficient tables need (re)computing for the current dt, nu
    msc_params params;
    // graphs
    cudaGraph_t g_march;
    cudaGraphExec_t x_march;
    cudaGraph_t g_ex;
    cudaGraphExec_t x_ex;
    cudaGraphExec_t x_adj[2];  // transposed solve of one adjoint step, BDF1 and BDF2
    int sweep_blocks;
    int march_prefix;  // straight-line inner iterations per step in the march graph
};

namespace {

template <typename P>
P* at(msc_ctx* c, size_t off) {
    return reinterpret_cast<P*>(c->ws + off);
}

int sweep_blocks_for(int dim, int n, int precision) {
    if (dim == 2) {  // the march's sweep and the explicit step (no partials, sized for both)
        const int b0 = sweep2_geometry(n).blocks, b1 = sweep2_geometry(n, kExplicitMinRows).blocks;
        return b0 > b1 ? b0 : b1;
    }
    return sweep3p_geometry(n, precision == MSC_FP64 ? 8 : 4).blocks;
}

// off-design TRT rates in effect (0 means the operating point)
bool params_trt(const msc_params& p) {
    const double wp = p.omega[0] > 0.0 ? p.omega[0] : 1.0, wm = p.omega[1] > 0.0 ? p.omega[1] : 1.0;
    return wp != 1.0 || wm != 1.0;
}
bool ctx_trt(const msc_ctx* c) { return c->params_set && params_trt(c->params); }
bool params_force(const msc_params& p) { return p.force[0] != 0.0 || p.force[1] != 0.0 || p.force[2] != 0.0; }

// the step-end kernel of a context: with or without the body-force terms
template <class L, typename T, typename FS>
const void* step_end_kernel(const msc_ctx* c) {
    return c->params_set && params_force(c->params) ? (const void*)k_step_end<L, T, FS, true>
                                                    : (const void*)k_step_end<L, T, FS, false>;
}

// the 2D sweep kernel of a context: operating point or general TRT collision
template <typename T, typename FS, bool EXPLICIT, bool GRAPH>
const void* sweep2_kernel(const msc_ctx* c) {
    return ctx_trt(c) ? (const void*)k_sweep2<T, FS, EXPLICIT, GRAPH, true>
                      : (const void*)k_sweep2<T, FS, EXPLICIT, GRAPH, false>;
}

size_t spec_bytes(int dim, int n, int precision) {
    const size_t celem = precision == MSC_FP64 ? 16 : 8;
    if (dim == 2) return (size_t)3 * n * (n / 4 + 1) * celem;
    return spec3_bytes(n, celem);
}

bool compute_layout(const msc_lattice_desc* d, Layout* L) {
    if (!d || !valid_lattice(d->dim, d->n, d->precision)) return false;
    if (d->max_steps < 1 || d->hist_cap < 1) return false;
    const size_t n = d->n;
    const size_t sites = d->dim == 2 ? n * n : n * n * n;
    const size_t Q = lattice_q(d->dim);
    const size_t F = d->dim + 1;
    const size_t e = field_elem(d->precision);
    const size_t ep = pop_elem(d->precision);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t r = o;
        o = align_up(o + bytes, 256);
        return r;
    };
    L->state = take(sizeof(DevState));
    L->fstride = Q * sites * ep;
    L->fbuf = take(kNumFBuf * L->fstride);
    // D3Q19: P f of every ring slot (the halo-free sweep reads its input's moments from there)
    L->pfstride = F * sites;
    L->pf = take(d->dim == 3 ? kNumFBuf * F * sites * ep : 0);
    L->mbuf = take(2 * F * sites * 8);
    L->h = take(F * sites * e * (e == 4 ? 2 : 1));  // binary32 storage: h as a hi + lo pair
    L->pr = take(F * sites * e);
    L->dm = take(F * sites * e);
    L->spec = take(spec_bytes(d->dim, d->n, d->precision));
    L->tw = take(n * 2 * e);
    L->coef = take(2 * 4 * solve_modes(d->dim, d->n) * sizeof(double));
    L->partial = take((size_t)sweep_blocks_for(d->dim, d->n, d->precision) * 8);
    L->counter = take(256);
    L->adj = take(kAdjBytes);  // adjoint run: position, per-step arguments and outcomes
    L->adjw = take(d->dim == 2 ? F * sites * e : 0);  // adjoint warm start: theta - c of the last step
    L->iters = take((size_t)d->max_steps * 4);
    L->hist = take((size_t)d->hist_cap * 8);
    L->replay = take((size_t)d->max_steps * 4);
    L->total = o;
    return true;
}

// grid of the grid-stride field kernels: at most 12 blocks of 256 threads per SM (A/B at N = 1024,
// march 2.83 ms at 16 per SM, 2.81 at 12, 2.85 at 6, 2.92 at 32)
int grid_for(size_t sites) {
    size_t b = (sites + kFieldThreads - 1) / kFieldThreads;
    if (b > 148 * 12) b = 148 * 12;
    if (b < 1) b = 1;
    return (int)b;
}

// ---- typed helpers ------------------------------------------------------------------------------

template <typename T, typename FS = T>
Sweep2Args<T, FS> sweep2_args_graph(msc_ctx* c, bool explicit_step = false) {
    Sweep2Args<T, FS> A;
    memset(&A, 0, sizeof(A));
    const Sweep2Geom g = sweep2_geometry(c->desc.n, explicit_step ? kExplicitMinRows : kSweepMinRows);
    A.dm = at<T>(c, c->lay.dm);
    A.h = at<T>(c, c->lay.h);
    A.pr = at<T>(c, c->lay.pr);
    A.partial = at<double>(c, c->lay.partial);
    A.counter = at<unsigned int>(c, c->lay.counter);
    A.n = c->desc.n;
    A.nstrips = g.nstrips;
    A.hb = g.hb;
    A.nrowblk = g.nrowblk;
    A.st = at<DevState>(c, c->lay.state);
    A.fbase = at<FS>(c, c->lay.fbuf);
    A.fstride = c->lay.fstride / sizeof(FS);
    A.fscale = 1.0;
    A.hist = at<double>(c, c->lay.hist);
    A.hist_cap = c->desc.hist_cap;
    A.replay_counts = at<int>(c, c->lay.replay);
    A.max_steps = c->desc.max_steps;
    return A;
}

template <typename T>
Sweep3Args<T> sweep3_args_graph(msc_ctx* c) {
    Sweep3Args<T> A;
    memset(&A, 0, sizeof(A));
    const Sweep3Geom g = sweep3_geometry(c->desc.n, sizeof(T));
    A.dm = at<T>(c, c->lay.dm);
    A.h = at<T>(c, c->lay.h);
    A.pr = at<T>(c, c->lay.pr);
    A.partial = at<double>(c, c->lay.partial);
    A.counter = at<unsigned int>(c, c->lay.counter);
    A.n = c->desc.n;
    A.g = g;
    A.st = at<DevState>(c, c->lay.state);
    A.fbase = at<T>(c, c->lay.fbuf);
    A.fstride = c->lay.fstride / sizeof(T);
    A.hist = at<double>(c, c->lay.hist);
    A.hist_cap = c->desc.hist_cap;
    A.replay_counts = at<int>(c, c->lay.replay);
    A.max_steps = c->desc.max_steps;
    return A;
}

// the D3Q19 sweep of the march: halo-free, reading and writing the P f field of its ring slots
template <typename T>
Sweep3PArgs<T> sweep3p_args_graph(msc_ctx* c) {
    Sweep3PArgs<T> A;
    memset(&A, 0, sizeof(A));
    A.g = sweep3p_geometry(c->desc.n, sizeof(T));
    A.dm = at<T>(c, c->lay.dm);
    A.h = at<T>(c, c->lay.h);
    A.pr = at<T>(c, c->lay.pr);
    A.partial = at<double>(c, c->lay.partial);
    A.counter = at<unsigned int>(c, c->lay.counter);
    A.n = c->desc.n;
    A.st = at<DevState>(c, c->lay.state);
    A.fbase = at<T>(c, c->lay.fbuf);
    A.fstride = c->lay.fstride / sizeof(T);
    A.pfbase = at<T>(c, c->lay.pf);
    A.pfstride = c->lay.pfstride;
    A.hist = at<double>(c, c->lay.hist);
    A.hist_cap = c->desc.hist_cap;
    A.replay_counts = at<int>(c, c->lay.replay);
    A.max_steps = c->desc.max_steps;
    return A;
}

// P f field base of a context's ring (D3Q19), null for D2Q9
template <typename FS>
FS* pf_base(msc_ctx* c) {
    return c->desc.dim == 3 ? at<FS>(c, c->lay.pf) : nullptr;
}

// Programmatic edges between consecutive kernel nodes of the march graph: the successor is launched
// while its predecessor drains and waits (wait_for_predecessor) before reading its results.
constexpr bool kProgrammaticEdges = true;
// the same for the explicit LBM graph's chain of steps (the baseline: N = 128 2.97 -> 2.78 us per
// step, N = 1024 12.95 -> 12.74 us; the march itself gains 0.6 .. 1.2 % from its own edges)
constexpr bool kExplicitProgrammatic = true;

// a kernel node that depends on the kernel node prev only, through a programmatic edge
cudaGraphNode_t add_kernel_after(cudaGraph_t g, cudaGraphNode_t prev, const void* fn, dim3 grid, dim3 block,
                                 size_t smem, void** args, cudaError_t* err) {
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams* p = reinterpret_cast<cudaGraphNodeParams*>(raw);
    p->type = cudaGraphNodeTypeKernel;
    p->kernel.func = const_cast<void*>(fn);
    p->kernel.gridDim = grid;
    p->kernel.blockDim = block;
    p->kernel.sharedMemBytes = (unsigned)smem;
    p->kernel.kernelParams = args;
    cudaGraphEdgeData ed;
    memset(&ed, 0, sizeof(ed));
    if (kProgrammaticEdges) {
        ed.from_port = cudaGraphKernelNodePortProgrammatic;
        ed.type = cudaGraphDependencyTypeProgrammatic;
    }
    cudaGraphNode_t node = nullptr;
    cudaError_t e = cudaGraphAddNode(&node, g, &prev, &ed, 1, p);
    if (e != cudaSuccess && *err == cudaSuccess) *err = e;
    return node;
}

cudaGraphNode_t add_kernel(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, const void* fn,
                           dim3 grid, dim3 block, size_t smem, void** args, cudaError_t* err) {
    cudaKernelNodeParams p;
    memset(&p, 0, sizeof(p));
    p.func = const_cast<void*>(fn);
    p.gridDim = grid;
    p.blockDim = block;
    p.sharedMemBytes = (unsigned)smem;
    p.kernelParams = args;
    cudaGraphNode_t node = nullptr;
    cudaError_t e = cudaGraphAddKernelNode(&node, g, deps.empty() ? nullptr : deps.data(), deps.size(), &p);
    if (e != cudaSuccess && *err == cudaSuccess) *err = e;
    return node;
}

cudaGraphNode_t add_cond(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps,
                         cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                         cudaGraph_t* body, cudaError_t* err) {
    // the parameter union has no default constructor: build it in zeroed raw storage
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams* p = reinterpret_cast<cudaGraphNodeParams*>(raw);
    p->type = cudaGraphNodeTypeConditional;
    p->conditional.handle = h;
    p->conditional.type = type;
    p->conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    cudaError_t e = cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), p);
    if (e != cudaSuccess) {
        if (*err == cudaSuccess) *err = e;
        *body = nullptr;
        return nullptr;
    }
    *body = p->conditional.phGraph_out[0];
    return node;
}

// spectral correction nodes: 2D forward row FFT, column FFT + solve + inverse, inverse row FFT;
// 3D the five passes of spectral3d.cuh.  All take the same argument block.  The first pass follows
// prev (if any) on a programmatic edge; gate: the passes check that the sweep before them asked for
// the correction (the march graph has no branch node for it).  Returns the last pass.
template <typename T>
cudaGraphNode_t add_spectral_nodes(msc_ctx* c, cudaGraph_t g, cudaGraphNode_t prev, int gate, cudaError_t* err) {
    using C = typename Cplx<T>::type;
    const int n = c->desc.n;
    Spec2Args<T> S = spec3_args<T>(n, c->logn, 0.0, c->params.nu, at<T>(c, c->lay.pr), at<C>(c, c->lay.spec),
                                   at<T>(c, c->lay.dm), at<C>(c, c->lay.tw), at<DevState>(c, c->lay.state),
                                   at<double>(c, c->lay.coef));
    S.gate = gate;
    void* args[] = {&S};
    if (c->desc.dim == 2) {
        S.nf = 3;
        S.rows = n;
        S.nscale = 1.0 / ((double)n * n);
        Spec2Launch L[3];
        S.P = spectral2_launches<T>(n, L);
        for (int i = 0; i < 3; ++i)
            prev = prev ? add_kernel_after(g, prev, L[i].fn, L[i].grid, L[i].block, L[i].smem, args, err)
                        : add_kernel(g, {}, L[i].fn, L[i].grid, L[i].block, L[i].smem, args, err);
    } else {
        LaunchDesc L[5];
        spectral3_launches<T>(n, L);
        for (int i = 0; i < 5; ++i) {
            spec3_pass_args<T>(n, &S, i);  // node parameters are copied when the node is added
            prev = prev ? add_kernel_after(g, prev, L[i].fn, L[i].grid, L[i].block, L[i].smem, args, err)
                        : add_kernel(g, {}, L[i].fn, L[i].grid, L[i].block, L[i].smem, args, err);
        }
    }
    return prev;
}

// The first n_min - 1 inner iterations of a step can never be accepted (Algorithm 1: l >= n_min), so
// the march graph runs them as straight-line nodes ahead of the conditional inner loop: no loop node
// per iteration, and programmatic edges from each sweep into its correction and on into the next
// sweep.  Replay mode (the counts are given) runs only the first sweep ahead of the loop.
constexpr int kMaxMarchPrefix = 7;
// physical steps per iteration of the march graph's step loop (one loop node and one ordinary edge
// into a step's first sweep per group instead of per step)
constexpr int kMarchStepsPerLoop = 4;
inline int march_prefix_count(const msc_params& p) {
    if (p.replay) return 0;
    return p.nmin - 1 < 0 ? 0 : (p.nmin - 1 > kMaxMarchPrefix ? kMaxMarchPrefix : p.nmin - 1);
}

// the march's sweep as a graph node in g (after prev on a programmatic edge, if given); it sets the
// inner loop's condition h_iter to "not accepted"
template <class L, typename T, typename FS>
cudaGraphNode_t add_sweep_node(msc_ctx* c, cudaGraph_t g, cudaGraphNode_t prev, cudaGraphConditionalHandle h_iter,
                               cudaError_t* err) {
    if (L::D == 2) {
        Sweep2Args<T, FS> A = sweep2_args_graph<T, FS>(c);
        A.h_iter = h_iter;
        A.cond = 1;
        void* a_sw[] = {&A};
        const void* fn = sweep2_kernel<T, FS, false, true>(c);
        const dim3 grid(sweep2_geometry(c->desc.n).blocks), block(kSweepWarps * 32);
        return prev ? add_kernel_after(g, prev, fn, grid, block, 0, a_sw, err)
                    : add_kernel(g, {}, fn, grid, block, 0, a_sw, err);
    }
    Sweep3PArgs<T> A = sweep3p_args_graph<T>(c);
    A.h_iter = h_iter;
    A.cond = 1;
    void* a_sw[] = {&A};
    const void* fn = (const void*)k_sweep3p<T, true>;
    return prev ? add_kernel_after(g, prev, fn, dim3(A.g.blocks), dim3(kP3Threads), A.g.smem, a_sw, err)
                : add_kernel(g, {}, fn, dim3(A.g.blocks), dim3(kP3Threads), A.g.smem, a_sw, err);
}

template <typename T>
int set_smem_limits(int dim, int n) {
    if (dim == 2) {
        const RowGeom rg = row_geometry(n, 3, n);
        CK(cudaFuncSetAttribute(k_rowfft_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)spec_row_smem<T>(n, rg.P)));
        CK(cudaFuncSetAttribute(k_rowfft_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)spec_row_smem<T>(n, rg.P)));
        CK(cudaFuncSetAttribute(k_colsolve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)spec2_col_smem<T>(n)));
        Spec2Launch L[3];
        spectral2_launches<T>(n, L);
        for (int i = 0; i < 3; ++i)
            CK(cudaFuncSetAttribute(L[i].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L[i].smem));
    } else {
        if (set_spec3_smem_limits<T>(n) != 0) return MSC_ERR_CUDA;
        if (set_sweep3_smem_limits<T>(n) != 0) return MSC_ERR_CUDA;
        if (set_sweep3p_smem_limits<T>(n) != 0) return MSC_ERR_CUDA;
    }
    return MSC_OK;
}

template <class L, typename T, typename FS>
int build_march_graph(msc_ctx* c) {
    cudaError_t err = cudaSuccess;
    int rc = set_smem_limits<T>(c->desc.dim, c->desc.n);
    if (rc) return rc;
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    DevState* st = at<DevState>(c, c->lay.state);
    FS* fbase = at<FS>(c, c->lay.fbuf);
    const size_t fstride = c->lay.fstride / sizeof(FS);
    double* mbuf = at<double>(c, c->lay.mbuf);
    T* h = at<T>(c, c->lay.h);
    int* iters = at<int>(c, c->lay.iters);
    size_t sites = c->sites;
    int max_steps = c->desc.max_steps;
    const int fgrid = grid_for(sites);

    // prologue: arm the step loop, set up the first step and form its h and trial; every later
    // step is set up by the previous step's k_step_finish_graph, its h and trial formed by k_step_end
    cudaGraphConditionalHandle h_step, h_iter;
    CK(cudaGraphConditionalHandleCreate(&h_step, g, 0, 0));
    void* a_arm[] = {&st, &h_step};
    cudaGraphNode_t arm = add_kernel(g, {}, (const void*)k_arm_setup, dim3(1), dim3(1), 0, a_arm, &err);
    FS* pfbase = pf_base<FS>(c);
    size_t pfstride = c->lay.pfstride;
    void* a_begin[] = {&st, &fbase, (void*)&fstride, &mbuf, &h, &sites, &pfbase, &pfstride};
    cudaGraphNode_t begin = add_kernel(g, {arm}, (const void*)k_step_begin<L, T, FS>, dim3(fgrid),
                                       dim3(kFieldThreads), 0, a_begin, &err);
    cudaGraph_t body_step;
    add_cond(g, {begin}, h_step, cudaGraphCondTypeWhile, &body_step, &err);
    if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }

    // kMarchStepsPerLoop physical steps per iteration of the step loop (a step after the march's last
    // one finds no live step: its kernels return at once).  One physical step: the inner iterations
    // that cannot be accepted, straight-line; the next sweep; then, while the last sweep was not
    // accepted, its correction and another sweep (every sweep sets the step's inner-loop handle);
    // acceptance with the next step's h and trial; the history rotation and the step loop's condition
    const int npre = march_prefix_count(c->params);
    c->march_prefix = npre;
    cudaGraphNode_t prev = nullptr;
    for (int k = 0; k < kMarchStepsPerLoop; ++k) {
        CK(cudaGraphConditionalHandleCreate(&h_iter, body_step, 0u, cudaGraphCondAssignDefault));
        cudaGraphNode_t pre = prev;
        for (int i = 0; i < npre; ++i) {
            pre = add_sweep_node<L, T, FS>(c, body_step, pre, h_iter, &err);
            pre = add_spectral_nodes<T>(c, body_step, pre, 1, &err);
        }
        pre = add_sweep_node<L, T, FS>(c, body_step, pre, h_iter, &err);
        if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
        cudaGraph_t body_iter;
        cudaGraphNode_t wit = add_cond(body_step, {pre}, h_iter, cudaGraphCondTypeWhile, &body_iter, &err);
        if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
        void* a_end[] = {&st, &fbase, (void*)&fstride, &mbuf, &h, &sites, &pfbase, &pfstride};
        cudaGraphNode_t end = add_kernel(body_step, {wit}, step_end_kernel<L, T, FS>(c), dim3(fgrid),
                                         dim3(kFieldThreads), 0, a_end, &err);
        void* a_fin[] = {&st, &iters, &max_steps, &h_step};
        prev = add_kernel_after(body_step, end, (const void*)k_step_finish_graph, dim3(1), dim3(1), 0, a_fin, &err);

        cudaGraphNode_t cor = add_spectral_nodes<T>(c, body_iter, nullptr, 1, &err);
        add_sweep_node<L, T, FS>(c, body_iter, cor, h_iter, &err);
        if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    }

    cudaGraphExec_t x;
    if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    c->g_march = g;
    c->x_march = x;
    return MSC_OK;
}

template <class L, typename T, typename FS>
int build_explicit_graph(msc_ctx* c) {
    cudaError_t err = cudaSuccess;
    int rc = set_smem_limits<T>(c->desc.dim, c->desc.n);
    if (rc) return rc;
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    DevState* st = at<DevState>(c, c->lay.state);
    cudaGraphConditionalHandle h_ex;
    CK(cudaGraphConditionalHandleCreate(&h_ex, g, 0, 0));
    void* a_arm[] = {&st, &h_ex};
    cudaGraphNode_t arm = add_kernel(g, {}, (const void*)k_ex_arm, dim3(1), dim3(1), 0, a_arm, &err);
    cudaGraph_t body;
    add_cond(g, {arm}, h_ex, cudaGraphCondTypeWhile, &body, &err);
    if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    // kExplicitUnroll steps per loop iteration, alternating a->b and b->a; the last one counts
    cudaGraphNode_t prev = nullptr;
    for (int i = 0; i < kExplicitUnroll; ++i) {
        std::vector<cudaGraphNode_t> deps;
        if (prev) deps.push_back(prev);
        if (L::D == 2) {
            Sweep2Args<T, FS> A = sweep2_args_graph<T, FS>(c, true);
            A.ex_dir = i & 1;
            A.ex_count = i == kExplicitUnroll - 1;
            A.h_ex = h_ex;
            void* aa[] = {&A};
            const dim3 eg(sweep2_geometry(c->desc.n, kExplicitMinRows).blocks);
            prev = prev && kExplicitProgrammatic
                       ? add_kernel_after(body, prev, sweep2_kernel<T, FS, true, true>(c), eg, dim3(kSweepWarps * 32), 0,
                                          aa, &err)
                       : add_kernel(body, deps, sweep2_kernel<T, FS, true, true>(c), eg, dim3(kSweepWarps * 32), 0, aa,
                                    &err);
        } else {
            Sweep3Args<T> A = sweep3_args_graph<T>(c);
            A.ex_dir = i & 1;
            A.ex_count = i == kExplicitUnroll - 1;
            A.h_ex = h_ex;
            void* aa[] = {&A};
            prev = prev && kExplicitProgrammatic
                       ? add_kernel_after(body, prev, (const void*)k_sweep3<T, true, true>, dim3(A.g.blocks),
                                          dim3(A.g.threads), A.g.smem, aa, &err)
                       : add_kernel(body, deps, (const void*)k_sweep3<T, true, true>, dim3(A.g.blocks),
                                    dim3(A.g.threads), A.g.smem, aa, &err);
        }
    }
    if (err != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    cudaGraphExec_t x;
    if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) { cudaGraphDestroy(g); return MSC_ERR_CUDA; }
    c->g_ex = g;
    c->x_ex = x;
    return MSC_OK;
}

template <class L, typename T, typename FS>
int run_explicit(msc_ctx* c, int n_steps) {
    if (!c->x_ex) {
        int rc = build_explicit_graph<L, T, FS>(c);
        if (rc) return rc;
    }
    DevState* st = at<DevState>(c, c->lay.state);
    const int blocks = n_steps / kExplicitUnroll;
    const int rem = n_steps % kExplicitUnroll;
    const int odd = rem & 1;
    k_ex_setup<<<1, 1, 0, c->stream>>>(st, blocks);
    CK(cudaGetLastError());
    if (blocks > 0) CK(cudaGraphLaunch(c->x_ex, c->stream));
    for (int i = 0; i < rem; ++i) {  // the remainder alternates a->b, b->a, ... as in the loop body
        if (L::D == 2) {
            Sweep2Args<T, FS> A = sweep2_args_graph<T, FS>(c, true);
            A.ex_dir = i & 1;
            void* aa[] = {&A};
            CK(cudaLaunchKernel(sweep2_kernel<T, FS, true, true>(c),
                                dim3(sweep2_geometry(c->desc.n, kExplicitMinRows).blocks), dim3(kSweepWarps * 32), aa,
                                0, c->stream));
        } else {
            Sweep3Args<T> A = sweep3_args_graph<T>(c);
            A.ex_dir = i & 1;
            k_sweep3<T, true, true><<<A.g.blocks, A.g.threads, A.g.smem, c->stream>>>(A);
        }
        CK(cudaGetLastError());
    }
    k_ex_finish<<<1, 1, 0, c->stream>>>(st, odd);
    CK(cudaGetLastError());
    // m^n = P f^n, m^{n-1} = m^n: read the new slot from the state on the device
    k_moments_state<L, T, FS><<<grid_for(c->sites), kFieldThreads, 0, c->stream>>>(
        st, at<FS>(c, c->lay.fbuf), c->lay.fstride / sizeof(FS), at<double>(c, c->lay.mbuf), c->sites);
    CK(cudaGetLastError());
    return MSC_OK;
}

template <class L, typename T, typename FS>
int run_init(msc_ctx* c, const double* p, const double* u, int on_device) {
    DevState* st = at<DevState>(c, c->lay.state);
    double* m0 = at<double>(c, c->lay.mbuf);
    double* m1 = m0 + (size_t)(L::D + 1) * c->sites;
    const size_t fb = c->sites * sizeof(double);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // stage (p, u) in the m^{n-1} slot, build f^0 in ring slot 0, then m^0 = P f^0 in both slots
    CK(cudaMemcpyAsync(m1, p, fb, kind, c->stream));
    CK(cudaMemcpyAsync(m1 + c->sites, u, fb * L::D, kind, c->stream));
    k_reset_history<<<1, 1, 0, c->stream>>>(st);
    CK(cudaGetLastError());
    FS* f0 = at<FS>(c, c->lay.fbuf);
    if (std::is_same<FS, __half>::value) {  // storage scale sigma from max |f^0|
        k_feq_absmax<L><<<grid_for(c->sites), kFieldThreads, 0, c->stream>>>(m1, m1 + c->sites, c->sites, st);
        CK(cudaGetLastError());
        k_set_scale<<<1, 1, 0, c->stream>>>(st);
        CK(cudaGetLastError());
    }
    k_equilibrium<L, FS><<<grid_for(c->sites), kFieldThreads, 0, c->stream>>>(m1, m1 + c->sites, f0, c->sites, st);
    CK(cudaGetLastError());
    k_moments<L, FS><<<grid_for(c->sites), kFieldThreads, 0, c->stream>>>(f0, m0, m1, c->sites, st);
    CK(cudaGetLastError());
    return MSC_OK;
}

int refresh_tables(msc_ctx* c) {
    if (!c->coef_dirty) return MSC_OK;
    const size_t nm = solve_modes(c->desc.dim, c->desc.n);
    int blocks = (int)((2 * nm + 255) / 256);
    if (blocks > 148 * 16) blocks = 148 * 16;
    k_solve_tables<<<blocks, 256, 0, c->stream>>>(at<double>(c, c->lay.coef), c->desc.dim, c->desc.n,
                                                  c->params.dt, c->params.nu);
    CK(cudaGetLastError());
    c->coef_dirty = false;
    return MSC_OK;
}

int read_state(msc_ctx* c, DevState* hs);

// Call fn(L{}, T{}, FS{}) for the context's lattice, arithmetic/field type T and population
// storage type FS (FP16 storage exists for D2Q9 only).
template <typename Fn>
int dispatch(const msc_ctx* c, Fn&& fn) {
    if (c->desc.dim == 2) {
        if (c->desc.precision == MSC_FP64) return fn(D2Q9{}, double{}, double{});
        if (c->desc.precision == MSC_FP32) return fn(D2Q9{}, float{}, float{});
        return fn(D2Q9{}, float{}, __half{});
    }
    if (c->desc.precision == MSC_FP64) return fn(D3Q19{}, double{}, double{});
    return fn(D3Q19{}, float{}, float{});
}
#define MSC_TYPES(l, t, s) decltype(l), decltype(t), decltype(s)

// The march of msc_march driven from the host: the same kernels launched one by one, with the
// acceptance decision read back after every sweep.  For profilers that do not descend into
// conditional graph nodes, and for debugging.
template <class L, typename T, typename FS>
int run_stepwise(msc_ctx* c, int n_steps) {
    using C = typename Cplx<T>::type;
    int rc = set_smem_limits<T>(c->desc.dim, c->desc.n);
    if (rc) return rc;
    DevState* st = at<DevState>(c, c->lay.state);
    FS* fbase = at<FS>(c, c->lay.fbuf);
    const size_t fstride = c->lay.fstride / sizeof(FS);
    double* mbuf = at<double>(c, c->lay.mbuf);
    T* h = at<T>(c, c->lay.h);
    const int fgrid = grid_for(c->sites);
    cudaGraphConditionalHandle none = 0;
    Spec2Args<T> S = spec3_args<T>(c->desc.n, c->logn, 0.0, c->params.nu, at<T>(c, c->lay.pr), at<C>(c, c->lay.spec),
                                   at<T>(c, c->lay.dm), at<C>(c, c->lay.tw), st, at<double>(c, c->lay.coef));
    LaunchDesc spec[5];
    int nspec = 0;
    if (c->desc.dim == 2) {
        const int n = c->desc.n;
        S.nf = 3;
        S.rows = n;
        S.nscale = 1.0 / ((double)n * n);
        Spec2Launch SL[3];
        S.P = spectral2_launches<T>(n, SL);
        for (int i = 0; i < 3; ++i) spec[i] = {SL[i].fn, SL[i].grid, SL[i].block, SL[i].smem};
        nspec = 3;
    } else {
        spectral3_launches<T>(c->desc.n, spec);
        nspec = 5;
    }
    void* sargs[] = {&S};
    k_set_target<<<1, 1, 0, c->stream>>>(st, n_steps);
    DevState hs;
    for (int step = 0; step < n_steps; ++step) {
        k_step_setup<<<1, 1, 0, c->stream>>>(st, none, 0);
        k_step_begin<L, T, FS><<<fgrid, kFieldThreads, 0, c->stream>>>(st, fbase, fstride, mbuf, h, c->sites,
                                                                        pf_base<FS>(c), c->lay.pfstride);
        for (;;) {
            if (L::D == 2) {
                Sweep2Args<T, FS> A = sweep2_args_graph<T, FS>(c);
                void* aa[] = {&A};
                CK(cudaLaunchKernel(sweep2_kernel<T, FS, false, true>(c), dim3(sweep2_geometry(c->desc.n).blocks),
                                    dim3(kSweepWarps * 32), aa, 0, c->stream));
            } else {
                Sweep3PArgs<T> A = sweep3p_args_graph<T>(c);
                k_sweep3p<T, true><<<A.g.blocks, kP3Threads, A.g.smem, c->stream>>>(A);
            }
            CK(cudaGetLastError());
            rc = read_state(c, &hs);
            if (rc) return rc;
            if (hs.lift)
                for (int i = 0; i < nspec; ++i) {
                    if (c->desc.dim == 3) spec3_pass_args<T>(c->desc.n, &S, i);
                    CK(cudaLaunchKernel(spec[i].fn, spec[i].grid, spec[i].block, sargs, spec[i].smem, c->stream));
                }
            if (hs.accepted || hs.status != MSC_OK) break;
        }
        {
            FS* pfb = pf_base<FS>(c);
            size_t pfs = c->lay.pfstride;
            void* ea[] = {&st, &fbase, (void*)&fstride, &mbuf, &h, (void*)&c->sites, &pfb, &pfs};
            CK(cudaLaunchKernel(step_end_kernel<L, T, FS>(c), dim3(fgrid), dim3(kFieldThreads), ea, 0, c->stream));
        }
        k_step_finish<<<1, 1, 0, c->stream>>>(st, at<int>(c, c->lay.iters), c->desc.max_steps, none, 0);
        CK(cudaGetLastError());
        rc = read_state(c, &hs);
        if (rc) return rc;
        if (hs.status != MSC_OK || hs.steps_target <= 0) break;
    }
    return MSC_OK;
}

int read_state(msc_ctx* c, DevState* hs) {
    CK(cudaMemcpyAsync(hs, c->ws + c->lay.state, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MSC_OK;
}

}  // namespace

// ================================================================================================
extern "C" {

const char* msc_strerror(int s) {
    switch (s) {
        case MSC_OK: return "ok";
        case MSC_ERR_ARG: return "invalid argument";
        case MSC_ERR_NONCONVERGED: return "physical step reached K_max without passing the residual test";
        case MSC_ERR_NONFINITE: return "non-finite raw residual";
        case MSC_ERR_TIMEOUT: return "device wait exceeded its budget";
        case MSC_ERR_CUDA: return "CUDA runtime error";
        case MSC_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

size_t msc_workspace_bytes(const msc_lattice_desc* desc) {
    Layout L;
    if (!compute_layout(desc, &L)) return 0;
    return L.total;
}

int msc_create(msc_ctx** out, const msc_lattice_desc* desc, void* ws, size_t bytes, void* stream) {
    if (!out) return MSC_ERR_ARG;
    *out = nullptr;
    Layout L;
    if (!compute_layout(desc, &L) || !ws || bytes < L.total) return MSC_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % 256) return MSC_ERR_ARG;
    msc_ctx* c = (msc_ctx*)calloc(1, sizeof(msc_ctx));
    if (!c) return MSC_ERR_ARG;
    c->desc = *desc;
    c->Q = lattice_q(desc->dim);
    c->logn = ilog2(desc->n);
    c->sites = desc->dim == 2 ? (size_t)desc->n * desc->n : (size_t)desc->n * desc->n * desc->n;
    c->elem = field_elem(desc->precision);
    c->lay = L;
    c->ws = (unsigned char*)ws;
    c->stream = (cudaStream_t)stream;
    c->coef_dirty = true;
    // zero the state, the reduction counter, h (read by stateless timing sweeps before any step) and
    // the adjoint warm start (a first warm step starts cold)
    if (cudaMemsetAsync(c->ws + L.state, 0, sizeof(DevState), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->ws + L.h, 0, L.pr - L.h, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->ws + L.counter, 0, 256, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->ws + L.adjw, 0, L.iters - L.adjw, c->stream) != cudaSuccess) {
        free(c);
        return MSC_ERR_CUDA;
    }
    k_reset_history<<<1, 1, 0, c->stream>>>(at<DevState>(c, L.state));  // sigma = 1 until init
    const int n = desc->n;
    if (desc->precision == MSC_FP64)
        k_twiddles<double2><<<(n + 255) / 256, 256, 0, c->stream>>>((double2*)(c->ws + L.tw), n);
    else
        k_twiddles<float2><<<(n + 255) / 256, 256, 0, c->stream>>>((float2*)(c->ws + L.tw), n);
    if (cudaGetLastError() != cudaSuccess) {
        free(c);
        return MSC_ERR_CUDA;
    }
    *out = c;
    return MSC_OK;
}

void msc_destroy(msc_ctx* c) {
    if (!c) return;
    if (c->x_march) cudaGraphExecDestroy(c->x_march);
    if (c->g_march) cudaGraphDestroy(c->g_march);
    if (c->x_ex) cudaGraphExecDestroy(c->x_ex);
    if (c->g_ex) cudaGraphDestroy(c->g_ex);
    for (int i = 0; i < 2; ++i)
        if (c->x_adj[i]) cudaGraphExecDestroy(c->x_adj[i]);
    free(c);
}

int msc_set_params(msc_ctx* c, const msc_params* p) {
    if (!c || !p) return MSC_ERR_ARG;
    if (!(p->dt > 0.0) || !(p->eps >= 0.0) || !(p->nu > 0.0) || p->kmax < 1 || p->nmin < 1 ||
        (p->corrector != 0 && p->corrector != 1) || (p->replay != 0 && p->replay != 1) || p->warm_order < 0 ||
        p->warm_order > 3 || p->count_multiple < 0 || p->count_multiple > 2 || !std::isfinite(p->force[0]) ||
        !std::isfinite(p->force[1]) || !std::isfinite(p->force[2]) || !(p->omega[0] >= 0.0 && p->omega[0] < 2.0) ||
        !(p->omega[1] >= 0.0 && p->omega[1] < 2.0))
        return MSC_ERR_ARG;
    if (params_trt(*p) && c->desc.dim != 2) return MSC_ERR_ARG;  // the general TRT sweep exists for D2Q9
    // the shadow solve bakes nu into the graph, the collision kind picks the sweep kernel: rebuild
    const bool kind_changes = c->params_set && (params_trt(*p) != params_trt(c->params) ||
                                                params_force(*p) != params_force(c->params));
    // so do n_min and replay, which set the straight-line iterations of each step
    const bool prefix_changes = c->x_march && march_prefix_count(*p) != c->march_prefix;
    if (c->params_set && (p->nu != c->params.nu || kind_changes || prefix_changes) && c->x_march) {
        cudaGraphExecDestroy(c->x_march);
        cudaGraphDestroy(c->g_march);
        c->x_march = nullptr;
        c->g_march = nullptr;
    }
    if (kind_changes && c->x_ex) {
        cudaGraphExecDestroy(c->x_ex);
        cudaGraphDestroy(c->g_ex);
        c->x_ex = nullptr;
        c->g_ex = nullptr;
    }
    if (!c->params_set || p->dt != c->params.dt || p->nu != c->params.nu) c->coef_dirty = true;
    c->params = *p;
    if (c->params.warm_order == 0)  // FP32 storage: the cubic rule grows rounding in weakly damped modes
        c->params.warm_order = c->desc.precision == MSC_FP64 ? 3 : (c->desc.dim == 2 ? 2 : 1);
    if (c->params.count_multiple == 0)  // FP32 D2Q9: keep the staggered modes' per-step factor positive
        c->params.count_multiple = c->desc.precision != MSC_FP64 && c->desc.dim == 2 ? 2 : 1;
    c->params_set = true;
    k_set_params<<<1, 1, 0, c->stream>>>(at<DevState>(c, c->lay.state), c->params);
    CK(cudaGetLastError());
    return MSC_OK;
}

int msc_init_fields(msc_ctx* c, const double* p, const double* u, int on_device) {
    if (!c || !p || !u) return MSC_ERR_ARG;
    int rc = dispatch(c, [&](auto l, auto t, auto s) { return run_init<MSC_TYPES(l, t, s)>(c, p, u, on_device); });
    if (rc == MSC_OK) c->fields_set = true;
    return rc;
}

int msc_march(msc_ctx* c, int n_steps) {
    if (!c || n_steps < 0) return MSC_ERR_ARG;
    if (!c->params_set || !c->fields_set) return MSC_ERR_STATE;
    if (!c->x_march) {
        int rc = dispatch(c, [&](auto l, auto t, auto s) { return build_march_graph<MSC_TYPES(l, t, s)>(c); });
        if (rc) return rc;
    }
    if (c->params.replay && n_steps > c->desc.max_steps) return MSC_ERR_ARG;
    int rc = refresh_tables(c);
    if (rc) return rc;
    k_set_target<<<1, 1, 0, c->stream>>>(at<DevState>(c, c->lay.state), n_steps);
    CK(cudaGetLastError());
    CK(cudaGraphLaunch(c->x_march, c->stream));
    return MSC_OK;
}

int msc_march_stepwise(msc_ctx* c, int n_steps) {
    if (!c || n_steps < 0) return MSC_ERR_ARG;
    if (!c->params_set || !c->fields_set) return MSC_ERR_STATE;
    if (c->params.replay && n_steps > c->desc.max_steps) return MSC_ERR_ARG;
    int rc = refresh_tables(c);
    if (rc) return rc;
    return dispatch(c, [&](auto l, auto t, auto s) { return run_stepwise<MSC_TYPES(l, t, s)>(c, n_steps); });
}

int msc_explicit_march(msc_ctx* c, int n_steps) {
    if (!c || n_steps < 0) return MSC_ERR_ARG;
    if (!c->fields_set) return MSC_ERR_STATE;
    if (n_steps == 0) return MSC_OK;
    return dispatch(c, [&](auto l, auto t, auto s) { return run_explicit<MSC_TYPES(l, t, s)>(c, n_steps); });
}

int msc_get_stats(msc_ctx* c, msc_stats* out) {
    if (!c || !out) return MSC_ERR_ARG;
    DevState s;
    int rc = read_state(c, &s);
    if (rc) return rc;
    out->steps_done = s.steps_done;
    out->inner_total = s.inner_total;
    out->steps_in_call = s.steps_in_call;
    out->last_iters = s.last_iters;
    out->last_q = s.last_q;
    out->status = s.status;
    out->last_R = s.R_last;
    return MSC_OK;
}

int msc_read_fields(msc_ctx* c, double* p, double* u, int on_device) {
    if (!c || !p || !u) return MSC_ERR_ARG;
    DevState s;
    int rc = read_state(c, &s);
    if (rc) return rc;
    const size_t F = c->desc.dim + 1;
    const double* m = at<double>(c, c->lay.mbuf) + (size_t)s.m_cur * F * c->sites;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(p, m, c->sites * 8, kind, c->stream));
    CK(cudaMemcpyAsync(u, m + c->sites, c->sites * 8 * c->desc.dim, kind, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MSC_OK;
}

int msc_copy_fields_async(msc_ctx* c, double* m) {
    if (!c || !m) return MSC_ERR_ARG;
    const size_t count = (size_t)(c->desc.dim + 1) * c->sites;
    k_copy_fields<<<grid_for(count), kFieldThreads, 0, c->stream>>>(at<const DevState>(c, c->lay.state),
                                                                     at<const double>(c, c->lay.mbuf), m, count);
    CK(cudaGetLastError());
    return MSC_OK;
}

int msc_read_populations(msc_ctx* c, double* f, int on_device) {
    if (!c || !f) return MSC_ERR_ARG;
    DevState s;
    int rc = read_state(c, &s);
    if (rc) return rc;
    const size_t cnt = (size_t)c->Q * c->sites;
    const unsigned char* src = c->ws + c->lay.fbuf + (size_t)s.slot_fn[0] * c->lay.fstride;
    if (c->desc.precision == MSC_FP64) {
        CK(cudaMemcpyAsync(f, src, cnt * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return MSC_OK;
    }
    if (on_device) return MSC_ERR_ARG;  // FP32 / FP16 storage: host read-back only
    const size_t ep = pop_elem(c->desc.precision);
    void* tmp = malloc(cnt * ep);
    if (!tmp) return MSC_ERR_ARG;
    if (cudaMemcpyAsync(tmp, src, cnt * ep, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        free(tmp);
        return MSC_ERR_CUDA;
    }
    if (c->desc.precision == MSC_FP32) {
        for (size_t i = 0; i < cnt; ++i) f[i] = (double)((const float*)tmp)[i];
    } else {  // FP16: stored f / sigma
        for (size_t i = 0; i < cnt; ++i) f[i] = s.fscale * (double)__half2float(((const __half*)tmp)[i]);
    }
    free(tmp);
    return MSC_OK;
}

int msc_get_residual_history(msc_ctx* c, double* R, int cap, int* n) {
    if (!c || !R || !n || cap < 0) return MSC_ERR_ARG;
    DevState s;
    int rc = read_state(c, &s);
    if (rc) return rc;
    const int64_t total = s.hist_pos;
    const int64_t keep = total < c->desc.hist_cap ? total : c->desc.hist_cap;
    const int64_t cnt = keep < cap ? keep : cap;
    std::vector<double> h(c->desc.hist_cap);
    CK(cudaMemcpy(h.data(), c->ws + c->lay.hist, (size_t)c->desc.hist_cap * 8, cudaMemcpyDeviceToHost));
    // oldest kept value first
    const int64_t first = total - keep;
    for (int64_t i = 0; i < cnt; ++i) R[i] = h[(first + i) % c->desc.hist_cap];
    *n = (int)cnt;
    return MSC_OK;
}

int msc_get_step_iters(msc_ctx* c, int* iters, int cap, int* n) {
    if (!c || !iters || !n || cap < 0) return MSC_ERR_ARG;
    DevState s;
    int rc = read_state(c, &s);
    if (rc) return rc;
    int cnt = s.steps_in_call < c->desc.max_steps ? s.steps_in_call : c->desc.max_steps;
    if (cnt > cap) cnt = cap;
    if (cnt > 0) CK(cudaMemcpy(iters, c->ws + c->lay.iters, (size_t)cnt * 4, cudaMemcpyDeviceToHost));
    *n = cnt;
    return MSC_OK;
}

int msc_set_replay_counts(msc_ctx* c, const int* counts, int n) {
    if (!c || !counts || n < 0 || n > c->desc.max_steps) return MSC_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (counts[i] < 1) return MSC_ERR_ARG;
    CK(cudaMemcpyAsync(c->ws + c->lay.replay, counts, (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MSC_OK;
}

// blob: [magic, dim, n, precision, n_avail, e] int32 x6 (population scale sigma = 2^e), steps_done
// int64, then n_avail population arrays (storage type, newest first), then m^n and m^{n-1} (double)
int msc_save_state(msc_ctx* c, void* blob, size_t* bytes) {
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
    unsigned char* b = (unsigned char*)blob;
    int sig_exp = 0;
    frexp(s.fscale > 0.0 ? s.fscale : 1.0, &sig_exp);
    int32_t hdr[6] = {0x4d53434c, c->desc.dim, c->desc.n, c->desc.precision, s.n_avail, sig_exp - 1};
    memcpy(b, hdr, 24);
    int64_t sd = s.steps_done;
    memcpy(b + 24, &sd, 8);
    size_t o = 32;
    for (int i = 0; i < s.n_avail; ++i) {
        CK(cudaMemcpy(b + o, c->ws + c->lay.fbuf + (size_t)s.slot_fn[i] * c->lay.fstride, c->lay.fstride,
                      cudaMemcpyDeviceToHost));
        o += c->lay.fstride;
    }
    const double* mb = at<double>(c, c->lay.mbuf);
    CK(cudaMemcpy(b + o, mb + (size_t)s.m_cur * F * c->sites, F * c->sites * 8, cudaMemcpyDeviceToHost));
    o += F * c->sites * 8;
    CK(cudaMemcpy(b + o, mb + (size_t)s.m_prev * F * c->sites, F * c->sites * 8, cudaMemcpyDeviceToHost));
    *bytes = need;
    return MSC_OK;
}

int msc_load_state(msc_ctx* c, const void* blob, size_t bytes) {
    if (!c || !blob || bytes < 32) return MSC_ERR_ARG;
    const unsigned char* b = (const unsigned char*)blob;
    int32_t hdr[6];
    memcpy(hdr, b, 24);
    if (hdr[0] != 0x4d53434c || hdr[1] != c->desc.dim || hdr[2] != c->desc.n || hdr[3] != c->desc.precision ||
        hdr[4] < 1 || hdr[4] > 3 || hdr[5] < -1000 || hdr[5] > 1000)
        return MSC_ERR_ARG;
    int64_t sd;
    memcpy(&sd, b + 24, 8);
    const size_t F = c->desc.dim + 1;
    const size_t need = 32 + (size_t)hdr[4] * c->lay.fstride + 2 * F * c->sites * 8;
    if (bytes < need) return MSC_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream));
    DevState s;
    int rc = read_state(c, &s);
    if (rc) return rc;
    size_t o = 32;
    for (int i = 0; i < hdr[4]; ++i) {
        CK(cudaMemcpy(c->ws + c->lay.fbuf + (size_t)i * c->lay.fstride, b + o, c->lay.fstride,
                      cudaMemcpyHostToDevice));
        o += c->lay.fstride;
    }
    double* mb = at<double>(c, c->lay.mbuf);
    CK(cudaMemcpy(mb, b + o, F * c->sites * 8, cudaMemcpyHostToDevice));
    o += F * c->sites * 8;
    CK(cudaMemcpy(mb + F * c->sites, b + o, F * c->sites * 8, cudaMemcpyHostToDevice));
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
    CK(cudaMemcpy(c->ws + c->lay.state, &s, sizeof(DevState), cudaMemcpyHostToDevice));
    c->fields_set = true;
    return MSC_OK;
}

int msc_bounds_check_report(unsigned long long* count, unsigned long long* first, int reset) {
    if (!count || !first) return MSC_ERR_ARG;
    *count = 0;
    *first = 0;
#ifdef MSC_BOUNDS_CHECK
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpyFromSymbol(count, g_oob_count, sizeof(unsigned long long)));
    CK(cudaMemcpyFromSymbol(first, g_oob_first, sizeof(unsigned long long)));
    if (reset) {
        const unsigned long long zero = 0;
        CK(cudaMemcpyToSymbol(g_oob_count, &zero, sizeof(zero)));
        CK(cudaMemcpyToSymbol(g_oob_first, &zero, sizeof(zero)));
    }
    return MSC_OK;
#else
    (void)reset;
    return MSC_ERR_STATE;
#endif
}

// ---- stage entry points ------------------------------------------------------------------------

size_t msc_stage_scratch_bytes(int dim, int n, int precision) {
    if (!valid_lattice(dim, n, precision)) return 0;
    size_t o = 0;
    o = align_up(o + 256, 256);                                  // counter
    o = align_up(o + (size_t)sweep_blocks_for(dim, n, precision) * 8, 256);  // partials
    o = align_up(o + (size_t)n * (precision == MSC_FP64 ? 16 : 8), 256);  // twiddles
    o = align_up(o + spec_bytes(dim, n, precision), 256);         // half spectrum
    if (dim == 3) o = align_up(o + (size_t)2 * 4 * n * n * n * field_elem(precision), 256);  // P f in, out
    return o;
}

}  // extern "C"

namespace {
struct StageScratch {
    unsigned int* counter;
    double* partial;
    void* tw;
    void* spec;
    void* pf;  // D3Q19 sweep: P f of the input, then of the output
};
StageScratch stage_scratch(int dim, int n, int precision, void* base) {
    StageScratch s;
    unsigned char* b = (unsigned char*)base;
    size_t o = 0;
    s.counter = (unsigned int*)(b + o);
    o = align_up(o + 256, 256);
    s.partial = (double*)(b + o);
    o = align_up(o + (size_t)sweep_blocks_for(dim, n, precision) * 8, 256);
    s.tw = b + o;
    o = align_up(o + (size_t)n * (precision == MSC_FP64 ? 16 : 8), 256);
    s.spec = b + o;
    o = align_up(o + spec_bytes(dim, n, precision), 256);
    s.pf = dim == 3 ? b + o : nullptr;
    return s;
}

template <typename T, typename FS = T>
int stage_sweep(int dim, int n, double a, const void* fin, const void* dm, const void* h, void* fout,
                void* pr, double* sumsq, void* scratch, cudaStream_t stream, double wp = 0.0, double wm = 0.0,
                bool hpair = false) {
    StageScratch S = stage_scratch(dim, n, sizeof(T) == 8 ? MSC_FP64 : MSC_FP32, scratch);
    CK(cudaMemsetAsync(S.counter, 0, 4, stream));
    if (dim == 2) {
        Sweep2Args<T, FS> A;
        memset(&A, 0, sizeof(A));
        const Sweep2Geom g = sweep2_geometry(n);
        A.fin = (const FS*)fin;
        A.dm = (const T*)dm;
        A.h = (const T*)h;
        A.fout = (FS*)fout;
        A.pr = (T*)pr;
        A.a = a;
        A.inv = 1.0 / (1.0 + a / 2.0);
        A.fscale = 1.0;
        A.omega_p = wp;
        A.omega_m = wm;
        A.lift = dm != nullptr;
        A.sumsq_out = sumsq;
        A.partial = S.partial;
        A.counter = S.counter;
        A.n = n;
        A.nstrips = g.nstrips;
        A.hb = g.hb;
        A.nrowblk = g.nrowblk;
        if (wp > 0.0)
            k_sweep2<T, FS, false, false, true><<<g.blocks, kSweepWarps * 32, 0, stream>>>(A);
        else if (hpair)
            k_sweep2<T, FS, false, false, false, std::is_same<T, float>::value><<<g.blocks, kSweepWarps * 32, 0,
                                                                                 stream>>>(A);
        else
            k_sweep2<T, FS, false, false><<<g.blocks, kSweepWarps * 32, 0, stream>>>(A);
    } else if constexpr (std::is_same<T, FS>::value) {
        // the march's halo-free D3Q19 sweep: P f of the input first, then the sweep
        if (set_sweep3p_smem_limits<T>(n) != 0) return MSC_ERR_CUDA;
        const size_t sites = (size_t)n * n * n;
        T* pfin = (T*)S.pf;
        T* pfout = pfin + 4 * sites;
        size_t b = (sites + kFieldThreads - 1) / kFieldThreads;
        if (b > 148 * 12) b = 148 * 12;
        k_pop_moments3<T><<<(int)b, kFieldThreads, 0, stream>>>((const T*)fin, pfin, sites);
        Sweep3PArgs<T> A;
        memset(&A, 0, sizeof(A));
        A.g = sweep3p_geometry(n, sizeof(T));
        A.fin = (const T*)fin;
        A.pfin = pfin;
        A.dm = (const T*)dm;
        A.h = (const T*)h;
        A.fout = (T*)fout;
        A.pfout = pfout;
        A.pr = (T*)pr;
        A.a = a;
        A.inv = 1.0 / (1.0 + a / 2.0);
        A.lift = dm != nullptr;
        A.sumsq_out = sumsq;
        A.partial = S.partial;
        A.counter = S.counter;
        A.n = n;
        k_sweep3p<T, false><<<A.g.blocks, kP3Threads, A.g.smem, stream>>>(A);
    }
    CK(cudaGetLastError());
    return MSC_OK;
}

template <typename T>
int stage_shadow(int dim, int n, double a, double nu, const void* pr, void* dm, void* scratch,
                 cudaStream_t stream) {
    using C = typename Cplx<T>::type;
    StageScratch S = stage_scratch(dim, n, sizeof(T) == 8 ? MSC_FP64 : MSC_FP32, scratch);
    k_twiddles<C><<<(n + 255) / 256, 256, 0, stream>>>((C*)S.tw, n);
    CK(cudaGetLastError());
    int rc = set_smem_limits<T>(dim, n);
    if (rc) return rc;
    if (dim == 2) {
        Spec2Args<T> A;
        memset(&A, 0, sizeof(A));
        A.pr = (const T*)pr;
        A.spec = (C*)S.spec;
        A.dm = (T*)dm;
        A.tw = (const C*)S.tw;
        A.n = n;
        A.logn = ilog2(n);
        A.nf = 3;
        A.rows = n;
        A.a = a;
        A.nu = nu;
        A.kunit = 6.283185307179586476925286766559 / (double)n;
        A.nscale = 1.0 / ((double)n * n);
        A.st = nullptr;
        Spec2Launch L[3];
        A.P = spectral2_launches<T>(n, L);
        void* args[] = {&A};
        for (int i = 0; i < 3; ++i) CK(cudaLaunchKernel(L[i].fn, L[i].grid, L[i].block, args, L[i].smem, stream));
        return MSC_OK;
    }
    return launch_spectral3<T>(n, ilog2(n), a, nu, (const T*)pr, (C*)S.spec, (T*)dm, (const C*)S.tw, stream);
}
}  // namespace

extern "C" {

int msc_sweep(int dim, int n, int precision, double a, const void* f_in, const void* dm, const void* h,
              void* f_out, void* pr_out, double* sumsq_out, void* scratch, size_t scratch_bytes,
              void* stream) {
    if (!valid_lattice(dim, n, precision) || !f_in || !h || !f_out || !pr_out || !sumsq_out || !scratch ||
        f_in == f_out || scratch_bytes < msc_stage_scratch_bytes(dim, n, precision) || !(a >= 0.0))
        return MSC_ERR_ARG;
    if (precision == MSC_FP64)
        return stage_sweep<double>(dim, n, a, f_in, dm, h, f_out, pr_out, sumsq_out, scratch, (cudaStream_t)stream);
    if (precision == MSC_FP16)
        return stage_sweep<float, __half>(dim, n, a, f_in, dm, h, f_out, pr_out, sumsq_out, scratch,
                                          (cudaStream_t)stream);
    return stage_sweep<float>(dim, n, a, f_in, dm, h, f_out, pr_out, sumsq_out, scratch, (cudaStream_t)stream);
}

int msc_sweep_d3q19_pf(int n, int precision, double a, const void* f_in, const void* pf_in, const void* dm,
                       const void* h, void* f_out, void* pf_out, void* pr_out, double* sumsq_out, void* scratch,
                       size_t scratch_bytes, void* stream) {
    if (!valid_lattice(3, n, precision) || precision == MSC_FP16 || !f_in || !pf_in || !h || !f_out || !pf_out ||
        !pr_out || !sumsq_out || !scratch || f_in == f_out || pf_in == pf_out ||
        scratch_bytes < msc_stage_scratch_bytes(3, n, precision) || !(a >= 0.0))
        return MSC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    auto run = [&](auto tag) -> int {
        using T = decltype(tag);
        if (set_sweep3p_smem_limits<T>(n) != 0) return MSC_ERR_CUDA;
        StageScratch S = stage_scratch(3, n, precision, scratch);
        CK(cudaMemsetAsync(S.counter, 0, 4, st));
        Sweep3PArgs<T> A;
        memset(&A, 0, sizeof(A));
        A.g = sweep3p_geometry(n, sizeof(T));
        A.fin = (const T*)f_in;
        A.pfin = (const T*)pf_in;
        A.dm = (const T*)dm;
        A.h = (const T*)h;
        A.fout = (T*)f_out;
        A.pfout = (T*)pf_out;
        A.pr = (T*)pr_out;
        A.a = a;
        A.inv = 1.0 / (1.0 + a / 2.0);
        A.lift = dm != nullptr;
        A.sumsq_out = sumsq_out;
        A.partial = S.partial;
        A.counter = S.counter;
        A.n = n;
        // the march's kernel: with binary32 storage h is the high / low pair the march holds
        k_sweep3p<T, false, std::is_same<T, float>::value><<<A.g.blocks, kP3Threads, A.g.smem, st>>>(A);
        CK(cudaGetLastError());
        return MSC_OK;
    };
    return precision == MSC_FP64 ? run(double{}) : run(float{});
}

int msc_sweep_hpair(int n, int precision, double a, const void* f_in, const void* dm, const void* h,
                    void* f_out, void* pr_out, double* sumsq_out, void* scratch, size_t scratch_bytes,
                    void* stream) {
    if (!valid_lattice(2, n, precision) || !f_in || !h || !f_out || !pr_out || !sumsq_out || !scratch ||
        f_in == f_out || scratch_bytes < msc_stage_scratch_bytes(2, n, precision) || !(a >= 0.0))
        return MSC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == MSC_FP64)
        return stage_sweep<double>(2, n, a, f_in, dm, h, f_out, pr_out, sumsq_out, scratch, st);
    if (precision == MSC_FP16)
        return stage_sweep<float, __half>(2, n, a, f_in, dm, h, f_out, pr_out, sumsq_out, scratch, st, 0.0, 0.0,
                                          true);
    return stage_sweep<float>(2, n, a, f_in, dm, h, f_out, pr_out, sumsq_out, scratch, st, 0.0, 0.0, true);
}

int msc_sweep_trt(int n, int precision, double a, double omega_p, double omega_m, const void* f_in, const void* dm,
                  const void* h, void* f_out, void* pr_out, double* sumsq_out, void* scratch, size_t scratch_bytes,
                  void* stream) {
    if (!valid_lattice(2, n, precision) || !f_in || !h || !f_out || !pr_out || !sumsq_out || !scratch ||
        f_in == f_out || scratch_bytes < msc_stage_scratch_bytes(2, n, precision) || !(a >= 0.0) ||
        !(omega_p > 0.0 && omega_p < 2.0) || !(omega_m > 0.0 && omega_m < 2.0))
        return MSC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == MSC_FP64)
        return stage_sweep<double>(2, n, a, f_in, dm, h, f_out, pr_out, sumsq_out, scratch, st, omega_p, omega_m);
    if (precision == MSC_FP16)
        return stage_sweep<float, __half>(2, n, a, f_in, dm, h, f_out, pr_out, sumsq_out, scratch, st, omega_p,
                                          omega_m);
    return stage_sweep<float>(2, n, a, f_in, dm, h, f_out, pr_out, sumsq_out, scratch, st, omega_p, omega_m);
}

int msc_shadow_solve(int dim, int n, int precision, double a, double nu, const void* pr, void* dm,
                     void* scratch, size_t scratch_bytes, void* stream) {
    if (!valid_lattice(dim, n, precision) || !pr || !dm || pr == dm || !scratch ||
        scratch_bytes < msc_stage_scratch_bytes(dim, n, precision) || !(a > 0.0) || !(nu > 0.0))
        return MSC_ERR_ARG;
    if (precision == MSC_FP64)
        return stage_shadow<double>(dim, n, a, nu, pr, dm, scratch, (cudaStream_t)stream);
    return stage_shadow<float>(dim, n, a, nu, pr, dm, scratch, (cudaStream_t)stream);
}

int msc_equilibrium(int dim, int n, int precision, const double* p, const double* u, void* f_out,
                    void* stream) {
    if (!valid_lattice(dim, n, precision) || !p || !u || !f_out) return MSC_ERR_ARG;
    const size_t sites = dim == 2 ? (size_t)n * n : (size_t)n * n * n;
    cudaStream_t s = (cudaStream_t)stream;
    if (dim == 2) {
        if (precision == MSC_FP64)
            k_equilibrium<D2Q9, double><<<grid_for(sites), kFieldThreads, 0, s>>>(p, u, (double*)f_out, sites);
        else if (precision == MSC_FP16)
            k_equilibrium<D2Q9, __half><<<grid_for(sites), kFieldThreads, 0, s>>>(p, u, (__half*)f_out, sites);
        else
            k_equilibrium<D2Q9, float><<<grid_for(sites), kFieldThreads, 0, s>>>(p, u, (float*)f_out, sites);
    } else {
        if (precision == MSC_FP64)
            k_equilibrium<D3Q19, double><<<grid_for(sites), kFieldThreads, 0, s>>>(p, u, (double*)f_out, sites);
        else
            k_equilibrium<D3Q19, float><<<grid_for(sites), kFieldThreads, 0, s>>>(p, u, (float*)f_out, sites);
    }
    CK(cudaGetLastError());
    return MSC_OK;
}

}  // extern "C"

#include "sweep_noalloc.cuh"
#include "batch_api.cuh"
#include "adjoint_api.cuh"
#include "fullsym_api.cuh"
#include "selftest.cuh"
