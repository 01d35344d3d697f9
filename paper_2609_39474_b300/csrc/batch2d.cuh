// Batched D2Q9 march: many independent periodic lattices of uneven n (and their own nu, dt, eps,
// Re) advanced by one CUDA graph.  Every instance keeps its own context (device state, population
// ring, BDF history, spectrum, solve tables) and runs exactly the per-instance algorithm of the
// single march (Algorithm 1, Section 3); the batch only changes how the work is scheduled.
//
// One round of the graph's loop performs one inner iteration of every active instance:
//   k_bsweep2   persistent sweep: a fixed grid of warps walks the work list of (instance, strip,
//               row block) units of all active instances; the last unit of an instance reduces its
//               residual norm in a fixed order and takes the acceptance decision (Algorithm 1)
//   k_browfft   forward / inverse row transforms and k_bcolsolve the column FFT + FP64 solve, for
//               the instances whose sweep asked for a shadow correction
//   k_bstep_end acceptance (m^{n+1}) and the next step's h and warm start, accepted instances only
//   k_bfinish   history rotation per instance, the loop condition (any instance still active) and
//               the next round's work list
// Instances therefore drift apart in phase (each converges in its own number of inner
// iterations) without waiting for one another; an instance leaves the work list when its steps
// are done or it stops with an error.  The work list is compacted at every round (BAct): its
// prefix tables cover the active instances only.  The sweep and the field kernels run grids of at
// most one resident wave that stride over the list, so the tail rounds, in which a few small
// instances are still iterating, run no work for the finished ones; the spectral kernels keep one
// block per row (column) block of the whole batch, and those past the list's total leave at once.
#pragma once

#include "common.cuh"
#include "march.cuh"
#include "spectral2d.cuh"
#include "sweep2d.cuh"

namespace msc {

constexpr int kBatchMax = 64;

// per-instance arguments, in device memory
template <typename T>
struct BInst {
    Sweep2Args<T> sw;       // graph-mode sweep arguments (hist, replay counts, pointers, geometry)
    Spec2Args<T> sp;        // graph-mode spectral arguments with this instance's P and G
    DevState* st;
    T* fbase;
    size_t fstride;         // elements
    double* mbuf;
    T* h;
    size_t sites;
    int* iters;
    int max_steps;
    int units;              // sweep warp units (nstrips x nrowblk)
    double* upart;          // per-unit partial sums of r^2 (batch workspace)
    unsigned int* ucount;   // finished units of the current sweep (batch workspace)
    // tuning mode: stateless sweep from t_fin into t_fout, norm into t_sumsq
    const T* t_fin;
    T* t_fout;
    double* t_sumsq;
};

// work-list prefix tables: instance i owns units [unit_off[i], unit_off[i+1]) and so on
struct BMap {
    int n_inst;
    int unit_off[kBatchMax + 1];
    int row_off[kBatchMax + 1];
    int col_off[kBatchMax + 1];
    int fld_off[kBatchMax + 1];
    int col_g[kBatchMax];       // columns per block of the column solve
    DevState* st[kBatchMax];
    int* iters[kBatchMax];
    int max_steps[kBatchMax];
};

// the round's work list: the active instances in batch order and prefix tables over their sweep
// units, row blocks, column blocks and field blocks (written on the device by k_bsetup / k_bfinish)
struct BAct {
    int n_act;
    int inst[kBatchMax];
    int unit_off[kBatchMax + 1];
    int row_off[kBatchMax + 1];
    int col_off[kBatchMax + 1];
    int fld_off[kBatchMax + 1];
};

// a prefix-table view of the work: entry j is instance ids[j] (ids null: instance j) and owns the
// items [off[j], off[j + 1])
struct BList {
    const int* off;
    const int* ids;
    int n;
    __device__ __forceinline__ int total() const { return __ldg(off + n); }
};

// MODE 0 (the march) walks the compacted list of active instances; the tuning and explicit modes
// walk every instance of the batch
template <int MODE>
__device__ __forceinline__ BList blist(const BMap* __restrict__ M, const BAct* __restrict__ A, int which) {
    if (MODE == 0) {
        const int* o = which == 0 ? A->unit_off : which == 1 ? A->row_off : which == 2 ? A->col_off : A->fld_off;
        return {o, A->inst, __ldg(&A->n_act)};
    }
    const int* o = which == 0 ? M->unit_off : which == 1 ? M->row_off : which == 2 ? M->col_off : M->fld_off;
    return {o, nullptr, __ldg(&M->n_inst)};
}

// per-call step counts (kernel parameter)
struct BSteps {
    int n[kBatchMax];
};

// largest i with off[i] <= x, for off[0] = 0 <= x < off[n_inst]
__device__ __forceinline__ int find_inst(const int* __restrict__ off, int n_inst, int x) {
    int lo = 0, hi = n_inst;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// item x of a list -> (entry j, instance, first item of the entry)
__device__ __forceinline__ int list_entry(const BList& L, int x, int* inst, int* first) {
    const int j = find_inst(L.off, L.n, x);
    *inst = L.ids ? __ldg(L.ids + j) : j;
    *first = __ldg(L.off + j);
    return j;
}

__device__ __forceinline__ bool inst_active(const DevState* vs) {
    return vs->params_ok && vs->status == MSC_OK && vs->steps_target > 0;
}

// MODE 0: march (state from the device), 1: tuning (stateless, every instance), 2: explicit LBM
// step `ex_node` of the unrolled explicit loop body.
template <typename T, int MODE>
__global__ void __launch_bounds__(kSweepWarps * 32) k_bsweep2(const BInst<T>* __restrict__ I,
                                                             const BMap* __restrict__ M,
                                                             const BAct* __restrict__ W, int ex_node) {
    if constexpr (MODE == 2) wait_for_predecessor();  // the batched explicit graph chains its steps (programmatic)
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * kSweepWarps;
    const BList L = blist<MODE>(M, W, 0);
    const int total = L.total();
    for (int u = blockIdx.x * kSweepWarps + (threadIdx.x >> 5); u < total; u += nw) {  // warp-uniform
        int i, u0;
        list_entry(L, u, &i, &u0);
        const BInst<T>& B = I[i];
        const int lu = u - u0;
        const Sweep2Args<T>& A = B.sw;
        const T* fin;
        T* fout;
        T a, inv;
        int lift;
        if (MODE == 0) {
            const DevState* vs = B.st;
            if (!inst_active(vs)) continue;
            fin = B.fbase + (size_t)vs->slot_cur * B.fstride;
            fout = B.fbase + (size_t)vs->slot_nxt * B.fstride;
            a = (T)vs->a;
            inv = (T)vs->inv_a;
            lift = vs->lift;
        } else if (MODE == 1) {
            fin = B.t_fin;
            fout = B.t_fout;
            a = (T)A.a;
            inv = (T)A.inv;
            lift = 1;
        } else {
            const DevState* vs = B.st;
            if (vs->ex_loops_left <= ex_node) continue;
            const int sa = vs->ex_a, sb = vs->ex_b;
            fin = B.fbase + (size_t)((ex_node & 1) ? sb : sa) * B.fstride;
            fout = B.fbase + (size_t)((ex_node & 1) ? sa : sb) * B.fstride;
            a = T(0);
            inv = T(1);
            lift = 0;
        }
        // the march and the tuning mode read the instance's h, a binary32 pair for FP32 storage
        double ssq = sweep2_unit<T, T, MODE == 2, false, MODE != 2 && std::is_same<T, float>::value>(
            fin, A.dm, A.h, fout, A.pr, a, inv, lift, A.n, A.hb, lu % A.nstrips, lu / A.nstrips, lane);
        if constexpr (MODE != 2) {  // residual norm of the instance (not for the explicit step)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, off);
            unsigned int last = 0;
            if (lane == 0) {
                B.upart[lu] = ssq;
                __threadfence();
                last = atomicAdd(B.ucount, 1u) == (unsigned int)(B.units - 1);
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (!last) continue;
            // the last unit of instance i: every partial of the sweep is visible, sum in a fixed order
            __threadfence();
            double s = 0.0;
            for (int k = lane; k < B.units; k += 32) s += __ldcg(B.upart + k);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) {
                *B.ucount = 0u;
                if (MODE == 0)
                    march_after_sweep(B.st, s, 9.0 * (double)B.sites, A.hist, A.hist_cap, A.replay_counts, A.max_steps,
                                      0, 0);
                else
                    *B.t_sumsq = s;
            }
        }
    }
}

// spectral passes; MODE 0 runs for instances whose last sweep asked for a correction, MODE 1 (tuning)
// for every instance with the solve coefficients evaluated in place
template <typename T, int MODE>
__device__ __forceinline__ bool spec_inst(const BInst<T>& B, Spec2Args<T>* A) {
    *A = B.sp;
    if (MODE == 1) {
        A->st = nullptr;
        A->coef = nullptr;
        return true;
    }
    const DevState* vs = B.st;
    return inst_active(vs) && vs->lift;
}

// The spectral kernels take one row (column) block of the list per thread block, over a grid of
// the whole batch's blocks; the blocks past the list's total leave at once.  (A grid-stride loop over
// the items would launch fewer blocks in the tail rounds, but a transform inside any loop needs
// twice the registers, 190-255 per thread, and the column solve spills.)  Whether an instance takes
// the correction is read from its state.
template <typename T, bool INV, int MODE>
__global__ void __launch_bounds__(kFftThreads) k_browfft(const BInst<T>* __restrict__ I, const BMap* __restrict__ M,
                                                         const BAct* __restrict__ W) {
    const BList L = blist<MODE>(M, W, 1);
    const int x = blockIdx.x;
    if (x >= L.total()) return;
    int i, x0;
    list_entry(L, x, &i, &x0);
    Spec2Args<T> A;
    if (!spec_inst<T, MODE>(I[i], &A)) return;
    if (A.n <= kSpec2Radix4Max) {  // the single march's radix-4 form at small n (block-uniform)
        if (INV) rowfft_inv_block<T, false, true>(A, x - x0);
        else rowfft_fwd_block<T, true>(A, x - x0);
    } else {
        if (INV) rowfft_inv_block<T>(A, x - x0);
        else rowfft_fwd_block<T>(A, x - x0);
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 384 : 768) k_bcolsolve(const BInst<T>* __restrict__ I,
                                                                          const BMap* __restrict__ M,
                                                                          const BAct* __restrict__ W) {
    const BList L = blist<MODE>(M, W, 2);
    const int x = blockIdx.x;
    if (x >= L.total()) return;
    int i, x0;
    list_entry(L, x, &i, &x0);
    Spec2Args<T> A;
    if (!spec_inst<T, MODE>(I[i], &A)) return;
    if (A.n <= kSpec2Radix4Max) colsolve_block<T, false, true>(A, x - x0, __ldg(M->col_g + i));
    else colsolve_block<T>(A, x - x0, __ldg(M->col_g + i));
}

// field kernels: list entry j owns the field blocks [off[j], off[j + 1]), which cover its
// instance's sites with a grid-stride loop; item x -> instance, first site and stride
__device__ __forceinline__ int fld_item(const BList& L, int x, size_t* i0, size_t* istride) {
    int i, b0;
    const int j = list_entry(L, x, &i, &b0);
    const int nb = __ldg(L.off + j + 1) - b0;
    *i0 = (size_t)(x - b0) * blockDim.x + threadIdx.x;
    *istride = (size_t)nb * blockDim.x;
    return i;
}

template <typename T>
__global__ void __launch_bounds__(kFieldThreads) k_bstep_begin(const BInst<T>* __restrict__ I,
                                                               const BMap* __restrict__ M,
                                                               const BAct* __restrict__ W) {
    const BList L = blist<0>(M, W, 3);
    const int total = L.total();
    for (int x = blockIdx.x; x < total; x += gridDim.x) {
        size_t i0, is;
        const BInst<T>& B = I[fld_item(L, x, &i0, &is)];
        if (inst_active(B.st)) step_begin_range<D2Q9, T>(B.st, B.fbase, B.fstride, B.mbuf, B.h, B.sites, i0, is);
    }
}

template <typename T, bool FORCE>
__global__ void __launch_bounds__(kFieldThreads) k_bstep_end(const BInst<T>* __restrict__ I,
                                                             const BMap* __restrict__ M,
                                                             const BAct* __restrict__ W) {
    const BList L = blist<0>(M, W, 3);
    const int total = L.total();
    for (int x = blockIdx.x; x < total; x += gridDim.x) {
        size_t i0, is;
        const BInst<T>& B = I[fld_item(L, x, &i0, &is)];
        step_end_range<D2Q9, T, T, FORCE>(B.st, B.fbase, B.fstride, B.mbuf, B.h, B.sites, i0, is);  // accepted only
    }
}

// m^n = P f^n after a batched explicit march, for the instances that took steps
template <typename T>
__global__ void __launch_bounds__(kFieldThreads) k_bmoments_state(const BInst<T>* __restrict__ I,
                                                                  const BMap* __restrict__ M, BSteps steps) {
    const BList L = blist<1>(M, nullptr, 3);
    const int total = L.total();
    for (int x = blockIdx.x; x < total; x += gridDim.x) {
        size_t i0, is;
        const int i = fld_item(L, x, &i0, &is);
        if (steps.n[i] <= 0) continue;
        const BInst<T>& B = I[i];
        moments_state_range<D2Q9, T>(B.st, B.fbase, B.fstride, B.mbuf, B.sites, i0, is);
    }
}

// ---- control kernels: one thread per instance, one block ---------------------------------------

__global__ void k_btargets(const BMap* __restrict__ M, BSteps steps) {
    const int i = threadIdx.x;
    if (i < M->n_inst) set_target(M->st[i], steps.n[i]);
}

// Compact the instances whose thread passes on = true into the work list W, in batch order.  One
// block of kBatchMax threads, thread i = instance i: a block-wide inclusive scan (two warps) of
// (on, units, row blocks, column blocks, field blocks); an active instance writes its entry at its
// exclusive prefix, the last thread the totals.  Returns whether any instance is on.
__device__ inline bool build_work_list(const BMap* __restrict__ M, BAct* __restrict__ W, bool on) {
    static_assert(kBatchMax == 64, "the scan below covers two warps");
    __shared__ int s_tot[2][5];
    const int i = threadIdx.x, lane = i & 31, w = i >> 5;
    int v[5] = {0, 0, 0, 0, 0};
    if (on) {
        v[0] = 1;
        v[1] = M->unit_off[i + 1] - M->unit_off[i];
        v[2] = M->row_off[i + 1] - M->row_off[i];
        v[3] = M->col_off[i + 1] - M->col_off[i];
        v[4] = M->fld_off[i + 1] - M->fld_off[i];
    }
    int inc[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        int x = v[k];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        inc[k] = x;
        if (lane == 31) s_tot[w][k] = x;
    }
    __syncthreads();
    if (w == 1) {
#pragma unroll
        for (int k = 0; k < 5; ++k) inc[k] += s_tot[0][k];
    }
    if (on) {
        const int j = inc[0] - 1;
        W->inst[j] = i;
        W->unit_off[j] = inc[1] - v[1];
        W->row_off[j] = inc[2] - v[2];
        W->col_off[j] = inc[3] - v[3];
        W->fld_off[j] = inc[4] - v[4];
    }
    if (i == kBatchMax - 1) {
        const int n = inc[0];
        W->n_act = n;
        W->unit_off[n] = inc[1];
        W->row_off[n] = inc[2];
        W->col_off[n] = inc[3];
        W->fld_off[n] = inc[4];
    }
    return s_tot[0][0] + s_tot[1][0] > 0;
}

// first step of every instance that runs, the first round's work list and the loop condition
__global__ void k_bsetup(const BMap* __restrict__ M, BAct* __restrict__ W, cudaGraphConditionalHandle h_round) {
    const int i = threadIdx.x;
    bool go = false;
    if (i < M->n_inst) {
        DevState* st = M->st[i];
        if (arm_state(st)) {
            step_setup(st);
            go = true;
        }
    }
    go = build_work_list(M, W, go);
    if (threadIdx.x == 0) cudaGraphSetConditional(h_round, go ? 1u : 0u);
}

__global__ void k_bfinish(const BMap* __restrict__ M, BAct* __restrict__ W, cudaGraphConditionalHandle h_round) {
    const int i = threadIdx.x;
    bool active = false;
    if (i < M->n_inst) {
        DevState* st = M->st[i];
        if (st->accepted) {
            step_finish(st, M->iters[i], M->max_steps[i]);
            st->accepted = 0;  // k_bstep_end of the next round must not see this step again
        }
        active = inst_active(st);
    }
    active = build_work_list(M, W, active);
    if (threadIdx.x == 0) cudaGraphSetConditional(h_round, active ? 1u : 0u);
}

// explicit march: ping-pong from the accepted slot, `left` = steps still to take
__global__ void k_bex_setup(const BMap* __restrict__ M, BSteps steps) {
    const int i = threadIdx.x;
    if (i < M->n_inst) {
        DevState* st = M->st[i];
        const int n = steps.n[i];
        st->ex_a = st->slot_fn[0];
        st->ex_b = (st->slot_fn[0] + 1) % kNumFBuf;
        st->ex_loops_left = n > 0 ? n : 0;
    }
}

// subtract the steps of one loop round and set the loop condition (unroll = 0: condition only)
__global__ void k_bex_count(const BMap* __restrict__ M, int unroll, cudaGraphConditionalHandle h_ex) {
    const int i = threadIdx.x;
    bool go = false;
    if (i < M->n_inst) {
        DevState* st = M->st[i];
        const int left = st->ex_loops_left - unroll;
        st->ex_loops_left = left > 0 ? left : 0;
        go = left > 0;
    }
    go = __syncthreads_or(go);
    if (threadIdx.x == 0) cudaGraphSetConditional(h_ex, go ? 1u : 0u);
}

__global__ void k_bex_finish(const BMap* __restrict__ M, BSteps steps) {
    const int i = threadIdx.x;
    if (i < M->n_inst && steps.n[i] > 0) ex_finish(M->st[i], steps.n[i] & 1);
}

}  // namespace msc
