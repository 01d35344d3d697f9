// Allocation-free variant of the D2Q9 fused sweep stage call (msc_sweep_d2q9_noalloc).
//
// msc_sweep needs a caller-provided scratch buffer for its residual-norm reduction (one partial
// sum per block plus a completion counter).  Some callers cannot provide one: host frameworks
// that own the whole device-memory budget and forbid plugins from calling cudaMalloc, bindings
// that can pass only the input and output arrays, and latency-critical loops in which a
// cudaMalloc/cudaFree pair would implicitly synchronise the device.  For them this entry point
// keeps the reduction scratch in a fixed file-scope device array instead.  The array exists once
// per device that loads the library and stays resident until the process exits.
//
// This file is included once, by msclbm.cu, so the array and its set-up live in that single
// translation unit.
#pragma once

#include "common.cuh"
#include "sweep2d.cuh"

namespace msc {

// Largest sweep grid the static scratch serves: 4096 blocks, which covers every D2Q9 lattice up
// to n = 4096 (n = 4096 launches 2192 blocks).  Layout: bytes [0, 256) hold the completion
// counter, then one double per block.
constexpr int kNoAllocMaxBlocks = 4096;
constexpr size_t kNoAllocBytes = 256 + (size_t)kNoAllocMaxBlocks * sizeof(double);

static __device__ __align__(256) unsigned char g_sweep_scratch[kNoAllocBytes];

// every D2Q9 lattice that the entry point accepts (n = 8 .. 4096, powers of two) launches at most
// kNoAllocMaxBlocks sweep blocks: checked at compile time against the sweep's own geometry rule
constexpr bool noalloc_covers_all_lattices() {
    for (int n = 8; n <= 4096; n *= 2)
        if (sweep2_geometry(n).blocks > kNoAllocMaxBlocks) return false;
    return true;
}
static_assert(noalloc_covers_all_lattices(), "the static sweep scratch is too small for some lattice");

// Device address of g_sweep_scratch on the current device.  In host code the symbol itself is only
// a host-side stand-in; kernels must be given the address that cudaGetSymbolAddress returns for the
// current device.  The lookup is repeated on every call (a host-side table lookup after the first
// call on a device has loaded the module), so the address stays right after a device reset, when
// the module may be loaded again at another address.
inline int noalloc_scratch(void** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sweep_scratch) != cudaSuccess || !p) return MSC_ERR_CUDA;
    *out = p;
    return MSC_OK;
}

template <typename T>
int sweep2_noalloc(int n, double a, const void* fin, const void* dm, const void* h, void* fout, void* pr,
                   double* sumsq, cudaStream_t stream) {
    const Sweep2Geom g = sweep2_geometry(n);
    if (g.blocks > kNoAllocMaxBlocks) return MSC_ERR_ARG;
    void* base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc != MSC_OK) return rc;
    unsigned int* counter = reinterpret_cast<unsigned int*>(base);
    // the counter must start at zero; the partials are fully rewritten by every call
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), stream) != cudaSuccess) return MSC_ERR_CUDA;
    Sweep2Args<T> A;
    memset(&A, 0, sizeof(A));
    A.fin = (const T*)fin;
    A.dm = (const T*)dm;
    A.h = (const T*)h;
    A.fout = (T*)fout;
    A.pr = (T*)pr;
    A.a = a;
    A.inv = 1.0 / (1.0 + a / 2.0);
    A.fscale = 1.0;
    A.lift = dm != nullptr;
    A.sumsq_out = sumsq;
    A.partial = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + 256);
    A.counter = counter;
    A.n = n;
    A.nstrips = g.nstrips;
    A.hb = g.hb;
    A.nrowblk = g.nrowblk;
    k_sweep2<T, T, false, false><<<g.blocks, kSweepWarps * 32, 0, stream>>>(A);
    return cudaGetLastError() == cudaSuccess ? MSC_OK : MSC_ERR_CUDA;
}

}  // namespace msc

extern "C" int msc_sweep_d2q9_noalloc(int n, int precision, double a, const void* f_in, const void* dm,
                                      const void* h, void* f_out, void* pr_out, double* sumsq_out,
                                      void* stream) {
    if (!msc::valid_lattice(2, n, precision) || precision == MSC_FP16 || !f_in || !h || !f_out || !pr_out ||
        !sumsq_out || f_in == f_out || !(a >= 0.0))
        return MSC_ERR_ARG;
    if (precision == MSC_FP64)
        return msc::sweep2_noalloc<double>(n, a, f_in, dm, h, f_out, pr_out, sumsq_out, (cudaStream_t)stream);
    return msc::sweep2_noalloc<float>(n, a, f_in, dm, h, f_out, pr_out, sumsq_out, (cudaStream_t)stream);
}
