// C ABI of the full-symbol reference correction (kernels in fullsym2d.cuh).  Included at the end of
// msclbm.cu (it uses that file's launch helpers).
#pragma once

#include "fullsym2d.cuh"

namespace {

struct FsScratch {
    void* tw;
    void* spec;
};

FsScratch fs_scratch(int n, int precision, void* base) {
    const size_t cb = precision == MSC_FP64 ? 16 : 8;
    unsigned char* b = (unsigned char*)base;
    FsScratch s;
    s.tw = b;
    s.spec = b + align_up((size_t)n * cb, 256);
    return s;
}

template <typename T>
int run_full_symbol(int n, double a, double wp, double wm, const void* f, const void* ft, void* out, void* scratch,
                    cudaStream_t stream) {
    using C = typename Cplx<T>::type;
    const FsScratch S = fs_scratch(n, sizeof(T) == 8 ? MSC_FP64 : MSC_FP32, scratch);
    FsArgs<T> A;
    memset(&A, 0, sizeof(A));
    A.f = (const T*)f;
    A.ft = (const T*)ft;
    A.out = (T*)out;
    A.spec = (C*)S.spec;
    A.tw = (const C*)S.tw;
    A.n = n;
    A.logn = ilog2(n);
    const RowGeom rg = row_geometry(n, 9, n);
    A.P = rg.P;
    A.d1 = (2.0 - wp - wm) / 2.0;
    A.d2 = (wm - wp) / 2.0;
    A.wp = wp;
    A.bp = (wp - a * (1.0 - wp / 2.0)) / (1.0 + a / 2.0);
    A.bm = (wm - a * (1.0 - wm / 2.0)) / (1.0 + a / 2.0);
    A.nscale = 1.0 / ((double)n * n);
    const size_t row_smem = spec_row_smem<T>(n, rg.P);
    const size_t col_smem = fs_col_smem<T>(n);
    CK(cudaFuncSetAttribute(k_fs_rowfwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));
    CK(cudaFuncSetAttribute(k_fs_rowinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));
    const bool large = fs_col_threads(n) > kFsColThreadsSmall;
    const void* col = large ? (const void*)k_fs_col<T, true> : (const void*)k_fs_col<T, false>;
    CK(cudaFuncSetAttribute(col, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem));
    k_twiddles<C><<<(n + 255) / 256, 256, 0, stream>>>((C*)S.tw, n);
    k_fs_rowfwd<T><<<rg.blocks, rg.threads, row_smem, stream>>>(A);
    if (large)
        k_fs_col<T, true><<<n / 2 + 1, fs_col_threads(n), col_smem, stream>>>(A);
    else
        k_fs_col<T, false><<<n / 2 + 1, fs_col_threads(n), col_smem, stream>>>(A);
    k_fs_rowinv<T><<<rg.blocks, rg.threads, row_smem, stream>>>(A);
    CK(cudaGetLastError());
    return MSC_OK;
}

}  // namespace

extern "C" {

size_t msc_full_symbol_scratch_bytes(int n, int precision) {
    if (precision != MSC_FP64 && precision != MSC_FP32) return 0;
    if (!is_pow2(n) || n < 8 || n > MSC_FULL_SYMBOL_MAX_N) return 0;
    const size_t cb = precision == MSC_FP64 ? 16 : 8;
    return align_up((size_t)n * cb, 256) + align_up((size_t)9 * (n / 2 + 1) * n * cb, 256);
}

int msc_full_symbol_correct(int n, int precision, double a, double omega_p, double omega_m, const void* f,
                            const void* f_swept, void* f_out, void* scratch, size_t scratch_bytes, void* stream) {
    const size_t need = msc_full_symbol_scratch_bytes(n, precision);
    if (need == 0 || !f || !f_swept || !f_out || !scratch || scratch_bytes < need || !(a > 0.0) ||
        !(omega_p > 0.0 && omega_p < 2.0) || !(omega_m > 0.0 && omega_m < 2.0))
        return MSC_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(scratch) % 256) return MSC_ERR_ARG;
    if (precision == MSC_FP64)
        return run_full_symbol<double>(n, a, omega_p, omega_m, f, f_swept, f_out, scratch, (cudaStream_t)stream);
    return run_full_symbol<float>(n, a, omega_p, omega_m, f, f_swept, f_out, scratch, (cudaStream_t)stream);
}

}  // extern "C"
