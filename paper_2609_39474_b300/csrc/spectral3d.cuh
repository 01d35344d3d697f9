// 3D periodic shadow correction (Section 3.2 with the third transform direction of Section 4.4):
// dm = F^{-1}[ chi(k) H(k)^{-1} F[P r] ] over the 4 residual-moment fields (r_p, r_mx, r_my, r_mz),
// with H(k) the 4 x 4 shadow matrix solved in closed form (Eq. schur).  Five kernels:
//   k_rowfft_fwd (x, real -> half spectrum 0 <= j_x <= n/4), k_ypass<fwd> (complex FFT along y),
//   k_zsolve (FFT along z, FP64 Schur solve at |j_y|, |j_z| <= n/4, inverse FFT along z; only the
//   n/2 + 1 masked j_y planes are visited), k_ypass<inv> (inverse along y reading only masked j_y),
//   k_rowfft_inv (Hermitian half spectrum -> real rows).
// Spectrum layout: spec[c][z][y][j_x], row stride n/4 + 1.
#pragma once

#include "common.cuh"
#include "fft.cuh"
#include "spectral2d.cuh"

namespace msc {

struct LaunchDesc {
    const void* fn;
    dim3 grid, block;
    size_t smem;
};

inline size_t spec3_bytes(int n, size_t celem) { return (size_t)4 * n * n * (n / 4 + 1) * celem; }

// j_x columns per block so that one block's shared arrays stay near 32 KB
template <typename T>
__host__ __device__ inline int ypass_cols(int n) {
    int g = (int)(32768 / ((size_t)n * sizeof(typename Cplx<T>::type)));
    const int nx4 = n / 4 + 1;
    if (g < 1) g = 1;
    if (g > nx4) g = nx4;
    return g;
}
template <typename T>
__host__ __device__ inline int zsolve_cols(int n) {
    int g = (int)(65536 / ((size_t)4 * n * sizeof(typename Cplx<T>::type)));
    const int nx4 = n / 4 + 1;
    if (g < 1) g = 1;
    if (g > nx4) g = nx4;
    return g;
}

// one block per (field c, plane z, chunk of G j_x columns): transform along y
template <typename T, bool INV>
__global__ void __launch_bounds__(kFftThreads) k_ypass(Spec2Args<T> A) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = A.n, logn = A.logn;
    const int nx4 = n / 4 + 1;
    const int G = ypass_cols<T>(n);
    const int nchunk = (nx4 + G - 1) / G;
    const int chunk = blockIdx.x % nchunk;
    const int plane = blockIdx.x / nchunk;  // c * n + z
    const int jx0 = chunk * G;
    const int ng = min(G, nx4 - jx0);
    C* base = A.spec + (size_t)plane * n * nx4;
    for (int t = threadIdx.x; t < G * n; t += blockDim.x) {
        const int g = t >> logn;
        const int y = t & (n - 1);
        C z;
        z.x = T(0); z.y = T(0);
        if (g < ng) {
            const int ys = y <= n / 2 ? y : y - n;
            if (!INV || (ys <= n / 4 && ys >= -(n / 4))) z = base[(size_t)y * nx4 + jx0 + g];
        }
        if (INV) s[g * n + y] = z;
        else s[g * n + bitrev(y, logn)] = z;
    }
    __syncthreads();
    if (INV) fft_dif(s, n, logn, G, A.tw, true);
    else fft_dit(s, n, logn, G, A.tw, false);
    for (int t = threadIdx.x; t < G * n; t += blockDim.x) {
        const int g = t >> logn;
        const int i = t & (n - 1);
        if (g >= ng) continue;
        const int y = INV ? bitrev(i, logn) : i;
        base[(size_t)y * nx4 + jx0 + g] = s[t];
    }
}

// one block per (masked j_y, chunk of G j_x columns): all 4 fields along z
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_zsolve(Spec2Args<T> A) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);  // [4][G][n]
    const int n = A.n, logn = A.logn;
    const int nx4 = n / 4 + 1;
    const int G = zsolve_cols<T>(n);
    const int nchunk = (nx4 + G - 1) / G;
    const int chunk = blockIdx.x % nchunk;
    const int jyk = blockIdx.x / nchunk;         // 0 .. n/2
    const int jys = jyk - n / 4;                  // signed j_y in [-n/4, n/4]
    const int jy = jys & (n - 1);
    const int jx0 = chunk * G;
    const int ng = min(G, nx4 - jx0);
    const size_t zstride = (size_t)n * nx4;
    const size_t fstride = (size_t)n * n * nx4;
    C* sp = A.spec;
    for (int t = threadIdx.x; t < 4 * G * n; t += blockDim.x) {
        const int z = t & (n - 1);
        const int cg = t >> logn;  // c * G + g
        const int c = cg / G;
        const int g = cg - c * G;
        C v;
        v.x = T(0); v.y = T(0);
        if (g < ng) v = sp[c * fstride + (size_t)z * zstride + (size_t)jy * nx4 + jx0 + g];
        s[cg * n + bitrev(z, logn)] = v;
    }
    __syncthreads();
    fft_dit(s, n, logn, 4 * G, A.tw, false);
    const double a = A.st ? ((const volatile DevState*)A.st)->a : A.a;
    const double nu = A.nu;
    const double two_pi_n = 6.283185307179586476925286766559 / (double)n;
    const double ky = two_pi_n * (double)jys;
    const double scale = 1.0 / ((double)n * (double)n * (double)n);
    for (int t = threadIdx.x; t < G * n; t += blockDim.x) {
        const int g = t >> logn;
        const int jz = t & (n - 1);
        const int jzs = jz <= n / 2 ? jz : jz - n;
        C* p0 = s + (0 * G + g) * n + jz;
        C* p1 = s + (1 * G + g) * n + jz;
        C* p2 = s + (2 * G + g) * n + jz;
        C* p3 = s + (3 * G + g) * n + jz;
        if (jzs > n / 4 || jzs < -(n / 4) || g >= ng) {
            C zz; zz.x = T(0); zz.y = T(0);
            *p0 = zz; *p1 = zz; *p2 = zz; *p3 = zz;
            continue;
        }
        const double kx = two_pi_n * (double)(jx0 + g);
        const double kz = two_pi_n * (double)jzs;
        const double k2 = kx * kx + ky * ky + kz * kz;
        const double dv = a + nu * k2;
        const double idv = 1.0 / dv;
        const double iD = 1.0 / (a + kCs2 * k2 * idv);
        const double rpx = (double)p0->x, rpy = (double)p0->y;
        const double r1x = (double)p1->x, r1y = (double)p1->y;
        const double r2x = (double)p2->x, r2y = (double)p2->y;
        const double r3x = (double)p3->x, r3y = (double)p3->y;
        const double krx = kx * r1x + ky * r2x + kz * r3x;
        const double kry = kx * r1y + ky * r2y + kz * r3y;
        const double dpx = (rpx + kry * idv) * iD;
        const double dpy = (rpy - krx * idv) * iD;
        C v;
        v.x = (T)(dpx * scale); v.y = (T)(dpy * scale); *p0 = v;
        v.x = (T)((r1x + kCs2 * kx * dpy) * idv * scale); v.y = (T)((r1y - kCs2 * kx * dpx) * idv * scale); *p1 = v;
        v.x = (T)((r2x + kCs2 * ky * dpy) * idv * scale); v.y = (T)((r2y - kCs2 * ky * dpx) * idv * scale); *p2 = v;
        v.x = (T)((r3x + kCs2 * kz * dpy) * idv * scale); v.y = (T)((r3y - kCs2 * kz * dpx) * idv * scale); *p3 = v;
    }
    __syncthreads();
    fft_dif(s, n, logn, 4 * G, A.tw, true);
    for (int t = threadIdx.x; t < 4 * G * n; t += blockDim.x) {
        const int i = t & (n - 1);
        const int cg = t >> logn;
        const int c = cg / G;
        const int g = cg - c * G;
        if (g >= ng) continue;
        const int z = bitrev(i, logn);
        sp[c * fstride + (size_t)z * zstride + (size_t)jy * nx4 + jx0 + g] = s[t];
    }
}

template <typename T>
inline void spectral3_launches(int n, LaunchDesc* L) {
    using C = typename Cplx<T>::type;
    const int nx4 = n / 4 + 1;
    const int rows = n * n;
    const size_t rsm = (size_t)ffts_per_block(n) * n * sizeof(C);
    const int yg = ypass_cols<T>(n), zg = zsolve_cols<T>(n);
    const int ych = (nx4 + yg - 1) / yg, zch = (nx4 + zg - 1) / zg;
    L[0] = {(const void*)k_rowfft_fwd<T>, dim3(spec_row_blocks(n, 4, rows)), dim3(kFftThreads), rsm};
    L[1] = {(const void*)k_ypass<T, false>, dim3(4 * n * ych), dim3(kFftThreads), (size_t)yg * n * sizeof(C)};
    L[2] = {(const void*)k_zsolve<T>, dim3((n / 2 + 1) * zch), dim3(kFftThreads), (size_t)4 * zg * n * sizeof(C)};
    L[3] = {(const void*)k_ypass<T, true>, dim3(4 * n * ych), dim3(kFftThreads), (size_t)yg * n * sizeof(C)};
    L[4] = {(const void*)k_rowfft_inv<T>, dim3(spec_row_blocks(n, 4, rows)), dim3(kFftThreads), rsm};
}

template <typename T>
int set_spec3_smem_limits(int n) {
    LaunchDesc L[5];
    spectral3_launches<T>(n, L);
    for (int i = 0; i < 5; ++i)
        if (cudaFuncSetAttribute(L[i].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L[i].smem) != cudaSuccess)
            return 1;
    return 0;
}

template <typename T>
inline Spec2Args<T> spec3_args(int n, int logn, double a, double nu, const T* pr, typename Cplx<T>::type* spec,
                               T* dm, const typename Cplx<T>::type* tw, const DevState* st) {
    Spec2Args<T> A;
    memset(&A, 0, sizeof(A));
    A.pr = pr;
    A.spec = spec;
    A.dm = dm;
    A.tw = tw;
    A.n = n;
    A.logn = logn;
    A.nf = 4;
    A.rows = n * n;
    A.a = a;
    A.nu = nu;
    A.st = st;
    return A;
}

template <typename T>
int launch_spectral3(int n, int logn, double a, double nu, const T* pr, typename Cplx<T>::type* spec, T* dm,
                     const typename Cplx<T>::type* tw, cudaStream_t stream) {
    if (set_spec3_smem_limits<T>(n)) return MSC_ERR_CUDA;
    Spec2Args<T> A = spec3_args<T>(n, logn, a, nu, pr, spec, dm, tw, nullptr);
    LaunchDesc L[5];
    spectral3_launches<T>(n, L);
    void* args[] = {&A};
    for (int i = 0; i < 5; ++i)
        if (cudaLaunchKernel(L[i].fn, L[i].grid, L[i].block, args, L[i].smem, stream) != cudaSuccess)
            return MSC_ERR_CUDA;
    return MSC_OK;
}

}  // namespace msc
