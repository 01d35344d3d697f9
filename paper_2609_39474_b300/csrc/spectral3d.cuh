// 3D periodic shadow correction (Section 3.2 with the third transform direction of Section 4.4):
// dm = F^{-1}[ chi(k) H(k)^{-1} F[P r] ] over the 4 residual-moment fields (r_p, r_mx, r_my, r_mz),
// with H(k) the 4 x 4 shadow matrix solved in closed form (Eq. schur).  Five kernels:
//   k_rowfft_fwd (x, real -> half spectrum 0 <= j_x <= n/4), k_ypass<fwd> (complex FFT along y),
//   k_zsolve (FFT along z, FP64 Schur solve at |j_y|, |j_z| <= n/4, inverse FFT along z; only the
//   n/2 + 1 masked j_y lines are visited), k_ypass<inv> (inverse along y reading only masked j_y),
//   k_rowfft_inv (Hermitian half spectrum -> real rows).
// Spectrum layout: spec[c][j_x][z][y] (the row index of the x pass is z n + y), so the y lines
// are contiguous and the z lines of G consecutive j_y are G-element contiguous segments.
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

// y pass: G consecutive z planes per block, one radix-16 butterfly per thread (G n / 16 <= 256)
__host__ __device__ inline int ypass_lines(int n) {
    int g = 4096 / n;
    return g > n ? n : (g < 1 ? 1 : g);
}
// z pass: 4 fields x G masked j_y lines per block (4 G n / 16 <= 768 FP32, 384 FP64).  G = 512 / n
// (FP32; 256 / n FP64): at N = 128, 561 blocks of 128 threads instead of 165 of 512, which left most
// SMs with one block of long serial FFT and FP64-solve chains (D3Q19 march 36.5 -> 34.8 ms alone)
template <typename T>
__host__ __device__ inline int zsolve_lines(int n) {
    int g = (sizeof(T) == 8 ? 256 : 512) / n;  // power of two
    return g < 1 ? 1 : g;
}

// x passes of the 3D correction: the 2D row rule with at most 8 row pairs per block (N = 128: 4096
// blocks of 64 threads instead of 1024 of 256; with the z pass above the D3Q19 march 36.5 -> 33.4 ms,
// same inner counts; 4 pairs per block, or 2 z lines per block, gained nothing more)
inline RowGeom row_geometry3(int n) {
    RowGeom rg = row_geometry(n, 4, n * n);
    if (rg.P > 8) {
        rg.blocks = rg.blocks * rg.P / 8;
        rg.P = 8;
        rg.threads = (8 * n / 16 + 31) / 32 * 32;
        if (rg.threads < 32) rg.threads = 32;
    }
    return rg;
}

template <typename T, bool INV>
__global__ void __launch_bounds__(kFftThreads) k_ypass(Spec2Args<T> A) {
    wait_for_predecessor();
    if (spec_gated_off(A)) return;
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = A.n, logn = A.logn, plen = padded_len(n);
    const int G = A.G;
    const int zch = n / G;
    const int line0 = blockIdx.x * G;         // (c * nx4 + jx) * n + z0, G divides n
    C* base = A.spec + (size_t)line0 * n;     // G contiguous lines of length n
    (void)zch;
    // binary32: two consecutive y per thread, one 16-byte access (the lines are contiguous and the
    // spectrum 16-byte aligned; y even keeps both in one padded 16-block of s)
    constexpr bool VEC = sizeof(C) == 8;
    const int lv = VEC ? 1 : 0;
    auto kept = [&](int y) {
        const int ys = y <= n / 2 ? y : y - n;
        return !INV || (ys <= n / 4 && ys >= -(n / 4));
    };
#pragma unroll 8
    for (int t = threadIdx.x; t < (G * n >> lv); t += blockDim.x) {
        const int e = t << lv;  // first element
        const int g = e >> logn;
        const int y = e & (n - 1);
        if constexpr (VEC) {
            const bool k0 = kept(y), k1 = kept(y + 1);
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k0 || k1) w = *reinterpret_cast<const float4*>(base + e);
            C z0, z1;
            z0.x = k0 ? w.x : T(0); z0.y = k0 ? w.y : T(0);
            z1.x = k1 ? w.z : T(0); z1.y = k1 ? w.w : T(0);
            s[g * plen + pad(y)] = z0;
            s[g * plen + pad(y) + 1] = z1;
        } else {
            C z;
            z.x = T(0); z.y = T(0);
            if (kept(y)) z = base[e];
            s[g * plen + pad(y)] = z;
        }
    }
    __syncthreads();
    fft_stockham<C, INV>(s, n, logn, G, A.tw);
    for (int t = threadIdx.x; t < (G * n >> lv); t += blockDim.x) {
        const int e = t << lv;
        const int g = e >> logn;
        const int y = e & (n - 1);
        if constexpr (VEC) {
            const C z0 = s[g * plen + pad(y)], z1 = s[g * plen + pad(y) + 1];
            *reinterpret_cast<float4*>(base + e) = make_float4(z0.x, z0.y, z1.x, z1.y);
        } else {
            base[e] = s[g * plen + pad(y)];
        }
    }
}

// one block per (j_x, chunk of G masked j_y): the z lines of all 4 fields
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 384 : 768) k_zsolve(Spec2Args<T> A) {
    wait_for_predecessor();
    if (spec_gated_off(A)) return;
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);  // line (c, g) at (c G + g) plen
    const int n = A.n, logn = A.logn, plen = padded_len(n);
    const int nx4 = n / 4 + 1, ny = n / 2 + 1;
    const int G = A.G;  // a power of two
    const int lg = __ffs(G) - 1;
    const int nch = (ny + G - 1) / G;
    const int jx = blockIdx.x / nch;
    const int jyk0 = (blockIdx.x - jx * nch) * G;
    const int ng = min(G, ny - jyk0);
    const size_t n2 = (size_t)n * n;
    const size_t fstride = (size_t)nx4 * n2;
    C* sp = A.spec + (size_t)jx * n2;  // + c * fstride + z * n + jy
    // binary32 (G >= 2): lines g, g + 1 (g even) hold adjacent j_y values, one 16-byte access
    constexpr int lv = sizeof(C) == 8 ? 1 : 0;
#pragma unroll 4
    for (int t = threadIdx.x; t < (4 * G * n >> lv); t += blockDim.x) {
        const int e = t << lv;
        const int g = e & (G - 1);
        const int cz = e >> lg;
        const int z = cz & (n - 1);
        const int c = cz >> logn;
        const int jy = (jyk0 + g - n / 4) & (n - 1);
        if constexpr (lv == 1) {
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g < ng) w = *reinterpret_cast<const float4*>(sp + c * fstride + (size_t)z * n + jy);
            s[(c * G + g) * plen + pad(z)] = make_float2(w.x, w.y);
            s[(c * G + g + 1) * plen + pad(z)] = g + 1 < ng ? make_float2(w.z, w.w) : make_float2(0.f, 0.f);
        } else {
            C v;
            v.x = T(0); v.y = T(0);
            if (g < ng) v = sp[c * fstride + (size_t)z * n + jy];
            s[(c * G + g) * plen + pad(z)] = v;
        }
    }
    __syncthreads();
    fft_stockham<C, false>(s, n, logn, 4 * G, A.tw);
    const double a = A.st ? A.st->a : A.a;
    const double* tab = solve_table(A.coef, A.st, 3, n);
    const double two_pi_n = A.kunit;
    const double scale = A.nscale;
    for (int t = threadIdx.x; t < G * n; t += blockDim.x) {
        const int g = t >> logn;
        const int jz = t & (n - 1);
        const int jzs = jz <= n / 2 ? jz : jz - n;
        C* v[4] = {s + (0 * G + g) * plen + pad(jz), s + (1 * G + g) * plen + pad(jz),
                   s + (2 * G + g) * plen + pad(jz), s + (3 * G + g) * plen + pad(jz)};
        if (jzs > n / 4 || jzs < -(n / 4) || g >= ng) {
            C zz; zz.x = T(0); zz.y = T(0);
            *v[0] = zz; *v[1] = zz; *v[2] = zz; *v[3] = zz;
            continue;
        }
        const int jys = jyk0 + g - n / 4;
        const double kv[3] = {two_pi_n * (double)jx, two_pi_n * (double)jys, two_pi_n * (double)jzs};
        double cf[4];
        if (tab) {
            const size_t mi = (size_t)jx + (size_t)nx4 * ((size_t)(jyk0 + g) + (size_t)ny * (jzs + n / 4));
            const double* tt = tab + 4 * mi;
            cf[0] = tt[0]; cf[1] = tt[1]; cf[2] = tt[2]; cf[3] = tt[3];
        } else {
            solve_coefficients(a, A.nu, kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2], scale, cf);
        }
        schur_apply<C, 3, true>(v, kv, cf);
    }
    __syncthreads();
    fft_stockham<C, true>(s, n, logn, 4 * G, A.tw);
    for (int t = threadIdx.x; t < (4 * G * n >> lv); t += blockDim.x) {
        const int e = t << lv;
        const int g = e & (G - 1);
        const int cz = e >> lg;
        const int z = cz & (n - 1);
        const int c = cz >> logn;
        if (g >= ng) continue;
        const int jy = (jyk0 + g - n / 4) & (n - 1);
        C* d = sp + c * fstride + (size_t)z * n + jy;
        const C z0 = s[(c * G + g) * plen + pad(z)];
        if constexpr (lv == 1) {
            if (g + 1 < ng) {
                const C z1 = s[(c * G + g + 1) * plen + pad(z)];
                *reinterpret_cast<float4*>(d) = make_float4(z0.x, z0.y, z1.x, z1.y);
            } else {
                *d = z0;
            }
        } else {
            *d = z0;
        }
    }
}

template <typename T>
inline void spectral3_launches(int n, LaunchDesc* L) {
    using C = typename Cplx<T>::type;
    const int nx4 = n / 4 + 1, ny = n / 2 + 1;
    const RowGeom rg = row_geometry3(n);
    const size_t rsm = spec_row_smem<T>(n, rg.P);
    const int yg = ypass_lines(n), zg = zsolve_lines<T>(n);
    const int yth = ((yg * n / 16 + 31) / 32) * 32;
    const int zth = ((4 * zg * n / 16 + 31) / 32) * 32;
    const size_t ysm = (size_t)yg * padded_len(n) * sizeof(C);
    const size_t zsm = (size_t)4 * zg * padded_len(n) * sizeof(C);
    const int zblocks = nx4 * ((ny + zg - 1) / zg);
    L[0] = {(const void*)k_rowfft_fwd<T>, dim3(rg.blocks), dim3(rg.threads), rsm};
    L[1] = {(const void*)k_ypass<T, false>, dim3(4 * nx4 * n / yg), dim3(yth < 32 ? 32 : yth), ysm};
    L[2] = {(const void*)k_zsolve<T>, dim3(zblocks), dim3(zth < 32 ? 32 : zth), zsm};
    L[3] = {(const void*)k_ypass<T, true>, dim3(4 * nx4 * n / yg), dim3(yth < 32 ? 32 : yth), ysm};
    L[4] = {(const void*)k_rowfft_inv<T>, dim3(rg.blocks), dim3(rg.threads), rsm};
}

// The five launches take one argument block whose P and G fields differ per pass: the row
// passes read P, the y pass and the z pass read G.  The launchers below set both.
template <typename T>
inline void spec3_pass_args(int n, Spec2Args<T>* A, int pass) {
    A->P = row_geometry3(n).P;
    A->G = pass == 2 ? zsolve_lines<T>(n) : ypass_lines(n);
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
                               T* dm, const typename Cplx<T>::type* tw, const DevState* st,
                               const double* coef = nullptr) {
    Spec2Args<T> A;
    memset(&A, 0, sizeof(A));
    A.coef = coef;
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
    A.kunit = 6.283185307179586476925286766559 / (double)n;
    A.nscale = 1.0 / ((double)n * (double)n * (double)n);  // 3D; the 2D callers replace it
    A.st = st;
    spec3_pass_args<T>(n, &A, 0);
    return A;
}

template <typename T>
int launch_spectral3(int n, int logn, double a, double nu, const T* pr, typename Cplx<T>::type* spec, T* dm,
                     const typename Cplx<T>::type* tw, cudaStream_t stream) {
    if (set_spec3_smem_limits<T>(n)) return MSC_ERR_CUDA;
    Spec2Args<T> A = spec3_args<T>(n, logn, a, nu, pr, spec, dm, tw, nullptr);
    LaunchDesc L[5];
    spectral3_launches<T>(n, L);
    for (int i = 0; i < 5; ++i) {
        spec3_pass_args<T>(n, &A, i);
        void* args[] = {&A};
        if (cudaLaunchKernel(L[i].fn, L[i].grid, L[i].block, args, L[i].smem, stream) != cudaSuccess)
            return MSC_ERR_CUDA;
    }
    return MSC_OK;
}

}  // namespace msc
