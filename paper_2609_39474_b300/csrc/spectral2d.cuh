// 2D periodic shadow correction (Section 3.2, Eqs. shadow-cont .. shadow-update):
//   dm = F^{-1}[ chi(k) H(k)^{-1} F[P r] ]
// as three kernels over the 3 residual-moment fields (r_p, r_mx, r_my):
//   k_rowfft_fwd   real rows -> half spectrum along x, keeping 0 <= j_x <= n/4 (the mask,
//                  Eq. shadow-mask; negative j_x follow from Hermitian symmetry).  Two real rows
//                  share one complex FFT.
//   k_colsolve     per kept j_x column: FFT along y, closed-form Schur solve (Eq. schur) in FP64
//                  at |j_y| <= n/4, zero elsewhere, scaling by 1/N_Omega, inverse FFT along y.
//   k_rowfft_inv   Hermitian-extended half spectrum -> real rows (two rows per complex FFT).
// Half-spectrum layout: spec[c][y][j_x], c in {p, x, y}, j_x in [0, n/4], row stride n/4 + 1.
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace msc {

constexpr int kFftThreads = 256;
constexpr double kCs2 = 1.0 / 3.0;

// number of length-n transforms one block runs together so that every thread has butterflies
__host__ __device__ inline int ffts_per_block(int n) {
    const int p = (2 * kFftThreads) / n;
    return p < 1 ? 1 : p;
}

template <typename T>
struct Spec2Args {
    const T* pr;       // 3 x n^2 residual moments
    typename Cplx<T>::type* spec;  // 3 x n x (n/4+1)
    T* dm;             // 3 x n^2 correction
    const typename Cplx<T>::type* tw;
    int n, logn;
    int nf;              // number of fields (d + 1)
    int rows;            // rows of length n per field (n in 2D, n^2 in 3D)
    double a, nu;
    const DevState* st;  // graph mode: a from the state
};

// rows (c, y) and (c, y+1) of the 3 fields form one complex row; 3n/2 row pairs in total
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_rowfft_fwd(Spec2Args<T> A) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = A.n, logn = A.logn;
    const int nx4 = n / 4 + 1;
    const int P = ffts_per_block(n);
    const int hr = A.rows / 2;
    const int npairs = A.nf * hr;
    const int pair0 = blockIdx.x * P;
    const size_t NN = (size_t)n * A.rows;
    // load with bit-reversed placement
    for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
        const int p = t >> logn;
        const int x = t & (n - 1);
        const int pair = pair0 + p;
        C z;
        z.x = T(0); z.y = T(0);
        if (pair < npairs) {
            const int c = pair / hr;
            const int y = 2 * (pair - c * hr);
            const T* row = A.pr + c * NN + (size_t)y * n;
            z.x = row[x];
            z.y = row[n + x];
        }
        s[p * n + bitrev(x, logn)] = z;
    }
    __syncthreads();
    fft_dit(s, n, logn, P, A.tw, false);
    // split the two real transforms and keep 0 <= j <= n/4
    for (int t = threadIdx.x; t < P * nx4; t += blockDim.x) {
        const int p = t / nx4;
        const int jx = t - p * nx4;
        const int pair = pair0 + p;
        if (pair >= npairs) continue;
        const int c = pair / hr;
        const int y = 2 * (pair - c * hr);
        const C zj = s[p * n + jx];
        const C zm = s[p * n + ((n - jx) & (n - 1))];
        C xa, xb;
        xa.x = T(0.5) * (zj.x + zm.x);
        xa.y = T(0.5) * (zj.y - zm.y);
        // (zj - conj(zm)) / (2i)
        xb.x = T(0.5) * (zj.y + zm.y);
        xb.y = T(-0.5) * (zj.x - zm.x);
        C* out = A.spec + (size_t)c * A.rows * nx4;
        out[(size_t)y * nx4 + jx] = xa;
        out[(size_t)(y + 1) * nx4 + jx] = xb;
    }
}

// one block per kept j_x column, all three fields
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_colsolve(Spec2Args<T> A) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = A.n, logn = A.logn;
    const int nx4 = n / 4 + 1;
    const int jx = blockIdx.x;
    C* sp = A.spec;
    for (int t = threadIdx.x; t < 3 * n; t += blockDim.x) {
        const int c = t >> logn;
        const int y = t & (n - 1);
        s[c * n + bitrev(y, logn)] = sp[((size_t)c * n + y) * nx4 + jx];
    }
    __syncthreads();
    fft_dit(s, n, logn, 3, A.tw, false);
    // Schur solve of H(k) [dp, du] = [r_p, r_m] at every masked wavevector (Eq. schur)
    const double a = A.st ? ((const volatile DevState*)A.st)->a : A.a;
    const double nu = A.nu;
    const double two_pi_n = 6.283185307179586476925286766559 / (double)n;
    const double kx = two_pi_n * (double)jx;
    const double scale = 1.0 / ((double)n * (double)n);
    for (int jy = threadIdx.x; jy < n; jy += blockDim.x) {
        const int jys = jy <= n / 2 ? jy : jy - n;
        C* p0 = s + jy;
        C* p1 = s + n + jy;
        C* p2 = s + 2 * n + jy;
        if (jys > n / 4 || jys < -(n / 4)) {
            C z; z.x = T(0); z.y = T(0);
            *p0 = z; *p1 = z; *p2 = z;
            continue;
        }
        const double ky = two_pi_n * (double)jys;
        const double k2 = kx * kx + ky * ky;
        const double dv = a + nu * k2;
        const double idv = 1.0 / dv;
        const double iD = 1.0 / (a + kCs2 * k2 * idv);
        const double rpx = (double)p0->x, rpy = (double)p0->y;
        const double rxx = (double)p1->x, rxy = (double)p1->y;
        const double ryx = (double)p2->x, ryy = (double)p2->y;
        // kr = k . r_m (complex)
        const double krx = kx * rxx + ky * ryx, kry = kx * rxy + ky * ryy;
        // dp = (r_p - i kr / dv) / D ;  -i z = (z.y, -z.x)
        const double dpx = (rpx + kry * idv) * iD;
        const double dpy = (rpy - krx * idv) * iD;
        // du = (r_m - cs2 i k dp) / dv ;  i dp = (-dp.y, dp.x)
        const double uxx = (rxx + kCs2 * kx * dpy) * idv;
        const double uxy = (rxy - kCs2 * kx * dpx) * idv;
        const double uyx = (ryx + kCs2 * ky * dpy) * idv;
        const double uyy = (ryy - kCs2 * ky * dpx) * idv;
        C z;
        z.x = (T)(dpx * scale); z.y = (T)(dpy * scale); *p0 = z;
        z.x = (T)(uxx * scale); z.y = (T)(uxy * scale); *p1 = z;
        z.x = (T)(uyx * scale); z.y = (T)(uyy * scale); *p2 = z;
    }
    __syncthreads();
    fft_dif(s, n, logn, 3, A.tw, true);
    for (int t = threadIdx.x; t < 3 * n; t += blockDim.x) {
        const int c = t >> logn;
        const int i = t & (n - 1);
        sp[((size_t)c * n + bitrev(i, logn)) * nx4 + jx] = s[t];
    }
}

template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_rowfft_inv(Spec2Args<T> A) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = A.n, logn = A.logn;
    const int nx4 = n / 4 + 1;
    const int P = ffts_per_block(n);
    const int hr = A.rows / 2;
    const int npairs = A.nf * hr;
    const int pair0 = blockIdx.x * P;
    const size_t NN = (size_t)n * A.rows;
    for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
        const int p = t >> logn;
        const int j = t & (n - 1);
        const int pair = pair0 + p;
        C z;
        z.x = T(0); z.y = T(0);
        if (pair < npairs) {
            const int c = pair / hr;
            const int y = 2 * (pair - c * hr);
            const C* ra = A.spec + ((size_t)c * A.rows + y) * nx4;
            const C* rb = ra + nx4;
            if (j <= n / 4) {  // Z = Xa + i Xb
                const C xa = ra[j], xb = rb[j];
                z.x = xa.x - xb.y;
                z.y = xa.y + xb.x;
            } else if (n - j <= n / 4) {  // Z = conj(Xa[n-j]) + i conj(Xb[n-j])
                const C xa = ra[n - j], xb = rb[n - j];
                z.x = xa.x + xb.y;
                z.y = xb.x - xa.y;
            }
        }
        s[t] = z;
    }
    __syncthreads();
    fft_dif(s, n, logn, P, A.tw, true);
    for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
        const int p = t >> logn;
        const int i = t & (n - 1);
        const int pair = pair0 + p;
        if (pair >= npairs) continue;
        const int c = pair / hr;
        const int y = 2 * (pair - c * hr);
        const int x = bitrev(i, logn);
        const C z = s[t];
        T* row = A.dm + c * NN + (size_t)y * n;
        row[x] = z.x;
        row[n + x] = z.y;
    }
}

template <typename T>
inline size_t spec2_row_smem(int n) {
    return (size_t)ffts_per_block(n) * n * sizeof(typename Cplx<T>::type);
}
template <typename T>
inline size_t spec2_col_smem(int n) {
    return (size_t)3 * n * sizeof(typename Cplx<T>::type);
}
inline int spec_row_blocks(int n, int nf, int rows) {
    const int P = ffts_per_block(n);
    return (nf * (rows / 2) + P - 1) / P;
}
inline int spec2_row_blocks(int n) { return spec_row_blocks(n, 3, n); }

}  // namespace msc
