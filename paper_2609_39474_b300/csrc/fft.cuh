// Hand-written radix-2 FFT building blocks in shared memory.
//
// A block transforms `nfft` independent arrays of length n (power of two) stored contiguously
// in shared memory.  Forward transforms use e^{-2 pi i j x / n}; inverse transforms use the
// conjugate twiddles and are unnormalised (the 1/N_Omega of Eq. fft-convention is applied by
// the caller).  Two orderings are provided so that no explicit permutation pass is needed:
//   dit: input in bit-reversed order, output in natural order (Cooley-Tukey decimation in time)
//   dif: input in natural order, output in bit-reversed order (decimation in frequency)
// Twiddles come from a table tw[j] = e^{-2 pi i j / n}, j < n/2, built once per context in FP64.
#pragma once

#include "common.cuh"

namespace msc {

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int bitrev(int i, int logn) { return (int)(__brev((unsigned)i) >> (32 - logn)); }

template <typename C>
__device__ __forceinline__ C twiddle(const C* tw, int idx, bool inverse) {
    C w = tw[idx];
    if (inverse) w.y = -w.y;
    return w;
}

// In-place decimation-in-time passes over nfft arrays (bit-reversed in, natural out).
template <typename C>
__device__ void fft_dit(C* s, int n, int logn, int nfft, const C* __restrict__ tw, bool inverse) {
    const int hn = n >> 1;
    const int total = nfft * hn;
    for (int lg = 1; lg <= logn; ++lg) {
        const int half = 1 << (lg - 1);
        const int len = half << 1;
        const int tstride = n >> lg;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int f = b >> (logn - 1);
            const int bb = b & (hn - 1);
            const int grp = bb >> (lg - 1);
            const int pos = bb & (half - 1);
            const int i = f * n + grp * len + pos;
            const int j = i + half;
            const C w = twiddle(tw, pos * tstride, inverse);
            const C u = s[i];
            const C v = cmul(s[j], w);
            s[i] = cadd(u, v);
            s[j] = csub(u, v);
        }
        __syncthreads();
    }
}

// In-place decimation-in-frequency passes over nfft arrays (natural in, bit-reversed out).
template <typename C>
__device__ void fft_dif(C* s, int n, int logn, int nfft, const C* __restrict__ tw, bool inverse) {
    const int hn = n >> 1;
    const int total = nfft * hn;
    for (int lg = logn; lg >= 1; --lg) {
        const int half = 1 << (lg - 1);
        const int len = half << 1;
        const int tstride = n >> lg;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int f = b >> (logn - 1);
            const int bb = b & (hn - 1);
            const int grp = bb >> (lg - 1);
            const int pos = bb & (half - 1);
            const int i = f * n + grp * len + pos;
            const int j = i + half;
            const C w = twiddle(tw, pos * tstride, inverse);
            const C u = s[i];
            const C v = s[j];
            s[i] = cadd(u, v);
            s[j] = cmul(csub(u, v), w);
        }
        __syncthreads();
    }
}

// tw[j] = exp(-2 pi i j / n) for j < n/2, evaluated in FP64 and rounded to the storage type.
template <typename C>
__global__ void k_twiddles(C* tw, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n / 2) {
        double s, c;
        sincospi(2.0 * (double)j / (double)n, &s, &c);
        C w;
        w.x = (decltype(w.x))c;
        w.y = (decltype(w.y))(-s);
        tw[j] = w;
    }
}

}  // namespace msc
