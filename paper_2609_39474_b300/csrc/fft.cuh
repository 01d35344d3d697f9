// Hand-written radix-2 FFT building blocks in shared memory.
//
// A block transforms `nfft` independent arrays of length n (power of two) stored contiguously
// in shared memory.  Forward transforms use e^{-2 pi i j x / n}; inverse transforms use the
// conjugate twiddles and are unnormalised (the 1/N_Omega of Eq. fft-convention is applied by
// the caller).  Input and output are in natural order (Stockham autosort, no permutation pass).
// Twiddles come from a table tw[j] = e^{-2 pi i j / n}, j < n, built once per context in FP64.
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

template <typename C>
__device__ __forceinline__ C twiddle(const C* __restrict__ tw, int idx, bool inverse) {
    C w = __ldg(tw + idx);
    if (inverse) w.y = -w.y;
    return w;
}

// ---- small DFTs in registers (forward: e^{-2 pi i jk/R}; INV: conjugate) -----------------------

template <typename C>
__device__ __forceinline__ C mul_minus_i(C d, bool inv) {  // d * (-i) forward, d * (+i) inverse
    C r;
    if (inv) { r.x = -d.y; r.y = d.x; }
    else { r.x = d.y; r.y = -d.x; }
    return r;
}

// multiply by e^{-+ 2 pi i m / 16} with (c, s) = (cos, sin) of 2 pi m / 16
template <typename C>
__device__ __forceinline__ C rot(C v, double c, double s, bool inv) {
    using R = decltype(v.x);
    const R cc = (R)c, ss = inv ? (R)s : (R)(-s);
    C r;
    r.x = v.x * cc - v.y * ss;
    r.y = v.x * ss + v.y * cc;
    return r;
}

template <typename C, bool INV>
__device__ __forceinline__ void dft4(C& a, C& b, C& c, C& d) {
    const C a0 = cadd(a, c), a1 = csub(a, c), a2 = cadd(b, d);
    const C a3 = mul_minus_i(csub(b, d), INV);
    a = cadd(a0, a2);
    b = cadd(a1, a3);
    c = csub(a0, a2);
    d = csub(a1, a3);
}

template <typename C, int R, bool INV> struct SmallDft;

template <typename C, bool INV> struct SmallDft<C, 2, INV> {
    __device__ __forceinline__ static void run(C* v) {
        const C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};
template <typename C, bool INV> struct SmallDft<C, 4, INV> {
    __device__ __forceinline__ static void run(C* v) { dft4<C, INV>(v[0], v[1], v[2], v[3]); }
};
// 8 = 2 x 4: n = q + 2p, k = s + 4t
template <typename C, bool INV> struct SmallDft<C, 8, INV> {
    __device__ __forceinline__ static void run(C* v) {
        const double h = 0.70710678118654752440;
        C a0 = v[0], a1 = v[2], a2 = v[4], a3 = v[6];
        C b0 = v[1], b1 = v[3], b2 = v[5], b3 = v[7];
        dft4<C, INV>(a0, a1, a2, a3);
        dft4<C, INV>(b0, b1, b2, b3);
        b1 = rot(b1, h, h, INV);
        b2 = mul_minus_i(b2, INV);
        b3 = rot(b3, -h, h, INV);
        v[0] = cadd(a0, b0); v[4] = csub(a0, b0);
        v[1] = cadd(a1, b1); v[5] = csub(a1, b1);
        v[2] = cadd(a2, b2); v[6] = csub(a2, b2);
        v[3] = cadd(a3, b3); v[7] = csub(a3, b3);
    }
};
// 16 = 4 x 4: n = q + 4p, k = s + 4t; twiddles e^{-2 pi i q s / 16}
template <typename C, bool INV> struct SmallDft<C, 16, INV> {
    __device__ __forceinline__ static void run(C* v) {
        const double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173, h = 0.70710678118654752440;
        C A[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            A[q][0] = v[q]; A[q][1] = v[q + 4]; A[q][2] = v[q + 8]; A[q][3] = v[q + 12];
            dft4<C, INV>(A[q][0], A[q][1], A[q][2], A[q][3]);
        }
        // q = 1: m = s;  q = 2: m = 2s;  q = 3: m = 3s
        A[1][1] = rot(A[1][1], c1, s1, INV);
        A[1][2] = rot(A[1][2], h, h, INV);
        A[1][3] = rot(A[1][3], s1, c1, INV);
        A[2][1] = rot(A[2][1], h, h, INV);
        A[2][2] = mul_minus_i(A[2][2], INV);
        A[2][3] = rot(A[2][3], -h, h, INV);
        A[3][1] = rot(A[3][1], s1, c1, INV);
        A[3][2] = rot(A[3][2], -h, h, INV);
        A[3][3] = rot(A[3][3], -c1, -s1, INV);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            C a = A[0][s], b = A[1][s], c = A[2][s], d = A[3][s];
            dft4<C, INV>(a, b, c, d);
            v[s] = a; v[s + 4] = b; v[s + 8] = c; v[s + 12] = d;
        }
    }
};

// Shared-memory layout of the transforms: array f of length n starts at f * padded_len(n) and
// element i sits at i + i/16.  The padding breaks the power-of-two strides of the Stockham stores
// that would otherwise hit one shared-memory bank.
__host__ __device__ __forceinline__ int padded_len(int n) { return n + (n >> 4); }
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

// One in-place Stockham stage of radix R over nfft arrays of length n: every butterfly j reads the
// R values j + r n/R, multiplies value r by w^(k r n/(Ns R)) with k = j mod Ns, does the R-point DFT
// in registers and writes value r to (j - k) R + k + r Ns.  All reads of the stage complete before
// any write (block barrier), so one buffer suffices.  Each thread handles at most MB butterflies
// (the host geometry launches at least nfft n / (R MB) threads): 16/R in the radix-16 form (n/16
// threads per array), 1 in the radix-4 form (n/4 threads per array).
template <typename C, int R, bool INV, int MB = 16 / R>
__device__ __forceinline__ void stockham_stage(C* x, int n, int logn, int Ns, int nfft, const C* __restrict__ tw) {
    constexpr int LR = R == 2 ? 1 : (R == 4 ? 2 : (R == 8 ? 3 : 4));
    const int lnb = logn - LR;
    const int nb = 1 << lnb;
    const int tstride = n / (Ns * R);
    const int total = nfft << lnb;
    const int plen = padded_len(n);
    C v[MB][R];
#pragma unroll
    for (int m = 0; m < MB; ++m) {
        const int b = threadIdx.x + m * blockDim.x;
        if (b < total) {
            const int f = b >> lnb;
            const int j = b & (nb - 1);
            const C* xs = x + f * plen;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (MSC_INB(f * plen + pad(j + r * nb), nfft * plen, 7)) v[m][r] = xs[pad(j + r * nb)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < MB; ++m) {
        const int b = threadIdx.x + m * blockDim.x;
        if (b < total) {
            const int f = b >> lnb;
            const int j = b & (nb - 1);
            const int k = j & (Ns - 1);
            if (Ns > 1) {
                const int kt = k * tstride;
                if (R == 16) {
                    // two table reads, the other powers by products (at most four deep)
                    C w[16];
                    w[1] = twiddle(tw, kt, INV);
                    w[4] = twiddle(tw, 4 * kt, INV);
                    w[2] = cmul(w[1], w[1]);
                    w[3] = cmul(w[2], w[1]);
                    w[8] = cmul(w[4], w[4]);
#pragma unroll
                    for (int r = 5; r < 8; ++r) w[r] = cmul(w[4], w[r - 4]);
#pragma unroll
                    for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
#pragma unroll
                    for (int r = 1; r < 16; ++r) v[m][r] = cmul(v[m][r], w[r]);
                } else {
#pragma unroll
                    for (int r = 1; r < R; ++r) v[m][r] = cmul(v[m][r], twiddle(tw, r * kt, INV));
                }
            }
            SmallDft<C, R, INV>::run(v[m]);
            C* ys = x + f * plen;
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (MSC_INB(f * plen + pad(base + r * Ns), nfft * plen, 8)) ys[pad(base + r * Ns)] = v[m][r];
        }
    }
    __syncthreads();
}

// In-place Stockham autosort FFT (natural order in and out) over nfft padded arrays of length n
// in shared memory.  Mixed radix: one radix-2/4/8 stage for log2(n) mod 4, then radix-16 stages.
// Must be called by all threads of the block, with blockDim.x >= nfft * n / 16.
template <typename C, bool INV>
__device__ void fft_stockham(C* x, int n, int logn, int nfft, const C* __restrict__ tw) {
    int Ns = 1;
    const int first = logn & 3;
    if (first == 1) stockham_stage<C, 2, INV>(x, n, logn, Ns, nfft, tw);
    else if (first == 2) stockham_stage<C, 4, INV>(x, n, logn, Ns, nfft, tw);
    else if (first == 3) stockham_stage<C, 8, INV>(x, n, logn, Ns, nfft, tw);
    Ns <<= first;
    for (int rem = logn - first; rem > 0; rem -= 4) {
        stockham_stage<C, 16, INV>(x, n, logn, Ns, nfft, tw);
        Ns <<= 4;
    }
}

// The same transform in radix-4 stages (a radix-2 stage first when log2(n) is odd) with n/4 threads
// per array: for small n, where the radix-16 form gives an array only n/16 threads and each thread a
// long serial chain of 16-point butterflies (N = 256: 16 threads per line).  Twice the stages and
// barriers, a quarter of the work per thread per stage.  Must be called by all threads of the
// block, with blockDim.x >= nfft * n / 4.
template <typename C, bool INV>
__device__ void fft_stockham_n4(C* x, int n, int logn, int nfft, const C* __restrict__ tw) {
    int Ns = 1;
    if (logn & 1) {
        stockham_stage<C, 2, INV, 2>(x, n, logn, Ns, nfft, tw);
        Ns = 2;
    }
    for (int rem = logn - (logn & 1); rem > 0; rem -= 2) {
        stockham_stage<C, 4, INV, 1>(x, n, logn, Ns, nfft, tw);
        Ns <<= 2;
    }
}

// cos(pi k / 16) for 0 <= k <= 16 (the 32-point DFT's rotations; sin(pi k / 16) = cos_pi16(|8 - k|))
__host__ __device__ constexpr double cos_pi16(int k) {
    return k > 8 ? -cos_pi16(16 - k)
                 : (k == 0 ? 1.0
                    : k == 1 ? 0.98078528040323044913
                    : k == 2 ? 0.92387953251128675613
                    : k == 3 ? 0.83146961230254523708
                    : k == 4 ? 0.70710678118654752440
                    : k == 5 ? 0.55557023301960222474
                    : k == 6 ? 0.38268343236508977173
                    : k == 7 ? 0.19509032201612826785
                             : 0.0);
}

// 32 = 2 x 16: X[k] = E[k] + W^k O[k], X[k + 16] = E[k] - W^k O[k] with E, O the 16-point DFTs of the
// even and odd samples and W = exp(-+ 2 pi i / 32)
template <typename C, bool INV> struct SmallDft<C, 32, INV> {
    __device__ __forceinline__ static void run(C* v) {
        C e[16], o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
        SmallDft<C, 16, INV>::run(e);
        SmallDft<C, 16, INV>::run(o);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int sk = 8 - k < 0 ? k - 8 : 8 - k;
            const C t = k == 0 ? o[0] : rot(o[k], cos_pi16(k), cos_pi16(sk), INV);
            v[k] = cadd(e[k], t);
            v[k + 16] = csub(e[k], t);
        }
    }
};

// ---- one warp per line of 1024 points: two radix-32 Stockham stages --------------------------------
// The line sits in shared memory in the padded layout (element i at pad(i)).  Lane j holds, on entry
// to stage 1, the samples x[j + 32 r] (r = 0 .. 31) in v; stage 1 forms their 32-point DFT and stores
// it at 32 j + r; stage 2 reads y[j + 32 r], applies the twiddles w_1024^(j r) and forms the second
// 32-point DFT, leaving X[j + 32 r] in v (natural order).  Only __syncwarp separates the stages, so
// the warps of a block proceed independently.  `s` may hold the stage-1 input (then the caller's
// loads from s are complete before stage 1 stores: the __syncwarp at its start orders them).
template <typename C, bool INV>
__device__ __forceinline__ void fft1024_warp(C* v, C* s, const C* __restrict__ tw) {
    const int j = threadIdx.x & 31;
    SmallDft<C, 32, INV>::run(v);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 32; ++r)
        if (MSC_INB(pad(32 * j + r), padded_len(1024), 9)) s[pad(32 * j + r)] = v[r];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 32; ++r)
        if (MSC_INB(pad(j + 32 * r), padded_len(1024), 10)) v[r] = s[pad(j + 32 * r)];
#pragma unroll
    for (int r = 1; r < 32; ++r) v[r] = cmul(v[r], twiddle(tw, j * r, INV));
    SmallDft<C, 32, INV>::run(v);
    __syncwarp();  // every lane's stage-2 reads are done before the caller stores into s
}

// tw[j] = exp(-2 pi i j / n) for j < n, evaluated in FP64 and rounded to the storage type.
template <typename C>
__global__ void k_twiddles(C* tw, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        double s, c;
        sincospi(2.0 * (double)j / (double)n, &s, &c);
        C w;
        w.x = (decltype(w.x))c;
        w.y = (decltype(w.y))(-s);
        tw[j] = w;
    }
}

}  // namespace msc
