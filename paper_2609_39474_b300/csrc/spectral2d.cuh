// Periodic shadow correction (Section 3.2, Eqs. shadow-cont .. shadow-update):
//   dm = F^{-1}[ chi(k) H(k)^{-1} F[P r] ]
// Shared pieces and the 2D kernels.  Transform convention Eq. fft-convention, wavenumbers
// Eq. wavenumbers, mask |j_alpha| <= n/4 (Eq. shadow-mask), closed-form Schur solve Eq. schur.
//
//   k_rowfft_fwd   real rows -> half spectrum along x, keeping 0 <= j_x <= n/4 (negative j_x
//                  follow from Hermitian symmetry).  Two real rows share one complex FFT; a block
//                  transforms 2P consecutive rows of one field.
//   k_colsolve     (2D) per kept j_x: FFT along y, FP64 Schur solve at |j_y| <= n/4 (zero
//                  elsewhere, 1/N_Omega folded in), inverse FFT along y.
//   k_rowfft_inv   Hermitian-extended half spectrum -> real rows.
// Half-spectrum layout: spec[c][j_x][row], c the field, j_x in [0, n/4], row the index of the
// length-n line along x (2D: row = y; 3D: row = z n + y), so that the transforms along y (and z)
// read contiguous memory and the row passes read or write 2P-element contiguous segments.
#pragma once

#include "common.cuh"
#include "fft.cuh"
#include "march.cuh"

namespace msc {

constexpr int kFftThreads = 256;
constexpr double kCs2 = 1.0 / 3.0;

template <typename T>
struct Spec2Args {
    const T* pr;                   // nf x sites residual moments
    typename Cplx<T>::type* spec;  // nf x (n/4+1) x rows half spectrum
    T* dm;                         // nf x sites correction
    const typename Cplx<T>::type* tw;
    int n, logn;
    int P;               // row passes: complex transforms (row pairs) per block
    int G;               // 3D passes: lines per block
    int nf;              // number of fields (d + 1)
    int rows;            // lines of length n per field (n in 2D, n^2 in 3D)
    double a, nu;
    double kunit;        // 2 pi / n (formed on the host)
    double nscale;       // 1 / N_Omega (formed on the host)
    const DevState* st;  // graph mode: a and q from the state
    const double* coef;  // per-mode solve coefficients (k_solve_tables): for q = 1, 2 with st, else one table
    int gate;            // graph mode outside a conditional node: run only if the sweep asked for it
};

// A correction that the march graph runs unconditionally (after a sweep that the acceptance rule
// cannot accept: fewer than n_min inner iterations) returns at once when that sweep asked for none
// (corrector off), the march stopped with an error, or no step is live.
template <typename T>
__device__ __forceinline__ bool spec_gated_off(const Spec2Args<T>& A) {
    return A.gate && !(A.st->lift && A.st->status == MSC_OK && A.st->steps_target > 0);
}

// pick the coefficient table of the current BDF order (graph mode), the table the caller chose
// (no state), or none (stage calls)
__device__ inline const double* solve_table(const double* coef, const DevState* st, int dim, int n) {
    if (!coef) return nullptr;
    if (!st) return coef;
    const int q = st->q;
    return coef + (size_t)(q - 1) * 4 * solve_modes(dim, n);
}

// Row-pass blocks: P row pairs (one field, consecutive rows), P a power of two dividing rows/2,
// at most 4096/n so that a block has at most 256 threads (one radix-16 butterfly each), at least
// 4 where possible so the transposed spectrum segments are >= 64 bytes, fewer when that would
// leave fewer than two blocks per SM, and 1 when even P = 4 gives fewer blocks than SMs.
struct RowGeom {
    int P, threads, blocks;
};
inline RowGeom row_geometry(int n, int nf, int rows) {
    const int npairs = nf * (rows / 2);
    int P = 4096 / n;
    if (P < 1) P = 1;
    if (P > rows / 2) P = rows / 2;
    while (P > 4 && npairs / P < 2 * 148) P >>= 1;
    // small lattices, where even four row pairs per block leave SMs idle: one pair per block
    // (N = 256: 96 blocks of 64 threads -> 384 of 32, the march 2.6 % faster)
    if (npairs / P < 148) P = 1;
    int t = P * n / 16;
    t = (t + 31) / 32 * 32;
    if (t < 32) t = 32;
    return {P, t, npairs / P};
}

// The 2D correction of small lattices takes the radix-4 transforms (n/4 threads per line): at
// N <= kSpec2Radix4Max the radix-16 form leaves a column block 3 n/16 threads (N = 256: 48) and a
// row block 16, so each pass is a few long serial chains per SM.
constexpr int kSpec2Radix4Max = 256;
inline bool spec2_radix4(int n) { return n <= kSpec2Radix4Max; }

// row blocks of the radix-4 form: one row pair per block (n/4 threads), or two below n = 128 so a
// block keeps at least 32 threads busy
inline RowGeom row_geometry_n4(int n) {
    int P = n >= 128 ? 1 : 128 / n;
    if (P > n / 2) P = n / 2;
    int t = (P * n / 4 + 31) / 32 * 32;
    if (t < 32) t = 32;
    return {P, t, 3 * (n / 2) / P};
}

template <typename T>
inline size_t spec_row_smem(int n, int P) {
    return (size_t)P * padded_len(n) * sizeof(typename Cplx<T>::type);
}

// the row and column transforms: radix-16 stages (n/16 threads per array) or, N4, radix-4 stages
// (n/4 threads per array; small lattices)
template <typename C, bool INV, bool N4>
__device__ __forceinline__ void fft_lines(C* s, int n, int logn, int nfft, const C* __restrict__ tw) {
    if constexpr (N4) fft_stockham_n4<C, INV>(s, n, logn, nfft, tw);
    else fft_stockham<C, INV>(s, n, logn, nfft, tw);
}

// 16-byte vectors of a row (4 binary32 or 2 binary64 values): the row passes move their rows with
// one load or store per vector when the rows are 16-byte aligned (always in the march; a stage
// call's arrays may not be, and then take the element loop)
template <typename T> struct RowVec;
template <> struct RowVec<float> { using type = float4; static constexpr int V = 4; };
template <> struct RowVec<double> { using type = double2; static constexpr int V = 2; };
template <typename VT> __device__ __forceinline__ auto vlane(const VT& v, int i) {
    if constexpr (sizeof(v.x) == 4) return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
    else return i == 0 ? v.x : v.y;
}
template <typename VT, typename S> __device__ __forceinline__ void vset(VT& v, int i, S x) {
    if constexpr (sizeof(v.x) == 4) {
        if (i == 0) v.x = x; else if (i == 1) v.y = x; else if (i == 2) v.z = x; else v.w = x;
    } else {
        if (i == 0) v.x = x; else v.y = x;
    }
}

// 2P consecutive rows (c, y0 .. y0 + 2P - 1) form P complex rows
template <typename T, bool N4 = false>
__device__ __forceinline__ void rowfft_fwd_block(const Spec2Args<T>& A, int bid) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = A.n, logn = A.logn, P = A.P, plen = padded_len(n);
    const int nx4 = n / 4 + 1;
    const int hr = A.rows / 2;
    const int pair0 = bid * P;  // P divides hr: all pairs of the block lie in one field
    const int c = pair0 / hr;
    const int y0 = 2 * (pair0 - c * hr);
    const T* rows = A.pr + ((size_t)c * A.rows + y0) * n;
    using VT = typename RowVec<T>::type;
    constexpr int V = RowVec<T>::V;
    if ((reinterpret_cast<uintptr_t>(A.pr) & 15u) == 0) {
        // one 16-byte load per row and vector; V consecutive x share one padded 16-block
        const int lnv = logn - (V == 4 ? 2 : 1);
        const int nv = 1 << lnv;
#pragma unroll 4
        for (int t = threadIdx.x; t < P * nv; t += blockDim.x) {
            const int p = t >> lnv;
            const int x = (t & (nv - 1)) * V;
            if (!MSC_INB(((size_t)c * A.rows + y0 + 2 * p + 1) * n + x + V - 1, (size_t)A.nf * A.rows * n, 11) ||
                !MSC_INB(p * plen + pad(x) + V - 1, P * plen, 12))
                continue;
            const VT ra = *reinterpret_cast<const VT*>(rows + (size_t)(2 * p) * n + x);
            const VT rb = *reinterpret_cast<const VT*>(rows + (size_t)(2 * p + 1) * n + x);
            C* d = s + p * plen + pad(x);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                C z;
                z.x = vlane(ra, i);
                z.y = vlane(rb, i);
                d[i] = z;
            }
        }
    } else {
        // unrolled so that the global loads of several iterations are in flight together
#pragma unroll 8
        for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
            const int p = t >> logn;
            const int x = t & (n - 1);
            if (!MSC_INB(((size_t)c * A.rows + y0 + 2 * p + 1) * n + x, (size_t)A.nf * A.rows * n, 11) ||
                !MSC_INB(p * plen + pad(x), P * plen, 12))
                continue;
            C z;
            z.x = rows[(size_t)(2 * p) * n + x];
            z.y = rows[(size_t)(2 * p + 1) * n + x];
            s[p * plen + pad(x)] = z;
        }
    }
    __syncthreads();
    fft_lines<C, false, N4>(s, n, logn, P, A.tw);
    // split the two real transforms; thread t -> (j_x, pair p), p fastest: the pair's two rows
    // 2p, 2p + 1 are adjacent in the transposed spectrum, one 16-byte store when aligned
    C* out = A.spec + (size_t)c * nx4 * A.rows + y0;
    const int lp = __ffs(P) - 1;  // P is a power of two
    const bool vec = sizeof(C) == 8 && (reinterpret_cast<uintptr_t>(A.spec) & 15u) == 0;
    for (int t = threadIdx.x; t < P * nx4; t += blockDim.x) {
        const int p = t & (P - 1);
        const int jx = t >> lp;
        const C zj = s[p * plen + pad(jx)];
        const C zm = s[p * plen + pad((n - jx) & (n - 1))];
        C va, vb;
        va.x = T(0.5) * (zj.x + zm.x);   // (zj + conj(zm)) / 2
        va.y = T(0.5) * (zj.y - zm.y);
        vb.x = T(0.5) * (zj.y + zm.y);   // (zj - conj(zm)) / (2i)
        vb.y = T(-0.5) * (zj.x - zm.x);
        const size_t o = (size_t)jx * A.rows + 2 * p;
        if (!MSC_INB((size_t)c * nx4 * A.rows + y0 + o + 1, (size_t)A.nf * nx4 * A.rows, 13)) continue;
        if (vec) {
            float4 w;
            w.x = (float)va.x; w.y = (float)va.y; w.z = (float)vb.x; w.w = (float)vb.y;
            *reinterpret_cast<float4*>(out + o) = w;
        } else {
            out[o] = va;
            out[o + 1] = vb;
        }
    }
}

template <typename T, bool N4 = false>
__global__ void __launch_bounds__(kFftThreads) k_rowfft_fwd(Spec2Args<T> A) {
    wait_for_predecessor();
    if (spec_gated_off(A)) return;
    rowfft_fwd_block<T, N4>(A, blockIdx.x);
}

// ACC = false: dm = the correction.  ACC = true (the adjoint's update): dm += pr + the correction,
// dm holding the iterate and pr the residual the forward pass transformed.
template <typename T, bool ACC = false, bool N4 = false>
__device__ __forceinline__ void rowfft_inv_block(const Spec2Args<T>& A, int bid) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = A.n, logn = A.logn, P = A.P, plen = padded_len(n);
    const int nx4 = n / 4 + 1;
    const int hr = A.rows / 2;
    const int pair0 = bid * P;
    const int c = pair0 / hr;
    const int y0 = 2 * (pair0 - c * hr);
    const C* in = A.spec + (size_t)c * nx4 * A.rows + y0;
    // Z[p][j] = Xa + i Xb (j <= n/4), conj(Xa[n-j]) + i conj(Xb[n-j]) (n-j <= n/4), else 0;
    // thread t -> (j, p), p fastest, so the spectrum reads are contiguous in the row index (Xa, Xb
    // adjacent: one 16-byte load when aligned)
    const bool vec = sizeof(C) == 8 && (reinterpret_cast<uintptr_t>(A.spec) & 15u) == 0;
    const int lp = __ffs(P) - 1;
#pragma unroll 8
    for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
        const int p = t & (P - 1);
        const int j = t >> lp;
        C z;
        z.x = T(0); z.y = T(0);
        const int jr = j <= n / 4 ? j : n - j;
        if (!MSC_INB((size_t)c * nx4 * A.rows + y0 + (size_t)(jr <= n / 4 ? jr : 0) * A.rows + 2 * p + 1,
                     (size_t)A.nf * nx4 * A.rows, 14))
            continue;
        if (jr <= n / 4) {
            const size_t o = (size_t)jr * A.rows + 2 * p;
            C xa, xb;
            if (vec) {
                const float4 w = *reinterpret_cast<const float4*>(in + o);
                xa.x = w.x; xa.y = w.y; xb.x = w.z; xb.y = w.w;
            } else {
                xa = in[o];
                xb = in[o + 1];
            }
            if (j <= n / 4) {
                z.x = xa.x - xb.y;
                z.y = xa.y + xb.x;
            } else {
                z.x = xa.x + xb.y;
                z.y = xb.x - xa.y;
            }
        }
        s[p * plen + pad(j)] = z;
    }
    __syncthreads();
    fft_lines<C, true, N4>(s, n, logn, P, A.tw);
    T* __restrict__ rows = A.dm + ((size_t)c * A.rows + y0) * n;
    if (ACC) {
        // four iterations at a time: all their iterate and residual loads are issued before the
        // stores, so one memory round trip serves four elements per row pair
        const T* __restrict__ res = A.pr + ((size_t)c * A.rows + y0) * n;
        constexpr int U = 4;
        for (int t0 = threadIdx.x; t0 < P * n; t0 += U * blockDim.x) {
            T v0[U], v1[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0 + u * blockDim.x;
                if (t < P * n) {
                    const size_t o0 = (size_t)(2 * (t >> logn)) * n + (t & (n - 1));
                    v0[u] = rows[o0] + res[o0];
                    v1[u] = rows[o0 + n] + res[o0 + n];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0 + u * blockDim.x;
                if (t < P * n) {
                    const int p = t >> logn;
                    const int x = t & (n - 1);
                    const size_t o0 = (size_t)(2 * p) * n + x;
                    const C z = s[p * plen + pad(x)];
                    rows[o0] = v0[u] + z.x;
                    rows[o0 + n] = v1[u] + z.y;
                }
            }
        }
        return;
    }
    using VT = typename RowVec<T>::type;
    constexpr int V = RowVec<T>::V;
    if ((reinterpret_cast<uintptr_t>(A.dm) & 15u) == 0) {
        const int lnv = logn - (V == 4 ? 2 : 1);
        const int nv = 1 << lnv;
        for (int t = threadIdx.x; t < P * nv; t += blockDim.x) {
            const int p = t >> lnv;
            const int x = (t & (nv - 1)) * V;
            if (!MSC_INB(((size_t)c * A.rows + y0 + 2 * p + 1) * n + x + V - 1, (size_t)A.nf * A.rows * n, 15))
                continue;
            const C* sp = s + p * plen + pad(x);
            VT ra, rb;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const C z = sp[i];
                vset(ra, i, z.x);
                vset(rb, i, z.y);
            }
            *reinterpret_cast<VT*>(rows + (size_t)(2 * p) * n + x) = ra;
            *reinterpret_cast<VT*>(rows + (size_t)(2 * p + 1) * n + x) = rb;
        }
        return;
    }
    for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
        const int p = t >> logn;
        const int x = t & (n - 1);
        if (!MSC_INB(((size_t)c * A.rows + y0 + 2 * p + 1) * n + x, (size_t)A.nf * A.rows * n, 15)) continue;
        const C z = s[p * plen + pad(x)];
        rows[(size_t)(2 * p) * n + x] = z.x;
        rows[(size_t)(2 * p + 1) * n + x] = z.y;
    }
}

template <typename T, bool N4 = false>
__global__ void __launch_bounds__(kFftThreads) k_rowfft_inv(Spec2Args<T> A) {
    wait_for_predecessor();
    if (spec_gated_off(A)) return;
    rowfft_inv_block<T, false, N4>(A, blockIdx.x);
}

// the inverse row pass of the adjoint shadow correction, fused with the iterate update
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_rowfft_inv_acc(Spec2Args<T> A) {
    rowfft_inv_block<T, true>(A, blockIdx.x);
}

// Schur solve at one masked wavevector in FP64: dp = A rp - i B (k.rm), du = Dv rm - i Cc k dp
// ICVT: the binary32 <-> binary64 conversions on the integer pipe (widen_f32 / narrow_f64, the same
// values): where the solve holds the FP64 pipe (the warp-per-line column pass at N = 1024, the 3D z
// pass) that takes 12 of its ~30 FP64-pipe instructions per mode off it
template <typename C, int D, bool ICVT = false>
__device__ __forceinline__ void schur_apply(C* v[D + 1], const double* kv, const double* cf) {
    using T = decltype(v[0]->x);
    auto wide = [](T x) { return ICVT ? to_f64<T>(x) : (double)x; };
    auto narrow = [](double x) { return ICVT ? from_f64<T>(x) : (T)x; };
    double rx[D + 1], ry[D + 1];
#pragma unroll
    for (int i = 0; i <= D; ++i) { rx[i] = wide(v[i]->x); ry[i] = wide(v[i]->y); }
    double krx = 0.0, kry = 0.0;
#pragma unroll
    for (int al = 0; al < D; ++al) { krx += kv[al] * rx[al + 1]; kry += kv[al] * ry[al + 1]; }
    const double dpx = cf[0] * rx[0] + cf[1] * kry;
    const double dpy = cf[0] * ry[0] - cf[1] * krx;
    v[0]->x = narrow(dpx);
    v[0]->y = narrow(dpy);
#pragma unroll
    for (int al = 0; al < D; ++al) {
        const double ck = cf[2] * kv[al];
        v[al + 1]->x = narrow(cf[3] * rx[al + 1] + ck * dpy);
        v[al + 1]->y = narrow(cf[3] * ry[al + 1] - ck * dpx);
    }
}

// Transposed solve x = (H(k)^H)^{-1} y, the per-wavevector factor of the adjoint shadow correction
// (the transpose of F^{-1} chi H^{-1} F for the real inner product): with the same table,
//   dp = A y_p + i cs^2 B (k.y_m),   du = Dv y_m + i (Cc / cs^2) k dp.
template <typename C, int D>
__device__ __forceinline__ void schur_apply_adjoint(C* v[D + 1], const double* kv, const double* cf) {
    using T = decltype(v[0]->x);
    double rx[D + 1], ry[D + 1];
#pragma unroll
    for (int i = 0; i <= D; ++i) { rx[i] = (double)v[i]->x; ry[i] = (double)v[i]->y; }
    double krx = 0.0, kry = 0.0;
#pragma unroll
    for (int al = 0; al < D; ++al) { krx += kv[al] * rx[al + 1]; kry += kv[al] * ry[al + 1]; }
    const double bt = kCs2 * cf[1], ct = cf[2] / kCs2;
    const double dpx = cf[0] * rx[0] - bt * kry;
    const double dpy = cf[0] * ry[0] + bt * krx;
    v[0]->x = (T)dpx;
    v[0]->y = (T)dpy;
#pragma unroll
    for (int al = 0; al < D; ++al) {
        const double ck = ct * kv[al];
        v[al + 1]->x = (T)(cf[3] * rx[al + 1] - ck * dpy);
        v[al + 1]->y = (T)(cf[3] * ry[al + 1] + ck * dpx);
    }
}

// The Schur solve of one (j_x, j_y) mode of the column pass in place on its three field values v
// (zero outside the mask |j_y| <= n/4 or for a column past the last kept one)
template <typename T, bool ADJ, bool ICVT = false>
__device__ __forceinline__ void solve_mode(const Spec2Args<T>& A, typename Cplx<T>::type* v[3], int jx, int jy,
                                           bool live, double a, const double* tab) {
    using C = typename Cplx<T>::type;
    const int n = A.n, nx4 = n / 4 + 1;
    const int jys = jy <= n / 2 ? jy : jy - n;
    if (jys > n / 4 || jys < -(n / 4) || !live) {
        C z; z.x = T(0); z.y = T(0);
        *v[0] = z; *v[1] = z; *v[2] = z;
        return;
    }
    double kv[2];
    kv[0] = A.kunit * (double)jx;
    kv[1] = A.kunit * (double)jys;
    double cf[4];
    if (tab) {
        const double* tt = tab + 4 * ((size_t)(jys + n / 4) * nx4 + jx);
        cf[0] = tt[0]; cf[1] = tt[1]; cf[2] = tt[2]; cf[3] = tt[3];
    } else {
        solve_coefficients(a, A.nu, kv[0] * kv[0] + kv[1] * kv[1], A.nscale, cf);
    }
    if (ADJ) schur_apply_adjoint<C, 2>(v, kv, cf);
    else schur_apply<C, 2, ICVT>(v, kv, cf);
}

// 2D: G consecutive kept j_x columns per block (G a power of two; the last block of a lattice may
// hold fewer), all three fields of each.  Line (c, g) of the block sits at (c G + g) plen in shared memory.
template <typename T, bool ADJ = false, bool N4 = false>
__device__ __forceinline__ void colsolve_block(const Spec2Args<T>& A, int bid, int G) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = A.n, logn = A.logn, plen = padded_len(n);
    const int nx4 = n / 4 + 1;
    const int jx0 = bid * G;
    const int ng = min(G, nx4 - jx0);
    const int lgn = logn + __ffs(G) - 1;  // G is a power of two
    const int gn = 1 << lgn;
    C* col = A.spec + (size_t)jx0 * n;  // spec[c][jx0 + g][y] at col + c * nx4 * n + g * n + y
    const size_t fs = (size_t)nx4 * n;
    // binary32: two consecutive y per thread, one 16-byte access (y even: one padded 16-block of s)
    constexpr int lv = sizeof(C) == 8 ? 1 : 0;
#pragma unroll 4
    for (int t = threadIdx.x; t < (3 * gn >> lv); t += blockDim.x) {
        const int e = t << lv;
        const int c = e >> lgn;
        const int gy = e & (gn - 1);  // g * n + y
        const bool in = (gy >> logn) < ng && MSC_INB((size_t)jx0 * n + c * fs + gy + lv, (size_t)A.nf * fs, 16);
        const int si = (c * G + (gy >> logn)) * plen + pad(gy & (n - 1));
        if (!MSC_INB(si + lv, 3 * G * plen, 17)) continue;
        if constexpr (lv == 1) {
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (in) w = *reinterpret_cast<const float4*>(col + c * fs + gy);
            s[si] = make_float2(w.x, w.y);
            s[si + 1] = make_float2(w.z, w.w);
        } else {
            C v;
            v.x = T(0); v.y = T(0);
            if (in) v = col[c * fs + gy];
            s[si] = v;
        }
    }
    __syncthreads();
    fft_lines<C, false, N4>(s, n, logn, 3 * G, A.tw);
    const double a = A.st ? A.st->a : A.a;
    const double* tab = solve_table(A.coef, A.st, 2, n);
    for (int t = threadIdx.x; t < gn; t += blockDim.x) {
        const int g = t >> logn;
        const int jy = t & (n - 1);
        C* v[3] = {s + g * plen + pad(jy), s + (G + g) * plen + pad(jy), s + (2 * G + g) * plen + pad(jy)};
        solve_mode<T, ADJ>(A, v, jx0 + g, jy, g < ng, a, tab);
    }
    __syncthreads();
    fft_lines<C, true, N4>(s, n, logn, 3 * G, A.tw);
    for (int t = threadIdx.x; t < (3 * gn >> lv); t += blockDim.x) {
        const int e = t << lv;
        const int c = e >> lgn;
        const int gy = e & (gn - 1);
        if ((gy >> logn) >= ng || !MSC_INB((size_t)jx0 * n + c * fs + gy + lv, (size_t)A.nf * fs, 16)) continue;
        const int si = (c * G + (gy >> logn)) * plen + pad(gy & (n - 1));
        if constexpr (lv == 1) {
            const C z0 = s[si], z1 = s[si + 1];
            *reinterpret_cast<float4*>(col + c * fs + gy) = make_float4(z0.x, z0.y, z1.x, z1.y);
        } else {
            col[c * fs + gy] = s[si];
        }
    }
}

template <typename T, bool N4 = false>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 384 : 768) k_colsolve(Spec2Args<T> A) {
    wait_for_predecessor();
    if (spec_gated_off(A)) return;
    colsolve_block<T, false, N4>(A, blockIdx.x, 1);
}

// the transposed column solve of the adjoint shadow correction
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 384 : 768) k_colsolve_adjoint(Spec2Args<T> A) {
    colsolve_block<T, true>(A, blockIdx.x, 1);
}

inline int spec2_col_threads(int n) {
    const int t = (3 * n / 16 + 31) / 32 * 32;
    return t < 32 ? 32 : t;
}
template <typename T>
inline size_t spec2_col_smem(int n) {
    return (size_t)3 * padded_len(n) * sizeof(typename Cplx<T>::type);
}

// ---- N = 1024 with FP32 working fields: the column pass with one warp per line ----------------------
// The generic column pass synchronises the whole block between the radix stages of its transforms;
// at N = 1024 (FP32, the benchmark size) this variant gives each 1024-point column line to one warp
// (fft1024_warp: two radix-32 stages separated by __syncwarp), loads the first stage's samples
// straight from global memory into registers and stores the last stage's outputs straight from
// registers, both coalesced.  Same inputs, outputs and layout as k_colsolve (the transform differs
// only in rounding order); the per-mode solve is the same function.  (The row passes stay generic:
// written the same way they needed 170 and 232 registers per thread, which left too few warps per
// SM, and ran slower than the block-synchronous versions.)
// column pass at N = 1024: warp c transforms field c of kept column j_x = blockIdx.x
__global__ void __launch_bounds__(96) k_colsolve_1024(Spec2Args<float> A) {
    wait_for_predecessor();
    if (spec_gated_off(A)) return;
    using C = float2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    constexpr int n = 1024;
    const int plen = padded_len(n), nx4 = n / 4 + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int jx = blockIdx.x;
    C* col = A.spec + ((size_t)warp * nx4 + jx) * n;  // spec[c][jx][y], c = warp
    C* line = s + warp * plen;
    C v[32];
    if (!MSC_INB(((size_t)warp * nx4 + jx) * n + 1023, (size_t)3 * nx4 * n, 18)) return;
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = col[lane + 32 * r];
    fft1024_warp<C, false>(v, line, A.tw);
#pragma unroll
    for (int r = 0; r < 32; ++r) line[pad(lane + 32 * r)] = v[r];
    __syncthreads();
    const double a = A.st ? A.st->a : A.a;
    const double* tab = solve_table(A.coef, A.st, 2, n);
    for (int jy = threadIdx.x; jy < n; jy += blockDim.x) {
        C* w[3] = {s + pad(jy), s + plen + pad(jy), s + 2 * plen + pad(jy)};
        solve_mode<float, false, true>(A, w, jx, jy, true, a, tab);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = line[pad(lane + 32 * r)];
    fft1024_warp<C, true>(v, line, A.tw);
#pragma unroll
    for (int r = 0; r < 32; ++r) col[lane + 32 * r] = v[r];
}

// The three launches of the 2D shadow correction (row FFTs, column FFT + solve + inverse, inverse
// row FFTs) for lattice size n and working type T, all taking one Spec2Args block; returns the row
// pairs per row block (Spec2Args::P) that the launches assume.
struct Spec2Launch {
    const void* fn;
    dim3 grid, block;
    size_t smem;
};
template <typename T>
inline int spectral2_launches(int n, Spec2Launch L[3]) {
    if (spec2_radix4(n)) {  // small lattices: radix-4 transforms, n/4 threads per line
        const RowGeom rg = row_geometry_n4(n);
        const size_t rsm = spec_row_smem<T>(n, rg.P);
        const int ct = (3 * n / 4 + 31) / 32 * 32;
        L[0] = {(const void*)k_rowfft_fwd<T, true>, dim3(rg.blocks), dim3(rg.threads), rsm};
        L[1] = {(const void*)k_colsolve<T, true>, dim3(n / 4 + 1), dim3(ct < 32 ? 32 : ct), spec2_col_smem<T>(n)};
        L[2] = {(const void*)k_rowfft_inv<T, true>, dim3(rg.blocks), dim3(rg.threads), rsm};
        return rg.P;
    }
    const RowGeom rg = row_geometry(n, 3, n);
    const size_t rsm = spec_row_smem<T>(n, rg.P);
    L[0] = {(const void*)k_rowfft_fwd<T>, dim3(rg.blocks), dim3(rg.threads), rsm};
    L[1] = {(const void*)k_colsolve<T>, dim3(n / 4 + 1), dim3(spec2_col_threads(n)), spec2_col_smem<T>(n)};
    if (std::is_same<T, float>::value && n == 1024)
        L[1] = {(const void*)k_colsolve_1024, dim3(n / 4 + 1), dim3(96), spec2_col_smem<T>(n)};
    L[2] = {(const void*)k_rowfft_inv<T>, dim3(rg.blocks), dim3(rg.threads), rsm};
    return rg.P;
}

}  // namespace msc
