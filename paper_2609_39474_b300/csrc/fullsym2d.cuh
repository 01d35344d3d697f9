// Full-symbol reference correction for D2Q9 (Section 4.1, Eq. full-symbol), for off-design
// collisions (omega+- != 1, Eq. collision) where the three-field shadow correction loses its
// contraction:
//     f_out = f + F^{-1}[ (I - Z(k) J)^{-1} F[f_T - f] ]   at every wavevector, all 9 fields,
// with J the collision Jacobian at rest, Z(k) = diag(exp(-i k . c_q)) the streaming symbol and
// f_T the swept iterate.  It is the linearised Newton step about rest.
//
// J in closed form.  Linearising Eq. collision at rest (u = 0, s = 0; m = R(f) with the history h
// fixed, so dm = P df / (1 + a/2) and ds = -a dm):
//     J = (1 - w+) Pi+ + (1 - w-) Pi- + U P,
//     U = [ b+ w_q,  b- w_q c_qx / cs^2,  b- w_q c_qy / cs^2 ],   b+- = (w+- - a (1 - w+-/2)) / (1 + a/2),
// Pi+- the even/odd projectors of the pairs (q, qbar) with c_qbar = -c_q, P the moment rows
// (1, c_x, c_y).  (At w+- = 1 this is gamma E P, Eq. symbol.)  Hence I - Z J = A - (Z U) P with
// A = I - Z((1 - w+) Pi+ + (1 - w-) Pi-) block diagonal over the pairs, and the Woodbury identity
//     (A - Z U P)^{-1} = A^{-1} + A^{-1} Z U (I_3 - P A^{-1} Z U)^{-1} P A^{-1}
// reduces every wavevector to four 2 x 2 pair solves (real determinant 1 - 2 d1 cos(k.c) + d1^2 - d2^2
// with d1 = (2 - w+ - w-)/2, d2 = (w- - w+)/2; |d1| + |d2| < 1 keeps it positive), one division for
// the rest particle (A_00 = w+) and one 3 x 3 complex solve, all in FP64.
//
// Passes (same transform conventions as the shadow correction, half spectrum over j_x <= n/2):
//   k_fs_rowfwd  rows of r = f_T - f -> half spectrum spec[q][j_x][y], two real rows per complex FFT
//   k_fs_col     per j_x: FFT along y of the 9 fields, the per-mode solve (1/N_Omega folded in),
//                inverse FFT along y
//   k_fs_rowinv  half spectrum -> real rows, written as f + df
#pragma once

#include "common.cuh"
#include "fft.cuh"
#include "spectral2d.cuh"

namespace msc {

template <typename T>
struct FsArgs {
    const T* f;                       // 9 x sites, the iterate
    const T* ft;                      // 9 x sites, the swept iterate
    T* out;                           // 9 x sites, f + df
    typename Cplx<T>::type* spec;     // 9 x (n/2 + 1) x n half spectrum
    const typename Cplx<T>::type* tw; // twiddles e^{-2 pi i j / n}
    int n, logn, P;                   // P: row pairs per block of the row passes
    double d1, d2, wp;                // pair-block constants and omega+
    double bp, bm;                    // b+ and b- of U
    double nscale;                    // 1 / N_Omega
};

// column-pass threads: 9 n / 16 (the column FFT's butterflies), at most 288 (n <= 512) or 576
// (n = 1024); the smaller bound leaves the FP64 solve more registers
constexpr int kFsColThreadsSmall = 288, kFsColThreadsLarge = 576;

inline int fs_col_threads(int n) {
    const int t = (9 * n / 16 + 31) / 32 * 32;
    return t < 32 ? 32 : t;
}
template <typename T>
inline size_t fs_col_smem(int n) {
    return (size_t)9 * padded_len(n) * sizeof(typename Cplx<T>::type);
}

// residual rows -> half spectrum over 0 <= j_x <= n/2 (negative j_x by Hermitian symmetry)
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_fs_rowfwd(FsArgs<T> A) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = A.n, logn = A.logn, P = A.P, plen = padded_len(n);
    const int nxh = n / 2 + 1;
    const int hr = n / 2;
    const int pair0 = blockIdx.x * P;  // P divides n/2: all pairs of the block lie in one field
    const int q = pair0 / hr;
    const int y0 = 2 * (pair0 - q * hr);
    const size_t off = ((size_t)q * n + y0) * n;
    const T* __restrict__ ft = A.ft + off;
    const T* __restrict__ f = A.f + off;
#pragma unroll 4
    for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
        const int p = t >> logn;
        const int x = t & (n - 1);
        const size_t o0 = (size_t)(2 * p) * n + x;
        C z;
        z.x = ft[o0] - f[o0];
        z.y = ft[o0 + n] - f[o0 + n];
        s[p * plen + pad(x)] = z;
    }
    __syncthreads();
    fft_stockham<C, false>(s, n, logn, P, A.tw);
    C* out = A.spec + (size_t)q * nxh * n + y0;
    const int l2p = __ffs(2 * P) - 1;
    for (int t = threadIdx.x; t < 2 * P * nxh; t += blockDim.x) {
        const int r = t & (2 * P - 1);
        const int jx = t >> l2p;
        const int p = r >> 1;
        const C zj = s[p * plen + pad(jx)];
        const C zm = s[p * plen + pad((n - jx) & (n - 1))];
        C v;
        if ((r & 1) == 0) {  // (zj + conj(zm)) / 2
            v.x = T(0.5) * (zj.x + zm.x);
            v.y = T(0.5) * (zj.y - zm.y);
        } else {             // (zj - conj(zm)) / (2i)
            v.x = T(0.5) * (zj.y + zm.y);
            v.y = T(-0.5) * (zj.x - zm.x);
        }
        out[(size_t)jx * n + r] = v;
    }
}

// half spectrum -> real rows, written as f + df
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_fs_rowinv(FsArgs<T> A) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = A.n, logn = A.logn, P = A.P, plen = padded_len(n);
    const int nxh = n / 2 + 1;
    const int hr = n / 2;
    const int pair0 = blockIdx.x * P;
    const int q = pair0 / hr;
    const int y0 = 2 * (pair0 - q * hr);
    const C* in = A.spec + (size_t)q * nxh * n + y0;
    const int lp = __ffs(P) - 1;
    // Z[p][j] = Xa + i Xb (j <= n/2), conj(Xa[n-j]) + i conj(Xb[n-j]) (j > n/2)
#pragma unroll 4
    for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
        const int p = t & (P - 1);
        const int j = t >> lp;
        C z;
        if (j <= n / 2) {
            const C xa = in[(size_t)j * n + 2 * p], xb = in[(size_t)j * n + 2 * p + 1];
            z.x = xa.x - xb.y;
            z.y = xa.y + xb.x;
        } else {
            const C xa = in[(size_t)(n - j) * n + 2 * p], xb = in[(size_t)(n - j) * n + 2 * p + 1];
            z.x = xa.x + xb.y;
            z.y = xb.x - xa.y;
        }
        s[p * plen + pad(j)] = z;
    }
    __syncthreads();
    fft_stockham<C, true>(s, n, logn, P, A.tw);
    const size_t off = ((size_t)q * n + y0) * n;
    const T* f = A.f + off;  // may alias out: each element is read, then written, by one thread
    T* out = A.out + off;
    for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
        const int p = t >> logn;
        const int x = t & (n - 1);
        const C z = s[p * plen + pad(x)];
        const size_t o0 = (size_t)(2 * p) * n + x;
        const T a0 = f[o0], a1 = f[o0 + n];
        out[o0] = a0 + z.x;
        out[o0 + n] = a1 + z.y;
    }
}

// ---- the per-wavevector solve (FP64) ------------------------------------------------------------

struct Cd {
    double x, y;
};
__device__ __forceinline__ Cd cd(double x, double y) { return Cd{x, y}; }
__device__ __forceinline__ Cd operator+(Cd a, Cd b) { return cd(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ Cd operator-(Cd a, Cd b) { return cd(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ Cd operator*(Cd a, Cd b) { return cd(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ Cd operator*(double s, Cd a) { return cd(s * a.x, s * a.y); }
__device__ __forceinline__ Cd operator*(Cd a, double s) { return cd(s * a.x, s * a.y); }
__device__ __forceinline__ Cd conjd(Cd a) { return cd(a.x, -a.y); }
__device__ __forceinline__ Cd cdiv(Cd a, Cd b) {
    const double d = 1.0 / (b.x * b.x + b.y * b.y);
    return cd((a.x * b.x + a.y * b.y) * d, (a.y * b.x - a.x * b.y) * d);
}

// The opposite pairs (q, qbar) of D2Q9 and the streaming symbol z_q = exp(-i k . c_q) =
// ex^{c_qx} ey^{c_qy} with ex = exp(-i k_x), ey = exp(-i k_y); z_qbar = conj(z_q).
__device__ __forceinline__ Cd fs_z(int q, Cd ex, Cd ey) {
    using L = D2Q9;
    Cd z = cd(1.0, 0.0);
    if (L::cx(q) == 1) z = ex;
    if (L::cx(q) == -1) z = conjd(ex);
    if (L::cy(q) == 1) z = z * ey;
    if (L::cy(q) == -1) z = z * conjd(ey);
    return z;
}

// value q of column j of U (j = 0: b+ w_q; j = 1, 2: b- w_q c_{qx,qy} / cs^2)
__device__ __forceinline__ double fs_u(int j, int q, double bp, double bm) {
    using L = D2Q9;
    return j == 0 ? bp * L::w(q) : (j == 1 ? bm * L::w(q) * 3.0 * L::cx(q) : bm * L::w(q) * 3.0 * L::cy(q));
}

// (x_q, x_qbar) = block^{-1} (b_q, b_qbar) for the pair block of A = I - Z((1 - w+) Pi+ + (1 - w-) Pi-),
// [[1 - z d1, -z d2], [-zb d2, 1 - zb d1]] with zb = conj(z); its inverse is
// [[1 - zb d1, z d2], [zb d2, 1 - z d1]] / det, det = 1 - 2 d1 Re z + d1^2 - d2^2 (|z| = 1)
__device__ __forceinline__ void fs_pair_solve(Cd z, double d1, double d2, Cd bq, Cd bb, Cd& xq, Cd& xb) {
    const Cd zb = conjd(z);
    const double id = 1.0 / (1.0 - 2.0 * d1 * z.x + d1 * d1 - d2 * d2);
    xq = id * ((cd(1.0, 0.0) - d1 * zb) * bq + d2 * (z * bb));
    xb = id * (d2 * (zb * bq) + (cd(1.0, 0.0) - d1 * z) * bb);
}

// accumulate P (rows 1, c_x, c_y) of value x at direction q
__device__ __forceinline__ void fs_pacc(int q, Cd x, Cd* m) {
    using L = D2Q9;
    m[0] = m[0] + x;
    if (L::cx(q)) m[1] = m[1] + (double)L::cx(q) * x;
    if (L::cy(q)) m[2] = m[2] + (double)L::cy(q) * x;
}

// the first member of pair i (1, 2, 5, 6; their opposites are 3, 4, 7, 8)
__host__ __device__ constexpr int fs_pair_q(int i) { return i == 0 ? 1 : (i == 1 ? 2 : (i == 2 ? 5 : 6)); }

// df = (I - Z J)^{-1} r at one wavevector, in place on v (9 values); (cx_, sx_) = (cos, sin) k_x
// and likewise for y.  Woodbury: y = A^{-1} r, S = I - P A^{-1} Z U, t = S^{-1} P y,
// df = y + A^{-1} Z U t; A^{-1} applied pair by pair so that no 9 x 3 block is held.
__device__ __forceinline__ void fs_solve(Cd* v, double ckx, double skx, double cky, double sky, double d1, double d2,
                                         double wp, double bp, double bm) {
    using L = D2Q9;
    const Cd ex = cd(ckx, -skx), ey = cd(cky, -sky);
    // y = A^{-1} r, in place, and P y
    v[0] = (1.0 / wp) * v[0];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int q = fs_pair_q(i), qb = L::opp(q);
        Cd xq, xb;
        fs_pair_solve(fs_z(q, ex, ey), d1, d2, v[q], v[qb], xq, xb);
        v[q] = xq;
        v[qb] = xb;
    }
    Cd py[3] = {cd(0.0, 0.0), cd(0.0, 0.0), cd(0.0, 0.0)};
#pragma unroll
    for (int q = 0; q < L::Q; ++q) fs_pacc(q, v[q], py);
    // S = I - P A^{-1} Z U, column by column (z_0 = 1 for the rest particle)
    Cd S[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        Cd pw[3] = {cd(0.0, 0.0), cd(0.0, 0.0), cd(0.0, 0.0)};
        fs_pacc(0, cd(fs_u(j, 0, bp, bm) / wp, 0.0), pw);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int q = fs_pair_q(i), qb = L::opp(q);
            const Cd z = fs_z(q, ex, ey);
            Cd xq, xb;
            fs_pair_solve(z, d1, d2, fs_u(j, q, bp, bm) * z, fs_u(j, qb, bp, bm) * conjd(z), xq, xb);
            fs_pacc(q, xq, pw);
            fs_pacc(qb, xb, pw);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) S[i][j] = (i == j ? cd(1.0, 0.0) : cd(0.0, 0.0)) - pw[i];
    }
    // t = S^{-1} P y by Cramer's rule
    const Cd c00 = S[1][1] * S[2][2] - S[1][2] * S[2][1];
    const Cd c01 = S[1][2] * S[2][0] - S[1][0] * S[2][2];
    const Cd c02 = S[1][0] * S[2][1] - S[1][1] * S[2][0];
    const Cd det = S[0][0] * c00 + S[0][1] * c01 + S[0][2] * c02;
    const Cd t0 = cdiv(py[0] * c00 + py[1] * (S[0][2] * S[2][1] - S[0][1] * S[2][2]) +
                           py[2] * (S[0][1] * S[1][2] - S[0][2] * S[1][1]),
                       det);
    const Cd t1 = cdiv(py[0] * c01 + py[1] * (S[0][0] * S[2][2] - S[0][2] * S[2][0]) +
                           py[2] * (S[0][2] * S[1][0] - S[0][0] * S[1][2]),
                       det);
    const Cd t2 = cdiv(py[0] * c02 + py[1] * (S[0][1] * S[2][0] - S[0][0] * S[2][1]) +
                           py[2] * (S[0][0] * S[1][1] - S[0][1] * S[1][0]),
                       det);
    // df = y + A^{-1} Z U t
    {
        const Cd g0 = fs_u(0, 0, bp, bm) * t0 + fs_u(1, 0, bp, bm) * t1 + fs_u(2, 0, bp, bm) * t2;
        v[0] = v[0] + (1.0 / wp) * g0;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int q = fs_pair_q(i), qb = L::opp(q);
        const Cd z = fs_z(q, ex, ey);
        const Cd gq = z * (fs_u(0, q, bp, bm) * t0 + fs_u(1, q, bp, bm) * t1 + fs_u(2, q, bp, bm) * t2);
        const Cd gb = conjd(z) * (fs_u(0, qb, bp, bm) * t0 + fs_u(1, qb, bp, bm) * t1 + fs_u(2, qb, bp, bm) * t2);
        Cd xq, xb;
        fs_pair_solve(z, d1, d2, gq, gb, xq, xb);
        v[q] = v[q] + xq;
        v[qb] = v[qb] + xb;
    }
}

// one kept j_x per block: FFT along y of the 9 fields, the solve at every j_y, inverse FFT
template <typename T, bool LARGE>
__global__ void __launch_bounds__(LARGE ? kFsColThreadsLarge : kFsColThreadsSmall) k_fs_col(FsArgs<T> A) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = A.n, logn = A.logn, plen = padded_len(n);
    const int nxh = n / 2 + 1;
    const int jx = blockIdx.x;
    C* col = A.spec + (size_t)jx * n;  // spec[q][jx][y] at col + q * nxh * n + y
    const size_t fs = (size_t)nxh * n;
    for (int t = threadIdx.x; t < 9 * n; t += blockDim.x) {
        const int q = t >> logn;
        const int y = t & (n - 1);
        s[q * plen + pad(y)] = col[q * fs + y];
    }
    __syncthreads();
    fft_stockham<C, false>(s, n, logn, 9, A.tw);
    double skx, ckx;
    sincospi(2.0 * (double)jx / (double)n, &skx, &ckx);  // k_x = 2 pi j_x / n
    for (int jy = threadIdx.x; jy < n; jy += blockDim.x) {
        const int jys = jy <= n / 2 ? jy : jy - n;
        double sky, cky;
        sincospi(2.0 * (double)jys / (double)n, &sky, &cky);
        Cd v[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const C e = s[q * plen + pad(jy)];
            v[q] = cd(A.nscale * (double)e.x, A.nscale * (double)e.y);
        }
        fs_solve(v, ckx, skx, cky, sky, A.d1, A.d2, A.wp, A.bp, A.bm);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            C e;
            e.x = (T)v[q].x;
            e.y = (T)v[q].y;
            s[q * plen + pad(jy)] = e;
        }
    }
    __syncthreads();
    fft_stockham<C, true>(s, n, logn, 9, A.tw);
    for (int t = threadIdx.x; t < 9 * n; t += blockDim.x) {
        const int q = t >> logn;
        const int y = t & (n - 1);
        col[q * fs + y] = s[q * plen + pad(y)];
    }
}

}  // namespace msc
