// D2Q9 fused collide-stream sweep (Eqs. macro-reconstruct, source-moments, source-distribution,
// collision-operating, sweep, residual) and the explicit LBM step (same kernel, no source).
//
// Design: one warp owns a strip of 32 consecutive x columns (30 output columns plus one halo
// column on each side) and marches down HB output rows of that strip.  For every row j it loads
// the 9 populations (plus h and the lifted correction) of its 32 columns with coalesced loads,
// forms the trial populations, the reconstructed field and the operating-point collision
// C = f_eq + Phi/2 at every column, and pushes the 9 post-collision values to their
// destinations x + c_k: x-shifts by warp shuffles, y-shifts by keeping the partial output rows
// j-1, j, j+1 in registers.  Row j-1 is complete after row j is collided, so the residual
// r = f_T - f, its moments P r and sum r^2 are formed there and the row is stored.  No shared
// memory and no block barriers in the main loop; each population is read once from memory
// except the two halo columns per strip and the two halo rows per row block.
#pragma once

#include "common.cuh"

namespace msc {

constexpr int kSweepWarps = 4;          // warps (strips) per block
constexpr int kStripOut = 30;           // output columns per warp strip

template <typename T, typename S = T>  // T: arithmetic and field type, S: population storage
struct Sweep2Args {
    // stateless mode: explicit pointers; graph mode: pointers resolved from the device state
    const S* fin;
    const T* dm;
    const T* h;
    S* fout;
    T* pr;
    double a;
    double inv;     // stateless mode: 1 / (1 + a/2), formed on the host
    double fscale;  // stateless mode: population storage scale (FP16 storage holds f / fscale)
    double omega_p, omega_m;  // stateless mode: TRT rates of the general collision (TRT kernels only)
    int lift;
    double* sumsq_out;
    // reduction scratch
    double* partial;
    unsigned int* counter;
    // geometry
    int n, nstrips, hb, nrowblk;
    // graph mode
    DevState* st;
    S* fbase;
    size_t fstride;  // elements
    double* hist;
    int hist_cap;
    const int* replay_counts;
    int max_steps;
    cudaGraphConditionalHandle h_iter;
    int cond;  // set the inner loop's graph conditional (0 when the march is driven from the host)
    // explicit graph mode: 0 = a->b, 1 = b->a; ex_count: decrement the pair counter
    int ex_dir, ex_count;
    cudaGraphConditionalHandle h_ex;
};

// Decide acceptance after the residual norm of inner iteration l is known (Algorithm 1).
__device__ inline void march_after_sweep(DevState* st, double total, double qsites, double* hist,
                                         int hist_cap, const int* replay_counts, int max_steps,
                                         cudaGraphConditionalHandle h_iter, int cond) {
    const double R = sqrt(total / qsites);
    const int ell = st->iter + 1;
    st->iter = ell;
    st->inner_total += 1;
    hist[st->hist_pos % hist_cap] = R;
    st->hist_pos += 1;
    st->R_last = R;
    // the sweep output becomes the base of the next trial
    const int t = st->slot_cur;
    st->slot_cur = st->slot_nxt;
    st->slot_nxt = t;
    int cont = 0, corr = 0;
    bool accept;
    if (st->replay) {
        const int idx = st->steps_in_call;
        accept = idx < max_steps && ell == replay_counts[idx];
    } else {
        accept = ell >= st->nmin && R < st->eps && ell % st->count_multiple == 0;  // a NaN never passes
    }
    if (!isfinite(R)) {
        st->status = MSC_ERR_NONFINITE;
    } else if (accept) {
        st->accepted = 1;
    } else if (ell >= st->kmax) {
        st->status = MSC_ERR_NONCONVERGED;
    } else {
        cont = 1;
        corr = st->corrector;
    }
    st->lift = corr;
    if (cond) cudaGraphSetConditional(h_iter, cont);  // another inner iteration (correction, sweep)
}

// One warp unit of the sweep: output columns [strip*30, strip*30 + 30) of rows [rb*hb, rb*hb + hb).
// Returns this lane's share of sum r^2 (zero in EXPLICIT mode).  Called by all 32 lanes.
// HPAIR: h is a binary32 pair, the low parts at hh + 3 n^2 (the march's working field); the
// differences h - a m are then formed as fma(-a, m, h_hi) + h_lo.
template <typename T, typename S, bool EXPLICIT, bool TRT = false, bool HPAIR = false>
__device__ __forceinline__ double sweep2_unit(const S* fin, const T* dm, const T* hh, S* fout, T* pr, T a, T inv,
                                              int lift, int n, int hb, int strip, int rb, int lane,
                                              T sig = T(1), T isig = T(1), T wp = T(1), T wm = T(1)) {
    using L = D2Q9;
    const int nmask = n - 1;
    const size_t NN = (size_t)n * n;
    double ssq = 0.0;
    const int x0 = strip * kStripOut;
    const int y0 = rb * hb;
    const int x = (x0 - 1 + lane) & nmask;
    const bool out_lane = lane >= 1 && lane <= kStripOut && (x0 + lane - 1) < n;

    T Ar[9], Br[9], ftp[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) { Ar[k] = T(0); Br[k] = T(0); ftp[k] = T(0); }
    T ssq_f = T(0);

    // software pipeline, two rows deep: the loads of rows j+1 and j+2 are in flight while row j is
    // collided (a warp keeps ~2 rows x 15 values of 128 B outstanding; the kernel is bound by load
    // latency, not by issue)
    T nf[9], ndp = T(0), ndx = T(0), ndy = T(0), nh[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};  // row j+1
    T qf[9], qdp = T(0), qdx = T(0), qdy = T(0), qh[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};  // row j+2
    auto load_row = [&](int jr, T* g, T& gdp, T& gdx, T& gdy, T* gh) {
        const size_t id = (size_t)(jr & nmask) * n + x;
        if (!MSC_INB(id, NN, 1)) return;
#pragma unroll
        for (int k = 0; k < 9; ++k) g[k] = ld_pop<T, S>(fin, k * NN + id, sig);
        if (!EXPLICIT) {
            if (lift) { gdp = dm[id]; gdx = dm[NN + id]; gdy = dm[2 * NN + id]; }
#pragma unroll
            for (int c = 0; c < (HPAIR ? 6 : 3); ++c) gh[c] = hh[c * NN + id];
        }
    };
    load_row(y0 - 1, nf, ndp, ndx, ndy, nh);
    load_row(y0, qf, qdp, qdx, qdy, qh);
    for (int j = y0 - 1; j <= y0 + hb; ++j) {
        T f[9], hv[6];
#pragma unroll
        for (int k = 0; k < 9; ++k) { f[k] = nf[k]; nf[k] = qf[k]; }
#pragma unroll
        for (int c = 0; c < 6; ++c) { hv[c] = nh[c]; nh[c] = qh[c]; }
        const T dp = ndp, dux = ndx, duy = ndy;
        ndp = qdp; ndx = qdx; ndy = qdy;
        if (j + 2 <= y0 + hb) load_row(j + 2, qf, qdp, qdx, qdy, qh);
        if (!EXPLICIT && lift) {  // trial f = f_T,prev + E dm   (Eq. lift)
#pragma unroll
            for (int k = 0; k < 9; ++k)
                f[k] += wmul<T>(L::w(k), dp + T(3) * (T(L::cx(k)) * dux + T(L::cy(k)) * duy));
        }
        // moments (Eq. moments)
        T rho = T(0), jx = T(0), jy = T(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            rho += f[k];
            if (L::cx(k)) jx += T(L::cx(k)) * f[k];
            if (L::cy(k)) jy += T(L::cy(k)) * f[k];
        }
        T p, ux, uy, s0 = T(0), sx = T(0), sy = T(0);
        T yx = T(0), yy = T(0);  // HPAIR: u = (jx + yx, jy + yy) kept unrounded for the collision
        if (EXPLICIT) {
            p = rho; ux = jx; uy = jy;
        } else {  // half-source reconstruction and source moments (Eqs. macro-reconstruct, source-moments)
            // m = (P f + h/2) / (1 + a/2) written as P f + (h - a P f) / (2 (1 + a/2)): the rounded
            // 1/(1 + a/2) then scales only the O(a) term, not m itself, so it cannot bias the moments
            // by a relative unit roundoff (which the long-wave solve would amplify by ~1/a)
            const T hinv = T(0.5) * inv;
            if constexpr (HPAIR) {
                // d = h - a P f with h = hi + lo: the FMA forms hi - a P f exactly and rounds once, then
                // lo is added, so d keeps its own relative accuracy where h ~ a m.  The source follows
                // from d alone, s = h - a m = (h - a P f) / (1 + a/2): it never sees the rounding of m
                // (a u_r |m| = u_r |h| absolute, as large as the rounding of a single binary32 h).
                const T d0 = fma(-a, rho, hv[0]) + hv[3];
                const T dx = fma(-a, jx, hv[1]) + hv[4];
                const T dy = fma(-a, jy, hv[2]) + hv[5];
                p = rho + d0 * hinv;
                yx = dx * hinv;
                yy = dy * hinv;
                ux = jx + yx;
                uy = jy + yy;
                s0 = d0 * inv;
                sx = dx * inv;
                sy = dy * inv;
            } else {
                p = rho + (hv[0] - a * rho) * hinv;
                ux = jx + (hv[1] - a * jx) * hinv;
                uy = jy + (hv[2] - a * jy) * hinv;
                s0 = hv[0] - a * p;
                sx = hv[1] - a * ux;
                sy = hv[2] - a * uy;
            }
        }
        T C[9];
        // the exact dominant term serves FP32 storage (the matched-accuracy march); binary16 storage
        // rounds every stored population to 2^-11, which swamps the binary32 collision rounding that
        // the exact term removes, and takes the plain collision below (fewer instructions per site)
        if constexpr (!TRT && HPAIR && std::is_same<S, float>::value) {
            // operating-point collision C = f_eq + Phi/2 (Eq. collision-operating) in binary32 with the
            // dominant term kept exact.  With u = J + Y (J = P_u f the moment sums, Y the O(a) correction)
            // C_k = (3 w_k) c_k.J + w_k (A0 + 3 c_k.Y + 1.5 c_k.s + 4.5 c_k.u (c_k.u + c_k.s)): the first
            // term is ~10^3 times the rest and is formed exactly (two-sum of c_k.J, two-product with the
            // split weight 3 w_k = hi + lo), the rest is small and rounds relative to its own size, and
            // the sum rounds once.  Forming u = J + Y in binary32 instead would quantise the slowly
            // varying Y on the grid of J: a rounding error that is smooth across sites, so that the
            // collision's mass and momentum are off by a long-wave field which the shadow solve's
            // 1/(a + nu |k|^2) and the march's steps accumulate (at N = 1024, dt = 307, ~40 times the
            // level of independent per-site rounding errors).
            const T A0 = p + T(0.5) * s0 - T(1.5) * (ux * ux + uy * uy) - T(1.5) * (ux * sx + uy * sy);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const T cs = T(L::cx(k)) * sx + T(L::cy(k)) * sy;
                if (L::cx(k) == 0 && L::cy(k) == 0) {
                    C[k] = wmul<T>(L::w(k), A0 + T(1.5) * cs);
                    continue;
                }
                T cjh, cje = T(0);  // c_k.J = cjh + cje exactly
                if (L::cx(k) != 0 && L::cy(k) != 0) two_sum(T(L::cx(k)) * jx, T(L::cy(k)) * jy, cjh, cje);
                else cjh = L::cx(k) != 0 ? T(L::cx(k)) * jx : T(L::cy(k)) * jy;
                const T cyk = T(L::cx(k)) * yx + T(L::cy(k)) * yy;
                const T cu = cjh + (cje + cyk);
                const T small = A0 + T(3) * (cje + cyk) + T(1.5) * cs + T(4.5) * cu * (cu + cs);
                const T w3h = (T)(3.0 * L::w(k)), w3l = (T)(3.0 * L::w(k) - (double)w3h);
                const T ph = w3h * cjh;
                const T pe = fma(w3h, cjh, -ph) + w3l * cjh;
                C[k] = ph + (pe + wmul<T>(L::w(k), small));
            }
        } else if constexpr (!TRT) {
            // operating-point collision C = f_eq + Phi/2 (Eq. collision-operating)
            const T A0 = p + T(0.5) * s0 - T(1.5) * (ux * ux + uy * uy) - T(1.5) * (ux * sx + uy * sy);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const T cu = T(L::cx(k)) * ux + T(L::cy(k)) * uy;
                const T cs = T(L::cx(k)) * sx + T(L::cy(k)) * sy;
                C[k] = wmul<T>(L::w(k), A0 + T(3) * cu + T(1.5) * cs + T(4.5) * cu * (cu + cs));
            }
        } else {
            // general TRT collision (Eq. collision): even / odd parts of f, f_eq (Eq. feq) and the
            // source distribution Phi (Eq. source-distribution) relax at omega+ / omega-
            const T B0 = p - T(1.5) * (ux * ux + uy * uy);
            const T us = ux * sx + uy * sy;
            T E[9], Ph[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const T cu = T(L::cx(k)) * ux + T(L::cy(k)) * uy;
                const T cs = T(L::cx(k)) * sx + T(L::cy(k)) * sy;
                E[k] = wmul<T>(L::w(k), B0 + T(3) * cu + T(4.5) * cu * cu);
                Ph[k] = wmul<T>(L::w(k), s0 + T(3) * (cs - us) + T(9) * cu * cs);
            }
            const T hp = T(1) - T(0.5) * wp, hm = T(1) - T(0.5) * wm;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int o = L::opp(k);
                const T fp = T(0.5) * (f[k] + f[o]), fm = T(0.5) * (f[k] - f[o]);
                const T ep = T(0.5) * (E[k] + E[o]), em = T(0.5) * (E[k] - E[o]);
                const T pp = T(0.5) * (Ph[k] + Ph[o]), pm = T(0.5) * (Ph[k] - Ph[o]);
                C[k] = f[k] - wp * (fp - ep) - wm * (fm - em) + hp * pp + hm * pm;
            }
        }
        // push streaming in x: value for column x comes from column x - c_kx
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (L::cx(k) == 1) C[k] = __shfl_up_sync(0xffffffffu, C[k], 1);
            else if (L::cx(k) == -1) C[k] = __shfl_down_sync(0xffffffffu, C[k], 1);
        }
        // row j-1 receives the c_y = -1 directions and is complete
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (L::cy(k) == -1) Ar[k] = C[k];
        if (j - 1 >= y0 && out_lane && MSC_INB((size_t)((j - 1) & nmask) * n + x, NN, 2)) {
            const size_t oidx = (size_t)((j - 1) & nmask) * n + x;
#pragma unroll
            for (int k = 0; k < 9; ++k) st_pop<T, S>(fout, k * NN + oidx, Ar[k], isig);
            if (!EXPLICIT) {
                T r0 = T(0), r1 = T(0), r2 = T(0), rr = T(0);
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const T r = Ar[k] - ftp[k];
                    r0 += r;
                    if (L::cx(k)) r1 += T(L::cx(k)) * r;
                    if (L::cy(k)) r2 += T(L::cy(k)) * r;
                    rr += r * r;
                }
                pr[oidx] = r0;
                pr[NN + oidx] = r1;
                pr[2 * NN + oidx] = r2;
                ssq_f += rr;
                if (((j - y0) & 7) == 0) { ssq += (double)ssq_f; ssq_f = T(0); }
            }
        }
        // rotate: row j keeps its c_y = 0 values and the c_y = +1 values of row j-1
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (L::cy(k) == 0) Ar[k] = C[k];
            else if (L::cy(k) == 1) { Ar[k] = Br[k]; Br[k] = C[k]; }
            ftp[k] = f[k];
        }
    }
    ssq += (double)ssq_f;
    return ssq;
}

// FP32 operating-point sweeps keep five blocks (20 warps, two rows of loads in flight each) per SM
// HPAIR: h is the march's binary32 pair and the collision keeps its dominant term exact (graph-mode
// march sweeps with binary32 arithmetic, or the stage call msc_sweep_hpair); the explicit LBM keeps
// the plain binary32 collision
template <typename T, typename S, bool EXPLICIT, bool GRAPH, bool TRT = false,
          bool HPAIR = GRAPH && !EXPLICIT && std::is_same<T, float>::value>
__global__ void __launch_bounds__(kSweepWarps * 32, sizeof(T) == 4 && !TRT ? 5 : 1) k_sweep2(Sweep2Args<T, S> A) {
    // the graphs chain the explicit steps, and the march's corrections and the sweeps that follow
    // them, on programmatic edges
    if constexpr (GRAPH) wait_for_predecessor();
    if constexpr (GRAPH && !EXPLICIT) {
        // no live step: the march stopped with an error (sweeps outside the conditional loop), or
        // its last step is done (the second step of the graph's unrolled pair); the step's inner
        // loop stays closed
        if (A.st->status != MSC_OK || A.st->steps_target <= 0) {
            if (A.cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(A.h_iter, 0u);
            return;
        }
    }
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int n = A.n;
    const size_t NN = (size_t)n * n;

    const S* fin = A.fin;
    const T* dm = A.dm;
    const T* hh = A.h;
    S* fout = A.fout;
    T* pr = A.pr;
    T a = (T)A.a;
    T inv = (T)A.inv;
    int lift = A.lift;
    double fs = A.fscale, ifs = 1.0;  // stateless FP16 calls use fscale = 1
    double wpd = A.omega_p, wmd = A.omega_m;
    if (GRAPH) {
        const DevState* vs = A.st;
        if constexpr (!std::is_same<S, T>::value) { fs = vs->fscale; ifs = vs->isig; }
        if constexpr (TRT) { wpd = vs->omega_p; wmd = vs->omega_m; }
        if (EXPLICIT) {
            const int sa = vs->ex_a, sb = vs->ex_b;
            fin = A.fbase + (size_t)(A.ex_dir ? sb : sa) * A.fstride;
            fout = A.fbase + (size_t)(A.ex_dir ? sa : sb) * A.fstride;
            if (A.ex_count && blockIdx.x == 0 && threadIdx.x == 0) {
                DevState* st = A.st;
                const int left = st->ex_loops_left - 1;
                st->ex_loops_left = left;
                cudaGraphSetConditional(A.h_ex, left > 0 ? 1u : 0u);
            }
        } else {
            fin = A.fbase + (size_t)vs->slot_cur * A.fstride;
            fout = A.fbase + (size_t)vs->slot_nxt * A.fstride;
            a = (T)vs->a;
            inv = (T)vs->inv_a;
            lift = vs->lift;
        }
    }

    const int unit = blockIdx.x * kSweepWarps + warp;
    double ssq = 0.0;
    if (unit < A.nstrips * A.nrowblk)  // warp-uniform
        ssq = sweep2_unit<T, S, EXPLICIT, TRT, HPAIR>(
            fin, dm, hh, fout, pr, a, inv, lift, n, A.hb, unit % A.nstrips, unit / A.nstrips, lane, (T)fs, (T)ifs,
            (T)wpd, (T)wmd);
    if (EXPLICIT) return;

    // ---- residual norm: block partials, last block reduces in a fixed order ----
    __shared__ double wsum[kSweepWarps];
    __shared__ bool is_last;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, off);
    if (lane == 0) wsum[warp] = ssq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < kSweepWarps; ++w) b += wsum[w];
        A.partial[blockIdx.x] = b;
        __threadfence();
        const unsigned int t = atomicAdd(A.counter, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(A.partial + i);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __syncthreads();
    if (lane == 0) wsum[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double total = 0.0;
        for (int w = 0; w < kSweepWarps; ++w) total += wsum[w];
        *A.counter = 0u;
        if (GRAPH) {
            march_after_sweep(A.st, total, 9.0 * (double)NN, A.hist, A.hist_cap, A.replay_counts,
                              A.max_steps, A.h_iter, A.cond);
        } else {
            *A.sumsq_out = total;
        }
    }
}

struct Sweep2Geom {
    int nstrips, hb, nrowblk, blocks;
};

// Rows per warp unit: the largest row block (<= 64, dividing n) that still gives 12 warps per SM:
// fewer halo rows, and one resident wave where 16 warps per SM would need 1.5 (N = 1024: 560 blocks
// instead of 1120, the sweep 34 -> 29 us and the march 4.5 % faster; N = 2048: 105 -> 97 us).  Small
// lattices never reach 12 warps per SM and take min_rows: 2 for the march's sweep, 1 for the explicit
// LBM step, whose row chain is shorter (A/B at N = 128 / 256, FP32: march 7.73 / 16.38 ms with 4
// rows, 7.44 / 16.27 with 2, 7.48 / 17.04 with 1; explicit step 3.99 / 4.06 us with 4 rows, 3.14 /
// 3.50 with 2, 2.78 / 3.41 with 1; N >= 512 unchanged).
constexpr int kSweepMinRows = 2;
constexpr int kExplicitMinRows = 1;

constexpr Sweep2Geom sweep2_geometry(int n, int min_rows = kSweepMinRows) {
    Sweep2Geom g{};
    g.nstrips = (n + kStripOut - 1) / kStripOut;
    const int target_units = 148 * 12;
    int hb = min_rows;
    for (int c = 64; c >= min_rows; c >>= 1) {
        if (c <= n && g.nstrips * (n / c) >= target_units) { hb = c; break; }
    }
    if (hb > n) hb = n;
    g.hb = hb;
    g.nrowblk = n / hb;
    const int units = g.nstrips * g.nrowblk;
    g.blocks = (units + kSweepWarps - 1) / kSweepWarps;
    return g;
}

}  // namespace msc
