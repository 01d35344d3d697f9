// D3Q19 collide-stream sweep in push form with population halos: the explicit D3Q19 LBM step (the
// baseline, EXPLICIT) and, in its general form, the fused sweep of the corrected iteration (Eqs.
// macro-reconstruct, source-moments, source-distribution, collision-operating, sweep, residual).
// The march and the stage call use the halo-free sweep of sweep3p.cuh instead, so only the explicit
// step is instantiated.
//
// Design: a block owns a 32 x TYB tile of (x, y) columns (30 x (TYB-2) output columns plus a
// one-column halo on each side) and marches along z over HB output planes.  For each plane it
// loads the 19 populations of its tile with coalesced row loads, collides every site, writes the
// 16 directions that move in x or y to shared memory, and gathers from there the value that
// arrives at each output column; the z component of streaming is handled by keeping the partial
// output planes z-1, z, z+1 in registers, as in the 2D sweep.  Plane z-1 is complete after plane
// z is collided, so its residual moments and sum r^2 are formed and it is stored.
#pragma once

#include "common.cuh"
#include "sweep2d.cuh"

namespace msc {

struct Sweep3Geom {
    int tyb, nsx, nsy, hb, nzblk, blocks, threads;
    size_t smem;
};

template <typename T>
struct Sweep3Args {
    const T* fin;
    const T* dm;
    const T* h;
    T* fout;
    T* pr;
    double a;
    double inv;  // stateless mode: 1 / (1 + a/2), formed on the host
    int lift;
    double* sumsq_out;
    double* partial;
    unsigned int* counter;
    int n;
    Sweep3Geom g;
    DevState* st;
    T* fbase;
    size_t fstride;
    double* hist;
    int hist_cap;
    const int* replay_counts;
    int max_steps;
    cudaGraphConditionalHandle h_iter;
    int cond;
    int ex_dir, ex_count;
    cudaGraphConditionalHandle h_ex;
};

// index of a direction that moves in x or y among the 16 such directions (k not in {0, 5, 6})
__host__ __device__ constexpr int shift_slot(int k) { return k - (k > 0) - (k > 5) - (k > 6); }

inline Sweep3Geom sweep3_geometry(int n, int elem) {
    Sweep3Geom g;
    // 32 x 8 tiles in both precisions: at 127 registers per thread (FP32) a 512-thread block of 32 x 16
    // leaves one block per SM, whose two barriers per plane stall all 16 warps at once; two
    // independent 256-thread blocks per SM hide them better despite the extra halo rows (A/B at
    // N = 128 FP32: tiles 32 x 16 with 16 planes 162 us, 32 x 8 with 16 planes 149 us, with 32 or 64
    // planes 160-170 us; the march 5.10 -> 4.85 ms)
    g.tyb = 8;
    g.nsx = (n + kStripOut - 1) / kStripOut;
    g.nsy = (n + (g.tyb - 2) - 1) / (g.tyb - 2);
    const int target_blocks = elem == 8 ? 2 * 148 : 4 * 148;
    int hb = 4;
    for (int c = 64; c >= 4; c >>= 1) {
        if (c <= n && g.nsx * g.nsy * (n / c) >= target_blocks) { hb = c; break; }
    }
    if (hb > n) hb = n;
    g.hb = hb;
    g.nzblk = n / hb;
    g.blocks = g.nsx * g.nsy * g.nzblk;
    g.threads = 32 * g.tyb;
    g.smem = (size_t)2 * 16 * g.tyb * 32 * elem;  // two exchange buffers, alternating by plane
    return g;
}

template <typename T, bool EXPLICIT, bool GRAPH>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512) k_sweep3(Sweep3Args<T> A) {
    if constexpr (EXPLICIT && GRAPH) wait_for_predecessor();  // the explicit graph chains its steps on programmatic edges
    using L = D3Q19;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sC0 = reinterpret_cast<T*>(smem_raw);  // [2][16][TYB][32]: plane j uses buffer j & 1
    const int tyb = A.g.tyb;
    const int tx = threadIdx.x & 31;
    const int ty = threadIdx.x >> 5;
    const int n = A.n;
    const int m = n - 1;
    const size_t NNN = (size_t)n * n * n;

    const T* fin = A.fin;
    const T* dm = A.dm;
    const T* hh = A.h;
    T* fout = A.fout;
    T* pr = A.pr;
    T a = (T)A.a;
    T inv = (T)A.inv;
    int lift = A.lift;
    if (GRAPH) {
        const DevState* vs = A.st;
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

    const int b = blockIdx.x;
    const int sx = b % A.g.nsx;
    const int sy = (b / A.g.nsx) % A.g.nsy;
    const int zb = b / (A.g.nsx * A.g.nsy);
    const int x0 = sx * kStripOut;
    const int y0 = sy * (tyb - 2);
    const int z0 = zb * A.g.hb;
    const int x = (x0 - 1 + tx) & m;
    const int y = (y0 - 1 + ty) & m;
    const bool out_site = tx >= 1 && tx <= kStripOut && ty >= 1 && ty <= tyb - 2 &&
                          (x0 + tx - 1) < n && (y0 + ty - 1) < n;
    const size_t col = (size_t)y * n + x;

    T Ar[19], Br[19], ftp[19];
#pragma unroll
    for (int k = 0; k < 19; ++k) { Ar[k] = T(0); Br[k] = T(0); ftp[k] = T(0); }
    double ssq = 0.0;
    T ssq_f = T(0);

    for (int j = z0 - 1; j <= z0 + A.g.hb; ++j) {
        const size_t idx = (size_t)(j & m) * n * n + col;
        T f[19];
        const bool idx_ok = MSC_INB(idx, NNN, 3);
        if (idx_ok) {
#pragma unroll
            for (int k = 0; k < 19; ++k) f[k] = fin[k * NNN + idx];
        }
        if (!EXPLICIT && lift && idx_ok) {
            const T dp = dm[idx], dux = dm[NNN + idx], duy = dm[2 * NNN + idx], duz = dm[3 * NNN + idx];
#pragma unroll
            for (int k = 0; k < 19; ++k)
                f[k] += wmul<T>(L::w(k), dp + T(3) * (T(L::cx(k)) * dux + T(L::cy(k)) * duy + T(L::cz(k)) * duz));
        }
        T rho = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            rho += f[k];
            if (L::cx(k)) jx += T(L::cx(k)) * f[k];
            if (L::cy(k)) jy += T(L::cy(k)) * f[k];
            if (L::cz(k)) jz += T(L::cz(k)) * f[k];
        }
        T p, ux, uy, uz, s0 = T(0), sxx = T(0), syy = T(0), szz = T(0);
        if (EXPLICIT) {
            p = rho; ux = jx; uy = jy; uz = jz;
        } else {
            const size_t hi_ = idx_ok ? idx : 0;
            const T h0 = hh[hi_], h1 = hh[NNN + hi_], h2 = hh[2 * NNN + hi_], h3 = hh[3 * NNN + hi_];
            // m = P f + (h - a P f) / (2 (1 + a/2)): the rounded 1/(1 + a/2) scales only the O(a) term
            const T hinv = T(0.5) * inv;
            p = rho + (h0 - a * rho) * hinv;
            ux = jx + (h1 - a * jx) * hinv;
            uy = jy + (h2 - a * jy) * hinv;
            uz = jz + (h3 - a * jz) * hinv;
            s0 = h0 - a * p;
            sxx = h1 - a * ux;
            syy = h2 - a * uy;
            szz = h3 - a * uz;
        }
        const T A0 = p + T(0.5) * s0 - T(1.5) * (ux * ux + uy * uy + uz * uz) -
                     T(1.5) * (ux * sxx + uy * syy + uz * szz);
        T C[19];
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            const T cu = T(L::cx(k)) * ux + T(L::cy(k)) * uy + T(L::cz(k)) * uz;
            const T cs = T(L::cx(k)) * sxx + T(L::cy(k)) * syy + T(L::cz(k)) * szz;
            C[k] = wmul<T>(L::w(k), A0 + T(3) * cu + T(1.5) * cs + T(4.5) * cu * (cu + cs));
        }
        // x/y streaming through shared memory: the planes alternate between two buffers, so one
        // barrier per plane suffices (a buffer is rewritten two planes later, after every thread
        // has passed the barrier of the plane in between, hence finished reading it)
        T* sC = sC0 + (size_t)(j & 1) * 16 * tyb * 32;
#pragma unroll
        for (int k = 0; k < 19; ++k)
            if ((L::cx(k) != 0 || L::cy(k) != 0) && MSC_INB((shift_slot(k) * tyb + ty) * 32 + tx, 16 * tyb * 32, 4))
                sC[(shift_slot(k) * tyb + ty) * 32 + tx] = C[k];
        __syncthreads();
        if (out_site) {
#pragma unroll
            for (int k = 0; k < 19; ++k)
                if ((L::cx(k) != 0 || L::cy(k) != 0) && MSC_INB(ty - L::cy(k), tyb, 5) && MSC_INB(tx - L::cx(k), 32, 5))
                    C[k] = sC[(shift_slot(k) * tyb + (ty - L::cy(k))) * 32 + (tx - L::cx(k))];
        }
        // plane j-1 receives the c_z = -1 directions and is complete
#pragma unroll
        for (int k = 0; k < 19; ++k)
            if (L::cz(k) == -1) Ar[k] = C[k];
        if (j - 1 >= z0 && out_site && MSC_INB((size_t)((j - 1) & m) * n * n + col, NNN, 6)) {
            const size_t oidx = (size_t)((j - 1) & m) * n * n + col;
#pragma unroll
            for (int k = 0; k < 19; ++k) fout[k * NNN + oidx] = Ar[k];
            if (!EXPLICIT) {
                T r0 = T(0), r1 = T(0), r2 = T(0), r3 = T(0), rr = T(0);
#pragma unroll
                for (int k = 0; k < 19; ++k) {
                    const T r = Ar[k] - ftp[k];
                    r0 += r;
                    if (L::cx(k)) r1 += T(L::cx(k)) * r;
                    if (L::cy(k)) r2 += T(L::cy(k)) * r;
                    if (L::cz(k)) r3 += T(L::cz(k)) * r;
                    rr += r * r;
                }
                pr[oidx] = r0;
                pr[NNN + oidx] = r1;
                pr[2 * NNN + oidx] = r2;
                pr[3 * NNN + oidx] = r3;
                ssq_f += rr;
                if (((j - z0) & 7) == 0) { ssq += (double)ssq_f; ssq_f = T(0); }
            }
        }
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            if (L::cz(k) == 0) Ar[k] = C[k];
            else if (L::cz(k) == 1) { Ar[k] = Br[k]; Br[k] = C[k]; }
            ftp[k] = f[k];
        }
    }
    ssq += (double)ssq_f;
    if (EXPLICIT) return;

    __shared__ double wsum[16];
    __shared__ bool is_last;
    const int lane = tx, warp = ty, nwarps = tyb;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, off);
    if (lane == 0) wsum[warp] = ssq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double bs = 0.0;
        for (int w = 0; w < nwarps; ++w) bs += wsum[w];
        A.partial[blockIdx.x] = bs;
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
        for (int w = 0; w < nwarps; ++w) total += wsum[w];
        *A.counter = 0u;
        if (GRAPH) {
            march_after_sweep(A.st, total, 19.0 * (double)NNN, A.hist, A.hist_cap, A.replay_counts,
                              A.max_steps, A.h_iter, A.cond);
        } else {
            *A.sumsq_out = total;
        }
    }
}

template <typename T>
int set_sweep3_smem_limits(int n) {
    const Sweep3Geom g = sweep3_geometry(n, sizeof(T));
    const int bytes = (int)g.smem;
    if (cudaFuncSetAttribute(k_sweep3<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) return 1;
    return 0;
}

}  // namespace msc
