// D3Q19 fused sweep of the corrected iteration, halo-free form (same equations as the other sweeps:
// Eqs. macro-reconstruct, source-moments, source-distribution, collision-operating, sweep,
// residual).
//
// At the operating point the post-collision populations of a site depend on the site only through
// its reconstructed moments and source (Eq. collision-operating): C_k(y) = w_k (A0 + 3 c_k.u +
// 3/2 c_k.s + 9/2 c_k.u (c_k.u + c_k.s)) with A0 = p + s_0/2 - 3/2 u.u - 3/2 u.s.  The moments of
// a trial f = f_T + E dm are P f_T + dm (P E = I), so every sweep also writes P f_T of its output,
// and the next sweep finds the collision inputs K(y) = (A0, u, s) of any site from P f_T(y), dm(y)
// and h(y) alone: 4 + 4 + 4 (or 8 with the binary32 history pair) values instead of 19 populations
// and a full collision.  The streamed output at x is pulled, f_T,k(x) = C_k(x - c_k), from the K of
// the 18 neighbours.
//
// Design: a block owns a 32 x 8 tile of (x, y) columns, one thread per output column, and marches
// along z.  For every plane it computes K on the tile plus a one-site ring (34 x 10 sites, the ring
// costing moment loads only) into shared memory, in four rotating plane buffers so that one block
// barrier per plane separates the writers of plane z+1 from the readers of planes z-1, z, z+1.  A
// thread loads the 19 populations of its own site (coalesced, no halo), pulls its 19 outputs,
// forms the residual r = f_T - f, P r, sum r^2 and P f_T, and stores f_T, P f_T and P r.
#pragma once

#include "common.cuh"
#include "sweep2d.cuh"

namespace msc {

// 32 x 8 output tiles, four 256-thread blocks (64 registers) per SM.  A/B of the FP32 march's
// kernel (binary32 history pair): 32 x 4 tiles at eight blocks per SM 0.65 / 0.68 of the measured
// HBM bandwidth at N = 128 / 256, 32 x 8 at four 0.66 / 0.74, 32 x 16 at two 0.57 / 0.68 (the ring
// costs moment loads per output site in the ratio 204 : 128, 340 : 256, 612 : 512).
constexpr int kP3TX = 32, kP3TY = 8;                        // output tile (x, y)
constexpr int kP3RX = kP3TX + 2, kP3RY = kP3TY + 2;         // tile plus ring
constexpr int kP3Ring = kP3RX * kP3RY;                      // 340 sites per plane
constexpr int kP3Threads = kP3TX * kP3TY;                   // 256
constexpr int kP3K = 7;                                     // A0, ux, uy, uz, sx, sy, sz
constexpr int kP3Bufs = 4;

struct Sweep3PGeom {
    int nsx, nsy, hb, nzblk, blocks;
    size_t smem;
};

// A block marches one column (x, y tile) over hb planes, recomputing two ring planes at its start:
// the longest run that still gives about four blocks per SM.  (Runs balanced to fill exactly one
// resident wave, e.g. nine runs of 14-15 planes per column at N = 128, measured no faster at N = 128
// and 11 % slower at N = 256 than this rule's 1.7 waves.)
inline Sweep3PGeom sweep3p_geometry(int n, int elem) {
    Sweep3PGeom g;
    g.nsx = (n + kP3TX - 1) / kP3TX;
    g.nsy = (n + kP3TY - 1) / kP3TY;
    const int target_blocks = 4 * 148;
    int hb = 4;
    for (int c = 64; c >= 4; c >>= 1) {
        if (c <= n && g.nsx * g.nsy * (n / c) >= target_blocks) { hb = c; break; }
    }
    if (hb > n) hb = n;
    g.hb = hb;
    g.nzblk = n / hb;
    g.blocks = g.nsx * g.nsy * g.nzblk;
    g.smem = (size_t)kP3Bufs * kP3K * kP3Ring * elem;
    return g;
}

template <typename T>
struct Sweep3PArgs {
    // stateless mode: explicit pointers
    const T* fin;    // 19 x sites
    const T* pfin;   // 4 x sites: P fin
    const T* dm;     // 4 x sites (lift)
    const T* h;      // 4 x sites, or 8 x sites (high parts, then low parts) with HPAIR
    T* fout;
    T* pfout;        // 4 x sites: P fout
    T* pr;
    double a, inv;
    int lift;
    double* sumsq_out;
    double* partial;
    unsigned int* counter;
    int n;
    Sweep3PGeom g;
    // graph mode: population ring and the P f of each ring slot
    DevState* st;
    T* fbase;
    size_t fstride;  // elements
    T* pfbase;
    size_t pfstride; // elements
    double* hist;
    int hist_cap;
    const int* replay_counts;
    int max_steps;
    cudaGraphConditionalHandle h_iter;
    int cond;
};

// K of the ring sites of plane zz (periodic index) into buffer b: thread t takes ring sites t, t + 256, ...
template <typename T, bool HPAIR>
__device__ __forceinline__ void p3_ring_plane(T* __restrict__ kb, const T* __restrict__ pfin,
                                              const T* __restrict__ dm, const T* __restrict__ hh, int lift, T a,
                                              T inv, int n, int x0, int y0, int zz) {
    const int m = n - 1;
    const size_t NNN = (size_t)n * n * n;
    const size_t zoff = (size_t)(zz & m) * n * n;
    const T hinv = T(0.5) * inv;
#pragma unroll
    for (int rep = 0; rep < (kP3Ring + kP3Threads - 1) / kP3Threads; ++rep) {
        const int r = threadIdx.x + rep * kP3Threads;
        if (r >= kP3Ring) break;
        const int rx = r % kP3RX, ry = r / kP3RX;
        const size_t id = zoff + (size_t)((y0 - 1 + ry) & m) * n + ((x0 - 1 + rx) & m);
        if (!MSC_INB(id, NNN, 20)) continue;
        T M[4], d[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) M[c] = pfin[c * NNN + id];
        if (lift) {
#pragma unroll
            for (int c = 0; c < 4; ++c) M[c] += dm[c * NNN + id];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if constexpr (HPAIR) d[c] = fma(-a, M[c], hh[c * NNN + id]) + hh[(4 + c) * NNN + id];
            else d[c] = hh[c * NNN + id] - a * M[c];
        }
        // m = P f + (h - a P f) / (2 (1 + a/2)),  s = h - a m = (h - a P f) / (1 + a/2)
        const T p = M[0] + d[0] * hinv;
        const T ux = M[1] + d[1] * hinv, uy = M[2] + d[2] * hinv, uz = M[3] + d[3] * hinv;
        const T s0 = d[0] * inv, sx = d[1] * inv, sy = d[2] * inv, sz = d[3] * inv;
        const T A0 = p + T(0.5) * s0 - T(1.5) * (ux * ux + uy * uy + uz * uz) - T(1.5) * (ux * sx + uy * sy + uz * sz);
        kb[0 * kP3Ring + r] = A0;
        kb[1 * kP3Ring + r] = ux;
        kb[2 * kP3Ring + r] = uy;
        kb[3 * kP3Ring + r] = uz;
        kb[4 * kP3Ring + r] = sx;
        kb[5 * kP3Ring + r] = sy;
        kb[6 * kP3Ring + r] = sz;
    }
}

template <typename T, bool GRAPH, bool HPAIR = GRAPH && std::is_same<T, float>::value>
__global__ void __launch_bounds__(kP3Threads, sizeof(T) == 4 ? 4 : 1) k_sweep3p(Sweep3PArgs<T> A) {
    using L = D3Q19;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* K0 = reinterpret_cast<T*>(smem_raw);  // [kP3Bufs][kP3K][kP3Ring]
    const int n = A.n, m = n - 1;
    const size_t NNN = (size_t)n * n * n;

    const T* fin = A.fin;
    const T* pfin = A.pfin;
    T* fout = A.fout;
    T* pfout = A.pfout;
    T a = (T)A.a, inv = (T)A.inv;
    int lift = A.lift;
    if (GRAPH) {
        wait_for_predecessor();  // a sweep that follows a correction on a programmatic edge
        const DevState* vs = A.st;
        if (vs->status != MSC_OK || vs->steps_target <= 0) {  // no live step (as the D2Q9 sweep)
            if (A.cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(A.h_iter, 0u);
            return;
        }
        fin = A.fbase + (size_t)vs->slot_cur * A.fstride;
        fout = A.fbase + (size_t)vs->slot_nxt * A.fstride;
        pfin = A.pfbase + (size_t)vs->slot_cur * A.pfstride;
        pfout = A.pfbase + (size_t)vs->slot_nxt * A.pfstride;
        a = (T)vs->a;
        inv = (T)vs->inv_a;
        lift = vs->lift;
    }
    const T* dm = A.dm;
    const T* hh = A.h;
    T* pr = A.pr;

    const int b = blockIdx.x;
    const int sx = b % A.g.nsx;
    const int sy = (b / A.g.nsx) % A.g.nsy;
    const int zb = b / (A.g.nsx * A.g.nsy);
    const int x0 = sx * kP3TX, y0 = sy * kP3TY, z0 = zb * A.g.hb, z1 = z0 + A.g.hb;
    const int tx = threadIdx.x % kP3TX, ty = threadIdx.x / kP3TX;
    const bool out_site = (x0 + tx) < n && (y0 + ty) < n;
    const size_t col = (size_t)((y0 + ty) & m) * n + ((x0 + tx) & m);
    const int rc = (ty + 1) * kP3RX + (tx + 1);  // own ring index

    p3_ring_plane<T, HPAIR>(K0 + (size_t)((z0 - 1) & (kP3Bufs - 1)) * kP3K * kP3Ring, pfin, dm, hh, lift, a, inv, n, x0,
                            y0, z0 - 1);
    p3_ring_plane<T, HPAIR>(K0 + (size_t)(z0 & (kP3Bufs - 1)) * kP3K * kP3Ring, pfin, dm, hh, lift, a, inv, n, x0, y0,
                            z0);
    double ssq = 0.0;
    for (int z = z0; z < z1; ++z) {
        const size_t idx = (size_t)(z & m) * n * n + col;
        const bool idx_ok = MSC_INB(idx, NNN, 21);
        // this site's populations and lift, in flight while the next ring plane is computed
        T f[19];
        T ldp = T(0), ldx = T(0), ldy = T(0), ldz = T(0);
        if (out_site && idx_ok) {
#pragma unroll
            for (int k = 0; k < 19; ++k) f[k] = fin[k * NNN + idx];
            if (lift) { ldp = dm[idx]; ldx = dm[NNN + idx]; ldy = dm[2 * NNN + idx]; ldz = dm[3 * NNN + idx]; }
        }
        p3_ring_plane<T, HPAIR>(K0 + (size_t)((z + 1) & (kP3Bufs - 1)) * kP3K * kP3Ring, pfin, dm, hh, lift, a, inv, n,
                                x0, y0, z + 1);
        __syncthreads();
        if (!out_site || !idx_ok) continue;
        T q0 = T(0), q1 = T(0), q2 = T(0), q3 = T(0);   // P f_T
        T r0 = T(0), r1 = T(0), r2 = T(0), r3 = T(0), rr = T(0);
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            const int cx = L::cx(k), cy = L::cy(k), cz = L::cz(k);
            // source y = x - c_k: ring index and plane buffer
            const T* kb = K0 + (size_t)((z - cz) & (kP3Bufs - 1)) * kP3K * kP3Ring;
            const int rs = rc - cy * kP3RX - cx;
            if (!MSC_INB(rs, kP3Ring, 22)) continue;
            T cu = T(0), cs = T(0);
            if (cx) { cu += T(cx) * kb[1 * kP3Ring + rs]; cs += T(cx) * kb[4 * kP3Ring + rs]; }
            if (cy) { cu += T(cy) * kb[2 * kP3Ring + rs]; cs += T(cy) * kb[5 * kP3Ring + rs]; }
            if (cz) { cu += T(cz) * kb[3 * kP3Ring + rs]; cs += T(cz) * kb[6 * kP3Ring + rs]; }
            const T Ck = wmul<T>(L::w(k), kb[rs] + T(3) * cu + T(1.5) * cs + T(4.5) * cu * (cu + cs));
            fout[k * NNN + idx] = Ck;
            q0 += Ck;
            if (cx) q1 += T(cx) * Ck;
            if (cy) q2 += T(cy) * Ck;
            if (cz) q3 += T(cz) * Ck;
            // trial f = f_T,prev + E dm   (Eq. lift)
            T fk = f[k];
            if (lift) fk += wmul<T>(L::w(k), ldp + T(3) * (T(cx) * ldx + T(cy) * ldy + T(cz) * ldz));
            const T r = Ck - fk;
            r0 += r;
            if (cx) r1 += T(cx) * r;
            if (cy) r2 += T(cy) * r;
            if (cz) r3 += T(cz) * r;
            rr += r * r;
        }
        pfout[idx] = q0;
        pfout[NNN + idx] = q1;
        pfout[2 * NNN + idx] = q2;
        pfout[3 * NNN + idx] = q3;
        pr[idx] = r0;
        pr[NNN + idx] = r1;
        pr[2 * NNN + idx] = r2;
        pr[3 * NNN + idx] = r3;
        ssq += (double)rr;
    }

    // ---- residual norm: block partials, last block reduces in a fixed order ----
    __shared__ double wsum[kP3Threads / 32];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, off);
    if (lane == 0) wsum[warp] = ssq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double bs = 0.0;
        for (int w = 0; w < kP3Threads / 32; ++w) bs += wsum[w];
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
        for (int w = 0; w < kP3Threads / 32; ++w) total += wsum[w];
        *A.counter = 0u;
        if (GRAPH) {
            march_after_sweep(A.st, total, 19.0 * (double)NNN, A.hist, A.hist_cap, A.replay_counts, A.max_steps,
                              A.h_iter, A.cond);
        } else {
            *A.sumsq_out = total;
        }
    }
}

// P f of a population array in the storage type (the input of a stateless halo-free sweep)
template <typename T>
__global__ void k_pop_moments3(const T* __restrict__ f, T* __restrict__ pf, size_t sites) {
    using L = D3Q19;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sites; i += (size_t)gridDim.x * blockDim.x) {
        T q0 = T(0), q1 = T(0), q2 = T(0), q3 = T(0);
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            const T v = f[k * sites + i];
            q0 += v;
            if (L::cx(k)) q1 += T(L::cx(k)) * v;
            if (L::cy(k)) q2 += T(L::cy(k)) * v;
            if (L::cz(k)) q3 += T(L::cz(k)) * v;
        }
        pf[i] = q0;
        pf[sites + i] = q1;
        pf[2 * sites + i] = q2;
        pf[3 * sites + i] = q3;
    }
}

template <typename T>
int set_sweep3p_smem_limits(int n) {
    const int bytes = (int)sweep3p_geometry(n, sizeof(T)).smem;
    if (cudaFuncSetAttribute(k_sweep3p<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ||
        cudaFuncSetAttribute(k_sweep3p<T, false, std::is_same<T, float>::value>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ||
        cudaFuncSetAttribute(k_sweep3p<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))
        return 1;
    return 0;
}

}  // namespace msc
