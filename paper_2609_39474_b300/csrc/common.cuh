// Shared definitions of the MSC-LBM CUDA library: lattice constants, device state, launch
// helpers.  Internal header (not part of the C ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/msclbm.h"

namespace msc {

// ---- bounds-checked debug build ---------------------------------------------------------------
// Built with -DMSC_BOUNDS_CHECK (libmsclbm_check.so), MSC_INB(i, n, site) tests 0 <= i < n at the
// index computations of the sweep strips, tiles and halos and of the shared-memory transforms; a
// failing test records the number of failures and the first failing site and index (read by
// msc_bounds_check_report) and the guarded access is skipped, so a bad index never reaches memory
// and nothing traps.  In the normal build MSC_INB is the constant true and compiles away.
#ifdef MSC_BOUNDS_CHECK
__device__ unsigned long long g_oob_count;
__device__ unsigned long long g_oob_first;  // site << 40 | (index & (2^40 - 1))
__device__ __forceinline__ bool inb_check(long long i, long long n, unsigned int site) {
    if (i >= 0 && i < n) return true;
    if (atomicAdd(&g_oob_count, 1ull) == 0ull)
        g_oob_first = ((unsigned long long)site << 40) | ((unsigned long long)i & 0xffffffffffull);
    return false;
}
#define MSC_INB(i, n, site) ::msc::inb_check((long long)(i), (long long)(n), (site))
#else
#define MSC_INB(i, n, site) true
#endif

// ---- lattices (Appendix A, Eqs. d2q9 and d3q19) -------------------------------------------

struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int D = 2;
    __host__ __device__ static constexpr int cx(int k) {
        return (k == 1 || k == 5 || k == 8) ? 1 : (k == 3 || k == 6 || k == 7) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cy(int k) {
        return (k == 2 || k == 5 || k == 6) ? 1 : (k == 4 || k == 7 || k == 8) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int k) {
        return k == 0 ? 4.0 / 9.0 : (k < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    // the direction with c = -c_k (TRT even/odd pairs, Eq. trt)
    __host__ __device__ static constexpr int opp(int k) {
        return k == 0 ? 0 : (k < 5 ? (k + 1) % 4 + 1 : (k - 3) % 4 + 5);
    }
};

struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr int D = 3;
    __host__ __device__ static constexpr int cx(int k) {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[k];
    }
    __host__ __device__ static constexpr int cy(int k) {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[k];
    }
    __host__ __device__ static constexpr int cz(int k) {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return t[k];
    }
    __host__ __device__ static constexpr double w(int k) {
        return k == 0 ? 1.0 / 3.0 : (k < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

// ---- device-resident march state -------------------------------------------------------------
// One instance per context, in the workspace.  Scalars written by single-thread control kernels
// and by the last block of the sweep; everything else reads them at kernel start with ordinary
// (L1-cached) loads: a kernel that writes the state does so only after every thread of it has
// read the fields it uses, and the caches start clean at every launch.  (Uncached reads of the
// same few lines by every thread of a grid queue up on one L2 slice.)
struct DevState {
    // parameters (set by msc_set_params)
    double nu, dt, eps;
    int kmax, nmin, corrector, replay;
    int warm_order;         // accepted states used by the warm start (1..3)
    int count_multiple;     // accepted inner counts are multiples of this (1 or 2)
    double force[3];        // uniform body force, added to the momentum part of h_q
    double omega_p, omega_m;  // TRT relaxation rates (1, 1 at the operating point)
    int params_ok;
    // physical-step bookkeeping
    int64_t steps_done;     // accepted steps since init
    int64_t inner_total;    // inner sweeps in the current march call
    int steps_target;       // steps still to run in this call
    int steps_in_call;      // steps accepted in this call
    int n_avail;            // accepted population states available for the warm start (1..3)
    int slot_fn[3];         // population ring slots of f^n, f^{n-1}, f^{n-2}
    int slot_cur, slot_nxt; // working slots: sweep reads cur (+lift), writes nxt
    int m_cur, m_prev;      // moment history slots of m^n, m^{n-1}
    int q;                  // BDF order of the current step
    double a;               // a_q
    // constants of the current step, formed once by the single-thread control kernels (an FP64
    // division costs ~10 FP64 instructions on a pipe that runs at ~1/58 of the FP32 rate)
    double inv_a;           // 1 / (1 + a_q / 2)
    double c1, c2;          // h_q = c1 m^n - c2 m^{n-1}
    double k1, k2;          // c1 inv_a / 2, c2 inv_a / 2: the history weights of the reconstruction
    double n1, n2;          // BDF2 coefficients 4 / (2 dt), 1 / (2 dt) of the next step
    double qa[2], qinv[2], qc1[2], qc2[2];  // a_q, 1 / (1 + a_q / 2), c1, c2 for q = 1, 2 (set with dt)
    double isig;            // 1 / fscale
    int iter;               // inner iterations done in the current step
    int lift;               // next sweep applies f = f_cur + E dm
    int accepted;           // current step accepted
    int status;             // MSC_OK or the error that stopped the march
    int last_iters, last_q;
    double R_last;
    int64_t hist_pos;       // total residuals recorded in the ring this call
    // explicit march
    int ex_a, ex_b;
    int ex_loops_left;
    // the next physical step's h and trial populations were already formed by k_step_end
    int prepared;
    // population storage scale sigma (a power of two): FP16 storage holds f / sigma; 1 otherwise
    double fscale;
    unsigned long long fmax_bits;  // max |f^0| (bits of a non-negative double) while sigma is chosen
};

// Layout of the context workspace (byte offsets from the workspace base).
// workspace bytes of an adjoint run of up to MSC_ADJOINT_CHUNK steps (position block, argument and
// outcome blocks; sizes checked where the blocks are defined)
constexpr size_t kAdjCtlBytes = 256, kAdjArgBytes = 160, kAdjStatBytes = 32;
constexpr size_t kAdjBytes = kAdjCtlBytes + MSC_ADJOINT_CHUNK * (kAdjArgBytes + kAdjStatBytes);

struct Layout {
    size_t state, fbuf, pf, mbuf, h, pr, dm, spec, tw, coef, partial, counter, adj, adjw, iters, hist, replay, total;
    size_t fstride;   // bytes of one population array
    size_t pfstride;  // elements of one P f field set (D3Q19)
};

constexpr int kNumFBuf = 5;

inline int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}
inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int lattice_q(int dim) { return dim == 2 ? 9 : 19; }

// size limits: shared-memory transforms hold one full line (2D) or plane chunk (3D) per block;
// FP16 population storage exists for D2Q9
inline bool valid_lattice(int dim, int n, int precision) {
    if (precision != MSC_FP64 && precision != MSC_FP32 && precision != MSC_FP16) return false;
    if (!is_pow2(n) || n < 8) return false;
    if (dim == 2) return n <= (precision == MSC_FP64 ? 2048 : 4096);
    if (dim == 3) return precision != MSC_FP16 && n <= (precision == MSC_FP64 ? 128 : 256);
    return false;
}

// binary32 <-> binary64 conversions on the integer pipe (IEEE 754 formats; B300's FP64 pipe, which
// executes the conversion instructions, runs at ~1/58 of the FP32 rate).  Same results as the
// hardware conversions; values outside the normal ranges take the hardware path.
// widen: exact.  The exponent field is re-biased by 1023 - 127 = 896, the mantissa moves up 29 bits.
__device__ __forceinline__ double widen_f32(float x) {
    const unsigned int b = __float_as_uint(x);
    const unsigned int mag = b & 0x7fffffffu;
    if (mag - 0x00800000u >= 0x7f000000u) return (double)x;  // zero, subnormal, inf, nan
    const unsigned long long d = ((unsigned long long)(b >> 31) << 63) |
                                 (((unsigned long long)mag + (896ull << 23)) << 29);
    return __longlong_as_double((long long)d);
}
// narrow: round to nearest, ties to even, for results in the normal binary32 range (double
// exponents 897 .. 1150); a carry out of the mantissa increments the exponent (to inf at the top).
__device__ __forceinline__ float narrow_f64(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    const unsigned int e = (unsigned int)(mag >> 52);
    if (e - 897u > 253u) return (float)x;  // zero, binary32 subnormal or overflow range, inf, nan
    const unsigned long long t = mag - (896ull << 52);
    unsigned int r = (unsigned int)(t >> 29);
    const unsigned int rem = (unsigned int)t & 0x1fffffffu;
    r += (rem > 0x10000000u) | ((rem == 0x10000000u) & (r & 1u));
    return __uint_as_float(((unsigned int)(b >> 63) << 31) | r);
}
// x = hi + lo with hi = x rounded to the nearest binary32 (ties to even) and lo = x - hi rounded to
// binary32, on the integer pipe, for x whose exponent lies in the normal binary32 range (other x
// take the hardware conversion with lo = 0).  x - hi is an integer multiple m of x's binary64 ulp
// with m <= 2^28, so lo = m 2^(E - 1075), E the biased binary64 exponent of x; when that scale
// falls below the binary32 normal range (|x| < 2^-74) lo is dropped (below 2^-98 absolute).
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    const unsigned int e = (unsigned int)(mag >> 52);
    if (e - 897u > 253u) {
        hi = (float)x;
        lo = 0.0f;
        return;
    }
    const unsigned int sgn = (unsigned int)(b >> 63) << 31;
    const unsigned long long t = mag - (896ull << 52);
    const unsigned int r = (unsigned int)(t >> 29);
    const unsigned int rem = (unsigned int)t & 0x1fffffffu;
    const unsigned int up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (r & 1u));
    hi = __uint_as_float(sgn | (r + up));
    // rounded up: lo = -(2^29 - rem) ulp with the sign of x flipped; else lo = rem ulp
    const unsigned int m = up ? 0x20000000u - rem : rem;
    const int ef = (int)e - 948;  // binary32 exponent field of 2^(E - 1075)
    if (m == 0u || ef < 1) {
        lo = 0.0f;
        return;
    }
    const float v = __int2float_rn((int)m) * __uint_as_float((unsigned int)ef << 23);
    lo = __uint_as_float(__float_as_uint(v) ^ (up ? sgn ^ 0x80000000u : sgn));
}

// Programmatic dependent launch: a kernel that a graph starts on a programmatic edge may begin while its
// predecessor drains; it waits here, before its first read of the predecessor's results, until that
// grid has completed and its memory operations are visible.  Without such an edge (stream launches,
// ordinary graph edges) the instruction returns at once.
__device__ __forceinline__ void wait_for_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// s + e = a + b exactly (Knuth's two-sum, six binary32 operations, no ordering assumption)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <typename T>
__device__ __forceinline__ double to_f64(T x) {
    if constexpr (std::is_same<T, float>::value) return widen_f32(x);
    else return (double)x;
}
// w x for a lattice weight w (a compile-time constant).  In binary32 the weight is split into its
// rounded value and the remainder, w = hi + lo, and the product formed as fma(x, hi, x lo): one
// rounding and no bias from the rounded weight.  1/9, 1/36, 4/9 (and 1/3, 1/18) are not binary32
// numbers, and their fixed relative errors would shift the moments of every site's collision
// output by the same relative amount; the shadow solve divides the long waves of such a coherent
// shift by a + nu |k|^2 (Eq. schur), which at large physical steps is ~1e-4.
template <typename T>
__device__ __forceinline__ T wmul(double w, T x) {
    if constexpr (std::is_same<T, float>::value) {
        const float hi = (float)w;
        const float lo = (float)(w - (double)hi);
        return fmaf(x, hi, x * lo);
    } else {
        return (T)w * x;
    }
}

template <typename T>
__device__ __forceinline__ T from_f64(double x) {
    if constexpr (std::is_same<T, float>::value) return narrow_f64(x);
    else return (T)x;
}

// bytes of one stored population value and of one working-field value (h, P r, dm)
inline size_t pop_elem(int precision) { return precision == MSC_FP64 ? 8 : (precision == MSC_FP32 ? 4 : 2); }
inline size_t field_elem(int precision) { return precision == MSC_FP64 ? 8 : 4; }

// Population loads and stores in the compute type T.  FP16 storage (S = __half) holds f / sigma
// with sigma a power of two (exact scaling), rounded to nearest; other storage holds f itself.
template <typename T, typename S>
__device__ __forceinline__ T ld_pop(const S* p, size_t i, T sig) {
    if constexpr (std::is_same<S, __half>::value) return sig * (T)__half2float(p[i]);
    else return (T)p[i];
}
template <typename T, typename S>
__device__ __forceinline__ void st_pop(S* p, size_t i, T v, T isig) {
    if constexpr (std::is_same<S, __half>::value) p[i] = __float2half_rn((float)(v * isig));
    else p[i] = (S)v;
}

}  // namespace msc
