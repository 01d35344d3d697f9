// Shared definitions of the MSC-LBM CUDA library: lattice constants, device state, launch
// helpers.  Internal header (not part of the C ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/msclbm.h"

namespace msc {

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
// and by the last block of the sweep; everything else reads them at kernel start.
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
struct Layout {
    size_t state, fbuf, mbuf, h, pr, dm, spec, tw, coef, partial, counter, iters, hist, replay, total;
    size_t fstride;  // bytes of one population array
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
