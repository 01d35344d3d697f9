/*
 * msclbm.h - C ABI of the B300 (sm_103a) MSC-LBM library (libmsclbm.so).
 *
 * MSC-LBM is the macroscopic-shadow-corrected lattice Boltzmann method of
 * arxiv 2609.39474: a BDF dual-time inner iteration on periodic D2Q9 / D3Q19
 * lattices whose fixed point is the fully discrete population equation
 * T(f) - f = 0 (Eq. fixed-point-problem).  Each inner iteration runs one fused
 * TRT collide-stream sweep at the operating point Lambda = 1/4,
 * omega+ = omega- = 1 (Eqs. collision-operating, sweep), tests the raw
 * population RMS residual (Eq. residual), and otherwise corrects the conserved
 * residual moments by a masked Fourier-space solve of the shadow system and an
 * equilibrium lift (Eqs. schur, lift, shadow-update; Algorithm 1).
 *
 * Conventions shared by every entry point
 *  - Lattices are periodic and cubic: n sites per direction, n a power of two,
 *    8 <= n <= 4096 (FP32 storage) or 2048 (FP64) for D2Q9 (dim 2), and 8 <= n <= 256 (FP32)
 *    or 128 (FP64) for D3Q19 (dim 3): the shared-memory transforms hold whole lines.
 *  - Layout is structure of arrays with x fastest: populations f[k][z][y][x]
 *    (k in the paper's ordering, Appendix A), fields m[c][z][y][x] with
 *    c = 0 the pressure-like variable p_hat and c = 1..d the velocity
 *    components.  2D arrays drop the z index.  "sites" = n^dim.
 *  - Storage precision (MSC_FP64 / MSC_FP32 / MSC_FP16) fixes the element type of
 *    population arrays (double / float / half) and working-field arrays (double /
 *    float / float).  Host-facing fields (p_hat, u, residual norms, BDF moment history)
 *    are always double.
 *  - Device pointers must come from cudaMalloc-class allocations of the
 *    current device; the library never frees caller memory and never
 *    allocates device memory itself (the context lives in a caller-provided
 *    workspace).  Stream arguments are cudaStream_t values passed as void*;
 *    NULL means the legacy default stream.  Work is enqueued on that stream
 *    only.
 *  - Unless stated otherwise calls are asynchronous with respect to the host;
 *    msc_get_stats, msc_read_*, msc_get_* and msc_save_state synchronise
 *    the stream.
 *  - Every function returns MSC_OK (0) or one of the status codes below and
 *    performs no work when it returns MSC_ERR_ARG.
 */
#ifndef MSCLBM_H
#define MSCLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define MSC_OK 0
#define MSC_ERR_ARG 1          /* invalid argument: size, pointer, precision, parameter */
#define MSC_ERR_NONCONVERGED 2 /* a physical step reached K_max without passing the residual test
                                  (Section 4.1: recorded nonconvergent); the state stays at the
                                  last accepted step */
#define MSC_ERR_NONFINITE 3    /* a non-finite raw residual (never accepted, Section 4.1); the
                                  march stops with the state at the last accepted step */
#define MSC_ERR_TIMEOUT 4      /* reserved: a bounded device wait gave up */
#define MSC_ERR_CUDA 5         /* a CUDA runtime call failed */
#define MSC_ERR_STATE 6        /* call out of order (e.g. march before init or set_params) */

/* Storage precisions. */
#define MSC_FP64 0
#define MSC_FP32 1
#define MSC_FP16 2 /* D2Q9 only: populations in IEEE binary16 as f / sigma, sigma = the power of two
                      just above max |f^0| (chosen by msc_init_fields; exact scaling), rounded to
                      nearest on every store; h, P r, dm and the spectrum FP32, BDF moment history,
                      residual norm and per-wavenumber solve FP64, arithmetic FP32.  Stage entry
                      points take FP16 population arrays (sigma = 1) and FP32 field arrays. */

typedef struct msc_ctx msc_ctx; /* opaque; lives inside the caller's workspace */

typedef struct {
    int dim;        /* 2: D2Q9, 3: D3Q19 (Appendix A orderings) */
    int n;          /* sites per direction (power of two, see limits above) */
    int precision;  /* MSC_FP64, MSC_FP32 or MSC_FP16 (D2Q9) population storage */
    int max_steps;  /* capacity of the per-step statistics and replay tables (>= 1) */
    int hist_cap;   /* capacity of the inner-residual history ring (>= 1) */
} msc_lattice_desc;

typedef struct {
    double nu;      /* viscosity of the shadow solve, Eq. shadow-mom; the sweep itself runs at the
                       operating point omega+ = omega- = 1, i.e. nu = 1/6 (Eq. trt) */
    double dt;      /* physical BDF step Delta t in lattice time units (> 0), Eq. bdf2 */
    double eps;     /* acceptance tolerance on the raw RMS residual (>= 0), Algorithm 1 */
    int kmax;       /* maximum inner iterations per physical step (>= 1) */
    int nmin;       /* minimum accepted inner count (>= 1): 2 in 2D, 1 in 3D in the paper */
    int corrector;  /* 1: MSC-LBM shadow correction (Algorithm 1); 0: plain Picard */
    int replay;     /* 1: accept step i at the inner count set by msc_set_replay_counts,
                       regardless of the residual (parity testing); 0: normal acceptance */
    int warm_order; /* accepted population states used by the warm start of each step:
                       3 = 3f^n - 3f^{n-1} + f^{n-2} (Section 3.1), 2 = 2f^n - f^{n-1}, 1 = f^n;
                       0 = default: 3 for FP64 storage; for FP32 storage 2 on D2Q9 and 1 on
                       D3Q19 (extrapolation grows FP32 rounding in weakly damped modes that lie
                       outside the shadow mask).  The warm start sets only the first iterate,
                       never the accepted fixed point. */
    int count_multiple; /* a step is accepted only at an inner count that is a multiple of this:
                       1 = Algorithm 1 as printed; 2 = sweeps in pairs.  On D2Q9 the staggered
                       modes k = (pi,0), (0,pi) have sweep eigenvalue -1 and lie outside the mask,
                       so an odd count leaves them with a negative per-step factor that a warm
                       start extrapolation amplifies; even counts keep the factor positive.
                       0 = default: 2 for FP32 storage on D2Q9, else 1. */
    double force[3]; /* uniform body force F (d components used; the paper has none): added to the
                       momentum source, s_u = h_u - a u + F, i.e. (0, F) joins h_q in both the
                       reconstruction (Eq. macro-reconstruct) and the source (Eq. source-moments).
                       Zero reproduces the paper's march. */
    double omega[2]; /* TRT relaxation rates (omega+, omega-) of the general collision (Eq. collision)
                       for off-design runs, 0 < omega < 2; 0, 0 (or 1, 1) = the operating point
                       Lambda = 1/4, nu = 1/6 (Eq. collision-operating).  The viscosity of the shadow
                       solve stays `nu`: set nu = (1/omega+ - 1/2)/3 for a consistent corrector.
                       D2Q9 only; the batch and the adjoint run at the operating point only. */
} msc_params;

typedef struct {
    int64_t steps_done;   /* accepted physical steps since msc_init_fields */
    int64_t inner_total;  /* inner sweeps run by the last march call */
    int32_t steps_in_call;/* physical steps accepted by the last march call */
    int32_t last_iters;   /* inner count of the last accepted step */
    int32_t last_q;       /* BDF order of the last accepted step (1 or 2) */
    int32_t status;       /* MSC_OK or the code that stopped the last march */
    double last_R;        /* last raw RMS residual computed */
} msc_stats;

/* ---- Context: state of one periodic lattice (Sections 2.3, 3.1) -------------------------- */

/* Bytes of device workspace a context with this description needs (0 if the description is
   invalid).  The workspace holds the population ring (f^n, f^{n-1}, f^{n-2} and two working
   buffers), the FP64 moment histories m^n, m^{n-1}, the history term h, residual moments,
   the shadow correction, the half spectrum, twiddles, reduction partials and statistics. */
size_t msc_workspace_bytes(const msc_lattice_desc* desc);

/* Create a context in dev_workspace (device memory of >= msc_workspace_bytes bytes, 256-byte
   aligned; owned by the caller and used exclusively by this context until msc_destroy).  The
   context's host part is allocated with malloc; its CUDA graphs are built lazily on first use.
   The stream is where every later call of this context enqueues work. */
int msc_create(msc_ctx** out, const msc_lattice_desc* desc, void* dev_workspace, size_t bytes,
               void* stream);

/* Destroy the host part and graphs of a context (the workspace is not touched). */
void msc_destroy(msc_ctx* ctx);

/* Set the march parameters (validated here; returns MSC_ERR_ARG on nonsense). */
int msc_set_params(msc_ctx* ctx, const msc_params* params);

/* f^0 = f_eq(p_hat, u) (Eq. feq), m^0 = P f^0 (Eq. moments); no pre-march relaxation
   (Section 4.1).  p_hat has sites doubles, u has dim*sites doubles, both in the field layout
   above, on the host (on_device = 0) or the device (on_device = 1).  Resets the histories so
   that the next physical step is BDF1. */
int msc_init_fields(msc_ctx* ctx, const double* p_hat, const double* u, int on_device);

/* Run n_steps physical steps of Algorithm 1 (corrector = 1) or plain Picard dual-time
   stepping (corrector = 0) entirely on the device: per step the BDF coefficients and the
   population warm start (Section 3.1), then inner iterations sweep -> residual test ->
   shadow correction until acceptance, then reconstruction of m^{n+1} and history rotation.
   BDF1 is used on the first step after msc_init_fields, BDF2 after.  Asynchronous; read the
   outcome with msc_get_stats.  A nonconvergent or non-finite step stops the march with the
   state at the last accepted step. */
int msc_march(msc_ctx* ctx, int n_steps);

/* The same march as msc_march, driven from the host: the same kernels launched one at a time
   with the acceptance decision read back after every sweep (one stream synchronisation per inner
   iteration).  Results are identical to msc_march; it exists for profilers that do not descend
   into conditional graph nodes and for debugging, and is much slower at small lattices. */
int msc_march_stepwise(msc_ctx* ctx, int n_steps);

/* Run n_steps explicit LBM steps f <- S f_eq(P f) (same collision and streaming with no BDF
   source; Section 4.1) from the current accepted populations.  Afterwards m^n = P f and the
   dual-time history restarts (the next physical step is BDF1). */
int msc_explicit_march(msc_ctx* ctx, int n_steps);

/* Statistics of the last march call (synchronises the stream). */
int msc_get_stats(msc_ctx* ctx, msc_stats* out);

/* Copy the accepted macroscopic field m^n = (p_hat, u) (double, layout above) to host or
   device memory (synchronises). */
int msc_read_fields(msc_ctx* ctx, double* p_hat, double* u, int on_device);

/* Stream-ordered copy of m^n = (p_hat, u), (d+1) x sites doubles, into device memory m, without
   synchronising: a kernel on the context's stream reads which buffer holds m^n, so the copy may
   follow a march that has not finished (e.g. one step of a recorded replay).  Errors: MSC_ERR_ARG
   for a NULL context or pointer, MSC_ERR_CUDA for a failed launch. */
int msc_copy_fields_async(msc_ctx* ctx, double* m);

/* Copy the accepted populations f^n (converted to double, Q*sites values) out (synchronises). */
int msc_read_populations(msc_ctx* ctx, double* f, int on_device);

/* Copy up to cap raw residuals R_l of the last march call (oldest first) to the host; *n gets
   the number copied.  The ring keeps the last hist_cap values. */
int msc_get_residual_history(msc_ctx* ctx, double* R, int cap, int* n);

/* Copy the accepted inner count of each step of the last march call (host ints; *n copied). */
int msc_get_step_iters(msc_ctx* ctx, int* iters, int cap, int* n);

/* Set the inner counts that replay mode forces on the next march call's steps (host ints,
   1 <= counts[i] <= kmax, n <= max_steps). */
int msc_set_replay_counts(msc_ctx* ctx, const int* counts, int n);

/* Serialise the accepted state (f^n, f^{n-1}, f^{n-2}, m^n, m^{n-1}, step counters) into a
   host blob.  With blob == NULL only *bytes is set to the size needed. */
int msc_save_state(msc_ctx* ctx, void* host_blob, size_t* bytes);
int msc_load_state(msc_ctx* ctx, const void* host_blob, size_t bytes);

/* Human-readable text for a status code (static storage). */
const char* msc_strerror(int status);

/* Index checks of the bounds-checked debug build (libmsclbm_check.so, compiled with
   -DMSC_BOUNDS_CHECK; not part of the method).  That build tests the indices of the sweep strips,
   tiles and halos and of the shared-memory transforms before each guarded access, skips an access
   whose index is out of range (the results are then wrong, but no memory outside the arrays is
   touched and nothing traps) and counts it.  *count receives the number of failed checks since the
   last reset, *first the first failure as site << 40 | index (site numbers are those of the
   MSC_INB calls in the sources).  Synchronises the device; reset != 0 clears both afterwards.
   Returns MSC_OK in the checked build and MSC_ERR_STATE (with both outputs 0) in the normal build,
   which has no checks; MSC_ERR_ARG for NULL outputs. */
int msc_bounds_check_report(unsigned long long* count, unsigned long long* first, int reset);

/* ---- Stage entry points: one step of the hot path on caller-owned device arrays ----------- */

/* Scratch bytes the stage calls below need for this lattice (reduction partials and the half
   spectrum).  The scratch is device memory owned by the caller, 256-byte aligned. */
size_t msc_stage_scratch_bytes(int dim, int n, int precision);

/* One fused sweep (Eqs. macro-reconstruct .. sweep, residual):
     trial  f = f_in + E dm            (Eq. lift; skipped when dm == NULL)
     m = (P f + h/2)/(1 + a/2),  s = h - a m,  C = f_eq(m) + Phi(m, s)/2,
     f_out = S C (periodic push streaming),  r = f_out - f,
     pr_out = P r  ((dim+1)*sites values),  *sumsq_out = sum_x sum_k r_k(x)^2 (one double).
   f_in / f_out: Q*sites elements of the storage type, distinct arrays; dm, h, pr_out:
   (dim+1)*sites elements of the storage type; sumsq_out: device double.  With a = 0 and h all
   zero this is one explicit LBM step plus its change.  Scratch as above. */
int msc_sweep(int dim, int n, int precision, double a, const void* f_in, const void* dm,
              const void* h, void* f_out, void* pr_out, double* sumsq_out, void* scratch,
              size_t scratch_bytes, void* stream);

/* The D3Q19 sweep of the march in its halo-free form, as one stage (msc_sweep with dim = 3 is this
   call preceded by the moments P f_in).  At the operating point the post-collision populations of a
   site depend only on its reconstructed moments and source (Eq. collision-operating), and the
   moments of the trial f_in + E dm are P f_in + dm, so the collision inputs of every neighbour come
   from pf_in, dm and h alone and the outputs are pulled, f_out,k(x) = C_k(x - c_k).  Same results as
   msc_sweep (dim 3) up to rounding, plus pf_out = P f_out for the next sweep.  f_in / f_out:
   19*n^3 elements of the storage type (FP64 or FP32); pf_in / pf_out: 4*n^3 elements, P f_in and
   P f_out (density, then the three momentum components); dm (NULL: no lift), pr_out: 4*n^3.  h as
   the march holds it (Eq. bdf2): 4*n^3 doubles with FP64 storage; with FP32 storage a binary32 pair
   of 2*4*n^3 floats, the four high parts followed by the four low parts, every difference h - a m
   formed as fma(-a, m, hi) + lo (as msc_sweep_hpair does in 2D), so that this call runs the FP32
   march's sweep kernel itself.  f_in != f_out and pf_in != pf_out.  Scratch as msc_sweep
   (msc_stage_scratch_bytes(3, n, ...)).
   MSC_ERR_ARG for invalid sizes, pointers, scratch or FP16 storage. */
int msc_sweep_d3q19_pf(int n, int precision, double a, const void* f_in, const void* pf_in, const void* dm,
                       const void* h, void* f_out, void* pf_out, void* pr_out, double* sumsq_out, void* scratch,
                       size_t scratch_bytes, void* stream);

/* msc_sweep for D2Q9 with the history term h (Eq. bdf2) given as the march holds it.  With binary32
   storage (FP32, FP16) h is a pair of 2*3*n*n floats, the three high parts followed by the three low
   parts, h = hi + lo; the sweep forms every difference h - a m (in m = (P f + h/2)/(1 + a/2) written
   as P f + (h - a P f)/(2 (1 + a/2)), and in s = h - a m) as fma(-a, m, hi) + lo, so that the source
   keeps its own relative accuracy where h ~ a m.  This is the sweep kernel of the FP32 and FP16
   march.  With FP64 storage h has 3*n*n doubles and the call equals msc_sweep with dim = 2.  Other
   arguments, scratch and errors as msc_sweep. */
int msc_sweep_hpair(int n, int precision, double a, const void* f_in, const void* dm, const void* h,
                    void* f_out, void* pr_out, double* sumsq_out, void* scratch, size_t scratch_bytes,
                    void* stream);

/* Shadow correction of the residual moments (Eq. shadow-update, first two lines):
     dm = F^{-1}[ chi(k) H(k)^{-1} F[pr] ]
   with the paper's transform convention (Eq. fft-convention), wavenumbers k_j = 2 pi j / n
   (Eq. wavenumbers), the rectangular mask |j_alpha| <= n/4 (Eq. shadow-mask) and the closed-form
   Schur elimination of H(k) (Eq. schur) evaluated in FP64.  pr, dm: (dim+1)*sites elements of
   the storage type (may not alias). */
int msc_shadow_solve(int dim, int n, int precision, double a, double nu, const void* pr, void* dm,
                     void* scratch, size_t scratch_bytes, void* stream);

/* f_out = f_eq(p_hat, u) (Eq. feq) from double device fields; f_out in the storage type. */
int msc_equilibrium(int dim, int n, int precision, const double* p_hat, const double* u,
                    void* f_out, void* stream);

/* msc_sweep for D2Q9 with the general TRT collision (Eq. collision) at relaxation rates
   omega_p = 1/tau+, omega_m = 1/tau- (each in (0, 2)); with omega_p = omega_m = 1 it equals the
   operating-point sweep up to rounding.  Arguments otherwise as msc_sweep (dim = 2). */
int msc_sweep_trt(int n, int precision, double a, double omega_p, double omega_m, const void* f_in, const void* dm,
                  const void* h, void* f_out, void* pr_out, double* sumsq_out, void* scratch, size_t scratch_bytes,
                  void* stream);

/* Full-symbol reference correction for D2Q9 (Section 4.1, Eq. full-symbol; the reference operator
   of the off-design study, Section 4.6): the linearised Newton step about rest,
       f_out = f + F^{-1}[ (I - Z(k) J)^{-1} F[f_swept - f] ]
   at every wavevector and on all 9 population fields, where J is the Q x Q Jacobian of the general
   TRT collision (Eq. collision, rates omega_p, omega_m in (0, 2), BDF reaction a > 0) at the rest
   state and Z(k) = diag(exp(-i k . c_q)) the streaming symbol.  J is used in closed form (the
   exact derivative; the paper forms it by a forward difference of step 1e-7, which agrees to that
   difference error) and every wavevector is solved in FP64 through the pair structure of the TRT
   relaxation (four 2 x 2 blocks and one 3 x 3 system).  f, f_swept, f_out: 9 x n x n elements of
   the storage type (FP64 or FP32), f_swept the sweep of f (e.g. msc_sweep_trt); f_out may alias f
   or f_swept.  Scratch: msc_full_symbol_scratch_bytes(n, precision) bytes of device memory,
   256-byte aligned (twiddles and the 9-field half spectrum).  n a power of two in
   [8, MSC_FULL_SYMBOL_MAX_N].  Stream-ordered, no synchronisation.  MSC_ERR_ARG for invalid
   sizes, rates, pointers or scratch. */
#define MSC_FULL_SYMBOL_MAX_N 1024
size_t msc_full_symbol_scratch_bytes(int n, int precision);
int msc_full_symbol_correct(int n, int precision, double a, double omega_p, double omega_m, const void* f,
                            const void* f_swept, void* f_out, void* scratch, size_t scratch_bytes, void* stream);

/* Allocation-free variant of msc_sweep for D2Q9 (dim 2).  The paper has no counterpart: this is
   an interface convenience for callers that cannot allocate device memory, such as host
   frameworks that own the whole device-memory budget and forbid plugins from calling cudaMalloc,
   bindings that can only pass input and output arrays, or latency-critical loops in which an
   allocation would synchronise the device.  Same computation and arguments as msc_sweep with
   dim = 2, minus the scratch: the reduction scratch (a counter and one partial sum per block) is
   a fixed static device array of 33 KB that every device which loads the library holds until the
   process exits.  Limits: n a power of two with 8 <= n <= 2048 for FP64 storage and
   8 <= n <= 4096 for FP32 storage; FP16 storage is not supported; anything else returns
   MSC_ERR_ARG before any launch.  Every call looks the array's device address up for the current
   device (so it stays right after a device reset); the first call on a device also loads the
   library's device code there, so make that first call outside any stream capture.  Every call
   shares the same array and clears its counter itself, so calls that may overlap on the GPU
   (different streams, or host threads racing on one device) race with each other: serialise
   them. */
int msc_sweep_d2q9_noalloc(int n, int precision, double a, const void* f_in, const void* dm,
                           const void* h, void* f_out, void* pr_out, double* sumsq_out, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Discrete adjoint (D2Q9).  The accepted state of each physical step is the fixed point
 * f^{n+1} = T(f^{n+1}; h^n) (Eqs. fixed-point-problem, sweep) with h^n = h_q(m^n, m^{n-1}) +
 * (0, F) (Eq. bdf2 plus the body force of msc_params) and m^{n+1} = R(f^{n+1}; h^n)
 * (Eq. macro-reconstruct); the warm start only picks the first iterate.  A loss of the final fields
 * is differentiated step by step, last step first, by implicit differentiation of each fixed
 * point: (I - dT/df)^T lambda = P^T mu / (1 + a/2) with mu = dL/dm^{n+1}, then
 * dL/dh^n = (dT/dh)^T lambda + mu / (2 (1 + a/2)), passed to m^n, m^{n-1} through h^n and to F.
 * At the operating point lambda = P^T theta with a three-field unknown theta, iterated with the
 * transposed shadow correction (the per-wavevector factor (H(k)^H)^{-1} inside the mask).
 * Since m^0 = P f_eq(p_hat_0, u_0) = (p_hat_0, u_0), dL/dm^0 is the gradient with respect to the
 * initial fields.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    int iters;       /* transposed iterations run */
    int status;      /* MSC_OK, MSC_ERR_NONCONVERGED or MSC_ERR_NONFINITE */
    double residual; /* final RMS of the reduced adjoint residual relative to RMS(mu / (1 + a/2)) */
} msc_adjoint_stats;

/* Adjoint of physical step n -> n+1 (q = 1 for the first step of a march, else 2), with the
   context's dt, nu and force.  All arrays are device double, (d+1) x sites each, layout of
   msc_read_fields (p_hat first): m_new = m^{n+1}, m_cur = m^n, m_prev = m^{n-1} (unused, may be
   NULL, when q = 1) are the forward moments; abar_new = dL/dm^{n+1} (complete: every later step
   already processed); abar_cur += c1 dL/dh^n and abar_prev -= c2 dL/dh^n (abar_prev unused when
   q = 1); dforce[0..d-1] += the velocity parts of dL/dh^n summed over sites.  Stops when the
   relative residual falls below eps (> 0) or after kmax iterations (MSC_ERR_NONCONVERGED: the
   accumulators are then left untouched).  Uses the context's working arrays as scratch: the forward
   state is undefined afterwards, so load a state (msc_load_state / msc_load_state_device) before
   the next march.  The iteration runs on the device (a CUDA graph with conditional nodes); the call
   synchronises the stream once.  `out` may be NULL. */
int msc_adjoint_step(msc_ctx* ctx, int q, const double* m_new, const double* m_cur, const double* m_prev,
                     const double* abar_new, double* abar_cur, double* abar_prev, double* dforce, double eps,
                     int kmax, msc_adjoint_stats* out);

/* The arrays of one step of msc_adjoint_steps (meaning as in msc_adjoint_step), and its start. */
typedef struct {
    int q;
    const double* m_new;
    const double* m_cur;
    const double* m_prev;   /* may be NULL when q = 1 */
    const double* abar_new;
    double* abar_cur;
    double* abar_prev;      /* may be NULL when q = 1 */
    int warm;               /* 0: the transposed solve starts from theta = c (as msc_adjoint_step does);
                               1: from c + (theta - c) of the last step that converged on this
                               context (zero before the first), which a reverse pass sets for every
                               step after its first.  The result is the same fixed point within eps. */
} msc_adjoint_io;

/* `count` adjoint steps in array order (a reverse pass lists the last physical step first, so that
   each step's abar_new is complete when it runs), with one synchronisation per MSC_ADJOINT_CHUNK
   steps instead of one per step.  Each step is exactly msc_adjoint_step.  After the first step
   that fails (MSC_ERR_NONCONVERGED or MSC_ERR_NONFINITE) the later steps run no kernels, leave their
   arrays untouched and report status MSC_ERR_STATE with iters 0.  `out` (count entries) may be
   NULL.  Returns MSC_OK or the status of the first failing step; MSC_ERR_ARG for a NULL or invalid
   entry (nothing is run). */
#define MSC_ADJOINT_CHUNK 64
int msc_adjoint_steps(msc_ctx* ctx, int count, const msc_adjoint_io* steps, double* dforce, double eps, int kmax,
                      msc_adjoint_stats* out);

/* msc_adjoint_steps with every kernel launched from the host and the iteration decided on the host
   (same kernels in the same order, identical results; one synchronisation per iteration).  For
   profiling: profilers do not descend into the conditional graph nodes of msc_adjoint_steps. */
int msc_adjoint_steps_stepwise(msc_ctx* ctx, int count, const msc_adjoint_io* steps, double* dforce, double eps,
                               int kmax, msc_adjoint_stats* out);

/* Self-check of the library's binary32 <-> binary64 conversions (integer-pipe implementations of the
   IEEE 754 widening and round-to-nearest-even narrowing used by the FP32-storage step kernels)
   against the hardware conversions on blocks x 256 x per_thread random patterns; *mismatches
   receives the count (0 expected).  Allocates 4 bytes of device memory for the count and
   synchronises the device. */
int msc_selftest_conversions(int blocks, int per_thread, unsigned long long seed, int* mismatches);

/* msc_save_state / msc_load_state with the blob in device memory (same layout; checkpoints of a
   reverse pass stay on the device).  Synchronise the stream. */
int msc_save_state_device(msc_ctx* ctx, void* dev_blob, size_t* bytes);
int msc_load_state_device(msc_ctx* ctx, const void* dev_blob, size_t bytes);

/* ---------------------------------------------------------------------------------------------
 * Batched march (a parameter sweep, Section 4.6 "Operating envelope": the same method over a range
 * of Reynolds numbers and lattice sizes).  A batch groups up to MSC_BATCH_MAX existing D2Q9
 * contexts of one storage precision, created on one stream, with any mix of n (and each with its
 * own msc_set_params: nu, dt, eps, K_max, n_min, replay) and advances all of them in one CUDA
 * graph: every loop round performs one inner iteration (sweep, acceptance test, shadow correction
 * or step end) of every instance still running, so each instance converges in its own number of
 * inner iterations without waiting for the others.  Each instance computes exactly what
 * msc_march computes for its context; only the grid geometry of the kernels differs (the per-site
 * and per-line arithmetic is the same, the residual-norm summation order follows the tuned tiling).
 * Contexts stay owned by the caller and keep their own calls: msc_set_params, msc_init_fields,
 * msc_set_replay_counts before a batch march; msc_get_stats, msc_read_fields, msc_get_step_iters,
 * msc_get_residual_history after it.  A context must not be destroyed while a batch holds it.
 * ------------------------------------------------------------------------------------------- */
#define MSC_BATCH_MAX 64
#define MSC_BATCH_CLASSES 8 /* distinct lattice sizes in one batch */

typedef struct msc_batch msc_batch;

/* Kernel tiling of a batch, per distinct lattice size (class c, sizes in descending order).
   sweep_rows: output rows per warp unit of the sweep (4..64, a power of two, <= n);
   fft_rows: complex row transforms per block of the row passes (a power of two, <= n/2,
   fft_rows * n / 16 <= 256); col_lines: j_x columns per block of the column solve (a power of
   two, 3 col_lines n / 16 <= 768 threads for FP32, 384 for FP64); sweep_ctas_per_sm: resident
   blocks of 4 warps per SM of the persistent sweep (1..16).  The *_us fields are the last
   msc_batch_autotune timings of the chosen tiling (one launch over the whole batch, microseconds;
   0 when not measured). */
typedef struct {
    int n_classes;
    int n[MSC_BATCH_CLASSES];
    int sweep_rows[MSC_BATCH_CLASSES];
    int fft_rows[MSC_BATCH_CLASSES];
    int col_lines[MSC_BATCH_CLASSES];
    int sweep_ctas_per_sm;
    float sweep_us, rowfft_us, colsolve_us;
} msc_batch_tuning;

/* Device workspace bytes of a batch over n_inst contexts (0 if the list is invalid: NULL, more than
   MSC_BATCH_MAX, not D2Q9, mixed precision, more than MSC_BATCH_CLASSES distinct n). */
size_t msc_batch_workspace_bytes(msc_ctx* const* ctxs, int n_inst);

/* Create a batch over ctxs[0..n_inst) in a caller-provided device workspace (256-byte aligned,
   >= msc_batch_workspace_bytes).  Every context must have been created with `stream`.  The initial
   tiling is the single-context geometry of each size; msc_batch_autotune improves it. */
int msc_batch_create(msc_batch** out, msc_ctx* const* ctxs, int n_inst, void* dev_workspace, size_t bytes,
                     void* stream);
void msc_batch_destroy(msc_batch* b);

/* Advance instance i by n_steps[i] >= 0 physical steps (host array of n_inst counts, in the order
   of ctxs).  Asynchronous.  Each instance stops on its own at its count or at its first
   nonconvergent or non-finite step (its status, readable by msc_get_stats, says which; the other
   instances carry on).  MSC_ERR_STATE if a context with a nonzero count lacks parameters or
   fields; MSC_ERR_ARG for a negative count or a replay count list shorter than the steps. */
int msc_batch_march(msc_batch* b, const int* n_steps);

/* Explicit LBM steps for every instance (n_steps[i] >= 0 each), batched the same way; the same
   result as msc_explicit_march on each context. */
int msc_batch_explicit_march(msc_batch* b, const int* n_steps);

/* Project-written autotuner: times the batched sweep, row transforms and column solve on the
   instances' own arrays (stateless: no instance state changes; the next step's working arrays are
   scratch until a march rewrites them) for every candidate tiling, one class and one kernel at a
   time (coordinate descent, best of `reps` launches each, reps >= 1), keeps the fastest and
   rebuilds the batch graph.  Synchronises the stream.  `out` (optional) receives the result. */
int msc_batch_autotune(msc_batch* b, int reps, msc_batch_tuning* out);
int msc_batch_get_tuning(msc_batch* b, msc_batch_tuning* out);
/* Install a tiling (validated as described above; MSC_ERR_ARG otherwise, batch unchanged). */
int msc_batch_set_tuning(msc_batch* b, const msc_batch_tuning* t);
/* Time one batched kernel family with the current tiling, as the autotuner does (stateless: reads
   each instance's accepted populations, writes only working arrays that a march rewrites before
   reading): which = 0 the persistent sweep over every instance, 1 the forward + inverse row
   transforms, 2 the column solve.  Best of `reps` launches after one warm-up launch, in
   microseconds, into *us.  Synchronises the stream. */
int msc_batch_time_stage(msc_batch* b, int which, int reps, float* us);

#ifdef __cplusplus
}
#endif
#endif /* MSCLBM_H */
