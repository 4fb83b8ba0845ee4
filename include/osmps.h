/*
 * osmps.h -- C ABI of the GB300 two-site variational ground-state search.
 *
 * The operations follow "Open source Matrix Product States" (arXiv 1703.00387):
 * the effective Hamiltonian of Sec. 3.4 (Fig. LanczosMPS), its lowest
 * eigenpair by Lanczos, the eigendecomposition split of Sec. 2
 * (Eq. AAD_ULLUD, Eq. ThetaAL) with the truncation rule of Eq. elocal, and the
 * sweeps of Sec. 3.4; and real-time evolution by the two-site TDVP of
 * Sec. 5.4 with the Krylov propagator of Sec. 5.2.
 *
 * Conventions (tensors real float64 unless a call says complex, which means
 * interleaved (re, im) float64 pairs; row-major, contiguous):
 *   MPS site tensor      A[a, s, b]        (chi_l, d, chi_r)            Eq. mps
 *   MPO site tensor      W[w, t, s, w2]    (w_left, d, d, w_right)      Eq. mpo / Eq. MPOdef
 *                        t = outgoing (bra) physical index, s = incoming (ket);
 *                        W[w,:,:,w2] is the operator in row w, column w2 of M^[k].
 *                        Lower-triangular channel order: the left environment's
 *                        last channel and the right environment's first channel
 *                        are the identity channels.
 *   Environments         L[a2, w, a], R[b2, w, b]: first index bra, last ket.
 *   Two-site tensor      theta[a, s1, s2, c]  (chi_l, d1, d2, chi_r)
 *
 * Memory: every pointer argument named as a tensor is a DEVICE pointer owned
 * by the caller, unless the comment says "host". The caller keeps it alive
 * until the stream has been synchronised. Scalars returned through "host"
 * pointers are written after the call synchronises its stream.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream). Calls are asynchronous on it unless they return host values.
 *
 * Errors: every call returns an osmps_status, never aborts and never prints.
 * osmps_last_error() returns a message for the calling thread's last failure.
 * No call falls back to the CPU: a missing GPU or a CUDA error is reported.
 */
#ifndef OSMPS_H
#define OSMPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OSMPS_OK = 0,
  OSMPS_EINVAL = 1,   /* null pointer, aliasing output, bad enum value     */
  OSMPS_ESHAPE = 2,   /* inconsistent or non-positive dimensions            */
  OSMPS_ENOMEM = 3,   /* device allocation failed                           */
  OSMPS_ECUDA = 4,    /* a CUDA / cuSOLVER call failed                      */
  OSMPS_ENOCONV = 5,  /* Lanczos hit max_iter above tol (best pair written) */
  OSMPS_ETIMEOUT = 6, /* a bounded device wait gave up                      */
  OSMPS_ENAN = 7,     /* non-finite value detected                          */
  OSMPS_EUNSUPPORTED = 8
} osmps_status;

/* Arithmetic of the contractions (H_eff.theta and the environment updates).
 * Lanczos orthogonalisation, the tridiagonal eigensolve, the Gram matrix and
 * its eigendecomposition, and energies are always float64.               */
typedef enum {
  OSMPS_PREC_FP64 = 0,   /* plain float64 on CUDA cores / DMMA                       */
  OSMPS_PREC_BF16X3 = 1, /* tcgen05 bf16 tensor cores, hi+lo split, 3 products, f32 acc */
  OSMPS_PREC_TF32X3 = 2, /* tcgen05 tf32 tensor cores, hi+lo split, 3 products, f32 acc */
  OSMPS_PREC_FP64_EMU = 3 /* float64-accurate products emulated on the bf16 tensor cores:
                             8 exact 7-bit slices per operand, 36 slice pairs, exact
                             float32 partial sums added in float64                     */
} osmps_precision;

typedef struct osmps_ctx osmps_ctx;

const char* osmps_last_error(void);
const char* osmps_status_string(osmps_status s);

/* Create a context on `device` (makes it current for the calling thread).
 * ws_bytes: initial device workspace; the context grows it on demand.
 * Owns the workspace, a cuSOLVER handle and a device error flag.            */
osmps_status osmps_ctx_create(int device, size_t ws_bytes, osmps_ctx** out);
osmps_status osmps_ctx_destroy(osmps_ctx* ctx);
/* Eigensolver used by the split (osmps_split and the sweeps):
 *   OSMPS_EIG_AUTO     (default) the faster of the two as measured on
 *                      GB300: this library's route for Gram dimension
 *                      n >= 64, cuSOLVER below;
 *   OSMPS_EIG_CUSOLVER cuSOLVER dsyevd / dsyevdx (largest pairs) always;
 *   OSMPS_EIG_TRIDIAG  this library's Householder reduction (osmps_sytrd;
 *                      cuSOLVER dsytrd above n = 8192), multisection on
 *                      Sturm counts, inverse iteration, Cholesky QR (cuSOLVER
 *                      dpotrf for the factor, this library's triangular
 *                      inverse) and blocked back-transformation
 *                      (float64-accurate emulated GEMMs) for every Gram
 *                      dimension >= 2.
 * Both are float64-accurate. EINVAL for another value.                      */
typedef enum { OSMPS_EIG_AUTO = 0, OSMPS_EIG_CUSOLVER = 1, OSMPS_EIG_TRIDIAG = 2 } osmps_eig_solver;
osmps_status osmps_ctx_set_eig_solver(osmps_ctx* ctx, int solver);
/* How Lanczos (osmps_lanczos_ground, its projected and U(1) forms, and the
 * sweeps) drives its steps:
 *   OSMPS_LANCZOS_HOST  the host launches every step and reads the Ritz
 *                       value, residual estimate and beta after each one;
 *   OSMPS_LANCZOS_GRAPH the first step runs as above without the read; the
 *                       remaining steps are one CUDA graph whose conditional
 *                       while-node repeats the recorded step until the device
 *                       takes the same stopping decision (at most max_iter
 *                       steps in all); the host synchronises once at the end.
 *                       The graph is kept in the context and replayed by later
 *                       calls with the same operator shape and parameters (up
 *                       to 16 graphs, least recently used dropped first);
 *   OSMPS_LANCZOS_AUTO  (default) the graph for Krylov vectors of at most
 *                       2^20 entries, the host loop above that (where the
 *                       products take milliseconds) and on the worker threads
 *                       of osmps_sweep_batch (where many streams run at once
 *                       and the host loop measured faster).
 * Both run the same kernels on the same data and give bit-identical results.
 * The graph is not used while kernel profiling is on, nor for max_iter = 1.
 * A context serves one host thread at a time. EINVAL for another value.     */
typedef enum { OSMPS_LANCZOS_AUTO = 0, OSMPS_LANCZOS_HOST = 1, OSMPS_LANCZOS_GRAPH = 2 } osmps_lanczos_mode;
osmps_status osmps_ctx_set_lanczos_mode(osmps_ctx* ctx, int mode);
/* Identity environment channels in the split-precision H_eff.theta (Sec. 3.2:
 * the identity corners of a lower-triangular MPO make one channel of a
 * left-canonical L, and one of a right-canonical R, the unit matrix). When
 * L's last (else first) channel and R's first (else last) channel equal the
 * unit matrix to within 1e-3 per entry (built by split-precision updates
 * from canonical tensors, it carries a few 1e-6 of rounding per site of the
 * chain; other channels are O(1) away), both GEMM stages leave them out
 * (theta itself feeds the W-steps; the W-steps' output for R's channel is
 * added in the last GEMM's epilogue): (wl - 1)/wl and (wr - 1)/wr of the
 * tensor-core work. The test reads two channels of L and R once per
 * prepared operator and synchronises the stream.
 *   OSMPS_IDENTITY_OFF    never;
 *   OSMPS_IDENTITY_SOLVER operators applied many times: Lanczos, TDVP and
 *                         excited-state solves, sweeps (default);
 *   OSMPS_IDENTITY_ALWAYS also every osmps_heff_apply.
 * Only for the MPO shapes with the fused W-step (d = 2; w in {1, 3, 5}).
 * EINVAL for another value.                                                */
typedef enum { OSMPS_IDENTITY_OFF = 0, OSMPS_IDENTITY_SOLVER = 1, OSMPS_IDENTITY_ALWAYS = 2 } osmps_identity_mode;
osmps_status osmps_ctx_set_identity_skip(osmps_ctx* ctx, int mode);
/* Tile-width autotuning of the tcgen05 GEMMs (H_eff stages, environment
 * updates, the U(1) grouped products). Each output tile is 128 rows by 256,
 * 128 or 64 columns; the arithmetic per element does not depend on the
 * width, so results are bit-identical. With OSMPS_AUTOTUNE_ON (default) the
 * first product of a size class (output tiles counted at 128 x 64, K in
 * steps of 512; grouped: problem count, tile count, K) that runs outside
 * stream capture and kernel profiling is run at all three widths, each
 * timed with CUDA events after one untimed run, and the fastest is kept in
 * the context for the class; later products of the class use it. With
 * OSMPS_AUTOTUNE_OFF every product uses 256 (unless a choice was set).
 * EINVAL for another mode.                                                  */
typedef enum { OSMPS_AUTOTUNE_OFF = 0, OSMPS_AUTOTUNE_ON = 1 } osmps_autotune_mode;
osmps_status osmps_ctx_set_autotune(osmps_ctx* ctx, int mode);
/* The context's tuning table: number of entries, and entry i (0-based):
 * key[6] (class fields), the chosen width, and the measured microseconds
 * at widths 256, 128, 64 (0 for a choice set by osmps_ctx_set_tuning).
 * HOST outputs; EINVAL for i out of range.                                 */
int64_t osmps_ctx_tuning_count(const osmps_ctx* ctx);
osmps_status osmps_ctx_tuning_entry(const osmps_ctx* ctx, int64_t i, int64_t* key, int* width,
                                    float* us3);
/* Set (or replace) the width for a class key, e.g. from a table saved by an
 * earlier run. EINVAL for a width other than 64, 128, 256.                 */
osmps_status osmps_ctx_set_tuning(osmps_ctx* ctx, const int64_t* key, int width);
/* Bytes of device memory currently held by the context's workspace.         */
size_t osmps_ctx_workspace_bytes(const osmps_ctx* ctx);

/* Kernel timing with CUDA events recorded on the launching stream around
 * every launch of the listed kernels made through this context (profiling
 * support; not part of the paper's method).                                 */
typedef enum {
  OSMPS_KERNEL_GEMM_TC = 0,  /* tcgen05 split-precision GEMM                   */
  OSMPS_KERNEL_GEMM_F64 = 1, /* float64 DMMA GEMM                             */
  OSMPS_KERNEL_GEMM_EMU = 2, /* float64-accurate GEMM on bf16 tensor cores      */
  OSMPS_KERNEL_SYTRD_PANEL = 3, /* Householder panel of the tridiagonalisation  */
  OSMPS_KERNEL_U1_WSTEP = 4     /* fused W-step of the U(1) H_eff (its "flops"
                                 * field carries algorithmic bytes instead)     */
} osmps_kernel;
/* Turn recording on (1) or off (0); both clear earlier records. Syncs the device. */
osmps_status osmps_profile_enable(osmps_ctx* ctx, int enable);
/* Totals over the records of one kernel since the last enable: launches,
 * summed event time (ms), credited FLOPs (2 M N K per GEMM) and tensor FLOPs
 * (3x credited for the three-product split, = credited for float64).
 * Host outputs; synchronises the device.                                   */
osmps_status osmps_profile_read(osmps_ctx* ctx, int kernel, int64_t* launches, double* total_ms,
                                double* flops, double* tensor_flops);
/* Number of kernels this library has launched since it was loaded (its own
 * kernels only; cuSOLVER's are not counted).                               */
int64_t osmps_kernel_launches(void);

/* H_eff . theta (Sec. 3.4, Fig. LanczosMPS: L, M^[k], M^[k+1] and R contracted
 * step by step with theta instead of forming the (chi^2 d^2)^2 matrix):
 *   y[a2,t1,t2,c2] = sum L[a2,w,a] W1[w,t1,s1,w1] W2[w1,t2,s2,w2] R[c2,w2,c] theta[a,s1,s2,c]
 * L: (chi_l, wl, chi_l); W1: (wl, d1, d1, wm); W2: (wm, d2, d2, wr);
 * R: (chi_r, wr, chi_r); theta, y: (chi_l, d1, d2, chi_r).
 * y must not alias theta (EINVAL). Scratch comes from the context workspace. */
osmps_status osmps_heff_apply(osmps_ctx* ctx, const double* L, const double* W1, const double* W2,
                              const double* R, const double* theta, double* y, int64_t chi_l,
                              int64_t d1, int64_t d2, int64_t chi_r, int64_t wl, int64_t wm,
                              int64_t wr, int precision, void* stream);

/* H_eff . theta for callers that cannot allocate device memory. (The paper
 * has no counterpart: this is a deployment variant of osmps_heff_apply.)
 * Some callers cannot call cudaMalloc: a serving process that reserved its
 * whole memory budget up front, a real-time loop that must not take the
 * implicit device synchronisation an allocation may cause, or a plug-in
 * that is not allowed to own allocations. This call needs no osmps_ctx and
 * allocates nothing. It computes the same float64 product as
 * osmps_heff_apply(..., OSMPS_PREC_FP64, ...) with the same arguments and
 * layouts, on the device current on the calling thread (all pointers must
 * be on that device); `stream` as everywhere else.
 * Its scratch is one fixed 32 MiB array compiled into the library: every
 * GPU that loads the library holds it until the process exits. Dimensions
 * whose intermediates would not fit are rejected with OSMPS_ESHAPE (the
 * message gives the bytes needed); use osmps_heff_apply for those.
 * The first call on each device looks up the array's device address with
 * that device current; make that first call before any stream capture.
 * The address is kept per device ordinal for the life of the process: after
 * cudaDeviceReset (or any release and re-creation of the device's primary
 * context) it is stale, so do not call this entry point again in a process
 * that has reset the device.
 * Every call shares the one array and it keeps the previous call's
 * contents (nothing in it is read before the call writes it), so calls
 * that can overlap on the GPU (other streams or threads) race: serialise
 * them.                                                                      */
osmps_status osmps_heff_apply_noalloc(const double* L, const double* W1, const double* W2,
                                      const double* R, const double* theta, double* y,
                                      int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r,
                                      int64_t wl, int64_t wm, int64_t wr, void* stream);

/* Float64-accurate matrix product on the tensor cores, C = A B with A
 * (M, K), B (K, N), C (M, N) row-major float64 device arrays. A support
 * routine of the float64 split (Sec. 2, Eq. AAD_ULLUD: the Gram matrix and
 * the projection are such products): every row of A and column of B is
 * scaled by a power of two and cut into 8 exact 7-bit bf16 slices; the 36
 * slice pairs whose weight is above 2^-56 are multiplied on tcgen05 with
 * exact float32 partial sums of 256 products, accumulated in float64.
 * C must not alias A or B. Scratch from the context.                       */
osmps_status osmps_dgemm_emu(osmps_ctx* ctx, const double* A, const double* B, double* C,
                             int64_t M, int64_t N, int64_t K, void* stream);

/* Householder reduction of a symmetric matrix to tridiagonal form, the first
 * step of the float64 eigendecomposition of the split (Sec. 2, Eq.
 * AAD_ULLUD): Q^T A Q = T with d (n) its diagonal, e (n-1) its off-diagonal,
 * Q = H(0) ... H(n-2), H(j) = I - tau[j] v v^T, v = (0..0, 1 at j+1,
 * A[j+2.., j]) stored below the subdiagonal of column j (column-major view;
 * the layout of LAPACK's dsytrd with uplo = L). A: n x n device array
 * holding the full symmetric matrix (both triangles), overwritten. Panels of
 * 32 columns on a cooperative kernel with two grid barriers per column, the
 * trailing updates on the float64-accurate emulated tensor-core GEMM.
 * 2 <= n <= 8192, else ESHAPE; ETIMEOUT if a bounded barrier wait gave up. */
osmps_status osmps_sytrd(osmps_ctx* ctx, double* A, int64_t n, double* d, double* e, double* tau,
                         void* stream);

/* Block operations for block-sparse (U(1)) tensors. With a conserved
 * particle number every tensor of the sweep (Sec. 3.4 with symmetries) is a
 * set of dense blocks, one per combination of charge sectors; theta
 * formation (Sec. 2 "Contractions"), the per-sector Gram matrices and
 * projections of the split (Eq. AAD_ULLUD) and the environment updates are
 * then lists of products and copies of strided views of those blocks.
 * All pointers are device pointers; element (r, c) of a view is at
 * base[r * row_stride + c * col_stride], strides of either sign.          */
typedef struct {
  const double* A; int64_t sam, sak;   /* A (M x K) of this term            */
  const double* B; int64_t sbk, sbn;   /* B (K x N) of this term            */
  int64_t K;                           /* >= 1                              */
  double alpha;
} osmps_gemm_term;
typedef struct {
  double* C; int64_t scm, scn;         /* C (M x N)                         */
  int64_t M, N;
  double beta;
  int64_t term_begin, term_count;      /* its terms in the term array       */
} osmps_gemm_out;
/* Grouped products: for every output, C = sum over its terms of
 * alpha A B + beta C (no terms: C = beta C), all outputs in one launch of
 * the float64 DMMA kernel, one CTA per 64 x 64 output tile running through
 * the terms' K ranges in order (deterministic; no atomics). Outputs must
 * not overlap one another nor any term operand of the launch; beta = 0
 * never reads C. outs, terms: HOST arrays, read before the call returns.
 * EINVAL for a null pointer or a term range outside the term array,
 * ESHAPE for negative sizes, K < 1 or more than 2^31 tiles. Synchronises
 * `stream` (the descriptor upload).                                       */
osmps_status osmps_gemm_grouped(osmps_ctx* ctx, const osmps_gemm_out* outs, int64_t n_out,
                                const osmps_gemm_term* terms, int64_t n_terms, void* stream);
typedef struct {
  const double* src;                   /* NULL: the destination is zeroed   */
  double* dst;
  int64_t rows, cols;
  int64_t srs, scs;                    /* source element strides            */
  int64_t drs;                         /* destination row stride            */
  double alpha;                        /* dst[r drs + c] = alpha src[...]   */
} osmps_copy_desc;
/* All copies in one launch (their destinations must not overlap); descs:
 * HOST array, read before the call returns. Synchronises `stream`.        */
osmps_status osmps_copy_list(osmps_ctx* ctx, const osmps_copy_desc* descs, int64_t n,
                             void* stream);
/* The largest nev eigenpairs of the symmetric n x n device matrix G
 * (row-major, both triangles; overwritten) in float64: eigenvalues
 * ascending to the HOST array ev_host (nev), eigenvectors as the rows of the
 * device array Y (nev x n). This library's tridiagonal route from n = 64 on
 * (OSMPS_EIG_AUTO), cuSOLVER dsyevd below. Synchronises `stream`.         */
osmps_status osmps_sym_eig_top(osmps_ctx* ctx, double* G, int64_t n, int64_t nev,
                               double* ev_host, double* Y, void* stream);
/* ||x||^2 of a device vector of n >= 1 doubles, to the host.               */
osmps_status osmps_vec_norm2(osmps_ctx* ctx, const double* x, int64_t n, double* out_host,
                             void* stream);

/* Self-test of the failure path of the bounded device waits (the paper has
 * no counterpart: a robustness check of this library). Every wait in this
 * library's kernels gives up after a time limit, records the failure, frees
 * what the kernel holds and returns; the call then reports ETIMEOUT and the
 * context stays usable. This call makes one such wait run out on purpose,
 * with a limit of limit_us microseconds (1 .. 1e6, else EINVAL):
 *   which = 0: a kernel that holds tensor memory waits on an mbarrier that
 *              no thread arrives at, then frees the tensor memory;
 *   which = 1: a cooperative grid waits at a grid barrier one of its blocks
 *              never reaches.
 * Returns OSMPS_ETIMEOUT when the wait gave up (the expected outcome), OK
 * otherwise. Synchronises `stream`.                                          */
osmps_status osmps_selftest_wait_timeout(osmps_ctx* ctx, int which, double limit_us, void* stream);
/* Test support: y32[i] = (float)x64[i] (round to nearest, ties to even) and
 * y64[i] = (double)x32[i] computed with the integer-field conversions the
 * kernels use where the float64 pipe would be the bottleneck (device arrays
 * of n elements). Results must equal the IEEE conversions bit for bit.    */
osmps_status osmps_selftest_convert(osmps_ctx* ctx, const double* x64, float* y32,
                                    const float* x32, double* y64, int64_t n, void* stream);
/* Test support: the bf16 rounding of n doubles (device arrays) by the
 * integer-field route the U(1) operand split uses (y_int) and by CUDA's
 * __double2bfloat16 (y_hw), as raw 16-bit patterns. EINVAL for a null
 * pointer with n > 0 or n < 0.                                              */
osmps_status osmps_selftest_bf16(osmps_ctx* ctx, const double* x, uint16_t* y_int, uint16_t* y_hw,
                                 int64_t n, void* stream);

/* Environment update (Sec. 3.4: the fixed sites are contracted into L and R
 * one site at a time).
 * side 0 (grow L past site k):
 *   env_out[b2,w2,b] = sum A[a2,t,b2] env_in[a2,w,a] W[w,t,s,w2] A[a,s,b]
 *   env_in: (chi_l, w_in, chi_l), W: (w_in, d, d, w_out), env_out: (chi_r, w_out, chi_r)
 * side 1 (grow R past site k):
 *   env_out[a2,w,a] = sum A[a2,t,b2] W[w,t,s,w2] env_in[b2,w2,b] A[a,s,b]
 *   env_in: (chi_r, w_in, chi_r), W: (w_out, d, d, w_in), env_out: (chi_l, w_out, chi_l)
 * A: (chi_l, d, chi_r).                                                      */
osmps_status osmps_env_update(osmps_ctx* ctx, int side, const double* env_in, const double* A,
                              const double* W, double* env_out, int64_t chi_l, int64_t d,
                              int64_t chi_r, int64_t w_in, int64_t w_out, int precision,
                              void* stream);

/* Lowest eigenpair of H_eff (Sec. 3.4) by Lanczos with full float64
 * reorthogonalisation, starting from theta_inout (normalised internally).
 * Stops when the residual estimate beta_j |s_j| <= tol, after max_iter
 * matrix-vector products (1 <= max_iter <= 512), or when the Krylov space is
 * exhausted. On return theta_inout holds the normalised Ritz vector.
 * energy_out, iters_out, resid_out: host pointers (resid_out may be NULL).
 * Returns ENOCONV when max_iter was reached above tol (the best pair is still
 * written). Synchronises `stream`.                                          */
osmps_status osmps_lanczos_ground(osmps_ctx* ctx, const double* L, const double* W1,
                                  const double* W2, const double* R, double* theta_inout,
                                  int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r,
                                  int64_t wl, int64_t wm, int64_t wr, int max_iter, double tol,
                                  int precision, double* energy_out, int* iters_out,
                                  double* resid_out, void* stream);

/* Krylov propagator theta <- exp(-i tau H_eff) theta (Sec. 5.2, Eq. propSE
 * and Eq. krylov:approx), the local step of the two-site TDVP (Sec. 5.4).
 * L (chi_l, wl, chi_l), R (chi_r, wr, chi_r) and theta_inout
 * (chi_l, d1, d2, chi_r) are COMPLEX: interleaved (re, im) float64 pairs,
 * the layout of C99 double complex / complex128; W1, W2 are real, as in
 * osmps_heff_apply. H_eff is the same contraction as in osmps_heff_apply;
 * the environments' first index is the conjugated (bra) one, so a Hermitian
 * MPO gives a Hermitian H_eff. A one-site H_eff is the case d2 = 1 with
 * W2[w,0,0,w2] = delta(w, w2).
 * The Krylov basis starts from theta / ||theta|| with full float64
 * reorthogonalisation; with m vectors the result is
 * ||theta|| V exp(-i tau T_m) e_1. It stops when the weight leaving the
 * space, beta_m |[exp(-i tau T_m) e_1]_m|, is <= tol, when the space is
 * exhausted, or at max_iter vectors (1 <= max_iter <= 128). The norm is kept
 * (the propagator is unitary). iters_out, err_out (may be NULL): host
 * pointers to the vector count and the last estimate. Returns ENOCONV at
 * max_iter above tol (the result is still written), ENAN on non-finite
 * Krylov data (theta_inout unchanged). Uses the same workspace as
 * osmps_lanczos_ground (the Krylov basis holds 4 chi_l d1 d2 chi_r doubles
 * per vector), plus three slots for the real embedding of L, R and theta
 * (32 chi_l^2 wl, 32 chi_r^2 wr and 32 chi_l d1 d2 chi_r bytes).
 * Synchronises `stream`.                                                    */
osmps_status osmps_heff_expm(osmps_ctx* ctx, const double* L, const double* W1, const double* W2,
                             const double* R, double* theta_inout, int64_t chi_l, int64_t d1,
                             int64_t d2, int64_t chi_r, int64_t wl, int64_t wm, int64_t wr,
                             double tau, int max_iter, double tol, int precision, int* iters_out,
                             double* err_out, void* stream);

/* Two-site tensor (Sec. 2, "Contractions"): theta[a,s1,s2,c] = sum_b A1[a,s1,b] A2[b,s2,c].
 * A1: (chi_l, d1, chi_m), A2: (chi_m, d2, chi_r), theta: (chi_l, d1, d2, chi_r). */
osmps_status osmps_theta_form(osmps_ctx* ctx, const double* A1, const double* A2, double* theta,
                              int64_t chi_l, int64_t d1, int64_t chi_m, int64_t d2, int64_t chi_r,
                              void* stream);

/* Split theta with truncation by the eigendecomposition route (Sec. 2,
 * Eq. AAD_ULLUD and Eq. ThetaAL), Gram matrix and eigensolver in float64.
 * The eigenpairs are float64 (cuSOLVER dsyevdx for the largest
 * min(chi_max, rank) only). The Gram matrix and the projection run on the
 * float64 DMMA GEMM for precision OSMPS_PREC_FP64 and on the float64-accurate
 * emulated tensor-core GEMM for every other precision. The discarded weight
 * is 1 - (kept sum of lambda^2) / ||theta||^2 (the Gram route cannot resolve
 * the tail below ~n eps ||theta||^2).
 * move_right = 1: G = M M^T with M = theta as (chi_l d1) x (d2 chi_r);
 *   A1 = kept eigenvectors (left-canonical), A2 = U^T M renormalised.
 * move_right = 0: G = M^T M; A2 = V^T (right-canonical), A1 = M V renormalised.
 * Kept number chi' = min(chi_max, smallest n >= 1 with sum_{i>=n} lambda_i^2
 * <= eps_local), lambda^2 normalised to sum 1 (Eq. elocal; Sec. 3.4).
 * A1 must hold chi_l*d1*min(chi_max, chi_l*d1, d2*chi_r) doubles and A2
 * min(...)*d2*chi_r; they are written with the actual chi'.
 * Host outputs: chi_new_out, discarded_out (weight of the dropped lambda^2),
 * entropy_out (-sum lambda'^2 log lambda'^2 over kept, renormalised values),
 * lam2_out (optional host array of min(chi_l d1, d2 chi_r) values,
 * descending; only the first min(chi_max, rank) are computed, the rest are
 * written as 0). Synchronises `stream`.                                     */
osmps_status osmps_split(osmps_ctx* ctx, const double* theta, double* A1, double* A2,
                         int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r, int move_right,
                         int64_t chi_max, double eps_local, int64_t* chi_new_out,
                         double* discarded_out, double* entropy_out, double* lam2_out,
                         int precision, void* stream);

/* ---------------------------------------------------------------------------
 * Whole-chain handles and sweeps (Sec. 3.4).
 * ------------------------------------------------------------------------- */
typedef struct osmps_mps osmps_mps;
typedef struct osmps_mpo osmps_mpo;

/* MPS with L sites, physical dims d[L] and a bond-dimension cap chi_cap used to
 * size the device storage. host_tensors[k] points to a HOST array of
 * chi[k]*d[k]*chi[k+1] doubles (chi has L+1 entries, chi[0] = chi[L] = 1).
 * The tensors are copied to the device. No canonical form is assumed.      */
osmps_status osmps_mps_create(osmps_ctx* ctx, int64_t L, const int64_t* d, const int64_t* chi,
                              const double* const* host_tensors, int64_t chi_cap,
                              osmps_mps** out);
osmps_status osmps_mps_destroy(osmps_mps* mps);
/* Current bond dimensions (host array of L+1 entries).                     */
osmps_status osmps_mps_bond_dims(const osmps_mps* mps, int64_t* chi_out);
/* Copy site k to a HOST buffer of at least chi[k]*d[k]*chi[k+1] doubles.    */
osmps_status osmps_mps_get_tensor(const osmps_mps* mps, int64_t k, double* host_out);
/* Device pointer of site k (valid until the next sweep or destroy).        */
const double* osmps_mps_device_tensor(const osmps_mps* mps, int64_t k);

/* MPO with L sites; host_W[k] is a HOST array of w[k]*d[k]*d[k]*w[k+1]
 * doubles (w has L+1 entries, w[0] = w[L] = 1).                             */
osmps_status osmps_mpo_create(osmps_ctx* ctx, int64_t L, const int64_t* d, const int64_t* w,
                              const double* const* host_W, osmps_mpo** out);
osmps_status osmps_mpo_destroy(osmps_mpo* mpo);
/* Overwrite every site tensor of an existing MPO with new values of the same
 * shapes (HOST arrays as for osmps_mpo_create). Synchronises the device.  */
osmps_status osmps_mpo_set(osmps_mpo* mpo, const double* const* host_W);

typedef struct {
  int64_t chi_max;        /* maximal bond dimension                                  */
  double eps_local;       /* truncation tolerance (<0: 1e-12 / (4 L), Sec. 3.4)    */
  double lanczos_tol;     /* residual tolerance of each Lanczos solve              */
  int lanczos_max_iter;   /* Lanczos cap per step (paper default 100)              */
  int n_sweeps;           /* number of full L->R->L sweeps                          */
  int precision;          /* osmps_precision of the contractions                   */
  int refine_sweeps;      /* extra float64-accurate sweeps after n_sweeps (OSMPS_PREC_FP64_EMU
                             after tensor-core sweeps, OSMPS_PREC_FP64 otherwise)      */
} osmps_sweep_params;

typedef struct {
  double energy;             /* final <psi|H|psi>, evaluated in float64                */
  double last_step_energy;   /* Lanczos eigenvalue of the last step                    */
  double max_discarded;      /* largest discarded weight of any split                  */
  double entropy_center;     /* bond entropy at the centre bond (last visit)           */
  int64_t max_chi;           /* largest bond dimension reached                         */
  int64_t steps;             /* two-site steps performed                               */
  int64_t lanczos_iters;     /* total matrix-vector products                           */
  int64_t nonconverged;      /* steps whose Lanczos stopped at max_iter above tol      */
  double seconds;            /* wall time of the call                                  */
  double setup_seconds;      /* canonicalisation and environment build                 */
  double sweep_seconds;      /* the sweeps themselves                                  */
  double energy_seconds;     /* the final float64 energy                               */
  double* step_energies;     /* optional HOST array (caller-owned) of length
                                2 (L-1) (n_sweeps + refine_sweeps), or NULL          */
  int64_t* step_iters;       /* optional HOST array, same length, or NULL              */
} osmps_sweep_stats;

/* Bring `mps` to mixed-canonical form with the orthogonality centre at
 * site `center` (0 <= center < L-1) by QR shifts (Sec. 2 "Shifting", Eq. oc),
 * normalise it, and build the left environments of sites < center and the
 * right environments of sites > center+1 for `mpo` (contractions in
 * `precision`). Afterwards osmps_sweep_step may run at pair (center,
 * center+1). Synchronises `stream`.                                         */
osmps_status osmps_mps_canonicalize(osmps_ctx* ctx, osmps_mps* mps, const osmps_mpo* mpo,
                                    int64_t center, int precision, void* stream);

typedef struct {
  double energy;     /* Lanczos eigenvalue of H_eff (precision of the contractions) */
  double resid;      /* Lanczos residual estimate                                   */
  double discarded;  /* discarded weight of the split                               */
  double entropy;    /* bond entropy of the kept, renormalised spectrum             */
  int64_t chi_new;   /* new bond dimension between the two sites                   */
  int iters;         /* matrix-vector products used                                 */
  int converged;     /* 1 if the Lanczos residual met the tolerance                 */
} osmps_step_stats;

/* One two-site step at the pair (k, k+1) (Sec. 3.4): theta = A_k A_{k+1},
 * Lanczos on H_eff (params->lanczos_tol / lanczos_max_iter / precision), the
 * eigendecomposition split with truncation (params->chi_max, eps_local), and
 * the environment update on the side the centre leaves: move_right = 1 grows
 * L to site k+1 (centre moves to k+1), 0 grows R to site k (centre stays at k).
 * Requires the centre at k or k+1 with environments in place (after
 * osmps_mps_canonicalize or a previous step). out: host pointer or NULL.
 * Synchronises `stream` (the new bond dimension is decided on the host).   */
osmps_status osmps_sweep_step(osmps_ctx* ctx, osmps_mps* mps, const osmps_mpo* mpo, int64_t k,
                              int move_right, const osmps_sweep_params* params,
                              osmps_step_stats* out, void* stream);

/* Run two-site sweeps on `mps` in place: right-canonicalise it (QR shifts,
 * Sec. 2), build the right environments, then for every sweep optimise the
 * pairs (0,1)...(L-2,L-1) left to right and back (2 (L-1) steps per sweep):
 * theta formation, Lanczos, split with truncation, environment update.
 * Finally the energy is evaluated to float64 accuracy by contracting
 * <psi|H|psi> and <psi|psi> (float64-accurate emulated tensor-core GEMMs).
 * stats is a host pointer (may be NULL). Synchronises `stream`.            */
osmps_status osmps_sweep(osmps_ctx* ctx, osmps_mps* mps, const osmps_mpo* mpo,
                         const osmps_sweep_params* params, osmps_sweep_stats* stats,
                         void* stream);

/* <psi|H|psi> / <psi|psi> to float64 accuracy for the MPS as it stands (host
 * result; contractions on the float64-accurate emulated GEMM).            */
osmps_status osmps_energy(osmps_ctx* ctx, const osmps_mps* mps, const osmps_mpo* mpo,
                          double* energy_out, void* stream);

/* Energy and variance of the MPS as it stands (Sec. 3.4 convergence
 * parameters: V = <H^2> - <H>^2 of the normalised state). V is formed as
 * <psi|(H - E)^2|psi> / <psi|psi> to avoid cancelling against E^2: the MPO
 * of H - E (each site's local term, the block [start = w_l - 1, :, :, done =
 * 0] of the nearest-neighbour MPO form, shifted by -E/L) is squared site by
 * site and contracted with float64-accurate environment updates.
 * Squared blocks w^2 d above 64 give EUNSUPPORTED. Host outputs
 * (energy_out may be NULL). Synchronises `stream`.                          */
osmps_status osmps_variance(osmps_ctx* ctx, const osmps_mps* mps, const osmps_mpo* mpo,
                            double* energy_out, double* variance_out, void* stream);

/* Sweeps of many independent chains at once (the paper's data parallelism
 * over independent simulations, appendix "Convenient features", MPI item:
 * jobs are handed to workers one by one, largest systems first).
 * n_workers host threads each own ctxs[w] (distinct contexts on one device)
 * and a stream they create; they take chains in decreasing order of
 * estimated cost (sum over bonds of chi^3 times the sweep count) and run
 * osmps_sweep(ctxs[w], mps[i], mpo[i], &params[i], &stats[i], stream) on
 * each. Chains must not share an MPS handle (EINVAL); an MPO may be shared.
 * stats (n_chains entries, may be NULL) and chain_status (n_chains entries,
 * may be NULL) are HOST arrays; chain_status[i] is the chain's own status,
 * or -1 for a chain that was not started because another one failed.
 * Returns the first failure (message names the chain). Blocks until all
 * workers are done.                                                        */
osmps_status osmps_sweep_batch(osmps_ctx* const* ctxs, int n_workers, osmps_mps* const* mps,
                               const osmps_mpo* const* mpo, const osmps_sweep_params* params,
                               int64_t n_chains, osmps_sweep_stats* stats,
                               osmps_status* chain_status);

/* ------------------------------------------------------------------------
 * Excited states (Sec. 4.1 eMPS, Eq. emps_lagrange: Lagrange multipliers
 * keep the state orthogonal to the lower eigenstates; locally, the Lanczos
 * search runs in the orthogonal complement of the lower states' two-site
 * blocks seen in the current basis).
 * ---------------------------------------------------------------------- */

/* osmps_lanczos_ground on H_eff restricted to the orthogonal complement of
 * the k rows of P (k x n row-major device array, n = chi_l d1 d2 chi_r; any
 * linearly independent rows, 0 <= k <= 64; copied and orthonormalised
 * internally). theta_inout is projected into the complement first (EINVAL if
 * it lies in the span of P). Other arguments and results as
 * osmps_lanczos_ground.                                                    */
osmps_status osmps_lanczos_ground_projected(osmps_ctx* ctx, const double* L, const double* W1,
                                            const double* W2, const double* R,
                                            double* theta_inout, const double* P, int k,
                                            int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r,
                                            int64_t wl, int64_t wm, int64_t wr, int max_iter,
                                            double tol, int precision, double* energy_out,
                                            int* iters_out, double* resid_out, void* stream);

/* Overlap environment of the state being optimised (bra, site tensor A
 * (chi_l, d, chi_r)) with a lower state (ket, site tensor Bk (chik_l, d,
 * chik_r)), grown past one site (float64):
 *   side 0: env_out[b2, bk] = sum A[a2, t, b2] env_in[a2, ak] Bk[ak, t, bk]
 *           env_in (chi_l, chik_l), env_out (chi_r, chik_r)
 *   side 1: env_out[a2, ak] = sum A[a2, t, b2] env_in[b2, bk] Bk[ak, t, bk]
 *           env_in (chi_r, chik_r), env_out (chi_l, chik_l)                  */
osmps_status osmps_overlap_env_update(osmps_ctx* ctx, int side, const double* env_in,
                                      const double* A, const double* Bk, double* env_out,
                                      int64_t chi_l, int64_t d, int64_t chi_r, int64_t chik_l,
                                      int64_t chik_r, void* stream);

/* The lower state's two-site block in the current basis:
 *   v[a, s1, s2, c] = sum OL[a, ak] B1[ak, s1, m] B2[m, s2, ck] OR[c, ck]
 * OL (chi_l, chik_l), B1 (chik_l, d1, chik_m), B2 (chik_m, d2, chik_r),
 * OR (chi_r, chik_r), v (chi_l, d1, d2, chi_r) (float64).                  */
osmps_status osmps_projected_state(osmps_ctx* ctx, const double* OL, const double* B1,
                                   const double* B2, const double* OR, double* v, int64_t chi_l,
                                   int64_t d1, int64_t d2, int64_t chi_r, int64_t chik_l,
                                   int64_t chik_m, int64_t chik_r, void* stream);

/* ------------------------------------------------------------------------
 * U(1)-symmetric H_eff . theta (Sec. 3.4 with a conserved particle number:
 * block-sparse tensors; every sector block of a GEMM stage in one grouped
 * tcgen05 launch).
 * Every bond index carries a charge; a local state s carries charge s; MPO
 * channel w carries q_w. Allowed entries:
 *   theta[a,s1,s2,c], y[...]: q(a) + s1 + s2 = q(c)
 *   L[a2,w,a]: q(a2) = q(a) + q_wl[w];   R[c2,w,c]: q(c2) = q(c) + q_wr[w]
 * Packed format of theta, y, L, R: their allowed entries in C order of the
 * dense tensor (numpy: dense[mask]). A bond is given as its sectors in
 * index order: charge and size of each (charges distinct, sizes >= 1).
 * W1 (wl, d1, d1, wm) and W2 (wm, d2, d2, wr) are dense; the result is the
 * dense product restricted to the allowed entries of y.                   */
typedef struct {
  int64_t n_left;            /* sectors of the left bond (index of a, a2)          */
  const int64_t* q_left;     /* their charges (HOST array, n_left)                  */
  const int64_t* chi_left;   /* their sizes   (HOST array, n_left)                  */
  int64_t n_right;           /* sectors of the right bond (index of c, c2)         */
  const int64_t* q_right;
  const int64_t* chi_right;
  int64_t d1, d2;            /* local dimensions (state s has charge s)            */
  int64_t wl, wm, wr;        /* MPO bond dimensions                                 */
  const int64_t* q_wl;       /* charge of each left MPO channel (HOST, wl)         */
  const int64_t* q_wr;       /* charge of each right MPO channel (HOST, wr)        */
} osmps_u1_desc;
typedef struct osmps_u1_heff osmps_u1_heff;

/* Build the block plan for one (left bond, right bond, MPO) structure: sector
 * bookkeeping on the host, index tables and operand buffers on the device
 * (owned by the handle). EINVAL for repeated charges, ESHAPE for bad sizes. */
osmps_status osmps_u1_heff_create(osmps_ctx* ctx, const osmps_u1_desc* desc, osmps_u1_heff** out);
osmps_status osmps_u1_heff_destroy(osmps_u1_heff* plan);
/* Packed lengths of theta (= y), L and R, and the GEMM FLOPs of one product
 * (sum over the sector blocks of 2 M N K, both GEMM stages). Host outputs,
 * any may be NULL.                                                          */
osmps_status osmps_u1_heff_sizes(const osmps_u1_heff* plan, int64_t* n_theta, int64_t* n_L,
                                 int64_t* n_R, double* flops);
/* Element counts of the plan's intermediates: n_t1 float32 entries of the
 * stage-1 output T1, n_a4 entries of the stage-4 A operand that the fused
 * W-step writes (each as two split pieces), n_y float64 entries of the
 * stage-4 output. Host outputs, any may be NULL.                            */
osmps_status osmps_u1_heff_stage_sizes(const osmps_u1_heff* plan, int64_t* n_t1, int64_t* n_a4,
                                       int64_t* n_y);
/* Convert the operator (packed L and R, dense W1 and W2) into the plan's
 * tensor-core operands for `precision` (OSMPS_PREC_BF16X3 or TF32X3; others
 * EUNSUPPORTED). The operator stays prepared until the next prepare.       */
osmps_status osmps_u1_heff_prepare(osmps_ctx* ctx, osmps_u1_heff* plan, const double* L,
                                   const double* W1, const double* W2, const double* R,
                                   int precision, void* stream);
/* y = H_eff theta for the prepared operator (packed device arrays; y must not
 * alias theta). EINVAL if nothing was prepared.                           */
osmps_status osmps_u1_heff_apply(osmps_ctx* ctx, osmps_u1_heff* plan, const double* theta,
                                 double* y, void* stream);
/* Lowest eigenpair of the U(1) block of H_eff by Lanczos (as
 * osmps_lanczos_ground: float64 Krylov vectors, full reorthogonalisation,
 * residual estimate <= tol, 1 <= max_iter <= 512), on packed vectors; the
 * operator is prepared first. theta_inout: start vector in, normalised Ritz
 * vector out. Host outputs; ENOCONV with the best pair written.            */
osmps_status osmps_lanczos_ground_u1(osmps_ctx* ctx, osmps_u1_heff* plan, const double* L,
                                     const double* W1, const double* W2, const double* R,
                                     double* theta_inout, int max_iter, double tol, int precision,
                                     double* energy_out, int* iters_out, double* resid_out,
                                     void* stream);
/* y = H_eff theta on packed device arrays (layouts above): prepare + apply.
 * Calls with one plan must not overlap on the GPU (its buffers are reused). */
osmps_status osmps_heff_apply_u1(osmps_ctx* ctx, osmps_u1_heff* plan, const double* L,
                                 const double* W1, const double* W2, const double* R,
                                 const double* theta, double* y, int precision, void* stream);

/* ------------------------------------------------------------------------
 * Gradients (differentiation of the Sec. 3.4 operators; the paper has no
 * backward pass). Every quantity below is linear in the tensor it is
 * differentiated by, so each gradient is a full contraction of the incoming
 * cotangent with all other factors.
 * ---------------------------------------------------------------------- */

/* Vector-Jacobian product of y = H_eff(L, W1, W2, R) theta (osmps_heff_apply)
 * for an output cotangent gy (chi_l, d1, d2, chi_r):
 *   gtheta = H_eff^T gy   (the same four-stage contraction with bra and ket
 *            swapped in L, W1, W2 and R; computed in `precision`),
 *   gW1[w,t1,s1,w1] = sum gy[a2,t1,t2,c2] L[a2,w,a] theta[a,s1,s2,c] W2[w1,t2,s2,w2] R[c2,w2,c],
 *   gW2[w1,t2,s2,w2] = sum gy[a2,t1,t2,c2] L[a2,w,a] theta[a,s1,s2,c] W1[w,t1,s1,w1] R[c2,w2,c].
 * gtheta, gW1, gW2 are device outputs with the shapes of theta, W1 and W2;
 * any of them may be NULL (not computed). theta may be NULL when gW1 and gW2
 * are. gW1 and gW2 are float64-accurate in every precision (DMMA for
 * OSMPS_PREC_FP64, the emulated GEMM otherwise). gtheta must not alias gy or
 * theta (EINVAL). wl*d1, d1*wm, wm*d2, d2*wr above 64 give EUNSUPPORTED when
 * a weight gradient is requested.                                          */
osmps_status osmps_heff_backward(osmps_ctx* ctx, const double* L, const double* W1,
                                 const double* W2, const double* R, const double* theta,
                                 const double* gy, double* gtheta, double* gW1, double* gW2,
                                 int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r, int64_t wl,
                                 int64_t wm, int64_t wr, int precision, void* stream);

/* E = <psi|H|psi> / <psi|psi> of the MPS as it stands (Eq. mpo) and its
 * gradient with respect to every MPO site tensor:
 *   dE/dW_k[w,t,s,w2] = sum L_k[a2,w,a] A_k[a2,t,b2] A_k[a,s,b] R_{k+1}[b2,w2,b] / <psi|psi>
 * with L_k, R_{k+1} the environments of the MPS (no canonical form assumed).
 * gW: device output, the gradients of sites 0..L-1 concatenated, each
 * (w[k], d[k], d[k], w[k+1]) row-major; gW_count must equal the total.
 * checkpoint_every: 0 or 1 keeps all L right environments; s > 1 keeps only
 * every s-th one and rebuilds the others block by block (about L/s + s
 * environments alive, one extra right pass of work).
 * precision: OSMPS_PREC_FP64 (DMMA) or OSMPS_PREC_FP64_EMU (emulated GEMM);
 * others give EINVAL. energy_out, norm_out: host pointers, may be NULL.
 * MPO blocks w*d above 64 give EUNSUPPORTED. Synchronises `stream`.        */
osmps_status osmps_energy_grad(osmps_ctx* ctx, const osmps_mps* mps, const osmps_mpo* mpo,
                               double* gW, int64_t gW_count, int64_t checkpoint_every,
                               int precision, double* energy_out, double* norm_out, void* stream);

/* Chain rule from an MPO-tensor gradient to Hamiltonian couplings for an MPO
 * that is affine in them, W = W_0 + sum_p c_p B_p:
 *   g_par[p] = sum_{j = row_ptr[p]}^{row_ptr[p+1]-1} val[j] * gW[col[j]]
 * (B in compressed sparse rows: row p lists the nonzero entries of B_p by
 * their index into the concatenated MPO, as in osmps_energy_grad).
 * row_ptr (n_par + 1 entries), col and val (nnz entries), gW (n_w entries)
 * and g_par (n_par entries) are device arrays. A column outside [0, n_w) or
 * a bad row pointer contributes nothing and gives EINVAL. Sums run in a
 * fixed order. Synchronises `stream`.                                      */
osmps_status osmps_coupling_grad(osmps_ctx* ctx, int64_t n_par, const int64_t* row_ptr,
                                 const int64_t* col, const double* val, int64_t nnz,
                                 const double* gW, int64_t n_w, double* g_par, void* stream);

/* ---- Real-time evolution: two-site TDVP (Sec. 5.4) ------------------------
 * Complex tensors are interleaved (re, im) float64 pairs (C99 double complex
 * / complex128 layout). */

/* Split of a complex two-site tensor with truncation, the eigendecomposition
 * route of osmps_split (Sec. 2, Eq. AAD_ULLUD) for M = theta as the complex
 * (chi_l d1) x (d2 chi_r) matrix:
 *   move_right = 1: G = M M^dagger; A1 = kept eigenvectors (left-canonical),
 *                   A2 = U^dagger M renormalised to unit norm;
 *   move_right = 0: G = M^dagger M; A2 = V^dagger (right-canonical),
 *                   A1 = M V renormalised.
 * The Hermitian eigenproblem is solved by cuSOLVER zheevd in float64; the
 * Gram matrix and the projection run on float64 GEMMs (DMMA for
 * OSMPS_PREC_FP64, the emulated float64 GEMM otherwise). The kept number and
 * the discarded weight follow osmps_split's rule. theta (device, complex,
 * chi_l x d1 x d2 x chi_r); A1, A2 (device, complex) with room for
 * chi_l d1 min(chi_max, rank) and min(chi_max, rank) d2 chi_r elements;
 * chi_new_out, discarded_out, entropy_out, lam2_out (min(chi_l d1, d2 chi_r)
 * values, may be NULL): host. Synchronises `stream`.                       */
osmps_status osmps_split_complex(osmps_ctx* ctx, const double* theta, double* A1, double* A2,
                                 int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r,
                                 int move_right, int64_t chi_max, double eps_local,
                                 int64_t* chi_new_out, double* discarded_out,
                                 double* entropy_out, double* lam2_out, int precision,
                                 void* stream);

typedef struct {
  double dt;            /* time step: each step applies exp(-i H dt) (Eq. propSE)         */
  int n_steps;          /* number of steps                                                 */
  int64_t chi_max;      /* maximal bond dimension                                          */
  double eps_local;     /* truncation tolerance of each split (0: chi_max only)            */
  double krylov_tol;    /* error estimate at which a local propagator stops                */
  int krylov_max_iter;  /* Krylov vectors per local propagator, 1..128                     */
  int precision;        /* osmps_precision of the contractions                             */
} osmps_tdvp_params;

typedef struct {
  double* energy;          /* in: NULL or host array of n_steps; out: <H> after each step   */
  double* norm;            /* in: NULL or host array of n_steps; out: <psi|psi> after each  */
  int64_t max_chi;         /* largest bond dimension reached                                */
  int max_krylov;          /* most Krylov vectors one local propagator used                 */
  int64_t krylov_calls;    /* local propagators applied (two-site and one-site)             */
  int64_t krylov_vectors;  /* Krylov vectors over all of them (= H_eff products)            */
  int64_t nonconverged;    /* propagators that stopped at krylov_max_iter above tolerance   */
  double max_discarded;    /* largest discarded weight of a split                           */
  double seconds;          /* wall time of the call                                         */
} osmps_tdvp_stats;

/* Real-time evolution of a complex MPS by n_steps of the symmetric
 * second-order two-site TDVP (Sec. 5.4; Haegeman et al.'s two-site scheme,
 * which lets the bond dimension grow): each step is a left-to-right half
 * sweep with dt/2 then a right-to-left one with dt/2. At the pair (k, k+1)
 * theta = A_k A_{k+1} is propagated by exp(-i H_eff dt/2) with the Krylov
 * method of osmps_heff_expm (Sec. 5.2, Eq. krylov:approx), split and
 * truncated as in osmps_split_complex (chi <= chi_max and the exact bound
 * min(prod d left, prod d right)), the environment on the side the centre
 * leaves is grown, and the new centre tensor is propagated backwards by
 * exp(+i H1_eff dt/2) with the one-site H_eff (not at the chain ends).
 * Input: chi_in (L + 1 bond dimensions, chi_in[0] = chi_in[L] = 1, each at
 * most chi_max), host_in[k] (HOST, complex, chi_in[k] x d_k x chi_in[k+1]).
 * The input must have sites 1..L-1 right-canonical (sum_{s,b} A[a,s,b]
 * conj(A[a2,s,b]) = delta(a, a2)), the centre at site 0 (any norm: it is
 * normalised); a product state qualifies. The same gauge holds on return.
 * Output: chi_out (L + 1), host_out[k] (HOST, room for
 * chi_max d_k chi_max complex elements, or for the exact bound), stats (may
 * be NULL). The MPO must be Hermitian (real W as for osmps_sweep). All
 * tensors stay on the device during the call; the context's workspace holds
 * the Krylov basis (4 chi_l d^2 chi_r krylov_max_iter doubles at the largest
 * bond). Synchronises `stream`.                                             */
osmps_status osmps_tdvp_evolve(osmps_ctx* ctx, const osmps_mpo* mpo, const int64_t* chi_in,
                               const double* const* host_in, const osmps_tdvp_params* p,
                               int64_t* chi_out, double* const* host_out,
                               osmps_tdvp_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* OSMPS_H */
