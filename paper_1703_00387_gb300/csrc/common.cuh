// Internal declarations shared by the translation units of libosmps.
#pragma once

#include <cuda_runtime.h>
#include <cusolverDn.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <functional>
#include <vector>

#include "osmps.h"

namespace osmps {

// ---------------------------------------------------------------------------
// Errors: every failing path records a message (thread-local) and returns a
// status; nothing aborts or prints.
// ---------------------------------------------------------------------------
osmps_status set_error(osmps_status s, const char* fmt, ...);
void clear_error();

#define OSMPS_TRY(expr)                          \
  do {                                           \
    osmps_status st_ = (expr);                   \
    if (st_ != OSMPS_OK) return st_;             \
  } while (0)

#define OSMPS_CUDA(call)                                                                 \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return ::osmps::set_error(OSMPS_ECUDA, "%s failed: %s (%s:%d)", #call,             \
                                cudaGetErrorString(e_), __FILE__, __LINE__);             \
  } while (0)

#define OSMPS_LAUNCH_CHECK()                                                             \
  do {                                                                                   \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess)                                                               \
      return ::osmps::set_error(OSMPS_ECUDA, "kernel launch failed: %s (%s:%d)",         \
                                cudaGetErrorString(e_), __FILE__, __LINE__);             \
  } while (0)

#define OSMPS_SOLVER(call)                                                               \
  do {                                                                                   \
    cusolverStatus_t s_ = (call);                                                        \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                   \
      return ::osmps::set_error(OSMPS_ECUDA, "%s failed: cusolver status %d (%s:%d)",    \
                                #call, (int)s_, __FILE__, __LINE__);                     \
  } while (0)

// ---------------------------------------------------------------------------
// Workspace: named slots that grow on demand. A slot is owned by one code
// path at a time; nested calls use disjoint slots. Growing a slot
// synchronises the stream first, so earlier work on the old buffer is done.
// ---------------------------------------------------------------------------
enum Slot {
  SLOT_HEFF_T1 = 0,
  SLOT_HEFF_T2,
  SLOT_HEFF_T3,
  SLOT_HEFF_LOP,
  SLOT_HEFF_ROP,
  SLOT_HEFF_XOP,
  SLOT_HEFF_SMALL,
  SLOT_ENV_X,
  SLOT_ENV_Y,
  SLOT_ENV_OPA,
  SLOT_ENV_OPB,
  SLOT_ENV_MAT,
  SLOT_LZ_BASIS,
  SLOT_LZ_W,
  SLOT_LZ_SCAL,
  SLOT_LZ_PART,
  SLOT_LZ_PROJ,
  SLOT_LZ_X,
  SLOT_SPLIT_G,
  SLOT_SPLIT_EV,
  SLOT_SPLIT_WORK,
  SLOT_SPLIT_TMP,
  SLOT_SPLIT_TMP2,
  SLOT_QR_WORK,
  SLOT_QR_TAU,
  SLOT_QR_R,
  SLOT_SWEEP_THETA,
  SLOT_SWEEP_ENV,
  SLOT_SWEEP_ENV2,
  SLOT_RED,
  SLOT_NORM,
  SLOT_EMU_A,
  SLOT_EMU_B,
  SLOT_EMU_EXP,
  SLOT_EMU_MAX,
  SLOT_TRD,
  SLOT_VAR,
  SLOT_OV_X,
  SLOT_EIG_X,
  SLOT_EIG_F32,
  SLOT_EIG_R,
  SLOT_EIG_S,
  SLOT_EIG_P,
  SLOT_EIG_E,
  SLOT_EIG_SCAL,
  SLOT_GRAD_A,
  SLOT_GRAD_B,
  SLOT_GRAD_C,
  SLOT_GRAD_M,
  SLOT_GRAD_T,
  SLOT_GRAD_PART,
  SLOT_GRAD_ENVS,
  SLOT_CX_L,
  SLOT_CX_R,
  SLOT_CX_THETA,
  SLOT_HEFF_IDDEV,
  SLOT_COUNT
};

struct Buffer {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace osmps

struct osmps_ctx {
  int device = 0;
  int sm_count = 0;
  cusolverDnHandle_t solver = nullptr;
  osmps::Buffer slots[osmps::SLOT_COUNT];
  int* dev_flags = nullptr;      // device error flags (bit 0: bounded wait gave up)
  int* dev_info = nullptr;       // cuSOLVER info
  double* host_pinned = nullptr; // small pinned host staging area
  size_t host_pinned_count = 0;
  // Per-kernel CUDA-event records (osmps_profile_enable / osmps_profile_read).
  bool prof_on = false;
  struct ProfRec {
    cudaEvent_t a, b;
    int kernel;
    double flops, tensor_flops;
  };
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
  // Operator prepared by heff_prepare (converted L/R operands, reordered W).
  bool heff_ready = false;
  int heff_prec = -1;
  int64_t heff_dims[7] = {0, 0, 0, 0, 0, 0, 0};
  // identity environment channels of the prepared operator (-1: none), and
  // whether heff_prepare looks for them (split precisions only)
  int heff_skip_l = -1, heff_skip_r = -1;
  int identity_skip = OSMPS_IDENTITY_SOLVER;
  // eigensolver of the split: OSMPS_EIG_AUTO / OSMPS_EIG_CUSOLVER / OSMPS_EIG_TRIDIAG
  int eig_solver = 0;
  // Lanczos iteration driver: OSMPS_LANCZOS_AUTO / OSMPS_LANCZOS_HOST / OSMPS_LANCZOS_GRAPH
  int lanczos_mode = 0;
  // stream used only to record CUDA graphs (created on first use), and a flag
  // that makes workspace growth an error while a capture is open
  cudaStream_t capture_stream = nullptr;
  bool capturing = false;
  // tcgen05 GEMM tile widths chosen by measurement (OSMPS_AUTOTUNE_ON) per
  // size class: key, chosen width, microseconds at widths 256 / 128 / 64
  int tc_autotune = OSMPS_AUTOTUNE_ON;
  struct TcTuned {
    int64_t key[6];
    int bn;
    float us[3];
  };
  std::vector<TcTuned> tc_tuned;
  // Recorded Lanczos step graphs kept for replay (lanczos.cu), least recently
  // used first out, and a count of workspace (re)allocations that every
  // graph's key includes (a graph holds workspace addresses).
  struct LzGraph {
    std::vector<long long> key;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    long long body_launches = 0;
    unsigned long long last_use = 0;
  };
  std::vector<LzGraph> lz_graphs;
  unsigned long long lz_clock = 0;
  unsigned long long ws_epoch = 0;
};

namespace osmps {

// Returns a device pointer of at least `bytes` for `slot`, growing it if
// needed. On failure returns nullptr and records ENOMEM/ECUDA.
void* ws_get(osmps_ctx* ctx, Slot slot, size_t bytes, cudaStream_t stream, osmps_status* st);

// The context whose profiling records kernel launches made by the calling
// thread (set by every public entry point for the duration of the call).
struct CtxScope {
  explicit CtxScope(osmps_ctx* c);
  ~CtxScope();
  osmps_ctx* prev;
};
osmps_ctx* current_ctx();
// Bracket a launch with events on `stream` when profiling is on.
int prof_begin(cudaStream_t stream);
void prof_end(int handle, cudaStream_t stream, int kernel, double flops, double tensor_flops);

// Count of kernels this library has launched (all threads, all contexts).
void note_launch();
// Add k launches that ran as nodes of a replayed CUDA graph (k may be
// negative to take back a count made while recording).
void note_launches(long long k);
// Launches made by the calling thread so far.
long long thread_launch_count();
// Set by the batch scheduler on its worker threads (OSMPS_LANCZOS_AUTO then
// keeps the host loop: see lanczos.cu).
void set_batch_worker(bool on);
bool is_batch_worker();

// Ensure the pinned host staging area holds `count` doubles.
osmps_status pinned_reserve(osmps_ctx* ctx, size_t count);

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

// ---------------------------------------------------------------------------
// Float64 strided batched GEMM: C[b] = alpha * A[b] B[b] + beta * C[b] with
// element (m,k) of A at A[b*sab + m*sam + k*sak] (likewise B (k,n), C (m,n)).
// ---------------------------------------------------------------------------
struct GemmF64 {
  int64_t M = 0, N = 0, K = 0, batch = 1;
  const double* A = nullptr;
  int64_t sam = 0, sak = 0, sab = 0;
  const double* B = nullptr;
  int64_t sbk = 0, sbn = 0, sbb = 0;
  double* C = nullptr;
  int64_t scm = 0, scn = 0, scb = 0;
  double alpha = 1.0, beta = 0.0;
};
osmps_status gemm_f64(const GemmF64& g, cudaStream_t stream);

// ---------------------------------------------------------------------------
// Split-precision tensor-core GEMM (tcgen05):
//   C[M,N] = sum over the products (hi,hi), (hi,lo), (lo,hi) of A_p B_p^T
// A: M rows, B: N rows, each row holds [hi(0..Kp) | lo(0..Kp)] in the operand
// type (bf16 or tf32 in a 32-bit container), Kp a multiple of 64.
// Output: float32 or float64, row-major with leading dimension ldc.
// ---------------------------------------------------------------------------
enum TcKind { TC_BF16 = 0, TC_TF32 = 1 };
enum TcOut { TC_OUT_F32 = 0, TC_OUT_F64 = 1 };
struct GemmTc {
  int kind = TC_BF16;
  int64_t M = 0, N = 0, Kp = 0;
  int64_t K = 0;            // true inner size (for FLOP accounting; 0 = Kp)
  const void* A = nullptr;  // row stride = 2*Kp elements
  const void* B = nullptr;
  void* C = nullptr;
  int64_t ldc = 0;
  int out = TC_OUT_F32;
  const float* addend = nullptr;  // TC_OUT_F64 only: C = A B^T + addend (same ldc)
};
osmps_status gemm_tc(osmps_ctx* ctx, const GemmTc& g, cudaStream_t stream);
inline size_t tc_elem_bytes(int kind) { return kind == TC_BF16 ? 2 : 4; }

// Grouped split-precision GEMM: many independent problems in one persistent
// launch. Problem p computes
//   C[c_off + m ldc + n] = sum_{k < 64 nkb-ish} A[a_row0 + m][k] B[b_row0 + n][k]
// (the three split products) for m < M, n < N. A and B are packed split
// operands whose rows hold [hi(0..Kpl) | lo(0..Kpl)]; problem p reads the
// first nkb K slices of its rows, which must be zero beyond its own K.
struct GroupProblem {
  int a_row0, b_row0;  // first rows of the problem in the packed A / B operands
  int M, N;            // output rows / columns
  int nkb;             // K slices (128 bytes of K each) of the problem
  int tile0, tiles_n;  // first global tile, N tiles (filled by group_tiles)
  int pad;
  int64_t c_off, ldc;  // element offset of the problem's C[0,0], row stride
};
// Fill tile0 / tiles_n for tile width bn (64, 128 or 256); returns the tile count.
int64_t group_tiles(GroupProblem* probs, int n_prob, int bn);
bool tc_tile_width_ok(int bn);
struct GemmTcGrouped {
  int kind = TC_BF16, out = TC_OUT_F32;
  int bn = 256;             // tile width the problem table was built for
  const void* A = nullptr;  // packed operand rows, 2 * Kpl elements each
  int64_t rowsA = 0;
  const void* B = nullptr;
  int64_t rowsB = 0;
  int64_t Kpl = 0;          // lo-half offset (multiple of 64)
  void* C = nullptr;
  const GroupProblem* probs = nullptr;  // DEVICE table, tile0 ascending
  int n_prob = 0;
  int64_t n_tiles = 0;
  double logical_flops = 0.0;  // for profiling records
};
osmps_status gemm_tc_grouped(osmps_ctx* ctx, const GemmTcGrouped& g, cudaStream_t stream);

// Tile-width autotuning of the tcgen05 GEMMs (csrc/tune.cu). A size class
// (plain: tiles of the output at 128 x 64 granularity and K in 512s; grouped:
// problem count, 128 x 64 tile count, K) maps to the width measured fastest
// the first time the class ran; 0 = not yet measured.
struct TcKey {
  int64_t v[6];
};
TcKey tc_key(int grouped, int kind, int out, int64_t a, int64_t b, int64_t c);
int tc_tuned_width(osmps_ctx* ctx, const TcKey& key);
// true when a first product of an unmeasured class may be timed now (tuning
// on, no stream capture, no kernel profiling in progress)
bool tc_may_tune(osmps_ctx* ctx);
// us[w] = mean CUDA-event time of reps runs of fn on stream
osmps_status tc_time_launches(osmps_ctx* ctx, cudaStream_t stream, int reps, float* us,
                              const std::function<osmps_status(cudaStream_t)>& fn);
// store the fastest of widths[0..2] (times us) for key; returns it
int tc_record_tuning(osmps_ctx* ctx, const TcKey& key, const int* widths, const float* us);

// Split a float64 (or float32) matrix view into the hi|lo operand layout.
// Source element (row r, col k) with r = r0*n1 + r1 (r1 < n1) lives at
// src[r0*s0 + r1*s1 + k*sk]. Destination row r holds hi at [0,K), zeros at
// [K,Kp), lo at [Kp, Kp+K), zeros up to 2Kp.
struct SplitView {
  const void* src = nullptr;
  bool src_f32 = false;
  int64_t rows = 0, n1 = 1, K = 0;
  int64_t s0 = 0, s1 = 0, sk = 1;
};
osmps_status split_operand(const SplitView& v, int kind, void* dst, int64_t Kp, cudaStream_t stream);

// ---------------------------------------------------------------------------
// Float64-accurate GEMM on the bf16 tensor cores (error-free slicing):
// C[M,N] = sum_k a(m,k) b(n,k), with a and b given as views (SplitView: row
// m / n, column k; float64 sources). C is float64, row-major, ldc. With
// subtract, C[M,N] -= the product instead (C must not overlap a or b). With
// small_on_dmma, products that the float64 DMMA kernel finishes in an
// estimated 40 us (plain float64 views) run there instead of the emulation.
osmps_status gemm_emu(osmps_ctx* ctx, const SplitView& a, const SplitView& b, int64_t M,
                      int64_t N, int64_t K, double* C, int64_t ldc, cudaStream_t s,
                      bool subtract = false, bool small_on_dmma = true);

// ---------------------------------------------------------------------------
// Small contractions with an MPO tensor ("W-steps"): for every fiber
// (o1, o2, c): out[o1*os1 + o2*os2 + o*ostride + c] = sum_i Mat[i][o] in[o1*is1 + o2*is2 + i*istride + c]
// Mat is P x Q (row-major, float64, on the device).
// ---------------------------------------------------------------------------
struct Fiber {
  int64_t P = 0, Q = 0;
  int64_t n_o1 = 1, n_o2 = 1, nc = 0;
  int64_t is1 = 0, is2 = 0, istride = 0;
  int64_t os1 = 0, os2 = 0, ostride = 0;
};
osmps_status fiber_contract_f64(const Fiber& f, const double* Mat, const double* in, double* out,
                                cudaStream_t stream);
osmps_status fiber_contract_f32(const Fiber& f, const double* Mat, const float* in, float* out,
                                cudaStream_t stream);
// Same, but the output is written into a split operand: plain output offset
// off = row*Kcols + col is stored as hi at dst[row*2Kp + col], lo at
// dst[row*2Kp + Kp + col].
osmps_status fiber_contract_f32_split(const Fiber& f, const double* Mat, const float* in,
                                      void* dst, int kind, int64_t Kcols, int64_t Kp,
                                      cudaStream_t stream);
// Both W-steps of H_eff.theta fused (T1 -> split T3) for the d = 2 MPO
// shapes it is specialised for; *done = false means the caller must fall back
// to the two fiber contractions.
// Identity environment channels: with skip_l >= 0, T1 holds the wl - 1 other
// channels and channel skip_l is theta (L[:, skip_l, :] = 1); with
// skip_r >= 0, the split operand holds the wr - 1 other output channels and
// channel skip_r (R[:, skip_r, :] = 1) goes as float32 to yid (rows
// (a2, t1, t2), chi_r columns) for the stage-4 epilogue to add.
struct WStepIdentity {
  const double* theta = nullptr;
  int skip_l = -1, skip_r = -1;
  float* yid = nullptr;
};
bool fused_wsteps_supported(int64_t d1, int64_t d2, int64_t wl, int64_t wm, int64_t wr);
osmps_status fused_wsteps_f32_split(const float* T1, const double* Mat1, const double* Mat2,
                                    void* dst, int kind, int64_t chi_l, int64_t d1, int64_t d2,
                                    int64_t chi_r, int64_t wl, int64_t wm, int64_t wr, int64_t Kp,
                                    const WStepIdentity& id, cudaStream_t s, bool* done);
// Largest |E[a, w, b] - delta_ab| over (a, b) for the channels w = 0 and
// w = w_count - 1 of an environment E (chi x w_count x chi): two doubles to
// dev_out (device), for the identity-channel test of heff_prepare.
osmps_status identity_channel_deviation(const double* E, int64_t chi, int64_t w_count,
                                        double* dev_out, cudaStream_t s);
osmps_status zero_pad_columns(void* dst, int kind, int64_t rows, int64_t Kcols, int64_t Kp,
                              cudaStream_t stream);

// Reorder an MPO tensor for a W-step: Mat[i][o] with i and o composed from
// the four indices of W[w,t,s,w2] (dims dw, d, d, dw2) by the given maps.
// code selects one of the fixed orders used by the contractions.
enum WOrder {
  WORD_IN_W_S__OUT_T_W2 = 0,   // i = (w, s),  o = (t, w2)   [left side]
  WORD_IN_S_W2__OUT_W_T = 1,   // i = (s, w2), o = (w, t)    [right side]
  WORD_IN_T_W2__OUT_W_S = 2    // i = (t, w2), o = (w, s)    [left side, transposed]
};
osmps_status w_reorder(const double* W, int64_t dw, int64_t d, int64_t dw2, int order, double* Mat,
                       cudaStream_t stream);

// ---------------------------------------------------------------------------
// Vector primitives (float64) used by Lanczos and normalisations.
// ---------------------------------------------------------------------------
osmps_status vec_norm2(osmps_ctx* ctx, const double* x, int64_t n, double* dev_out, cudaStream_t s);
osmps_status vec_scale_by_inv_sqrt(double* x, int64_t n, const double* dev_norm2, cudaStream_t s);
osmps_status vec_scale_by_inv(double* y, const double* x, int64_t n, const double* dev_div,
                              cudaStream_t s);
osmps_status check_finite(osmps_ctx* ctx, const double* x, int64_t n, cudaStream_t s, bool* ok);

// Internal entry points shared between translation units (no argument checks).
osmps_status heff_apply_impl(osmps_ctx* ctx, const double* L, const double* W1, const double* W2,
                             const double* R, const double* theta, double* y, int64_t chi_l,
                             int64_t d1, int64_t d2, int64_t chi_r, int64_t wl, int64_t wm,
                             int64_t wr, int precision, cudaStream_t stream, bool prepared);
osmps_status heff_prepare(osmps_ctx* ctx, const double* L, const double* W1, const double* W2,
                          const double* R, int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r,
                          int64_t wl, int64_t wm, int64_t wr, int precision, cudaStream_t stream, bool find_identity = true);
osmps_status env_update_impl(osmps_ctx* ctx, int side, const double* env_in, const double* A,
                             const double* W, double* env_out, int64_t chi_l, int64_t d,
                             int64_t chi_r, int64_t w_in, int64_t w_out, int precision,
                             cudaStream_t stream);
osmps_status lanczos_impl(osmps_ctx* ctx, const double* L, const double* W1, const double* W2,
                          const double* R, double* theta, int64_t chi_l, int64_t d1, int64_t d2,
                          int64_t chi_r, int64_t wl, int64_t wm, int64_t wr, int max_iter,
                          double tol, int precision, double* energy, int* iters, double* resid,
                          cudaStream_t stream);
// y = H x on stream q. Inside the Lanczos step graph the calls are recorded
// by stream capture: launches only, no allocation, no synchronisation.
using Matvec = std::function<osmps_status(const double* x, double* y, cudaStream_t q)>;
// Lanczos ground state of a symmetric operator given as a Matvec (device
// vectors of length n, work launched on s). Float64 Krylov basis with full
// reorthogonalisation; theta is the start vector and receives the Ritz vector.
// P (kp rows, stride ldp): orthonormal rows whose span the search avoids.
// mkey[0..nmkey): identifies everything the matvec's launches depend on
// besides workspace addresses (shapes, precision, operator identity); with
// it, the recorded step graph is kept in the context and replayed by later
// calls with the same key. Without it (nmkey = 0) the graph is recorded for
// this call only.
osmps_status lanczos_core(osmps_ctx* ctx, int64_t n, double* theta, int max_iter, double tol,
                          const Matvec& matvec, double* energy, int* iters, double* resid,
                          cudaStream_t s, const double* P = nullptr, int64_t ldp = 0, int kp = 0,
                          const long long* mkey = nullptr, int nmkey = 0);
osmps_status theta_form_tc(osmps_ctx* ctx, const double* A1, const double* A2, double* theta,
                           int64_t chi_l, int64_t d1, int64_t chi_m, int64_t d2, int64_t chi_r,
                           int precision, cudaStream_t stream);
osmps_status theta_form_impl(const double* A1, const double* A2, double* theta, int64_t chi_l,
                             int64_t d1, int64_t chi_m, int64_t d2, int64_t chi_r,
                             cudaStream_t stream);
// Householder tridiagonalisation (dsytrd layout: reflectors below the
// subdiagonal of column j, d, e, tau) of a full symmetric n x n matrix.
bool sytrd_supported(int64_t n);
osmps_status sytrd_tc(osmps_ctx* ctx, double* A, int64_t n, double* d, double* e, double* tau,
                      cudaStream_t s);
// Largest nev eigenpairs of the symmetric n x n matrix G (overwritten):
// eigenvalues ascending in ev, eigenvectors as the rows of Y (nev x n).
osmps_status eig_top(osmps_ctx* ctx, double* G, int64_t n, int64_t nev, double* ev, double* Y,
                     cudaStream_t s);
// Krylov propagator (lanczos.cu) on the real 2x2 embedding of complex
// tensors: X[r, w, c] (interleaved complex) -> X~[(p, r), w, (q, c)], with
// conj applied first when set.
osmps_status embed_complex(const double* z, double* out, int64_t r, int64_t w, int64_t c,
                           bool conj, cudaStream_t s);
// exp(-i tau H) theta~ for the embedded start vector theta_emb (length
// 4 n_c, n_c = chi_l D chi_r complex elements) and the embedded operator
// matvec; the result goes to theta_out as interleaved complex, or embedded
// (may alias theta_emb) with out_embedded.
osmps_status expm_core(osmps_ctx* ctx, int64_t n_c, const double* theta_emb, double* theta_out,
                       int64_t chi_l, int64_t D, int64_t chi_r, double tau, int max_iter,
                       double tol, const Matvec& matvec, int* iters, double* err, cudaStream_t s,
                       bool out_embedded);
// Truncation of a Gram spectrum (split.cu): ev (any order, nev values) with
// tr = ||theta||^2; keeps min(chi_max, rank, the local-tolerance count).
struct Trunc {
  int64_t keep = 0;
  double discarded = 0.0, entropy = 0.0;
  std::vector<int> order;   // indices of the kept values, descending
  std::vector<double> lam2;  // all values / tr, descending
};
osmps_status truncate_spectrum(const double* ev, int64_t nev, double tr, int64_t rank,
                               int64_t chi_max, double eps_local, Trunc* t);
osmps_status split_impl(osmps_ctx* ctx, const double* theta, double* A1, double* A2,
                        int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r, int move_right,
                        int64_t chi_max, double eps_local, int64_t* chi_new, double* discarded,
                        double* entropy, double* lam2_out, int precision, cudaStream_t stream);

// Gradients. fiber_weight_grad: dMat[i][o] = sum over the fibers of f of
// X[fiber, i] Y[fiber, o] (X in the input layout of f, Y in its output
// layout); P, Q <= 64. site_energy_grad: the MPO-energy gradient of one
// site, scale * sum L[a2,w,a] A[a2,t,b2] A[a,s,b] R[b2,w2,b], written as
// gW[w,t,s,w2]; precision FP64 (DMMA) or anything else (emulated float64).
osmps_status fiber_weight_grad(osmps_ctx* ctx, const Fiber& f, const double* X, const double* Y,
                               double* dMat, cudaStream_t s);
osmps_status site_energy_grad(osmps_ctx* ctx, const double* Lenv, const double* A,
                              const double* Renv, double* gW, int64_t chi_l, int64_t d,
                              int64_t chi_r, int64_t wl, int64_t wr, double scale, int precision,
                              cudaStream_t s);

inline bool valid_precision(int p) {
  return p == OSMPS_PREC_FP64 || p == OSMPS_PREC_BF16X3 || p == OSMPS_PREC_TF32X3 ||
         p == OSMPS_PREC_FP64_EMU;
}

}  // namespace osmps
