// Internal kernel launchers of the D-NGD library.
#pragma once

#include <vector>

#include "common.cuh"

namespace dngd {

template <typename T>
struct LayerPtrs {
  T* p[kMaxLayers];
};

// ---- jets.cu --------------------------------------------------------------
struct Tc3Scratch;
// tc3 (FP32 only, optional): hidden-layer GEMMs on the TF32 tensor cores
// (3xTF32, ~2^-21 per product) instead of FP32 SIMT.  Without `streams` the
// sweep is forward-only (losses): the activations are handed to the next
// GEMM as its split operand and Z / H are not kept for a reverse sweep.
template <typename T>
dngd_status jets_forward(const NetInfo& net, const T* theta, const double* X, const double* target,
                         LayerPtrs<T> Z, LayerPtrs<T> H, double* r, int* status, cudaStream_t st,
                         const Tc3Scratch* tc3 = nullptr, bool streams = false);

// G forward-only sweeps of line-search trials at once (FP32, 3xTF32 hidden
// layers; see jets.cu).
dngd_status jets_forward_trials(const NetInfo& net, int G, const float* theta_b, long long n, const double* X,
                                const double* target, float* Zb, float* Hb, double* rb, int* status, cudaStream_t st,
                                const Tc3Scratch& tc3);

// df64 (FP64 data): J's entries in double-float arithmetic (k_jac_write,
// ~2^-46 relative), for Jacobians whose consumer keeps fewer bits.
template <typename T, typename TJ>
dngd_status jets_backward_jacobian(const NetInfo& net, const T* theta, const double* X, LayerPtrs<T> Z,
                                   LayerPtrs<T> H, LayerPtrs<T> D, T* Hbar, TJ* J, long long ldJ,
                                   __nv_bfloat16* Jb, long long ldb, cudaStream_t st,
                                   const Tc3Scratch* tc3 = nullptr, int* status = nullptr,
                                   unsigned* rowmax = nullptr, bool df64 = false);

template <typename T>
dngd_status jets_fvv(const NetInfo& net, const T* theta, const T* v, const double* X, T* Z3, T* H3a,
                     T* H3b, double* fvv, cudaStream_t st, const Tc3Scratch* tc3 = nullptr,
                     int* status = nullptr);

// ---- linalg.cu ------------------------------------------------------------
// C[M x N] = alpha * A[M x K] * B^T + beta * C, B is [N x K] (both row-major).
// lower: skip output tiles strictly above the diagonal (syrk-style use).
template <typename T>
dngd_status gemm_nt(int M, int N, int K, T alpha, const T* A, long long lda, const T* B, long long ldb,
                    T beta, T* C, long long ldc, bool lower, cudaStream_t st);

// C[M x N] = alpha * A[M x K] * B[K x N] + beta * C (row-major).
template <typename T>
dngd_status gemm_nn(int M, int N, int K, T alpha, const T* A, long long lda, const T* B, long long ldb,
                    T beta, T* C, long long ldc, cudaStream_t st);

// C[M x N] = alpha * A^T diag(kscale) B + beta * C, A [K x M], B [K x N]
// row-major; kscale [K] may be null.  lower: as gemm_nt.
template <typename T>
dngd_status gemm_tn(int M, int N, int K, T alpha, const T* A, long long lda, const T* B, long long ldb, T beta,
                    T* C, long long ldc, const T* kscale, cudaStream_t st, bool lower = false);

// Lower triangle of the FP64 Gram C [M x M] = A^T A (at: A [K x M]) or
// A A^T (A [M x K]), row-major.  With a workspace ws of gram_f64_splits(M, K)
// x M x ldc doubles (when that is > 1) the K range is split over that many
// slices of blocks, so that a small M still fills the GPU, and the slices'
// partial products are added in a fixed order; ws = nullptr: one pass.
int gram_f64_splits(int M, int K);
dngd_status gram_f64(bool at, int M, int K, const double* A, long long lda, double* C, long long ldc, double* ws,
                     cudaStream_t st);

// FP32 GEMMs with compensated (Kahan over BK-slabs) accumulation.
dngd_status gemm_nt_comp(int M, int N, int K, float alpha, const float* A, long long lda, const float* B,
                         long long ldb, float beta, float* C, long long ldc, cudaStream_t st);
dngd_status gemm_tn_comp(int M, int N, int K, float alpha, const float* A, long long lda, const float* B,
                         long long ldb, float beta, float* C, long long ldc, const float* kscale, cudaStream_t st);

// In-place blocked Cholesky of the lower triangle of A [m x m] (lda).
// TA = double: everything in FP64.  TA = float: FP32 panels and trailing
// updates with every diagonal block factored in FP64.
// On a non-positive pivot sets status bit ST_NOT_SPD and status[1] = column.
template <typename TA>
dngd_status cholesky(int m, TA* A, long long lda, int* status, double* work, cudaStream_t st);

// FP32 factorisation of the mixed path: A = L L^T in place (lower) and the
// inverses of the 64 x 64 diagonal blocks of L written into Linv, which the
// caller zero-initialises; trtri_offdiag_f32 then completes Linv = L^{-1}.
// tc3 (optional): the trailing / inverse GEMMs on the TF32 tensor cores
// (3xTF32) — the factor only preconditions the refinement.  status: the
// context's four status words, all zero on entry; status[3] counts the
// block-factor CTAs within a launch and is zero again after it, except after
// a failed factorisation (ST_NOT_SPD), which the caller clears with the other
// words before the next one.
dngd_status cholesky_f32_inv(int m, float* A, long long lda, float* Linv, long long ldi, int* status,
                             cudaStream_t st, const Tc3Scratch* tc3 = nullptr);
dngd_status trtri_offdiag_f32(int m, const float* L, long long ldl, float* Linv, long long ldi, float* work,
                              cudaStream_t st, const Tc3Scratch* tc3 = nullptr, int* status = nullptr);

// x = (L L^T)^{-1} b with the FP64 factor (two triangular solves).
dngd_status chol_solve_f64(int m, const double* L, long long ldl, const double* b, double* x, cudaStream_t st);
// Inverses of the 64 x 64 diagonal blocks of an FP64 factor ([ceil(m/64)] x
// 64 x 64) and the blocked solve that uses them (w, y: work vectors [m]).
dngd_status trtri_diag64(int m, const double* L, long long ldl, double* Dinv, cudaStream_t st);
// L32 = fl32(L) (lower) and the diagonal 64-blocks of Linv = fl32(Dinv),
// zero elsewhere (both [m x ldk]).
dngd_status factor_to_f32(int m, const double* L, long long ldl, const double* Dinv, float* L32, float* Linv,
                          long long ldk, cudaStream_t st);
// The small nodes (n1 + n2 <= 512) of trtri_offdiag_f32's recursion only,
// bottom-up; the large nodes (k0, n1, n2) are returned bottom-up.
dngd_status trtri_small_nodes_f32(int m, const float* L, long long ldl, float* Linv, long long ldi, float* work,
                                  cudaStream_t st, std::vector<int3>* large_out);
dngd_status chol_solve_f64_dinv(int m, const double* L, long long ldl, const double* Dinv, const double* b, double* x,
                                double* w, double* y, cudaStream_t st);

// ---- pcg_persist.cu: one cooperative kernel per exact-Gram PCG solve ------
size_t pcg_persist_state_bytes();
// Runs the grid barrier with one arrival missing, so its bounded wait
// expires after limit_ms (records ST_TIMEOUT).
dngd_status barrier_expiry(void* state, int* status, double limit_ms, cudaStream_t st);
dngd_status transpose_f32(int m, const float* A, long long lda, float* T, long long ldt, cudaStream_t st);
// INVALID_ARG when the cooperative grid cannot be formed (callers then use
// the per-kernel loop).  Results in scal (S_ITERS, S_RR, S_BB, ...).
// work: [7 m] doubles.
dngd_status pcg_persist_solve(int m, const float2* K, long long ldk, double lambda, const float* Linv,
                              const float* LinvT, long long ldi, const double* b, double* x, double* work,
                              double* parts, long long parts_cap, double* scal, double tol, int maxit, void* state,
                              int* status, cudaStream_t st);

// ---- tc3.cu: FP32 GEMM on TF32 tensor cores with hi/lo splits -----------
struct OzGemm;
struct Tc3Scratch {
  float* buf = nullptr;
  size_t bytes = 0;
  OzGemm* ozg = nullptr;   // FP64 layer GEMMs from exact slice products (FP64 jets)
};
size_t tc3_scratch_bytes(int M, int N, int K);
// The scratch's two halves: the A operand's split [M x 2 Kp] and the B
// operand's split [N x 2 Kp] (row r: tf32 hi in [0, Kp), lo in [Kp, 2 Kp),
// Kp = K rounded up to 32, zero tails).
void tc3_halves(const Tc3Scratch& sc, float** a_half, float** b_half);
enum : unsigned {
  TC3_A_PRESPLIT = 1u,   // the A half already holds A_op's split (no split launch)
  TC3_B_PRESPLIT = 2u,   // the B half already holds B_op's split
  TC3_C_SPLIT = 4u,      // the epilogue also writes the result's split into the A half,
                         // as the A operand of a following GEMM with K = N (N <= 128, not lower)
};
// C = alpha A_op B_op^T + beta C; A_op = A [M x K] (or A^T with transA,
// A then [K x M]), B_op = B [N x K] (or B^T with transB); lower: only
// C[i][j], j <= i.  INVALID_ARG when the scratch is too small (callers then
// use the SIMT GEMM).
// kscale_a (optional, [K]): op(A)'s columns scaled by it (a diagonal in the
// product) as A is split.
dngd_status gemm_tc3(int M, int N, int K, float alpha, const float* A, long long lda, bool transA, const float* B,
                     long long ldb, bool transB, float beta, float* C, long long ldc, bool lower, const Tc3Scratch& sc,
                     int* status, cudaStream_t st, unsigned flags = 0u, const float* kscale_a = nullptr);

dngd_status gemm_tc3_trials(int G, int M, int N, int K, const float* B0, long long ldb, long long b_z, float* C,
                            long long ldc, long long c_z, const Tc3Scratch& sc, int* status, cudaStream_t st);

// ---- gram_oz.cu: exact Gram of an FP32 or FP64 matrix from BF16 integer slices ----
// Four 8-bit slices per entry; ng = 5 keeps the slice products of levels
// s + t <= 4 (13 products), ng = 6 levels <= 5 (15 products).  J is float*
// (j64 false) or double* (j64 true); ldJ a multiple of 4 and the row pad
// beyond n zero.
struct OzPlan;
size_t gram_oz_partial_bytes(int m, int n, int ng);
size_t gram_oz_slice_bytes(int m, int n);   // slices + row exponents
// K: FP32 lower triangle + shift; F: full symmetric Gram as double-float
// pairs (no shift)
// Its tile list is uploaded on st (the stream its runs are issued on).
dngd_status gram_oz_plan(OzPlan** plan, const void* J, bool j64, int ng, long long ldJ, int m, int n, void* slices,
                         float* K, long long ldk, float2* F, long long ldf, double* partials, size_t partial_bytes,
                         cudaStream_t st);
dngd_status gram_oz_read(const OzPlan* plan, double* out, cudaStream_t st);  // F as FP64 [m x ldf]
dngd_status gram_oz_set_shift(OzPlan* plan, double shift);
dngd_status gram_oz_run(OzPlan* plan, int* status, cudaStream_t st, cudaEvent_t ev_before_mma,
                        cudaEvent_t ev_after_mma);
// Per-row largest |J| (float bits) that the writer of J fills for the slicing
// (jets_backward_jacobian's rowmax); gram_oz_run reads it.
unsigned* gram_oz_rowmax(OzPlan* plan);
dngd_status gram_oz_reduce(OzPlan* plan, cudaStream_t st);
void gram_oz_free(OzPlan* plan);
int gram_oz_nsplit(const OzPlan* plan);
// The exact Gram's reduction also writes K + shift as FP64 (lower) into Kd
// when set (the FP64 factorisation's input), or not when Kd is null.
void gram_oz_set_fp64_out(OzPlan* plan, double* Kd);

// Blocked Cholesky (64-column steps) of the lower triangle of the FP64
// matrix C in place: diagonal blocks, panel solves and the first 64 columns
// of each trailing update in double-float arithmetic (~2^-47); the rest of
// each update exactly from six 8-bit slices per entry of the panel on the
// BF16 tensor cores (products of levels <= 6, each entry kept to 2^-49 of
// its row's largest), on a side stream beside the next step.
struct OzFactor;
size_t oz_factor_bytes(int m);   // panel slices + row exponents + tile list
dngd_status oz_factor_plan(OzFactor** plan, int m, double* C, long long ldc, void* work, cudaStream_t st);
dngd_status oz_factor_run(OzFactor* plan, int* status, cudaStream_t st);
void oz_factor_free(OzFactor* plan);
// Batched factorisation of n independent instances (each with its own
// OzFactor plan and status word): per 64-column step, one launch each for
// every instance's diagonal block, panel solve and whole trailing update
// (double-float).  A plan of one instance computes the same factor.
struct OzBatchFactor;
dngd_status oz_factor_batched_plan(OzBatchFactor** plan, int n, OzFactor* const* f, int* const* status,
                                   cudaStream_t st);
dngd_status oz_factor_batched_run(OzBatchFactor* plan, cudaStream_t st);
void oz_factor_batched_free(OzBatchFactor* plan);

// C = alpha A B^T + beta C in FP64 (A [M x K] ld lda; B [N x K] ld ldb, or
// with b_kn B given as [K x N]) from four 8-bit slices of every row of A and
// of B^T on the BF16 tensor cores (15 slice products, levels <= 5): each entry of A and B
// kept to 2^-33 of its row's largest, the products exact, so C is accurate
// to ~2^-33 of the row scales times K.  M, N, K within the plan's capacity.
size_t oz_gemm_bytes(int max_m, int max_n, int max_k);
dngd_status oz_gemm_plan(OzGemm** plan, int max_m, int max_n, int max_k, void* work);
dngd_status oz_gemm(OzGemm* plan, int M, int N, int K, double alpha, const double* A, long long lda, const double* B,
                    long long ldb, bool b_kn, double beta, double* C, long long ldc, int* status, cudaStream_t st);
void oz_gemm_free(OzGemm* plan);
// The preconditioner's inverse factor: Linv = fl32(L^{-1}) and LinvT =
// fl32(L^{-T}) (FP32, [m x ld]) of a lower FP64 factor L, from its diagonal
// blocks' inverses Dinv (trtri_diag64); small recursion nodes in FP32, large
// ones as FP64 sliced products through Li, LiT ([m x ld] FP64).  Scratch:
// L32 [m x ld] FP32, work32 >= m^2 / 4 floats, work >= (m/2 + 64)^2
// doubles; the plan's capacity >= (m, m, m).
dngd_status oz_trtri(OzGemm* plan, int m, const double* L, long long ldl, const double* Dinv, float* L32, float* Linv,
                     float* LinvT, double* Li, double* LiT, long long ld, float* work32, double* work, int* status,
                     cudaStream_t st);

// Explicit inverse of a lower-triangular FP32 factor: Linv = L^{-1} (lower).
dngd_status trtri_lower_f32(int m, const float* L, long long ldl, float* Linv, long long ldi, float* work,
                            cudaStream_t st);

// y = alpha * A x + add_scale * add  (FP32 A, double-float accumulation)
dngd_status gemv_n_f32(int m, int n, const float* A, long long lda, const double* x, double alpha, double* y,
                       const double* add, double add_scale, float2* xs, cudaStream_t st);

// y = alpha * A^T x  (A [m x n] row-major, x [m], y [n]); partials: [splits x n]
template <typename TA>
dngd_status gemv_t(int m, int n, const TA* A, long long lda, const double* x, double alpha, double* y,
                   double* partials, cudaStream_t st);

// y = alpha * A x + beta_y * y0 + gamma * z   (A [m x n] row-major, y [m])
template <typename TA>
dngd_status gemv_n(int m, int n, const TA* A, long long lda, const double* x, double alpha, double* y,
                   cudaStream_t st);

// ---- refine.cu: FP32 matrices with double-float accumulation ---------------
// y = alpha A^T x (A [m x n] FP32, lda % 4 == 0, padding columns zero).
// xs: scratch of round_up(max(m, n), 4) + 4 float2; partial_cap: doubles in partials.
// Queries the GEMV launch shape once (outside any stream capture).
void gemv_init();
dngd_status gemv_t_f32(int m, int n, const float* A, long long lda, const double* x, double alpha, double* y,
                       double* partials, long long partial_cap, float2* xs, cudaStream_t st);

// Preconditioned CG on (J J^T + lambda I) x = b with the FP32 J as operator
// and M^{-1} = Linv^T Linv as preconditioner; all scalars on the device.
struct PcgMixed {
  int m, n;
  const float* J;
  long long ldJ;
  const float* Linv;
  long long ldk;
  double lambda;
  double *res, *z, *p, *Ap, *u, *y;   // work vectors (u has n entries)
  float2* xs;
  double* partials;
  long long partial_cap;
  double* dotp;                       // >= 1024 doubles
  double* scal;                       // device scalars (S_COUNT)
  double* scal_h;                     // pinned host copy
  cudaEvent_t* ev;                    // optional: 4 events bracketing the first
                                      // J^T p and J u launches of the solve
  // exact-Gram mode: operator A = K64 (full symmetric double-float Gram, one GEMV)
  const float2* K64 = nullptr;
  long long ldk64 = 0;
  // exact-Gram synchronous solves: the persistent cooperative PCG kernel
  // (needs Linv^T and a barrier state word)
  const float* LinvT = nullptr;
  void* pstate = nullptr;
  double* pwork = nullptr;            // [7 m]
  int* status = nullptr;
  // synchronous solves: chunks of iterations captured once into a graph on
  // the stream cap and replayed (key: lambda, chunk size, kernels per chunk,
  // solution pointer)
  cudaGraphExec_t* chunk_exec = nullptr;
  double* chunk_key = nullptr;
  cudaStream_t cap = nullptr;
};
// async: enqueue exactly maxit iterations (kernels become no-ops after
// convergence) and never synchronise; iters/relres are then left untouched and
// the per-solve record (S_IT*, S_RR*, S_BB*) holds the result.
dngd_status pcg_mixed_solve(const PcgMixed& P, const double* b, double* x, double tol, int maxit, int check_every,
                            int* iters, double* relres, cudaStream_t st, bool async = false, int slot = 0);

// K[i,i] += shift for i < m.
template <typename T>
dngd_status add_diag(int m, T* K, long long ldk, double shift, cudaStream_t st);

// Deterministic dot products / norms into a device scalar.
dngd_status dot_dev(int n, const double* x, const double* y, double* out, double* partials, cudaStream_t st);
// out[g] = <x_g, x_g> for G vectors x_g = x + g n (one block each, fixed order).
dngd_status sqnorm_batch(int n, int G, const double* x, double* out, cudaStream_t st);

// Device-side vector kernels used by the refinement / PCG loops.
dngd_status axpy_dev(int n, double alpha, const double* x, double* y, cudaStream_t st);

// ---- matfree.cu: matrix-free operator and Nystrom preconditioner -----------
struct MatFree {
  const NetInfo* net;
  const double* X;
  LayerPtrs<float> H, D;   // stream activations / adjoints of the hidden layers
  float* vrow;             // [R]
  float* g32;              // [n]
  float* Y;                // [R x max_w]
  float* Hin;              // [R x d_in] input streams of layer 0
  int ell, RI;             // landmarks, their stream rows
  const int* lm;           // [ell] landmark residual (point) indices
  const int* lrows;        // [RI] stream rows of the landmarks
  const int* lrow0;        // [ell] first gathered row of landmark j
  const int* lS;           // [ell] streams of landmark j
  float *DI, *HI;          // [RI x max_w]
  float *P, *Q;            // [R x RI]
  float* KCI;              // [m x ell]
  float *Fo, *FoI, *fb;    // output-layer features [m x w_L], [ell x w_L], [m]
  float *KII, *LIIinv, *M, *C, *LCinv, *work;
  double *t1, *t2, *t3;
  float2* xs;
  double* partials;
  long long partial_cap;
  const Tc3Scratch* tc3;   // the factor-form GEMMs on the TF32 tensor cores (3xTF32), or null: SIMT
  int* status;
};
dngd_status mf_jtv(const MatFree& F, const double* v, float* g, cudaStream_t st);
dngd_status mf_jv(const MatFree& F, const float* u, double* y, cudaStream_t st);
dngd_status mf_kvp(const MatFree& F, const double* v, double lambda, double* w, cudaStream_t st);
dngd_status mf_kci(const MatFree& F, cudaStream_t st);
dngd_status mf_nystrom(const MatFree& F, double lambda, double nu, int* status, cudaStream_t st);
dngd_status mf_precond(const MatFree& F, double lambda, const double* x, double* z, cudaStream_t st);
dngd_status mf_input_rows(const MatFree& F, cudaStream_t st);
dngd_status mf_g_to_double(long long n, const float* g, double alpha, double* out, cudaStream_t st);
dngd_status mf_kii_trace(const MatFree& F, double* out, cudaStream_t st);

// ---- gram_tc.cu -----------------------------------------------------------
// K (FP32, lower 128x256 tiles) = Jlow Jlow^T with tcgen05 tensor cores.
// kind: 0 = BF16 operands (Jlow is bf16 [rows x ld]), 1 = TF32 (float).
struct GramPlan;
// The tile list is uploaded on st, the stream the runs are issued on (a copy
// on the legacy stream would not be ordered before work on a non-blocking
// stream).
dngd_status gram_tc_plan(GramPlan** plan, int kind, const void* Jlow, int m, int n, long long ld, float* K,
                         long long ldk, float* partials, size_t partial_bytes, cudaStream_t st);
dngd_status gram_tc_run(GramPlan* plan, int* status, cudaStream_t st, cudaEvent_t ev_before_mma,
                        cudaEvent_t ev_after_mma);
void gram_tc_free(GramPlan* plan);
size_t gram_tc_partial_bytes(int m, int n);

}  // namespace dngd
