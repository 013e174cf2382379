// C ABI of the D-NGD step: context set-up, workspace, and the step pipeline
//   jets + J  ->  Gram K + lambda I  ->  factor  ->  alpha  ->  v = -J^T alpha
//   -> f_vv  ->  beta (same factor / preconditioner)  ->  a  ->  GA test  ->  delta
// following Alg. DenseDualSolve of the paper (push-through recovery).
#include <chrono>
#include <math.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "step_kernels.h"

using namespace dngd;

namespace dngd {
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace dngd

struct dngd_ctx {
  dngd_problem_desc desc;
  NetInfo net;
  cudaStream_t st = nullptr;
  int m = 0, R = 0;
  long long n = 0;
  int prec = 0;
  double lambda = 0.0;
  bool timing = false;
  bool have_step = false;
  std::vector<void*> allocs;

  // staging for host inputs / outputs
  double *theta_s = nullptr, *X_s = nullptr, *target_s = nullptr, *nvec_s = nullptr, *mvec_s = nullptr;
  double* theta_tmp = nullptr;  // line search
  float *theta32 = nullptr, *v32 = nullptr;
  float2* xs = nullptr;  // hi/lo split of the vector of an FP32 GEMV

  // jets
  void* Z[kMaxLayers] = {};
  void* H[kMaxLayers] = {};
  void* D[kMaxLayers] = {};
  void* Hbar = nullptr;
  void *Z3 = nullptr, *H3a = nullptr, *H3b = nullptr;

  // Jacobian and Gram
  void* J = nullptr;
  long long ldJ = 0;
  __nv_bfloat16* Jb = nullptr;
  long long ldb = 0;
  void* K = nullptr;
  long long ldk = 0;
  void* Kcopy = nullptr;
  float* Linv = nullptr;
  float* trtri_work = nullptr;
  OzPlan* oz = nullptr;       // exact-Gram mode
  OzFactor* ozf = nullptr;    // its FP64 factorisation (exact sliced trailing updates)
  OzBatchFactor* ozb = nullptr;   // the same with double-float trailing updates (factor_update = DF)
  int phase = 0;              // batched steps: 1 stops before the factor, 2 starts after it
  OzGemm* ozi = nullptr;      // FP64 GEMMs of the factor's inverse (exact-Gram modes)
  void* ozi_work = nullptr;
  double *Li64 = nullptr, *LiT64 = nullptr;   // the factor's FP64 inverse and its transpose
  OzGemm* ozg = nullptr;      // FP64 jets' layer GEMMs from exact slice products (MIXED_OZ64)
  void* ozg_work = nullptr;
  Tc3Scratch ozs;             // hands ozg to the FP64 jets
  double* Kd = nullptr;       // exact Gram + (lambda + mu) I, FP64 lower: factored in place
  void* ozf_work = nullptr;
  void* oz_slices = nullptr;
  double* oz_partials = nullptr;
  float2* K64 = nullptr;      // exact Gram as double-float pairs (full symmetric, no shift)
  float* LinvT = nullptr;     // transpose of Linv (exact-Gram persistent PCG)
  void* pstate = nullptr;     // grid-barrier state of the persistent PCG
  double* pwork = nullptr;    // [7 m] vectors of the persistent PCG
  Tc3Scratch tc3;             // split operands of the TF32 tensor-core GEMMs (mixed paths)
  cudaStream_t cap_st = nullptr;                 // capture stream of the PCG chunk graphs
  cudaGraphExec_t pcg_chunk[2] = {nullptr, nullptr};
  double pcg_chunk_key[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};   // lambda, chunk, kernels, x
  double* Dinv = nullptr;     // FP64 path: inverses of the factor's 64 x 64 diagonal blocks
  double* tw = nullptr;       // FP64 path: [2 ms] triangular-solve work
  // FP64 path: the dense system's space (Prop. 3.1 primal, n x n, or
  // Thm. 3.1 dual, m x m) and its dimension ms; gp [n]: -J^T of the
  // right-hand side of a primal solve
  bool primal = false;
  int ms = 0;
  double* gp = nullptr;
  double* gws = nullptr;      // FP64 path: the split Gram's partial products (null: one pass)
  float* gram_partials = nullptr;
  size_t gram_partial_bytes = 0;
  GramPlan* gram = nullptr;

  // vectors
  double *r = nullptr, *alpha = nullptr, *v = nullptr, *fvv = nullptr, *beta = nullptr, *a = nullptr,
         *delta = nullptr;
  double *cg_res = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_Ap = nullptr, *cg_u = nullptr,
         *cg_y = nullptr, *xsol = nullptr;
  double* partials = nullptr;
  double* dot_partials = nullptr;
  double* scal = nullptr;
  double* scal_h = nullptr;  // pinned
  int* status = nullptr;
  int* status_h = nullptr;  // pinned
  int iters[2] = {0, 0};
  double shift_used = 0.0;
  double mu_sticky = 0.0;  // preconditioner shift that factored last time
  int factor_attempts = 0;
  void* K0 = nullptr;      // mixed path: Gram + (lambda + mu0) I before factorisation
  double relres[2] = {0.0, 0.0};
  cudaEvent_t ev[10] = {};
  cudaEvent_t kev[4] = {};  // first J^T p / J u launches of the first solve

  // asynchronous (graph-capturable) stepping
  bool async = false;        // current step enqueues without host synchronisation
  bool async_ok = false;     // a synchronous step has fixed the shift: async allowed
  cudaGraphExec_t graph = nullptr;
  double graph_lambda = 0.0;
  double* ls_dev = nullptr;          // line search: etas [64], losses [64], result [2]
  double* ls_host = nullptr;         // pinned copy of the etas
  double* loss_dev = nullptr;        // trial losses of dngd_loss [64]
  double* loss_host = nullptr;       // pinned copy [64]
  int ls_k = 0;
  float* ls_th32 = nullptr;          // FP32 parameters of the batched line-search trials
  double* ls_r = nullptr;            // their residuals [G m]
  float *ls_Z = nullptr, *ls_H = nullptr;  // their pre-activations / activations [G R max_w]
  int ls_G = 0;                            // trials per batched sweep
  double graph_mu = 0.0;
  // refinement iterations of a captured (asynchronous) solve, which cannot
  // stop on the host: twice the last synchronous step's count plus two (at
  // least 8, at most refine_max_it); iterations after convergence are no-ops,
  // and a captured solve that has not converged by then is redone
  // synchronously (batch) or makes the next step synchronous
  int async_it = 0;
  int graph_it = 0;
  cudaStream_t gst = nullptr;        // private stream for capture / replay
  unsigned long long graph_kernels = 0;  // kernel launches captured in the graph
  cudaEvent_t gev[2] = {};           // fences between st and gst

  // matrix-free Nystrom-PCG solver (solver == DNGD_PCG)
  bool pcg = false;
  MatFree mf{};
  std::vector<int> lm_host;             // landmark point indices
  int* d_lm = nullptr;
  int* d_lrows = nullptr;
  int* d_lrow0 = nullptr;
  int* d_lS = nullptr;
  int RI_max = 0;
  double nu_sticky = 0.0;
  double nu_used = 0.0;
};

namespace {

constexpr const char* kVersion = "dngd-gb300 0.1 (sm_103a)";
constexpr int kTrials = 8;  // most line-search trials per batched forward sweep

// trials per batched sweep: up to kTrials while their activations stay
// within 2^26 floats per buffer (at least 2)
int trials_of(const NetInfo& net) {
  const long long per = (long long)net.R * net.max_w;
  long long g = per > 0 ? (1LL << 26) / per : kTrials;
  return (int)(g > kTrials ? kTrials : (g < 2 ? 2 : g));
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
dngd_status dalloc(dngd_ctx* c, T** p, size_t count) {
  if (count == 0) count = 1;
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return DNGD_ERR_OOM;
  }
  c->allocs.push_back(q);
  *p = (T*)q;
  return DNGD_OK;
}

long long round_up(long long a, long long b) { return ((a + b - 1) / b) * b; }

// FP64 jets, residuals and Jacobian (the FP64 path and the exact-Gram mode
// of an FP64 Jacobian)
bool jets64(int prec) { return prec == DNGD_FP64 || prec == DNGD_MIXED_OZ64; }
// exact Gram from integer slices on the tensor cores
bool oz_mode(int prec) { return prec == DNGD_MIXED_OZ || prec == DNGD_MIXED_OZ64; }

// lambda > 0 everywhere; an FP64 context also takes a finite lambda <= 0
// (K + lambda I may then be indefinite, which its Cholesky reports)
bool lambda_ok(int prec, double lambda) {
  return prec == DNGD_FP64 ? isfinite(lambda) != 0 : lambda > 0.0 && isfinite(lambda) != 0;
}

dngd_status build_net(const dngd_problem_desc* d, NetInfo* net) {
  memset(net, 0, sizeof(*net));
  if (d->n_layers < 1 || d->n_layers > kMaxLayers) return DNGD_ERR_INVALID_ARG;
  if (d->widths[0] < 1 || d->widths[0] > kMaxDim) return DNGD_ERR_INVALID_ARG;
  if (d->widths[d->n_layers] != 1) return DNGD_ERR_INVALID_ARG;
  if (d->n_classes < 1 || d->n_classes > kMaxClasses) return DNGD_ERR_INVALID_ARG;
  net->n_layers = d->n_layers;
  net->d_in = d->widths[0];
  long long off = 0;
  int maxw = 1;
  for (int l = 0; l <= d->n_layers; ++l) {
    if (d->widths[l] < 1 || d->widths[l] > 65536) return DNGD_ERR_INVALID_ARG;
    net->widths[l] = d->widths[l];
  }
  for (int l = 0; l < d->n_layers; ++l) {
    net->w_off[l] = off;
    off += (long long)d->widths[l + 1] * d->widths[l];
    net->b_off[l] = off;
    off += d->widths[l + 1];
    if (l + 1 < d->n_layers) maxw = d->widths[l + 1] > maxw ? d->widths[l + 1] : maxw;
  }
  net->n = off;
  net->max_w = maxw;
  int p0 = 0, row0 = 0;
  for (int c = 0; c < d->n_classes; ++c) {
    const dngd_class_desc& cd = d->classes[c];
    if (cd.count < 1) return DNGD_ERR_INVALID_ARG;
    ClassInfo& ci = net->cls[c];
    ci.p0 = p0;
    ci.count = cd.count;
    ci.c_val = cd.c_val;
    ci.c_lap = cd.c_lap;
    ci.scale = 1.0 / sqrt((double)cd.count);
    ci.nD = 0;
    bool any_lap = false;
    for (int k = 0; k < net->d_in; ++k) {
      const bool lap = cd.lap_mask[k] != 0 && cd.c_lap != 0.0;
      if (cd.c_grad[k] != 0.0 || lap) {
        ci.D[ci.nD] = k;
        ci.c_gradD[ci.nD] = cd.c_grad[k];
        ci.lapD[ci.nD] = lap ? 1 : 0;
        ci.nD++;
      }
      any_lap = any_lap || lap;
    }
    ci.has_lap = any_lap ? 1 : 0;
    ci.S = 1 + ci.nD + ci.has_lap;
    ci.row0 = row0;
    row0 += ci.S * cd.count;
    p0 += cd.count;
  }
  net->n_classes = d->n_classes;
  net->m = p0;
  net->R = row0;
  return DNGD_OK;
}

struct Sizes {
  size_t total = 0;
};

void evrec(dngd_ctx* c, int i) {
  if (c->timing) cudaEventRecord(c->ev[i], c->st);
}

// Resolve an input pointer: device pointers are used in place, host pointers
// are copied into the staging buffer.
const double* in_ptr(dngd_ctx* c, const double* p, double* stage, size_t count) {
  if (!p) return nullptr;
  if (is_device_ptr(p)) return p;
  cudaMemcpyAsync(stage, p, count * sizeof(double), cudaMemcpyHostToDevice, c->st);
  return stage;
}

// The dense system's space: 1 primal (n x n, Prop. 3.1), 0 dual (m x m,
// Thm. 3.1), -1 an invalid request.  Automatic: the smaller system, primal
// only where it is built (FP64, dense solver).
int resolve_space(const dngd_problem_desc* d, const NetInfo& net) {
  const bool can = d->precision == DNGD_FP64 && d->solver == DNGD_DENSE;
  switch (d->solve_space) {
    case DNGD_SPACE_DUAL: return 0;
    case DNGD_SPACE_PRIMAL: return can ? 1 : -1;
    case DNGD_SPACE_AUTO: return can && net.n < net.m ? 1 : 0;
    default: return -1;
  }
}

dngd_status read_status(dngd_ctx* c) {
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->status_h, c->status, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->st));
  DNGD_CUDA_CHECK(cudaStreamSynchronize(c->st));
  const int s = c->status_h[0];
  if (s & ST_TIMEOUT) return DNGD_ERR_TIMEOUT;
  if (s & ST_NOT_SPD) return DNGD_ERR_NOT_SPD;
  if (s & ST_NONFINITE) return DNGD_ERR_NONFINITE;
  if (s & ST_NO_CONVERGE) return DNGD_ERR_NO_CONVERGE;
  return DNGD_OK;
}

// The damping rule lambda_k = min(L(theta_k), cap) of the paper's experiments
// (App. A.3), L = 1/2 ||r||^2 of the residuals just computed: one reduction
// and one read-back before K + lambda I is formed.
dngd_status apply_lambda_rule(dngd_ctx* c) {
  const double cap = c->desc.lambda_cap;
  if (!(cap > 0.0) || c->async) return DNGD_OK;
  dngd_status s = dot_dev(c->m, c->r, c->r, c->scal + S_LOSS, c->dot_partials, c->st);
  if (s) return s;
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->scal_h + S_LOSS, c->scal + S_LOSS, sizeof(double), cudaMemcpyDeviceToHost,
                                  c->st));
  DNGD_CUDA_CHECK(cudaStreamSynchronize(c->st));
  const double loss = 0.5 * c->scal_h[S_LOSS];
  c->lambda = (loss > 0.0 && isfinite(loss) && loss < cap) ? loss : cap;
  return DNGD_OK;
}

template <typename T>
LayerPtrs<T> lp(void* const* a) {
  LayerPtrs<T> r;
  for (int l = 0; l < kMaxLayers; ++l) r.p[l] = (T*)a[l];
  return r;
}

// ---------------------------------------------------------------------------
// Residuals + Jacobian in the context's precision
// ---------------------------------------------------------------------------

template <typename T>
const T* theta_in_T(dngd_ctx* c, const double* theta);
template <>
const double* theta_in_T<double>(dngd_ctx* c, const double* theta) {
  (void)c;
  return theta;
}
template <>
const float* theta_in_T<float>(dngd_ctx* c, const double* theta) {
  to_float(c->n, theta, c->theta32, c->st);
  return c->theta32;
}

template <typename T>
dngd_status forward_only(dngd_ctx* c, const T* thT, const double* X, const double* target, double* r,
                         bool tensor = false) {
  return jets_forward<T>(c->net, thT, X, target, lp<T>(c->Z), lp<T>(c->H), r, c->status, c->st,
                         tensor && c->tc3.buf ? &c->tc3 : nullptr);
}

// FP32 paths: the hidden-layer GEMMs of the jets, J's reverse sweep and f_vv
// run on the TF32 tensor cores (3xTF32) when the context has the scratch.
const Tc3Scratch* tc3p(dngd_ctx* c);

// The tensor-core GEMM handle of the jets: 3xTF32 (FP32 jets) or the FP64
// GEMM from slice products (FP64 jets of MIXED_OZ64); null: SIMT GEMMs.
template <typename T>
const Tc3Scratch* jets_tc(dngd_ctx* c) {
  if (std::is_same<T, float>::value) return tc3p(c);
  return c->ozg ? &c->ozs : nullptr;
}

template <typename T>
dngd_status residual_jacobian_T(dngd_ctx* c, const T* thT, const double* X, const double* target) {
  const Tc3Scratch* t3 = jets_tc<T>(c);
  dngd_status s = jets_forward<T>(c->net, thT, X, target, lp<T>(c->Z), lp<T>(c->H), c->r, c->status, c->st, t3,
                                  true);
  if (s) return s;
  // the exact Gram's slicing takes each row's largest |J| from the writer;
  // its FP64 Jacobian is written in double-float arithmetic: ~46 bits,
  // where the slices keep 33 of each row's largest entry and the map-back
  // J^T x needs no more)
  return jets_backward_jacobian<T, T>(c->net, thT, X, lp<T>(c->Z), lp<T>(c->H), lp<T>(c->D), (T*)c->Hbar,
                                      (T*)c->J, c->ldJ, c->prec == DNGD_MIXED_BF16 ? c->Jb : nullptr, c->ldb,
                                      c->st, t3, c->status, c->oz ? gram_oz_rowmax(c->oz) : nullptr,
                                      c->prec == DNGD_MIXED_OZ64);
}

// ---------------------------------------------------------------------------
// Solves with the factor of the last step
// ---------------------------------------------------------------------------

long long partial_cap(const dngd_ctx* c) { return 16LL * (c->n > c->m ? c->n : c->m); }

// y = alpha J^T x in the context's precision
template <typename T>
dngd_status jt_x(dngd_ctx* c, const double* x, double alpha, double* y);
template <>
dngd_status jt_x<double>(dngd_ctx* c, const double* x, double alpha, double* y) {
  return gemv_t<double>(c->m, (int)c->n, (const double*)c->J, c->ldJ, x, alpha, y, c->partials, c->st);
}
template <>
dngd_status jt_x<float>(dngd_ctx* c, const double* x, double alpha, double* y) {
  return gemv_t_f32(c->m, (int)c->n, (const float*)c->J, c->ldJ, x, alpha, y, c->partials, partial_cap(c),
                    c->xs, c->st);
}

dngd_status pcg_mixed(dngd_ctx* c, const double* b, double* x, int slot) {
  PcgMixed P;
  P.m = c->m;
  P.n = (int)c->n;
  P.J = (const float*)c->J;
  P.ldJ = c->ldJ;
  P.Linv = c->Linv;
  P.ldk = c->ldk;
  P.lambda = c->lambda;
  P.res = c->cg_res;
  P.z = c->cg_z;
  P.p = c->cg_p;
  P.Ap = c->cg_Ap;
  P.u = c->cg_u;
  P.y = c->cg_y;
  P.xs = c->xs;
  P.partials = c->partials;
  P.partial_cap = partial_cap(c);
  P.dotp = c->dot_partials + 256;
  P.scal = c->scal;
  P.scal_h = c->scal_h;
  P.ev = (c->timing && slot == 0) ? c->kev : nullptr;
  const double tol = c->desc.refine_tol > 0 ? c->desc.refine_tol : 1e-10;
  int maxit = c->desc.refine_max_it > 0 ? c->desc.refine_max_it : 200;
  if (c->async && c->async_it > 0 && c->async_it < maxit) maxit = c->async_it;
  if (oz_mode(c->prec)) {
    // the exact FP64 Gram is the operator: one m x m GEMV per iteration; the
    // synchronous solve is one persistent cooperative kernel
    P.K64 = c->K64;
    P.ldk64 = c->ldk;
    P.LinvT = c->LinvT;
    P.pstate = c->pstate;
    P.pwork = c->pwork;
    P.status = c->status;
  }
  if (!c->async) {
    if (!c->cap_st) DNGD_CUDA_CHECK(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
    P.chunk_exec = &c->pcg_chunk[slot];
    P.chunk_key = c->pcg_chunk_key[slot];
    P.cap = c->cap_st;
  }
  return pcg_mixed_solve(P, b, x, tol, maxit, 4, &c->iters[slot], &c->relres[slot], c->st, c->async, slot);
}

dngd_status pcg_matfree(dngd_ctx* c, const double* b, double* x, int slot);

dngd_status solve_last(dngd_ctx* c, const double* b, double* x, int slot) {
  if (c->pcg) return pcg_matfree(c, b, x, slot);
  if (c->prec == DNGD_FP64) {
    c->iters[slot] = 0;
    c->relres[slot] = 0.0;
    return chol_solve_f64_dinv(c->ms, (const double*)c->K, c->ldk, c->Dinv, b, x, c->tw, c->tw + c->ms, c->st);
  }
  return pcg_mixed(c, b, x, slot);
}

// ---------------------------------------------------------------------------
// The step
// ---------------------------------------------------------------------------

const Tc3Scratch* tc3p(dngd_ctx* c) { return c->tc3.buf ? &c->tc3 : nullptr; }

// Scratch for the largest TF32 tensor-core GEMM of the context: a jets layer
// (R x w x w; the f_vv sweep's three stacked streams 3R x w x w), a factor
// update (m x m x 64) or the top level of the recursive inverse
// (m/2 x m/2 x m/2).
size_t tc3_bytes(const dngd_ctx* c) {
  const int m = c->net.m, w = c->net.max_w;
  size_t b = tc3_scratch_bytes(trials_of(c->net) * c->net.R, w, w);   // line-search trials stacked by rows
  const size_t f = tc3_scratch_bytes(m, m, 64);
  const size_t t = tc3_scratch_bytes(m, 0, m / 2 + 64);
  if (f > b) b = f;
  if (t > b) b = t;
  return b;
}

// The low-precision Gram writes K + shift I (FP32 lower) for the factor: the
// tcgen05 BF16 / TF32 syrk, or the exact sliced Gram (which also writes the
// FP64 refinement operator).
void gram_set_shift(dngd_ctx* c, double shift) {
  if (c->oz) gram_oz_set_shift(c->oz, shift);
  else gram_tc_set_shift(c->gram, shift);
}
dngd_status gram_run(dngd_ctx* c, bool timed) {
  cudaEvent_t before = timed ? c->ev[9] : nullptr, after = timed ? c->ev[8] : nullptr;
  return c->oz ? gram_oz_run(c->oz, c->status, c->st, before, after)
               : gram_tc_run(c->gram, c->status, c->st, before, after);
}

template <typename T>
dngd_status step_T(dngd_ctx* c, const double* theta, const double* X, const double* target, dngd_step_info* info) {
  dngd_status s;
  const int m = c->m;
  const int n = (int)c->n;
  // c->phase: 0 the whole step; in a batch of exact-Gram instances, 1 up to
  // the factorisation and 2 from the factor's inverse on (the batch factors
  // every instance in between)
  if (c->phase != 2) {
    DNGD_CUDA_CHECK(cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->st));
    evrec(c, 0);
  }
  const T* thT = theta_in_T<T>(c, theta);
  if (c->phase != 2) {
    if ((s = residual_jacobian_T<T>(c, thT, X, target))) return s;
    if ((s = apply_lambda_rule(c))) return s;
    evrec(c, 1);
  }
  // K + lambda I (lower), or J^T J + lambda I in the primal space
  if (c->prec == DNGD_FP64) {
    const int ms = c->ms;
    if ((s = gram_f64(c->primal, ms, c->primal ? m : n, (const double*)c->J, c->ldJ, (double*)c->K, c->ldk,
                      c->gws, c->st)))
      return s;
    evrec(c, 8);
    if ((s = add_diag<double>(ms, (double*)c->K, c->ldk, c->lambda, c->st))) return s;
    if (c->Kcopy)
      DNGD_CUDA_CHECK(cudaMemcpyAsync(c->Kcopy, c->K, sizeof(double) * (size_t)ms * c->ldk,
                                      cudaMemcpyDeviceToDevice, c->st));
    evrec(c, 2);
    if ((s = cholesky<double>(ms, (double*)c->K, c->ldk, c->status, nullptr, c->st))) return s;
    if ((s = trtri_diag64(ms, (const double*)c->K, c->ldk, c->Dinv, c->st))) return s;
  } else if (c->ozf) {
    // exact Gram: FP64 factor of K + (lambda + mu) I with exact sliced
    // trailing updates (mu = 0 unless that fails at the Gram's own accuracy);
    // its FP32 rounding and inverse precondition PCG on the exact operator
    if (c->phase != 2) {
      double mu = c->mu_sticky > c->desc.shift_mu ? c->mu_sticky : c->desc.shift_mu;
      const double mu0 = mu;
      gram_set_shift(c, c->lambda + mu);
      if ((s = gram_run(c, c->timing))) return s;
      c->factor_attempts = 0;
      if (!c->async && (s = diag_sum<float>(m, (const float*)c->K, c->ldk, c->scal + S_TRACE, c->st))) return s;
      for (int attempt = 0;; ++attempt) {
        if (attempt > 0) {
          gram_set_shift(c, c->lambda + mu);
          if ((s = gram_oz_reduce(c->oz, c->st))) return s;
        }
        evrec(c, 2);
        c->factor_attempts++;
        if (c->phase == 1) {   // a batch factors all instances together
          c->shift_used = mu;
          return DNGD_OK;
        }
        if ((s = c->ozb ? oz_factor_batched_run(c->ozb, c->st) : oz_factor_run(c->ozf, c->status, c->st))) return s;
        if (c->async) break;   // a failure is reported by the status word
        const dngd_status fs = read_status(c);
        if (fs != DNGD_ERR_NOT_SPD || attempt >= 15) break;
        DNGD_CUDA_CHECK(cudaMemcpyAsync(c->scal_h, c->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, c->st));
        DNGD_CUDA_CHECK(cudaStreamSynchronize(c->st));
        const double tr = c->scal_h[S_TRACE] - m * (c->lambda + mu0);
        const double base = 1e-10 * (tr > 0 ? tr : 1.0) / m;
        mu = mu * 10.0 > base ? mu * 10.0 : base;
        DNGD_CUDA_CHECK(cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->st));
      }
      if (!c->async) c->mu_sticky = mu;
      c->shift_used = mu;
    }
    // the factor's inverse in FP64 from sliced products (its condition number
    // is the square root of K's, up to ~1e5 late in training, so an inverse
    // formed in FP32 arithmetic is off by far more than FP32 rounding), then
    // rounded to FP32: a relative perturbation of 2^-24 cond(L) of the ideal
    // preconditioner
    if ((s = trtri_diag64(m, c->Kd, c->ldk, c->Dinv, c->st))) return s;
    if ((s = oz_trtri(c->ozi, m, c->Kd, c->ldk, c->Dinv, (float*)c->K, c->Linv, c->LinvT, c->Li64, c->LiT64, c->ldk,
                      c->trtri_work, (double*)c->K0, c->status, c->st)))
      return s;
    if (c->async) goto factored;
  } else {
    // low-precision Gram + FP32 factor of K + (lambda + mu) I; a failed
    // factorisation is retried with a larger shift mu (it only preconditions
    // the refinement, whose operator keeps the exact lambda)
    double mu = c->mu_sticky > c->desc.shift_mu ? c->mu_sticky : c->desc.shift_mu;
    if (c->async) {
      // no host round trip: one factorisation with the shift of the last
      // synchronous step; a failure is reported by the status word
      gram_set_shift(c, c->lambda + mu);
      if ((s = gram_run(c, false))) return s;
      DNGD_CUDA_CHECK(cudaMemsetAsync(c->Linv, 0, sizeof(float) * (size_t)m * c->ldk, c->st));
      if ((s = cholesky_f32_inv(m, (float*)c->K, c->ldk, c->Linv, c->ldk, c->status, c->st, tc3p(c)))) return s;
      if ((s = trtri_offdiag_f32(m, (const float*)c->K, c->ldk, c->Linv, c->ldk, c->trtri_work, c->st, tc3p(c),
                                 c->status)))
        return s;
      c->shift_used = mu;
      c->factor_attempts = 1;
      goto factored;
    }
    gram_set_shift(c, c->lambda + mu);
    if ((s = gram_run(c, c->timing))) return s;
    // K0 = K + (lambda + mu0) I is kept, so a failed factorisation is retried
    // from the copy with a larger shift instead of recomputing the Gram
    DNGD_CUDA_CHECK(cudaMemcpyAsync(c->K0, c->K, sizeof(float) * (size_t)m * c->ldk, cudaMemcpyDeviceToDevice,
                                    c->st));
    if ((s = diag_sum<float>(m, (const float*)c->K, c->ldk, c->scal + S_TRACE, c->st))) return s;
    const double mu0 = mu;
    c->factor_attempts = 0;
    for (int attempt = 0;; ++attempt) {
      if (attempt > 0) {
        DNGD_CUDA_CHECK(cudaMemcpyAsync(c->K, c->K0, sizeof(float) * (size_t)m * c->ldk, cudaMemcpyDeviceToDevice,
                                        c->st));
        if ((s = add_diag<float>(m, (float*)c->K, c->ldk, mu - mu0, c->st))) return s;
      }
      evrec(c, 2);
      c->factor_attempts++;
      DNGD_CUDA_CHECK(cudaMemsetAsync(c->Linv, 0, sizeof(float) * (size_t)m * c->ldk, c->st));
      if ((s = cholesky_f32_inv(m, (float*)c->K, c->ldk, c->Linv, c->ldk, c->status, c->st, tc3p(c)))) return s;
      const dngd_status fs = read_status(c);
      if (fs != DNGD_ERR_NOT_SPD || attempt >= 15) break;
      DNGD_CUDA_CHECK(cudaMemcpyAsync(c->scal_h, c->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, c->st));
      DNGD_CUDA_CHECK(cudaStreamSynchronize(c->st));
      const double tr = c->scal_h[S_TRACE] - m * (c->lambda + mu0);
      const double base = 1e-6 * (tr > 0 ? tr : 1.0) / m;
      mu = mu * 3.0 > base ? mu * 3.0 : base;
      DNGD_CUDA_CHECK(cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->st));
    }
    if (c->Kcopy) {
      DNGD_CUDA_CHECK(cudaMemcpyAsync(c->Kcopy, c->K0, sizeof(float) * (size_t)m * c->ldk, cudaMemcpyDeviceToDevice,
                                      c->st));
      if ((s = add_diag<float>(m, (float*)c->Kcopy, c->ldk, mu - mu0, c->st))) return s;
    }
    c->mu_sticky = mu;
    c->shift_used = mu;
    if ((s = trtri_offdiag_f32(m, (const float*)c->K, c->ldk, c->Linv, c->ldk, c->trtri_work, c->st, tc3p(c),
                               c->status)))
      return s;
    // row-oriented access to Linv^T for the persistent solve
    if (c->LinvT && (s = transpose_f32(m, c->Linv, c->ldk, c->LinvT, c->ldk, c->st))) return s;
  }
  // a failed factorisation stops the (synchronous) step here
  if (!c->async && (s = read_status(c))) return s;
factored:
  evrec(c, 3);
  // alpha = (K + lambda I)^{-1} r ; v = -J^T alpha
  // (primal: v = (J^T J + lambda I)^{-1} (-J^T r))
  if (c->primal) {
    if ((s = jt_x<T>(c, c->r, -1.0, c->gp))) return s;
    if ((s = solve_last(c, c->gp, c->v, 0))) return s;
  } else {
    if ((s = solve_last(c, c->r, c->alpha, 0))) return s;
    if ((s = jt_x<T>(c, c->alpha, -1.0, c->v))) return s;
  }
  evrec(c, 4);
  if (c->desc.use_ga) {
    const T* vT;
    if (sizeof(T) == sizeof(double)) {
      vT = (const T*)c->v;
    } else {
      to_float(n, c->v, c->v32, c->st);
      vT = (const T*)c->v32;
    }
    if ((s = jets_fvv<T>(c->net, thT, vT, X, (T*)c->Z3, (T*)c->H3a, (T*)c->H3b, c->fvv, c->st, jets_tc<T>(c),
                         c->status)))
      return s;
    evrec(c, 5);
    if (c->primal) {
      if ((s = jt_x<T>(c, c->fvv, -1.0, c->gp))) return s;
      if ((s = solve_last(c, c->gp, c->a, 1))) return s;
    } else {
      if ((s = solve_last(c, c->fvv, c->beta, 1))) return s;
      if ((s = jt_x<T>(c, c->beta, -1.0, c->a))) return s;
    }
    evrec(c, 6);
  } else {
    evrec(c, 5);
    evrec(c, 6);
  }
  if ((s = ga_finish(n, c->v, c->a, c->desc.use_ga, c->desc.eps_norm,
                     c->desc.ga_ratio_max > 0 ? c->desc.ga_ratio_max : 0.5, c->delta, c->scal, c->dot_partials,
                     c->status, c->st)))
    return s;
  if ((s = dot_dev(m, c->r, c->r, c->scal + S_LOSS, c->dot_partials, c->st))) return s;
  evrec(c, 7);
  c->have_step = true;
  (void)info;
  return DNGD_OK;
}

// ---------------------------------------------------------------------------
// Matrix-free Nystrom-PCG step (Alg. PCGStep; push-through recovery)
// ---------------------------------------------------------------------------

dngd_status upload_landmarks(dngd_ctx* c) {
  const NetInfo& net = c->net;
  const int ell = (int)c->lm_host.size();
  std::vector<int> rows, row0(ell), S(ell);
  for (int j = 0; j < ell; ++j) {
    const int p = c->lm_host[j];
    const ClassInfo& ci = class_of(net, p);
    const int r = ci.row0 + (p - ci.p0) * ci.S;
    row0[j] = (int)rows.size();
    S[j] = ci.S;
    for (int t = 0; t < ci.S; ++t) rows.push_back(r + t);
  }
  if ((int)rows.size() > c->RI_max) return DNGD_ERR_INVALID_ARG;
  c->mf.RI = (int)rows.size();
  c->mf.ell = ell;
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->d_lm, c->lm_host.data(), sizeof(int) * ell, cudaMemcpyHostToDevice, c->st));
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->d_lrows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, c->st));
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->d_lrow0, row0.data(), sizeof(int) * ell, cudaMemcpyHostToDevice, c->st));
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->d_lS, S.data(), sizeof(int) * ell, cudaMemcpyHostToDevice, c->st));
  return DNGD_OK;
}

// PCG on (K + lambda I) x = b with the factor-form operator and the Nystrom
// preconditioner; host-driven loop (one synchronisation per iteration, small
// next to a kernel-vector product).
dngd_status pcg_matfree(dngd_ctx* c, const double* b, double* x, int slot) {
  const int m = c->m;
  double* sc = c->scal;
  const MatFree& F = c->mf;
  dngd_status s;
  const double tol = c->desc.pcg_tol > 0 ? c->desc.pcg_tol : 1e-6;
  const int maxit = c->desc.pcg_max_it > 0 ? c->desc.pcg_max_it : 500;
  DNGD_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * m, c->st));
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->cg_res, b, sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st));
  DNGD_CUDA_CHECK(cudaMemsetAsync(sc + S_BREAK, 0, sizeof(double), c->st));
  if ((s = dot_dev(m, b, b, sc + S_BB, c->dot_partials, c->st))) return s;
  if ((s = mf_precond(F, c->lambda, c->cg_res, c->cg_z, c->st))) return s;
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->cg_p, c->cg_z, sizeof(double) * m, cudaMemcpyDeviceToDevice, c->st));
  if ((s = dot_dev(m, c->cg_res, c->cg_z, sc + S_RHO, c->dot_partials, c->st))) return s;
  int it = 0;
  double rel = 1.0;
  for (it = 0; it < maxit;) {
    if ((s = mf_kvp(F, c->cg_p, c->lambda, c->cg_Ap, c->st))) return s;
    if ((s = dot_dev(m, c->cg_p, c->cg_Ap, sc + S_PAP, c->dot_partials, c->st))) return s;
    if ((s = cg_alpha(sc, c->st))) return s;
    if ((s = cg_update_x(m, sc, x, c->cg_res, c->cg_p, c->cg_Ap, c->st))) return s;
    if ((s = dot_dev(m, c->cg_res, c->cg_res, sc + S_RR, c->dot_partials, c->st))) return s;
    ++it;
    DNGD_CUDA_CHECK(cudaMemcpyAsync(c->scal_h, sc, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, c->st));
    DNGD_CUDA_CHECK(cudaStreamSynchronize(c->st));
    const double bb = c->scal_h[S_BB];
    rel = bb > 0 ? sqrt(c->scal_h[S_RR] / bb) : 0.0;
    if (rel <= tol || bb == 0.0 || c->scal_h[S_BREAK] != 0.0) break;
    if ((s = mf_precond(F, c->lambda, c->cg_res, c->cg_z, c->st))) return s;
    if ((s = dot_dev(m, c->cg_res, c->cg_z, sc + S_RHONEW, c->dot_partials, c->st))) return s;
    if ((s = cg_beta(sc, c->st))) return s;
    if ((s = cg_update_p(m, sc, c->cg_z, c->cg_p, c->st))) return s;
  }
  c->iters[slot] = it;
  c->relres[slot] = rel;
  return DNGD_OK;
}

dngd_status step_pcg(dngd_ctx* c, const double* theta, const double* X, const double* target) {
  dngd_status s;
  const int m = c->m;
  const long long n = c->n;
  DNGD_CUDA_CHECK(cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->st));
  evrec(c, 0);
  const float* th = theta_in_T<float>(c, theta);
  // jets: r, stream activations H and adjoints D (J is not formed); their
  // layer GEMMs on the TF32 tensor cores
  if ((s = jets_forward<float>(c->net, th, X, target, lp<float>(c->Z), lp<float>(c->H), c->r, c->status, c->st,
                               tc3p(c), true)))
    return s;
  if ((s = jets_backward_jacobian<float, float>(c->net, th, X, lp<float>(c->Z), lp<float>(c->H), lp<float>(c->D),
                                                (float*)c->Hbar, (float*)nullptr, 0, nullptr, 0, c->st, tc3p(c),
                                                c->status)))
    return s;
  if ((s = apply_lambda_rule(c))) return s;
  evrec(c, 1);
  c->mf.X = X;
  if ((s = mf_input_rows(c->mf, c->st))) return s;
  if ((s = mf_kci(c->mf, c->st))) return s;
  evrec(c, 8);
  // Nystrom factors; K_II + nu I is shifted up only if it does not factor
  double nu = c->nu_sticky;
  for (int attempt = 0;; ++attempt) {
    evrec(c, 2);
    if ((s = mf_nystrom(c->mf, c->lambda, nu, c->status, c->st))) return s;
    const dngd_status fs = read_status(c);
    if (fs != DNGD_ERR_NOT_SPD || attempt >= 15) break;
    if ((s = mf_kii_trace(c->mf, c->scal + S_TRACE, c->st))) return s;
    DNGD_CUDA_CHECK(cudaMemcpyAsync(c->scal_h, c->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, c->st));
    DNGD_CUDA_CHECK(cudaStreamSynchronize(c->st));
    const double base = 1e-7 * (c->scal_h[S_TRACE] > 0 ? c->scal_h[S_TRACE] : 1.0) / c->mf.ell;
    nu = nu * 3.0 > base ? nu * 3.0 : base;
    DNGD_CUDA_CHECK(cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->st));
  }
  c->nu_sticky = nu;
  c->nu_used = nu;
  if ((s = read_status(c))) return s;
  evrec(c, 3);
  if ((s = pcg_matfree(c, c->r, c->alpha, 0))) return s;
  if ((s = mf_jtv(c->mf, c->alpha, c->mf.g32, c->st))) return s;
  if ((s = mf_g_to_double(n, c->mf.g32, -1.0, c->v, c->st))) return s;
  evrec(c, 4);
  if (c->desc.use_ga) {
    to_float(n, c->v, c->v32, c->st);
    if ((s = jets_fvv<float>(c->net, th, c->v32, X, (float*)c->Z3, (float*)c->H3a, (float*)c->H3b, c->fvv, c->st,
                             tc3p(c), c->status)))
      return s;
    evrec(c, 5);
    if ((s = pcg_matfree(c, c->fvv, c->beta, 1))) return s;
    if ((s = mf_jtv(c->mf, c->beta, c->mf.g32, c->st))) return s;
    if ((s = mf_g_to_double(n, c->mf.g32, -1.0, c->a, c->st))) return s;
    evrec(c, 6);
  } else {
    evrec(c, 5);
    evrec(c, 6);
  }
  if ((s = ga_finish((int)n, c->v, c->a, c->desc.use_ga, c->desc.eps_norm,
                     c->desc.ga_ratio_max > 0 ? c->desc.ga_ratio_max : 0.5, c->delta, c->scal, c->dot_partials,
                     c->status, c->st)))
    return s;
  if ((s = dot_dev(m, c->r, c->r, c->scal + S_LOSS, c->dot_partials, c->st))) return s;
  evrec(c, 7);
  c->have_step = true;
  return DNGD_OK;
}

dngd_status alloc_pcg(dngd_ctx* c, bool dry, size_t* bytes_out) {
  const NetInfo& net = c->net;
  const int m = net.m;
  const long long n = net.n;
  const int L = net.n_layers - 1;
  const int ell = c->desc.pcg_rank > 0 ? (c->desc.pcg_rank < m ? c->desc.pcg_rank : m) : (m < 512 ? m : 512);
  int Smax = 1;
  for (int k = 0; k < net.n_classes; ++k) Smax = net.cls[k].S > Smax ? net.cls[k].S : Smax;
  c->RI_max = ell * Smax;
  const int RI = c->RI_max;
  const int wl = net.widths[L];
  const int wmax = net.max_w > net.d_in ? net.max_w : net.d_in;
  size_t tot = 0;
  auto add = [&](size_t b) { tot += (b + 255) & ~(size_t)255; };
  const size_t rb = (size_t)net.R * wmax;
  add(8 * (3 * n + (size_t)m * net.d_in + 2 * m));          // staging
  add(4 * 2 * n);                                            // theta32, v32
  for (int l = 0; l < L; ++l) add(4 * 3 * (size_t)net.R * net.widths[l + 1]);
  add(4 * rb * 10);                                          // Hbar, Z3, H3a, H3b
  add(4 * ((size_t)net.R + n + rb + (size_t)net.R * net.d_in));  // vrow, g32, Y, Hin
  add(4 * 2 * (size_t)RI * wmax + 4 * 2 * (size_t)net.R * RI); // DI, HI, P, Q
  add(4 * ((size_t)m * ell + (size_t)m * wl + (size_t)ell * wl + m));
  add(4 * (4 * (size_t)ell * ell + (size_t)m * ell + (size_t)ell * ell));
  add(8 * ((size_t)m * 12 + 3 * n + 16 * (size_t)(n > m ? n : m)));
  // split operands of the 3xTF32 GEMMs: the jets' layers (R x w x w), J u
  // (R x w_out x w_in), the landmark columns (R x RI x w) and J^T v (w_out x
  // w_in x R)
  size_t t3 = tc3_scratch_bytes(net.R, net.max_w, net.max_w);
  const size_t t3b = tc3_scratch_bytes(net.R, RI, wmax);
  const size_t t3c = tc3_scratch_bytes(3 * net.R, net.max_w, net.max_w);   // the f_vv sweep's stacked streams
  const size_t t3d = tc3_scratch_bytes(net.max_w, net.max_w, net.R);
  t3 = t3 > t3b ? t3 : t3b;
  t3 = t3 > t3c ? t3 : t3c;
  t3 = t3 > t3d ? t3 : t3d;
  add(t3);
  if (bytes_out) *bytes_out = tot;
  if (dry) return DNGD_OK;
  dngd_status s;
#define A_(p, T, cnt) \
  if ((s = dalloc<T>(c, (T**)&(p), (cnt)))) return s;
  c->tc3.bytes = t3;
  A_(c->tc3.buf, float, t3 / sizeof(float));
  A_(c->theta_s, double, n);
  A_(c->X_s, double, (size_t)m * net.d_in);
  A_(c->target_s, double, m);
  A_(c->nvec_s, double, n);
  A_(c->mvec_s, double, m);
  A_(c->theta_tmp, double, n);
  A_(c->theta32, float, n);
  A_(c->v32, float, n);
  for (int l = 0; l < L; ++l) {
    const size_t cnt = (size_t)net.R * net.widths[l + 1];
    A_(c->Z[l], float, cnt);
    A_(c->H[l], float, cnt);
    A_(c->D[l], float, cnt);
  }
  A_(c->Hbar, float, rb);
  A_(c->Z3, float, 3 * rb);
  A_(c->H3a, float, 3 * rb);
  A_(c->H3b, float, 3 * rb);
  MatFree& F = c->mf;
  F.net = &c->net;
  for (int l = 0; l < kMaxLayers; ++l) {
    F.H.p[l] = (float*)c->H[l];
    F.D.p[l] = (float*)c->D[l];
  }
  A_(F.vrow, float, net.R);
  A_(F.g32, float, n);
  A_(F.Y, float, rb);
  A_(F.Hin, float, (size_t)net.R * net.d_in);
  A_(F.DI, float, (size_t)RI * wmax);
  A_(F.HI, float, (size_t)RI * wmax);
  A_(F.P, float, (size_t)net.R * RI);
  A_(F.Q, float, (size_t)net.R * RI);
  A_(F.KCI, float, (size_t)m * ell);
  A_(F.Fo, float, (size_t)m * wl);
  A_(F.FoI, float, (size_t)ell * wl);
  A_(F.fb, float, m);
  A_(F.KII, float, (size_t)ell * ell);
  A_(F.LIIinv, float, (size_t)ell * ell);
  A_(F.C, float, (size_t)ell * ell);
  A_(F.LCinv, float, (size_t)ell * ell);
  A_(F.work, float, (size_t)ell * ell);
  A_(F.M, float, (size_t)m * ell);
  A_(F.t1, double, ell > m ? ell : m);
  A_(F.t2, double, ell > m ? ell : m);
  A_(F.t3, double, m);
  A_(c->d_lm, int, ell);
  A_(c->d_lrows, int, RI);
  A_(c->d_lrow0, int, ell);
  A_(c->d_lS, int, ell);
  F.lm = c->d_lm;
  F.lrows = c->d_lrows;
  F.lrow0 = c->d_lrow0;
  F.lS = c->d_lS;
  A_(c->r, double, m);
  A_(c->alpha, double, m);
  A_(c->fvv, double, m);
  A_(c->beta, double, m);
  A_(c->v, double, n);
  A_(c->a, double, n);
  A_(c->delta, double, n);
  A_(c->cg_res, double, m);
  A_(c->cg_z, double, m);
  A_(c->cg_p, double, m);
  A_(c->cg_Ap, double, m);
  A_(c->cg_y, double, m);
  A_(c->xsol, double, m);
  A_(c->cg_u, double, n);
  A_(c->partials, double, (size_t)16 * (n > m ? n : m));
  A_(c->dot_partials, double, 256 + 1024 + (size_t)m / 4 + 64);
  A_(c->xs, float2, (size_t)round_up(n > m ? n : m, 4) + 4);
  A_(c->scal, double, S_COUNT);
  A_(c->status, int, 4);
#undef A_
  F.xs = c->xs;
  F.partials = c->partials;
  F.partial_cap = 16LL * (n > m ? n : m);
  // the factor-form operator's GEMMs: 3xTF32 tensor cores, or compensated
  // FP32 SIMT (null)
  F.tc3 = c->desc.pcg_operator == DNGD_PCG_OP_COMPENSATED ? nullptr : &c->tc3;
  F.status = c->status;
  DNGD_CUDA_CHECK(cudaMemsetAsync(c->a, 0, sizeof(double) * n, c->st));
  DNGD_CUDA_CHECK(cudaMemsetAsync(c->scal, 0, sizeof(double) * S_COUNT, c->st));
  DNGD_CUDA_CHECK(cudaMemsetAsync(c->status, 0, sizeof(int) * 4, c->st));
  DNGD_CUDA_CHECK(cudaMallocHost(&c->scal_h, sizeof(double) * S_COUNT));
  DNGD_CUDA_CHECK(cudaMallocHost(&c->status_h, sizeof(int) * 4));
  for (int i = 0; i < 10; ++i) DNGD_CUDA_CHECK(cudaEventCreate(&c->ev[i]));
  for (int i = 0; i < 4; ++i) DNGD_CUDA_CHECK(cudaEventCreate(&c->kev[i]));
  // default landmarks: evenly spaced residual indices
  c->lm_host.resize(ell);
  for (int j = 0; j < ell; ++j) c->lm_host[j] = (int)(((long long)j * m) / ell);
  return upload_landmarks(c);
}

dngd_status status_from_host(const int* h) {
  const int s = h[0];
  if (s & ST_TIMEOUT) return DNGD_ERR_TIMEOUT;
  if (s & ST_NOT_SPD) return DNGD_ERR_NOT_SPD;
  if (s & ST_NONFINITE) return DNGD_ERR_NONFINITE;
  if (s & ST_NO_CONVERGE) return DNGD_ERR_NO_CONVERGE;
  return DNGD_OK;
}

void info_from_host(dngd_ctx* c, dngd_step_info* info);

// Fill info after an asynchronous step whose graph copied scal/status to the
// pinned host buffers (the stream must have been synchronised).
// A captured solve that stopped at async_it (below the full budget) above
// the refinement tolerance.
bool async_capped(const dngd_ctx* c) {
  if (c->pcg || c->prec == DNGD_FP64 || c->async_it <= 0) return false;
  const int maxit = c->desc.refine_max_it > 0 ? c->desc.refine_max_it : 200;
  const double tol = c->desc.refine_tol > 0 ? c->desc.refine_tol : 1e-10;
  if (c->async_it >= maxit) return false;
  return c->relres[0] > tol || c->relres[1] > tol;
}

dngd_status finish_async(dngd_ctx* c, dngd_step_info* info) {
  const double* h = c->scal_h;
  for (int k = 0; k < 2; ++k) {
    const int rec = k == 0 ? S_IT0 : S_IT1;
    c->iters[k] = (int)h[rec];
    c->relres[k] = h[rec + 2] > 0 ? sqrt(h[rec + 1] / h[rec + 2]) : 0.0;
  }
  if (info) info_from_host(c, info);
  return status_from_host(c->status_h);
}

dngd_status fill_info(dngd_ctx* c, dngd_step_info* info) {
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->scal_h, c->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, c->st));
  dngd_status s = read_status(c);
  if (!info) return s;
  info_from_host(c, info);
  return s;
}

void info_from_host(dngd_ctx* c, dngd_step_info* info) {
  memset(info, 0, sizeof(*info));
  info->loss = 0.5 * c->scal_h[S_LOSS];
  info->norm_v = sqrt(c->scal_h[S_NV2]);
  info->norm_a = sqrt(c->scal_h[S_NA2]);
  info->ga_ratio = c->scal_h[S_RATIO];
  info->ga_accepted = c->scal_h[S_ACCEPT] != 0.0;
  info->solve_iters[0] = c->iters[0];
  info->solve_iters[1] = c->iters[1];
  info->solve_relres[0] = c->relres[0];
  info->solve_relres[1] = c->relres[1];
  info->device_status = c->status_h[0];
  info->not_spd_column = (c->status_h[0] & ST_NOT_SPD) ? c->status_h[1] : -1;
  info->shift_used = c->pcg ? c->nu_used : c->shift_used;
  info->factor_attempts = c->factor_attempts;
  info->lambda_used = c->lambda;
  if (c->timing) {
    // event order: 0 start, 1 jets+J, 8 Gram kernel, 2 Gram epilogue, 3 factor,
    // 4 solve r, 5 f_vv, 6 solve f_vv, 7 end
    const int a[7] = {0, 1, 8, 3, 4, 5, 6}, b[7] = {1, 8, 3, 4, 5, 6, 7};
    for (int i = 0; i < 7; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->ev[a[i]], c->ev[b[i]]);
      info->phase_ms[i] = ms;
    }
    float tot = 0.f;
    cudaEventElapsedTime(&tot, c->ev[0], c->ev[7]);
    info->phase_ms[7] = tot;
    if (c->prec != DNGD_FP64 && !c->pcg) cudaEventElapsedTime(&info->gram_kernel_ms, c->ev[9], c->ev[8]);
    if (!c->pcg && c->prec != DNGD_FP64 && c->iters[0] > 0) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, c->kev[0], c->kev[1]);
      cudaEventElapsedTime(&b, c->kev[1], c->kev[2]);
      info->jt_ms = a;
      info->j_ms = b;
    }
    cudaGetLastError();  // an unrecorded event only leaves a timing field at 0
  }
}

dngd_status alloc_workspace(dngd_ctx* c, bool dry, size_t* bytes_out) {
  const NetInfo& net = c->net;
  const int m = net.m;
  const long long n = net.n;
  const int L = net.n_layers - 1;
  const bool f64 = c->prec == DNGD_FP64;          // FP64 Gram, factor and solves
  const bool j64 = jets64(c->prec);                // FP64 jets and Jacobian
  const size_t es = j64 ? sizeof(double) : sizeof(float);     // jets / J elements
  const size_t ek = f64 ? sizeof(double) : sizeof(float);     // K elements
  size_t tot = 0;
  auto add = [&](size_t b) { tot += (b + 255) & ~(size_t)255; };
  c->ldJ = f64 ? n : round_up(n, 64);
  c->ldb = round_up(n, 64);
  const int ms = c->primal ? (int)n : m;          // FP64 system dimension
  c->ms = ms;
  c->ldk = round_up(f64 ? ms : m, 4);
  const bool oz = oz_mode(c->prec);
  const int ng = c->prec == DNGD_MIXED_OZ64 ? 6 : 5;   // exact-Gram levels kept
  const bool bf = c->prec == DNGD_MIXED_BF16;
  add(sizeof(double) * n);        // theta_s
  add(sizeof(double) * m * net.d_in);
  add(sizeof(double) * m);        // target_s
  add(sizeof(double) * n);        // nvec_s
  add(sizeof(double) * m);        // mvec_s
  add(sizeof(double) * n);        // theta_tmp
  if (!f64) {
    add(sizeof(float) * n);
    add(sizeof(float) * n);
  }
  for (int l = 0; l < L; ++l) {
    const size_t b = es * (size_t)net.R * net.widths[l + 1];
    add(b);
    add(b);
    add(b);
  }
  const size_t rowbuf = es * (size_t)net.R * net.max_w;
  add(rowbuf);            // Hbar
  add(3 * rowbuf);        // Z3
  add(3 * rowbuf);        // H3a
  add(3 * rowbuf);        // H3b
  add(es * (size_t)m * c->ldJ);
  if (bf) add(sizeof(__nv_bfloat16) * (size_t)m * c->ldb);
  const int mk = f64 ? ms : m;    // rows of K
  add(ek * (size_t)mk * c->ldk);
  if (c->desc.keep_gram) add(ek * (size_t)mk * c->ldk);
  if (f64) add(sizeof(double) * ((size_t)cdiv(ms, 64) * 64 * 64 + 2 * (size_t)ms));   // Dinv, tw
  if (c->primal) add(sizeof(double) * n);                                              // gp
  const int gsplit = f64 ? gram_f64_splits(ms, c->primal ? m : (int)n) : 1;
  if (gsplit > 1) add(sizeof(double) * gsplit * (size_t)ms * c->ldk);                   // gws
  if (!f64) {
    add(ek * (size_t)m * c->ldk);                 // K0
    add(sizeof(float) * (size_t)m * c->ldk);      // Linv
    add(sizeof(float) * (size_t)m * m);           // trtri work
    add(tc3_bytes(c));                            // TF32 tensor-core GEMM splits
    add(sizeof(float) * trials_of(net) * n);      // line-search trial parameters
    add(sizeof(double) * trials_of(net) * m);     // line-search trial residuals
    add(2 * sizeof(float) * trials_of(net) * (size_t)net.R * net.max_w);   // their activations
    if (oz) {
      add(sizeof(float2) * (size_t)m * c->ldk);   // K64
      add(sizeof(float) * (size_t)m * c->ldk);    // LinvT
      add(256);                                   // persistent-PCG barrier state
      add(sizeof(double) * 7 * (size_t)m);        // persistent-PCG vectors
      add(gram_oz_slice_bytes(m, (int)n));
      add(gram_oz_partial_bytes(m, (int)n, ng));
      add(sizeof(double) * (size_t)m * c->ldk);                                  // Kd
      add(sizeof(double) * (size_t)cdiv(m, 64) * 64 * 64);                       // Dinv
      add(oz_factor_bytes(m));
      add(oz_gemm_bytes(m, m, m));                                               // inverse's GEMMs
      add(2 * sizeof(double) * (size_t)m * c->ldk);                              // Li64, LiT64
      if (j64) add(oz_gemm_bytes(3 * net.R, net.max_w, net.max_w));              // FP64 jets' GEMMs
    } else {
      add(gram_tc_partial_bytes(m, (int)n));
    }
  }
  add(sizeof(double) * m * 4 + sizeof(double) * n * 3);
  add(sizeof(double) * m * 6 + sizeof(double) * n);
  add(sizeof(double) * (size_t)16 * (n > m ? n : m));
  add(sizeof(double) * (256 + 1024 + (size_t)m / 4 + 64) + sizeof(double) * S_COUNT + 16);
  add(sizeof(float2) * ((size_t)round_up(n > m ? n : m, 4) + 4));
  if (bytes_out) *bytes_out = tot;
  if (dry) return DNGD_OK;

  dngd_status s;
#define A_(p, T, cnt) \
  if ((s = dalloc<T>(c, (T**)&(p), (cnt)))) return s;
  A_(c->theta_s, double, n);
  A_(c->X_s, double, (size_t)m * net.d_in);
  A_(c->target_s, double, m);
  A_(c->nvec_s, double, n);
  A_(c->mvec_s, double, m);
  A_(c->theta_tmp, double, n);
  if (!f64) {
    A_(c->theta32, float, n);
    A_(c->v32, float, n);
  }
  for (int l = 0; l < L; ++l) {
    const size_t cnt = (size_t)net.R * net.widths[l + 1];
    if (j64) {
      A_(c->Z[l], double, cnt);
      A_(c->H[l], double, cnt);
      A_(c->D[l], double, cnt);
    } else {
      A_(c->Z[l], float, cnt);
      A_(c->H[l], float, cnt);
      A_(c->D[l], float, cnt);
    }
  }
  const size_t rb = (size_t)net.R * net.max_w;
  if (j64) {
    A_(c->Hbar, double, rb);
    A_(c->Z3, double, 3 * rb);
    A_(c->H3a, double, 3 * rb);
    A_(c->H3b, double, 3 * rb);
    A_(c->J, double, (size_t)m * c->ldJ);
    // the exact-Gram slicing reads whole padded rows: the pad stays zero
    if (!f64) DNGD_CUDA_CHECK(cudaMemsetAsync(c->J, 0, sizeof(double) * (size_t)m * c->ldJ, c->st));
  } else {
    A_(c->Hbar, float, rb);
    A_(c->Z3, float, 3 * rb);
    A_(c->H3a, float, 3 * rb);
    A_(c->H3b, float, 3 * rb);
    A_(c->J, float, (size_t)m * c->ldJ);
    DNGD_CUDA_CHECK(cudaMemsetAsync(c->J, 0, sizeof(float) * (size_t)m * c->ldJ, c->st));
  }
  if (f64) {
    A_(c->K, double, (size_t)ms * c->ldk);
    if (c->desc.keep_gram) A_(c->Kcopy, double, (size_t)ms * c->ldk);
    A_(c->Dinv, double, (size_t)cdiv(ms, 64) * 64 * 64);
    A_(c->tw, double, 2 * (size_t)ms);
    if (c->primal) A_(c->gp, double, n);
    if (gsplit > 1) A_(c->gws, double, gsplit * (size_t)ms * c->ldk);
  } else {
    if (bf) {
      A_(c->Jb, __nv_bfloat16, (size_t)m * c->ldb);
      DNGD_CUDA_CHECK(cudaMemsetAsync(c->Jb, 0, sizeof(__nv_bfloat16) * (size_t)m * c->ldb, c->st));
    }
    A_(c->K, float, (size_t)m * c->ldk);
    A_(c->K0, float, (size_t)m * c->ldk);
    if (c->desc.keep_gram) A_(c->Kcopy, float, (size_t)m * c->ldk);
    A_(c->Linv, float, (size_t)m * c->ldk);
    A_(c->trtri_work, float, (size_t)m * m);
    c->tc3.bytes = tc3_bytes(c);
    A_(c->tc3.buf, float, c->tc3.bytes / sizeof(float));
    c->ls_G = trials_of(net);
    A_(c->ls_th32, float, c->ls_G * n);
    A_(c->ls_r, double, c->ls_G * m);
    A_(c->ls_Z, float, c->ls_G * (size_t)net.R * net.max_w);
    A_(c->ls_H, float, c->ls_G * (size_t)net.R * net.max_w);
    if (oz) {
      A_(c->K64, float2, (size_t)m * c->ldk);
      A_(c->LinvT, float, (size_t)m * c->ldk);
      A_(c->pstate, unsigned char, 256);
      A_(c->pwork, double, 7 * (size_t)m);
      A_(c->oz_slices, unsigned char, gram_oz_slice_bytes(m, (int)n));
      c->gram_partial_bytes = gram_oz_partial_bytes(m, (int)n, ng);
      A_(c->oz_partials, double, c->gram_partial_bytes / sizeof(double));
      A_(c->Kd, double, (size_t)m * c->ldk);
      A_(c->Dinv, double, (size_t)cdiv(m, 64) * 64 * 64);
      A_(c->ozf_work, unsigned char, oz_factor_bytes(m));
      A_(c->ozi_work, unsigned char, oz_gemm_bytes(m, m, m));
      A_(c->Li64, double, (size_t)m * c->ldk);
      A_(c->LiT64, double, (size_t)m * c->ldk);
      if (j64) A_(c->ozg_work, unsigned char, oz_gemm_bytes(3 * net.R, net.max_w, net.max_w));
    } else {
      c->gram_partial_bytes = gram_tc_partial_bytes(m, (int)n);
      A_(c->gram_partials, float, c->gram_partial_bytes / sizeof(float));
    }
  }
  A_(c->r, double, m);
  A_(c->alpha, double, m);
  A_(c->fvv, double, m);
  A_(c->beta, double, m);
  A_(c->v, double, n);
  A_(c->a, double, n);
  A_(c->delta, double, n);
  A_(c->cg_res, double, m);
  A_(c->cg_z, double, m);
  A_(c->cg_p, double, m);
  A_(c->cg_Ap, double, m);
  A_(c->cg_y, double, m);
  A_(c->xsol, double, m);
  A_(c->cg_u, double, n);
  A_(c->partials, double, (size_t)16 * (n > m ? n : m));
  A_(c->dot_partials, double, 256 + 1024 + (size_t)m / 4 + 64);
  A_(c->xs, float2, (size_t)round_up(n > m ? n : m, 4) + 4);
  A_(c->scal, double, S_COUNT);
  A_(c->status, int, 4);
#undef A_
  DNGD_CUDA_CHECK(cudaMemsetAsync(c->a, 0, sizeof(double) * n, c->st));
  DNGD_CUDA_CHECK(cudaMemsetAsync(c->scal, 0, sizeof(double) * S_COUNT, c->st));
  DNGD_CUDA_CHECK(cudaMemsetAsync(c->status, 0, sizeof(int) * 4, c->st));
  DNGD_CUDA_CHECK(cudaMallocHost(&c->scal_h, sizeof(double) * S_COUNT));
  DNGD_CUDA_CHECK(cudaMallocHost(&c->status_h, sizeof(int) * 4));
  if (oz) {
    s = gram_oz_plan(&c->oz, c->J, j64, ng, c->ldJ, m, (int)n, c->oz_slices, (float*)c->K, c->ldk, c->K64, c->ldk,
                     c->oz_partials, c->gram_partial_bytes, c->st);
    if (s) return s;
    gram_oz_set_fp64_out(c->oz, c->Kd);
    if ((s = oz_factor_plan(&c->ozf, m, c->Kd, c->ldk, c->ozf_work, c->st))) return s;
    if (c->desc.factor_update == DNGD_FACTOR_DF) {
      OzFactor* f1[1] = {c->ozf};
      int* s1[1] = {c->status};
      if ((s = oz_factor_batched_plan(&c->ozb, 1, f1, s1, c->st))) return s;
    }
    if ((s = oz_gemm_plan(&c->ozi, m, m, m, c->ozi_work))) return s;
    if (c->ozg_work) {
      if ((s = oz_gemm_plan(&c->ozg, 3 * net.R, net.max_w, net.max_w, c->ozg_work))) return s;
      c->ozs.ozg = c->ozg;
    }
  } else if (!f64) {
    const void* Jlow = bf ? (const void*)c->Jb : (const void*)c->J;
    const long long ld = bf ? c->ldb : c->ldJ;
    s = gram_tc_plan(&c->gram, bf ? 0 : 1, Jlow, m, (int)n, ld, (float*)c->K, c->ldk, c->gram_partials,
                     c->gram_partial_bytes, c->st);
    if (s) return s;
  }
  for (int i = 0; i < 10; ++i) DNGD_CUDA_CHECK(cudaEventCreate(&c->ev[i]));
  for (int i = 0; i < 4; ++i) DNGD_CUDA_CHECK(cudaEventCreate(&c->kev[i]));
  return DNGD_OK;
}

void free_ctx(dngd_ctx* c) {
  for (int i = 0; i < 2; ++i)
    if (c->pcg_chunk[i]) cudaGraphExecDestroy(c->pcg_chunk[i]);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  if (c->ls_host) cudaFreeHost(c->ls_host);
  if (c->loss_host) cudaFreeHost(c->loss_host);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->gst) cudaStreamDestroy(c->gst);
  for (int i = 0; i < 2; ++i)
    if (c->gev[i]) cudaEventDestroy(c->gev[i]);
  for (void* p : c->allocs) cudaFree(p);
  if (c->scal_h) cudaFreeHost(c->scal_h);
  if (c->status_h) cudaFreeHost(c->status_h);
  if (c->gram) gram_tc_free(c->gram);
  if (c->oz) gram_oz_free(c->oz);
  if (c->ozb) oz_factor_batched_free(c->ozb);
  if (c->ozf) oz_factor_free(c->ozf);
  if (c->ozg) oz_gemm_free(c->ozg);
  if (c->ozi) oz_gemm_free(c->ozi);
  for (int i = 0; i < 10; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  for (int i = 0; i < 4; ++i)
    if (c->kev[i]) cudaEventDestroy(c->kev[i]);
  delete c;
}

dngd_status out_copy(dngd_ctx* c, double* dst, const double* src, size_t count) {
  if (dst == src) return DNGD_OK;
  DNGD_CUDA_CHECK(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, c->st));
  if (!is_device_ptr(dst)) DNGD_CUDA_CHECK(cudaStreamSynchronize(c->st));
  return DNGD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Exported C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char* dngd_status_string(dngd_status s) {
  switch (s) {
    case DNGD_OK: return "ok";
    case DNGD_ERR_INVALID_ARG: return "invalid argument";
    case DNGD_ERR_NOT_SPD: return "matrix not positive definite";
    case DNGD_ERR_NO_CONVERGE: return "iteration did not converge";
    case DNGD_ERR_NONFINITE: return "non-finite value";
    case DNGD_ERR_BUDGET: return "memory budget exceeded";
    case DNGD_ERR_TIMEOUT: return "device wait timed out";
    case DNGD_ERR_CUDA: return "CUDA error";
    case DNGD_ERR_STATE: return "call out of order";
    case DNGD_ERR_OOM: return "out of device memory";
    default: return "unknown status";
  }
}

const char* dngd_version(void) { return kVersion; }

uint64_t dngd_launch_count(void) { return dngd::g_launches.load(std::memory_order_relaxed); }

int64_t dngd_num_params(const dngd_problem_desc* desc) {
  NetInfo net;
  if (!desc || build_net(desc, &net)) return -1;
  return net.n;
}

dngd_status dngd_workspace_bytes(const dngd_problem_desc* desc, size_t* bytes) {
  if (!desc || !bytes) return DNGD_ERR_INVALID_ARG;
  dngd_ctx tmp;
  tmp.desc = *desc;
  dngd_status s = build_net(desc, &tmp.net);
  if (s) return s;
  tmp.prec = desc->precision;
  const int sp = resolve_space(desc, tmp.net);
  if (sp < 0) return DNGD_ERR_INVALID_ARG;
  tmp.primal = sp == 1;
  if (desc->solver == DNGD_PCG) return alloc_pcg(&tmp, true, bytes);
  return alloc_workspace(&tmp, true, bytes);
}

dngd_status dngd_create(dngd_ctx** out, const dngd_problem_desc* desc, void* stream) {
  if (!out || !desc) return DNGD_ERR_INVALID_ARG;
  *out = nullptr;
  if (desc->precision < DNGD_FP64 || desc->precision > DNGD_MIXED_OZ64) return DNGD_ERR_INVALID_ARG;
  if (desc->solver != DNGD_DENSE && desc->solver != DNGD_PCG) return DNGD_ERR_INVALID_ARG;
  if (desc->solver == DNGD_PCG && jets64(desc->precision)) return DNGD_ERR_INVALID_ARG;
  if (!lambda_ok(desc->precision, desc->lambda) || !(desc->lambda_cap >= 0.0) || !isfinite(desc->lambda_cap))
    return DNGD_ERR_INVALID_ARG;
  if (desc->pcg_operator != DNGD_PCG_OP_TC3 && desc->pcg_operator != DNGD_PCG_OP_COMPENSATED)
    return DNGD_ERR_INVALID_ARG;
  if (desc->factor_update != DNGD_FACTOR_SLICED && desc->factor_update != DNGD_FACTOR_DF)
    return DNGD_ERR_INVALID_ARG;
  if (desc->solve_space < DNGD_SPACE_DUAL || desc->solve_space > DNGD_SPACE_AUTO ||
      (desc->solve_space == DNGD_SPACE_PRIMAL && (desc->precision != DNGD_FP64 || desc->solver != DNGD_DENSE)))
    return DNGD_ERR_INVALID_ARG;
  gemv_init();
  dngd_ctx* c = new dngd_ctx();
  c->desc = *desc;
  dngd_status s = build_net(desc, &c->net);
  if (s) {
    delete c;
    return s;
  }
  c->st = (cudaStream_t)stream;
  c->m = c->net.m;
  c->n = c->net.n;
  c->R = c->net.R;
  c->prec = desc->precision;
  c->lambda = desc->lambda;
  c->pcg = desc->solver == DNGD_PCG;
  c->primal = resolve_space(desc, c->net) == 1;   // valid: checked above
  if ((s = c->pcg ? alloc_pcg(c, false, nullptr) : alloc_workspace(c, false, nullptr))) {
    free_ctx(c);
    return s;
  }
  *out = c;
  return DNGD_OK;
}

int dngd_solve_space_of(const dngd_ctx* c) { return c ? (c->primal ? DNGD_SPACE_PRIMAL : DNGD_SPACE_DUAL) : -1; }

dngd_status dngd_destroy(dngd_ctx* c) {
  if (!c) return DNGD_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->st);
  free_ctx(c);
  return DNGD_OK;
}

dngd_status dngd_set_timing(dngd_ctx* c, int enable) {
  if (!c) return DNGD_ERR_INVALID_ARG;
  c->timing = enable != 0;
  return DNGD_OK;
}

dngd_status dngd_set_lambda(dngd_ctx* c, double lambda) {
  if (!c || !lambda_ok(c->prec, lambda)) return DNGD_ERR_INVALID_ARG;
  c->lambda = lambda;
  return DNGD_OK;
}

dngd_status dngd_step(dngd_ctx* c, const double* theta, const double* X, const double* target, double* delta_out,
                      dngd_step_info* info) {
  if (!c || !theta || !X || !target || !delta_out) return DNGD_ERR_INVALID_ARG;
  const double* th = in_ptr(c, theta, c->theta_s, c->n);
  const double* x = in_ptr(c, X, c->X_s, (size_t)c->m * c->net.d_in);
  const double* tg = in_ptr(c, target, c->target_s, c->m);
  c->have_step = false;
  dngd_status s = c->pcg ? step_pcg(c, th, x, tg)
                         : (jets64(c->prec) ? step_T<double>(c, th, x, tg, info) : step_T<float>(c, th, x, tg, info));
  if (s) {
    dngd_status ds = read_status(c);
    if (info) fill_info(c, info);
    return ds ? ds : s;
  }
  if ((s = out_copy(c, delta_out, c->delta, c->n))) return s;
  if (!c->pcg && c->prec != DNGD_FP64) {
    const int maxit = c->desc.refine_max_it > 0 ? c->desc.refine_max_it : 200;
    const int used = c->iters[0] > c->iters[1] ? c->iters[0] : c->iters[1];
    c->async_it = 2 * used + 2 < 8 ? 8 : (2 * used + 2 > maxit ? maxit : 2 * used + 2);
  }
  if (info) return fill_info(c, info);
  return DNGD_OK;
}

dngd_status dngd_solve(dngd_ctx* c, const double* rhs, double* x_out) {
  if (!c || !rhs || !x_out) return DNGD_ERR_INVALID_ARG;
  if (!c->have_step) return DNGD_ERR_STATE;
  if (c->primal) {
    const double* b = in_ptr(c, rhs, c->nvec_s, c->n);
    dngd_status s = solve_last(c, b, c->gp, 0);
    if (s) return s;
    return out_copy(c, x_out, c->gp, c->n);
  }
  const double* b = in_ptr(c, rhs, c->mvec_s, c->m);
  dngd_status s = solve_last(c, b, c->xsol, 0);
  if (s) return s;
  return out_copy(c, x_out, c->xsol, c->m);
}

dngd_status dngd_residual_jacobian(dngd_ctx* c, const double* theta, const double* X, const double* target,
                                   double* r_out, double* J_out) {
  if (!c || !theta || !X || !target || !r_out) return DNGD_ERR_INVALID_ARG;
  const double* th = in_ptr(c, theta, c->theta_s, c->n);
  const double* x = in_ptr(c, X, c->X_s, (size_t)c->m * c->net.d_in);
  const double* tg = in_ptr(c, target, c->target_s, c->m);
  DNGD_CUDA_CHECK(cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->st));
  dngd_status s;
  if (c->pcg) {
    if (J_out) return DNGD_ERR_INVALID_ARG;  // the matrix-free context never forms J
    s = forward_only<float>(c, theta_in_T<float>(c, th), x, tg, c->r);
    if (s) return s;
    c->have_step = false;
    if ((s = out_copy(c, r_out, c->r, c->m))) return s;
    return read_status(c);
  }
  if (jets64(c->prec)) s = residual_jacobian_T<double>(c, theta_in_T<double>(c, th), x, tg);
  else s = residual_jacobian_T<float>(c, theta_in_T<float>(c, th), x, tg);
  if (s) return s;
  c->have_step = false;
  if ((s = out_copy(c, r_out, c->r, c->m))) return s;
  if (J_out) {
    double* dst = J_out;
    const bool dev = is_device_ptr(J_out);
    std::vector<double> tmp;
    double* dbuf = nullptr;
    if (!dev) {
      if (cudaMalloc(&dbuf, sizeof(double) * (size_t)c->m * c->n) != cudaSuccess) return DNGD_ERR_OOM;
      dst = dbuf;
    }
    if (jets64(c->prec)) s = rows_to_f64<double>(c->m, c->n, (const double*)c->J, c->ldJ, dst, c->st);
    else s = rows_to_f64<float>(c->m, c->n, (const float*)c->J, c->ldJ, dst, c->st);
    if (!s && !dev) {
      cudaMemcpyAsync(J_out, dbuf, sizeof(double) * (size_t)c->m * c->n, cudaMemcpyDeviceToHost, c->st);
      cudaStreamSynchronize(c->st);
    }
    if (dbuf) cudaFree(dbuf);
    if (s) return s;
  }
  return read_status(c);
}

dngd_status dngd_fvv(dngd_ctx* c, const double* theta, const double* X, const double* target, const double* v,
                     double* fvv_out) {
  if (!c || !theta || !X || !v || !fvv_out) return DNGD_ERR_INVALID_ARG;
  (void)target;
  const double* th = in_ptr(c, theta, c->theta_s, c->n);
  const double* x = in_ptr(c, X, c->X_s, (size_t)c->m * c->net.d_in);
  const double* vv = in_ptr(c, v, c->nvec_s, c->n);
  dngd_status s;
  if (jets64(c->prec)) {
    s = jets_fvv<double>(c->net, th, vv, x, (double*)c->Z3, (double*)c->H3a, (double*)c->H3b, c->fvv, c->st,
                         jets_tc<double>(c), c->status);
  } else {
    const float* t32 = theta_in_T<float>(c, th);
    to_float(c->n, vv, c->v32, c->st);
    s = jets_fvv<float>(c->net, t32, c->v32, x, (float*)c->Z3, (float*)c->H3a, (float*)c->H3b, c->fvv, c->st,
                        tc3p(c), c->status);
  }
  if (s) return s;
  c->have_step = false;
  return out_copy(c, fvv_out, c->fvv, c->m);
}

// ||r(theta + etas[j] delta)||^2 into sq[j] for j < k: in the FP32 modes
// up to kTrials trials share each launch of the forward sweep, otherwise one
// trial at a time.
dngd_status trial_sqnorms(dngd_ctx* c, const double* theta, const double* X, const double* target,
                          const double* delta, const double* etas, int k, double* sq) {
  dngd_status s;
  if (c->prec != DNGD_FP64 && c->ls_th32 && c->tc3.buf) {
    for (int j = 0; j < k; j += c->ls_G) {
      const int G = k - j < c->ls_G ? k - j : c->ls_G;
      if ((s = axpy_to_float_batch(c->n, G, theta, etas + j, delta, c->ls_th32, c->st))) return s;
      if ((s = jets_forward_trials(c->net, G, c->ls_th32, c->n, X, target, c->ls_Z, c->ls_H, c->ls_r,
                                   c->status, c->st, c->tc3)))
        return s;
      if ((s = sqnorm_batch(c->m, G, c->ls_r, sq + j, c->st))) return s;
    }
    return DNGD_OK;
  }
  for (int j = 0; j < k; ++j) {
    if ((s = axpy_to(c->n, theta, etas[j], delta, c->theta_tmp, c->st))) return s;
    if (c->prec == DNGD_FP64) s = forward_only<double>(c, c->theta_tmp, X, target, c->cg_res);
    else s = forward_only<float>(c, theta_in_T<float>(c, c->theta_tmp), X, target, c->cg_res, true);
    if (s) return s;
    if ((s = dot_dev(c->m, c->cg_res, c->cg_res, sq + j, c->dot_partials, c->st))) return s;
  }
  return DNGD_OK;
}

dngd_status dngd_loss(dngd_ctx* c, const double* theta, const double* X, const double* target, const double* delta,
                      const double* etas, int k, double* loss_out) {
  if (!c || !theta || !X || !target || !etas || !loss_out || k < 1) return DNGD_ERR_INVALID_ARG;
  const double* th = in_ptr(c, theta, c->theta_s, c->n);
  const double* x = in_ptr(c, X, c->X_s, (size_t)c->m * c->net.d_in);
  const double* tg = in_ptr(c, target, c->target_s, c->m);
  const double* dl = delta ? in_ptr(c, delta, c->nvec_s, c->n) : nullptr;
  DNGD_CUDA_CHECK(cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->st));
  // the trial losses stay on the device (64 per round trip), so the trials'
  // kernels queue back to back
  if (!c->loss_dev) {
    if (cudaMalloc(&c->loss_dev, sizeof(double) * 64) != cudaSuccess) return DNGD_ERR_OOM;
    c->allocs.push_back(c->loss_dev);
    DNGD_CUDA_CHECK(cudaMallocHost(&c->loss_host, sizeof(double) * 64));
  }
  for (int j0 = 0; j0 < k; j0 += 64) {
    const int kk = (k - j0) < 64 ? (k - j0) : 64;
    dngd_status s = trial_sqnorms(c, th, x, tg, dl, etas + j0, kk, c->loss_dev);
    if (s) return s;
    DNGD_CUDA_CHECK(cudaMemcpyAsync(c->loss_host, c->loss_dev, sizeof(double) * kk, cudaMemcpyDeviceToHost, c->st));
    DNGD_CUDA_CHECK(cudaStreamSynchronize(c->st));
    for (int j = 0; j < kk; ++j) loss_out[j0 + j] = 0.5 * c->loss_host[j];
  }
  c->have_step = false;
  return read_status(c);
}

dngd_status dngd_line_search(dngd_ctx* c, const double* theta, const double* X, const double* target,
                             const double* delta, const double* etas, int k, double* theta_out, double* eta_out) {
  if (!c || !theta || !delta || !etas || !theta_out || !eta_out || k < 1) return DNGD_ERR_INVALID_ARG;
  std::vector<double> losses(k);
  dngd_status s = dngd_loss(c, theta, X, target, delta, etas, k, losses.data());
  if (s) return s;
  int best = 0;
  for (int j = 1; j < k; ++j)
    if (losses[j] < losses[best]) best = j;
  *eta_out = etas[best];
  const double* th = in_ptr(c, theta, c->theta_s, c->n);
  const double* dl = in_ptr(c, delta, c->nvec_s, c->n);
  if ((s = axpy_to(c->n, th, etas[best], dl, c->theta_tmp, c->st))) return s;
  return out_copy(c, theta_out, c->theta_tmp, c->n);
}

dngd_status dngd_line_search_async(dngd_ctx* c, double* theta, const double* X, const double* target,
                                   const double* delta, const double* etas, int k) {
  if (!c || !theta || !X || !target || !delta || !etas || k < 1 || k > 64) return DNGD_ERR_INVALID_ARG;
  if (!is_device_ptr(theta) || !is_device_ptr(X) || !is_device_ptr(target) || !is_device_ptr(delta))
    return DNGD_ERR_INVALID_ARG;
  if (!c->ls_dev) {
    if (cudaMalloc(&c->ls_dev, sizeof(double) * 132) != cudaSuccess) return DNGD_ERR_OOM;
    c->allocs.push_back(c->ls_dev);
    DNGD_CUDA_CHECK(cudaMallocHost(&c->ls_host, sizeof(double) * 64));
  }
  // the device grid is reloaded only when it changes (then after the stream
  // has consumed the previous pinned copy)
  bool same = c->ls_k == k;
  for (int j = 0; j < k && same; ++j) same = c->ls_host[j] == etas[j];
  if (!same) {
    DNGD_CUDA_CHECK(cudaStreamSynchronize(c->st));
    for (int j = 0; j < k; ++j) c->ls_host[j] = etas[j];
    DNGD_CUDA_CHECK(cudaMemcpyAsync(c->ls_dev, c->ls_host, sizeof(double) * k, cudaMemcpyHostToDevice, c->st));
    c->ls_k = k;
  }
  double* losses = c->ls_dev + 64;
  // the step's status word, before the trial evaluations add their own flags
  int* step_flags = (int*)(c->ls_dev + 130);
  DNGD_CUDA_CHECK(cudaMemcpyAsync(step_flags, c->status, sizeof(int), cudaMemcpyDeviceToDevice, c->st));
  dngd_status s = trial_sqnorms(c, theta, X, target, delta, etas, k, losses);
  if (s) return s;
  return ls_finish(c->n, k, losses, c->ls_dev, step_flags, c->ls_dev + 128, delta, theta, c->st);
}

dngd_status dngd_train(dngd_ctx* c, double* theta, double* X, double* target, const dngd_train_cfg* cfg,
                       double* loss_history, dngd_train_result* result) {
  if (!c || !theta || !X || !target || !cfg || !result || cfg->max_iters < 1) return DNGD_ERR_INVALID_ARG;
  if (cfg->resample_every < 0 || (cfg->resample_every > 0 && !cfg->resample)) return DNGD_ERR_INVALID_ARG;
  if (cfg->etas && (cfg->k < 1 || cfg->k > 64)) return DNGD_ERR_INVALID_ARG;
  if (!is_device_ptr(theta) || !is_device_ptr(X) || !is_device_ptr(target)) return DNGD_ERR_INVALID_ARG;
  double grid[64];
  int k = 31;
  if (cfg->etas) {
    k = cfg->k;
    for (int j = 0; j < k; ++j) grid[j] = cfg->etas[j];
  } else {
    for (int j = 0; j < k; ++j) grid[j] = 1.0 / (double)(1ull << j);
  }
  memset(result, 0, sizeof(*result));
  result->stop = DNGD_STOP_ITERS;
  const auto t0 = std::chrono::steady_clock::now();
  auto elapsed = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  dngd_status s = DNGD_OK;
  for (int it = 0; it < cfg->max_iters; ++it) {
    if (cfg->time_budget_s > 0.0 && elapsed() >= cfg->time_budget_s) {
      result->stop = DNGD_STOP_BUDGET;
      break;
    }
    if (it > 0 && cfg->resample_every > 0 && it % cfg->resample_every == 0) {
      // the device is idle on the context's stream before the callback
      // rewrites the points the last line search read
      DNGD_CUDA_CHECK(cudaStreamSynchronize(c->st));
      if ((s = cfg->resample(cfg->user, it, X, target))) break;
    }
    dngd_step_info info;
    s = dngd_step(c, theta, X, target, c->delta, &info);
    if (s == DNGD_ERR_NO_CONVERGE) s = DNGD_OK;
    if (s) break;
    if (loss_history) loss_history[it] = info.loss;
    if (cfg->loss_target > 0.0 && info.loss <= cfg->loss_target) {
      result->stop = DNGD_STOP_LOSS;
      result->loss = info.loss;
      break;
    }
    if ((s = dngd_line_search_async(c, theta, X, target, c->delta, grid, k))) break;
    result->iters = it + 1;
  }
  if (!s && result->stop != DNGD_STOP_LOSS) {
    double l = 0.0;
    s = dngd_loss(c, theta, X, target, nullptr, grid, 1, &l);
    result->loss = l;
  }
  result->elapsed_s = elapsed();
  return s;
}

dngd_status dngd_get_stage(dngd_ctx* c, int which, double* dst) {
  if (!c || !dst) return DNGD_ERR_INVALID_ARG;
  if (!c->have_step) return DNGD_ERR_STATE;
  const int m = c->m;
  if (c->primal && (which == 1 || which == 4)) return DNGD_ERR_STATE;
  switch (which) {
    case 0: return out_copy(c, dst, c->r, m);
    case 1: return out_copy(c, dst, c->alpha, m);
    case 2: return out_copy(c, dst, c->v, c->n);
    case 3: return out_copy(c, dst, c->fvv, m);
    case 4: return out_copy(c, dst, c->beta, m);
    case 5: return out_copy(c, dst, c->a, c->n);
    case 6:
    case 7:
    case 10:
    case 11: {
      // 7: the FP64 path's factor; 10: the explicit inverse factor of the
      // mixed paths (FP32); 11: the exact-Gram modes' FP64 factor
      const void* src = which == 6 ? c->Kcopy : which == 7 ? c->K : which == 10 ? (void*)c->Linv : (void*)c->Kd;
      if (!src) return DNGD_ERR_STATE;
      const bool k64 = which == 11 || (which != 10 && c->prec == DNGD_FP64);
      if (which == 7 && !k64) return DNGD_ERR_STATE;
      const int d = c->prec == DNGD_FP64 ? c->ms : m;   // n in the primal space
      double* buf = nullptr;
      if (cudaMalloc(&buf, sizeof(double) * (size_t)d * d) != cudaSuccess) return DNGD_ERR_OOM;
      dngd_status s = k64 ? lower_to_f64<double>(d, (const double*)src, c->ldk, buf, c->st)
                                           : lower_to_f64<float>(d, (const float*)src, c->ldk, buf, c->st);
      if (!s) {
        cudaMemcpyAsync(dst, buf, sizeof(double) * (size_t)d * d, cudaMemcpyDefault, c->st);
        cudaStreamSynchronize(c->st);
      }
      cudaFree(buf);
      return s;
    }
    case 8: {
      if (!c->pcg) return DNGD_ERR_STATE;
      double* buf = nullptr;
      const long long cnt = (long long)m * c->mf.ell;
      if (cudaMalloc(&buf, sizeof(double) * cnt) != cudaSuccess) return DNGD_ERR_OOM;
      dngd_status s = mf_g_to_double(cnt, c->mf.KCI, 1.0, buf, c->st);
      if (!s) {
        cudaMemcpyAsync(dst, buf, sizeof(double) * cnt, cudaMemcpyDefault, c->st);
        cudaStreamSynchronize(c->st);
      }
      cudaFree(buf);
      return s;
    }
    case 9: {
      // the exact FP64 Gram (MIXED_OZ), full symmetric, no shift
      if (!c->oz) return DNGD_ERR_STATE;
      double* buf = nullptr;
      if (cudaMalloc(&buf, sizeof(double) * (size_t)m * c->ldk) != cudaSuccess) return DNGD_ERR_OOM;
      dngd_status s = gram_oz_read(c->oz, buf, c->st);
      if (!s) {
        cudaMemcpy2DAsync(dst, sizeof(double) * m, buf, sizeof(double) * c->ldk, sizeof(double) * m, m,
                          cudaMemcpyDefault, c->st);
        cudaStreamSynchronize(c->st);
      }
      cudaFree(buf);
      return s;
    }
    default: return DNGD_ERR_INVALID_ARG;
  }
}

dngd_status dngd_check_wait_expiry(dngd_ctx* c, double limit_ms) {
  if (!c || !(limit_ms > 0.0) || limit_ms > 1000.0) return DNGD_ERR_INVALID_ARG;
  void* state = c->pstate;
  bool own = false;
  if (!state) {
    if (cudaMalloc(&state, 256) != cudaSuccess) return DNGD_ERR_OOM;
    own = true;
  }
  DNGD_CUDA_CHECK(cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->st));
  dngd_status s = barrier_expiry(state, c->status, limit_ms, c->st);
  if (!s) s = read_status(c);
  if (own) cudaFree(state);
  return s;
}

dngd_status dngd_set_landmarks(dngd_ctx* c, const int64_t* idx, int ell) {
  if (!c || !idx || !c->pcg || ell < 1 || ell > c->mf.ell || ell > c->m) return DNGD_ERR_INVALID_ARG;
  std::vector<int> keep = c->lm_host;
  c->lm_host.assign(ell, 0);
  for (int j = 0; j < ell; ++j) {
    if (idx[j] < 0 || idx[j] >= c->m) {
      c->lm_host = keep;
      return DNGD_ERR_INVALID_ARG;
    }
    c->lm_host[j] = (int)idx[j];
  }
  c->nu_sticky = 0.0;
  return upload_landmarks(c);
}

dngd_status dngd_kvp(dngd_ctx* c, const double* v, double* w_out) {
  if (!c || !v || !w_out) return DNGD_ERR_INVALID_ARG;
  if (!c->pcg || !c->have_step) return DNGD_ERR_STATE;
  const double* vv = in_ptr(c, v, c->mvec_s, c->m);
  dngd_status s = mf_kvp(c->mf, vv, c->lambda, c->xsol, c->st);
  if (s) return s;
  return out_copy(c, w_out, c->xsol, c->m);
}

dngd_status dngd_precond_apply(dngd_ctx* c, const double* x, double* z_out) {
  if (!c || !x || !z_out) return DNGD_ERR_INVALID_ARG;
  if (!c->pcg || !c->have_step) return DNGD_ERR_STATE;
  const double* xx = in_ptr(c, x, c->mvec_s, c->m);
  dngd_status s = mf_precond(c->mf, c->lambda, xx, c->xsol, c->st);
  if (s) return s;
  return out_copy(c, z_out, c->xsol, c->m);
}


}  // extern "C"

// ---------------------------------------------------------------------------
// Asynchronous, graph-captured stepping and batches of independent instances
// ---------------------------------------------------------------------------

namespace {

// Enqueue one asynchronous step of a dense context on its stream, reading the
// staging inputs and ending with copies of the status word and scalars to the
// pinned host buffers.  No host synchronisation: capturable.
dngd_status enqueue_async(dngd_ctx* c) {
  c->async = true;
  const bool timing = c->timing;
  c->timing = false;
  dngd_status s = jets64(c->prec) ? step_T<double>(c, c->theta_s, c->X_s, c->target_s, nullptr)
                                       : step_T<float>(c, c->theta_s, c->X_s, c->target_s, nullptr);
  c->timing = timing;
  c->async = false;
  if (s) return s;
  if (c->phase == 1) return DNGD_OK;   // the step goes on after the batch's factorisation
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->scal_h, c->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, c->st));
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->status_h, c->status, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->st));
  return DNGD_OK;
}

dngd_status stage_inputs(dngd_ctx* c, const double* theta, const double* X, const double* target,
                         cudaStream_t st) {
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->theta_s, theta, sizeof(double) * c->n, cudaMemcpyDefault, st));
  DNGD_CUDA_CHECK(
      cudaMemcpyAsync(c->X_s, X, sizeof(double) * (size_t)c->m * c->net.d_in, cudaMemcpyDefault, st));
  DNGD_CUDA_CHECK(cudaMemcpyAsync(c->target_s, target, sizeof(double) * c->m, cudaMemcpyDefault, st));
  return DNGD_OK;
}

}  // namespace

struct dngd_batch {
  std::vector<dngd_ctx*> ctx;
  std::vector<cudaEvent_t> join;
  cudaStream_t master = nullptr;
  bool own_master = false;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool first = true;
  unsigned long long graph_kernels = 0;
  OzBatchFactor* ozb = nullptr;     // every exact-Gram instance's factorisation together
  cudaEvent_t fork2 = nullptr;      // after the batched factorisation
};

extern "C" {

dngd_status dngd_step_async(dngd_ctx* c, const double* theta, const double* X, const double* target,
                            double* delta_out) {
  if (!c || !theta || !X || !target || !delta_out) return DNGD_ERR_INVALID_ARG;
  if (c->pcg) return DNGD_ERR_INVALID_ARG;
  if (!c->async_ok) {
    // the first step is synchronous: it fixes the preconditioner shift
    // (a refinement that stopped at its iteration cap still gives a step)
    dngd_status s = dngd_step(c, theta, X, target, delta_out, nullptr);
    if (s && s != DNGD_ERR_NO_CONVERGE) return s;
    c->async_ok = true;
    DNGD_CUDA_CHECK(cudaMemcpyAsync(c->scal_h, c->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, c->st));
    DNGD_CUDA_CHECK(cudaMemcpyAsync(c->status_h, c->status, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    return DNGD_OK;
  }
  dngd_status s = stage_inputs(c, theta, X, target, c->st);
  if (s) return s;
  // the graph is captured and replayed on a private stream (the context's
  // stream may be the legacy default stream, which cannot be captured);
  // events keep it ordered with the context's stream
  if (!c->gst) {
    DNGD_CUDA_CHECK(cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking));
    DNGD_CUDA_CHECK(cudaEventCreateWithFlags(&c->gev[0], cudaEventDisableTiming));
    DNGD_CUDA_CHECK(cudaEventCreateWithFlags(&c->gev[1], cudaEventDisableTiming));
  }
  cudaStream_t user = c->st;
  // the graph bakes in lambda and the preconditioner shift of the last
  // synchronous step; either changing means a new capture
  const double mu_now = c->mu_sticky > c->desc.shift_mu ? c->mu_sticky : c->desc.shift_mu;
  if (!c->graph || c->graph_lambda != c->lambda || c->graph_mu != mu_now || c->graph_it != c->async_it) {
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    c->st = c->gst;
    cudaError_t e = cudaStreamBeginCapture(c->gst, cudaStreamCaptureModeThreadLocal);
    const unsigned long long k0 = dngd::g_launches.load();
    if (e == cudaSuccess) {
      s = enqueue_async(c);
      e = cudaStreamEndCapture(c->gst, &g);
    }
    c->graph_kernels = dngd::g_launches.load() - k0;
    dngd::g_launches.fetch_sub(c->graph_kernels);
    c->st = user;
    if (s) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    DNGD_CUDA_CHECK(e);
    DNGD_CUDA_CHECK(cudaGraphInstantiate(&c->graph, g, 0));
    cudaGraphDestroy(g);
    c->graph_lambda = c->lambda;
    c->graph_mu = mu_now;
    c->graph_it = c->async_it;
  }
  DNGD_CUDA_CHECK(cudaEventRecord(c->gev[0], user));
  DNGD_CUDA_CHECK(cudaStreamWaitEvent(c->gst, c->gev[0], 0));
  DNGD_CUDA_CHECK(cudaGraphLaunch(c->graph, c->gst));
  dngd::g_launches.fetch_add(c->graph_kernels);
  DNGD_CUDA_CHECK(cudaEventRecord(c->gev[1], c->gst));
  DNGD_CUDA_CHECK(cudaStreamWaitEvent(user, c->gev[1], 0));
  DNGD_CUDA_CHECK(cudaMemcpyAsync(delta_out, c->delta, sizeof(double) * c->n, cudaMemcpyDefault, user));
  c->have_step = true;
  return DNGD_OK;
}

dngd_status dngd_step_wait(dngd_ctx* c, dngd_step_info* info) {
  if (!c) return DNGD_ERR_INVALID_ARG;
  DNGD_CUDA_CHECK(cudaStreamSynchronize(c->st));
  dngd_status s = finish_async(c, info);
  // a failed factor or a capped solve that did not converge: the next step
  // runs synchronously (shift search, full iteration budget)
  if (s == DNGD_ERR_NOT_SPD || async_capped(c)) c->async_ok = false;
  return s;
}

dngd_status dngd_batch_create(dngd_batch** out, const dngd_problem_desc* descs, int count, void* stream) {
  if (!out || !descs || count < 1) return DNGD_ERR_INVALID_ARG;
  *out = nullptr;
  dngd_batch* b = new dngd_batch();
  for (int i = 0; i < count; ++i) {
    if (descs[i].solver != DNGD_DENSE) {
      dngd_batch_destroy(b);
      return DNGD_ERR_INVALID_ARG;
    }
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      dngd_batch_destroy(b);
      return DNGD_ERR_CUDA;
    }
    // exact-Gram instances factor with double-float trailing updates, the
    // form the batch runs for all of them in one launch per kernel (also in
    // each instance's synchronous steps, so they compute the same factor)
    dngd_problem_desc d = descs[i];
    if (d.precision == DNGD_MIXED_OZ || d.precision == DNGD_MIXED_OZ64) d.factor_update = DNGD_FACTOR_DF;
    dngd_ctx* c = nullptr;
    dngd_status s = dngd_create(&c, &d, st);
    if (s) {
      cudaStreamDestroy(st);
      dngd_batch_destroy(b);
      return s;
    }
    b->ctx.push_back(c);
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    b->join.push_back(ev);
  }
  if (stream) {
    b->master = (cudaStream_t)stream;
  } else {
    cudaStreamCreateWithFlags(&b->master, cudaStreamNonBlocking);
    b->own_master = true;
  }
  cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&b->fork2, cudaEventDisableTiming);
  bool all_oz = true;
  for (dngd_ctx* c : b->ctx) all_oz = all_oz && c->ozf != nullptr;
  if (all_oz) {
    std::vector<OzFactor*> f;
    std::vector<int*> st;
    for (dngd_ctx* c : b->ctx) {
      f.push_back(c->ozf);
      st.push_back(c->status);
    }
    dngd_status s = oz_factor_batched_plan(&b->ozb, (int)f.size(), f.data(), st.data(), b->master);
    if (s) {
      dngd_batch_destroy(b);
      return s;
    }
  }
  *out = b;
  return DNGD_OK;
}

dngd_status dngd_batch_destroy(dngd_batch* b) {
  if (!b) return DNGD_ERR_INVALID_ARG;
  if (b->master) cudaStreamSynchronize(b->master);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    cudaStream_t st = b->ctx[i]->st;
    dngd_destroy(b->ctx[i]);
    cudaStreamDestroy(st);
    cudaEventDestroy(b->join[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->fork2) cudaEventDestroy(b->fork2);
  if (b->ozb) oz_factor_batched_free(b->ozb);
  if (b->own_master) cudaStreamDestroy(b->master);
  delete b;
  return DNGD_OK;
}

int dngd_batch_size(const dngd_batch* b) { return b ? (int)b->ctx.size() : 0; }

dngd_status dngd_batch_step(dngd_batch* b, const double* const* theta, const double* const* X,
                            const double* const* target, double* const* delta_out, dngd_step_info* infos) {
  if (!b || !theta || !X || !target || !delta_out) return DNGD_ERR_INVALID_ARG;
  const int nb = (int)b->ctx.size();
  dngd_status worst = DNGD_OK;
  if (b->first) {
    // synchronous first step per instance (fixes each preconditioner shift)
    for (int i = 0; i < nb; ++i) {
      dngd_status s = dngd_step(b->ctx[i], theta[i], X[i], target[i], delta_out[i], infos ? &infos[i] : nullptr);
      if (s && !worst) worst = s;
      b->ctx[i]->async_ok = (s == DNGD_OK);
    }
    b->first = false;
    return worst;
  }
  for (int i = 0; i < nb; ++i) {
    dngd_status s = stage_inputs(b->ctx[i], theta[i], X[i], target[i], b->master);
    if (s) return s;
  }
  if (!b->exec) {
    // one graph: fork to every instance stream, one asynchronous step each, join
    cudaGraph_t g = nullptr;
    DNGD_CUDA_CHECK(cudaStreamBeginCapture(b->master, cudaStreamCaptureModeThreadLocal));
    const unsigned long long k0 = dngd::g_launches.load();
    dngd_status s = DNGD_OK;
    if (cudaEventRecord(b->fork, b->master) != cudaSuccess) s = DNGD_ERR_CUDA;
    // exact-Gram batches in two halves around one batched factorisation of
    // every instance; otherwise one whole step per instance
    const int halves = b->ozb ? 2 : 1;
    for (int h = 0; h < halves && !s; ++h) {
      cudaEvent_t ev = h == 0 ? b->fork : b->fork2;
      for (int i = 0; i < nb && !s; ++i) {
        dngd_ctx* c = b->ctx[i];
        c->phase = b->ozb ? h + 1 : 0;
        if (cudaStreamWaitEvent(c->st, ev, 0) != cudaSuccess) s = DNGD_ERR_CUDA;
        if (!s) s = enqueue_async(c);
        if (!s && cudaEventRecord(b->join[i], c->st) != cudaSuccess) s = DNGD_ERR_CUDA;
        if (!s && cudaStreamWaitEvent(b->master, b->join[i], 0) != cudaSuccess) s = DNGD_ERR_CUDA;
      }
      if (!s && h == 0 && b->ozb) {
        s = oz_factor_batched_run(b->ozb, b->master);
        if (!s && cudaEventRecord(b->fork2, b->master) != cudaSuccess) s = DNGD_ERR_CUDA;
      }
    }
    for (dngd_ctx* c : b->ctx) c->phase = 0;
    const cudaError_t e = cudaStreamEndCapture(b->master, &g);
    b->graph_kernels = dngd::g_launches.load() - k0;
    dngd::g_launches.fetch_sub(b->graph_kernels);
    if (s || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return s ? s : DNGD_ERR_CUDA;
    }
    DNGD_CUDA_CHECK(cudaGraphInstantiate(&b->exec, g, 0));
    cudaGraphDestroy(g);
  }
  DNGD_CUDA_CHECK(cudaGraphLaunch(b->exec, b->master));
  dngd::g_launches.fetch_add(b->graph_kernels);
  for (int i = 0; i < nb; ++i)
    DNGD_CUDA_CHECK(cudaMemcpyAsync(delta_out[i], b->ctx[i]->delta, sizeof(double) * b->ctx[i]->n,
                                    cudaMemcpyDefault, b->master));
  DNGD_CUDA_CHECK(cudaStreamSynchronize(b->master));
  bool recapture = false;
  for (int i = 0; i < nb; ++i) {
    dngd_ctx* c = b->ctx[i];
    c->have_step = true;
    dngd_status s = finish_async(c, infos ? &infos[i] : nullptr);
    if (s == DNGD_ERR_NOT_SPD || async_capped(c)) {
      // redo this instance synchronously (the shift search raises mu) and
      // rebuild the batch graph with the new shift
      s = dngd_step(c, theta[i], X[i], target[i], delta_out[i], infos ? &infos[i] : nullptr);
      recapture = true;
    }
    if (s && !worst) worst = s;
  }
  if (recapture && b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return worst;
}

dngd_ctx* dngd_batch_context(dngd_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
  return b->ctx[i];
}

}  // extern "C"
