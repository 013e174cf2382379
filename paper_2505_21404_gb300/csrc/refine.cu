// Refinement of the mixed-precision dual solve: preconditioned CG on
// (J J^T + lambda I) x = b with the FP32 Jacobian as operator, applied as two
// HBM-bound GEMVs that accumulate in double-float arithmetic, and the explicit
// inverse factor of the low-precision Gram as preconditioner
// (M^{-1} = Linv^T Linv).  This is the iterative counterpart of the paper's
// direct solve (Alg. DenseDualSolve): the low-precision factor only steers the
// iteration, the operator keeps the exact lambda.
//
// All CG scalars live on the device.  Every kernel of an iteration first
// reads the device "done" flag and returns at once after convergence, so the
// host only synchronises once per `check_every` iterations.  Reductions use a
// fixed order, so results are reproducible bit for bit.
#include "common.cuh"
#include "kernels.h"
#include "step_kernels.h"

namespace dngd {

namespace {

__device__ __forceinline__ bool stopped(const double* scal) { return scal && scal[S_DONE] != 0.0; }

__device__ __forceinline__ void df_axpy2(dfloat& acc, float a, float2 x) {
  acc = df_fma(acc, a, x.x);
  acc.lo = fmaf(a, x.y, acc.lo);
}

// xs[i] = (hi, lo): hi = fl32(x[i]), lo = fl32(x[i] - hi); tail zeroed.
__global__ void k_split_vec(int n, int npad, const double* __restrict__ x, float2* __restrict__ xs,
                            const double* scal) {
  if (stopped(scal)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  float2 v = make_float2(0.f, 0.f);
  if (i < n) {
    const double xv = x[i];
    v.x = (float)xv;
    v.y = (float)(xv - (double)v.x);
  }
  xs[i] = v;
}

// partials[split][c] = sum_{rows of split} A[i, c] x[i]; a thread owns 4
// columns and keeps 8 rows of float4 loads in flight.
__global__ void __launch_bounds__(256) k_gemv_t_f32(int m, int n, const float* __restrict__ A, long long lda,
                                                     const float2* __restrict__ xs, int rows_per_split,
                                                     double* __restrict__ partials, const double* scal) {
  if (stopped(scal)) return;
  const int c4 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (c4 >= n) return;
  const int i0 = blockIdx.y * rows_per_split;
  const int i1 = min(m, i0 + rows_per_split);
  dfloat acc[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[j] = {0.f, 0.f};
  constexpr int U = 8;
  int i = i0;
  for (; i + U <= i1; i += U) {
    float4 a[U];
    float2 xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a[u] = __ldg(reinterpret_cast<const float4*>(A + (long long)(i + u) * lda + c4));
      xv[u] = xs[i + u];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      df_axpy2(acc[0], a[u].x, xv[u]);
      df_axpy2(acc[1], a[u].y, xv[u]);
      df_axpy2(acc[2], a[u].z, xv[u]);
      df_axpy2(acc[3], a[u].w, xv[u]);
    }
  }
  for (; i < i1; ++i) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(A + (long long)i * lda + c4));
    const float2 xv = xs[i];
    df_axpy2(acc[0], a.x, xv);
    df_axpy2(acc[1], a.y, xv);
    df_axpy2(acc[2], a.z, xv);
    df_axpy2(acc[3], a.w, xv);
  }
  double* out = partials + (long long)blockIdx.y * n + c4;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (c4 + j < n) out[j] = (double)acc[j].hi + (double)acc[j].lo;
}

__global__ void k_reduce_splits(int n, int splits, const double* __restrict__ partials, double alpha,
                                double* __restrict__ y, const double* scal) {
  if (stopped(scal)) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double s = 0.0;
  for (int k = 0; k < splits; ++k) s += partials[(long long)k * n + p];
  y[p] = alpha * s;
}

// y[r] = alpha * sum_c A[r, c] x[c] + add_scale * add[r] for 4 rows per block;
// optionally dotp[block] = sum_r dotw[r] * y[r] (the block's share of <w, y>).
constexpr int kRows = 4;
__global__ void __launch_bounds__(256) k_gemv_n_f32(int m, int n, const float* __restrict__ A, long long lda,
                                                     const float2* __restrict__ xs, double alpha,
                                                     const double* __restrict__ add, double add_scale,
                                                     double* __restrict__ y, const double* __restrict__ dotw,
                                                     double* __restrict__ dotp, const double* scal) {
  if (stopped(scal)) return;
  const int r0 = blockIdx.x * kRows;
  const int nrow = min(kRows, m - r0);
  dfloat acc[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) acc[r] = {0.f, 0.f};
  for (int c4 = threadIdx.x * 4; c4 < n; c4 += blockDim.x * 4) {
    const float4 xa = *reinterpret_cast<const float4*>(xs + c4);
    const float4 xb = *reinterpret_cast<const float4*>(xs + c4 + 2);
    float4 a[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
      a[r] = r < nrow ? __ldg(reinterpret_cast<const float4*>(A + (long long)(r0 + r) * lda + c4))
                      : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      df_axpy2(acc[r], a[r].x, make_float2(xa.x, xa.y));
      df_axpy2(acc[r], a[r].y, make_float2(xa.z, xa.w));
      df_axpy2(acc[r], a[r].z, make_float2(xb.x, xb.y));
      df_axpy2(acc[r], a[r].w, make_float2(xb.z, xb.w));
    }
  }
  __shared__ double red[kRows][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    const dfloat t = df_warp_sum(acc[r]);
    if (lane == 0) red[r][warp] = (double)t.hi + (double)t.lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double d = 0.0;
    for (int r = 0; r < nrow; ++r) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[r][w];
      const double yr = alpha * t + (add ? add_scale * add[r0 + r] : 0.0);
      y[r0 + r] = yr;
      if (dotw) d += dotw[r0 + r] * yr;
    }
    if (dotp) dotp[blockIdx.x] = d;
  }
}

// Double-float matrix (pairs hi + lo): y[r] = sum_c A[r, c] x[c] +
// add_scale * add[r] for 4 rows per block with double-float products and
// accumulation (x split on the fly), optionally dotp[block] = sum_r dotw[r] y[r].
__global__ void __launch_bounds__(256) k_gemv_n_df(int m, int n, const float2* __restrict__ A, long long lda,
                                                    const double* __restrict__ x, const double* __restrict__ add,
                                                    double add_scale, double* __restrict__ y,
                                                    const double* __restrict__ dotw, double* __restrict__ dotp,
                                                    const double* scal) {
  if (stopped(scal)) return;
  const int r0 = blockIdx.x * kRows;
  const int nrow = min(kRows, m - r0);
  dfloat acc[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) acc[r] = {0.f, 0.f};
  for (int c2 = threadIdx.x * 2; c2 < n; c2 += blockDim.x * 2) {
    const bool pair = c2 + 1 < n;
    const double x0 = x[c2], x1 = pair ? x[c2 + 1] : 0.0;
    const float x0h = (float)x0, x1h = (float)x1;
    const float x0l = (float)(x0 - (double)x0h), x1l = (float)(x1 - (double)x1h);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      if (r < nrow) {
        const float2* a = A + (long long)(r0 + r) * lda + c2;
        float4 v;
        if (pair) {
          v = __ldg(reinterpret_cast<const float4*>(a));
        } else {
          const float2 t = a[0];
          v = make_float4(t.x, t.y, 0.f, 0.f);
        }
        acc[r] = df_fma(acc[r], v.x, x0h);
        acc[r].lo = fmaf(v.x, x0l, fmaf(v.y, x0h, acc[r].lo));
        acc[r] = df_fma(acc[r], v.z, x1h);
        acc[r].lo = fmaf(v.z, x1l, fmaf(v.w, x1h, acc[r].lo));
      }
    }
  }
  __shared__ double red[kRows][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    const dfloat t = df_warp_sum(acc[r]);
    if (lane == 0) red[r][warp] = (double)t.hi + (double)t.lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double d = 0.0;
    for (int r = 0; r < nrow; ++r) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[r][w];
      const double yr = t + (add ? add_scale * add[r0 + r] : 0.0);
      y[r0 + r] = yr;
      if (dotw) d += dotw[r0 + r] * yr;
    }
    if (dotp) dotp[blockIdx.x] = d;
  }
}

// Fixed-order reduction of `parts` partial sums by one block of 256 threads.
__device__ double block_reduce_parts(int parts, const double* __restrict__ p) {
  double s = 0.0;
  for (int i = threadIdx.x; i < parts; i += blockDim.x) s += p[i];
  s = warp_sum(s);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < 8; ++w) t += red[w];
  return t;  // valid in thread 0
}

// alpha = rho / <p, Ap>; breakdown ends the iteration.
__global__ void k_cg_alpha(int parts, const double* __restrict__ pap_parts, double* scal) {
  if (stopped(scal)) return;
  const double pAp = block_reduce_parts(parts, pap_parts);
  if (threadIdx.x == 0) {
    scal[S_PAP] = pAp;
    if (!(pAp > 1e-300)) {
      scal[S_ALPHA] = 0.0;
      scal[S_BREAK] = 1.0;
      scal[S_DONE] = 1.0;
    } else {
      scal[S_ALPHA] = scal[S_RHO] / pAp;
    }
  }
}

// x += alpha p ; res -= alpha Ap ; per-block partials of <res, res>.
__global__ void k_cg_update_x(int m, const double* scal, double* __restrict__ x, double* __restrict__ res,
                              const double* __restrict__ p, const double* __restrict__ Ap, double* __restrict__ rr) {
  if (stopped(scal)) return;
  const double al = scal[S_ALPHA];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    x[i] += al * p[i];
    const double ri = res[i] - al * Ap[i];
    res[i] = ri;
    s += ri * ri;
  }
  s = warp_sum(s);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    rr[blockIdx.x] = t;
  }
}

// Convergence test ||res||^2 <= tol^2 ||b||^2 and iteration count.
__global__ void k_cg_check(int parts, const double* __restrict__ rr_parts, double* scal) {
  if (stopped(scal)) return;
  const double rr = block_reduce_parts(parts, rr_parts);
  if (threadIdx.x == 0) {
    scal[S_RR] = rr;
    scal[S_ITERS] += 1.0;
    if (rr <= scal[S_TOL2]) scal[S_DONE] = 1.0;
  }
}

// per-block partials of <a, b>
__global__ void k_dot_parts(int m, const double* __restrict__ a, const double* __restrict__ b,
                            double* __restrict__ parts, const double* scal) {
  if (stopped(scal)) return;
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) s += a[i] * b[i];
  s = warp_sum(s);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    parts[blockIdx.x] = t;
  }
}

// beta = rho_new / rho ; rho = rho_new
__global__ void k_cg_beta(int parts, const double* __restrict__ rz_parts, double* scal) {
  if (stopped(scal)) return;
  const double rn = block_reduce_parts(parts, rz_parts);
  if (threadIdx.x == 0) {
    if (rn == 0.0 || scal[S_RHO] == 0.0) {
      scal[S_BETA] = 0.0;
      scal[S_BREAK] = 1.0;
      scal[S_DONE] = 1.0;
    } else {
      scal[S_BETA] = rn / scal[S_RHO];
    }
    scal[S_RHO] = rn;
  }
}

// p = z + beta p
__global__ void k_cg_update_p(int m, const double* scal, const double* __restrict__ z, double* __restrict__ p) {
  if (stopped(scal)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) p[i] = z[i] + scal[S_BETA] * p[i];
}

// set-up: rho = <res, z> , bb = <b, b>, tol2 = tol^2 bb, done = (bb == 0)
__global__ void k_cg_init(int parts, const double* __restrict__ rz_parts, const double* __restrict__ bb_parts,
                          double tol, double* scal) {
  const double rz = block_reduce_parts(parts, rz_parts);
  __syncthreads();
  const double bb = block_reduce_parts(parts, bb_parts);
  if (threadIdx.x == 0) {
    scal[S_RHO] = rz;
    scal[S_BB] = bb;
    scal[S_TOL2] = tol * tol * bb;
    scal[S_RR] = bb;
    scal[S_ITERS] = 0.0;
    scal[S_BREAK] = 0.0;
    scal[S_DONE] = (bb == 0.0) ? 1.0 : 0.0;
  }
}

constexpr int kVecBlocks = 64;

// Resident blocks of k_gemv_t_f32 on the whole device (one wave).
int gemv_t_wave() {
  static int wave = 0;
  if (!wave) {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 152;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gemv_t_f32, 256, 0) != cudaSuccess || per < 1) per = 4;
    cudaGetLastError();
    wave = nsm * per;
  }
  return wave;
}

dngd_status gemv_t_f32_s(int m, int n, const float* A, long long lda, const double* x, double alpha, double* y,
                         double* partials, long long partial_cap, float2* xs, const double* scal,
                         cudaStream_t st) {
  const int mpad = (m + 3) & ~3;
  DNGD_NOTE_LAUNCH();
  k_split_vec<<<cdiv(mpad, 256), 256, 0, st>>>(m, mpad, x, xs, scal);
  // row splits: as many as fill one wave of resident blocks (a second, partly
  // filled wave would leave the memory system idle at its end)
  const int gx = cdiv(n, 1024);
  int splits = max(1, gemv_t_wave() / gx);
  splits = min(splits, max(1, m / 16));
  while (splits > 1 && (long long)splits * n > partial_cap) --splits;
  const int rows = cdiv(m, splits);
  splits = cdiv(m, rows);
  DNGD_NOTE_LAUNCH();
  k_gemv_t_f32<<<dim3(gx, splits), 256, 0, st>>>(m, n, A, lda, xs, rows, partials, scal);
  DNGD_NOTE_LAUNCH();
  k_reduce_splits<<<cdiv(n, 256), 256, 0, st>>>(n, splits, partials, alpha, y, scal);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

dngd_status gemv_n_f32_s(int m, int n, const float* A, long long lda, const double* x, double alpha, double* y,
                         const double* add, double add_scale, float2* xs, const double* dotw, double* dotp,
                         const double* scal, cudaStream_t st) {
  const int npad = (n + 3) & ~3;
  DNGD_NOTE_LAUNCH();
  k_split_vec<<<cdiv(npad, 256), 256, 0, st>>>(n, npad, x, xs, scal);
  DNGD_NOTE_LAUNCH();
  k_gemv_n_f32<<<cdiv(m, kRows), 256, 0, st>>>(m, n, A, lda, xs, alpha, add, add_scale, y, dotw, dotp, scal);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// z = Linv^T (Linv q)
dngd_status precond(const PcgMixed& P, const double* q, double* z, cudaStream_t st) {
  dngd_status s = gemv_n_f32_s(P.m, P.m, P.Linv, P.ldk, q, 1.0, P.y, nullptr, 0.0, P.xs, nullptr, nullptr, P.scal,
                               st);
  if (s) return s;
  return gemv_t_f32_s(P.m, P.m, P.Linv, P.ldk, P.y, 1.0, z, P.partials, P.partial_cap, P.xs, P.scal, st);
}

}  // namespace

void gemv_init() { gemv_t_wave(); }

dngd_status gemv_t_f32(int m, int n, const float* A, long long lda, const double* x, double alpha, double* y,
                       double* partials, long long partial_cap, float2* xs, cudaStream_t st) {
  return gemv_t_f32_s(m, n, A, lda, x, alpha, y, partials, partial_cap, xs, nullptr, st);
}

dngd_status gemv_n_f32(int m, int n, const float* A, long long lda, const double* x, double alpha, double* y,
                       const double* add, double add_scale, float2* xs, cudaStream_t st) {
  return gemv_n_f32_s(m, n, A, lda, x, alpha, y, add, add_scale, xs, nullptr, nullptr, nullptr, st);
}

namespace {

// One PCG iteration (no-ops once the device "done" flag is set).
dngd_status pcg_iteration(const PcgMixed& P, double* x, bool timed, cudaStream_t st) {
  const int m = P.m;
  double* sc = P.scal;
  double* part_a = P.dotp;
  double* part_b = P.dotp + 512;
  double* pap_parts = P.dotp + 1024;
  const int nAp = cdiv(m, kRows);
  dngd_status s;
  if (P.K64) {
    // Ap = K p + lambda p with the exact Gram, block partials of <p, Ap>
    DNGD_NOTE_LAUNCH();
    k_gemv_n_df<<<cdiv(m, kRows), 256, 0, st>>>(m, m, P.K64, P.ldk64, P.p, P.p, P.lambda, P.Ap, P.p, pap_parts, sc);
    DNGD_LAUNCH_CHECK();
  } else {
    // Ap = J (J^T p) + lambda p, with the block partials of <p, Ap>
    if (timed) cudaEventRecord(P.ev[0], st);
    if ((s = gemv_t_f32_s(m, P.n, P.J, P.ldJ, P.p, 1.0, P.u, P.partials, P.partial_cap, P.xs, sc, st))) return s;
    if (timed) cudaEventRecord(P.ev[1], st);
    if ((s = gemv_n_f32_s(m, P.n, P.J, P.ldJ, P.u, 1.0, P.Ap, P.p, P.lambda, P.xs, P.p, pap_parts, sc, st)))
      return s;
    if (timed) cudaEventRecord(P.ev[2], st);
  }
  DNGD_NOTE_LAUNCH();
  k_cg_alpha<<<1, 256, 0, st>>>(nAp, pap_parts, sc);
  DNGD_NOTE_LAUNCH();
  k_cg_update_x<<<kVecBlocks, 256, 0, st>>>(m, sc, x, P.res, P.p, P.Ap, part_a);
  DNGD_NOTE_LAUNCH();
  k_cg_check<<<1, 256, 0, st>>>(kVecBlocks, part_a, sc);
  if ((s = precond(P, P.res, P.z, st))) return s;
  DNGD_NOTE_LAUNCH();
  k_dot_parts<<<kVecBlocks, 256, 0, st>>>(m, P.res, P.z, part_b, sc);
  DNGD_NOTE_LAUNCH();
  k_cg_beta<<<1, 256, 0, st>>>(kVecBlocks, part_b, sc);
  DNGD_NOTE_LAUNCH();
  k_cg_update_p<<<cdiv(m, 256), 256, 0, st>>>(m, sc, P.z, P.p);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

}  // namespace

dngd_status pcg_mixed_solve(const PcgMixed& P, const double* b, double* x, double tol, int maxit, int check_every,
                            int* iters, double* relres, cudaStream_t st, bool async, int slot) {
  if (!async && P.K64 && P.LinvT && P.pstate && P.pwork) {
    const dngd_status ps = pcg_persist_solve(P.m, P.K64, P.ldk64, P.lambda, P.Linv, P.LinvT, P.ldk, b, x, P.pwork,
                                             P.partials, P.partial_cap, P.scal, tol, maxit, P.pstate, P.status, st);
    if (ps == DNGD_OK) {
      double* sc = P.scal;
      const int rec = slot == 0 ? S_IT0 : S_IT1;
      DNGD_CUDA_CHECK(cudaMemcpyAsync(sc + rec, sc + S_ITERS, sizeof(double), cudaMemcpyDeviceToDevice, st));
      DNGD_CUDA_CHECK(cudaMemcpyAsync(sc + rec + 1, sc + S_RR, sizeof(double), cudaMemcpyDeviceToDevice, st));
      DNGD_CUDA_CHECK(cudaMemcpyAsync(sc + rec + 2, sc + S_BB, sizeof(double), cudaMemcpyDeviceToDevice, st));
      DNGD_CUDA_CHECK(cudaMemcpyAsync(P.scal_h, sc, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st));
      DNGD_CUDA_CHECK(cudaStreamSynchronize(st));
      const double bb = P.scal_h[S_BB];
      *iters = (int)P.scal_h[S_ITERS];
      *relres = bb > 0 ? sqrt(P.scal_h[S_RR] / bb) : 0.0;
      return DNGD_OK;
    }
    if (ps != DNGD_ERR_INVALID_ARG) return ps;
  }
  const int m = P.m;
  double* sc = P.scal;
  double* part_a = P.dotp;          // kVecBlocks partials
  double* part_b = P.dotp + 512;    // kVecBlocks partials
  dngd_status s;
  DNGD_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * m, st));
  DNGD_CUDA_CHECK(cudaMemcpyAsync(P.res, b, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
  DNGD_CUDA_CHECK(cudaMemsetAsync(sc + S_DONE, 0, sizeof(double), st));
  // z = M^{-1} res, p = z, rho = <res, z>, bb = <b, b>
  if ((s = precond(P, P.res, P.z, st))) return s;
  DNGD_CUDA_CHECK(cudaMemcpyAsync(P.p, P.z, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
  DNGD_NOTE_LAUNCH();
  k_dot_parts<<<kVecBlocks, 256, 0, st>>>(m, P.res, P.z, part_a, nullptr);
  DNGD_NOTE_LAUNCH();
  k_dot_parts<<<kVecBlocks, 256, 0, st>>>(m, b, b, part_b, nullptr);
  DNGD_NOTE_LAUNCH();
  k_cg_init<<<1, 256, 0, st>>>(kVecBlocks, part_a, part_b, tol, sc);
  DNGD_LAUNCH_CHECK();
  const int nAp = cdiv(m, kRows);
  double* pap_parts = P.dotp + 1024;  // m / 4 partials of <p, Ap>
  int it = 0;
  for (;;) {
    const int chunk = check_every > 0 ? check_every : 4;
    const bool timed = P.ev && it == 0;
    if (!async && P.chunk_exec && !timed && it + chunk <= maxit) {
      // the chunk of iterations as one captured graph (cached per solve
      // slot and lambda): one launch instead of ~12 per iteration
      const double xkey = (double)(uintptr_t)x;
      if (!*P.chunk_exec || P.chunk_key[0] != P.lambda || P.chunk_key[1] != (double)chunk || P.chunk_key[3] != xkey) {
        if (*P.chunk_exec) {
          cudaGraphExecDestroy(*P.chunk_exec);
          *P.chunk_exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        const unsigned long long n0 = dngd_launch_count();
        DNGD_CUDA_CHECK(cudaStreamBeginCapture(P.cap, cudaStreamCaptureModeThreadLocal));
        dngd_status cs = DNGD_OK;
        for (int k = 0; k < chunk && !cs; ++k) cs = pcg_iteration(P, x, false, P.cap);
        const cudaError_t e = cudaStreamEndCapture(P.cap, &g);
        P.chunk_key[2] = (double)(dngd_launch_count() - n0);
        if (cs) {
          if (g) cudaGraphDestroy(g);
          return cs;
        }
        DNGD_CUDA_CHECK(e);
        DNGD_CUDA_CHECK(cudaGraphInstantiate(P.chunk_exec, g, 0));
        cudaGraphDestroy(g);
        P.chunk_key[0] = P.lambda;
        P.chunk_key[1] = (double)chunk;
        P.chunk_key[3] = xkey;
      }
      DNGD_CUDA_CHECK(cudaGraphLaunch(*P.chunk_exec, st));
      for (int k = 0; k < (int)P.chunk_key[2]; ++k) note_launch();
      it += chunk;
    } else {
      for (int k = 0; k < chunk && it < maxit; ++k, ++it)
        if ((s = pcg_iteration(P, x, P.ev && it == 0, st))) return s;
    }
    if (async) {
      if (it >= maxit) break;
      continue;
    }
    DNGD_CUDA_CHECK(cudaMemcpyAsync(P.scal_h, sc, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st));
    DNGD_CUDA_CHECK(cudaStreamSynchronize(st));
    if (P.scal_h[S_DONE] != 0.0 || it >= maxit) break;
  }
  // per-solve record: iterations, ||res||^2, ||b||^2
  const int rec = slot == 0 ? S_IT0 : S_IT1;
  DNGD_CUDA_CHECK(cudaMemcpyAsync(sc + rec, sc + S_ITERS, sizeof(double), cudaMemcpyDeviceToDevice, st));
  DNGD_CUDA_CHECK(cudaMemcpyAsync(sc + rec + 1, sc + S_RR, sizeof(double), cudaMemcpyDeviceToDevice, st));
  DNGD_CUDA_CHECK(cudaMemcpyAsync(sc + rec + 2, sc + S_BB, sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (async) return DNGD_OK;
  const double bb = P.scal_h[S_BB];
  *iters = (int)P.scal_h[S_ITERS];
  *relres = bb > 0 ? sqrt(P.scal_h[S_RR] / bb) : 0.0;
  return DNGD_OK;
}

}  // namespace dngd
