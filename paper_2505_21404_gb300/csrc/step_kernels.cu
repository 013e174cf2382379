// Small device kernels of the step: precision conversion, the geodesic
// acceleration acceptance test, and the scalar / vector updates of the
// preconditioned CG loops (all scalars stay on the device).
#include "common.cuh"
#include "kernels.h"
#include "step_kernels.h"

namespace dngd {

__global__ void k_to_float(long long n, const double* __restrict__ x, float* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

dngd_status to_float(long long n, const double* x, float* y, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_to_float<<<cdiv(n, 256), 256, 0, st>>>(n, x, y);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// theta_out = theta + eta * delta
__global__ void k_axpy_to(long long n, const double* __restrict__ x, double eta, const double* __restrict__ d,
                          double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] + eta * (d ? d[i] : 0.0);
}

dngd_status axpy_to(long long n, const double* x, double eta, const double* d, double* y, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_axpy_to<<<cdiv(n, 256), 256, 0, st>>>(n, x, eta, d, y);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// theta32_g = fl32(theta + eta_g delta) for up to 8 line-search trials
// (grid.y = trial, outputs n apart)
struct Etas8 {
  double e[8];
};
__global__ void k_axpy_to_float_batch(long long n, const double* __restrict__ x, Etas8 eta,
                                      const double* __restrict__ d, float* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[(long long)blockIdx.y * n + i] = (float)(x[i] + eta.e[blockIdx.y] * (d ? d[i] : 0.0));
}

dngd_status axpy_to_float_batch(long long n, int G, const double* x, const double* etas, const double* d, float* y,
                                cudaStream_t st) {
  if (G < 1 || G > 8) return DNGD_ERR_INVALID_ARG;
  Etas8 e = {};
  for (int g = 0; g < G; ++g) e.e[g] = etas[g];
  DNGD_NOTE_LAUNCH();
  k_axpy_to_float_batch<<<dim3(cdiv(n, 256), G), 256, 0, st>>>(n, x, e, d, y);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// GA acceptance (Alg. DenseDualSolve): scal[S_NV2], scal[S_NA2] hold ||v||^2,
// ||a||^2.  Writes ratio / accepted to scal and delta = v (+ a/2).
__global__ void k_ga_decide(double* scal, int use_ga, double eps_norm, double ratio_max) {
  const double nv = sqrt(scal[S_NV2]);
  const double na = sqrt(scal[S_NA2]);
  double ratio = nan("");
  int acc = 0;
  if (use_ga && nv > eps_norm) {
    ratio = 2.0 * na / nv;
    acc = ratio <= ratio_max ? 1 : 0;
  }
  scal[S_RATIO] = ratio;
  scal[S_ACCEPT] = (double)acc;
}

__global__ void k_ga_delta(long long n, const double* __restrict__ v, const double* __restrict__ a,
                           const double* __restrict__ scal, double* __restrict__ delta, int* status) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool acc = scal[S_ACCEPT] != 0.0;
  const double d = acc ? v[i] + 0.5 * a[i] : v[i];
  delta[i] = d;
  if (!isfinite(d)) atomicOr(status, ST_NONFINITE);
}

dngd_status ga_finish(int n, const double* v, const double* a, int use_ga, double eps_norm, double ratio_max,
                      double* delta, double* scal, double* partials, int* status, cudaStream_t st) {
  dngd_status s = dot_dev(n, v, v, scal + S_NV2, partials, st);
  if (s) return s;
  if (use_ga) {
    s = dot_dev(n, a, a, scal + S_NA2, partials, st);
    if (s) return s;
  } else {
    DNGD_CUDA_CHECK(cudaMemsetAsync(scal + S_NA2, 0, sizeof(double), st));
  }
  DNGD_NOTE_LAUNCH();
  k_ga_decide<<<1, 1, 0, st>>>(scal, use_ga, eps_norm, ratio_max);
  DNGD_NOTE_LAUNCH();
  k_ga_delta<<<cdiv(n, 256), 256, 0, st>>>(n, v, use_ga ? a : v, scal, delta, status);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// ---- preconditioned CG helpers (device scalars) ---------------------------

// alpha = rho / pAp (breakdown if pAp <= 1e-300)
__global__ void k_cg_alpha(double* scal) {
  const double pAp = scal[S_PAP];
  if (!(pAp > 1e-300)) {
    scal[S_ALPHA] = 0.0;
    scal[S_BREAK] = 1.0;
  } else {
    scal[S_ALPHA] = scal[S_RHO] / pAp;
  }
}

// x += alpha p ; res -= alpha Ap
__global__ void k_cg_update_x(int m, const double* scal, double* __restrict__ x, double* __restrict__ res,
                              const double* __restrict__ p, const double* __restrict__ Ap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double al = scal[S_ALPHA];
  x[i] += al * p[i];
  res[i] -= al * Ap[i];
}

// beta = rho_new / rho ; rho = rho_new
__global__ void k_cg_beta(double* scal) {
  const double rn = scal[S_RHONEW];
  if (rn == 0.0 || scal[S_RHO] == 0.0) {
    scal[S_BETA] = 0.0;
    scal[S_BREAK] = 1.0;
  } else {
    scal[S_BETA] = rn / scal[S_RHO];
  }
  scal[S_RHO] = rn;
}

// p = z + beta p
__global__ void k_cg_update_p(int m, const double* scal, const double* __restrict__ z, double* __restrict__ p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  p[i] = z[i] + scal[S_BETA] * p[i];
}

dngd_status cg_alpha(double* scal, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_cg_alpha<<<1, 1, 0, st>>>(scal);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}
dngd_status cg_update_x(int m, const double* scal, double* x, double* res, const double* p, const double* Ap,
                        cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_cg_update_x<<<cdiv(m, 256), 256, 0, st>>>(m, scal, x, res, p, Ap);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}
dngd_status cg_beta(double* scal, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_cg_beta<<<1, 1, 0, st>>>(scal);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}
dngd_status cg_update_p(int m, const double* scal, const double* z, double* p, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_cg_update_p<<<cdiv(m, 256), 256, 0, st>>>(m, scal, z, p);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// y = y + s * x  (s a host scalar)
__global__ void k_axpby(int m, double s, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) y[i] += s * x[i];
}
dngd_status add_scaled(int m, double s, const double* x, double* y, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_axpby<<<cdiv(m, 256), 256, 0, st>>>(m, s, x, y);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

template <typename T>
__global__ void k_diag_sum(int m, const T* __restrict__ A, long long lda, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += (double)A[(long long)i * lda + i];
  s = warp_sum(s);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

template <typename T>
dngd_status diag_sum(int m, const T* A, long long lda, double* scal_out, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_diag_sum<T><<<1, 256, 0, st>>>(m, A, lda, scal_out);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}
template dngd_status diag_sum<double>(int, const double*, long long, double*, cudaStream_t);
template dngd_status diag_sum<float>(int, const float*, long long, double*, cudaStream_t);

// Copy the lower triangle of a [m x m] matrix to float64 (upper = 0).
template <typename T>
__global__ void k_lower_to_f64(int m, const T* __restrict__ A, long long lda, double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * m) return;
  const int i = (int)(idx / m), j = (int)(idx % m);
  out[idx] = j <= i ? (double)A[(long long)i * lda + j] : 0.0;
}

template <typename T>
dngd_status lower_to_f64(int m, const T* A, long long lda, double* out, cudaStream_t st) {
  const long long tot = (long long)m * m;
  DNGD_NOTE_LAUNCH();
  k_lower_to_f64<T><<<(int)((tot + 255) / 256), 256, 0, st>>>(m, A, lda, out);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}
template dngd_status lower_to_f64<double>(int, const double*, long long, double*, cudaStream_t);
template dngd_status lower_to_f64<float>(int, const float*, long long, double*, cudaStream_t);

// Row-major [m x n] (ld) -> dense float64 [m x n]
template <typename T>
__global__ void k_rows_to_f64(int m, long long n, const T* __restrict__ A, long long lda, double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * n) return;
  const long long i = idx / n, j = idx % n;
  out[idx] = (double)A[i * lda + j];
}

template <typename T>
dngd_status rows_to_f64(int m, long long n, const T* A, long long lda, double* out, cudaStream_t st) {
  const long long tot = (long long)m * n;
  DNGD_NOTE_LAUNCH();
  k_rows_to_f64<T><<<(int)((tot + 255) / 256), 256, 0, st>>>(m, n, A, lda, out);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}
template dngd_status rows_to_f64<double>(int, long long, const double*, long long, double*, cudaStream_t);
template dngd_status rows_to_f64<float>(int, long long, const float*, long long, double*, cudaStream_t);

// Line search finish (Alg. D-NGD Workflow): eta* = the first minimiser of the
// k losses (ties go to the earlier grid point), then theta += eta* delta.
// First minimum of the trial losses over the grid (non-finite trials never
// win).  A step whose status word reports a failed factorisation, a
// non-finite value or a timeout is not applied (eta* = 0).
__global__ void k_ls_argmin(int k, const double* __restrict__ losses, const double* __restrict__ etas,
                            const int* __restrict__ step_flags, double* __restrict__ out) {
  int best = -1;
  for (int j = 0; j < k; ++j)
    if (isfinite(losses[j]) && (best < 0 || losses[j] < losses[best])) best = j;
  const bool ok = best >= 0 && (step_flags[0] & (ST_NOT_SPD | ST_NONFINITE | ST_TIMEOUT)) == 0;
  out[0] = ok ? etas[best] : 0.0;
  out[1] = ok ? losses[best] : nan("");
}

__global__ void k_ls_update(long long n, const double* __restrict__ eta, const double* __restrict__ delta,
                            double* __restrict__ theta) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && eta[0] != 0.0) theta[i] += eta[0] * delta[i];
}

dngd_status ls_finish(long long n, int k, const double* losses, const double* etas, const int* step_flags,
                      double* out, const double* delta, double* theta, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_ls_argmin<<<1, 1, 0, st>>>(k, losses, etas, step_flags, out);
  DNGD_NOTE_LAUNCH();
  k_ls_update<<<cdiv(n, 256), 256, 0, st>>>(n, out, delta, theta);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

}  // namespace dngd
