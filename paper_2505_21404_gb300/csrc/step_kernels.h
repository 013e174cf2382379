// Device-scalar slots and small step kernels (internal).
#pragma once

#include "common.cuh"

namespace dngd {

// Slots of the per-context device scalar array.
enum : int {
  S_NV2 = 0, S_NA2, S_RATIO, S_ACCEPT,
  S_RHO, S_RHONEW, S_PAP, S_ALPHA, S_BETA, S_BREAK, S_RR, S_BB, S_LOSS, S_TRACE,
  S_DONE, S_ITERS, S_TOL2,
  S_IT0, S_RR0, S_BB0, S_IT1, S_RR1, S_BB1,
  S_COUNT = 26
};

dngd_status to_float(long long n, const double* x, float* y, cudaStream_t st);
dngd_status axpy_to(long long n, const double* x, double eta, const double* d, double* y, cudaStream_t st);
// y_g = fl32(x + etas[g] d) for g < G <= 8 (etas on the host), y_g = y + g n.
dngd_status axpy_to_float_batch(long long n, int G, const double* x, const double* etas, const double* d, float* y,
                                cudaStream_t st);
dngd_status ga_finish(int n, const double* v, const double* a, int use_ga, double eps_norm, double ratio_max,
                      double* delta, double* scal, double* partials, int* status, cudaStream_t st);
dngd_status cg_alpha(double* scal, cudaStream_t st);
dngd_status cg_update_x(int m, const double* scal, double* x, double* res, const double* p, const double* Ap,
                        cudaStream_t st);
dngd_status cg_beta(double* scal, cudaStream_t st);
dngd_status cg_update_p(int m, const double* scal, const double* z, double* p, cudaStream_t st);
// scal_out = sum_i A[i,i]
template <typename T>
dngd_status diag_sum(int m, const T* A, long long lda, double* scal_out, cudaStream_t st);
dngd_status add_scaled(int m, double s, const double* x, double* y, cudaStream_t st);
template <typename T>
dngd_status lower_to_f64(int m, const T* A, long long lda, double* out, cudaStream_t st);
template <typename T>
dngd_status rows_to_f64(int m, long long n, const T* A, long long lda, double* out, cudaStream_t st);

// theta += eta* delta with eta* the first minimiser of losses[0..k) (out[0] =
// eta*, out[1] = its loss)
dngd_status ls_finish(long long n, int k, const double* losses, const double* etas, const int* step_flags,
                      double* out, const double* delta, double* theta, cudaStream_t st);

dngd_status gram_tc_set_shift(struct GramPlan* p, double shift);
int gram_tc_nsplit(const struct GramPlan* p);
int gram_tc_ntiles(const struct GramPlan* p);

}  // namespace dngd
