// Dense linear algebra of the dual solve: SIMT GEMMs (FP64 / FP32), the
// blocked Cholesky factorisation of K + lambda I, triangular solves and
// inverses, and the HBM-bound J^T x / J x products.
//
// All reductions use a fixed order (no atomics on floating point), so every
// result is bitwise reproducible run to run.
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace dngd {

// ---------------------------------------------------------------------------
// SIMT GEMM, register-tiled: C = alpha * A * op(B) + beta * C.
// BT = true: B is [N x K] (C = A B^T); BT = false: B is [K x N].
// ---------------------------------------------------------------------------

// COMP: compensated accumulation.  Each BK-slab of products is summed in a
// plain accumulator, then added into (acc, cmp) with Kahan compensation, so
// the error does not grow with K (used where the operator must stay
// consistent over thousands of PCG applications).
// kchunk > 0: split K; the block with blockIdx.z = z sums k in
// [z kchunk, (z + 1) kchunk) and writes C + z cz (k_sum_splits adds the
// partial products up in a fixed order).
template <typename T, int BM, int BN, int BK, int TM, int TN, bool BT, bool AT = false, bool COMP = false>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm(int M, int N, int K, T alpha, const T* __restrict__ A, long long lda, const T* __restrict__ B,
       long long ldb, T beta, T* __restrict__ C, long long ldc, int lower, const T* __restrict__ kscale = nullptr,
       int kchunk = 0, long long cz = 0) {
  constexpr int NT = (BM / TM) * (BN / TN);
  const int kb = kchunk > 0 ? (int)blockIdx.z * kchunk : 0;
  const int ke = kchunk > 0 && kb + kchunk < K ? kb + kchunk : K;
  C += (long long)blockIdx.z * cz;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
  if (lower && bn > bm + BM - 1) return;
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  T acc[TM][TN];
  T cmp[COMP ? TM : 1][COMP ? TN : 1];
  T part[COMP ? TM : 1][COMP ? TN : 1];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  if (COMP) {
#pragma unroll
    for (int i = 0; i < (COMP ? TM : 1); ++i)
#pragma unroll
      for (int j = 0; j < (COMP ? TN : 1); ++j) cmp[i][j] = T(0);
  }
  for (int k0 = kb; k0 < ke; k0 += BK) {
    if (AT) {
      // A is [K x M] row-major (C = A^T op(B)); optional per-k scale of A
#pragma unroll
      for (int e = tid; e < BM * BK; e += NT) {
        const int kk = e / BM, r = e % BM;
        const int gr = bm + r, gk = k0 + kk;
        T v = (gr < M && gk < ke) ? A[(long long)gk * lda + gr] : T(0);
        if (kscale && gk < ke) v *= kscale[gk];
        As[kk][r] = v;
      }
    } else {
#pragma unroll
      for (int e = tid; e < BM * BK; e += NT) {
        const int r = e / BK, kk = e % BK;
        const int gr = bm + r, gk = k0 + kk;
        As[kk][r] = (gr < M && gk < ke) ? A[(long long)gr * lda + gk] : T(0);
      }
    }
    if (BT) {
#pragma unroll
      for (int e = tid; e < BN * BK; e += NT) {
        const int c = e / BK, kk = e % BK;
        const int gc = bn + c, gk = k0 + kk;
        Bs[kk][c] = (gc < N && gk < ke) ? B[(long long)gc * ldb + gk] : T(0);
      }
    } else {
#pragma unroll
      for (int e = tid; e < BN * BK; e += NT) {
        const int kk = e / BN, c = e % BN;
        const int gc = bn + c, gk = k0 + kk;
        Bs[kk][c] = (gc < N && gk < ke) ? B[(long long)gk * ldb + gc] : T(0);
      }
    }
    __syncthreads();
    if (COMP) {
#pragma unroll
      for (int i = 0; i < (COMP ? TM : 1); ++i)
#pragma unroll
        for (int j = 0; j < (COMP ? TN : 1); ++j) part[i][j] = T(0);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
      if (COMP) {
#pragma unroll
        for (int i = 0; i < (COMP ? TM : 1); ++i)
#pragma unroll
          for (int j = 0; j < (COMP ? TN : 1); ++j) part[i][j] += a[i] * b[j];
      } else {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
      }
    }
    if (COMP) {
#pragma unroll
      for (int i = 0; i < (COMP ? TM : 1); ++i)
#pragma unroll
        for (int j = 0; j < (COMP ? TN : 1); ++j) {
          const T y = part[i][j] - cmp[i][j];
          const T t = acc[i][j] + y;
          cmp[i][j] = (t - acc[i][j]) - y;
          acc[i][j] = t;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gr = bm + ty * TM + i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gc = bn + tx * TN + j;
      if (gc >= N) continue;
      T* cp = C + (long long)gr * ldc + gc;
      *cp = (beta == T(0)) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *cp;
    }
  }
}

template <typename T>
struct GemmCfg;
template <>
struct GemmCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};
template <>
struct GemmCfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};

template <typename T>
dngd_status gemm_nt(int M, int N, int K, T alpha, const T* A, long long lda, const T* B, long long ldb, T beta,
                    T* C, long long ldc, bool lower, cudaStream_t st) {
  if (M <= 0 || N <= 0) return DNGD_OK;
  using G = GemmCfg<T>;
  dim3 grid(cdiv(N, G::BN), cdiv(M, G::BM));
  DNGD_NOTE_LAUNCH();
  k_gemm<T, G::BM, G::BN, G::BK, G::TM, G::TN, true>
      <<<grid, (G::BM / G::TM) * (G::BN / G::TN), 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                          lower ? 1 : 0);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// C[r][c] = sum over s = 0..S-1 (in that order) of W[s][r][c], the lower
// triangle (c <= r) of an M x M result.
__global__ void k_sum_splits(int M, int S, const double* __restrict__ W, long long ldw, long long wz,
                             double* __restrict__ C, long long ldc) {
  const int r = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= r && c < M; c += gridDim.x * blockDim.x) {
    double acc = W[(long long)r * ldw + c];
    for (int z = 1; z < S; ++z) acc += W[(long long)z * wz + (long long)r * ldw + c];
    C[(long long)r * ldc + c] = acc;
  }
}

int gram_f64_splits(int M, int K) {
  using G = GemmCfg<double>;
  const int t = cdiv(M, G::BM);
  const int tiles = t * (t + 1) / 2;                 // lower-triangle tiles
  int S = cdiv(2 * 152, tiles);                      // about two blocks per SM
  if (S > 16) S = 16;
  if (S > K / 256) S = K / 256;                      // at least 256 k per split
  return S < 1 ? 1 : S;
}

dngd_status gram_f64(bool at, int M, int K, const double* A, long long lda, double* C, long long ldc, double* ws,
                     cudaStream_t st) {
  if (M <= 0) return DNGD_OK;
  using G = GemmCfg<double>;
  const int S = ws ? gram_f64_splits(M, K) : 1;
  if (S == 1)
    return at ? gemm_tn<double>(M, M, K, 1.0, A, lda, A, lda, 0.0, C, ldc, nullptr, st, true)
              : gemm_nt<double>(M, M, K, 1.0, A, lda, A, lda, 0.0, C, ldc, true, st);
  const int kchunk = cdiv(cdiv(K, S), G::BK) * G::BK;
  const int Sz = cdiv(K, kchunk);
  const long long ldw = ldc, wz = (long long)M * ldw;
  dim3 grid(cdiv(M, G::BN), cdiv(M, G::BM), Sz);
  DNGD_NOTE_LAUNCH();
  if (at)
    k_gemm<double, G::BM, G::BN, G::BK, G::TM, G::TN, false, true>
        <<<grid, (G::BM / G::TM) * (G::BN / G::TN), 0, st>>>(M, M, K, 1.0, A, lda, A, lda, 0.0, ws, ldw, 1,
                                                            nullptr, kchunk, wz);
  else
    k_gemm<double, G::BM, G::BN, G::BK, G::TM, G::TN, true>
        <<<grid, (G::BM / G::TM) * (G::BN / G::TN), 0, st>>>(M, M, K, 1.0, A, lda, A, lda, 0.0, ws, ldw, 1,
                                                            nullptr, kchunk, wz);
  DNGD_LAUNCH_CHECK();
  DNGD_NOTE_LAUNCH();
  k_sum_splits<<<dim3(cdiv(M, 256), M), 256, 0, st>>>(M, Sz, ws, ldw, wz, C, ldc);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

template <typename T>
dngd_status gemm_nn(int M, int N, int K, T alpha, const T* A, long long lda, const T* B, long long ldb, T beta,
                    T* C, long long ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return DNGD_OK;
  using G = GemmCfg<T>;
  dim3 grid(cdiv(N, G::BN), cdiv(M, G::BM));
  DNGD_NOTE_LAUNCH();
  k_gemm<T, G::BM, G::BN, G::BK, G::TM, G::TN, false>
      <<<grid, (G::BM / G::TM) * (G::BN / G::TN), 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 0);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// C[M x N] = alpha * A^T B + beta * C with A [K x M], B [K x N] row-major and
// an optional scale of A's rows (the K index): C = A^T diag(kscale) B.
// lower: skip output tiles strictly above the diagonal (syrk-style use).
template <typename T>
dngd_status gemm_tn(int M, int N, int K, T alpha, const T* A, long long lda, const T* B, long long ldb, T beta,
                    T* C, long long ldc, const T* kscale, cudaStream_t st, bool lower) {
  if (M <= 0 || N <= 0) return DNGD_OK;
  using G = GemmCfg<T>;
  dim3 grid(cdiv(N, G::BN), cdiv(M, G::BM));
  DNGD_NOTE_LAUNCH();
  k_gemm<T, G::BM, G::BN, G::BK, G::TM, G::TN, false, true>
      <<<grid, (G::BM / G::TM) * (G::BN / G::TN), 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                          lower ? 1 : 0, kscale);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}
template dngd_status gemm_tn<float>(int, int, int, float, const float*, long long, const float*, long long, float,
                                    float*, long long, const float*, cudaStream_t, bool);

// FP32 GEMMs with compensated accumulation (64 x 128 tiles, 4 x 8 per thread).
dngd_status gemm_nt_comp(int M, int N, int K, float alpha, const float* A, long long lda, const float* B,
                         long long ldb, float beta, float* C, long long ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return DNGD_OK;
  dim3 grid(cdiv(N, 128), cdiv(M, 64));
  DNGD_NOTE_LAUNCH();
  k_gemm<float, 64, 128, 8, 4, 8, true, false, true>
      <<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 0, nullptr);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

dngd_status gemm_tn_comp(int M, int N, int K, float alpha, const float* A, long long lda, const float* B,
                         long long ldb, float beta, float* C, long long ldc, const float* kscale, cudaStream_t st) {
  if (M <= 0 || N <= 0) return DNGD_OK;
  dim3 grid(cdiv(N, 128), cdiv(M, 64));
  DNGD_NOTE_LAUNCH();
  k_gemm<float, 64, 128, 8, 4, 8, false, true, true>
      <<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 0, kscale);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}
template dngd_status gemm_tn<double>(int, int, int, double, const double*, long long, const double*, long long,
                                     double, double*, long long, const double*, cudaStream_t, bool);

template dngd_status gemm_nt<double>(int, int, int, double, const double*, long long, const double*, long long,
                                     double, double*, long long, bool, cudaStream_t);
template dngd_status gemm_nt<float>(int, int, int, float, const float*, long long, const float*, long long, float,
                                    float*, long long, bool, cudaStream_t);
template dngd_status gemm_nn<double>(int, int, int, double, const double*, long long, const double*, long long,
                                     double, double*, long long, cudaStream_t);
template dngd_status gemm_nn<float>(int, int, int, float, const float*, long long, const float*, long long, float,
                                    float*, long long, cudaStream_t);

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky (lower).  Per block column k:
//   1. factor the diagonal block in FP64 in shared memory,
//   2. panel: A21 <- A21 L11^{-T} by row-wise forward substitution,
//   3. trailing update A22 <- A22 - A21 A21^T (lower tiles, SIMT GEMM).
// ---------------------------------------------------------------------------

constexpr int kCholNB = 64;

template <typename TA>
__global__ void __launch_bounds__(256) k_potrf_diag(int k0, int kb, TA* A, long long lda, int* status) {
  __shared__ double S[kCholNB][kCholNB + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, j = e % kb;
    S[i][j] = (j <= i) ? (double)A[(long long)(k0 + i) * lda + k0 + j] : 0.0;
  }
  __syncthreads();
  __shared__ int bad;
  if (tid == 0) bad = -1;
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    const double piv = S[j][j];
    if (!(piv > 0.0)) {  // not SPD (or NaN): record and stop this block
      if (tid == 0) bad = j;
      break;
    }
    const double d = sqrt(piv);
    // thread per row i > j: scale column j, then rank-1 update of row i
    for (int i = j + 1 + tid; i < kb; i += blockDim.x) S[i][j] /= d;
    __syncthreads();
    if (tid == 0) S[j][j] = d;
    for (int i = j + 1 + tid; i < kb; i += blockDim.x) {
      const double lij = S[i][j];
      for (int c = j + 1; c <= i; ++c) S[i][c] -= lij * S[c][j];
    }
    __syncthreads();
  }
  __syncthreads();
  if (bad >= 0) {
    if (tid == 0) {
      const int old = atomicOr(status, ST_NOT_SPD);
      if (!(old & ST_NOT_SPD)) status[1] = k0 + bad;
    }
    return;
  }
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, j = e % kb;
    if (j <= i) A[(long long)(k0 + i) * lda + k0 + j] = (TA)S[i][j];
  }
}

// Panel rows i in [k0+kb, m): x L11^T = a, solved left to right; one thread
// per row, the row kept in shared memory.
template <typename TA>
__global__ void __launch_bounds__(64) k_trsm_panel(int m, int k0, int kb, TA* A, long long lda,
                                                    const int* status) {
  if (status[0] & ST_NOT_SPD) return;
  extern __shared__ unsigned char trsm_smem[];
  TA(*Lsh)[kCholNB + 1] = reinterpret_cast<TA(*)[kCholNB + 1]>(trsm_smem);
  TA(*X)[kCholNB + 1] = Lsh + kCholNB;
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, j = e % kb;
    Lsh[i][j] = (j <= i) ? A[(long long)(k0 + i) * lda + k0 + j] : TA(0);
  }
  const int r0 = k0 + kb + blockIdx.x * 64;
  for (int e = tid; e < 64 * kb; e += blockDim.x) {
    const int rr = e / kb, j = e % kb;
    const int gr = r0 + rr;
    X[rr][j] = (gr < m) ? A[(long long)gr * lda + k0 + j] : TA(0);
  }
  __syncthreads();
  const int gr = r0 + tid;
  if (gr < m) {
    for (int j = 0; j < kb; ++j) {
      TA s = X[tid][j];
      for (int p = 0; p < j; ++p) s -= X[tid][p] * Lsh[j][p];
      X[tid][j] = s / Lsh[j][j];
    }
  }
  __syncthreads();
  for (int e = tid; e < 64 * kb; e += blockDim.x) {
    const int rr = e / kb, j = e % kb;
    const int g = r0 + rr;
    if (g < m) A[(long long)g * lda + k0 + j] = X[rr][j];
  }
}

template <typename TA>
dngd_status cholesky(int m, TA* A, long long lda, int* status, double* work, cudaStream_t st) {
  (void)work;
  const int trsm_smem = 2 * kCholNB * (kCholNB + 1) * (int)sizeof(TA);
  static bool attr_set = false;
  if (!attr_set) {
    DNGD_CUDA_CHECK(cudaFuncSetAttribute(k_trsm_panel<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, trsm_smem));
    attr_set = true;
  }
  for (int k0 = 0; k0 < m; k0 += kCholNB) {
    const int kb = (m - k0) < kCholNB ? (m - k0) : kCholNB;
    DNGD_NOTE_LAUNCH();
    k_potrf_diag<TA><<<1, 256, 0, st>>>(k0, kb, A, lda, status);
    DNGD_LAUNCH_CHECK();
    const int rest = m - k0 - kb;
    if (rest <= 0) break;
    DNGD_NOTE_LAUNCH();
    k_trsm_panel<TA><<<cdiv(rest, 64), 64, trsm_smem, st>>>(m, k0, kb, A, lda, status);
    DNGD_LAUNCH_CHECK();
    TA* P = A + (long long)(k0 + kb) * lda + k0;
    TA* A22 = A + (long long)(k0 + kb) * lda + k0 + kb;
    dngd_status s = gemm_nt<TA>(rest, rest, kb, TA(-1), P, lda, P, lda, TA(1), A22, lda, true, st);
    if (s) return s;
  }
  return DNGD_OK;
}

template dngd_status cholesky<double>(int, double*, long long, int*, double*, cudaStream_t);

// ---------------------------------------------------------------------------
// FP32 factorisation for the mixed path (a preconditioner, whose accuracy the
// refinement restores).  One kernel factors a 64 x 64 diagonal block and
// builds its inverse; the panel solve is then a GEMM with that inverse, and
// the inverse fills the diagonal blocks of the explicit L^{-1}.
//
// The 64-block is taken as 2 x 2 blocks of 32: one warp factors a 32 x 32
// diagonal block in registers (lane i holds row i of the block and of its
// inverse; column j's entries travel by warp shuffles, so no block barrier
// per column), and the rest are 32 x 32 products over the whole CTA:
// L10 = S10 Y00^T, S11 -= L10 L10^T, and (L^{-1})10 = -Y11 (L10 Y00).
// ---------------------------------------------------------------------------

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u = (u + 0x1000u) & 0xFFFFE000u;
  return __uint_as_float(u);
}

// Cholesky of a 32 x 32 SPD block held by one warp (a[c] = S[lane][c] for
// c <= lane, zero above): on return a holds row `lane` of L and y row `lane`
// of L^{-1}.  Column J: the pivot, column J of L, row J of the inverse
// (scaled), the rank-1 update of the trailing rows, and the elimination of
// column J from the inverse rows below.  A non-positive pivot is recorded in
// `bad` (the same in every lane) and the remaining columns run on, their
// values unused.  The column index is a template parameter so that every
// register index is static.
template <int J>
__device__ __forceinline__ void chol32_col(float (&a)[32], float (&y)[32], int lane, int& bad) {
  const unsigned full = 0xffffffffu;
  const float piv = __shfl_sync(full, a[J], J);
  if (!(piv > 0.f) && bad < 0) bad = J;
  // the column's chain runs through this pivot: one hardware reciprocal
  // square root (a preconditioner needs no correctly rounded sqrt)
  const float inv_d = rsqrtf(piv);
  const float d = piv * inv_d;
  if (lane > J) a[J] *= inv_d;
  if (lane == J) {
    a[J] = d;
#pragma unroll
    for (int c = 0; c <= J; ++c) y[c] *= inv_d;
  }
#pragma unroll
  for (int c = J + 1; c < 32; ++c) {
    const float lc = __shfl_sync(full, a[J], c);
    if (lane >= c) a[c] -= a[J] * lc;
  }
#pragma unroll
  for (int c = 0; c <= J; ++c) {
    const float yc = __shfl_sync(full, y[c], J);
    if (lane > J) y[c] -= a[J] * yc;
  }
  if constexpr (J + 1 < 32) chol32_col<J + 1>(a, y, lane, bad);
}

// Returns -1, or the first column whose pivot is not positive.
__device__ __forceinline__ int warp_chol32_inv(float (&a)[32], float (&y)[32], int lane) {
  int bad = -1;
#pragma unroll
  for (int c = 0; c < 32; ++c) y[c] = (c == lane) ? 1.f : 0.f;
  chol32_col<0>(a, y, lane, bad);
  return bad;
}

// Grid: 1 + ceil(rest / 64) CTAs.  CTA 0 stores the block's inverse into
// Linv; CTA b >= 1 solves panel rows k0 + kb + 64 (b - 1) .. (+64) and, with
// asplit given, also writes them as the trailing update's split A operand
// (row r of the panel: TF32 hi of its kp = kb rounded up to 32 values, then
// lo; zero beyond kb).  The factored block itself goes back into A from the
// last CTA to have read it (status[3] counts the arrivals).
__global__ void __launch_bounds__(256) k_potrf_inv_f32(int k0, int kb, float* A, long long lda, float* Linv,
                                                        long long ldi, int rest, float* asplit, int* status) {
  __shared__ float S[kCholNB][kCholNB + 1];
  __shared__ float X[kCholNB][kCholNB + 1];
  __shared__ float T[32][33];
  __shared__ int bad;
  if (status[0] & ST_NOT_SPD) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // lower triangle of the block; rows past kb are identity rows
  for (int e = tid; e < kCholNB * kCholNB; e += blockDim.x) {
    const int i = e / kCholNB, j = e % kCholNB;
    S[i][j] = (i < kb && j <= i) ? A[(long long)(k0 + i) * lda + k0 + j] : (i == j ? 1.f : 0.f);
    X[i][j] = 0.f;
  }
  if (tid == 0) bad = -1;
  __syncthreads();
  // every CTA computes the same factor; the diagonal block of A is
  // overwritten with it only by the last CTA to have read the block, so no
  // CTA that starts late reads a half-written block (status[3] counts the
  // arrivals and is zero again once the last one has arrived)
  __shared__ int writer;
  if (tid == 0) {
    const int old = atomicAdd(status + 3, 1);
    writer = (old == (int)gridDim.x - 1) ? 1 : 0;
    if (writer) status[3] = 0;
  }
  // 2 x 2 output elements per thread in the 32 x 32 products
  const int r0 = 2 * (tid >> 4), c0 = 2 * (tid & 15);
  for (int half = 0; half < 2; ++half) {
    const int o = 32 * half;
    if (warp == 0) {
      float a[32], y[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) a[c] = (c <= lane) ? S[o + lane][o + c] : 0.f;
      const int b = warp_chol32_inv(a, y, lane);
      if (b >= 0) {
        if (lane == 0) bad = o + b;
      } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          S[o + lane][o + c] = (c <= lane) ? a[c] : 0.f;
          X[o + lane][o + c] = (c <= lane) ? y[c] : 0.f;
        }
      }
    }
    __syncthreads();
    if (bad >= 0) break;
    if (half == 1) break;
    // L10 = S10 Y00^T
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float s0 = S[32 + r0][k], s1 = S[33 + r0][k];
      const float y0 = X[c0][k], y1 = X[c0 + 1][k];
      acc[0][0] += s0 * y0;
      acc[0][1] += s0 * y1;
      acc[1][0] += s1 * y0;
      acc[1][1] += s1 * y1;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) S[32 + r0 + p][c0 + q] = acc[p][q];
    __syncthreads();
    // S11 -= L10 L10^T (lower triangle)
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) acc[p][q] = 0.f;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float l0 = S[32 + r0][k], l1 = S[33 + r0][k];
      const float m0 = S[32 + c0][k], m1 = S[33 + c0][k];
      acc[0][0] += l0 * m0;
      acc[0][1] += l0 * m1;
      acc[1][0] += l1 * m0;
      acc[1][1] += l1 * m1;
    }
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q)
        if (c0 + q <= r0 + p) S[32 + r0 + p][32 + c0 + q] -= acc[p][q];
    __syncthreads();
  }
  if (bad >= 0) {
    if (blockIdx.x == 0 && tid == 0 && bad < kb) {
      const int old = atomicOr(status, ST_NOT_SPD);
      if (!(old & ST_NOT_SPD)) status[1] = k0 + bad;
    }
    return;
  }
  // (L^{-1})10 = -Y11 (L10 Y00)
  {
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float l0 = S[32 + r0][k], l1 = S[33 + r0][k];
      const float y0 = X[k][c0], y1 = X[k][c0 + 1];
      acc[0][0] += l0 * y0;
      acc[0][1] += l0 * y1;
      acc[1][0] += l1 * y0;
      acc[1][1] += l1 * y1;
    }
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) T[r0 + p][c0 + q] = acc[p][q];
    __syncthreads();
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) acc[p][q] = 0.f;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float y0 = X[32 + r0][32 + k], y1 = X[33 + r0][32 + k];
      const float t0 = T[k][c0], t1 = T[k][c0 + 1];
      acc[0][0] += y0 * t0;
      acc[0][1] += y0 * t1;
      acc[1][0] += y1 * t0;
      acc[1][1] += y1 * t1;
    }
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) X[32 + r0 + p][c0 + q] = -acc[p][q];
    __syncthreads();
  }
  if (writer) {
    for (int e = tid; e < kCholNB * kCholNB; e += blockDim.x) {
      const int i = e / kCholNB, c = e % kCholNB;
      if (i < kb && c <= i) A[(long long)(k0 + i) * lda + k0 + c] = S[i][c];
    }
  }
  if (blockIdx.x == 0) {
    for (int e = tid; e < kCholNB * kCholNB; e += blockDim.x) {
      const int i = e / kCholNB, c = e % kCholNB;
      if (i < kb && c < kb) Linv[(long long)(k0 + i) * ldi + k0 + c] = (c <= i) ? X[i][c] : 0.f;
    }
    return;
  }
  __syncthreads();   // S is reused for the panel rows below
  // CTA b >= 1: panel rows k0 + kb + 64 (b - 1) .. (+64): P <- P L11^{-T}
  // (P[r][c] = sum_{k <= c} P[r][k] X[c][k]), written back into A and, for
  // the trailing update, as its split A operand (rows from the panel's first
  // row, 2 kp floats each: TF32 hi, then lo)
  const int kp = (kb + 31) & ~31;
  const int rb0 = (blockIdx.x - 1) * kCholNB;
  const int nr = min(kCholNB, rest - rb0);
  const long long grow0 = (long long)k0 + kb + rb0;
  for (int e = tid; e < kCholNB * kCholNB; e += blockDim.x) {
    const int i = e / kCholNB, c = e % kCholNB;
    S[i][c] = (i < nr && c < kb) ? A[(grow0 + i) * lda + k0 + c] : 0.f;
  }
  __syncthreads();
  // 4 x 4 outputs per thread: rows 4 (tid / 16) .., columns (tid % 16) + 16 q
  const int rr = 4 * (tid >> 4), cc = tid & 15;
  float acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
#pragma unroll 4
  for (int k = 0; k < kCholNB; ++k) {
    float pv[4], xv[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) pv[p] = S[rr + p][k];
#pragma unroll
    for (int q = 0; q < 4; ++q) xv[q] = X[cc + 16 * q][k];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] += pv[p] * xv[q];
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = rr + p;
    if (i >= nr) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = cc + 16 * q;
      if (c < kb) A[(grow0 + i) * lda + k0 + c] = acc[p][q];
      if (asplit && c < kp) {
        const float x = c < kb ? acc[p][q] : 0.f;
        const float hi = tf32_round(x);
        float* sp = asplit + (long long)(rb0 + i) * 2 * kp;
        sp[c] = hi;
        sp[kp + c] = tf32_round(x - hi);
      }
    }
  }
}

// A 64-column step is two launches: the block factor with the panel solve
// (every CTA factors the 64 x 64 diagonal block and its inverse, CTA 0 stores
// them, CTA b >= 1 solves 64 panel rows in FP32 and also writes them as the
// trailing update's split operand), then the trailing update.
dngd_status cholesky_f32_inv(int m, float* A, long long lda, float* Linv, long long ldi, int* status,
                             cudaStream_t st, const Tc3Scratch* tc3) {
  const bool tc = tc3 && tc3->buf && tc3_scratch_bytes(m, m, kCholNB) <= tc3->bytes;
  float *a_half = nullptr, *b_half = nullptr;
  if (tc) tc3_halves(*tc3, &a_half, &b_half);
  for (int k0 = 0; k0 < m; k0 += kCholNB) {
    const int kb = (m - k0) < kCholNB ? (m - k0) : kCholNB;
    const int rest = m - k0 - kb;
    DNGD_NOTE_LAUNCH();
    k_potrf_inv_f32<<<1 + cdiv(rest, kCholNB), 256, 0, st>>>(k0, kb, A, lda, Linv, ldi, rest,
                                                              (tc && rest > 0) ? a_half : nullptr, status);
    DNGD_LAUNCH_CHECK();
    if (rest <= 0) break;
    float* P = A + (long long)(k0 + kb) * lda + k0;
    float* A22 = A + (long long)(k0 + kb) * lda + k0 + kb;
    // trailing update A22 -= P P^T (lower); the tensor-core form reads P from
    // the split the panel solve wrote
    dngd_status s = tc ? gemm_tc3(rest, rest, kb, -1.0f, P, lda, false, P, lda, false, 1.0f, A22, lda, true, *tc3,
                                  status, st, TC3_A_PRESPLIT)
                       : gemm_nt<float>(rest, rest, kb, -1.0f, P, lda, P, lda, 1.0f, A22, lda, true, st);
    if (s) return s;
  }
  return DNGD_OK;
}

// ---------------------------------------------------------------------------
// Triangular solves with the FP64 factor, blocked: one small kernel solves a
// diagonal block, a second applies that block to the remaining rows.
// ---------------------------------------------------------------------------

constexpr int kTrsvNB = 64;

// forward: x[k0:k0+kb] = L_blk^{-1} x[k0:k0+kb]
// backward: x[k0:k0+kb] = L_blk^{-T} x[k0:k0+kb]
__global__ void k_trsv_diag(int k0, int kb, const double* __restrict__ L, long long ldl, double* x, int trans) {
  __shared__ double Ls[kTrsvNB][kTrsvNB + 1];
  __shared__ double xs[kTrsvNB];
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, j = e % kb;
    Ls[i][j] = (j <= i) ? L[(long long)(k0 + i) * ldl + k0 + j] : 0.0;
  }
  for (int i = tid; i < kb; i += blockDim.x) xs[i] = x[k0 + i];
  __syncthreads();
  if (!trans) {
    for (int j = 0; j < kb; ++j) {
      const double xj = xs[j] / Ls[j][j];
      __syncthreads();
      if (tid == 0) xs[j] = xj;
      for (int i = j + 1 + tid; i < kb; i += blockDim.x) xs[i] -= Ls[i][j] * xj;
      __syncthreads();
    }
  } else {
    for (int j = kb - 1; j >= 0; --j) {
      const double xj = xs[j] / Ls[j][j];
      __syncthreads();
      if (tid == 0) xs[j] = xj;
      for (int i = tid; i < j; i += blockDim.x) xs[i] -= Ls[j][i] * xj;
      __syncthreads();
    }
  }
  for (int i = tid; i < kb; i += blockDim.x) x[k0 + i] = xs[i];
}

// forward update: x[i] -= sum_{j in blk} L[i,j] x[j] for i >= k0+kb (warp per row)
__global__ void k_trsv_upd_fwd(int m, int k0, int kb, const double* __restrict__ L, long long ldl, double* x) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int i = k0 + kb + warp;
  if (i >= m) return;
  double s = 0.0;
  for (int j = lane; j < kb; j += 32) s += L[(long long)i * ldl + k0 + j] * x[k0 + j];
  s = warp_sum(s);
  if (lane == 0) x[i] -= s;
}

// backward update: x[i] -= sum_{j in blk} L[j,i] x[j] for i < k0 (thread per i)
__global__ void k_trsv_upd_bwd(int k0, int kb, const double* __restrict__ L, long long ldl, double* x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k0) return;
  double s = 0.0;
  for (int j = 0; j < kb; ++j) s += L[(long long)(k0 + j) * ldl + i] * x[k0 + j];
  x[i] -= s;
}

dngd_status chol_solve_f64(int m, const double* L, long long ldl, const double* b, double* x, cudaStream_t st) {
  if (x != b) DNGD_CUDA_CHECK(cudaMemcpyAsync(x, b, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
  for (int k0 = 0; k0 < m; k0 += kTrsvNB) {
    const int kb = (m - k0) < kTrsvNB ? (m - k0) : kTrsvNB;
    DNGD_NOTE_LAUNCH();
    k_trsv_diag<<<1, 64, 0, st>>>(k0, kb, L, ldl, x, 0);
    const int rest = m - k0 - kb;
    if (rest > 0) {
      DNGD_NOTE_LAUNCH();
      k_trsv_upd_fwd<<<cdiv((long long)rest * 32, 256), 256, 0, st>>>(m, k0, kb, L, ldl, x);
    }
  }
  const int nblk = cdiv(m, kTrsvNB);
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int k0 = bi * kTrsvNB;
    const int kb = (m - k0) < kTrsvNB ? (m - k0) : kTrsvNB;
    DNGD_NOTE_LAUNCH();
    k_trsv_diag<<<1, 64, 0, st>>>(k0, kb, L, ldl, x, 1);
    if (k0 > 0) {
      DNGD_NOTE_LAUNCH();
      k_trsv_upd_bwd<<<cdiv(k0, 128), 128, 0, st>>>(k0, kb, L, ldl, x);
    }
  }
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// ---------------------------------------------------------------------------
// Faster FP64 triangular solves: the inverses of the 64 x 64 diagonal blocks
// of L are formed once per factorisation, and each block step is one launch
// that applies the block inverse (a 64 x 64 GEMV, recomputed by every CTA)
// and updates the rows still to be solved.
// ---------------------------------------------------------------------------

// Dinv[b] = inverse of the diagonal block b of L (64 x 64, lower; thread per
// column, forward substitution on the identity).
__global__ void __launch_bounds__(64) k_trtri_diag64(int m, const double* __restrict__ L, long long ldl,
                                                     double* __restrict__ Dinv) {
  __shared__ double Ls[kTrsvNB][kTrsvNB + 1];
  __shared__ double Xs[kTrsvNB][kTrsvNB + 1];
  const int k0 = blockIdx.x * kTrsvNB;
  const int kb = min(kTrsvNB, m - k0);
  const int c = threadIdx.x;
  for (int e = c; e < kTrsvNB * kTrsvNB; e += blockDim.x) {
    const int i = e / kTrsvNB, j = e % kTrsvNB;
    Ls[i][j] = (i < kb && j <= i) ? L[(long long)(k0 + i) * ldl + k0 + j] : (i == j ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int i = 0; i < kTrsvNB; ++i) {
    double s = (i == c) ? 1.0 : 0.0;
    for (int p = c; p < i; ++p) s -= Ls[i][p] * Xs[p][c];
    Xs[i][c] = (i >= c) ? s / Ls[i][i] : 0.0;
  }
  __syncthreads();
  double* D = Dinv + (long long)blockIdx.x * kTrsvNB * kTrsvNB;
  for (int e = c; e < kTrsvNB * kTrsvNB; e += blockDim.x) D[e] = Xs[e / kTrsvNB][e % kTrsvNB];
}

// Forward block step: y_blk = Dinv_k w_blk; w_i -= L[i, blk] y_blk for the
// rows i >= k0 + kb this CTA owns (warp per row).  w_blk is only read here.
__global__ void __launch_bounds__(256) k_trsv_fwd_step(int m, int k0, int kb, const double* __restrict__ L,
                                                       long long ldl, const double* __restrict__ D,
                                                       double* __restrict__ w, double* __restrict__ y) {
  __shared__ double xb[kTrsvNB], yb[kTrsvNB];
  const int tid = threadIdx.x;
  if (tid < kTrsvNB) xb[tid] = tid < kb ? w[k0 + tid] : 0.0;
  __syncthreads();
  if (tid < kTrsvNB) {
    double s = 0.0;
    for (int j = 0; j <= tid; ++j) s += D[tid * kTrsvNB + j] * xb[j];
    yb[tid] = s;
    if (blockIdx.x == 0 && tid < kb) y[k0 + tid] = s;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  const int i = k0 + kb + blockIdx.x * 8 + warp;
  if (i >= m) return;
  const double* Li = L + (long long)i * ldl + k0;
  double s = 0.0;
  for (int j = lane; j < kb; j += 32) s += Li[j] * yb[j];
  s = warp_sum(s);
  if (lane == 0) w[i] -= s;
}

// Backward block step: x_blk = Dinv_k^T w_blk; w_i -= sum_j L[k0+j, i] x_j
// for i < k0 (thread per i).
__global__ void __launch_bounds__(256) k_trsv_bwd_step(int k0, int kb, const double* __restrict__ L, long long ldl,
                                                       const double* __restrict__ D, double* __restrict__ w,
                                                       double* __restrict__ x) {
  __shared__ double xb[kTrsvNB], yb[kTrsvNB];
  const int tid = threadIdx.x;
  if (tid < kTrsvNB) xb[tid] = tid < kb ? w[k0 + tid] : 0.0;
  __syncthreads();
  if (tid < kTrsvNB) {
    double s = 0.0;
    for (int j = tid; j < kTrsvNB; ++j) s += D[j * kTrsvNB + tid] * xb[j];
    yb[tid] = s;
    if (blockIdx.x == 0 && tid < kb) x[k0 + tid] = s;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + tid;
  if (i >= k0) return;
  double s = 0.0;
  for (int j = 0; j < kb; ++j) s += L[(long long)(k0 + j) * ldl + i] * yb[j];
  w[i] -= s;
}

dngd_status trtri_diag64(int m, const double* L, long long ldl, double* Dinv, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_trtri_diag64<<<cdiv(m, kTrsvNB), kTrsvNB, 0, st>>>(m, L, ldl, Dinv);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// x = (L L^T)^{-1} b with the diagonal-block inverses; w, y: work vectors [m].
dngd_status chol_solve_f64_dinv(int m, const double* L, long long ldl, const double* Dinv, const double* b, double* x,
                                double* w, double* y, cudaStream_t st) {
  DNGD_CUDA_CHECK(cudaMemcpyAsync(w, b, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
  const int nblk = cdiv(m, kTrsvNB);
  for (int bi = 0; bi < nblk; ++bi) {
    const int k0 = bi * kTrsvNB;
    const int kb = (m - k0) < kTrsvNB ? (m - k0) : kTrsvNB;
    const int rest = m - k0 - kb;
    DNGD_NOTE_LAUNCH();
    k_trsv_fwd_step<<<rest > 0 ? cdiv(rest, 8) : 1, 256, 0, st>>>(m, k0, kb, L, ldl,
                                                                  Dinv + (long long)bi * kTrsvNB * kTrsvNB, w, y);
  }
  // y holds L^{-1} b; solve L^T x = y with y as the working vector
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int k0 = bi * kTrsvNB;
    const int kb = (m - k0) < kTrsvNB ? (m - k0) : kTrsvNB;
    DNGD_NOTE_LAUNCH();
    k_trsv_bwd_step<<<k0 > 0 ? cdiv(k0, 256) : 1, 256, 0, st>>>(k0, kb, L, ldl,
                                                                Dinv + (long long)bi * kTrsvNB * kTrsvNB, y, x);
  }
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// ---------------------------------------------------------------------------
// Explicit inverse of a lower-triangular FP32 factor (recursive 2x2 blocks:
// inv([[A,0],[B,C]]) = [[A^-1, 0], [-C^-1 B A^-1, C^-1]]); the diagonal blocks
// are inverted in FP64 in shared memory.  Linv must be zero-initialised.
// ---------------------------------------------------------------------------

__global__ void k_trtri_diag(int k0, int kb, const float* __restrict__ L, long long ldl, float* Linv,
                             long long ldi) {
  extern __shared__ unsigned char trtri_smem[];
  double(*Ls)[kCholNB + 1] = reinterpret_cast<double(*)[kCholNB + 1]>(trtri_smem);
  double(*Xs)[kCholNB + 1] = Ls + kCholNB;
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, j = e % kb;
    Ls[i][j] = (j <= i) ? (double)L[(long long)(k0 + i) * ldl + k0 + j] : 0.0;
  }
  __syncthreads();
  // column c of the inverse by forward substitution (thread per column)
  for (int c = tid; c < kb; c += blockDim.x) {
    for (int i = 0; i < kb; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int p = c; p < i; ++p) s -= Ls[i][p] * Xs[p][c];
      Xs[i][c] = (i < c) ? 0.0 : s / Ls[i][i];
    }
  }
  __syncthreads();
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, j = e % kb;
    Linv[(long long)(k0 + i) * ldi + k0 + j] = (j <= i) ? (float)Xs[i][j] : 0.0f;
  }
}

static dngd_status trtri_rec(int k0, int n, const float* L, long long ldl, float* Linv, long long ldi, float* work,
                             cudaStream_t st, bool have_diag, const Tc3Scratch* tc3, int* status) {
  if (n <= kCholNB && have_diag) return DNGD_OK;
  if (n <= kCholNB) {
    const int smem = 2 * kCholNB * (kCholNB + 1) * (int)sizeof(double);
    static bool attr_set = false;
    if (!attr_set) {
      DNGD_CUDA_CHECK(cudaFuncSetAttribute(k_trtri_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      attr_set = true;
    }
    DNGD_NOTE_LAUNCH();
    k_trtri_diag<<<1, 64, smem, st>>>(k0, n, L, ldl, Linv, ldi);
    DNGD_LAUNCH_CHECK();
    return DNGD_OK;
  }
  const int n1 = ((n / 2 + kCholNB - 1) / kCholNB) * kCholNB;
  const int n2 = n - n1;
  dngd_status s = trtri_rec(k0, n1, L, ldl, Linv, ldi, work, st, have_diag, tc3, status);
  if (s) return s;
  s = trtri_rec(k0 + n1, n2, L, ldl, Linv, ldi, work, st, have_diag, tc3, status);
  if (s) return s;
  // T = L21 * Linv11  (n2 x n1), stored in work with ld n1
  const float* L21 = L + (long long)(k0 + n1) * ldl + k0;
  const float* I11 = Linv + (long long)k0 * ldi + k0;
  const float* I22 = Linv + (long long)(k0 + n1) * ldi + k0 + n1;
  float* I21 = Linv + (long long)(k0 + n1) * ldi + k0;
  if (tc3 && status) {
    s = gemm_tc3(n2, n1, n1, 1.0f, L21, ldl, false, I11, ldi, true, 0.0f, work, n1, false, *tc3, status, st);
    if (s == DNGD_OK)
      s = gemm_tc3(n2, n1, n2, -1.0f, I22, ldi, false, work, n1, true, 0.0f, I21, ldi, false, *tc3, status, st);
    if (s != DNGD_ERR_INVALID_ARG) return s;
  }
  s = gemm_nn<float>(n2, n1, n1, 1.0f, L21, ldl, I11, ldi, 0.0f, work, n1, st);
  if (s) return s;
  return gemm_nn<float>(n2, n1, n2, -1.0f, I22, ldi, work, n1, 0.0f, I21, ldi, st);
}

dngd_status trtri_lower_f32(int m, const float* L, long long ldl, float* Linv, long long ldi, float* work,
                            cudaStream_t st) {
  DNGD_CUDA_CHECK(cudaMemsetAsync(Linv, 0, sizeof(float) * (size_t)m * ldi, st));
  return trtri_rec(0, m, L, ldl, Linv, ldi, work, st, false, nullptr, nullptr);
}

// ---------------------------------------------------------------------------
// Off-diagonal blocks of L^{-1} level by level.  The recursion splits a block
// of n rows at n1 = n/2 rounded up to 64: with L = [L11 0; L21 L22] and the
// inverses I11, I22 of the halves, (L^{-1})21 = -I22 (L21 I11).  Nodes of one
// depth are independent, so all small nodes of a depth (n <= 512) go into
// one batched FP32 SIMT GEMM launch for T = L21 I11 and one for
// -I22 T; the few large nodes at the top use the 3xTF32 tensor-core GEMMs.
// ---------------------------------------------------------------------------

struct GemmNode {
  const float* A;
  const float* B;
  float* C;
  int M, N, K, lda, ldb, ldc;
  float alpha;
  int pad;
};

// C = alpha A B for every node (A [M x K], B [K x N], row-major), 64 x 64
// tiles, blockIdx.z = node.
__global__ void __launch_bounds__(256) k_gemm_nodes(const GemmNode* __restrict__ nodes) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const GemmNode nd = nodes[blockIdx.z];
  const int bm = blockIdx.y * 64, bn = blockIdx.x * 64;
  if (bm >= nd.M || bn >= nd.N) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < nd.K; k0 += 16) {
    for (int e = tid; e < 64 * 16; e += 256) {
      const int r = e >> 4, kk = e & 15;
      const int gr = bm + r, gk = k0 + kk;
      As[kk][r] = (gr < nd.M && gk < nd.K) ? nd.A[(long long)gr * nd.lda + gk] : 0.f;
    }
    for (int e = tid; e < 16 * 64; e += 256) {
      const int kk = e >> 6, c = e & 63;
      const int gc = bn + c, gk = k0 + kk;
      Bs[kk][c] = (gc < nd.N && gk < nd.K) ? nd.B[(long long)gk * nd.ldb + gc] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = bm + ty * 4 + i;
    if (gr >= nd.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = bn + tx * 4 + j;
      if (gc < nd.N) nd.C[(long long)gr * nd.ldc + gc] = nd.alpha * acc[i][j];
    }
  }
}

namespace {

constexpr int kSmallNode = 512;   // nodes up to this size go into the batched launches

struct TrtriNode {
  int k0, n1, n2;
};

void trtri_tree(int k0, int n, int depth, std::vector<std::vector<TrtriNode>>& levels) {
  if (n <= kCholNB) return;   // the factor's 64-blocks are the leaves
  const int n1 = ((n / 2 + kCholNB - 1) / kCholNB) * kCholNB;
  const int n2 = n - n1;
  trtri_tree(k0, n1, depth + 1, levels);
  trtri_tree(k0 + n1, n2, depth + 1, levels);
  if ((int)levels.size() <= depth) levels.resize(depth + 1);
  levels[depth].push_back({k0, n1, n2});
}

// Device node tables of one (m, L, Linv, work) layout, built once.
struct TrtriPlan {
  int m;
  const float* L;
  long long ldl;
  float* Linv;
  long long ldi;
  float* work;
  std::vector<std::vector<TrtriNode>> levels;
  GemmNode* d_nodes = nullptr;          // per depth: [count] T nodes then [count] I21 nodes
  std::vector<int> first, count, maxM, maxN1;
};
std::mutex g_trtri_mu;
std::vector<TrtriPlan*> g_trtri_plans;

TrtriPlan* trtri_plan(int m, const float* L, long long ldl, float* Linv, long long ldi, float* work,
                      cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_trtri_mu);
  for (TrtriPlan* p : g_trtri_plans)
    if (p->m == m && p->L == L && p->ldl == ldl && p->Linv == Linv && p->ldi == ldi && p->work == work) return p;
  // building a plan allocates and copies: not inside a stream capture.  The
  // node table is uploaded on st, ahead of the launches that read it there
  // (a copy on the legacy stream would not be ordered before them when st is
  // a non-blocking stream); a later context can match the plan only once the
  // buffers it names were released, which synchronised the device
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
  TrtriPlan* p = new TrtriPlan();
  p->m = m;
  p->L = L;
  p->ldl = ldl;
  p->Linv = Linv;
  p->ldi = ldi;
  p->work = work;
  trtri_tree(0, m, 0, p->levels);
  std::vector<GemmNode> h;
  for (size_t d = 0; d < p->levels.size(); ++d) {
    std::vector<GemmNode> t, u;
    long long woff = 0;
    int mm = 0, mn = 0;
    for (const TrtriNode& nd : p->levels[d]) {
      if (nd.n1 + nd.n2 > kSmallNode) continue;
      float* T = work + woff;   // n2 x n1, ld n1
      woff += (long long)nd.n1 * nd.n2;
      const float* L21 = L + (long long)(nd.k0 + nd.n1) * ldl + nd.k0;
      const float* I11 = Linv + (long long)nd.k0 * ldi + nd.k0;
      const float* I22 = Linv + (long long)(nd.k0 + nd.n1) * ldi + nd.k0 + nd.n1;
      float* I21 = Linv + (long long)(nd.k0 + nd.n1) * ldi + nd.k0;
      t.push_back({L21, I11, T, nd.n2, nd.n1, nd.n1, (int)ldl, (int)ldi, nd.n1, 1.0f, 0});
      u.push_back({I22, T, I21, nd.n2, nd.n1, nd.n2, (int)ldi, nd.n1, (int)ldi, -1.0f, 0});
      mm = nd.n2 > mm ? nd.n2 : mm;
      mn = nd.n1 > mn ? nd.n1 : mn;
    }
    p->first.push_back((int)h.size());
    p->count.push_back((int)t.size());
    p->maxM.push_back(mm);
    p->maxN1.push_back(mn);
    h.insert(h.end(), t.begin(), t.end());
    h.insert(h.end(), u.begin(), u.end());
  }
  if (!h.empty()) {
    if (cudaMalloc(&p->d_nodes, sizeof(GemmNode) * h.size()) != cudaSuccess ||
        cudaMemcpyAsync(p->d_nodes, h.data(), sizeof(GemmNode) * h.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
      cudaGetLastError();
      delete p;
      return nullptr;
    }
  }
  // plans are kept for the process (a few KB each; a released workspace's
  // plan may still be read by work in flight on another stream)
  g_trtri_plans.push_back(p);
  return p;
}

}  // namespace

// Only the small nodes (two batched FP32 launches per depth, products
// accumulated in FP32 over at most 448 terms), bottom-up; the large nodes are
// the caller's, listed (k0, n1, n2) bottom-up in large_out.
dngd_status trtri_small_nodes_f32(int m, const float* L, long long ldl, float* Linv, long long ldi, float* work,
                                  cudaStream_t st, std::vector<int3>* large_out) {
  TrtriPlan* p = trtri_plan(m, L, ldl, Linv, ldi, work, st);
  if (!p) return DNGD_ERR_INVALID_ARG;
  large_out->clear();
  for (int d = (int)p->levels.size() - 1; d >= 0; --d) {
    const int cnt = p->count[d];
    if (cnt > 0) {
      const dim3 gT(cdiv(p->maxN1[d], 64), cdiv(p->maxM[d], 64), cnt);
      DNGD_NOTE_LAUNCH();
      k_gemm_nodes<<<gT, 256, 0, st>>>(p->d_nodes + p->first[d]);
      DNGD_NOTE_LAUNCH();
      k_gemm_nodes<<<gT, 256, 0, st>>>(p->d_nodes + p->first[d] + cnt);
      DNGD_LAUNCH_CHECK();
    }
    for (const TrtriNode& nd : p->levels[d])
      if (nd.n1 + nd.n2 > kSmallNode) large_out->push_back(make_int3(nd.k0, nd.n1, nd.n2));
  }
  return DNGD_OK;
}

// The FP64 factor as FP32 inputs of the inverse: L32 = fl32(L) (lower,
// upper zero) and the diagonal 64-blocks of Linv = fl32(Dinv), zero
// elsewhere (ldi = ldk).
__global__ void k_factor_to_f32(int m, const double* __restrict__ L, long long ldl, const double* __restrict__ Dinv,
                                float* __restrict__ L32, long long ldk, float* __restrict__ Linv) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * ldk) return;
  const int i = (int)(idx / ldk), j = (int)(idx % ldk);
  L32[idx] = (j <= i) ? (float)L[(long long)i * ldl + j] : 0.f;
  float d = 0.f;
  if (j <= i && j / kTrsvNB == i / kTrsvNB) {
    const int b = i / kTrsvNB;
    d = (float)Dinv[(long long)b * kTrsvNB * kTrsvNB + (i - b * kTrsvNB) * kTrsvNB + (j - b * kTrsvNB)];
  }
  Linv[idx] = d;
}

dngd_status factor_to_f32(int m, const double* L, long long ldl, const double* Dinv, float* L32, float* Linv,
                          long long ldk, cudaStream_t st) {
  const long long cnt = (long long)m * ldk;
  DNGD_NOTE_LAUNCH();
  k_factor_to_f32<<<(int)((cnt + 255) / 256), 256, 0, st>>>(m, L, ldl, Dinv, L32, ldk, Linv);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

dngd_status trtri_offdiag_f32(int m, const float* L, long long ldl, float* Linv, long long ldi, float* work,
                              cudaStream_t st, const Tc3Scratch* tc3, int* status) {
  TrtriPlan* p = (tc3 && status) ? trtri_plan(m, L, ldl, Linv, ldi, work, st) : nullptr;
  if (!p) return trtri_rec(0, m, L, ldl, Linv, ldi, work, st, true, tc3, status);
  for (int d = (int)p->levels.size() - 1; d >= 0; --d) {
    // small nodes of this depth: two batched launches
    const int cnt = p->count[d];
    if (cnt > 0) {
      const dim3 gT(cdiv(p->maxN1[d], 64), cdiv(p->maxM[d], 64), cnt);
      DNGD_NOTE_LAUNCH();
      k_gemm_nodes<<<gT, 256, 0, st>>>(p->d_nodes + p->first[d]);
      DNGD_NOTE_LAUNCH();
      k_gemm_nodes<<<gT, 256, 0, st>>>(p->d_nodes + p->first[d] + cnt);
      DNGD_LAUNCH_CHECK();
    }
    // large nodes: 3xTF32 tensor-core GEMMs, one node at a time
    for (const TrtriNode& nd : p->levels[d]) {
      if (nd.n1 + nd.n2 <= kSmallNode) continue;
      const float* L21 = L + (long long)(nd.k0 + nd.n1) * ldl + nd.k0;
      const float* I11 = Linv + (long long)nd.k0 * ldi + nd.k0;
      const float* I22 = Linv + (long long)(nd.k0 + nd.n1) * ldi + nd.k0 + nd.n1;
      float* I21 = Linv + (long long)(nd.k0 + nd.n1) * ldi + nd.k0;
      dngd_status s = gemm_tc3(nd.n2, nd.n1, nd.n1, 1.0f, L21, ldl, false, I11, ldi, true, 0.0f, work, nd.n1, false,
                               *tc3, status, st);
      if (s == DNGD_OK)
        s = gemm_tc3(nd.n2, nd.n1, nd.n2, -1.0f, I22, ldi, false, work, nd.n1, true, 0.0f, I21, ldi, false, *tc3,
                     status, st);
      if (s == DNGD_ERR_INVALID_ARG) {
        s = gemm_nn<float>(nd.n2, nd.n1, nd.n1, 1.0f, L21, ldl, I11, ldi, 0.0f, work, nd.n1, st);
        if (s == DNGD_OK) s = gemm_nn<float>(nd.n2, nd.n1, nd.n2, -1.0f, I22, ldi, work, nd.n1, 0.0f, I21, ldi, st);
      }
      if (s) return s;
    }
  }
  return DNGD_OK;
}

// ---------------------------------------------------------------------------
// GEMV.  FP64 data accumulates in FP64; FP32 data accumulates the exact
// products of the FP32 entry with the hi/lo FP32 split of the FP64 vector in
// double-float arithmetic, so the FP32 operator is applied without adding
// FP32 rounding of its own, at HBM speed.
// ---------------------------------------------------------------------------

template <typename TA>
struct Acc;
template <>
struct Acc<double> {
  double v;
  __device__ void init() { v = 0.0; }
  __device__ void add(double a, double xhi, double xlo) { v = fma(a, xhi, v); (void)xlo; }
  __device__ double get() const { return v; }
  __device__ void warp_reduce() { v = warp_sum(v); }
};
template <>
struct Acc<float> {
  dfloat v;
  __device__ void init() { v.hi = 0.f; v.lo = 0.f; }
  __device__ void add(float a, float xhi, float xlo) {
    v = df_fma(v, a, xhi);
    v.lo = fmaf(a, xlo, v.lo);
  }
  // hi + lo is exact in float64 (|lo| <= ulp(hi)/2)
  __device__ double get() const { return (double)v.hi + (double)v.lo; }
  __device__ void warp_reduce() { v = df_warp_sum(v); }
};

template <typename TA>
__device__ __forceinline__ void split_x(double x, TA& hi, TA& lo);
template <>
__device__ __forceinline__ void split_x<double>(double x, double& hi, double& lo) { hi = x; lo = 0.0; }
template <>
__device__ __forceinline__ void split_x<float>(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

constexpr int kGemvSplits = 16;

// partials[split][p] = sum_{i in split rows} A[i,p] x[i]
template <typename TA>
__global__ void __launch_bounds__(256) k_gemv_t(int m, int n, const TA* __restrict__ A, long long lda,
                                                 const double* __restrict__ x, double* __restrict__ partials) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int split = blockIdx.y;
  const int rows = (m + gridDim.y - 1) / gridDim.y;
  const int i0 = split * rows, i1 = min(m, i0 + rows);
  if (p >= n) return;
  Acc<TA> acc;
  acc.init();
  for (int i = i0; i < i1; ++i) {
    TA hi, lo;
    split_x<TA>(x[i], hi, lo);
    acc.add(A[(long long)i * lda + p], hi, lo);
  }
  partials[(long long)split * n + p] = acc.get();
}

__global__ void k_reduce_splits(int n, int splits, const double* __restrict__ partials, double alpha,
                                double* __restrict__ y) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double s = 0.0;
  for (int k = 0; k < splits; ++k) s += partials[(long long)k * n + p];
  y[p] = alpha * s;
}

template <typename TA>
dngd_status gemv_t(int m, int n, const TA* A, long long lda, const double* x, double alpha, double* y,
                   double* partials, cudaStream_t st) {
  const int splits = m >= kGemvSplits * 8 ? kGemvSplits : 1;
  dim3 grid(cdiv(n, 256), splits);
  DNGD_NOTE_LAUNCH();
  k_gemv_t<TA><<<grid, 256, 0, st>>>(m, n, A, lda, x, partials);
  DNGD_NOTE_LAUNCH();
  k_reduce_splits<<<cdiv(n, 256), 256, 0, st>>>(n, splits, partials, alpha, y);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// y[i] = alpha * sum_p A[i,p] x[p]; 4 rows per block of 256 threads.
template <typename TA>
__global__ void __launch_bounds__(256) k_gemv_n(int m, int n, const TA* __restrict__ A, long long lda,
                                                 const double* __restrict__ x, double alpha, double* __restrict__ y) {
  constexpr int RPB = 4;
  const int i0 = blockIdx.x * RPB;
  Acc<TA> acc[RPB];
#pragma unroll
  for (int r = 0; r < RPB; ++r) acc[r].init();
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    TA hi, lo;
    split_x<TA>(x[p], hi, lo);
#pragma unroll
    for (int r = 0; r < RPB; ++r)
      if (i0 + r < m) acc[r].add(A[(long long)(i0 + r) * lda + p], hi, lo);
  }
  __shared__ double red[RPB][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < RPB; ++r) {
    acc[r].warp_reduce();
    if (lane == 0) red[r][warp] = acc[r].get();
  }
  __syncthreads();
  if (threadIdx.x < RPB && i0 + (int)threadIdx.x < m) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[threadIdx.x][w];
    y[i0 + threadIdx.x] = alpha * t;
  }
}

template <typename TA>
dngd_status gemv_n(int m, int n, const TA* A, long long lda, const double* x, double alpha, double* y,
                   cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_gemv_n<TA><<<cdiv(m, 4), 256, 0, st>>>(m, n, A, lda, x, alpha, y);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

template dngd_status gemv_t<double>(int, int, const double*, long long, const double*, double, double*, double*,
                                    cudaStream_t);
template dngd_status gemv_n<double>(int, int, const double*, long long, const double*, double, double*,
                                    cudaStream_t);


template <typename T>
__global__ void k_add_diag(int m, T* K, long long ldk, double shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) K[(long long)i * ldk + i] += (T)shift;
}

template <typename T>
dngd_status add_diag(int m, T* K, long long ldk, double shift, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_add_diag<T><<<cdiv(m, 256), 256, 0, st>>>(m, K, ldk, shift);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}
template dngd_status add_diag<double>(int, double*, long long, double, cudaStream_t);
template dngd_status add_diag<float>(int, float*, long long, double, cudaStream_t);

// ---------------------------------------------------------------------------
// Deterministic dot product: fixed grid, per-block partial, second pass.
// ---------------------------------------------------------------------------

constexpr int kDotBlocks = 128;

__global__ void k_dot_partial(int n, const double* __restrict__ x, const double* __restrict__ y,
                              double* __restrict__ partials) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += x[i] * y[i];
  s = warp_sum(s);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void k_dot_final(int nb, const double* __restrict__ partials, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) s += partials[i];
  s = warp_sum(s);
  if (threadIdx.x == 0) *out = s;
}

dngd_status dot_dev(int n, const double* x, const double* y, double* out, double* partials, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_dot_partial<<<kDotBlocks, 256, 0, st>>>(n, x, y, partials);
  DNGD_NOTE_LAUNCH();
  k_dot_final<<<1, 32, 0, st>>>(kDotBlocks, partials, out);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

__global__ void k_sqnorm_batch(int n, const double* __restrict__ x, double* __restrict__ out) {
  const double* v = x + (long long)blockIdx.x * n;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i] * v[i];
  s = warp_sum(s);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

dngd_status sqnorm_batch(int n, int G, const double* x, double* out, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_sqnorm_batch<<<G, 256, 0, st>>>(n, x, out);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

__global__ void k_axpy(int n, double alpha, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += alpha * x[i];
}

dngd_status axpy_dev(int n, double alpha, const double* x, double* y, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_axpy<<<cdiv(n, 256), 256, 0, st>>>(n, alpha, x, y);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

}  // namespace dngd
