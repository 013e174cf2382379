// Persistent PCG for the exact-Gram path: the whole solve of
// (K + lambda I) x = b (Alg. DenseDualSolve's refinement, preconditioned by
// the FP32 factor M^{-1} = Linv^T Linv) is one cooperative kernel.
//
// One 512-thread block per SM (the vector every block stages is read from L2
// by half as many blocks as with two smaller ones).  Every block owns a
// contiguous range of rows; each phase of an iteration is a row-parallel
// GEMV (warp per row, rows taken in pairs (p, m-1-p) so that every warp's
// share of the triangular factor is the same; 16-byte loads with eight in
// flight per lane; the input vector staged in shared memory as separate hi
// and lo float arrays; double-float accumulation) followed by a grid
// barrier; block partial sums are reduced by every block in the same order,
// so all blocks take the same decisions and the result is deterministic.
// Vectors written during the kernel are read with L2-only loads (another SM
// may have written them).
// p and r are double-buffered, so each iteration needs three barriers:
//   p = z + beta p_prev (staged whole by every block), Ap = K p + lambda p,
//     <p, Ap>                                                    | barrier
//   r_new = r - alpha Ap staged whole by every block (each forms the same
//     ||r_new||^2: the stop test needs no barrier), x += alpha p on owned
//     rows, y = Linv r_new (lower triangle only)                 | barrier
//   z = Linv^T y (upper triangle of the stored transpose), <r_new, z> | barrier
// The grid barrier is an arrival counter plus a generation word; every wait
// is bounded by a global-timer deadline after which the kernel records
// ST_TIMEOUT and all blocks leave.  The launch is cooperative, so all blocks
// are co-resident.
#include <cooperative_groups.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "step_kernels.h"

namespace dngd {

namespace {

constexpr int PT = 512;                         // threads per block (one block per SM)
constexpr unsigned long long kBarrierNs = 2000000000ull;

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct PcgState {
  unsigned int count;       // arrivals at the current barrier
  unsigned int gen;         // barrier generation
  int abort;                // set by a block whose wait ran out
  int pad;
};

// Returns false (all threads) if the barrier timed out or another block did.
__device__ bool grid_barrier(PcgState* gs, unsigned nblocks, int* status,
                             unsigned long long limit_ns = kBarrierNs) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &gs->gen;
    volatile int* ab = &gs->abort;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&gs->count, 1u) + 1u;
    int ok = 1;
    if (arrived == nblocks) {
      gs->count = 0;
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    } else {
      const unsigned long long t0 = gtime();
      while (*gen == g) {
        if (*ab) {
          ok = 0;
          break;
        }
        if (gtime() - t0 > limit_ns) {
          atomicOr(status, ST_TIMEOUT);
          atomicExch(&gs->abort, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    ok_sh = ok && !*ab;
  }
  __syncthreads();
  return ok_sh != 0;
}

// Fixed-order sum of nb block partials (valid in every thread).
__device__ double sum_parts(const double* parts, int nb) {
  __shared__ double red[PT / 32];
  __shared__ double tot;
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += PT) s += __ldcg(parts + i);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < PT / 32; ++w) t += red[w];
    tot = t;
  }
  __syncthreads();
  const double v = tot;
  __syncthreads();
  return v;
}

// Block sum of v (valid in thread 0).
__device__ double block_sum(double v) {
  __shared__ double red[PT / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < PT / 32; ++w) t += red[w];
  __syncthreads();
  return t;
}

// Stage v[0, m) in shared memory as hi and lo floats (sh[j], sl[j]).
__device__ void stage(const double* __restrict__ v, float* __restrict__ sh, float* __restrict__ sl, int m) {
  __syncthreads();
  for (int j0 = threadIdx.x; j0 < m; j0 += 8 * PT) {
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + u * PT;
      x[u] = j < m ? __ldcg(v + j) : 0.0;   // written by other blocks: bypass L1
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + u * PT;
      if (j < m) {
        const float h = (float)x[u];
        sh[j] = h;
        sl[j] = (float)(x[u] - (double)h);
      }
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void acc_f32(dfloat& acc, float a, float xh, float xl) {
  acc = df_fma(acc, a, xh);
  acc.lo = fmaf(a, xl, acc.lo);
}

// Row of an FP32 matrix (columns [c0, c1)) times the staged vector: a scalar
// head up to a 4-aligned column, float4 loads (eight in flight per lane),
// a scalar tail; two double-float accumulators.  The row must start on a
// 16-byte boundary (the caller checks base and leading dimension).
__device__ double row_dot_f32(const float* __restrict__ A, int c0, int c1, const float* __restrict__ sh,
                              const float* __restrict__ sl) {
  const int lane = threadIdx.x & 31;
  dfloat acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};
  const int a0 = min(c1, (c0 + 3) & ~3);
  if (c0 + lane < a0) acc_f32(acc0, __ldg(A + c0 + lane), sh[c0 + lane], sl[c0 + lane]);
  const int n4 = (c1 - a0) >> 2;
  const float4* A4 = reinterpret_cast<const float4*>(A + a0);
  const float4* h4 = reinterpret_cast<const float4*>(sh + a0);
  const float4* l4 = reinterpret_cast<const float4*>(sl + a0);
  int q = lane;
  for (; q + 7 * 32 < n4; q += 8 * 32) {
    float4 a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = __ldg(A4 + q + 32 * u);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float4 xh = h4[q + 32 * u], xl = l4[q + 32 * u];
      acc_f32(acc0, a[u].x, xh.x, xl.x);
      acc_f32(acc1, a[u].y, xh.y, xl.y);
      acc_f32(acc0, a[u].z, xh.z, xl.z);
      acc_f32(acc1, a[u].w, xh.w, xl.w);
    }
  }
  for (; q < n4; q += 32) {
    const float4 a = __ldg(A4 + q);
    const float4 xh = h4[q], xl = l4[q];
    acc_f32(acc0, a.x, xh.x, xl.x);
    acc_f32(acc1, a.y, xh.y, xl.y);
    acc_f32(acc0, a.z, xh.z, xl.z);
    acc_f32(acc1, a.w, xh.w, xl.w);
  }
  const int b0 = a0 + 4 * n4;
  if (b0 + lane < c1) acc_f32(acc1, __ldg(A + b0 + lane), sh[b0 + lane], sl[b0 + lane]);
  dfloat acc = df_warp_sum(df_add(acc0, acc1));
  return (double)acc.hi + (double)acc.lo;
}

__device__ __forceinline__ void acc_df(dfloat& acc, float ah, float al, float xh, float xl) {
  acc = df_fma(acc, ah, xh);
  acc.lo = fmaf(ah, xl, fmaf(al, xh, acc.lo));
}

// Row of the double-float Gram (float2 (hi, lo) per entry) times the staged
// vector: float4 loads = two entries, eight in flight per lane.  The row must
// start on a 16-byte boundary.
__device__ double row_dot_df(const float2* __restrict__ A, int m, const float* __restrict__ sh,
                             const float* __restrict__ sl) {
  const int lane = threadIdx.x & 31;
  dfloat acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};
  const float4* A4 = reinterpret_cast<const float4*>(A);
  const float2* h2 = reinterpret_cast<const float2*>(sh);
  const float2* l2 = reinterpret_cast<const float2*>(sl);
  const int m2 = m >> 1;
  int q = lane;
  for (; q + 7 * 32 < m2; q += 8 * 32) {
    float4 a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = __ldg(A4 + q + 32 * u);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float2 xh = h2[q + 32 * u], xl = l2[q + 32 * u];
      acc_df(acc0, a[u].x, a[u].y, xh.x, xl.x);
      acc_df(acc1, a[u].z, a[u].w, xh.y, xl.y);
    }
  }
  for (; q < m2; q += 32) {
    const float4 a = __ldg(A4 + q);
    const float2 xh = h2[q], xl = l2[q];
    acc_df(acc0, a.x, a.y, xh.x, xl.x);
    acc_df(acc1, a.z, a.w, xh.y, xl.y);
  }
  if ((m & 1) && lane == 0) {
    const float2 a = __ldg(A + m - 1);
    acc_df(acc0, a.x, a.y, sh[m - 1], sl[m - 1]);
  }
  dfloat acc = df_warp_sum(df_add(acc0, acc1));
  return (double)acc.hi + (double)acc.lo;
}

__global__ void __launch_bounds__(PT, 1) k_pcg_persist(int m, const float2* __restrict__ K, long long ldk, double lambda,
                                                    const float* __restrict__ Linv, const float* __restrict__ LinvT,
                                                    long long ldi, const double* __restrict__ b,
                                                    double* __restrict__ x, double* __restrict__ r0b,
                                                    double* __restrict__ r1b, double* __restrict__ p0b,
                                                    double* __restrict__ p1b, double* __restrict__ z,
                                                    double* __restrict__ Ap, double* __restrict__ y,
                                                    double* __restrict__ parts, double* scal, double tol, int maxit,
                                                    PcgState* gs, int* status) {
  extern __shared__ float4 sv_raw[];
  const int mpad = (m + 3) & ~3;
  float* sh = reinterpret_cast<float*>(sv_raw);   // [mpad] hi
  float* sl = sh + mpad;                          // [mpad] lo
  __shared__ double red_sh[PT / 32];
  const unsigned nb = gridDim.x;
  const int per = (m + (int)nb - 1) / (int)nb;
  const int ra = min(m, (int)blockIdx.x * per), rb = min(m, ra + per);   // rows this block updates
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = PT / 32;
  // GEMV rows go round-robin over all warps of the grid (the triangular
  // factor's rows differ in length)
  const int gw = (int)blockIdx.x * nw + warp, GW = (int)nb * nw;
  double* p_pap = parts;           // [nb] per quantity, rewritten once per iteration
  double* p_rz = parts + nb;
  double* p_bb = parts + 2 * nb;
  double* rbuf[2] = {r0b, r1b};
  double* pbuf[2] = {p0b, p1b};

  // x = 0, r = b; z = M^{-1} r
  for (int i = ra + threadIdx.x; i < rb; i += PT) {
    x[i] = 0.0;
    r0b[i] = b[i];
  }
  if (!grid_barrier(gs, nb, status)) return;
  stage(r0b, sh, sl, m);
  for (int p = gw; p < (m + 1) / 2; p += GW)
      for (int h = 0; h < 2 && (h == 0 || m - 1 - p != p); ++h) {
        const int i = h ? m - 1 - p : p;
    const double v = row_dot_f32(Linv + (long long)i * ldi, 0, i + 1, sh, sl);
    if (lane == 0) y[i] = v;
  }
  if (!grid_barrier(gs, nb, status)) return;
  stage(y, sh, sl, m);
  {
    double rz = 0.0, bb = 0.0;
    for (int p = gw; p < (m + 1) / 2; p += GW)
      for (int h = 0; h < 2 && (h == 0 || m - 1 - p != p); ++h) {
        const int i = h ? m - 1 - p : p;
      const double v = row_dot_f32(LinvT + (long long)i * ldi, i, m, sh, sl);
      if (lane == 0) {
        z[i] = v;
        rz += __ldcg(r0b + i) * v;
        bb += b[i] * b[i];
      }
    }
    rz = block_sum(rz);
    bb = block_sum(bb);
    if (threadIdx.x == 0) {
      p_rz[blockIdx.x] = rz;
      p_bb[blockIdx.x] = bb;
    }
  }
  if (!grid_barrier(gs, nb, status)) return;
  double rho = sum_parts(p_rz, nb);
  const double bbt = sum_parts(p_bb, nb);
  const double tol2 = tol * tol * bbt;
  double rr = bbt, beta = 0.0;
  int it = 0;
  bool done = bbt == 0.0, brk = false;
  while (!done && it < maxit) {
    double* pc = pbuf[it & 1];
    const double* pp = pbuf[(it + 1) & 1];
    const double* rc = rbuf[it & 1];
    double* rn = rbuf[(it + 1) & 1];
    // A: p = z + beta p_prev (every block stages all of it, the owners store
    //    their rows); Ap = K p + lambda p with the block partials of <p, Ap>
    __syncthreads();
    for (int j0 = threadIdx.x; j0 < m; j0 += 8 * PT) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u * PT;
        v[u] = j < m ? (it == 0 ? __ldcg(z + j) : __ldcg(z + j) + beta * __ldcg(pp + j)) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u * PT;
        if (j < m) {
          const float h = (float)v[u];
          sh[j] = h;
          sl[j] = (float)(v[u] - (double)h);
          if (j >= ra && j < rb) pc[j] = v[u];
        }
      }
    }
    __syncthreads();
    double pap = 0.0;
    for (int p = gw; p < (m + 1) / 2; p += GW)
      for (int h = 0; h < 2 && (h == 0 || m - 1 - p != p); ++h) {
        const int i = h ? m - 1 - p : p;
      const double pi = (double)sh[i] + (double)sl[i];
      const double v = row_dot_df(K + (long long)i * ldk, m, sh, sl) + lambda * pi;
      if (lane == 0) {
        Ap[i] = v;
        pap += pi * v;
      }
    }
    pap = block_sum(pap);
    if (threadIdx.x == 0) p_pap[blockIdx.x] = pap;
    if (!grid_barrier(gs, nb, status)) return;
    const double pAp = sum_parts(p_pap, nb);
    if (!(pAp > 1e-300)) {
      brk = true;
      break;
    }
    const double alpha = rho / pAp;
    // B: r_new = r - alpha Ap for all rows (staged; every block forms the same
    //    ||r_new||^2 in the same order), x += alpha p on the owned rows, stop
    //    test, y = Linv r_new
    __syncthreads();
    double rrl = 0.0;
    for (int j0 = threadIdx.x; j0 < m; j0 += 8 * PT) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u * PT;
        v[u] = j < m ? __ldcg(rc + j) - alpha * __ldcg(Ap + j) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u * PT;
        if (j < m) {
          rrl += v[u] * v[u];
          const float h = (float)v[u];
          sh[j] = h;
          sl[j] = (float)(v[u] - (double)h);
          if (j >= ra && j < rb) {
            rn[j] = v[u];
            x[j] = __ldcg(x + j) + alpha * __ldcg(pc + j);
          }
        }
      }
    }
    rrl = warp_sum(rrl);
    if (lane == 0) red_sh[warp] = rrl;
    __syncthreads();
    rr = 0.0;
    for (int w = 0; w < nw; ++w) rr += red_sh[w];
    ++it;
    if (rr <= tol2) {
      done = true;
      break;
    }
    for (int p = gw; p < (m + 1) / 2; p += GW)
      for (int h = 0; h < 2 && (h == 0 || m - 1 - p != p); ++h) {
        const int i = h ? m - 1 - p : p;
      const double v = row_dot_f32(Linv + (long long)i * ldi, 0, i + 1, sh, sl);
      if (lane == 0) y[i] = v;
    }
    if (!grid_barrier(gs, nb, status)) return;
    // C: z = Linv^T y with the block partials of <r_new, z>
    stage(y, sh, sl, m);
    double rz = 0.0;
    for (int p = gw; p < (m + 1) / 2; p += GW)
      for (int h = 0; h < 2 && (h == 0 || m - 1 - p != p); ++h) {
        const int i = h ? m - 1 - p : p;
      const double v = row_dot_f32(LinvT + (long long)i * ldi, i, m, sh, sl);
      if (lane == 0) {
        z[i] = v;
        rz += __ldcg(rn + i) * v;
      }
    }
    rz = block_sum(rz);
    if (threadIdx.x == 0) p_rz[blockIdx.x] = rz;
    if (!grid_barrier(gs, nb, status)) return;
    const double rho_new = sum_parts(p_rz, nb);
    if (rho_new == 0.0 || rho == 0.0) {
      brk = true;
      break;
    }
    beta = rho_new / rho;
    rho = rho_new;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    scal[S_ITERS] = (double)it;
    scal[S_RR] = rr;
    scal[S_BB] = bbt;
    scal[S_TOL2] = tol2;
    scal[S_RHO] = rho;
    scal[S_BREAK] = brk ? 1.0 : 0.0;
    scal[S_DONE] = 1.0;
  }
}

// Expiry of the bounded grid barrier: the blocks wait for one more arrival
// than there are blocks, so the wait runs out after limit_ns and the kernel
// records ST_TIMEOUT and returns (the check that a stuck wait ends cleanly).
__global__ void k_barrier_expiry(PcgState* gs, int* status, unsigned long long limit_ns) {
  grid_barrier(gs, gridDim.x + 1, status, limit_ns);
}

// Linv^T, tile-transposed (ld of both: ldi).
__global__ void k_transpose_f32(int m, const float* __restrict__ A, long long lda, float* __restrict__ T,
                                long long ldt) {
  __shared__ float t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8) {
    const int r = by + i, c = bx + tx;
    t[i][tx] = (r < m && c < m) ? A[(long long)r * lda + c] : 0.f;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int r = bx + i, c = by + tx;
    if (r < m && c < m) T[(long long)r * ldt + c] = t[tx][i];
  }
}

}  // namespace

dngd_status transpose_f32(int m, const float* A, long long lda, float* T, long long ldt, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_transpose_f32<<<dim3(cdiv(m, 32), cdiv(m, 32)), 256, 0, st>>>(m, A, lda, T, ldt);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

size_t pcg_persist_state_bytes() { return sizeof(PcgState); }

dngd_status barrier_expiry(void* state, int* status, double limit_ms, cudaStream_t st) {
  DNGD_CUDA_CHECK(cudaMemsetAsync(state, 0, sizeof(PcgState), st));
  DNGD_NOTE_LAUNCH();
  k_barrier_expiry<<<2, PT, 0, st>>>((PcgState*)state, status, (unsigned long long)(limit_ms * 1e6));
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

static size_t persist_smem(int m) { return 2 * sizeof(float) * (size_t)((m + 3) & ~3); }

// Blocks of the cooperative grid (co-resident), or 0 if the launch cannot fit.
static int persist_blocks(int m) {
  // one block per SM, so the grid only depends on whether a block with this
  // m's shared memory fits on an SM at all
  static std::mutex mu;
  static bool attr = false;
  std::lock_guard<std::mutex> lk(mu);
  if (!attr) {
    if (allow_max_dynamic_smem((const void*)k_pcg_persist) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    attr = true;
  }
  int dev = 0, nsm = 0, per = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_persist, PT, persist_smem(m)) != cudaSuccess) {
    cudaGetLastError();
    per = 0;
  }
  if (per > 1) per = 1;
  return coop ? per * nsm : 0;
}

dngd_status pcg_persist_solve(int m, const float2* K, long long ldk, double lambda, const float* Linv,
                              const float* LinvT, long long ldi, const double* b, double* x, double* work,
                              double* parts, long long parts_cap, double* scal, double tol, int maxit, void* state,
                              int* status, cudaStream_t st) {
  const int nb = persist_blocks(m);
  if (nb <= 0 || 3LL * nb > parts_cap || persist_smem(m) > 200 * 1024) return DNGD_ERR_INVALID_ARG;
  // the row products use 16-byte loads: every row of K (float2) and of the
  // factor (float) must start on a 16-byte boundary
  if ((reinterpret_cast<uintptr_t>(K) & 15) || (ldk & 1) || (reinterpret_cast<uintptr_t>(Linv) & 15) ||
      (reinterpret_cast<uintptr_t>(LinvT) & 15) || (ldi & 3))
    return DNGD_ERR_INVALID_ARG;
  DNGD_CUDA_CHECK(cudaMemsetAsync(state, 0, sizeof(PcgState), st));
  PcgState* gs = (PcgState*)state;
  double* r0b = work;
  double* r1b = work + m;
  double* p0b = work + 2 * (size_t)m;
  double* p1b = work + 3 * (size_t)m;
  double* z = work + 4 * (size_t)m;
  double* Ap = work + 5 * (size_t)m;
  double* y = work + 6 * (size_t)m;
  void* args[] = {&m,  &K,  &ldk, &lambda, &Linv, &LinvT, &ldi,  &b,   &x,      &r0b,   &r1b, &p0b,
                  &p1b, &z, &Ap,  &y,      &parts, &scal, &tol, &maxit, &gs, &status};
  DNGD_NOTE_LAUNCH();
  DNGD_CUDA_CHECK(cudaLaunchCooperativeKernel((const void*)k_pcg_persist, dim3(nb), dim3(PT), args,
                                              persist_smem(m), st));
  return DNGD_OK;
}

}  // namespace dngd
