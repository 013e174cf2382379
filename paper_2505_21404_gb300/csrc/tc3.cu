// FP32 GEMM on the TF32 tensor cores with FP32-like accuracy ("3xTF32"):
// C = alpha * A_op B_op^T + beta * C, A_op [M x K], B_op [N x K].
//
// Every operand x is split into x_hi = tf32(x) and x_lo = tf32(x - x_hi)
// (both rounded to nearest, so the tensor cores see exact TF32 values), and
// A_op B_op^T ~= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T; the dropped
// A_lo B_lo^T and the rounding of x_lo leave ~2^-21 relative error per
// product (FP32 SIMT: 2^-24).  The tensor cores' FP32 accumulation is not
// round-to-nearest and its error grows with the reduction length, so the
// TMEM accumulator only ever runs over 128 K-elements: chunks alternate
// between two TMEM buffers and the epilogue adds each into round-to-nearest
// FP32 registers while the next chunk is computed.
//
// The split copies (and, for a transposed operand, the transpose) go to a
// caller-owned scratch as [rows x 2 Kp] FP32 (hi in columns [0, Kp), lo in
// [Kp, 2 Kp), Kp = K rounded up to 32, zero tails), so TMA needs no
// alignment from the caller's matrices.  Kernel: one 128 x 128 output tile
// per CTA (lower-triangle tiles only when asked), a 3-stage TMA ring of
// 64 KB stages (A_hi, A_lo, B_hi, B_lo for 32 K), warp 1 issuing 12
// tcgen05.mma kind::tf32 per stage into the current TMEM buffer, warps 2..5
// draining each chunk.  Waits are bounded (ST_TIMEOUT).
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace dngd {

namespace {

using namespace tc;

constexpr int T3 = 128;                     // tile rows = columns
constexpr int KB3 = 32;                     // K per stage (128-byte rows)
constexpr int ST3 = 3;
constexpr int TILE3 = T3 * 128;             // 16 KB
constexpr int STAGE3 = 4 * TILE3;           // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM3 = ST3 * STAGE3 + 1024;
constexpr int THREADS3 = 192;
constexpr int CH3 = 4;                      // stages per TMEM accumulation chunk (4 x 32 = 128 K)
static_assert(4 * 4 * 32 * 33 * 4 <= ST3 * STAGE3, "the epilogue stages its accumulators in the operand ring");

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;   // inf / nan unchanged
  u = (u + 0x1000u) & 0xFFFFE000u;
  return __uint_as_float(u);
}

// dst[r, 0:Kp] = hi, dst[r, Kp:2Kp] = lo of op[r, k]; op = src (row-major
// [rows x K], ld) or, with trans, src^T (src row-major [K x rows]).
__global__ void k_tc3_split(int rows, int K, int Kp, const float* __restrict__ src, long long ld, int trans,
                            float* __restrict__ dst, long long src_z = 0, const float* __restrict__ kscale = nullptr) {
  // grid.z: independent operands (line-search trials), src + z src_z, dst
  // z rows further on
  src += blockIdx.z * src_z;
  dst += (long long)blockIdx.z * rows * 2 * Kp;
  __shared__ float t[32][33];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    float v = 0.f;
    if (trans) {
      const int k = k0 + i, r = r0 + tx;
      if (k < K && r < rows) v = src[(long long)k * ld + r] * (kscale ? kscale[k] : 1.f);
      t[tx][i] = v;   // t[r][k]
    } else {
      const int r = r0 + i, k = k0 + tx;
      if (k < K && r < rows) v = src[(long long)r * ld + k] * (kscale ? kscale[k] : 1.f);
      t[i][tx] = v;
    }
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, k = k0 + tx;
    if (r < rows && k < Kp) {
      const float x = t[i][tx];
      const float hi = tf32_rn(x);
      float* row = dst + (long long)r * 2 * Kp;
      row[k] = hi;
      row[Kp + k] = tf32_rn(x - hi);
    }
  }
}

// TF32 x TF32 -> FP32, both K-major, N = M = 128.
__device__ __forceinline__ uint32_t tc3_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(T3 >> 3) << 17) | ((uint32_t)(T3 >> 4) << 24);
}

__global__ void __launch_bounds__(THREADS3, 1)
k_tc3(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N, int Kp,
      float alpha, float beta, float* __restrict__ C, long long ldc, int lower, float* __restrict__ csplit, int kpc,
      int* status, int a_zrows = 0, int b_zrows = 0, long long c_z = 0) {
  // grid.z: independent products (line-search trials) whose operands are
  // stacked by rows in the split buffers and whose outputs are c_z apart
  const int bn = blockIdx.x, bm = blockIdx.y;
  const int ay = (int)blockIdx.z * a_zrows + bm * T3, by = (int)blockIdx.z * b_zrows + bn * T3;
  C += blockIdx.z * c_z;
  if (lower && bn * T3 > bm * T3 + T3 - 1) return;
  // a factorisation that already failed (the host retries it with a larger
  // shift) needs no further updates
  if (status[0] & ST_NOT_SPD) return;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[ST3];
  __shared__ __align__(8) uint64_t empty_bar[ST3];
  __shared__ __align__(8) uint64_t accf_bar[2];   // MMA -> epilogue: chunk in buffer b done
  __shared__ __align__(8) uint64_t acce_bar[2];   // epilogue -> MMA: buffer b drained
  __shared__ __align__(8) uint64_t fin_bar;       // teardown: every issued MMA retired
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int nk = Kp / KB3;
  const int nchunk = (nk + CH3 - 1) / CH3;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST3; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf_bar[b]), 1);
      mbar_init(smem_u32(&acce_bar[b]), 4);
    }
    mbar_init(smem_u32(&fin_bar), 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(2 * T3));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;
  volatile int* abort_flag = &abort_sh;

  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int st = it % ST3;
        const uint32_t ph = (uint32_t)((it / ST3) & 1);
        if (*abort_flag || !mbar_wait(smem_u32(&empty_bar[st]), ph ^ 1u, status, 21)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t fb = smem_u32(&full_bar[st]);
        mbar_expect_tx(fb, STAGE3);
        const uint32_t sb = smem_base + st * STAGE3;
        const int kc = it * KB3;
        tma_load_2d(sb, &mapA, fb, kc, ay);
        tma_load_2d(sb + TILE3, &mapA, fb, Kp + kc, ay);
        tma_load_2d(sb + 2 * TILE3, &mapB, fb, kc, by);
        tma_load_2d(sb + 3 * TILE3, &mapB, fb, Kp + kc, by);
        ++issued;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tc3_idesc();
      // CH3 stages per chunk, alternating between two TMEM buffers; a buffer
      // is reused once the epilogue has drained its previous chunk
      for (int c = 0; c < nchunk && !*abort_flag; ++c) {
        const int b = c & 1;
        if (c >= 2 && !mbar_wait(smem_u32(&acce_bar[b]), (uint32_t)(((c >> 1) - 1) & 1), status, 26)) {
          *abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t dbuf = tmem + (uint32_t)(b * T3);
        const int it1 = min(nk, (c + 1) * CH3);
        bool stop = false;
        for (int it = c * CH3; it < it1; ++it) {
          const int st = it % ST3;
          const uint32_t ph = (uint32_t)((it / ST3) & 1);
          if (!mbar_wait(smem_u32(&full_bar[st]), ph, status, 22)) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t sb = smem_base + st * STAGE3;
          const uint64_t ahi = sw128_desc(sb), alo = sw128_desc(sb + TILE3);
          const uint64_t bhi = sw128_desc(sb + 2 * TILE3), blo = sw128_desc(sb + 3 * TILE3);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint64_t dk = (uint64_t)((32 * k) >> 4);
            umma<1>(dbuf, ahi + dk, bhi + dk, idesc, (it > c * CH3 || k > 0) ? 1u : 0u);
            umma<1>(dbuf, ahi + dk, blo + dk, idesc, 1u);
            umma<1>(dbuf, alo + dk, bhi + dk, idesc, 1u);
          }
          umma_commit(smem_u32(&empty_bar[st]));
        }
        if (stop) break;
        umma_commit(smem_u32(&accf_bar[b]));
      }
    }
  } else {
    // epilogue warps 2..5: warp w reads TMEM lanes 32 (w % 4).. (its 32 rows)
    // and adds each chunk into round-to-nearest FP32 registers (the tensor
    // cores' own accumulation is not round-to-nearest, so it only ever runs
    // over CH3 x 32 products)
    const int q = warp & 3;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    float acc[T3];
#pragma unroll
    for (int j = 0; j < T3; ++j) acc[j] = 0.f;
    bool ok = true;
    for (int c = 0; c < nchunk; ++c) {
      const int b = c & 1;
      ok = __all_sync(0xffffffffu,
                      (!*abort_flag && mbar_wait(smem_u32(&accf_bar[b]), (uint32_t)((c >> 1) & 1), status, 23)) ? 1
                                                                                                                 : 0) != 0;
      if (!ok) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int j4 = 0; j4 < T3 / 32; ++j4) {
        uint32_t r[32];
        TMEM_LD_32(lane_base + (uint32_t)(b * T3 + j4 * 32), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[j4 * 32 + i] += __uint_as_float(r[i]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[b])) : "memory");
    }
    if (ok && !*abort_flag) {
      // all MMAs (hence all TMA stages) are done: stage 0 holds each warp's
      // 32 x 33 transpose buffer, so C is written row by row, coalesced
      float* tb4 = reinterpret_cast<float*>(smem_raw + (smem_base - smem_u32(smem_raw))) + (warp - 2) * 4 * 32 * 33;
      const int row0 = bm * T3 + q * 32;
      // the whole accumulator row goes to shared memory first, so no
      // accumulator register stays live across the read-modify-write of C
#pragma unroll
      for (int j4 = 0; j4 < T3 / 32; ++j4)
#pragma unroll
        for (int i = 0; i < 32; ++i) tb4[j4 * 32 * 33 + lane * 33 + i] = acc[j4 * 32 + i];
      __syncwarp();
#pragma unroll 1
      for (int j4 = 0; j4 < T3 / 32; ++j4) {
        const float* tb = tb4 + j4 * 32 * 33;
        const int col = bn * T3 + j4 * 32 + lane;
        if (col < N && nk > 0) {
          // all 32 reads of C are issued before the first write, so the
          // read-modify-write costs one memory latency per 32 rows
          float cv[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int row = row0 + i;
            cv[i] = (beta != 0.f && row < M && (!lower || col <= row)) ? C[(long long)row * ldc + col] : 0.f;
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int row = row0 + i;
            if (row < M && (!lower || col <= row)) {
              const float v = alpha * tb[i * 33 + lane] + beta * cv[i];
              C[(long long)row * ldc + col] = v;
              if (csplit) {
                // this tile's rows of the A half were read by this CTA alone
                // (one column tile) and every MMA reading them has completed
                const float hi = tf32_rn(v);
                float* sp = csplit + (long long)row * 2 * kpc;
                sp[col] = hi;
                sp[kpc + col] = tf32_rn(v - hi);
              }
            }
          }
        } else if (csplit && col < kpc && nk > 0) {
          for (int i = 0; i < 32; ++i) {
            const int row = row0 + i;
            if (row < M) {
              float* sp = csplit + (long long)row * 2 * kpc;
              sp[col] = 0.f;
              sp[kpc + col] = 0.f;
            }
          }
        }
        __syncwarp();
      }
    }
  }
  __syncwarp();
  if (warp == 0 && lane == 0 && *abort_flag) {
    for (int it = 0; it < issued; ++it) {
      const int st = it % ST3;
      mbar_wait(smem_u32(&full_bar[st]), (uint32_t)((it / ST3) & 1), status, 24);
    }
  }
  // on abort, the MMAs already issued must retire before TMEM is freed
  if (warp == 1 && lane == 0 && *abort_flag) {
    umma_commit(smem_u32(&fin_bar));
    mbar_wait(smem_u32(&fin_bar), 0u, status, 25);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * T3));
  }
}

bool encode_split_map(CUtensorMap* map, float* base, int rows, int Kp) {
  EncodeTiledFn enc = (EncodeTiledFn)tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)(2 * Kp), (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)(2 * Kp) * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)KB3, (cuuint32_t)T3};
  cuuint32_t estride[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, gdim, gstride, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// The scratch is used as two fixed halves (A split, B split), so a tensor map
// depends only on the half's base and Kp and is encoded once: rows past the
// operand's size are read but their results are never stored.
size_t tc3_scratch_bytes(int M, int N, int K) {
  const long long Kp = ((K + KB3 - 1) / KB3) * KB3;
  const long long rows = M > N ? M : N;
  return (size_t)2 * rows * 2 * Kp * sizeof(float) + 1024;
}

void tc3_halves(const Tc3Scratch& sc, float** a_half, float** b_half) {
  const size_t half = sc.bytes > 1024 ? ((sc.bytes - 1024) / 2) / sizeof(float) / 32 * 32 : 0;   // floats per half
  *a_half = sc.buf;
  *b_half = sc.buf + half;
}

namespace {

struct MapEntry {
  const float* base;
  int Kp, rows;
  CUtensorMap map;
};
std::mutex g_map_mu;
std::vector<MapEntry> g_maps;

bool cached_map(float* base, int rows, int Kp, CUtensorMap* out) {
  std::lock_guard<std::mutex> lk(g_map_mu);
  // the key includes the row capacity, so a new scratch at a reused address
  // never inherits a map with a larger extent
  for (const MapEntry& e : g_maps)
    if (e.base == base && e.Kp == Kp && e.rows == rows) {
      *out = e.map;
      return true;
    }
  MapEntry e;
  e.base = base;
  e.Kp = Kp;
  e.rows = rows;
  if (!encode_split_map(&e.map, base, rows, Kp)) return false;
  if (g_maps.size() > 256) g_maps.clear();
  g_maps.push_back(e);
  *out = e.map;
  return true;
}

}  // namespace

dngd_status gemm_tc3(int M, int N, int K, float alpha, const float* A, long long lda, bool transA, const float* B,
                     long long ldb, bool transB, float beta, float* C, long long ldc, bool lower, const Tc3Scratch& sc,
                     int* status, cudaStream_t st, unsigned flags, const float* kscale_a) {
  if (M <= 0 || N <= 0) return DNGD_OK;
  if (!sc.buf || tc3_scratch_bytes(M, N, K) > sc.bytes || K <= 0) return DNGD_ERR_INVALID_ARG;
  if ((flags & TC3_C_SPLIT) && (lower || N > T3)) return DNGD_ERR_INVALID_ARG;
  const int Kp = ((K + KB3 - 1) / KB3) * KB3;
  const int kpc = ((N + KB3 - 1) / KB3) * KB3;
  if ((flags & TC3_C_SPLIT) && tc3_scratch_bytes(M, 0, N) > sc.bytes) return DNGD_ERR_INVALID_ARG;
  float *Ab, *Bh;
  tc3_halves(sc, &Ab, &Bh);
  const int cap_rows = (int)((size_t)(Bh - Ab) / (2 * (size_t)Kp));
  const bool same = A == B && lda == ldb && transA == transB && M == N;
  float* Bb = same ? Ab : Bh;
  if (!(flags & TC3_A_PRESPLIT)) {
    DNGD_NOTE_LAUNCH();
    k_tc3_split<<<dim3(Kp / 32, cdiv(M, 32)), 256, 0, st>>>(M, K, Kp, A, lda, transA ? 1 : 0, Ab, 0, kscale_a);
  }
  if (!same && !(flags & TC3_B_PRESPLIT)) {
    DNGD_NOTE_LAUNCH();
    k_tc3_split<<<dim3(Kp / 32, cdiv(N, 32)), 256, 0, st>>>(N, K, Kp, B, ldb, transB ? 1 : 0, Bb);
  }
  DNGD_LAUNCH_CHECK();
  CUtensorMap mapA, mapB;
  if (!cached_map(Ab, cap_rows, Kp, &mapA) || !cached_map(Bb, cap_rows, Kp, &mapB)) return DNGD_ERR_CUDA;
  static bool attr = false;
  if (!attr) {
    DNGD_CUDA_CHECK(cudaFuncSetAttribute(k_tc3, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM3));
    attr = true;
  }
  DNGD_NOTE_LAUNCH();
  k_tc3<<<dim3(cdiv(N, T3), cdiv(M, T3)), THREADS3, SMEM3, st>>>(mapA, mapB, M, N, Kp, alpha, beta, C, ldc,
                                                                 lower ? 1 : 0,
                                                                 (flags & TC3_C_SPLIT) ? Ab : nullptr, kpc, status);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// G independent products C_g = A_g B_g^T (line-search trials): A_g is
// already split in the scratch's A half as rows [g M, (g+1) M) of a
// [G M x 2 Kp] stack; B_g = B0 + g b_z ([N x K], ld ldb) is split here into
// the B half; C_g = C + g c_z.  One launch per operand kind.
dngd_status gemm_tc3_trials(int G, int M, int N, int K, const float* B0, long long ldb, long long b_z, float* C,
                            long long ldc, long long c_z, const Tc3Scratch& sc, int* status, cudaStream_t st) {
  if (G <= 0 || M <= 0 || N <= 0) return DNGD_OK;
  if (!sc.buf || K <= 0) return DNGD_ERR_INVALID_ARG;
  const int Kp = ((K + KB3 - 1) / KB3) * KB3;
  float *Ab, *Bh;
  tc3_halves(sc, &Ab, &Bh);
  const long long cap_rows = (long long)(Bh - Ab) / (2 * (long long)Kp);
  if ((long long)G * M > cap_rows || (long long)G * N > cap_rows) return DNGD_ERR_INVALID_ARG;
  DNGD_NOTE_LAUNCH();
  k_tc3_split<<<dim3(Kp / 32, cdiv(N, 32), G), 256, 0, st>>>(N, K, Kp, B0, ldb, 0, Bh, b_z);
  DNGD_LAUNCH_CHECK();
  CUtensorMap mapA, mapB;
  if (!cached_map(Ab, (int)cap_rows, Kp, &mapA) || !cached_map(Bh, (int)cap_rows, Kp, &mapB)) return DNGD_ERR_CUDA;
  static bool attr = false;
  if (!attr) {
    DNGD_CUDA_CHECK(cudaFuncSetAttribute(k_tc3, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM3));
    attr = true;
  }
  DNGD_NOTE_LAUNCH();
  k_tc3<<<dim3(cdiv(N, T3), cdiv(M, T3), G), THREADS3, SMEM3, st>>>(mapA, mapB, M, N, Kp, 1.0f, 0.0f, C, ldc, 0,
                                                                    nullptr, 0, status, M, N, c_z);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

}  // namespace dngd
