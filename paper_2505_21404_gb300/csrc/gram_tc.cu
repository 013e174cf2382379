// Residual Gramian K = J J^T on the 5th-generation tensor cores (tcgen05).
//
// K is symmetric (Def. 3.1 of the paper; its assembly algorithm fills one
// triangle and mirrors), so only the 128 x 256 output tiles that touch the
// lower triangle are computed.  Per CTA (one output tile, one K-range):
//   - warp 0 / lane 0 streams 128 x 64 (A) and 256 x 64 (B) operand tiles of
//     the low-precision J into a 4-stage shared-memory ring with TMA
//     (cp.async.bulk.tensor, 128-byte swizzle), signalling mbarriers;
//   - warp 1 / lane 0 issues tcgen05.mma (M = 128, N = 256, FP32 accumulator
//     in tensor memory, 256 columns) and releases each stage with
//     tcgen05.commit;
//   - all four warps drain the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w..32w+31 = tile rows) and store FP32 partial tiles.
// Operands: BF16 (kind::f16) or TF32 (kind::tf32); both use 128-byte K
// blocks (64 bf16 / 32 tf32) and 32-byte K steps per instruction.
// Split-K partials are summed in a fixed order by a reduction kernel that also
// adds the diagonal shift, so results are deterministic.
// Every mbarrier wait is bounded by a global-timer deadline; on expiry the
// kernel records ST_TIMEOUT, drains what it issued and frees its TMEM.
#include <cuda.h>

#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace dngd {

namespace {

using namespace tc;

constexpr int BM = 128, BN = 256, STAGES = 4;
constexpr int KBLK_BYTES = 128;                       // bytes of K per stage row
constexpr int A_BYTES = BM * KBLK_BYTES;              // 16 KB
constexpr int B_BYTES = BN * KBLK_BYTES;              // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;        // 48 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;

// Instruction descriptor: FP32 accumulator, A/B format (1 = BF16, 2 = TF32),
// both K-major, N = 256, M = 128.
template <int KIND>
__device__ __forceinline__ uint32_t make_idesc() {
  const uint32_t fmt = KIND == 0 ? 1u : 2u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// grid.x: tile index into tiles[] (pairs of row-block I, col-block J);
// grid.y: split index over the K blocks.
//
// Accumulation: a tensor-core accumulator that runs over tens of thousands of
// products loses accuracy (its FP32 additions are not round-to-nearest), and
// the Gram's error must stay far below lambda relative to ||K|| for the
// factor to precondition well.  So the MMAs accumulate only CH k-blocks
// (CH * 64 BF16 / 32 TF32 elements) in one of two TMEM buffers; eight
// epilogue warps then add that partial tile into round-to-nearest FP32
// registers (128 columns per thread) while the MMA warp fills the other
// buffer.  Warps: 0 = TMA producer, 1 = MMA issuer (+ TMEM owner), 2..9 =
// epilogue (warp w reads TMEM lanes 32*(w%4).., column half (w-2)/4).
constexpr int CH = 4;
constexpr int GRAM_THREADS = 320;
constexpr uint32_t TMEM_COLS2 = 512;

template <int KIND>
__global__ void __launch_bounds__(GRAM_THREADS, 1)
k_gram_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
          const int2* __restrict__ tiles, int m, int num_kblk, float* __restrict__ out, long long ldo,
          long long split_stride, int* status) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2];   // MMA -> epilogue: chunk ready in buffer b
  __shared__ __align__(8) uint64_t acce_bar[2];   // epilogue -> MMA: buffer b drained
  __shared__ __align__(8) uint64_t fin_bar;   // teardown: every issued MMA retired
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int2 tile = tiles[blockIdx.x];
  const int split = blockIdx.y, nsplit = gridDim.y;
  const int kb_per = (num_kblk + nsplit - 1) / nsplit;
  const int kb0 = split * kb_per;
  const int kb1 = min(num_kblk, kb0 + kb_per);
  const int nk = max(0, kb1 - kb0);
  const int nchunk = (nk + CH - 1) / CH;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf_bar[b]), 1);
      mbar_init(smem_u32(&acce_bar[b]), 8);
    }
    mbar_init(smem_u32(&fin_bar), 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TMEM_COLS2));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;
  volatile int* abort_flag = &abort_sh;

  int issued = 0;  // producer: stages issued (for draining on abort)
  if (warp == 0) {
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)((it / STAGES) & 1);
        if (*abort_flag || !mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, status, 1)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t fb = smem_u32(&full_bar[s]);
        mbar_expect_tx(fb, STAGE_BYTES);
        const uint32_t sa = smem_base + s * STAGE_BYTES;
        const int kcoord = (kb0 + it) * (KIND == 0 ? 64 : 32);
        tma_load_2d(sa, &mapA, fb, kcoord, tile.x * BM);
        tma_load_2d(sa + A_BYTES, &mapB, fb, kcoord, tile.y * BN);
        ++issued;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc<KIND>();
      for (int c = 0; c < nchunk && !*abort_flag; ++c) {
        const int b = c & 1, use = c >> 1;
        if (!mbar_wait(smem_u32(&acce_bar[b]), (uint32_t)((use & 1) ^ 1), status, 5)) {
          *abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t dbuf = tmem + (uint32_t)(b * BN);
        const int it0 = c * CH, it1 = min(nk, it0 + CH);
        for (int it = it0; it < it1; ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)((it / STAGES) & 1);
          if (*abort_flag || !mbar_wait(smem_u32(&full_bar[s]), ph, status, 2)) {
            *abort_flag = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t sa = smem_base + s * STAGE_BYTES;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            umma<KIND>(dbuf, sw128_desc(sa + 32 * k), sw128_desc(sa + A_BYTES + 32 * k), idesc,
                       (it > it0 || k > 0) ? 1u : 0u);
          }
          umma_commit(smem_u32(&empty_bar[s]));
        }
        umma_commit(smem_u32(&accf_bar[b]));  // fires when the chunk's MMAs are done
      }
    }
  } else {
    // epilogue warps 2..9
    const int q = warp & 3;             // TMEM lane quadrant this warp may access
    const int h = (warp - 2) >> 2;      // column half of the 256-column tile
    float acc[128];
#pragma unroll
    for (int j = 0; j < 128; ++j) acc[j] = 0.f;
    for (int c = 0; c < nchunk; ++c) {
      const int b = c & 1, use = c >> 1;
      const bool ok = __all_sync(0xffffffffu,
                                 (!*abort_flag && mbar_wait(smem_u32(&accf_bar[b]), (uint32_t)(use & 1), status, 3))
                                     ? 1
                                     : 0) != 0;
      if (!ok) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + h * 128);
#pragma unroll
      for (int j4 = 0; j4 < 4; ++j4) {
        uint32_t r[32];
        TMEM_LD_32(base + (uint32_t)(j4 * 32), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[j4 * 32 + i] += __uint_as_float(r[i]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[b])) : "memory");
    }
    const int row = tile.x * BM + q * 32 + lane;
    const int col0 = tile.y * BN + h * 128;
    if (row < m && !*abort_flag) {
      float* orow = out + (long long)split * split_stride + (long long)row * ldo;
      if (col0 + 128 <= m) {
        float4* dst = reinterpret_cast<float4*>(orow + col0);
#pragma unroll
        for (int j = 0; j < 32; ++j) dst[j] = make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 128; ++j)
          if (col0 + j < m) orow[col0 + j] = acc[j];
      }
    }
  }
  __syncwarp();

  // teardown: on abort, let issued TMA copies land before the CTA exits
  if (warp == 0 && lane == 0 && *abort_flag) {
    for (int it = 0; it < issued; ++it) {
      const int s = it % STAGES;
      mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((it / STAGES) & 1), status, 4);
    }
  }
  // on abort, the MMAs already issued must retire before TMEM is freed
  if (warp == 1 && lane == 0 && *abort_flag) {
    umma_commit(smem_u32(&fin_bar));
    mbar_wait(smem_u32(&fin_bar), 0u, status, 6);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS2));
  }
}

// K[i,j] (j <= i) = sum_s P_s[i,j] (+ shift on the diagonal); upper set to 0.
__global__ void k_gram_reduce(int m, int nsplit, const float* __restrict__ P, long long ldp, long long sstride,
                              float* __restrict__ K, long long ldk, double shift) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * m) return;
  const int i = (int)(idx / m), j = (int)(idx % m);
  float v = 0.f;
  if (j <= i) {
    for (int s = 0; s < nsplit; ++s) v += P[(long long)s * sstride + (long long)i * ldp + j];
    if (i == j) v += (float)shift;
  }
  K[(long long)i * ldk + j] = v;
}



EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

}  // namespace

void* tensor_map_encoder() { return (void*)get_encode(); }

struct GramPlan {
  int kind, m, n;
  long long ld;
  CUtensorMap mapA, mapB;
  int2* d_tiles = nullptr;
  int ntiles = 0, nsplit = 1, num_kblk = 0;
  float* K = nullptr;
  long long ldk = 0;
  float* partials = nullptr;
  long long ldp = 0, sstride = 0;
  double shift = 0.0;
};

int choose_splits(int ntiles, int num_kblk, int nsm) {
  int best = 1;
  double best_eff = 0.0;
  for (int s = 1; s <= 8; ++s) {
    if (num_kblk / s < 8) break;
    const long long units = (long long)ntiles * s;
    const long long waves = (units + nsm - 1) / nsm;
    const double eff = (double)units / (double)(waves * nsm);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = s;
    }
  }
  return best;
}

size_t gram_tc_partial_bytes(int m, int n) {
  // the split count gram_tc_plan will choose for this shape (K blocks of 64)
  const int nI = (m + BM - 1) / BM;
  int ntiles = 0;
  for (int I = 0; I < nI; ++I)
    for (int Jc = 0; Jc * BN <= I * BM + BM - 1 && Jc * BN < m; ++Jc) ++ntiles;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int nsplit = choose_splits(ntiles, (n + 31) / 32, nsm);
  const long long ldp = ((m + 3) / 4) * 4 + 4;
  return (size_t)nsplit * nI * BM * ldp * sizeof(float);
}

dngd_status gram_tc_plan(GramPlan** out, int kind, const void* Jlow, int m, int n, long long ld, float* K,
                         long long ldk, float* partials, size_t partial_bytes, cudaStream_t st) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return DNGD_ERR_CUDA;
  GramPlan* p = new GramPlan();
  p->kind = kind;
  p->m = m;
  p->n = n;
  p->ld = ld;
  p->K = K;
  p->ldk = ldk;
  const int elem = kind == 0 ? 2 : 4;
  const int kblk = KBLK_BYTES / elem;
  p->num_kblk = (n + kblk - 1) / kblk;
  if ((ld * elem) % 16 != 0) {
    delete p;
    return DNGD_ERR_INVALID_ARG;
  }
  const CUtensorMapDataType dt = kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  cuuint64_t gdim[2] = {(cuuint64_t)n, (cuuint64_t)m};
  cuuint64_t gstride[1] = {(cuuint64_t)(ld * elem)};
  cuuint32_t estride[2] = {1, 1};
  cuuint32_t boxA[2] = {(cuuint32_t)kblk, (cuuint32_t)BM};
  cuuint32_t boxB[2] = {(cuuint32_t)kblk, (cuuint32_t)BN};
  CUresult r1 = enc(&p->mapA, dt, 2, const_cast<void*>(Jlow), gdim, gstride, boxA, estride,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = enc(&p->mapB, dt, 2, const_cast<void*>(Jlow), gdim, gstride, boxB, estride,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
    delete p;
    return DNGD_ERR_CUDA;
  }
  std::vector<int2> tiles;
  const int nI = (m + BM - 1) / BM;
  for (int I = 0; I < nI; ++I)
    for (int Jc = 0; Jc * BN <= I * BM + BM - 1 && Jc * BN < m; ++Jc) tiles.push_back(make_int2(I, Jc));
  p->ntiles = (int)tiles.size();
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  p->nsplit = choose_splits(p->ntiles, p->num_kblk, nsm);
  const int mp = nI * BM;
  p->ldp = ((m + 3) / 4) * 4 + 4;
  p->sstride = (long long)mp * p->ldp;
  if ((size_t)p->nsplit * p->sstride * sizeof(float) > partial_bytes) p->nsplit = 1;
  if ((size_t)p->sstride * sizeof(float) > partial_bytes) {
    delete p;
    return DNGD_ERR_INVALID_ARG;
  }
  p->partials = partials;
  if (cudaMalloc(&p->d_tiles, sizeof(int2) * tiles.size()) != cudaSuccess) {
    delete p;
    return DNGD_ERR_OOM;
  }
  // stream-ordered before the runs (the host list is staged before return)
  if (cudaMemcpyAsync(p->d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, st) !=
      cudaSuccess) {
    cudaFree(p->d_tiles);
    delete p;
    return DNGD_ERR_CUDA;
  }
  static bool attr0 = false, attr1 = false;
  if (kind == 0 && !attr0) {
    cudaFuncSetAttribute(k_gram_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr0 = true;
  }
  if (kind == 1 && !attr1) {
    cudaFuncSetAttribute(k_gram_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr1 = true;
  }
  *out = p;
  return DNGD_OK;
}

dngd_status gram_tc_set_shift(GramPlan* p, double shift) {
  p->shift = shift;
  return DNGD_OK;
}

dngd_status gram_tc_run(GramPlan* p, int* status, cudaStream_t st, cudaEvent_t ev_before_mma,
                        cudaEvent_t ev_after_mma) {
  dim3 grid(p->ntiles, p->nsplit);
  if (ev_before_mma) cudaEventRecord(ev_before_mma, st);
  DNGD_NOTE_LAUNCH();
  if (p->kind == 0)
    k_gram_tc<0><<<grid, GRAM_THREADS, SMEM_BYTES, st>>>(p->mapA, p->mapB, p->d_tiles, p->m, p->num_kblk, p->partials,
                                                p->ldp, p->sstride, status);
  else
    k_gram_tc<1><<<grid, GRAM_THREADS, SMEM_BYTES, st>>>(p->mapA, p->mapB, p->d_tiles, p->m, p->num_kblk, p->partials,
                                                p->ldp, p->sstride, status);
  DNGD_LAUNCH_CHECK();
  if (ev_after_mma) cudaEventRecord(ev_after_mma, st);
  const long long tot = (long long)p->m * p->m;
  DNGD_NOTE_LAUNCH();
  k_gram_reduce<<<(int)((tot + 255) / 256), 256, 0, st>>>(p->m, p->nsplit, p->partials, p->ldp, p->sstride, p->K,
                                                          p->ldk, p->shift);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

void gram_tc_free(GramPlan* p) {
  if (!p) return;
  if (p->d_tiles) cudaFree(p->d_tiles);
  delete p;
}

int gram_tc_nsplit(const GramPlan* p) { return p->nsplit; }
int gram_tc_ntiles(const GramPlan* p) { return p->ntiles; }

}  // namespace dngd

// ---------------------------------------------------------------------------
// Allocation-free Gram entry point.
//
// Some callers cannot allocate device memory at the moment they need the
// Gram: code running under a framework that owns every device allocation (a
// caching allocator or a fixed memory pool), code inside a region where an
// allocation would synchronise the device and stall the surrounding work, or
// small embedded users that reserve memory once at start-up.  This
// entry point computes the same K = J J^T + shift I as the context's Gram
// (same tcgen05 kernel, same reduction) but takes its split-K partial tiles,
// its tile list and its status word from one file-scope device array of fixed
// size instead of cudaMalloc.
// ---------------------------------------------------------------------------

namespace dngd {
namespace {

constexpr size_t kNoAllocBytes = (size_t)16 << 20;       // 16 MiB per device
constexpr size_t kNoAllocStatusOff = 0;                   // int[4]
constexpr size_t kNoAllocTilesOff = 256;                  // int2 tile list
constexpr size_t kNoAllocTilesMax = 512;                  // tiles (m <= 2000 needs 72)
constexpr int kNoAllocMaxM = 2000;                        // largest m accepted
constexpr size_t kNoAllocPartOff = 256 + kNoAllocTilesMax * sizeof(int2);

// Every GPU that loads the library holds this array until the process exits.
// Host code must not use its name as a device address: the per-device address
// comes from cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char g_gram_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
unsigned char* g_scratch_addr[kNoAllocMaxDevices] = {};

// Writes the lower-triangle 128 x 256 tile list (row block I, column block J)
// into the scratch; one thread, ntiles is small.
__global__ void k_noalloc_tiles(int m, int2* tiles) {
  int t = 0;
  const int nI = (m + BM - 1) / BM;
  for (int I = 0; I < nI; ++I)
    for (int Jc = 0; Jc * BN <= I * BM + BM - 1 && Jc * BN < m; ++Jc) tiles[t++] = make_int2(I, Jc);
}

}  // namespace

}  // namespace dngd

extern "C" dngd_status dngd_gram_bf16_noalloc(const void* J, int m, int n, long long ld, float* K, long long ldk,
                                              double shift, void* stream) {
  using namespace dngd;
  if (!J || !K || m < 1 || n < 1 || ld < n || ldk < m) return DNGD_ERR_INVALID_ARG;
  if ((ld * 2) % 16 != 0 || ((uintptr_t)J % 16) != 0) return DNGD_ERR_INVALID_ARG;
  if (m > kNoAllocMaxM) {
    fprintf(stderr, "dngd_gram_bf16_noalloc: m = %d is above the maximum m = %d that its static scratch "
                    "array holds\n", m, kNoAllocMaxM);
    return DNGD_ERR_INVALID_ARG;
  }
  const int nI = (m + BM - 1) / BM;
  const long long mp = (long long)nI * BM;
  const long long ldp = ((m + 3) / 4) * 4 + 4;
  const size_t per_split = (size_t)mp * ldp * sizeof(float);
  const size_t cap = kNoAllocBytes - kNoAllocPartOff;
  // m <= 2000 needs at most 2048 x 2008 floats (16.4 MB) of one split
  static_assert((size_t)((kNoAllocMaxM + BM - 1) / BM) * BM * (((kNoAllocMaxM + 3) / 4) * 4 + 4) * sizeof(float) <=
                    kNoAllocBytes - kNoAllocPartOff,
                "the static scratch must hold one split of the largest accepted m");
  if (per_split > cap) return DNGD_ERR_INVALID_ARG;
  int ntiles = 0;
  for (int I = 0; I < nI; ++I)
    for (int Jc = 0; Jc * BN <= I * BM + BM - 1 && Jc * BN < m; ++Jc) ++ntiles;
  if ((size_t)ntiles > kNoAllocTilesMax) return DNGD_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return DNGD_ERR_CUDA;
  // once per device, with that device current: the device address of the array
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "dngd_gram_bf16_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
      return DNGD_ERR_CUDA;
    }
    if (cudaFuncSetAttribute(k_gram_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) !=
        cudaSuccess)
      return DNGD_ERR_CUDA;
    g_scratch_addr[dev] = (unsigned char*)p;
  }
  EncodeTiledFn enc = get_encode();
  if (!enc) return DNGD_ERR_CUDA;
  CUtensorMap mapA, mapB;
  cuuint64_t gdim[2] = {(cuuint64_t)n, (cuuint64_t)m};
  cuuint64_t gstride[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t estride[2] = {1, 1};
  cuuint32_t boxA[2] = {64, (cuuint32_t)BM};
  cuuint32_t boxB[2] = {64, (cuuint32_t)BN};
  if (enc(&mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(J), gdim, gstride, boxA, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      enc(&mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(J), gdim, gstride, boxB, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return DNGD_ERR_CUDA;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int num_kblk = (n + 63) / 64;
  int nsplit = choose_splits(ntiles, num_kblk, nsm);
  while (nsplit > 1 && (size_t)nsplit * per_split > cap) --nsplit;
  unsigned char* base = g_scratch_addr[dev];
  int* status = (int*)(base + kNoAllocStatusOff);
  int2* tiles = (int2*)(base + kNoAllocTilesOff);
  float* partials = (float*)(base + kNoAllocPartOff);
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear the status word
  if (cudaMemsetAsync(status, 0, 4 * sizeof(int), st) != cudaSuccess) return DNGD_ERR_CUDA;
  DNGD_NOTE_LAUNCH();
  k_noalloc_tiles<<<1, 1, 0, st>>>(m, tiles);
  DNGD_NOTE_LAUNCH();
  k_gram_tc<0><<<dim3(ntiles, nsplit), GRAM_THREADS, SMEM_BYTES, st>>>(mapA, mapB, tiles, m, num_kblk, partials, ldp,
                                                              (long long)mp * ldp, status);
  const long long tot = (long long)m * m;
  DNGD_NOTE_LAUNCH();
  k_gram_reduce<<<(int)((tot + 255) / 256), 256, 0, st>>>(m, nsplit, partials, ldp, (long long)mp * ldp, K, ldk,
                                                          shift);
  if (cudaGetLastError() != cudaSuccess) return DNGD_ERR_CUDA;
  int hs[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(hs, status, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DNGD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DNGD_ERR_CUDA;
  return (hs[0] & ST_TIMEOUT) ? DNGD_ERR_TIMEOUT : DNGD_OK;
}
