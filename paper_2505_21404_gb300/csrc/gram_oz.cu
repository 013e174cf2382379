// Exact Gram K = J J^T of an FP32 matrix on the BF16 tensor cores.
//
// The dual solve needs K accurate to far below lambda: at lambda = 1e-5 and
// ||K|| ~ 1e4 (Sec. 3.1's K + lambda I, with cond ~ 1e9 late in training) a
// BF16 or FP32 Gram is indefinite at the lambda scale, and only an exact
// Gram factored in FP64 makes the refinement converge in one iteration; with
// an exact FP64 Gram the refinement operator is also one m x m GEMV instead
// of two GEMVs over J.  GB300's FP64 rate is ~1 TFLOP/s, so the Gram is
// built from exact integer products (an error-free splitting in the spirit
// of Ozaki et al.):
//
//   * each row i of J is scaled by 2^-E_i (E_i = exponent of the row's
//     largest entry, plus one) and split into four signed 8-bit integers,
//       J[i,k] = 2^E_i sum_{s<4} sigma_s[i,k] 2^(-8(s+1)) + r,
//       |sigma_s| <= 128,  |r| <= 2^(E_i - 33);
//     the slices are exact in BF16;
//   * with L_g = sum_{s+t=g} sigma_s sigma_t^T (integer matrices),
//       K[i,j] = 2^(E_i+E_j-48) sum_{g<=4} 2^(8(4-g)) L_g[i,j]
//     (13 slice products; the dropped s+t >= 5 terms are below 2^-40 of the
//     row scales);
//   * products of slices are exact in the tensor cores; for levels 0-2 every
//     chunk the MMAs accumulate in TMEM stays within 2^24 in magnitude
//     (level g with n_g products is drained every 2^10 / n_g K columns), so
//     the FP32 accumulator is exact; levels 3 and 4 (weights 2^-24 and
//     2^-32 of level 0) are drained every 2048 columns and round in FP32
//     (chunks below 2^27 units of level 3, so a unit is at most 8): even
//     with each of a chunk's 896 MMA additions (levels 3 and 4 share one
//     accumulator) off by a full unit in the same direction this adds at
//     most 2^-38 of the row scales times n (896 x 8 x 2^8 x 2^-48 / 2048),
//     below the slicing's own 2^-32; the epilogue adds each chunk into
//     double-float registers (48-bit significand).
//
// Kernel roles (one 128 x TN output tile touching the lower triangle and
// one K range per CTA; TN = 128 for an FP32 Jacobian, 96 for an FP64 one):
// warp 0 lane 0 streams, per 32-wide K block, all four A slices and all
// four B slices with TMA (64-byte swizzle) into a ring of stages, so one
// stage feeds every slice product; warp 1 lane 0 issues tcgen05.mma (M =
// 128, N = TN) into four or five TMEM accumulators (levels 0, 1, 2 and the
// rounded levels; the slices are stored pre-scaled by 2^(-8 s), so a
// product carries its level's weight and levels can share an accumulator)
// and commits an accumulator at the end of its chunk; the chunk boundaries
// are staggered and an accumulator that starts a chunk is issued last in
// its stage, so its drain overlaps the other accumulators' MMAs; warps
// 2..9 drain an accumulator as soon as it is committed (two warps per TMEM
// lane quadrant, TN / 2 columns each), release it to the MMA warp, and add
// it into double-float registers.
// Split-K partial tiles (FP64) are summed in a fixed order by the reduction,
// which applies the row scales and writes the full FP64 Gram (the
// refinement operator) and its FP32 lower triangle plus the diagonal shift
// (the matrix the FP32 preconditioner factors).  Every wait is bounded
// (ST_TIMEOUT, drain, free TMEM).
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>

#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "step_kernels.h"
#include "tc_ptx.cuh"

namespace dngd {

namespace {

using namespace tc;

// Configurations <NS, NG>: NS 8-bit slices per value; the products
// sigma_s sigma_t^T are summed by level g = s + t <= NG - 1.  A level's
// products go to one of NA TMEM accumulators of TN columns (NA x TN <= 512):
// accumulator a takes the levels [lo(a), hi(a)].
// * PRE (pre-scaled slices): slice s is stored as sigma_s 2^(-8 s), exact in
//   BF16, so every product already carries its level's weight 2^(-8 g) and
//   levels may share an accumulator.  The exact levels 0-2 keep one each
//   (their chunks sum integers times 2^(-8 g), exact below 2^24 units); the
//   rounded levels >= 3 share one, whose FP32 rounding is relative to level
//   3's magnitude, ~2^-48 of level 0.  Without PRE (integer slices) every
//   level has its own accumulator and the epilogue applies the weights.
// * <4, 5>: levels g <= 4 (13 of the 16 products), for the FP32 Jacobian,
//   whose own rounding is far larger than the dropped terms.
// * <4, 6>: also level 5 (15 products), for the FP64 Jacobian.  The dropped
//   levels are not unbiased noise (on the diagonal they are a sum of
//   squares), so for an accurate J the truncation is what limits the Gram,
//   not the slicing: level 5 brings the step error at a trained theta from
//   1.5e-4 to 6e-6 (CPU emulation), as close as a fifth slice would.
// * <6, 7>: six integer slices, levels g <= 6 (26 of 36 products), for the
//   trailing updates of the FP64 factorisation (K extent 64: every chunk
//   exact, one accumulator per level).
template <int NS, int NG>
struct OzCfg;
template <>
struct OzCfg<4, 5> {
  static constexpr int TN = 128, OST = 3, NA = 4;
  static constexpr bool PRE = true;
  __host__ __device__ static constexpr int lo(int a) { return a; }
  __host__ __device__ static constexpr int hi(int a) { return a < 3 ? a : 4; }
  // Stages per chunk of accumulator a.  Levels 0-2 are exact: n_g = g_hi -
  // g_lo + 1 products of |sigma| <= 128 over period x 32 columns stay within
  // 2^24 units (1 x 32 x 32, 2 x 16 x 32, 3 x 10 x 32, times 2^14).  The
  // rounded levels run 64 stages (their error bound is in the header).
  __host__ __device__ static constexpr int period(int a) { return a == 0 ? 32 : a == 1 ? 16 : a == 2 ? 10 : 64; }
  // Offsets that stagger the accumulators' chunk boundaries (the first chunk
  // of accumulator a is period - offset stages long): chunk ends fall on
  // stages 31, 10/26, 7 + 10 i (modulo 32) and 52 (modulo 64).
  __host__ __device__ static constexpr int offset(int a) { return a == 0 ? 0 : a == 1 ? 5 : a == 2 ? 2 : 11; }
};
template <>
struct OzCfg<4, 6> {
  // With an FP64 Jacobian the rounded levels must not share one accumulator:
  // with levels 3-5 together (128 x 128 tiles) the step error at a trained
  // theta rose from 1.3e-5 to 2.0e-4 (measured), the smaller levels' sums
  // being cut at the ulps of level 3's.  Level 3 keeps its own accumulator
  // and level 5 (2 products, weight 2^-8 of level 4) shares level 4's: five
  // accumulators of 96 columns.
  static constexpr int TN = 96, OST = 4, NA = 5;
  static constexpr bool PRE = true;
  __host__ __device__ static constexpr int lo(int a) { return a; }
  __host__ __device__ static constexpr int hi(int a) { return a < 4 ? a : 5; }
  __host__ __device__ static constexpr int period(int a) { return a == 0 ? 32 : a == 1 ? 16 : a == 2 ? 10 : 64; }
  // chunk ends on stages 31, 10/26, 7 + 10 i (modulo 32), 52 and 38 (modulo 64)
  __host__ __device__ static constexpr int offset(int a) {
    return a == 0 ? 0 : a == 1 ? 5 : a == 2 ? 2 : a == 3 ? 11 : 25;
  }
};
template <>
struct OzCfg<6, 7> {
  static constexpr int TN = 64, OST = 2, NA = 7;
  static constexpr bool PRE = false;
  __host__ __device__ static constexpr int lo(int a) { return a; }
  __host__ __device__ static constexpr int hi(int a) { return a; }
  // K extent 64 = two stages: one chunk per level, 2 x 32 x 6 x 2^14 < 2^24,
  // so every level is exact.
  __host__ __device__ static constexpr int period(int a) { return a >= 0 ? 2 : 2; }
  __host__ __device__ static constexpr int offset(int a) { return a >= 0 ? 0 : 0; }
};

constexpr int TM = 128;                     // output tile rows
constexpr int KS = 32;                      // K per stage (64-byte rows, 64-byte swizzle)
constexpr int A_TILE = TM * 64;             // 8 KB
constexpr uint32_t OTMEM = 512;             // NA accumulators of TN columns

// Warps: 0 TMA, 1 MMA, then the epilogue warps, epi_warps / 4 per TMEM lane
// quadrant, each draining cpw of the tile's columns: sixteen for the FP64-J
// Gram and GEMM and for the factor's sliced update (shorter drains, so an
// accumulator that starts a new chunk waits less; in the update the
// epilogue sets the persistent kernel's period per tile), eight for the
// FP32-J Gram.
template <int NS, int NG>
__host__ __device__ constexpr int epi_warps() { return (NS == 6 || NG == 6) ? 16 : 8; }
template <int NS, int NG>
__host__ __device__ constexpr int cpw() { return OzCfg<NS, NG>::TN * 4 / epi_warps<NS, NG>(); }
template <int NS, int NG>
__host__ __device__ constexpr int othreads() { return 64 + 32 * epi_warps<NS, NG>(); }
template <int NS, int NG>
__host__ __device__ constexpr int b_tile() { return OzCfg<NS, NG>::TN * 64; }
template <int NS, int NG>
__host__ __device__ constexpr int ostage() { return NS * (A_TILE + b_tile<NS, NG>()); }
// The update configuration (six slices) also holds each epilogue warp's
// 32 x (cpw + 1) FP64 block of C.
template <int NS, int NG>
__host__ __device__ constexpr int cstage() {
  return NS == 6 ? epi_warps<NS, NG>() * 32 * (cpw<NS, NG>() + 1) * (int)sizeof(double) : 0;
}
template <int NS, int NG>
__host__ __device__ constexpr int osmem() { return OzCfg<NS, NG>::OST * ostage<NS, NG>() + cstage<NS, NG>() + 1024; }

template <int NS>
__host__ __device__ __forceinline__ int g_lo(int g) { return g > NS - 1 ? g - (NS - 1) : 0; }
template <int NS>
__host__ __device__ __forceinline__ int g_hi(int g) { return g < NS - 1 ? g : NS - 1; }

static_assert(32 * 32 * 1 <= 1024 && 16 * 32 * 2 <= 1024 && 10 * 32 * 3 <= 1024 && 2 * 32 * 6 <= 1024,
              "an exact chunk must stay within 2^24 = 2^10 x 2^14");
static_assert(OzCfg<4, 5>::NA * OzCfg<4, 5>::TN <= (int)OTMEM && OzCfg<4, 6>::NA * OzCfg<4, 6>::TN <= (int)OTMEM &&
                  OzCfg<6, 7>::NA * OzCfg<6, 7>::TN <= (int)OTMEM,
              "the accumulators must fit the TMEM allocation");
static_assert(OzCfg<4, 5>::hi(OzCfg<4, 5>::NA - 1) == 4 && OzCfg<4, 6>::hi(OzCfg<4, 6>::NA - 1) == 5 &&
                  OzCfg<6, 7>::hi(OzCfg<6, 7>::NA - 1) == 6,
              "the accumulators cover every kept level");
static_assert(osmem<4, 5>() <= 227 * 1024 && osmem<4, 6>() <= 227 * 1024 && osmem<6, 7>() <= 227 * 1024,
              "shared-memory ring too large");
static_assert(epi_warps<6, 7>() * 32 * (cpw<6, 7>() + 1) * (int)sizeof(double) == cstage<6, 7>(),
              "the update epilogue keeps one block of C per epilogue warp");
static_assert(cpw<6, 7>() % 8 == 0 && cpw<6, 7>() <= 32 && cpw<4, 5>() % 8 == 0 && cpw<4, 6>() % 8 == 0 &&
                  cpw<4, 5>() <= 64 && cpw<4, 6>() <= 64,
              "an epilogue warp drains whole 8-column blocks (at most 32 for the update's staged sub-tile)");
static_assert(b_tile<4, 5>() % 1024 == 0 && b_tile<4, 6>() % 1024 == 0 && b_tile<6, 7>() % 1024 == 0,
              "tiles keep 1024-byte alignment");

// Chunk c of accumulator a covers stages [start, end]: start = 0 for c = 0,
// else c period - offset; end = (c + 1) period - offset - 1, clamped to
// nk - 1.
template <int NS, int NG>
__device__ __forceinline__ int chunk_end(int a, int c, int nk) {
  return min(nk - 1, (c + 1) * OzCfg<NS, NG>::period(a) - OzCfg<NS, NG>::offset(a) - 1);
}

// BF16 x BF16 -> FP32, both K-major, M = 128, N = TN.
template <int TN>
__device__ __forceinline__ uint32_t oz_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// Epilogue modes of the sliced product kernel:
//   OZ_PARTIAL  the tile's raw level sum into the split-K partial tiles;
//   OZ_UPDATE   the factorisation's trailing update C[i, j] -= 2^(E_i + E_j -
//               eshift) acc for the entries j <= i of the trailing block
//               (rows and columns row_off + index, exponents rexpA);
//   OZ_GEMM     C[i, j] = alpha 2^(EA_i + EB_j - eshift) acc + beta C[i, j]
//               (i < m, j < ncols; tiles from blockIdx, ntn column tiles).
enum { OZ_PARTIAL = 0, OZ_UPDATE = 1, OZ_GEMM = 2 };
struct OzEpi {
  double* C;
  long long ldc;
  const int* rexpA;
  const int* rexpB;
  int eshift;
  int ncols, ntn;
  double alpha, beta;
};

// (hi, lo) += c exactly as long as the sum needs at most ~48 bits.
__device__ __forceinline__ void df_add_exact(float& hi, float& lo, float c) {
  const float s = hi + c;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (c - bp);
  const float l = lo + e;
  const float t = s + l;
  lo = l - (t - s);
  hi = t;
}

// Weight 2^(-8 s) of slice s in the pre-scaled layout (exact in BF16 for the
// slice values |sigma| <= 128 and s <= 3).
__device__ __forceinline__ float slice_weight(int s) { return __int_as_float((127 - 8 * s) << 23); }

// The ND balanced base-256 digits of v = round(x 2^(8 ND - E)) for a double
// x with |x| < 2^(E - 1), from x's bits with integer operations only (FP64
// arithmetic is slow on this GPU): x 2^-E = sum_s d_s 2^-8(s+1) to within
// 2^-(8 ND + 1), every |d_s| <= 128 (so exact in BF16).  Zero and
// subnormal x give zero digits (subnormals lie far below that bound).
template <int ND>
__device__ __forceinline__ void oz_digits(double x, int E, float (&d)[ND]) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long v = 0;
  if (ex != 0 && ex != 0x7FF) {
    const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
    const int sh = 1075 - ex - 8 * ND + E;   // >= 6 for |x| < 2^(E - 1) and ND <= 6
    v = (sh >= 1 && sh < 64) ? (mant + (1LL << (sh - 1))) >> sh : 0;
    if (bits < 0) v = -v;
  }
#pragma unroll
  for (int s = ND - 1; s >= 1; --s) {
    int r = (int)(v & 255);    // v mod 256 (two's complement)
    if (r >= 128) r -= 256;    // balanced digit in [-128, 127]
    d[s] = (float)r;           // 32-bit conversion: a 64-bit one runs on the slow FP64 pipe
    v = (v - r) >> 8;          // exact
  }
  d[0] = (float)(int)v;        // |v| <= 128
}

// |x| as ordered integer bits (non-negative doubles compare like their bits)
__device__ __forceinline__ long long abs_bits(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL; }
// E with |x| / 2^E < 0.5 for the largest |x| given by its bits (1 for zero)
__device__ __forceinline__ int exp_of_abs_bits(long long b) {
  const int ex = (int)(b >> 52);
  return ex == 0 ? 1 : ex - 1021;   // |x| = f 2^(ex - 1022), f in [0.5, 1)
}

// Row scaling and slicing: one block per row, 16-byte loads (four FP32 or
// two pairs of FP64 entries) and 8-byte stores (ldJ and ldb are multiples of
// 4; the row's pad columns are zero).  The row's largest |J| (as a float)
// comes from the Jacobian's writer, so J is read once.  A float that rounded
// a double maximum down keeps |J| / 2^E below 0.5 (1 + 2^-24), so the first
// slice still stays within +-128.
template <typename TJ>
__global__ void __launch_bounds__(256) k_oz_slice(int m, int n, const TJ* __restrict__ J, long long ldJ,
                                                  __nv_bfloat16* __restrict__ S, long long ldS, int ldb,
                                                  const unsigned* __restrict__ rowmax, int* __restrict__ rowexp) {
  const int i = blockIdx.x;
  const TJ* row = J + (long long)i * ldJ;
  const int n4 = (n + 3) / 4, b4 = ldb / 4;
  const float a = __uint_as_float(rowmax[i]);
  int e = 0;
  if (a > 0.f && a <= 3.0e38f) frexpf(a, &e);   // a = f 2^e, f in [0.5, 1)
  const int E = e + 1;                          // |J| / 2^E < 0.5
  if (threadIdx.x == 0) rowexp[i] = E;
  __nv_bfloat16* srow = S + (long long)i * ldS;
  for (int k = threadIdx.x; k < b4; k += blockDim.x) {
    TJ x[4];
    if (k < n4) {
      if constexpr (sizeof(TJ) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(row) + k);
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
      } else {
        const double2 v0 = __ldg(reinterpret_cast<const double2*>(row) + 2 * k);
        const double2 v1 = __ldg(reinterpret_cast<const double2*>(row) + 2 * k + 1);
        x[0] = v0.x;
        x[1] = v0.y;
        x[2] = v1.x;
        x[3] = v1.y;
      }
    } else {
      x[0] = x[1] = x[2] = x[3] = TJ(0);
    }
    if constexpr (sizeof(TJ) == 4) {
#pragma unroll
      for (int c = 0; c < 4; ++c) x[c] = (4 * k + c < n) ? ldexpf(x[c], -E) : 0.f;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        __nv_bfloat16 q[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float t = x[c] * 256.f;
          const float sg = rintf(t);
          x[c] = t - sg;
          q[c] = __float2bfloat16_rn(sg * slice_weight(s));
        }
        *reinterpret_cast<uint2*>(srow + (long long)s * ldb + 4 * k) = *reinterpret_cast<const uint2*>(q);
      }
    } else {
      float d[4][4];
#pragma unroll
      for (int c = 0; c < 4; ++c) oz_digits<4>(4 * k + c < n ? (double)x[c] : 0.0, E, d[c]);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        __nv_bfloat16 q[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) q[c] = __float2bfloat16_rn(d[c][s] * slice_weight(s));
        *reinterpret_cast<uint2*>(srow + (long long)s * ldb + 4 * k) = *reinterpret_cast<const uint2*>(q);
      }
    }
  }
}

// One CTA per (output tile, K split).  m: rows of the output (for the
// Gram and the update also its columns); its row i sits at slice row
// row_off + i.  MODE: the epilogue (OZ_PARTIAL, OZ_UPDATE, OZ_GEMM).
template <int NS, int NG, int MODE>
__global__ void __launch_bounds__(othreads<NS, NG>(), 1)
k_gram_oz(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
          const int2* __restrict__ tiles, int m, int row_off, int num_kblk, int ldb, double* __restrict__ out,
          long long ldo, long long split_stride, OzEpi epi, int* status) {
  using Cfg = OzCfg<NS, NG>;
  constexpr int TN = Cfg::TN, OST = Cfg::OST, NA = Cfg::NA, EPI = epi_warps<NS, NG>();
  constexpr int B_TILE = b_tile<NS, NG>(), OSTAGE = ostage<NS, NG>();
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[OST];
  __shared__ __align__(8) uint64_t empty_bar[OST];
  __shared__ __align__(8) uint64_t accf_bar[NA];   // MMA -> epilogue: accumulator a committed
  __shared__ __align__(8) uint64_t acce_bar[NA];   // epilogue -> MMA: accumulator a drained
  __shared__ __align__(8) uint64_t fin_bar;    // teardown: every issued MMA retired
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  // OZ_UPDATE runs persistent: CTA b takes the tiles b, b + gridDim.x, ...
  // of the epi.ncols listed, one after another; tile c is chunk c of every
  // accumulator (its K extent is one chunk), so the MMA warp's chunk logic
  // carries over unchanged and the next tile's operands load while the
  // epilogue finishes the previous one
  constexpr bool PERSIST = MODE == OZ_UPDATE;
  const int my_tiles = PERSIST ? max(0, (epi.ncols - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x) : 1;
  const int2 tile = MODE == OZ_GEMM ? make_int2((int)blockIdx.x / epi.ntn, (int)blockIdx.x % epi.ntn)
                                    : tiles[blockIdx.x];
  const int split = blockIdx.y, nsplit = gridDim.y;
  const int kb_per = (num_kblk + nsplit - 1) / nsplit;
  const int kb0 = split * kb_per;
  const int kb1 = min(num_kblk, kb0 + kb_per);
  const int nk_tile = max(0, kb1 - kb0);
  const int nk = nk_tile * my_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OST; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int a = 0; a < NA; ++a) {
      mbar_init(smem_u32(&accf_bar[a]), 1);
      mbar_init(smem_u32(&acce_bar[a]), EPI);
    }
    mbar_init(smem_u32(&fin_bar), 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(OTMEM));
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
        const int st = it % OST;
        const uint32_t ph = (uint32_t)((it / OST) & 1);
        if (*abort_flag || !mbar_wait(smem_u32(&empty_bar[st]), ph ^ 1u, status, 11)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t fb = smem_u32(&full_bar[st]);
        mbar_expect_tx(fb, OSTAGE);
        const uint32_t sbase = smem_base + st * OSTAGE;
        const int2 tl = PERSIST ? tiles[blockIdx.x + (it / nk_tile) * gridDim.x] : tile;
        const int kc = (kb0 + (PERSIST ? it % nk_tile : it)) * KS;
#pragma unroll
        for (int sl = 0; sl < NS; ++sl) {
          tma_load_2d(sbase + sl * A_TILE, &mapA, fb, sl * ldb + kc, row_off + tl.x * TM);
          tma_load_2d(sbase + NS * A_TILE + sl * B_TILE, &mapB, fb, sl * ldb + kc, row_off + tl.y * TN);
        }
        ++issued;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = oz_idesc<TN>();
      // per accumulator: current chunk, its first and last stage
      int cidx[NA], cstart[NA], cend[NA];
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        cidx[a] = 0;
        cstart[a] = 0;
        cend[a] = chunk_end<NS, NG>(a, 0, nk);
      }
      for (int it = 0; it < nk && !*abort_flag; ++it) {
        const int st = it % OST;
        const uint32_t ph = (uint32_t)((it / OST) & 1);
        if (!mbar_wait(smem_u32(&full_bar[st]), ph, status, 12)) {
          *abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sbase = smem_base + st * OSTAGE;
        // descriptors of the stage's first A and B tiles; the others differ
        // only in the start-address field (byte offset / 16, no carry out)
        const uint64_t da0 = sw64_desc(sbase), db0 = sw64_desc(sbase + NS * A_TILE);
        // pass 0: accumulators inside a chunk; pass 1: those starting one,
        // which first wait until their previous chunk has been drained
        bool stop = false;
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
          for (int a = 0; a < NA; ++a) {
            const bool first = cstart[a] == it;
            if (first != (pass == 1) || stop) continue;
            if (first) {
              if (!mbar_wait(smem_u32(&acce_bar[a]), (uint32_t)((cidx[a] & 1) ^ 1), status, 15)) {
                *abort_flag = 1;
                stop = true;
                continue;
              }
              asm volatile("tcgen05.fence::after_thread_sync;");
            }
            const uint32_t dbuf = tmem + (uint32_t)(a * TN);
#pragma unroll
            for (int g = Cfg::lo(a); g <= Cfg::hi(a); ++g) {
#pragma unroll
              for (int sa = g_lo<NS>(g); sa <= g_hi<NS>(g); ++sa) {
#pragma unroll
                for (int k = 0; k < KS / 16; ++k) {
                  umma<0>(dbuf, da0 + (uint64_t)((sa * A_TILE + 32 * k) >> 4),
                          db0 + (uint64_t)(((g - sa) * B_TILE + 32 * k) >> 4), idesc,
                          (first && g == Cfg::lo(a) && sa == g_lo<NS>(g) && k == 0) ? 0u : 1u);
                }
              }
            }
            if (cend[a] == it) {
              umma_commit(smem_u32(&accf_bar[a]));
              ++cidx[a];
              cstart[a] = it + 1;
              cend[a] = chunk_end<NS, NG>(a, cidx[a], nk);
            }
          }
        }
        if (stop) break;
        umma_commit(smem_u32(&empty_bar[st]));
      }
    }
  } else {
    constexpr int CPW = cpw<NS, NG>();
    const int q = warp & 3;             // TMEM lane quadrant this warp may access
    const int cg = (warp - 2) >> 2;     // column half: CPW of the TN columns
    const int ncol = CPW;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cg * CPW);
    float hi[CPW], lo[CPW];
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
      hi[j] = 0.f;
      lo[j] = 0.f;
    }
    int2 tcur = PERSIST ? (my_tiles > 0 ? tiles[blockIdx.x] : make_int2(0, 0)) : tile;
    int row = tcur.x * TM + q * 32 + lane;
    int col0 = tcur.y * TN + cg * CPW;
    // OZ_UPDATE: the warp's 32 x cpw sub-tile of C (lane = column) is copied
    // into its own shared-memory block while the operands load and the MMAs
    // run
    double* cs = reinterpret_cast<double*>(smem_raw + (smem_base - smem_u32(smem_raw)) + OST * OSTAGE) +
                 (warp - 2) * 32 * (CPW + 1);
    auto prefetch_c = [&](int2 t) {
      const int col = t.y * TN + cg * CPW + lane;
#pragma unroll 8
      for (int rr = 0; rr < 32; ++rr) {
        const int rw = t.x * TM + q * 32 + rr;
        if (lane < ncol && rw < m && col <= rw)
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(cs + rr * (CPW + 1) + lane)),
                       "l"(epi.C + (long long)(row_off + rw) * epi.ldc + row_off + col)
                       : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // the update, scaled by 2^(E_row + E_col - eshift), is subtracted in the
    // shared copy by the thread of its row; the copy then goes back row by
    // row (lane = column), coalesced
    auto update_c = [&]() {
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncwarp();
      // row exponent per lane; the 32 column exponents loaded once (lane =
      // column) and broadcast
      const int er = row < m ? epi.rexpA[row_off + row] : 0;
      const int ecl = (lane < ncol && col0 + lane < m) ? epi.rexpA[row_off + col0 + lane] : 0;
      // all 32 values first (branch-free; the rare ones that need the FP64
      // path are fixed up afterwards), then the read-modify-write
      double vv[CPW];
      unsigned slow = 0u;
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        const int ec = __shfl_sync(0xffffffffu, ecl, j);
        bool sl;
        vv[j] = df_to_double_try(hi[j], lo[j], er + ec - epi.eshift, sl);
        slow |= sl ? (1u << j) : 0u;
      }
      if (__any_sync(0xffffffffu, slow != 0u)) {
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          const int ec = __shfl_sync(0xffffffffu, ecl, j);
          if ((slow >> j) & 1u) vv[j] = df_to_double_slow(hi[j], lo[j], er + ec - epi.eshift);
        }
      }
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        const int cj = col0 + j;
        if (j < ncol && row < m && cj <= row) cs[lane * (CPW + 1) + j] -= vv[j];
      }
      __syncwarp();
      if (!*abort_flag && lane < ncol) {
        const int col = col0 + lane;
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
          const int rw = tcur.x * TM + q * 32 + rr;
          if (rw < m && col <= rw)
            epi.C[(long long)(row_off + rw) * epi.ldc + row_off + col] = cs[rr * (CPW + 1) + lane];
        }
      }
      __syncwarp();
    };
    if (MODE == OZ_UPDATE && my_tiles > 0) prefetch_c(tcur);
    // the chunks in the order the MMA warp commits them: by last stage, a
    // chunk of one stage (issued in the second pass) after the others, then
    // by accumulator
    int cidx[NA], cstart[NA], cend[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      cidx[a] = 0;
      cstart[a] = 0;
      cend[a] = nk > 0 ? chunk_end<NS, NG>(a, 0, nk) : INT_MAX;
    }
    while (!*abort_flag) {
      int asel = -1, kbest = INT_MAX;
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        if (cend[a] == INT_MAX) continue;
        const int key = cend[a] * 2 + (cstart[a] == cend[a] ? 1 : 0);
        if (key < kbest) {
          kbest = key;
          asel = a;
        }
      }
      if (asel < 0) break;
      const bool ok =
          __all_sync(0xffffffffu, (!*abort_flag && mbar_wait(smem_u32(&accf_bar[asel]), (uint32_t)(cidx[asel] & 1),
                                                             status, 13))
                                      ? 1
                                      : 0) != 0;
      if (!ok) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      // the chunk times 2^(8 (NG - 1)) with pre-scaled slices, else times its
      // level's weight 2^(8 (NG - 1 - g)) (a power of two: exact), read in
      // blocks of 8 columns to keep the registers low
      const float sc = __int_as_float((127 + 8 * (NG - 1 - (Cfg::PRE ? 0 : asel))) << 23);
#pragma unroll
      for (int h = 0; h < CPW / 8; ++h) {
        uint32_t r[8];
        TMEM_LD_8(lane_base + (uint32_t)(asel * TN + 8 * h), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 8; ++i) df_add_exact(hi[8 * h + i], lo[8 * h + i], __uint_as_float(r[i]) * sc);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[asel])) : "memory");
      // next chunk of this accumulator
#pragma unroll
      for (int a = 0; a < NA; ++a)
        if (a == asel) {
          const int e = cend[a];
          ++cidx[a];
          cstart[a] = e + 1;
          cend[a] = e + 1 < nk ? chunk_end<NS, NG>(a, cidx[a], nk) : INT_MAX;
        }
      if (PERSIST && asel == NA - 1) {
        // every accumulator of tile c = cidx - 1 is drained: finish the tile,
        // start the next one's C copy
        update_c();
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          hi[j] = 0.f;
          lo[j] = 0.f;
        }
        const int cn = cidx[NA - 1];
        if (cn < my_tiles) {
          tcur = tiles[blockIdx.x + cn * gridDim.x];
          row = tcur.x * TM + q * 32 + lane;
          col0 = tcur.y * TN + cg * CPW;
          prefetch_c(tcur);
        }
      }
    }
    if (MODE == OZ_UPDATE) {
      // every tile was finished in the loop; copies still in flight after an
      // abort complete before the shared memory is released
      asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (MODE == OZ_GEMM) {
      // the tile, scaled by alpha 2^(EA_row + EB_col - eshift), goes through
      // shared memory (the operand ring is idle: every MMA has completed)
      // and is written row by row (lane = column), coalesced
      constexpr int TS = CPW + 1;
      static_assert(MODE != OZ_GEMM || EPI * 32 * TS * (int)sizeof(double) <= OST * OSTAGE,
                    "the GEMM epilogue stages its sub-tiles in the operand ring");
      double* tb = reinterpret_cast<double*>(smem_raw + (smem_base - smem_u32(smem_raw))) + (warp - 2) * 32 * TS;
      const int er = row < m ? epi.rexpA[row] : 0;
      const int eb0 = (lane < CPW && col0 + lane < epi.ncols) ? epi.rexpB[col0 + lane] : 0;
      const int eb1 = (lane + 32 < CPW && col0 + lane + 32 < epi.ncols) ? epi.rexpB[col0 + lane + 32] : 0;
      unsigned long long slow = 0ull;
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        const int eb = __shfl_sync(0xffffffffu, j < 32 ? eb0 : eb1, j & 31);
        bool sl;
        tb[lane * TS + j] = epi.alpha * df_to_double_try(hi[j], lo[j], er + eb - epi.eshift, sl);
        slow |= sl ? (1ull << j) : 0ull;
      }
      if (__any_sync(0xffffffffu, slow != 0ull)) {
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          const int eb = __shfl_sync(0xffffffffu, j < 32 ? eb0 : eb1, j & 31);
          if ((slow >> j) & 1ull) tb[lane * TS + j] = epi.alpha * df_to_double_slow(hi[j], lo[j], er + eb - epi.eshift);
        }
      }
      __syncwarp();
      if (!*abort_flag) {
        for (int rr = 0; rr < 32; ++rr) {
          const int rw = tile.x * TM + q * 32 + rr;
          if (rw >= m) break;
          double* crow = epi.C + (long long)rw * epi.ldc + col0;
#pragma unroll
          for (int j = lane; j < CPW; j += 32)
            if (col0 + j < epi.ncols) {
              const double v = tb[rr * TS + j];
              crow[j] = epi.beta == 0.0 ? v : v + epi.beta * crow[j];
            }
        }
      }
    } else if (row < m && !*abort_flag) {
      double* orow = out + (long long)split * split_stride + (long long)row * ldo + col0;
#pragma unroll
      for (int j = 0; j < CPW; ++j)
        if (col0 + j < m) orow[j] = df_to_double_bits(hi[j], lo[j]);
    }
  }
  __syncwarp();

  if (warp == 0 && lane == 0 && *abort_flag) {
    for (int it = 0; it < issued; ++it) {
      const int st = it % OST;
      mbar_wait(smem_u32(&full_bar[st]), (uint32_t)((it / OST) & 1), status, 14);
    }
  }
  // on abort, the MMAs already issued must retire before TMEM is freed
  if (warp == 1 && lane == 0 && *abort_flag) {
    umma_commit(smem_u32(&fin_bar));
    mbar_wait(smem_u32(&fin_bar), 0u, status, 16);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OTMEM));
  }
}

// v as an unevaluated sum of two floats (48 significant bits)
__device__ __forceinline__ float2 df_split(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

__global__ void k_df_to_double(long long cnt, const float2* __restrict__ F, double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) out[i] = (double)F[i].x + (double)F[i].y;
}

// Blocks of 32 x 32 entries (bj <= bi): sum the split partials once, scale
// by 2^(E_i+E_j-eshift) (eshift = 16 + 8 (NG - 1): the slices' 2^-8(s+1)
// weights and the epilogue's 2^(8 (NG - 1 - g)) level factors), write the full
// symmetric double-float Gram F (both the block
// and its mirror, through shared memory) and the FP32 lower triangle K with
// the diagonal shift (its upper triangle zeroed) for the FP32 factorisation.
__global__ void __launch_bounds__(256) k_oz_reduce(int m, int nsplit, const double* __restrict__ P, long long ldp,
                                                   long long sstride, const int* __restrict__ rowexp, int eshift,
                                                   double shift, float* __restrict__ K, long long ldk,
                                                   float2* __restrict__ F, long long ldf, double* __restrict__ Kd) {
  __shared__ double t[32][33];
  const int b = blockIdx.x;
  int bi = (int)((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
  while ((bi + 1) * (bi + 2) / 2 <= b) ++bi;
  while (bi * (bi + 1) / 2 > b) --bi;
  const int bj = b - bi * (bi + 1) / 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  // every partial this thread needs is loaded before the first sum (up to 16
  // loads in flight); the sums keep the split order (nsplit <= 4)
  double pv[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = bi * 32 + ty + 8 * q, j = bj * 32 + tx;
    const bool in = i < m && j < m && j <= i;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
      pv[q][sp] = (in && sp < nsplit) ? P[(long long)sp * sstride + (long long)i * ldp + j] : 0.0;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = ty + 8 * q;
    const int i = bi * 32 + r, j = bj * 32 + tx;
    double v = 0.0;
    if (i < m && j < m && j <= i) {
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
        if (sp < nsplit) v += pv[q][sp];
      v = ldexp(v, rowexp[i] + rowexp[j] - eshift);
    }
    t[r][tx] = v;
    if (i < m && j < m) {
      if (j <= i) F[(long long)i * ldf + j] = df_split(v);
      K[(long long)i * ldk + j] = (j <= i) ? (float)(i == j ? v + shift : v) : 0.f;
      if (Kd && j <= i) Kd[(long long)i * ldk + j] = i == j ? v + shift : v;
    }
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = bj * 32 + r, j = bi * 32 + tx;   // mirrored block, j > i
    if (i < m && j < m && j > i) {
      F[(long long)i * ldf + j] = df_split(t[tx][r]);
      if (bi != bj) K[(long long)i * ldk + j] = 0.f;
    }
  }
}

int oz_splits(int ntiles, int num_kblk, int nsm) {
  int best = 1;
  double best_eff = 0.0;
  for (int s = 1; s <= 4; ++s) {
    if (num_kblk / s < 16) break;
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

// Output tiles (I: 128-row block, J: 96-column block) touching the lower
// triangle; partial tiles are stored [split][mp rows][lp columns].  CTAs run
// roughly in tile-list order, one per SM, so the list goes by super-blocks of
// kSB x kSB tiles: the ~one wave of CTAs working at a time reads the slice
// rows of kSB row blocks and kSB column blocks (which L2 then serves to the
// other tiles of the super-block) instead of every column block of a few
// row blocks.
constexpr int kSB = 12;
int oz_tn(int ng) { return ng == 6 ? OzCfg<4, 6>::TN : OzCfg<4, 5>::TN; }
std::vector<int2> oz_tiles(int m, int ng) {
  std::vector<int2> t;
  const int TN = oz_tn(ng);
  const int nI = (m + TM - 1) / TM, nJ = (m + TN - 1) / TN;
  for (int I0 = 0; I0 < nI; I0 += kSB)
    for (int J0 = 0; J0 < nJ && J0 * TN <= (I0 + kSB) * TM - 1; J0 += kSB)
      for (int I = I0; I < I0 + kSB && I < nI; ++I)
        for (int Jc = J0; Jc < J0 + kSB && Jc < nJ && Jc * TN <= I * TM + TM - 1; ++Jc)
          t.push_back(make_int2(I, Jc));
  return t;
}
long long oz_mp(int m) { return (long long)((m + TM - 1) / TM) * TM; }
long long oz_lp(int m, int ng) { return (long long)((m + oz_tn(ng) - 1) / oz_tn(ng)) * oz_tn(ng); }

}  // namespace

struct OzPlan {
  int m, n, ldb;
  int ng;            // levels kept (5: g <= 4, 6: g <= 5)
  bool j64;          // J is FP64 (else FP32)
  long long ldJ, ldS;
  const void* J;
  __nv_bfloat16* S;
  int* rowexp;
  unsigned* rowmax;
  CUtensorMap mapA, mapB;
  int2* d_tiles = nullptr;
  int ntiles = 0, nsplit = 1, num_kblk = 0;
  double* partials = nullptr;
  long long ldp = 0, sstride = 0;
  float* K;          // FP32 lower + shift (factorisation)
  long long ldk;
  float2* F;         // double-float full symmetric (refinement operator)
  long long ldf;
  double shift = 0.0;
  double* Kd = nullptr;   // FP64 lower + shift (the FP64 factorisation), or null
};

size_t gram_oz_partial_bytes(int m, int n, int ng) {
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int nsplit = oz_splits((int)oz_tiles(m, ng).size(), (n + KS - 1) / KS, nsm);
  return (size_t)nsplit * oz_mp(m) * oz_lp(m, ng) * sizeof(double);
}

size_t gram_oz_slice_bytes(int m, int n) {
  const long long ldb = ((n + 63) / 64) * 64;
  return (size_t)m * 4 * ldb * sizeof(__nv_bfloat16) + 2 * (size_t)m * sizeof(int) + 256;
}

dngd_status gram_oz_plan(OzPlan** out, const void* J, bool j64, int ng, long long ldJ, int m, int n, void* slices,
                         float* K, long long ldk, float2* F, long long ldf, double* partials, size_t partial_bytes,
                         cudaStream_t st) {
  if (ng != 5 && ng != 6) return DNGD_ERR_INVALID_ARG;
  EncodeTiledFn enc = (EncodeTiledFn)tensor_map_encoder();
  if (!enc) return DNGD_ERR_CUDA;
  OzPlan* p = new OzPlan();
  p->m = m;
  p->n = n;
  p->ng = ng;
  p->j64 = j64;
  p->J = J;
  p->ldJ = ldJ;
  p->ldb = ((n + 63) / 64) * 64;
  p->ldS = (long long)4 * p->ldb;
  p->S = (__nv_bfloat16*)slices;
  p->rowexp = (int*)((char*)slices + (size_t)m * p->ldS * sizeof(__nv_bfloat16));
  p->rowmax = (unsigned*)(p->rowexp + m);
  p->K = K;
  p->ldk = ldk;
  p->F = F;
  p->ldf = ldf;
  p->num_kblk = p->ldb / KS;   // K stages
  const int TN = oz_tn(ng);
  cuuint64_t gdim[2] = {(cuuint64_t)p->ldS, (cuuint64_t)m};
  cuuint64_t gstride[1] = {(cuuint64_t)(p->ldS * 2)};
  cuuint32_t estride[2] = {1, 1};
  cuuint32_t boxA[2] = {(cuuint32_t)KS, (cuuint32_t)TM};
  cuuint32_t boxB[2] = {(cuuint32_t)KS, (cuuint32_t)TN};
  if (enc(&p->mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)p->S, gdim, gstride, boxA, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      enc(&p->mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)p->S, gdim, gstride, boxB, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    delete p;
    return DNGD_ERR_CUDA;
  }
  std::vector<int2> tiles = oz_tiles(m, ng);
  p->ntiles = (int)tiles.size();
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  p->nsplit = oz_splits(p->ntiles, p->num_kblk, nsm);
  p->ldp = oz_lp(m, ng);
  p->sstride = oz_mp(m) * p->ldp;
  if ((size_t)p->nsplit * p->sstride * sizeof(double) > partial_bytes) p->nsplit = 1;
  if ((size_t)p->sstride * sizeof(double) > partial_bytes) {
    delete p;
    return DNGD_ERR_INVALID_ARG;
  }
  p->partials = partials;
  if (cudaMalloc(&p->d_tiles, sizeof(int2) * tiles.size()) != cudaSuccess) {
    delete p;
    return DNGD_ERR_OOM;
  }
  if (cudaMemcpyAsync(p->d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, st) !=
      cudaSuccess) {
    cudaFree(p->d_tiles);
    delete p;
    return DNGD_ERR_CUDA;
  }
  static bool attr5 = false, attr6 = false;
  if (ng == 5 && !attr5) {
    cudaFuncSetAttribute(k_gram_oz<4, 5, OZ_PARTIAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, osmem<4, 5>());
    attr5 = true;
  }
  if (ng == 6 && !attr6) {
    cudaFuncSetAttribute(k_gram_oz<4, 6, OZ_PARTIAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, osmem<4, 6>());
    attr6 = true;
  }
  *out = p;
  return DNGD_OK;
}

dngd_status gram_oz_set_shift(OzPlan* p, double shift) {
  p->shift = shift;
  return DNGD_OK;
}

dngd_status gram_oz_run(OzPlan* p, int* status, cudaStream_t st, cudaEvent_t ev_before_mma,
                        cudaEvent_t ev_after_mma) {
  DNGD_NOTE_LAUNCH();
  if (p->j64)
    k_oz_slice<double><<<p->m, 256, 0, st>>>(p->m, p->n, (const double*)p->J, p->ldJ, p->S, p->ldS, p->ldb,
                                              p->rowmax, p->rowexp);
  else
    k_oz_slice<float><<<p->m, 256, 0, st>>>(p->m, p->n, (const float*)p->J, p->ldJ, p->S, p->ldS, p->ldb,
                                             p->rowmax, p->rowexp);
  DNGD_LAUNCH_CHECK();
  if (ev_before_mma) cudaEventRecord(ev_before_mma, st);
  DNGD_NOTE_LAUNCH();
  const OzEpi none{nullptr, 0, nullptr, nullptr, 0, 0, 0, 0.0, 0.0};
  if (p->ng == 5)
    k_gram_oz<4, 5, OZ_PARTIAL><<<dim3(p->ntiles, p->nsplit), othreads<4, 5>(), osmem<4, 5>(), st>>>(
        p->mapA, p->mapB, p->d_tiles, p->m, 0, p->num_kblk, p->ldb, p->partials, p->ldp, p->sstride, none, status);
  else
    k_gram_oz<4, 6, OZ_PARTIAL><<<dim3(p->ntiles, p->nsplit), othreads<4, 6>(), osmem<4, 6>(), st>>>(
        p->mapA, p->mapB, p->d_tiles, p->m, 0, p->num_kblk, p->ldb, p->partials, p->ldp, p->sstride, none, status);
  DNGD_LAUNCH_CHECK();
  if (ev_after_mma) cudaEventRecord(ev_after_mma, st);
  return gram_oz_reduce(p, st);
}

// Re-run only the reduction (e.g. with a new shift): the partial tiles of
// the last run stay valid.
dngd_status gram_oz_reduce(OzPlan* p, cudaStream_t st) {
  if (p->nsplit > 4) return DNGD_ERR_INVALID_ARG;   // the reduction sums at most four partial tiles
  const int nb = (p->m + 31) / 32;
  DNGD_NOTE_LAUNCH();
  k_oz_reduce<<<nb * (nb + 1) / 2, 256, 0, st>>>(p->m, p->nsplit, p->partials, p->ldp, p->sstride, p->rowexp,
                                                 16 + 8 * (p->ng - 1), p->shift, p->K, p->ldk, p->F, p->ldf, p->Kd);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// The exact Gram (rows of ldf float2) as FP64 [m x m] row-major on the device.
dngd_status gram_oz_read(const OzPlan* p, double* out, cudaStream_t st) {
  const long long cnt = (long long)p->m * p->ldf;
  DNGD_NOTE_LAUNCH();
  k_df_to_double<<<(int)((cnt + 255) / 256), 256, 0, st>>>(cnt, p->F, out);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

void gram_oz_free(OzPlan* p) {
  if (!p) return;
  if (p->d_tiles) cudaFree(p->d_tiles);
  delete p;
}

int gram_oz_nsplit(const OzPlan* p) { return p->nsplit; }

void gram_oz_set_fp64_out(OzPlan* p, double* Kd) { p->Kd = Kd; }

// ---------------------------------------------------------------------------
// Blocked Cholesky of an FP64 matrix: double-float diagonal blocks, panel
// solves and the first 64 columns of each trailing update; the rest of each
// update from exact slice products on the tensor cores (look-ahead)
// ---------------------------------------------------------------------------

namespace {

constexpr int FNS = 6, FNG = 7;                       // six slices, levels <= 6
constexpr int FNB = 64;                               // columns per step (the K extent of an update)
constexpr int FLD = FNS * FNB;                        // slice row: 6 x 64 BF16

// The factorisation's 64-column steps compute in double-float arithmetic
// (hi + lo FP32 pairs, ~2^-47 per operation) on the FP32 pipes: GB300's FP64
// pipe retires 2 FMA per clock per SM, and these kernels are the latency
// chain of the factorisation.  The factor preconditions a refinement against
// the exact Gram and is rounded to FP32 afterwards, so the pairs keep far
// more than it needs even at cond(K + lambda I) ~ 1e10.  The matrix itself
// stays FP64: operands are read from it and results rounded once into it.

// Entry e of the column-major numbering of a 64 x 64 lower triangle
// (column c starts at c (129 - c) / 2 and holds rows c .. 63).
__device__ __forceinline__ void tri64_entry(int e, int& i, int& c) {
  int cc = (int)((129.0f - sqrtf((float)(16641 - 8 * e))) * 0.5f);
  cc = max(0, min(63, cc));
  while (cc < 63 && (cc + 1) * (129 - (cc + 1)) / 2 <= e) ++cc;
  while (cc > 0 && cc * (129 - cc) / 2 > e) --cc;
  c = cc;
  i = cc + (e - cc * (129 - cc) / 2);
}

// Diagonal block A[k0 .. k0 + kb)^2 = L L^T (kb <= 64; rows beyond kb are
// padded with the identity).  Right-looking with one barrier per column:
// thread t keeps the entries e = t + 512 q of the lower triangle in
// registers; at step j every thread updates its entries (i, c), c > j, by
// a_ic -= a_ij a_cj / d_j from the unscaled column j, which sits in a
// shared double buffer (the owners of column j + 1 publish it as soon as
// their update makes it final).  A warp skips a slot whose 32 entries are
// all finished (they run through the triangle column by column).  At the
// end L_ic = a_ic / sqrt(d_c).  Outputs: L in A (FP64), L's strictly lower
// part as pairs in Ldf[64][64], the pivots' reciprocal square roots in
// rdf[64].  A pivot that is not positive sets ST_NOT_SPD with its column
// (status[1]).
constexpr int kDiagThreads = 512;
__device__ __forceinline__ void potrf_diag_df_body(int k0, int kb, double* A, long long lda,
                                                   float2* __restrict__ Ldf, float2* __restrict__ rdf, int* status) {
  constexpr int NB = FNB, NE = NB * (NB + 1) / 2, Q = (NE + kDiagThreads - 1) / kDiagThreads;
  static_assert(NB == 64, "the triangle numbering assumes 64 columns");
  __shared__ float2 col[2][NB];
  __shared__ float2 rs[NB];
  const int tid = threadIdx.x;
  int ri[Q], ci[Q];
  double a0[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int e = tid + kDiagThreads * q;
    ri[q] = 0;    // a slot past the triangle: never updated, published or stored
    ci[q] = -1;
    if (e < NE) tri64_entry(e, ri[q], ci[q]);
    a0[q] = (ci[q] >= 0 && ri[q] < kb) ? A[(long long)(k0 + ri[q]) * lda + k0 + ci[q]] : 0.0;
  }
  dfloat v[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    v[q] = ri[q] < kb ? df_from_double(a0[q]) : dfloat{ri[q] == ci[q] ? 1.f : 0.f, 0.f};
    if (ci[q] == 0) col[0][ri[q]] = make_float2(v[q].hi, v[q].lo);
  }
  __syncthreads();
  int bad = -1;
  for (int j = 0; j < NB; ++j) {
    const float2 dj = col[j & 1][j];
    if (!(dj.x > 0.f && dj.x < 3.0e38f)) {   // the same decision in every thread
      bad = j;
      break;
    }
    const dfloat inv = df_rcp({dj.x, dj.y});
    const float2* cj = col[j & 1];
    float2* cn = col[(j + 1) & 1];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if (__any_sync(0xffffffffu, ci[q] > j)) {
        const bool act = ci[q] > j;
        const float2 aij = cj[ri[q]], acj = cj[act ? ci[q] : 0];
        const dfloat nv = df_sub_mul(v[q], df_mul({aij.x, aij.y}, inv), {acj.x, acj.y});
        if (act) v[q] = nv;
        if (ci[q] == j + 1) cn[ri[q]] = make_float2(v[q].hi, v[q].lo);
      }
    }
    __syncthreads();
  }
  if (bad >= 0) {
    if (bad < kb && tid == 0) {
      const int old = atomicOr(status, ST_NOT_SPD);
      if (!(old & ST_NOT_SPD)) status[1] = k0 + bad;
    }
    return;
  }
  // r_c = 1 / sqrt(d_c) from the final diagonal entries
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    if (ri[q] == ci[q]) {
      const dfloat r = df_rsqrt(v[q]);
      rs[ri[q]] = make_float2(r.hi, r.lo);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = ri[q], c = ci[q];
    if (c < 0 || i >= kb) continue;
    const float2 r = rs[c];
    const dfloat l = df_mul(v[q], {r.x, r.y});
    A[(long long)(k0 + i) * lda + k0 + c] = df_to_double_bits(l.hi, l.lo);
    Ldf[i * NB + c] = i > c ? make_float2(l.hi, l.lo) : make_float2(0.f, 0.f);
  }
  // entries above the diagonal of Ldf and rows beyond kb are zero
  for (int e = tid; e < NB * NB; e += kDiagThreads) {
    const int i = e >> 6, c = e & (NB - 1);
    if (c > i || i >= kb) Ldf[e] = make_float2(0.f, 0.f);
  }
  if (tid < NB) rdf[tid] = tid < kb ? rs[tid] : make_float2(0.f, 0.f);
}
__global__ void __launch_bounds__(kDiagThreads) k_potrf_diag_df(int k0, int kb, double* A, long long lda,
                                                                float2* __restrict__ Ldf, float2* __restrict__ rdf,
                                                                int* status) {
  potrf_diag_df_body(k0, kb, A, lda, Ldf, rdf, status);
}

// Panel rows g in [k0 + kb, m): X L11^T = A_panel by forward substitution,
// x_j = (a_j - sum_{i<j} x_i L_ji) r_j, then the row's exponent and six
// 8-bit slices for the sliced trailing update.  A CTA takes 16 rows with 128
// threads, eight per row: thread (row, q) keeps columns q + 8 t of its row
// as pairs in registers; once x_j is final its owner scales it and a
// width-8 shuffle hands it to the row's other threads.  Outputs: the solved
// panel in A (FP64) and as pairs in P[(g - k0 - kb) * 64 + j] (for the
// first 64 columns of the update), and slices S[g] (FLD BF16 per row, zero
// beyond kb) with exponents rowexp[g] (|x| / 2^E < 0.5, entries kept to
// 2^(E - 49)).
// (Without slices, Sl = nullptr, the rows are only solved.)
constexpr int kPanelRows = 16;
__device__ __forceinline__ void trsm_panel_df_body(int m, int k0, int kb, double* A, long long lda,
                                                   const float2* __restrict__ Ldf, const float2* __restrict__ rdf,
                                                   float2* __restrict__ P, __nv_bfloat16* __restrict__ Sl,
                                                   int* __restrict__ rowexp, int blk) {
  constexpr int NB = FNB;
  __shared__ float2 Lsh[NB][NB + 1];
  __shared__ float2 rc[NB];
  const int tid = threadIdx.x;
  {
    float2 lv[NB * NB / 128];   // every load in flight before the first store
#pragma unroll
    for (int u = 0; u < NB * NB / 128; ++u) lv[u] = Ldf[tid + 128 * u];
#pragma unroll
    for (int u = 0; u < NB * NB / 128; ++u) Lsh[(tid + 128 * u) >> 6][(tid + 128 * u) & (NB - 1)] = lv[u];
  }
  if (tid < NB) rc[tid] = rdf[tid];
  const int q = tid & 7;
  const long long row = (long long)blk * kPanelRows + (tid >> 3);
  const long long g = (long long)k0 + kb + row;
  const bool live = g < m;
  dfloat x[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int j = q + 8 * t;
    x[t] = (live && j < kb) ? df_from_double(A[g * lda + k0 + j]) : dfloat{0.f, 0.f};
  }
  __syncthreads();
  const int base = (tid & 31) & ~7;
  // column j = 8 t + o: the register slot t is unrolled, the owner o is a
  // loop (a fully unrolled solve outgrows the instruction cache)
#pragma unroll
  for (int t = 0; t < 8; ++t) {
#pragma unroll 1
    for (int o = 0; o < 8; ++o) {
      const int j = 8 * t + o;
      dfloat xj = {0.f, 0.f};
      if (q == o) {
        x[t] = df_mul(x[t], {rc[j].x, rc[j].y});
        xj = x[t];
      }
      xj.hi = __shfl_sync(0xffffffffu, xj.hi, base + o);
      xj.lo = __shfl_sync(0xffffffffu, xj.lo, base + o);
      if (q > o) x[t] = df_sub_mul(x[t], xj, {Lsh[q + 8 * t][j].x, Lsh[q + 8 * t][j].y});
#pragma unroll
      for (int u = t + 1; u < 8; ++u) x[u] = df_sub_mul(x[u], xj, {Lsh[q + 8 * u][j].x, Lsh[q + 8 * u][j].y});
    }
  }
  double xd[8];
  long long amax = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    xd[t] = (live && q + 8 * t < kb) ? df_to_double_bits(x[t].hi, x[t].lo) : 0.0;
    amax = max(amax, abs_bits(xd[t]));
  }
  for (int o = 4; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o, 8));
  if (!live) return;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int j = q + 8 * t;
    if (j < kb) A[g * lda + k0 + j] = xd[t];
    P[row * NB + j] = j < kb ? make_float2(x[t].hi, x[t].lo) : make_float2(0.f, 0.f);
  }
  if (Sl == nullptr) return;
  // a non-finite entry (a failed factorisation upstream) slices as zero
  const bool bad = amax >= 0x7FF0000000000000LL;
  const int E = bad ? 1 : exp_of_abs_bits(amax);
  if (q == 0) rowexp[g] = E;
  __nv_bfloat16* sr = Sl + g * FLD;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int j = q + 8 * t;
    float d[FNS];
    oz_digits<FNS>(bad ? 0.0 : xd[t], E, d);
#pragma unroll
    for (int s = 0; s < FNS; ++s) sr[s * FNB + j] = __float2bfloat16_rn(d[s]);
  }
}
__global__ void __launch_bounds__(128) k_trsm_panel_df(int m, int k0, int kb, double* A, long long lda,
                                                       const float2* __restrict__ Ldf,
                                                       const float2* __restrict__ rdf, float2* __restrict__ P,
                                                       __nv_bfloat16* __restrict__ Sl, int* __restrict__ rowexp,
                                                       const int* status) {
  if (status[0] & ST_NOT_SPD) return;
  trsm_panel_df_body(m, k0, kb, A, lda, Ldf, rdf, P, Sl, rowexp, blockIdx.x);
}

// The trailing update's first 64 columns (the next diagonal block and
// panel): C[r0 + i, r0 + c] -= sum_t P_i,t P_c,t for rows i < r, columns
// c < min(64, r), c <= i, r0 = k0 + kb, from the solved panel's pairs P
// (row-major, 64 per row).  A CTA takes 16 rows x 64 columns with 256
// threads, each one row x 4 columns (columns tx + 16 u), the sums in
// double-float; the result is rounded once into the FP64 entry.
// (strip_update_df_body: rows 16 blk .. 16 blk + 15 and the 64 columns from
// c0 of the trailing block, c <= i.)
constexpr int kStripRows = 16;
__device__ __forceinline__ void strip_update_df_body(int m, int r0, const float2* __restrict__ P, double* C,
                                                     long long ldc, int blk, int c0) {
  constexpr int NB = FNB;
  __shared__ float2 Pt[NB][NB + 1];            // the first 64 panel rows (the strip's columns)
  __shared__ float2 Pr[kStripRows][NB + 1];    // this CTA's rows
  const int tid = threadIdx.x, r = m - r0, nc = min(NB, r - c0);
  const int i0 = blk * kStripRows;
  {
    // every load in flight before the first store
    float2 pv[NB * NB / 256], rv[kStripRows * NB / 256];
#pragma unroll
    for (int u = 0; u < NB * NB / 256; ++u) {
      const int e = tid + 256 * u;
      pv[u] = (e >> 6) < nc ? P[(long long)c0 * NB + e] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kStripRows * NB / 256; ++u) {
      const int e = tid + 256 * u;
      rv[u] = i0 + (e >> 6) < r ? P[(long long)i0 * NB + e] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < NB * NB / 256; ++u) Pt[(tid + 256 * u) >> 6][(tid + 256 * u) & (NB - 1)] = pv[u];
#pragma unroll
    for (int u = 0; u < kStripRows * NB / 256; ++u) Pr[(tid + 256 * u) >> 6][(tid + 256 * u) & (NB - 1)] = rv[u];
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;   // row ty; columns tx + 16 u
  dfloat s[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) s[u] = {0.f, 0.f};
#pragma unroll 4
  for (int t = 0; t < NB; ++t) {
    const float2 pa = Pr[ty][t];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 pb = Pt[tx + 16 * u][t];
      // s += pa pb, the low part accumulated without renormalising
      const float p = pa.x * pb.x;
      const float e = fmaf(pa.x, pb.y, fmaf(pa.y, pb.x, fmaf(pa.x, pb.x, -p)));
      float h, gq;
      two_sum(s[u].hi, p, h, gq);
      s[u].hi = h;
      s[u].lo += gq + e;
    }
  }
  const int i = i0 + ty;
  if (i >= r) return;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int c = tx + 16 * u;
    if (c >= nc || c0 + c > i) continue;
    const float hi = s[u].hi + s[u].lo;
    const float lo = s[u].lo - (hi - s[u].hi);
    C[(long long)(r0 + i) * ldc + r0 + c0 + c] -= df_to_double_bits(hi, lo);
  }
}
__global__ void __launch_bounds__(256) k_strip_update_df(int m, int r0, const float2* __restrict__ P, double* C,
                                                         long long ldc, const int* status) {
  if (status[0] & ST_NOT_SPD) return;
  strip_update_df_body(m, r0, P, C, ldc, blockIdx.x, 0);
}

}  // namespace

struct OzFactor {
  int m;
  double* C;
  long long ldc;
  __nv_bfloat16* S[2];       // panel slices of even / odd steps
  int* rowexp[2];
  int2* d_rest;              // tiles (I, J >= 1), row blocks in order
  float2* Ldf;               // the current diagonal block's L as pairs [64 x 64]
  float2* rdf;               // its pivots' reciprocal square roots [64]
  float2* Pdf;               // the solved panel as pairs [(m - k0 - 64) x 64]
  std::vector<int> rest_prefix;   // rest tiles with row block < I, for I = 0 .. nI
  CUtensorMap mapA[2], mapB[2];
  cudaStream_t side = nullptr;    // the rest of each trailing update
  int nsm = 148;                  // persistent CTAs of the sliced update
  cudaEvent_t ev_fork = nullptr, ev_slice = nullptr, ev_rest = nullptr;
};

namespace {
size_t oz_factor_slice_bytes(int m) { return ((size_t)m * FLD * sizeof(__nv_bfloat16) + 255) & ~(size_t)255; }
size_t oz_factor_exp_bytes(int m) { return ((size_t)m * sizeof(int) + 255) & ~(size_t)255; }
}  // namespace

size_t oz_factor_bytes(int m) {
  const int nI = (m + TM - 1) / TM, nJ = (m + OzCfg<FNS, FNG>::TN - 1) / OzCfg<FNS, FNG>::TN;
  return 2 * oz_factor_slice_bytes(m) + 2 * oz_factor_exp_bytes(m) + (size_t)nI * (nJ + 1) * sizeof(int2) + 256 +
         (size_t)(FNB * FNB + FNB) * sizeof(float2) + (size_t)m * FNB * sizeof(float2) + 1024;
}

// The trailing update of a block of r rows: its first 64 columns (the
// columns the next diagonal block and panel are cut from) in double-float
// on the step's stream, the other column tiles from slices in one launch on
// a side stream, so the next step's diagonal block, panel solve and slicing
// overlap the bulk of the update; slices alternate between two buffers so
// the next step's slicing does not overwrite what the side launch reads.
dngd_status oz_factor_plan(OzFactor** out, int m, double* C, long long ldc, void* work, cudaStream_t st) {
  EncodeTiledFn enc = (EncodeTiledFn)tensor_map_encoder();
  if (!enc) return DNGD_ERR_CUDA;
  constexpr int TN = OzCfg<FNS, FNG>::TN;
  OzFactor* p = new OzFactor();
  p->m = m;
  p->C = C;
  p->ldc = ldc;
  char* w = (char*)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  for (int b = 0; b < 2; ++b) {
    p->S[b] = (__nv_bfloat16*)w;
    w += oz_factor_slice_bytes(m);
  }
  for (int b = 0; b < 2; ++b) {
    p->rowexp[b] = (int*)w;
    w += oz_factor_exp_bytes(m);
  }
  const int nI = (m + TM - 1) / TM, nJ = (m + TN - 1) / TN;
  p->d_rest = (int2*)w;
  p->Ldf = (float2*)(((uintptr_t)(p->d_rest + (size_t)nI * nJ) + 255) & ~(uintptr_t)255);
  p->rdf = p->Ldf + FNB * FNB;
  p->Pdf = p->rdf + FNB;
  std::vector<int2> tiles;
  p->rest_prefix.assign(nI + 1, 0);
  for (int I = 0; I < nI; ++I) {
    for (int Jc = 1; Jc < nJ && Jc * TN <= I * TM + TM - 1; ++Jc) tiles.push_back(make_int2(I, Jc));
    p->rest_prefix[I + 1] = (int)tiles.size();
  }
  cuuint64_t gdim[2] = {(cuuint64_t)FLD, (cuuint64_t)m};
  cuuint64_t gstride[1] = {(cuuint64_t)(FLD * 2)};
  cuuint32_t estride[2] = {1, 1};
  cuuint32_t boxA[2] = {(cuuint32_t)KS, (cuuint32_t)TM};
  cuuint32_t boxB[2] = {(cuuint32_t)KS, (cuuint32_t)TN};
  for (int b = 0; b < 2; ++b) {
    if (enc(&p->mapA[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)p->S[b], gdim, gstride, boxA, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&p->mapB[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)p->S[b], gdim, gstride, boxB, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      delete p;
      return DNGD_ERR_CUDA;
    }
  }
  if (cudaMemcpyAsync(p->d_rest, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_slice, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_rest, cudaEventDisableTiming) != cudaSuccess) {
    oz_factor_free(p);
    return DNGD_ERR_CUDA;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gram_oz<FNS, FNG, OZ_UPDATE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         osmem<FNS, FNG>());
    attr = true;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev);
  *out = p;
  return DNGD_OK;
}

dngd_status oz_factor_run(OzFactor* p, int* status, cudaStream_t st) {
  const int m = p->m;
  // the side stream joins the caller's stream here and is joined back at
  // the end (also inside a stream capture)
  DNGD_CUDA_CHECK(cudaEventRecord(p->ev_fork, st));
  DNGD_CUDA_CHECK(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
  bool rest_pending = false;
  for (int k0 = 0, step = 0; k0 < m; k0 += FNB, ++step) {
    // diagonal block, panel solve and slicing (double-float): after the
    // previous step's first 64 columns of its update, which the stream order
    // gives
    const int kb = (m - k0) < FNB ? (m - k0) : FNB;
    const int row0 = k0 + kb, r = m - row0;
    const int b = step & 1;
    DNGD_NOTE_LAUNCH();
    k_potrf_diag_df<<<1, kDiagThreads, 0, st>>>(k0, kb, p->C, p->ldc, p->Ldf, p->rdf, status);
    DNGD_LAUNCH_CHECK();
    if (r <= 0) break;
    DNGD_NOTE_LAUNCH();
    k_trsm_panel_df<<<cdiv(r, kPanelRows), 128, 0, st>>>(m, k0, kb, p->C, p->ldc, p->Ldf, p->rdf, p->Pdf, p->S[b],
                                                        p->rowexp[b], status);
    DNGD_LAUNCH_CHECK();
    DNGD_CUDA_CHECK(cudaEventRecord(p->ev_slice, st));
    OzEpi upd{p->C, p->ldc, p->rowexp[b], nullptr, 16 + 8 * (FNG - 1), 0, 0, 0.0, 0.0};
    const int nIr = (r + TM - 1) / TM;
    // the first 64 columns (double-float, from the panel's pairs) also wait
    // for the previous step's rest, which updated the same columns
    if (rest_pending) DNGD_CUDA_CHECK(cudaStreamWaitEvent(st, p->ev_rest, 0));
    DNGD_NOTE_LAUNCH();
    k_strip_update_df<<<cdiv(r, kStripRows), 256, 0, st>>>(m, row0, p->Pdf, p->C, p->ldc, status);
    DNGD_LAUNCH_CHECK();
    const int nrest = p->rest_prefix[nIr];
    DNGD_CUDA_CHECK(cudaStreamWaitEvent(p->side, p->ev_slice, 0));
    if (nrest > 0) {
      upd.ncols = nrest;   // the tile count of the persistent launch
      DNGD_NOTE_LAUNCH();
      k_gram_oz<FNS, FNG, OZ_UPDATE><<<dim3(min(nrest, p->nsm), 1), othreads<FNS, FNG>(), osmem<FNS, FNG>(),
                                       p->side>>>(
          p->mapA[b], p->mapB[b], p->d_rest, r, row0, FNB / KS, FNB, nullptr, 0, 0, upd, status);
      DNGD_LAUNCH_CHECK();
    }
    DNGD_CUDA_CHECK(cudaEventRecord(p->ev_rest, p->side));
    rest_pending = true;
  }
  // join: every update has landed before the caller's stream goes on
  DNGD_CUDA_CHECK(cudaEventRecord(p->ev_rest, p->side));
  DNGD_CUDA_CHECK(cudaStreamWaitEvent(st, p->ev_rest, 0));
  return DNGD_OK;
}

void oz_factor_free(OzFactor* p) {
  if (!p) return;
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_slice) cudaEventDestroy(p->ev_slice);
  if (p->ev_rest) cudaEventDestroy(p->ev_rest);
  if (p->side) cudaStreamDestroy(p->side);
  delete p;
}


// ---------------------------------------------------------------------------
// Batched factorisation of independent exact-Gram instances: one plan over
// all of them, and per 64-column step three launches for every instance
// together (diagonal blocks; panel solves; the whole trailing update in
// double-float arithmetic, 16-row x 64-column units).  Many instances of
// modest size then fill the device instead of each running its own chain of
// small launches.  The per-instance arithmetic does not depend on the batch:
// a plan of one instance computes the same factor bit for bit.
// ---------------------------------------------------------------------------

namespace {

struct BInst {
  double* C;
  long long ldc;
  int m;
  int* status;
  float2 *Ldf, *rdf, *P;
};

// The participant of a launch that owns CTA b: parts are (instance, first
// CTA) pairs in CTA order.
__device__ __forceinline__ int2 find_part(const int2* __restrict__ parts, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (parts[mid].y <= b) lo = mid;
    else hi = mid - 1;
  }
  return parts[lo];
}

__global__ void __launch_bounds__(kDiagThreads) k_potrf_diag_df_b(const BInst* __restrict__ inst,
                                                                  const int* __restrict__ list, int k0) {
  const BInst I = inst[list[blockIdx.x]];
  if (I.status[0] & ST_NOT_SPD) return;
  potrf_diag_df_body(k0, min(FNB, I.m - k0), I.C, I.ldc, I.Ldf, I.rdf, I.status);
}

__global__ void __launch_bounds__(128) k_trsm_panel_df_b(const BInst* __restrict__ inst,
                                                         const int2* __restrict__ parts, int n, int k0) {
  const int2 pt = find_part(parts, n, blockIdx.x);
  const BInst I = inst[pt.x];
  if (I.status[0] & ST_NOT_SPD) return;
  trsm_panel_df_body(I.m, k0, FNB, I.C, I.ldc, I.Ldf, I.rdf, I.P, nullptr, nullptr, (int)blockIdx.x - pt.y);
}

// Unit u of an instance's trailing update: row block R (16 rows) has
// floor(R / 4) + 1 units (64-column blocks J <= R / 4), so groups of four
// row blocks hold 4 (q + 1) units and group q starts at unit 2 q (q + 1).
__global__ void __launch_bounds__(256) k_trail_df_b(const BInst* __restrict__ inst, const int2* __restrict__ parts,
                                                    int n, int k0) {
  const int2 pt = find_part(parts, n, blockIdx.x);
  const BInst I = inst[pt.x];
  if (I.status[0] & ST_NOT_SPD) return;
  const int u = (int)blockIdx.x - pt.y;
  int q = (int)((sqrtf(1.0f + 2.0f * (float)u) - 1.0f) * 0.5f);
  while (q > 0 && 2 * q * (q + 1) > u) --q;
  while (2 * (q + 1) * (q + 2) <= u) ++q;
  const int v = u - 2 * q * (q + 1);
  const int R = 4 * q + v / (q + 1), J = v % (q + 1);
  strip_update_df_body(I.m, k0 + FNB, I.P, I.C, I.ldc, R, FNB * J);
}

int trail_units(int r) {
  const int nR = (r + kStripRows - 1) / kStripRows;
  int u = 0;
  for (int R = 0; R < nR; ++R) u += R / 4 + 1;
  return u;
}

}  // namespace

struct OzBatchFactor {
  int n = 0, steps = 0;
  BInst* d_inst = nullptr;
  int* d_diag = nullptr;
  int2* d_parts = nullptr;
  std::vector<int> diag_off, diag_cnt, pan_off, pan_n, pan_cta, tr_off, tr_n, tr_cta;
};

void oz_factor_batched_free(OzBatchFactor* p) {
  if (!p) return;
  if (p->d_inst) cudaFree(p->d_inst);
  if (p->d_diag) cudaFree(p->d_diag);
  if (p->d_parts) cudaFree(p->d_parts);
  delete p;
}

dngd_status oz_factor_batched_plan(OzBatchFactor** out, int n, OzFactor* const* f, int* const* status,
                                   cudaStream_t st) {
  *out = nullptr;
  if (n < 1) return DNGD_ERR_INVALID_ARG;
  OzBatchFactor* p = new OzBatchFactor();
  p->n = n;
  std::vector<BInst> hi(n);
  int maxm = 0;
  for (int b = 0; b < n; ++b) {
    hi[b] = BInst{f[b]->C, f[b]->ldc, f[b]->m, status[b], f[b]->Ldf, f[b]->rdf, f[b]->Pdf};
    maxm = std::max(maxm, f[b]->m);
  }
  p->steps = (maxm + FNB - 1) / FNB;
  std::vector<int> diag;
  std::vector<int2> parts;
  for (int s = 0; s < p->steps; ++s) {
    const int k0 = s * FNB;
    p->diag_off.push_back((int)diag.size());
    for (int b = 0; b < n; ++b)
      if (hi[b].m > k0) diag.push_back(b);
    p->diag_cnt.push_back((int)diag.size() - p->diag_off.back());
    p->pan_off.push_back((int)parts.size());
    int cta = 0;
    for (int b = 0; b < n; ++b) {
      const int r = hi[b].m - k0 - FNB;
      if (r > 0) {
        parts.push_back(make_int2(b, cta));
        cta += (r + kPanelRows - 1) / kPanelRows;
      }
    }
    p->pan_n.push_back((int)parts.size() - p->pan_off.back());
    p->pan_cta.push_back(cta);
    p->tr_off.push_back((int)parts.size());
    cta = 0;
    for (int b = 0; b < n; ++b) {
      const int r = hi[b].m - k0 - FNB;
      if (r > 0) {
        parts.push_back(make_int2(b, cta));
        cta += trail_units(r);
      }
    }
    p->tr_n.push_back((int)parts.size() - p->tr_off.back());
    p->tr_cta.push_back(cta);
  }
  if (cudaMalloc(&p->d_inst, sizeof(BInst) * n) != cudaSuccess ||
      cudaMalloc(&p->d_diag, sizeof(int) * std::max<size_t>(1, diag.size())) != cudaSuccess ||
      cudaMalloc(&p->d_parts, sizeof(int2) * std::max<size_t>(1, parts.size())) != cudaSuccess) {
    oz_factor_batched_free(p);
    return DNGD_ERR_OOM;
  }
  if (cudaMemcpyAsync(p->d_inst, hi.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (!diag.empty() &&
       cudaMemcpyAsync(p->d_diag, diag.data(), sizeof(int) * diag.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      (!parts.empty() &&
       cudaMemcpyAsync(p->d_parts, parts.data(), sizeof(int2) * parts.size(), cudaMemcpyHostToDevice, st) !=
           cudaSuccess) ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    oz_factor_batched_free(p);
    return DNGD_ERR_CUDA;
  }
  *out = p;
  return DNGD_OK;
}

dngd_status oz_factor_batched_run(OzBatchFactor* p, cudaStream_t st) {
  for (int s = 0; s < p->steps; ++s) {
    const int k0 = s * FNB;
    DNGD_NOTE_LAUNCH();
    k_potrf_diag_df_b<<<p->diag_cnt[s], kDiagThreads, 0, st>>>(p->d_inst, p->d_diag + p->diag_off[s], k0);
    DNGD_LAUNCH_CHECK();
    if (p->pan_cta[s] > 0) {
      DNGD_NOTE_LAUNCH();
      k_trsm_panel_df_b<<<p->pan_cta[s], 128, 0, st>>>(p->d_inst, p->d_parts + p->pan_off[s], p->pan_n[s], k0);
      DNGD_LAUNCH_CHECK();
    }
    if (p->tr_cta[s] > 0) {
      DNGD_NOTE_LAUNCH();
      k_trail_df_b<<<p->tr_cta[s], 256, 0, st>>>(p->d_inst, p->d_parts + p->tr_off[s], p->tr_n[s], k0);
      DNGD_LAUNCH_CHECK();
    }
  }
  return DNGD_OK;
}

// ---------------------------------------------------------------------------
// FP64 GEMM from exact slice products: C = alpha A B^T + beta C
// ---------------------------------------------------------------------------

namespace {

// Rows of A [M x K] (ld lda), or with cols the columns of a [K x M] matrix,
// as four 8-bit slices of kp columns (zero beyond K) and the row exponent.
// One warp per row; two passes over the row (its largest |A|, then slices).
__global__ void __launch_bounds__(256) k_slice_rows_f64(int M, int K, int kp, const double* __restrict__ A,
                                                        long long lda, bool cols, __nv_bfloat16* __restrict__ S,
                                                        int* __restrict__ rexp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + warp;
  if (row >= M) return;
  auto at = [&](int k) -> double { return cols ? A[(long long)k * lda + row] : A[(long long)row * lda + k]; };
  long long a = 0;
  for (int k = lane; k < K; k += 32) a = max(a, abs_bits(at(k)));
  for (int o = 16; o > 0; o >>= 1) a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
  const bool bad = a >= 0x7FF0000000000000LL;   // a non-finite row slices as zero
  const int E = bad ? 1 : exp_of_abs_bits(a);
  if (lane == 0) rexp[row] = E;
  __nv_bfloat16* sr = S + (long long)row * 4 * kp;
  for (int k = lane; k < kp; k += 32) {
    float d[4];
    oz_digits<4>(k < K && !bad ? at(k) : 0.0, E, d);
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) sr[sl * kp + k] = __float2bfloat16_rn(d[sl] * slice_weight(sl));
  }
}

}  // namespace

struct OzGemm {
  int max_m, max_n, kp;
  __nv_bfloat16 *SA, *SB;
  int *ea, *eb;
  CUtensorMap mapA, mapB;
};

size_t oz_gemm_bytes(int max_m, int max_n, int max_k) {
  const size_t kp = (size_t)((max_k + 63) / 64) * 64;
  return ((size_t)max_m + max_n) * 4 * kp * sizeof(__nv_bfloat16) + ((size_t)max_m + max_n) * sizeof(int) + 1024;
}

dngd_status oz_gemm_plan(OzGemm** out, int max_m, int max_n, int max_k, void* work) {
  EncodeTiledFn enc = (EncodeTiledFn)tensor_map_encoder();
  if (!enc) return DNGD_ERR_CUDA;
  OzGemm* p = new OzGemm();
  p->max_m = max_m;
  p->max_n = max_n;
  p->kp = ((max_k + 63) / 64) * 64;
  p->SA = (__nv_bfloat16*)work;
  p->SB = p->SA + (size_t)max_m * 4 * p->kp;
  p->ea = (int*)(p->SB + (size_t)max_n * 4 * p->kp);
  p->eb = p->ea + max_m;
  constexpr int TN = OzCfg<4, 6>::TN;
  cuuint64_t gA[2] = {(cuuint64_t)(4 * p->kp), (cuuint64_t)max_m};
  cuuint64_t gB[2] = {(cuuint64_t)(4 * p->kp), (cuuint64_t)max_n};
  cuuint64_t stride[1] = {(cuuint64_t)(4 * p->kp * 2)};
  cuuint32_t estride[2] = {1, 1};
  cuuint32_t boxA[2] = {(cuuint32_t)KS, (cuuint32_t)TM};
  cuuint32_t boxB[2] = {(cuuint32_t)KS, (cuuint32_t)TN};
  if (enc(&p->mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)p->SA, gA, stride, boxA, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      enc(&p->mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)p->SB, gB, stride, boxB, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    delete p;
    return DNGD_ERR_CUDA;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gram_oz<4, 6, OZ_GEMM>, cudaFuncAttributeMaxDynamicSharedMemorySize, osmem<4, 6>());
    attr = true;
  }
  *out = p;
  return DNGD_OK;
}

dngd_status oz_gemm(OzGemm* p, int M, int N, int K, double alpha, const double* A, long long lda, const double* B,
                    long long ldb, bool b_kn, double beta, double* C, long long ldc, int* status, cudaStream_t st) {
  if (M <= 0 || N <= 0) return DNGD_OK;
  if (M > p->max_m || N > p->max_n || K > p->kp || K <= 0) return DNGD_ERR_INVALID_ARG;
  constexpr int TN = OzCfg<4, 6>::TN;
  DNGD_NOTE_LAUNCH();
  k_slice_rows_f64<<<(M + 7) / 8, 256, 0, st>>>(M, K, p->kp, A, lda, false, p->SA, p->ea);
  DNGD_NOTE_LAUNCH();
  k_slice_rows_f64<<<(N + 7) / 8, 256, 0, st>>>(N, K, p->kp, B, ldb, b_kn, p->SB, p->eb);
  DNGD_LAUNCH_CHECK();
  const int ntn = (N + TN - 1) / TN, ntm = (M + TM - 1) / TM;
  const OzEpi epi{C, ldc, p->ea, p->eb, 16 + 8 * 5, N, ntn, alpha, beta};
  DNGD_NOTE_LAUNCH();
  k_gram_oz<4, 6, OZ_GEMM><<<dim3(ntm * ntn, 1), othreads<4, 6>(), osmem<4, 6>(), st>>>(
      p->mapA, p->mapB, nullptr, M, 0, (K + KS - 1) / KS, p->kp, nullptr, 0, 0, epi, status);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

void oz_gemm_free(OzGemm* p) { delete p; }

// ---------------------------------------------------------------------------
// Inverse of a lower-triangular FP64 factor (the exact-Gram preconditioner)
// ---------------------------------------------------------------------------
//
// The recursion (L^{-1})21 = -I22 (L21 I11) over halves rounded to 64.  Its
// small nodes (n1 + n2 <= 512: products over at most 448 terms) run as the
// batched FP32 launches of trtri_offdiag_f32; a large node's products run
// over up to m/2 terms, where FP32 accumulation ruins the preconditioner at
// cond(L) ~ 1e5 (preconditioned condition number ~1e4 instead of ~2 on the
// 5-D benchmark late in training, CPU emulation), so they are FP64 products
// from exact slices: keeping L^{-1} and L^{-T},
//   T^T = I11^T L21^T,  I21 = -I22 T  (row-major products C = A B^T)
// and I21^T by a transpose.

namespace {

// B [cols x rows] = A^T for A [rows x cols] (FP64, 32 x 32 tiles).
__global__ void k_transpose_f64(int rows, int cols, const double* __restrict__ A, long long lda,
                                double* __restrict__ B, long long ldb) {
  __shared__ double t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int i = by + r, j = bx + tx;
    if (i < rows && j < cols) t[r][tx] = A[(long long)i * lda + j];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = bx + r, j = by + tx;   // B[i][j] = A[j][i]
    if (i < cols && j < rows) B[(long long)i * ldb + j] = t[tx][r];
  }
}

// Li = double(Linv) and LiT = its transpose (both [m x ld]).
__global__ void k_widen_inv(int m, const float* __restrict__ Linv, double* __restrict__ Li,
                            double* __restrict__ LiT, long long ld) {
  __shared__ float t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int i = by + r, j = bx + tx;
    const float v = (i < m && j < ld) ? Linv[(long long)i * ld + j] : 0.f;
    t[r][tx] = v;
    if (i < m && j < ld) Li[(long long)i * ld + j] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = bx + r, j = by + tx;   // LiT[i][j] = Linv[j][i]
    if (i < m && j < ld) LiT[(long long)i * ld + j] = (j < m) ? t[tx][r] : 0.f;
  }
}

}  // namespace

dngd_status oz_trtri(OzGemm* g, int m, const double* L, long long ldl, const double* Dinv, float* L32, float* Linv,
                     float* LinvT, double* Li, double* LiT, long long ld, float* work32, double* work, int* status,
                     cudaStream_t st) {
  dngd_status s = factor_to_f32(m, L, ldl, Dinv, L32, Linv, ld, st);
  if (s) return s;
  std::vector<int3> large;
  if ((s = trtri_small_nodes_f32(m, L32, ld, Linv, ld, work32, st, &large))) return s;
  if (!large.empty()) {
    DNGD_NOTE_LAUNCH();
    k_widen_inv<<<dim3((unsigned)((ld + 31) / 32), (unsigned)((m + 31) / 32)), 256, 0, st>>>(m, Linv, Li, LiT, ld);
    DNGD_LAUNCH_CHECK();
    for (const int3& nd : large) {
      const int k0 = nd.x, n1 = nd.y, n2 = nd.z;
      const double* L21 = L + (long long)(k0 + n1) * ldl + k0;        // [n2 x n1]
      const double* I11T = LiT + (long long)k0 * ld + k0;             // [n1 x n1]
      const double* I22 = Li + (long long)(k0 + n1) * ld + k0 + n1;   // [n2 x n2]
      double* TT = work;                                              // T^T [n1 x n2]
      if ((s = oz_gemm(g, n1, n2, n1, 1.0, I11T, ld, L21, ldl, false, 0.0, TT, n2, status, st))) return s;
      if ((s = oz_gemm(g, n2, n1, n2, -1.0, I22, ld, TT, n2, false, 0.0, Li + (long long)(k0 + n1) * ld + k0, ld,
                       status, st)))
        return s;
      // I21^T: the transpose of the block just formed
      DNGD_NOTE_LAUNCH();
      k_transpose_f64<<<dim3((unsigned)((n1 + 31) / 32), (unsigned)((n2 + 31) / 32)), 256, 0, st>>>(
          n2, n1, Li + (long long)(k0 + n1) * ld + k0, ld, LiT + (long long)k0 * ld + k0 + n1, ld);
      DNGD_LAUNCH_CHECK();
    }
    if ((s = to_float((long long)m * ld, Li, Linv, st))) return s;
    if ((s = to_float((long long)m * ld, LiT, LinvT, st))) return s;
    return DNGD_OK;
  }
  return transpose_f32(m, Linv, ld, LinvT, ld, st);
}

unsigned* gram_oz_rowmax(OzPlan* p) { return p->rowmax; }

}  // namespace dngd
