// Shared definitions of the D-NGD CUDA library (internal, not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/dngd.h"

namespace dngd {

constexpr int kMaxLayers = DNGD_MAX_LAYERS;
constexpr int kMaxDim = DNGD_MAX_DIM;
constexpr int kMaxClasses = DNGD_MAX_CLASSES;

// Device status word bits (ctx->d_status[0]); d_status[1] holds the first
// failing Cholesky column, d_status[2] a code for the wait that timed out.
enum : int {
  ST_NOT_SPD = 1,
  ST_NONFINITE = 2,
  ST_TIMEOUT = 4,
  ST_NO_CONVERGE = 8,
};

// One residual class laid out for the kernels.  Points of the class are
// [p0, p0 + count); each point owns S consecutive rows of every stream
// matrix starting at row0 + (i - p0) * S.  Stream order inside a point:
// 0 = value, 1..nD = first derivatives along coords D[0..nD-1], nD+1 =
// masked Laplacian (present when has_lap).
struct ClassInfo {
  int p0, count, S, row0, nD, has_lap;
  int D[kMaxDim];
  double c_val, c_lap, scale;      // scale = 1/sqrt(count)
  double c_gradD[kMaxDim];         // c_grad of coord D[j]
  int lapD[kMaxDim];               // 1 if D[j] is in the Laplacian mask
};

struct NetInfo {
  int n_layers;                    // affine layers; hidden = n_layers - 1
  int widths[kMaxLayers + 1];
  long long w_off[kMaxLayers], b_off[kMaxLayers];
  long long n;                     // parameters
  int d_in, m, R;                  // input dim, residuals, stream rows
  int n_classes;
  int max_w;                       // widest hidden layer
  ClassInfo cls[kMaxClasses];
};

__host__ __device__ inline const ClassInfo& class_of(const NetInfo& net, int p) {
  int c = 0;
  while (c + 1 < net.n_classes && p >= net.cls[c + 1].p0) ++c;
  return net.cls[c];
}

#define DNGD_CUDA_CHECK(expr)                                                     \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      fprintf(stderr, "dngd: CUDA error %s at %s:%d: %s\n", cudaGetErrorName(_e), \
              __FILE__, __LINE__, cudaGetErrorString(_e));                        \
      return DNGD_ERR_CUDA;                                                       \
    }                                                                             \
  } while (0)

#define DNGD_LAUNCH_CHECK() DNGD_CUDA_CHECK(cudaGetLastError())

// Host-side count of kernel launches issued by the library (all contexts).
void note_launch();
#define DNGD_NOTE_LAUNCH() ::dngd::note_launch()

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Lets func take up to the device's opt-in maximum of dynamic shared memory
// (less its static shared memory).  Called once per kernel whose dynamic
// size depends on the problem: the limit belongs to the function, shared by
// every context and stream of the process, so it is raised once to the
// maximum and never set per problem (which would lower it under launches of
// a larger problem still queued on another stream).
inline cudaError_t allow_max_dynamic_smem(const void* func) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  return e;
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// tanh in the working precision (library call; derivatives use t' = 1 - t^2).
__device__ __forceinline__ double tanh_t(double x) { return tanh(x); }
__device__ __forceinline__ float tanh_t(float x) { return tanhf(x); }

// (hi + lo) 2^e2 as an FP64 value, for a normalised double-float pair
// (|lo| <= ulp(hi) / 2), assembled with 32-bit integer operations: hi's
// sign, exponent (+ e2) and significand placed in the two words of the
// double, and lo's significand, shifted to hi's FP64 units (rounded), added
// to or subtracted from that bit pattern (one unit finer when it subtracts
// from the bottom of hi's binade, where the pattern steps into the binade
// below).  A zero pair gives a signed zero.  A subnormal or non-finite part,
// a pair that is not normalised or a result outside the normal range takes
// the FP64 path, which is a call: inlined, the compiler may predicate it
// into every use, and conversions and adds on GB300's slow FP64 pipe then
// cost every value.  (A first version with 64-bit variable shifts and
// lane-divergent branches took ~1,000 cycles a value in the sliced update's
// epilogue.)
static __device__ __noinline__ double df_to_double_slow(float hi, float lo, int e2) {
  return ldexp((double)hi + (double)lo, e2);
}

// The branch-free part: the value for the common case and, in slow, whether
// the FP64 path must replace it.  Loops over many values keep a mask of the
// slow ones and fix them up after the loop (checks with early returns in the
// loop body cost ~3x the conversion itself: measured).
__device__ __forceinline__ double df_to_double_try(float hi, float lo, int e2, bool& slow) {
  const unsigned hb = __float_as_uint(hi), lb = __float_as_uint(lo);
  const int eh = (int)((hb >> 23) & 0xFFu), el = (int)((lb >> 23) & 0xFFu);
  const unsigned lmag = lb & 0x7FFFFFFFu;
  const bool zero = ((hb & 0x7FFFFFFFu) | lmag) == 0u;
  const int k = el - eh + 29;       // lo's significand in units of hi's FP64 ulp: Ml 2^k
  const int eo = eh + 896 + e2;     // the result's biased exponent (1023 - 127 = 896)
  slow = !zero && (eh == 0 || eh == 0xFF || eo < 2 || eo > 2046 || (lmag != 0u && (el == 0 || el == 0xFF || k > 5)));
  const unsigned whi = (hb & 0x80000000u) | (((unsigned)eo & 0x7FFu) << 20) | ((hb & 0x7FFFFFu) >> 3);
  const unsigned wlo = (hb & 7u) << 29;
  unsigned long long d = ((unsigned long long)whi << 32) | wlo;
  const unsigned ml = (lb & 0x7FFFFFu) | 0x800000u;
  const bool opp = ((hb ^ lb) >> 31) != 0u;
  const int kk = k + ((opp && (hb & 0x7FFFFFu) == 0u) ? 1 : 0);
  const int r = -kk;
  unsigned c = kk >= 0 ? (ml << (kk < 6 ? kk : 6)) : (r < 25 ? (ml + (1u << (r - 1))) >> r : 0u);
  c = lmag != 0u ? c : 0u;
  d = opp ? d - c : d + c;
  d = zero ? (unsigned long long)(hb >> 31) << 63 : d;
  return __longlong_as_double((long long)d);
}

__device__ __forceinline__ double df_to_double_scaled(float hi, float lo, int e2) {
  bool slow;
  double v = df_to_double_try(hi, lo, e2, slow);
  if (slow) v = df_to_double_slow(hi, lo, e2);
  return v;
}

__device__ __forceinline__ double df_to_double_bits(float hi, float lo) { return df_to_double_scaled(hi, lo, 0); }

// Double-float ("float2 as hi+lo") accumulation for FP32 data that needs an
// accumulator with ~48 significant bits.  two_sum / two_prod are the
// error-free transformations of Knuth and Dekker (the latter with fma).
struct dfloat {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  float hi = s + e;
  float lo = e - (hi - s);
  return {hi, lo};
}

// a + x*y with x*y formed exactly (hi by rounding, lo by fma residual).
__device__ __forceinline__ dfloat df_fma(dfloat a, float x, float y) {
  float p = x * y;
  float pe = fmaf(x, y, -p);
  float s, e;
  two_sum(a.hi, p, s, e);
  e += pe + a.lo;
  float hi = s + e;
  float lo = e - (hi - s);
  return {hi, lo};
}

// Nearest double-float pair of an FP64 value (hi = RN(x), lo = RN(x - hi);
// |x| within the float range).
__device__ __forceinline__ dfloat df_from_double(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}

// a * b, ~2^-47 relative (the lo x lo term is dropped).
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float hi = p + e;
  return {hi, e - (hi - p)};
}

// acc - a * b.
__device__ __forceinline__ dfloat df_sub_mul(dfloat acc, dfloat a, dfloat b) {
  const float p = a.hi * b.hi;
  float pe = fmaf(a.hi, b.hi, -p);
  pe = fmaf(a.hi, b.lo, pe);
  pe = fmaf(a.lo, b.hi, pe);
  float s, e;
  two_sum(acc.hi, -p, s, e);
  e += acc.lo - pe;
  const float hi = s + e;
  return {hi, e - (hi - s)};
}

// 1 / d for d > 0 (float range): one Newton-Raphson step y + y (1 - d y)
// from the single-precision reciprocal, the residual 1 - d y formed in
// double-float.
__device__ __forceinline__ dfloat df_rcp(dfloat d) {
  const float y = __frcp_rn(d.hi);   // the correctly rounded reciprocal, as 1.0f / d.hi
  const float r = fmaf(-d.hi, y, 1.0f) - d.lo * y;   // 1 - d y (the first term exact)
  const float c = y * r;
  const float hi = y + c;
  return {hi, c - (hi - y)};
}

// 1 / sqrt(d) for d > 0 (float range): a single-precision Newton step on
// the rsqrt estimate, then one in double-float, y + y (1 - d y^2) / 2.
__device__ __forceinline__ dfloat df_rsqrt(dfloat d) {
  float y = rsqrtf(d.hi);
  y = y * fmaf(-0.5f * d.hi, y * y, 1.5f);
  const float p = y * y;
  const float pe = fmaf(y, y, -p);             // y^2 = p + pe exactly
  const float h = d.hi * p;
  const float he = fmaf(d.hi, p, -h) + fmaf(d.hi, pe, d.lo * p);   // d y^2 = h + he
  const float r = (1.0f - h) - he;             // 1 - h exact for h near 1
  const float c = 0.5f * y * r;
  const float hi = y + c;
  return {hi, c - (hi - y)};
}

__device__ __forceinline__ dfloat df_shfl_xor(dfloat v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

__device__ __forceinline__ dfloat df_warp_sum(dfloat v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  return v;
}

}  // namespace dngd
