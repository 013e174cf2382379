// Taylor-mode jets of the tanh MLP, residuals, Jacobian rows and f_vv.
//
// Every collocation point carries S "streams" through the network (Taylor-mode
// AD of Sec. 5 of the paper): the value, the first derivatives along the
// coordinates its operator needs, and one collapsed second-order stream for
// the masked Laplacian, using (t = tanh z, s = 1 - t^2)
//     h = t,   d_k h = s d_k z,   Lap h = s Lap z - 2 t s sum_{k in mask} (d_k z)^2.
// The residual of a class is linear in the output streams (Sec. 2.2), so the
// Jacobian row of point i w.r.t. layer l is the rank-S sum
//     dr_i/dW_l = sum_s delta_{l,i,s} h_{l-1,i,s}^T,   dr_i/db_l = delta_{l,i,value}
// where delta are the stream adjoints from one reverse sweep.  The dense
// matrix products of each layer run as GEMMs over all point-streams
// (linalg.cu); the kernels here are the per-point elementwise parts.
//
// f_vv (Sec. 3.2) propagates, for every stream, the Taylor coefficients in the
// parameter direction t of theta + t v: (q, q', q'') with
//     z' = W h' + V h + b_v,   z'' = W h'' + 2 V h'
// and the chain rules of tanh, s and t*s up to second order.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace dngd {

// ---------------------------------------------------------------------------
// Forward sweep
// ---------------------------------------------------------------------------

// Where a forward-only sweep feeds the next layer's 3xTF32 GEMM, the
// activations go out directly as that GEMM's A operand split (row r:
// tf32 hi of h[r][0..kp) then lo, zero beyond w) instead of as H, and the
// pre-activations (needed only by the reverse sweep) are not stored.
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u = (u + 0x1000u) & 0xFFFFE000u;
  return __uint_as_float(u);
}

// Per-trial strides of the line search's batched forward sweep (grid.z =
// trial): every pointer of trial z is offset by z times its stride.
struct TrialStride {
  long long theta = 0, z = 0, h = 0, hs = 0, r = 0;
};

template <typename T>
__device__ __forceinline__ void put_h(T* __restrict__ H, float* __restrict__ hs, int kp, long long row, int w, int a,
                                      T v) {
  if (hs) {
    const float x = (float)v, hi = tf32_hi(x);
    hs[row * 2 * kp + a] = hi;
    hs[row * 2 * kp + kp + a] = tf32_hi(x - hi);
  } else {
    H[row * w + a] = v;
  }
}

template <typename T>
__global__ void k_first_layer(NetInfo net, const T* __restrict__ theta, const double* __restrict__ X,
                              T* __restrict__ Z, T* __restrict__ H, float* __restrict__ hs, int kp,
                              TrialStride zs = TrialStride()) {
  theta += blockIdx.z * zs.theta;
  Z += blockIdx.z * zs.z;
  H += blockIdx.z * zs.h;
  if (hs) hs += blockIdx.z * zs.hs;
  const int p = blockIdx.x;
  const int a = blockIdx.y * blockDim.x + threadIdx.x;
  const int w = net.widths[1], din = net.d_in;
  const ClassInfo& c = class_of(net, p);
  const long long row = c.row0 + (long long)(p - c.p0) * c.S;
  if (a >= w) {
    if (hs && a < kp)
      for (int j = 0; j < c.S; ++j) put_h<T>(H, hs, kp, row + j, w, a, T(0));
    return;
  }
  const T* W = theta + net.w_off[0];
  T z = theta[net.b_off[0] + a];
  for (int k = 0; k < din; ++k) z += W[(long long)a * din + k] * (T)X[(long long)p * din + k];
  const T t = tanh_t(z), s = T(1) - t * t;
  if (!hs) Z[row * w + a] = z;
  put_h<T>(H, hs, kp, row, w, a, t);
  T Q = 0;
  for (int j = 0; j < c.nD; ++j) {
    const T zk = W[(long long)a * din + c.D[j]];
    if (!hs) Z[(row + 1 + j) * w + a] = zk;
    put_h<T>(H, hs, kp, row + 1 + j, w, a, s * zk);
    if (c.lapD[j]) Q += zk * zk;
  }
  if (c.has_lap) {
    if (!hs) Z[(row + 1 + c.nD) * w + a] = T(0);
    put_h<T>(H, hs, kp, row + 1 + c.nD, w, a, T(-2) * t * s * Q);
  }
}

// Hidden layer l >= 1: Z already holds W_l h_{l-1} for every stream row.
template <typename T>
__global__ void k_act_fwd(NetInfo net, int l, const T* __restrict__ theta, T* __restrict__ Z,
                          T* __restrict__ H, float* __restrict__ hs, int kp, TrialStride zs = TrialStride()) {
  theta += blockIdx.z * zs.theta;
  Z += blockIdx.z * zs.z;
  H += blockIdx.z * zs.h;
  if (hs) hs += blockIdx.z * zs.hs;
  const int p = blockIdx.x;
  const int a = blockIdx.y * blockDim.x + threadIdx.x;
  const int w = net.widths[l + 1];
  const ClassInfo& c = class_of(net, p);
  const long long row = c.row0 + (long long)(p - c.p0) * c.S;
  if (a >= w) {
    if (hs && a < kp)
      for (int j = 0; j < c.S; ++j) put_h<T>(H, hs, kp, row + j, w, a, T(0));
    return;
  }
  const T z = Z[row * w + a] + theta[net.b_off[l] + a];
  const T t = tanh_t(z), s = T(1) - t * t;
  if (!hs) Z[row * w + a] = z;
  put_h<T>(H, hs, kp, row, w, a, t);
  T Q = 0;
  for (int j = 0; j < c.nD; ++j) {
    const T zk = Z[(row + 1 + j) * w + a];
    put_h<T>(H, hs, kp, row + 1 + j, w, a, s * zk);
    if (c.lapD[j]) Q += zk * zk;
  }
  if (c.has_lap) {
    const T L = Z[(row + 1 + c.nD) * w + a];
    put_h<T>(H, hs, kp, row + 1 + c.nD, w, a, s * L - T(2) * t * s * Q);
  }
}

// Output layer and residual: one warp per point.
template <typename T>
__global__ void k_output(NetInfo net, const T* __restrict__ theta, const double* __restrict__ X,
                         const T* __restrict__ Hlast, const double* __restrict__ target,
                         double* __restrict__ r, int* __restrict__ status, TrialStride zs = TrialStride()) {
  theta += blockIdx.z * zs.theta;
  if (Hlast) Hlast += blockIdx.z * zs.h;
  r += blockIdx.z * zs.r;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= net.m) return;
  const int p = warp;
  const ClassInfo& c = class_of(net, p);
  const int L = net.n_layers - 1;
  const int w = net.widths[L];
  const T* wo = theta + net.w_off[L];
  T acc = 0;
  if (L == 0) {
    // no hidden layer: u = w.x + b, d_k u = w_k, Lap u = 0
    if (lane == 0) {
      T u = theta[net.b_off[0]];
      for (int k = 0; k < net.d_in; ++k) u += wo[k] * (T)X[(long long)p * net.d_in + k];
      acc = T(c.c_val) * u;
      for (int j = 0; j < c.nD; ++j) acc += T(c.c_gradD[j]) * wo[c.D[j]];
    }
  } else {
    const long long row = c.row0 + (long long)(p - c.p0) * c.S;
    for (int s = 0; s < c.S; ++s) {
      T coef;
      if (s == 0) coef = T(c.c_val);
      else if (s <= c.nD) coef = T(c.c_gradD[s - 1]);
      else coef = T(c.c_lap);
      if (coef == T(0)) continue;
      T u = 0;
      for (int a = lane; a < w; a += 32) u += wo[a] * Hlast[(row + s) * w + a];
      acc += coef * u;
    }
    if (lane == 0) acc += T(c.c_val) * theta[net.b_off[L]];
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    const double ri = (double)acc * c.scale - target[p] * c.scale;
    r[p] = ri;
    if (!isfinite(ri)) atomicOr(status, ST_NONFINITE);
  }
}

// ---------------------------------------------------------------------------
// Reverse sweep
// ---------------------------------------------------------------------------

// Stream adjoints through tanh for hidden layer l.  Hbar holds the adjoints of
// the layer's outputs (rows x w), or is null for the last hidden layer, whose
// output adjoints are ubar_s * w_out with ubar the class coefficients.
template <typename T>
__global__ void k_act_bwd(NetInfo net, int l, const T* __restrict__ theta, const T* __restrict__ Z,
                          const T* __restrict__ Hbar, T* __restrict__ Dl) {
  const int p = blockIdx.x;
  const int a = blockIdx.y * blockDim.x + threadIdx.x;
  const int w = net.widths[l + 1];
  if (a >= w) return;
  const ClassInfo& c = class_of(net, p);
  const long long row = c.row0 + (long long)(p - c.p0) * c.S;
  T hv, hk[kMaxDim], hL = 0;
  if (Hbar == nullptr) {
    const T wo = theta[net.w_off[net.n_layers - 1] + a];
    const T sc = T(c.scale);
    hv = sc * T(c.c_val) * wo;
    for (int j = 0; j < c.nD; ++j) hk[j] = sc * T(c.c_gradD[j]) * wo;
    if (c.has_lap) hL = sc * T(c.c_lap) * wo;
  } else {
    hv = Hbar[row * w + a];
    for (int j = 0; j < c.nD; ++j) hk[j] = Hbar[(row + 1 + j) * w + a];
    if (c.has_lap) hL = Hbar[(row + 1 + c.nD) * w + a];
  }
  const T z = Z[row * w + a];
  const T t = tanh_t(z), s = T(1) - t * t;
  const T ts = t * s, dts = s * (s - T(2) * t * t);
  T Q = 0, gsum = 0;
  T zk[kMaxDim];
  for (int j = 0; j < c.nD; ++j) {
    zk[j] = Z[(row + 1 + j) * w + a];
    if (c.lapD[j]) Q += zk[j] * zk[j];
    gsum += zk[j] * hk[j];
  }
  T Lz = c.has_lap ? Z[(row + 1 + c.nD) * w + a] : T(0);
  const T zbar = s * hv - T(2) * ts * gsum - (T(2) * ts * Lz + T(2) * dts * Q) * hL;
  Dl[row * w + a] = zbar;
  for (int j = 0; j < c.nD; ++j) {
    T zb = s * hk[j];
    if (c.lapD[j]) zb -= T(4) * ts * zk[j] * hL;
    Dl[(row + 1 + j) * w + a] = zb;
  }
  if (c.has_lap) Dl[(row + 1 + c.nD) * w + a] = s * hL;
}

// Jacobian rows: block (point p, layer l) writes dr_p/dW_l and dr_p/db_l.
// DF (FP64 data only): each entry sum_s d_s h_s is formed in double-float
// arithmetic on the FP32 pipes (both factors split into FP32 hi + lo, the
// hi products exact by fma, the cross terms added, the sum carried as an
// unevaluated hi + lo pair) and rounded to FP64 once: ~2^-46 of the sum of
// the terms' magnitudes, at FP32 instead of FP64 throughput.
template <typename T, typename TJ, bool DF = false>
__global__ void k_jac_write(NetInfo net, const T* __restrict__ theta, const double* __restrict__ X,
                            LayerPtrs<T> Hs, LayerPtrs<T> Ds, TJ* __restrict__ J, long long ldJ,
                            __nv_bfloat16* __restrict__ Jb, long long ldb, unsigned* __restrict__ rowmax) {
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int p = blockIdx.x;
  const int l = blockIdx.y;
  const ClassInfo& c = class_of(net, p);
  const int S = c.S;
  const int L = net.n_layers - 1;
  const int wout = net.widths[l + 1], win = net.widths[l];
  T* dsh = sm;                   // [S][wout]
  T* hsh = sm + S * wout;        // [S][win]
  const long long row = c.row0 + (long long)(p - c.p0) * S;
  // stream adjoints of this layer's pre-activations
  for (int e = threadIdx.x; e < S * wout; e += blockDim.x) {
    const int s = e / wout, a = e % wout;
    T v;
    if (l == L) {
      const T sc = T(c.scale);
      v = (s == 0) ? sc * T(c.c_val) : (s <= c.nD ? sc * T(c.c_gradD[s - 1]) : sc * T(c.c_lap));
    } else {
      v = Ds.p[l][(row + s) * wout + a];
    }
    dsh[e] = v;
  }
  // stream inputs of this layer
  for (int e = threadIdx.x; e < S * win; e += blockDim.x) {
    const int s = e / win, b = e % win;
    T v;
    if (l == 0) {
      if (s == 0) v = (T)X[(long long)p * net.d_in + b];
      else if (s <= c.nD) v = (b == c.D[s - 1]) ? T(1) : T(0);
      else v = T(0);
    } else {
      v = Hs.p[l - 1][(row + s) * win + b];
    }
    hsh[e] = v;
  }
  __syncthreads();
  TJ* Jrow = J + (long long)p * ldJ;
  __nv_bfloat16* Jbrow = Jb ? Jb + (long long)p * ldb : nullptr;
  const long long wo = net.w_off[l], bo = net.b_off[l];
  float amax = 0.f;   // largest |J| this block writes (as stored)
  if constexpr (DF && std::is_same<T, double>::value) {
    // adjoints as FP32 pairs after the two FP64 tiles
    float2* d2 = reinterpret_cast<float2*>(sm + S * wout + S * win);
    for (int e = threadIdx.x; e < S * wout; e += blockDim.x) {
      const double v = dsh[e];
      const float h = (float)v;
      d2[e] = make_float2(h, (float)(v - (double)h));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < win; b += blockDim.x) {
      float hh[2 + kMaxDim], hl[2 + kMaxDim];
#pragma unroll
      for (int s = 0; s < 2 + kMaxDim; ++s) {
        const double v = s < S ? hsh[s * win + b] : 0.0;
        hh[s] = (float)v;
        hl[s] = (float)(v - (double)hh[s]);
      }
      for (int a = 0; a < wout; ++a) {
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int s = 0; s < 2 + kMaxDim; ++s) {
          if (s >= S) break;
          const float2 d = d2[s * wout + a];
          const float pr = d.x * hh[s];
          float e = fmaf(d.x, hh[s], -pr);   // exact residual of the hi product
          e = fmaf(d.x, hl[s], e);
          e = fmaf(d.y, hh[s], e);
          float t, te;
          two_sum(hi, pr, t, te);
          hi = t;
          lo += te + e;
        }
        // renormalise (hi = fl32(hi + lo)), then assemble the FP64 value
        // with integer operations
        const float sh = hi + lo;
        lo = lo - (sh - hi);
        hi = sh;
        const double v = df_to_double_bits(hi, lo);
        Jrow[wo + (long long)a * win + b] = (TJ)v;
        amax = fmaxf(amax, fabsf(hi));
      }
    }
  } else
  for (int b = threadIdx.x; b < win; b += blockDim.x) {
    // the stream loops are unrolled to the largest S so hreg stays in registers
    T hreg[2 + kMaxDim];
#pragma unroll
    for (int s = 0; s < 2 + kMaxDim; ++s) hreg[s] = s < S ? hsh[s * win + b] : T(0);
    int a = 0;
    if constexpr (std::is_same<T, float>::value) {
      // four outputs per pass: one 16-byte broadcast load of the adjoints per
      // stream instead of four (the loop is bound by shared-memory loads)
      if ((wout & 3) == 0) {
        for (; a < wout; a += 4) {
          float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int s = 0; s < 2 + kMaxDim; ++s) {
            if (s >= S) break;
            const float4 d = *reinterpret_cast<const float4*>(dsh + s * wout + a);
            acc.x += d.x * hreg[s];
            acc.y += d.y * hreg[s];
            acc.z += d.z * hreg[s];
            acc.w += d.w * hreg[s];
          }
          const float o[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            Jrow[wo + (long long)(a + q) * win + b] = (TJ)o[q];
            if (Jbrow) Jbrow[wo + (long long)(a + q) * win + b] = __float2bfloat16_rn(o[q]);
            amax = fmaxf(amax, fabsf(o[q]));
          }
        }
      }
    }
    for (; a < wout; ++a) {
      T acc = 0;
#pragma unroll
      for (int s = 0; s < 2 + kMaxDim; ++s) {
        if (s >= S) break;
        acc += dsh[s * wout + a] * hreg[s];
      }
      Jrow[wo + (long long)a * win + b] = (TJ)acc;
      if (Jbrow) Jbrow[wo + (long long)a * win + b] = __float2bfloat16_rn((float)acc);
      amax = fmaxf(amax, fabsf((float)(TJ)acc));
    }
  }
  for (int a = threadIdx.x; a < wout; a += blockDim.x) {
    Jrow[bo + a] = (TJ)dsh[a];
    if (Jbrow) Jbrow[bo + a] = __float2bfloat16_rn((float)dsh[a]);
    amax = fmaxf(amax, fabsf((float)(TJ)dsh[a]));
  }
  if (rowmax) {
    // the row's largest magnitude over all layer blocks (non-negative floats
    // order like their bit patterns)
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float a = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = fmaxf(a, red[w]);
      atomicMax(rowmax + p, __float_as_uint(a));
    }
  }
}

// ---------------------------------------------------------------------------
// f_vv: second-order Taylor coefficients along the parameter direction v
// ---------------------------------------------------------------------------

// 2-jet (in t) of one unit's streams through tanh.
template <typename T>
__device__ __forceinline__ void act2_unit(const ClassInfo& c, T z0, T z1, T z2, const T* g0, const T* g1,
                                          const T* g2, T L0, T L1, T L2, T* h0, T* h1, T* h2,
                                          T* hk0, T* hk1, T* hk2, T* hL) {
  const T t = tanh_t(z0), s = T(1) - t * t;
  const T s_z = T(-2) * t * s;
  const T s_zz = T(-2) * s * s + T(4) * t * t * s;
  const T p = t * s;
  const T p_z = s * (s - T(2) * t * t);
  const T p_zz = T(-8) * t * s * s + T(4) * t * t * t * s;
  *h0 = t;
  *h1 = s * z1;
  *h2 = s * z2 + s_z * z1 * z1;
  const T S1 = s_z * z1, S2 = s_zz * z1 * z1 + s_z * z2;
  const T P1 = p_z * z1, P2 = p_zz * z1 * z1 + p_z * z2;
  T Q0 = 0, Q1 = 0, Q2 = 0;
  for (int j = 0; j < c.nD; ++j) {
    hk0[j] = s * g0[j];
    hk1[j] = S1 * g0[j] + s * g1[j];
    hk2[j] = S2 * g0[j] + T(2) * S1 * g1[j] + s * g2[j];
    if (c.lapD[j]) {
      Q0 += g0[j] * g0[j];
      Q1 += T(2) * g0[j] * g1[j];
      Q2 += T(2) * (g1[j] * g1[j] + g0[j] * g2[j]);
    }
  }
  hL[0] = s * L0 - T(2) * p * Q0;
  hL[1] = S1 * L0 + s * L1 - T(2) * (P1 * Q0 + p * Q1);
  hL[2] = S2 * L0 + T(2) * S1 * L1 + s * L2 - T(2) * (P2 * Q0 + T(2) * P1 * Q1 + p * Q2);
}

// Z3/H3 hold three blocks of R rows: coefficient 0, 1 (d/dt), 2 (d^2/dt^2).
template <typename T>
__global__ void k_first_layer_fvv(NetInfo net, const T* __restrict__ theta, const T* __restrict__ v,
                                  const double* __restrict__ X, T* __restrict__ H3) {
  const int p = blockIdx.x;
  const int a = blockIdx.y * blockDim.x + threadIdx.x;
  const int w = net.widths[1], din = net.d_in;
  if (a >= w) return;
  const ClassInfo& c = class_of(net, p);
  const T* W = theta + net.w_off[0];
  const T* V = v + net.w_off[0];
  T z0 = theta[net.b_off[0] + a], z1 = v[net.b_off[0] + a];
  for (int k = 0; k < din; ++k) {
    const T x = (T)X[(long long)p * din + k];
    z0 += W[(long long)a * din + k] * x;
    z1 += V[(long long)a * din + k] * x;
  }
  T g0[kMaxDim], g1[kMaxDim], g2[kMaxDim];
  for (int j = 0; j < c.nD; ++j) {
    g0[j] = W[(long long)a * din + c.D[j]];
    g1[j] = V[(long long)a * din + c.D[j]];
    g2[j] = 0;
  }
  T h0, h1, h2, hk0[kMaxDim], hk1[kMaxDim], hk2[kMaxDim], hL[3];
  act2_unit(c, z0, z1, T(0), g0, g1, g2, T(0), T(0), T(0), &h0, &h1, &h2, hk0, hk1, hk2, hL);
  const long long R = net.R;
  const long long row = c.row0 + (long long)(p - c.p0) * c.S;
  T* B0 = H3;
  T* B1 = H3 + R * w;
  T* B2 = H3 + 2 * R * w;
  B0[row * w + a] = h0; B1[row * w + a] = h1; B2[row * w + a] = h2;
  for (int j = 0; j < c.nD; ++j) {
    B0[(row + 1 + j) * w + a] = hk0[j];
    B1[(row + 1 + j) * w + a] = hk1[j];
    B2[(row + 1 + j) * w + a] = hk2[j];
  }
  if (c.has_lap) {
    B0[(row + 1 + c.nD) * w + a] = hL[0];
    B1[(row + 1 + c.nD) * w + a] = hL[1];
    B2[(row + 1 + c.nD) * w + a] = hL[2];
  }
}

// Hidden layer l >= 1: Z3 holds W h (block 0), W h' + V h (block 1) and
// W h'' + 2 V h' (block 2); add biases and apply the tanh 2-jet.
template <typename T>
__global__ void k_act_fvv(NetInfo net, int l, const T* __restrict__ theta, const T* __restrict__ v,
                          const T* __restrict__ Z3, T* __restrict__ H3) {
  const int p = blockIdx.x;
  const int a = blockIdx.y * blockDim.x + threadIdx.x;
  const int w = net.widths[l + 1];
  if (a >= w) return;
  const ClassInfo& c = class_of(net, p);
  const long long R = net.R;
  const long long row = c.row0 + (long long)(p - c.p0) * c.S;
  const T* Z0 = Z3;
  const T* Z1 = Z3 + R * w;
  const T* Z2 = Z3 + 2 * R * w;
  const T z0 = Z0[row * w + a] + theta[net.b_off[l] + a];
  const T z1 = Z1[row * w + a] + v[net.b_off[l] + a];
  const T z2 = Z2[row * w + a];
  T g0[kMaxDim], g1[kMaxDim], g2[kMaxDim];
  for (int j = 0; j < c.nD; ++j) {
    g0[j] = Z0[(row + 1 + j) * w + a];
    g1[j] = Z1[(row + 1 + j) * w + a];
    g2[j] = Z2[(row + 1 + j) * w + a];
  }
  T L0 = 0, L1 = 0, L2 = 0;
  if (c.has_lap) {
    L0 = Z0[(row + 1 + c.nD) * w + a];
    L1 = Z1[(row + 1 + c.nD) * w + a];
    L2 = Z2[(row + 1 + c.nD) * w + a];
  }
  T h0, h1, h2, hk0[kMaxDim], hk1[kMaxDim], hk2[kMaxDim], hL[3];
  act2_unit(c, z0, z1, z2, g0, g1, g2, L0, L1, L2, &h0, &h1, &h2, hk0, hk1, hk2, hL);
  T* B0 = H3;
  T* B1 = H3 + R * w;
  T* B2 = H3 + 2 * R * w;
  B0[row * w + a] = h0; B1[row * w + a] = h1; B2[row * w + a] = h2;
  for (int j = 0; j < c.nD; ++j) {
    B0[(row + 1 + j) * w + a] = hk0[j];
    B1[(row + 1 + j) * w + a] = hk1[j];
    B2[(row + 1 + j) * w + a] = hk2[j];
  }
  if (c.has_lap) {
    B0[(row + 1 + c.nD) * w + a] = hL[0];
    B1[(row + 1 + c.nD) * w + a] = hL[1];
    B2[(row + 1 + c.nD) * w + a] = hL[2];
  }
}

// Output layer of the t-2-jet: f_vv_p = scale * Op(u'') with
// u'' = w.h'' + 2 w_v.h' (the output bias moves linearly and drops out).
template <typename T>
__global__ void k_output_fvv(NetInfo net, const T* __restrict__ theta, const T* __restrict__ v,
                             const T* __restrict__ H3, double* __restrict__ fvv) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= net.m) return;
  const int p = warp;
  const ClassInfo& c = class_of(net, p);
  const int L = net.n_layers - 1;
  T acc = 0;
  if (L > 0) {
    const int w = net.widths[L];
    const long long R = net.R;
    const T* wo = theta + net.w_off[L];
    const T* wv = v + net.w_off[L];
    const T* B1 = H3 + R * w;
    const T* B2 = H3 + 2 * R * w;
    const long long row = c.row0 + (long long)(p - c.p0) * c.S;
    for (int s = 0; s < c.S; ++s) {
      T coef;
      if (s == 0) coef = T(c.c_val);
      else if (s <= c.nD) coef = T(c.c_gradD[s - 1]);
      else coef = T(c.c_lap);
      if (coef == T(0)) continue;
      T u = 0;
      for (int a = lane; a < w; a += 32)
        u += wo[a] * B2[(row + s) * w + a] + T(2) * wv[a] * B1[(row + s) * w + a];
      acc += coef * u;
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) fvv[p] = (double)acc * c.scale;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

// C = alpha A B^T + beta C (A [M x K], B [N x K]) or, with b_kn, B given as
// [K x N]: on the TF32 tensor cores (3xTF32) when a scratch is given and
// fits, else on the FP32 / FP64 SIMT GEMM.
template <typename T>
static dngd_status layer_gemm(int M, int N, int K, T alpha, const T* A, int lda, const T* B, int ldb, bool b_kn,
                              T beta, T* C, int ldc, const Tc3Scratch* tc3, int* status, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (tc3 && status) {
      const dngd_status s =
          gemm_tc3(M, N, K, alpha, A, lda, false, B, ldb, b_kn, beta, C, ldc, false, *tc3, status, st);
      if (s != DNGD_ERR_INVALID_ARG) return s;
    }
  } else {
    if (tc3 && tc3->ozg && status) {
      const dngd_status s = oz_gemm(tc3->ozg, M, N, K, alpha, A, lda, B, ldb, b_kn, beta, C, ldc, status, st);
      if (s != DNGD_ERR_INVALID_ARG) return s;
    }
  }
  return b_kn ? gemm_nn<T>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st)
              : gemm_nt<T>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, false, st);
}

template <typename T>
dngd_status jets_forward(const NetInfo& net, const T* theta, const double* X, const double* target,
                         LayerPtrs<T> Z, LayerPtrs<T> H, double* r, int* status, cudaStream_t st,
                         const Tc3Scratch* tc3, bool streams) {
  const int L = net.n_layers - 1;
  const int thr = 128;
  // forward-only sweep on the TF32 tensor cores: every hidden GEMM fits the
  // scratch, so each layer but the last hands its activations over as the
  // next GEMM's A operand split
  bool presplit = false;
  float *a_half = nullptr, *b_half = nullptr;
  if constexpr (std::is_same<T, float>::value) {
    if (tc3 && tc3->buf && !streams) {
      presplit = true;
      for (int l = 1; l < L; ++l)
        presplit = presplit && tc3_scratch_bytes(net.R, net.widths[l + 1], net.widths[l]) <= tc3->bytes;
      if (presplit) tc3_halves(*tc3, &a_half, &b_half);
    }
  }
  for (int l = 0; l < L; ++l) {
    const int w = net.widths[l + 1];
    const bool split_out = presplit && l + 1 < L;
    const int kp = (w + 31) & ~31;
    float* hs = split_out ? a_half : nullptr;
    dim3 grid(net.m, cdiv(split_out ? kp : w, thr));
    if (l == 0) {
      DNGD_NOTE_LAUNCH();
      k_first_layer<T><<<grid, thr, 0, st>>>(net, theta, X, Z.p[0], H.p[0], hs, kp);
    } else {
      dngd_status s = DNGD_ERR_INVALID_ARG;
      if constexpr (std::is_same<T, float>::value) {
        if (presplit)
          s = gemm_tc3(net.R, w, net.widths[l], 1.0f, H.p[l - 1], net.widths[l], false, theta + net.w_off[l],
                       net.widths[l], false, 0.0f, Z.p[l], w, false, *tc3, status, st, TC3_A_PRESPLIT);
        else if (tc3)
          s = gemm_tc3(net.R, w, net.widths[l], 1.0f, H.p[l - 1], net.widths[l], false, theta + net.w_off[l],
                       net.widths[l], false, 0.0f, Z.p[l], w, false, *tc3, status, st);
      }
      if (s == DNGD_ERR_INVALID_ARG && !presplit)
        s = layer_gemm<T>(net.R, w, net.widths[l], T(1), H.p[l - 1], net.widths[l], theta + net.w_off[l],
                          net.widths[l], false, T(0), Z.p[l], w, std::is_same<T, float>::value ? nullptr : tc3,
                          status, st);
      if (s) return s;
      DNGD_NOTE_LAUNCH();
      k_act_fwd<T><<<grid, thr, 0, st>>>(net, l, theta, Z.p[l], H.p[l], hs, kp);
    }
    DNGD_LAUNCH_CHECK();
  }
  const T* Hlast = L > 0 ? H.p[L - 1] : nullptr;
  DNGD_NOTE_LAUNCH();
  k_output<T><<<cdiv((long long)net.m * 32, 256), 256, 0, st>>>(net, theta, X, Hlast, target, r, status);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// Forward-only sweeps of G line-search trials at once (grid.z = trial): the
// trials' FP32 parameters are theta_b + g n; each layer's activations go to
// the next 3xTF32 GEMM as split operands stacked by trial in the scratch's A
// half, every hidden GEMM is one launch for all trials, the pre-activations
// of trial g sit at Zb + g R w, the last activations at Hb + g R w_L and the
// residuals at rb + g m.  INVALID_ARG when the scratch cannot hold G trials.
dngd_status jets_forward_trials(const NetInfo& net, int G, const float* theta_b, long long n, const double* X,
                                const double* target, float* Zb, float* Hb, double* rb, int* status, cudaStream_t st,
                                const Tc3Scratch& tc3) {
  const int L = net.n_layers - 1;
  const int thr = 128;
  const long long R = net.R;
  if (L < 2 || !tc3.buf) return DNGD_ERR_INVALID_ARG;
  float *a_half, *b_half;
  tc3_halves(tc3, &a_half, &b_half);
  for (int l = 1; l < L; ++l) {
    const long long kp = (net.widths[l] + 31) & ~31;
    if ((long long)G * R * 2 * kp > (long long)(b_half - a_half)) return DNGD_ERR_INVALID_ARG;
    if ((long long)G * net.widths[l + 1] * 2 * kp > (long long)(b_half - a_half)) return DNGD_ERR_INVALID_ARG;
  }
  for (int l = 0; l < L; ++l) {
    const int w = net.widths[l + 1];
    const bool split_out = l + 1 < L;
    const int kp = (w + 31) & ~31;
    TrialStride zs;
    zs.theta = n;
    zs.z = R * w;
    zs.h = R * w;
    zs.hs = R * 2 * kp;
    dim3 grid(net.m, cdiv(split_out ? kp : w, thr), G);
    if (l == 0) {
      DNGD_NOTE_LAUNCH();
      k_first_layer<float><<<grid, thr, 0, st>>>(net, theta_b, X, Zb, Hb, a_half, kp, zs);
    } else {
      dngd_status s = gemm_tc3_trials(G, (int)R, w, net.widths[l], theta_b + net.w_off[l], net.widths[l], n, Zb, w,
                                      R * w, tc3, status, st);
      if (s) return s;
      DNGD_NOTE_LAUNCH();
      k_act_fwd<float><<<grid, thr, 0, st>>>(net, l, theta_b, Zb, Hb, split_out ? a_half : nullptr, kp, zs);
    }
    DNGD_LAUNCH_CHECK();
  }
  TrialStride zo;
  zo.theta = n;
  zo.h = R * net.widths[L];
  zo.r = net.m;
  DNGD_NOTE_LAUNCH();
  k_output<float><<<dim3(cdiv((long long)net.m * 32, 256), 1, G), 256, 0, st>>>(net, theta_b, X, Hb, target, rb, status,
                                                                                 zo);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

template <typename T, typename TJ>
dngd_status jets_backward_jacobian(const NetInfo& net, const T* theta, const double* X, LayerPtrs<T> Z,
                                   LayerPtrs<T> H, LayerPtrs<T> D, T* Hbar, TJ* J, long long ldJ,
                                   __nv_bfloat16* Jb, long long ldb, cudaStream_t st, const Tc3Scratch* tc3,
                                   int* status, unsigned* rowmax, bool df64) {
  const int L = net.n_layers - 1;
  const int thr = 128;
  for (int l = L - 1; l >= 0; --l) {
    const int w = net.widths[l + 1];
    dim3 grid(net.m, cdiv(w, thr));
    DNGD_NOTE_LAUNCH();
    k_act_bwd<T><<<grid, thr, 0, st>>>(net, l, theta, Z.p[l], l == L - 1 ? nullptr : Hbar, D.p[l]);
    DNGD_LAUNCH_CHECK();
    if (l > 0) {
      // Hbar_{l-1} = D_l W_l  (rows x w_l)
      dngd_status s = layer_gemm<T>(net.R, net.widths[l], w, T(1), D.p[l], w, theta + net.w_off[l],
                                    net.widths[l], true, T(0), Hbar, net.widths[l], tc3, status, st);
      if (s) return s;
    }
  }
  int maxS = 1;
  for (int c = 0; c < net.n_classes; ++c) maxS = net.cls[c].S > maxS ? net.cls[c].S : maxS;
  int maxw = 1;
  for (int l = 0; l <= L; ++l) {
    const int ws = net.widths[l + 1] + net.widths[l];
    maxw = ws > maxw ? ws : maxw;
  }
  int maxwo = 1;
  for (int l = 0; l <= L; ++l) maxwo = net.widths[l + 1] > maxwo ? net.widths[l + 1] : maxwo;
  const bool df = df64 && std::is_same<T, double>::value;
  const size_t smem = (size_t)maxS * maxw * sizeof(T) + (df ? (size_t)maxS * maxwo * sizeof(float2) : 0);
  if (smem > 48 * 1024) {
    static bool attr = false, attr_df = false;
    if (!df && !attr) {
      DNGD_CUDA_CHECK(allow_max_dynamic_smem((const void*)k_jac_write<T, TJ, false>));
      attr = true;
    }
    if (df && !attr_df) {
      DNGD_CUDA_CHECK(allow_max_dynamic_smem((const void*)k_jac_write<T, TJ, true>));
      attr_df = true;
    }
  }
  if (J == nullptr) return DNGD_OK;  // matrix-free use: stream adjoints only
  dim3 grid(net.m, L + 1);
  if (rowmax) DNGD_CUDA_CHECK(cudaMemsetAsync(rowmax, 0, sizeof(unsigned) * net.m, st));
  DNGD_NOTE_LAUNCH();
  if (df)
    k_jac_write<T, TJ, true><<<grid, 256, smem, st>>>(net, theta, X, H, D, J, ldJ, Jb, ldb, rowmax);
  else
    k_jac_write<T, TJ, false><<<grid, 256, smem, st>>>(net, theta, X, H, D, J, ldJ, Jb, ldb, rowmax);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

template <typename T>
dngd_status jets_fvv(const NetInfo& net, const T* theta, const T* v, const double* X, T* Z3, T* H3a,
                     T* H3b, double* fvv, cudaStream_t st, const Tc3Scratch* tc3, int* status) {
  const int L = net.n_layers - 1;
  const int thr = 128;
  const long long R = net.R;
  T* Hprev = H3a;
  T* Hcur = H3b;
  for (int l = 0; l < L; ++l) {
    const int w = net.widths[l + 1];
    dim3 grid(net.m, cdiv(w, thr));
    if (l == 0) {
      DNGD_NOTE_LAUNCH();
      k_first_layer_fvv<T><<<grid, thr, 0, st>>>(net, theta, v, X, Hcur);
    } else {
      const int win = net.widths[l];
      const T* W = theta + net.w_off[l];
      const T* V = v + net.w_off[l];
      // blocks 0..2: W h^(j)
      dngd_status s = layer_gemm<T>(3 * net.R, w, win, T(1), Hprev, win, W, win, false, T(0), Z3, w, tc3, status, st);
      if (s) return s;
      // block 1 += V h ; block 2 += 2 V h'
      s = layer_gemm<T>(net.R, w, win, T(1), Hprev, win, V, win, false, T(1), Z3 + R * w, w, tc3, status, st);
      if (s) return s;
      s = layer_gemm<T>(net.R, w, win, T(2), Hprev + R * win, win, V, win, false, T(1), Z3 + 2 * R * w, w, tc3,
                        status, st);
      if (s) return s;
      DNGD_NOTE_LAUNCH();
      k_act_fvv<T><<<grid, thr, 0, st>>>(net, l, theta, v, Z3, Hcur);
    }
    DNGD_LAUNCH_CHECK();
    T* tmp = Hprev;
    Hprev = Hcur;
    Hcur = tmp;
  }
  DNGD_NOTE_LAUNCH();
  k_output_fvv<T><<<cdiv((long long)net.m * 32, 256), 256, 0, st>>>(net, theta, v, Hprev, fvv);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

template dngd_status jets_forward<double>(const NetInfo&, const double*, const double*, const double*,
                                          LayerPtrs<double>, LayerPtrs<double>, double*, int*, cudaStream_t,
                                          const Tc3Scratch*, bool);
template dngd_status jets_forward<float>(const NetInfo&, const float*, const double*, const double*,
                                         LayerPtrs<float>, LayerPtrs<float>, double*, int*, cudaStream_t,
                                         const Tc3Scratch*, bool);
template dngd_status jets_backward_jacobian<double, double>(const NetInfo&, const double*, const double*,
                                                            LayerPtrs<double>, LayerPtrs<double>,
                                                            LayerPtrs<double>, double*, double*, long long,
                                                            __nv_bfloat16*, long long, cudaStream_t,
                                                            const Tc3Scratch*, int*, unsigned*, bool);
template dngd_status jets_backward_jacobian<float, float>(const NetInfo&, const float*, const double*,
                                                          LayerPtrs<float>, LayerPtrs<float>,
                                                          LayerPtrs<float>, float*, float*, long long,
                                                          __nv_bfloat16*, long long, cudaStream_t,
                                                          const Tc3Scratch*, int*, unsigned*, bool);
template dngd_status jets_fvv<double>(const NetInfo&, const double*, const double*, const double*, double*,
                                      double*, double*, double*, cudaStream_t, const Tc3Scratch*, int*);
template dngd_status jets_fvv<float>(const NetInfo&, const float*, const float*, const double*, float*,
                                     float*, float*, double*, cudaStream_t, const Tc3Scratch*, int*);

}  // namespace dngd
