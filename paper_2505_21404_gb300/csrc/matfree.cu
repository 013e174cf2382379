// Matrix-free dual solve (Sec. 3.3 of the paper): the kernel-vector product
// w = J (J^T v) + lambda v (Def. 3.3) without forming J, the Nystrom
// preconditioner (Sec. 3.3.1) and preconditioned CG (Alg. PCGStep).
//
// J is never materialised.  One forward and one reverse sweep of the
// Taylor-mode jets leave, per hidden layer l, the stream activations H_l and
// the stream adjoints D_l (one row per point-stream).  With those factors the
// Jacobian block of layer l is sum_s delta_s h_s^T per point, hence
//   J^T v :  G_l = D_l^T diag(v~) H_{l-1}          (one GEMM per layer)
//   J u   :  (J u)_i = sum_l sum_s <delta_{l,i,s}, U_l h_{l-1,i,s}>
//                                                   (one GEMM + a row-dot)
// and the landmark columns of K (Nystrom) follow the same factorisation:
//   K_ij = sum_l sum_{s,s'} (D_l D_l,I^T)[s,s'] (H H_I^T + [value rows])[s,s'],
// two GEMMs per layer and a block reduction over stream pairs.
//
// The preconditioner is P^{-1} = (K_hat + lambda I)^{-1} with the column-
// sampling Nystrom approximation K_hat = K_{:,I} K_II^{-1} K_{I,:}; it is
// applied through the Woodbury identity with M = K_{:,I} L_II^{-T}:
//   P^{-1} x = (x - M (lambda I + M^T M)^{-1} M^T x) / lambda,
// which equals the paper's U (Lambda_hat + lambda I)^{-1} U^T +
// (I - U U^T) / lambda for the same K_hat (K_hat = U Lambda_hat U^T = M M^T).
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "step_kernels.h"

namespace dngd {

namespace {

// The 3xTF32 GEMM drains its TMEM accumulator every 128 K-elements into
// round-to-nearest FP32 registers, so the whole reduction runs in one launch.
// These optional cuts (point-stream rows of J^T v, layer-input columns of
// J u, added in FP32 with beta = 1) are compile-time parameters, off by
// default.
#ifndef DNGD_MF_CHUNK
#define DNGD_MF_CHUNK (1 << 30)
#endif
#ifndef DNGD_MF_KCHUNK
#define DNGD_MF_KCHUNK (1 << 30)
#endif
constexpr int kJtvChunk = DNGD_MF_CHUNK;
constexpr int kJuChunk = DNGD_MF_KCHUNK;

// Layer-0 and bias parts of J^T v.  Thread = one output unit a of layer l.
// Writes g[w_off[l] ...] and g[b_off[l] ...] for l = 0 (weights from the
// input streams) and the biases of every hidden layer.
__global__ void k_jtv_first_and_bias(NetInfo net, const double* __restrict__ v, const double* __restrict__ X,
                                     LayerPtrs<float> D, float* __restrict__ g) {
  const int l = blockIdx.y;  // hidden layer
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int w = net.widths[l + 1];
  if (a >= w) return;
  const float* Dl = D.p[l];
  const int din = net.d_in;
  double gb = 0.0;
  double gw[kMaxDim];
  for (int k = 0; k < din; ++k) gw[k] = 0.0;
  for (int c = 0; c < net.n_classes; ++c) {
    const ClassInfo& ci = net.cls[c];
    for (int i = 0; i < ci.count; ++i) {
      const int p = ci.p0 + i;
      const long long row = ci.row0 + (long long)i * ci.S;
      const double vi = v[p];
      const double dval = Dl[row * w + a];
      gb += vi * dval;
      if (l == 0) {
        for (int k = 0; k < din; ++k) gw[k] += vi * dval * X[(long long)p * din + k];
        for (int j = 0; j < ci.nD; ++j) gw[ci.D[j]] += vi * (double)Dl[(row + 1 + j) * w + a];
      }
    }
  }
  g[net.b_off[l] + a] = (float)gb;
  if (l == 0)
    for (int k = 0; k < din; ++k) g[net.w_off[0] + (long long)a * din + k] = (float)gw[k];
}

// Output-layer part of J^T v: g_W[b] = sum_i v_i sum_s ubar_s H_{L-1}[row_s][b],
// g_b = sum_i v_i ubar_val.  Thread = one input unit b (block 0 thread 0 also
// writes the bias).  With no hidden layer the inputs are the input streams.
__global__ void k_jtv_out(NetInfo net, const double* __restrict__ v, const double* __restrict__ X,
                          const float* __restrict__ Hlast, float* __restrict__ g) {
  const int L = net.n_layers - 1;
  const int w = net.widths[L];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < w) {
    double acc = 0.0;
    for (int c = 0; c < net.n_classes; ++c) {
      const ClassInfo& ci = net.cls[c];
      for (int i = 0; i < ci.count; ++i) {
        const int p = ci.p0 + i;
        const double vi = v[p] * ci.scale;
        if (L == 0) {
          double hv = X[(long long)p * net.d_in + b] * ci.c_val;
          for (int j = 0; j < ci.nD; ++j)
            if (ci.D[j] == b) hv += ci.c_gradD[j];
          acc += vi * hv;
        } else {
          const long long row = ci.row0 + (long long)i * ci.S;
          double hv = 0.0;
          for (int s = 0; s < ci.S; ++s) {
            const double coef = s == 0 ? ci.c_val : (s <= ci.nD ? ci.c_gradD[s - 1] : ci.c_lap);
            hv += coef * (double)Hlast[(row + s) * w + b];
          }
          acc += vi * hv;
        }
      }
    }
    g[net.w_off[L] + b] = (float)acc;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double acc = 0.0;
    for (int c = 0; c < net.n_classes; ++c) {
      const ClassInfo& ci = net.cls[c];
      for (int i = 0; i < ci.count; ++i) acc += v[ci.p0 + i] * ci.scale * ci.c_val;
    }
    g[net.b_off[L]] = (float)acc;
  }
}

// Row weights for the J^T v GEMMs: vrow[row] = v[point of row].
__global__ void k_expand_rows(NetInfo net, const double* __restrict__ v, float* __restrict__ vrow) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= net.m) return;
  const ClassInfo& ci = class_of(net, p);
  const long long row = ci.row0 + (long long)(p - ci.p0) * ci.S;
  for (int s = 0; s < ci.S; ++s) vrow[row + s] = (float)v[p];
}

// J u: y_p (+)= sum over the point's rows and units of D_l * (Y + bias on the
// value row).  For l == 0, Y is built on the fly from U_0 and the input
// streams.  One warp per point; FP32 partials, FP64 accumulation.
__global__ void k_jv_rowdot(NetInfo net, int l, const float* __restrict__ Dl, const float* __restrict__ Y,
                            const float* __restrict__ u, const double* __restrict__ X, double* __restrict__ y,
                            int accumulate) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= net.m) return;
  const int p = warp;
  const ClassInfo& ci = class_of(net, p);
  const int w = net.widths[l + 1];
  const long long row = ci.row0 + (long long)(p - ci.p0) * ci.S;
  const float* ub = u + net.b_off[l];
  double acc = 0.0;   // FP32 products are exact in FP64
  if (l == 0) {
    const float* U0 = u + net.w_off[0];
    const int din = net.d_in;
    for (int a = lane; a < w; a += 32) {
      double yv = ub[a];
      for (int k = 0; k < din; ++k) yv += (double)U0[(long long)a * din + k] * X[(long long)p * din + k];
      acc += (double)Dl[row * w + a] * yv;
      for (int j = 0; j < ci.nD; ++j) acc += (double)Dl[(row + 1 + j) * w + a] * (double)U0[(long long)a * din + ci.D[j]];
    }
  } else {
    for (int s = 0; s < ci.S; ++s)
      for (int a = lane; a < w; a += 32)
        acc += (double)Dl[(row + s) * w + a] * ((double)Y[(row + s) * w + a] + (s == 0 ? (double)ub[a] : 0.0));
  }
  const double t = warp_sum(acc);
  if (lane == 0) y[p] = accumulate ? y[p] + t : t;
}

// Output layer of J u: y_p += sum_s ubar_s (u_out . h_s) + ubar_val u_bout.
__global__ void k_jv_out(NetInfo net, const float* __restrict__ Hlast, const float* __restrict__ u,
                         const double* __restrict__ X, double* __restrict__ y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= net.m) return;
  const int p = warp;
  const ClassInfo& ci = class_of(net, p);
  const int L = net.n_layers - 1;
  const int w = net.widths[L];
  const float* uo = u + net.w_off[L];
  float acc = 0.f;
  if (L == 0) {
    if (lane == 0) {
      for (int k = 0; k < net.d_in; ++k) acc += (float)ci.c_val * uo[k] * (float)X[(long long)p * net.d_in + k];
      for (int j = 0; j < ci.nD; ++j) acc += (float)ci.c_gradD[j] * uo[ci.D[j]];
    }
  } else {
    const long long row = ci.row0 + (long long)(p - ci.p0) * ci.S;
    for (int s = 0; s < ci.S; ++s) {
      const float coef = s == 0 ? (float)ci.c_val : (s <= ci.nD ? (float)ci.c_gradD[s - 1] : (float)ci.c_lap);
      if (coef == 0.f) continue;
      float d = 0.f;
      for (int b = lane; b < w; b += 32) d += uo[b] * Hlast[(row + s) * w + b];
      acc += coef * d;
    }
  }
  double t = warp_sum((double)acc);
  if (lane == 0) {
    t += (double)ci.c_val * (double)u[net.b_off[L]];
    y[p] += ci.scale * t;
  }
}

// Input streams of layer 0 as explicit rows (value = x, derivative = e_k,
// Laplacian = 0): Hin [R x d_in].
__global__ void k_input_rows(NetInfo net, const double* __restrict__ X, float* __restrict__ Hin) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= net.m) return;
  const ClassInfo& ci = class_of(net, p);
  const long long row = ci.row0 + (long long)(p - ci.p0) * ci.S;
  const int din = net.d_in;
  for (int s = 0; s < ci.S; ++s)
    for (int k = 0; k < din; ++k) {
      float v = 0.f;
      if (s == 0) v = (float)X[(long long)p * din + k];
      else if (s <= ci.nD) v = (ci.D[s - 1] == k) ? 1.f : 0.f;
      Hin[(row + s) * din + k] = v;
    }
}

// Gather landmark rows: out[r][c] = in[rows[r]][c].
__global__ void k_gather_rows(int nr, int w, const int* __restrict__ rows, const float* __restrict__ in,
                              float* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nr * w) return;
  const int r = (int)(idx / w), c = (int)(idx % w);
  out[idx] = in[(long long)rows[r] * w + c];
}

// K_CI[p][j] (+)= sum_{s in rows(p), s' in rows(landmark j)} P[s][s'] (Q[s][s'] + [s, s' value rows])
__global__ void k_ghost_accum(NetInfo net, int ell, const int* __restrict__ lrow0, const int* __restrict__ lS,
                              const float* __restrict__ P, const float* __restrict__ Q, long long ldpq, int bias,
                              float* __restrict__ KCI, int accumulate) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)net.m * ell) return;
  const int p = (int)(idx / ell), j = (int)(idx % ell);
  const ClassInfo& ci = class_of(net, p);
  const long long row = ci.row0 + (long long)(p - ci.p0) * ci.S;
  const int r0 = lrow0[j], Sj = lS[j];
  float acc = 0.f;
  for (int s = 0; s < ci.S; ++s)
    for (int t = 0; t < Sj; ++t) {
      const long long e = (row + s) * ldpq + r0 + t;
      const float q = Q ? Q[e] : 0.f;
      acc += P[e] * (q + ((bias && s == 0 && t == 0) ? 1.f : 0.f));
    }
  KCI[idx] = accumulate ? KCI[idx] + acc : acc;
}

// Output-layer contribution: F[p][b] = scale_p sum_s coef_s H_{L-1}[row_s][b]
// (the output weight row of J), plus the output bias term c_val*scale.
__global__ void k_out_features(NetInfo net, const float* __restrict__ Hlast, const double* __restrict__ X,
                               float* __restrict__ F, float* __restrict__ fb) {
  const int p = blockIdx.x;
  const ClassInfo& ci = class_of(net, p);
  const int L = net.n_layers - 1;
  const int w = net.widths[L];
  for (int b = threadIdx.x; b < w; b += blockDim.x) {
    float hv = 0.f;
    if (L == 0) {
      hv = (float)X[(long long)p * net.d_in + b] * (float)ci.c_val;
      for (int j = 0; j < ci.nD; ++j)
        if (ci.D[j] == b) hv += (float)ci.c_gradD[j];
    } else {
      const long long row = ci.row0 + (long long)(p - ci.p0) * ci.S;
      for (int s = 0; s < ci.S; ++s) {
        const float coef = s == 0 ? (float)ci.c_val : (s <= ci.nD ? (float)ci.c_gradD[s - 1] : (float)ci.c_lap);
        hv += coef * Hlast[(row + s) * w + b];
      }
    }
    F[(long long)p * w + b] = (float)ci.scale * hv;
  }
  if (threadIdx.x == 0) fb[p] = (float)(ci.scale * ci.c_val);
}

// KCI[p][j] += fb[p] fb[I_j]
__global__ void k_add_outer_bias(int m, int ell, const int* __restrict__ lm, const float* __restrict__ fb,
                                 float* __restrict__ KCI) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * ell) return;
  const int p = (int)(idx / ell), j = (int)(idx % ell);
  KCI[idx] += fb[p] * fb[lm[j]];
}

// KII[a][b] = KCI[lm[a]][b] (+ nu on the diagonal)
__global__ void k_extract_kii(int ell, const int* __restrict__ lm, const float* __restrict__ KCI, double nu,
                              float* __restrict__ KII) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ell * ell) return;
  const int a = idx / ell, b = idx % ell;
  KII[idx] = KCI[(long long)lm[a] * ell + b] + (a == b ? (float)nu : 0.f);
}

__global__ void k_to_double(long long n, const float* __restrict__ x, double alpha, double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = alpha * (double)x[i];
}

// tr(K_II) = sum_j K_CI[lm[j]][j]
__global__ void k_kii_trace(int ell, const int* __restrict__ lm, const float* __restrict__ KCI, double* out) {
  double s = 0.0;
  for (int j = threadIdx.x; j < ell; j += blockDim.x) s += (double)KCI[(long long)lm[j] * ell + j];
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

// z = (x - t) / lambda
__global__ void k_woodbury_finish(int m, const double* __restrict__ x, const double* __restrict__ t, double lam,
                                  double* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) z[i] = (x[i] - t[i]) / lam;
}

}  // namespace

// ---------------------------------------------------------------------------

dngd_status mf_jtv(const MatFree& F, const double* v, float* g, cudaStream_t st) {
  const NetInfo& net = *F.net;
  const int L = net.n_layers - 1;
  DNGD_NOTE_LAUNCH();
  k_expand_rows<<<cdiv(net.m, 256), 256, 0, st>>>(net, v, F.vrow);
  for (int l = 1; l < L; ++l) {
    const int wo = net.widths[l + 1], wi = net.widths[l];
    if (F.tc3) {
      // G_l = D_l^T diag(v) H_{l-1} over all R point-stream rows (or in cuts
      // of kJtvChunk rows added with beta = 1)
      for (int r0 = 0; r0 < net.R; r0 += kJtvChunk) {
        const int cr = net.R - r0 < kJtvChunk ? net.R - r0 : kJtvChunk;
        dngd_status s = gemm_tc3(wo, wi, cr, 1.0f, F.D.p[l] + (long long)r0 * wo, wo, true,
                                 F.H.p[l - 1] + (long long)r0 * wi, wi, true, r0 ? 1.0f : 0.0f, g + net.w_off[l], wi,
                                 false, *F.tc3, F.status, st, 0u, F.vrow + r0);
        if (s) return s;
      }
      continue;
    }
    dngd_status s = gemm_tn_comp(wo, wi, net.R, 1.0f, F.D.p[l], wo, F.H.p[l - 1], wi, 0.0f, g + net.w_off[l], wi,
                                 F.vrow, st);
    if (s) return s;
  }
  if (L >= 1) {
    DNGD_NOTE_LAUNCH();
    k_jtv_first_and_bias<<<dim3(cdiv(net.max_w, 128), L), 128, 0, st>>>(net, v, F.X, F.D, g);
  }
  const int wlast = net.widths[L];
  DNGD_NOTE_LAUNCH();
  k_jtv_out<<<cdiv(wlast, 128), 128, 0, st>>>(net, v, F.X, L > 0 ? F.H.p[L - 1] : nullptr, g);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

dngd_status mf_jv(const MatFree& F, const float* u, double* y, cudaStream_t st) {
  const NetInfo& net = *F.net;
  const int L = net.n_layers - 1;
  const int blocks = cdiv((long long)net.m * 32, 256);
  DNGD_CUDA_CHECK(cudaMemsetAsync(y, 0, sizeof(double) * net.m, st));
  for (int l = 0; l < L; ++l) {
    const int wo = net.widths[l + 1], wi = net.widths[l];
    if (l > 0) {
      // Y = H_{l-1} U_l^T (K = the layer width)
      dngd_status s = DNGD_OK;
      if (F.tc3) {
        for (int k0 = 0; k0 < wi && !s; k0 += kJuChunk) {
          const int kc = wi - k0 < kJuChunk ? wi - k0 : kJuChunk;
          s = gemm_tc3(net.R, wo, kc, 1.0f, F.H.p[l - 1] + k0, wi, false, u + net.w_off[l] + k0, wi, false,
                       k0 ? 1.0f : 0.0f, F.Y, wo, false, *F.tc3, F.status, st);
        }
      } else {
        s = gemm_nt_comp(net.R, wo, wi, 1.0f, F.H.p[l - 1], wi, u + net.w_off[l], wi, 0.0f, F.Y, wo, st);
      }
      if (s) return s;
    }
    DNGD_NOTE_LAUNCH();
    k_jv_rowdot<<<blocks, 256, 0, st>>>(net, l, F.D.p[l], F.Y, u, F.X, y, 1);
  }
  DNGD_NOTE_LAUNCH();
  k_jv_out<<<blocks, 256, 0, st>>>(net, L > 0 ? F.H.p[L - 1] : nullptr, u, F.X, y);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// w = J (J^T v) + lambda v
dngd_status mf_kvp(const MatFree& F, const double* v, double lambda, double* w, cudaStream_t st) {
  dngd_status s = mf_jtv(F, v, F.g32, st);
  if (s) return s;
  s = mf_jv(F, F.g32, w, st);
  if (s) return s;
  return add_scaled(F.net->m, lambda, v, w, st);
}

// K_{:,I} (m x ell, FP32) by the ghost-Gram identity.
dngd_status mf_kci(const MatFree& F, cudaStream_t st) {
  const NetInfo& net = *F.net;
  const int L = net.n_layers - 1;
  const int m = net.m, ell = F.ell;
  const long long tot = (long long)m * ell;
  bool first = true;
  for (int l = 0; l < L; ++l) {
    const int wo = net.widths[l + 1];
    const int wi = l == 0 ? net.d_in : net.widths[l];
    const float* Hin = l == 0 ? F.Hin : F.H.p[l - 1];
    // landmark rows of D_l and of the layer input
    DNGD_NOTE_LAUNCH();
    k_gather_rows<<<cdiv((long long)F.RI * wo, 256), 256, 0, st>>>(F.RI, wo, F.lrows, F.D.p[l], F.DI);
    DNGD_NOTE_LAUNCH();
    k_gather_rows<<<cdiv((long long)F.RI * wi, 256), 256, 0, st>>>(F.RI, wi, F.lrows, Hin, F.HI);
    dngd_status s = F.tc3 ? gemm_tc3(net.R, F.RI, wo, 1.0f, F.D.p[l], wo, false, F.DI, wo, false, 0.0f, F.P, F.RI,
                                     false, *F.tc3, F.status, st)
                          : gemm_nt<float>(net.R, F.RI, wo, 1.0f, F.D.p[l], wo, F.DI, wo, 0.0f, F.P, F.RI, false, st);
    if (s) return s;
    s = F.tc3 ? gemm_tc3(net.R, F.RI, wi, 1.0f, Hin, wi, false, F.HI, wi, false, 0.0f, F.Q, F.RI, false, *F.tc3,
                         F.status, st)
              : gemm_nt<float>(net.R, F.RI, wi, 1.0f, Hin, wi, F.HI, wi, 0.0f, F.Q, F.RI, false, st);
    if (s) return s;
    DNGD_NOTE_LAUNCH();
    k_ghost_accum<<<cdiv(tot, 256), 256, 0, st>>>(net, ell, F.lrow0, F.lS, F.P, F.Q, F.RI, 1, F.KCI, first ? 0 : 1);
    first = false;
  }
  // output layer: F F_I^T + bias outer product
  const int wl = net.widths[L];
  DNGD_NOTE_LAUNCH();
  k_out_features<<<m, 128, 0, st>>>(net, L > 0 ? F.H.p[L - 1] : nullptr, F.X, F.Fo, F.fb);
  DNGD_NOTE_LAUNCH();
  k_gather_rows<<<cdiv((long long)ell * wl, 256), 256, 0, st>>>(ell, wl, F.lm, F.Fo, F.FoI);
  dngd_status s = gemm_nt<float>(m, ell, wl, 1.0f, F.Fo, wl, F.FoI, wl, first ? 0.0f : 1.0f, F.KCI, ell, false, st);
  if (s) return s;
  DNGD_NOTE_LAUNCH();
  k_add_outer_bias<<<cdiv(tot, 256), 256, 0, st>>>(m, ell, F.lm, F.fb, F.KCI);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

// Nystrom factors: L_II (with shift nu), M = K_CI L_II^{-T}, C = lambda I + M^T M
// and the explicit inverse of chol(C).  Returns NOT_SPD if K_II + nu I does
// not factor.
dngd_status mf_nystrom(const MatFree& F, double lambda, double nu, int* status, cudaStream_t st) {
  const int m = F.net->m, ell = F.ell;
  DNGD_NOTE_LAUNCH();
  k_extract_kii<<<cdiv(ell * ell, 256), 256, 0, st>>>(ell, F.lm, F.KCI, nu, F.KII);
  DNGD_CUDA_CHECK(cudaMemsetAsync(F.LIIinv, 0, sizeof(float) * (size_t)ell * ell, st));
  dngd_status s = cholesky_f32_inv(ell, F.KII, ell, F.LIIinv, ell, status, st);
  if (s) return s;
  if ((s = trtri_offdiag_f32(ell, F.KII, ell, F.LIIinv, ell, F.work, st))) return s;
  // M = K_CI L^{-T}  (m x ell)
  if ((s = gemm_nt<float>(m, ell, ell, 1.0f, F.KCI, ell, F.LIIinv, ell, 0.0f, F.M, ell, false, st))) return s;
  // C = M^T M + lambda I
  if ((s = gemm_tn<float>(ell, ell, m, 1.0f, F.M, ell, F.M, ell, 0.0f, F.C, ell, nullptr, st))) return s;
  if ((s = add_diag<float>(ell, F.C, ell, lambda, st))) return s;
  DNGD_CUDA_CHECK(cudaMemsetAsync(F.LCinv, 0, sizeof(float) * (size_t)ell * ell, st));
  if ((s = cholesky_f32_inv(ell, F.C, ell, F.LCinv, ell, status, st))) return s;
  return trtri_offdiag_f32(ell, F.C, ell, F.LCinv, ell, F.work, st);
}

// z = P^{-1} x = (x - M (L_C^{-T} (L_C^{-1} (M^T x)))) / lambda
dngd_status mf_precond(const MatFree& F, double lambda, const double* x, double* z, cudaStream_t st) {
  const int m = F.net->m, ell = F.ell;
  dngd_status s = gemv_t_f32(m, ell, F.M, ell, x, 1.0, F.t1, F.partials, F.partial_cap, F.xs, st);
  if (s) return s;
  if ((s = gemv_n_f32(ell, ell, F.LCinv, ell, F.t1, 1.0, F.t2, nullptr, 0.0, F.xs, st))) return s;
  if ((s = gemv_t_f32(ell, ell, F.LCinv, ell, F.t2, 1.0, F.t1, F.partials, F.partial_cap, F.xs, st))) return s;
  if ((s = gemv_n_f32(m, ell, F.M, ell, F.t1, 1.0, F.t3, nullptr, 0.0, F.xs, st))) return s;
  DNGD_NOTE_LAUNCH();
  k_woodbury_finish<<<cdiv(m, 256), 256, 0, st>>>(m, x, F.t3, lambda, z);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

dngd_status mf_input_rows(const MatFree& F, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_input_rows<<<cdiv(F.net->m, 256), 256, 0, st>>>(*F.net, F.X, F.Hin);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

dngd_status mf_g_to_double(long long n, const float* g, double alpha, double* out, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_to_double<<<cdiv(n, 256), 256, 0, st>>>(n, g, alpha, out);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

dngd_status mf_kii_trace(const MatFree& F, double* out, cudaStream_t st) {
  DNGD_NOTE_LAUNCH();
  k_kii_trace<<<1, 256, 0, st>>>(F.ell, F.lm, F.KCI, out);
  DNGD_LAUNCH_CHECK();
  return DNGD_OK;
}

}  // namespace dngd
