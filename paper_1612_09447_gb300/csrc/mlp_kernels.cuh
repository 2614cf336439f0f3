// Learned start vector of the M-solves: per-node 8-32-32-1 network with
// exact-erf GELU, BF16 weights (staged in shared memory as FP32) and FP32
// arithmetic/accumulation.  Start-vector estimation from earlier solutions
// is the subject of Section IV; this estimator is a project addition.
//
// Parameter layout (1377 values): W1 (32x8, row-major), b1 (32), W2 (32x32),
// b2 (32), w3 (32), b3.  Inputs at free node i: the last four solutions
// h1..h4 and their means over the free graph neighbours, divided by
// s_h = RMS(h1); output o; start vector z0 = h1 + s_h o.
#pragma once

#include <cuda_bf16.h>

#include "kernels.cuh"

namespace eqs {

constexpr int kNP = 1377;
constexpr int kTrainBlock = 128;

// splitmix64 finaliser (Steele, Lea, Flood 2014): value k of stream `seed`.
__device__ __forceinline__ uint64_t smix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_df(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__device__ __forceinline__ void load_weights(const __nv_bfloat16* __restrict__ wb, float* sw) {
  for (int k = threadIdx.x; k < kNP; k += blockDim.x) sw[k] = __bfloat162float(wb[k]);
  __syncthreads();
}

// Normalised inputs at free node i from four history vectors.
__device__ __forceinline__ void node_features(int i, const float* __restrict__ h0, const float* __restrict__ h1,
                                              const float* __restrict__ h2, const float* __restrict__ h3,
                                              const int32_t* __restrict__ adj_ptr,
                                              const int32_t* __restrict__ adj_col,
                                              const float* __restrict__ inv_deg, float inv_s, float x[8]) {
  x[0] = h0[i] * inv_s;
  x[1] = h1[i] * inv_s;
  x[2] = h2[i] * inv_s;
  x[3] = h3[i] * inv_s;
  float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
  const int e = adj_ptr[i + 1];
  for (int k = adj_ptr[i]; k < e; ++k) {
    const int j = adj_col[k];
    m0 += h0[j];
    m1 += h1[j];
    m2 += h2[j];
    m3 += h3[j];
  }
  const float w = inv_deg[i] * inv_s;
  x[4] = m0 * w;
  x[5] = m1 * w;
  x[6] = m2 * w;
  x[7] = m3 * w;
}

__device__ __forceinline__ float mlp_forward(const float* sw, const float x[8]) {
  const float* W1 = sw;
  const float* b1 = sw + 256;
  const float* W2 = sw + 288;
  const float* b2 = sw + 1312;
  const float* w3 = sw + 1344;
  float g1[32];
#pragma unroll
  for (int o = 0; o < 32; ++o) {
    float a = b1[o];
#pragma unroll
    for (int k = 0; k < 8; ++k) a = fmaf(W1[o * 8 + k], x[k], a);
    g1[o] = gelu_f(a);
  }
  float out = sw[1376];
#pragma unroll 4
  for (int o = 0; o < 32; ++o) {
    float a = b2[o];
#pragma unroll
    for (int k = 0; k < 32; ++k) a = fmaf(W2[o * 32 + k], g1[k], a);
    out = fmaf(w3[o], gelu_f(a), out);
  }
  return out;
}

// s_h = sqrt(mean(h1^2)) over the free nodes.
__global__ void k_rms(int n, const double* __restrict__ h, double* sh, double* partials,
                      unsigned int* counter, int max_blocks) {
  pdl_enter();
  double v[1] = {0.0};
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) v[0] += h[i] * h[i];
  double tot[1];
  if (grid_sum<1>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) *sh = sqrt(tot[0] / n);
}

// z0 = h1 + s_h MLP(features) for the solve with global index
// g = stepcount[0] + j (solves before this step + stage); the history ring
// holds solution k in slot k % 4.
// With fewer than four earlier solutions (or s_h = 0) z0 = h1.
__global__ void k_mlp_guess(int nf, const double* __restrict__ h1d, const float* __restrict__ ring,
                            const long long* __restrict__ stepcount, int s, int j,
                            const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj_col,
                            const float* __restrict__ inv_deg, const __nv_bfloat16* __restrict__ wb,
                            const double* __restrict__ sh, double* __restrict__ z0) {
  pdl_enter();
  __shared__ float sw[kNP + 3];
  load_weights(wb, sw);
  const long long g = stepcount[0] + j;
  const double s_h = *sh;
  const bool use = g >= 4 && s_h > 0.0;
  const float* hr[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) hr[l] = ring + (size_t)(((g - 1 - l) % 4 + 4) % 4) * nf;
  const float inv_s = use ? (float)(1.0 / s_h) : 0.f;
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    if (!use) {
      z0[i] = h1d[i];
      continue;
    }
    float x[8];
    node_features((int)i, hr[0], hr[1], hr[2], hr[3], adj_ptr, adj_col, inv_deg, inv_s, x);
    z0[i] = h1d[i] + s_h * (double)mlp_forward(sw, x);
  }
}

// ---- correction of the SPE start (the second mode of the network).
// Inputs at free node i: the increments d0 = x0 - h1 (the SPE step from the
// previous solution), d1 = h1 - h2, d2 = h2 - h3, d3 = h3 - h4 and their
// means over the free graph neighbours, divided by s = RMS(d0); output o;
// direction d = s o; start z0 = x0 + alpha d with the step alpha that
// minimises the M-norm error along d (so a poor direction costs nothing).
// Increments, not the solutions themselves: the information is in how the
// solutions change, small against their size, and BF16 weights could not
// cancel raw inputs to that precision.

// s = sqrt(mean((x0 - h1)^2)) over the free nodes; 0 without SPE history
// (*nuse == 0, when x0 is h1).
__global__ void k_rms_diff(int n, const double* __restrict__ a, const double* __restrict__ b,
                           const int* __restrict__ nuse, double* s, double* partials, unsigned int* counter,
                           int max_blocks) {
  pdl_enter();
  const bool has = *nuse > 0;
  double v[1] = {0.0};
  if (has)
    for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const double d = a[i] - b[i];
      v[0] = fma(d, d, v[0]);
    }
  double tot[1];
  if (grid_sum<1>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) *s = sqrt(tot[0] / n);
}

__device__ __forceinline__ void spe_node_features(int i, const double* __restrict__ x0, const double* __restrict__ h1d,
                                                  const float* __restrict__ r0, const float* __restrict__ r1,
                                                  const float* __restrict__ r2, const float* __restrict__ r3,
                                                  const int32_t* __restrict__ adj_ptr,
                                                  const int32_t* __restrict__ adj_col,
                                                  const float* __restrict__ inv_deg, float inv_s, float x[8]) {
  x[0] = (float)(x0[i] - h1d[i]) * inv_s;
  x[1] = (r0[i] - r1[i]) * inv_s;
  x[2] = (r1[i] - r2[i]) * inv_s;
  x[3] = (r2[i] - r3[i]) * inv_s;
  float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
  const int e = adj_ptr[i + 1];
  for (int k = adj_ptr[i]; k < e; ++k) {
    const int j = adj_col[k];
    m0 += (float)(x0[j] - h1d[j]);
    m1 += r0[j] - r1[j];
    m2 += r1[j] - r2[j];
    m3 += r2[j] - r3[j];
  }
  const float w = inv_deg[i] * inv_s;
  x[4] = m0 * w;
  x[5] = m1 * w;
  x[6] = m2 * w;
  x[7] = m3 * w;
}

// Direction d = s MLP(features) for the solve g = stepcount[0] + j from its
// SPE start x0; d = 0 without SPE history (*nuse == 0), with fewer than four
// earlier solutions, or when s = 0.
__global__ void k_mlp_dir_spe(int nf, const double* __restrict__ x0, const double* __restrict__ h1d,
                              const float* __restrict__ ring, const long long* __restrict__ stepcount, int j,
                              const int* __restrict__ nuse, const int32_t* __restrict__ adj_ptr,
                              const int32_t* __restrict__ adj_col, const float* __restrict__ inv_deg,
                              const __nv_bfloat16* __restrict__ wb, const double* __restrict__ sd,
                              double* __restrict__ d) {
  pdl_enter();
  __shared__ float sw[kNP + 3];
  load_weights(wb, sw);
  const long long g = stepcount[0] + j;
  const double s = *nuse > 0 ? *sd : 0.0;
  const bool use = g >= 4 && s > 0.0;
  const float* hr[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) hr[l] = ring + (size_t)(((g - 1 - l) % 4 + 4) % 4) * nf;
  const float inv_s = use ? (float)(1.0 / s) : 0.f;
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    if (!use) {
      d[i] = 0.0;
      continue;
    }
    float x[8];
    spe_node_features((int)i, x0, h1d, hr[0], hr[1], hr[2], hr[3], adj_ptr, adj_col, inv_deg, inv_s, x);
    d[i] = s * (double)mlp_forward(sw, x);
  }
}

// Line search along d from x0: q = M d and alpha = d.r0 / d.q (0 when
// d.q <= 0), r0 = R - M x0 given as r, or formed here from R and x0 when r
// is null.  The last block writes alpha.
__global__ void k_dir_alpha(DevSell<double> M, int nf, const double* __restrict__ d, const double* __restrict__ r,
                            const double* __restrict__ R, const double* __restrict__ x0, double* __restrict__ q,
                            double* __restrict__ alpha, double* partials, unsigned int* counter, int max_blocks) {
  pdl_enter();
  double v[2] = {0.0, 0.0};
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const double qi = mat_row<double>(M, i, nf, d);
    q[i] = qi;
    const double ri = r ? r[i] : R[i] - mat_row<double>(M, i, nf, x0);
    v[0] = fma(d[i], ri, v[0]);
    v[1] = fma(d[i], qi, v[1]);
  }
  double tot[2];
  if (grid_sum<2>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0)
    *alpha = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
}

// The corrected CG start: x += alpha d, r -= alpha q, the first V-cycle input
// and ||r||^2; the last block redoes the stopping test of the start
// (||R||^2 already in sc->bnorm2) and counts the solve as started from the
// learned direction when alpha != 0.
template <typename T>
__global__ void k_dir_apply(int nf, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ d,
                            const double* __restrict__ q, const double* __restrict__ alpha,
                            const T* __restrict__ dinv0, T inv_theta0, T* __restrict__ b0, T* __restrict__ x0v,
                            T* __restrict__ d0v, PcgScalars* sc, double* partials, unsigned int* counter,
                            int max_blocks, double tol2, int maxit, cudaGraphConditionalHandle h, int use_handle,
                            double* relres_out, int* kept_out) {
  pdl_enter();
  const double a = *alpha;
  double v[1] = {0.0};
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const double xi = fma(a, d[i], x[i]);
    const double ri = fma(-a, q[i], r[i]);
    x[i] = xi;
    r[i] = ri;
    const T bi = vc_in<T>(ri);
    b0[i] = bi;
    const T dd = dinv0[i] * bi * inv_theta0;
    x0v[i] = dd;
    d0v[i] = dd;
    v[0] = fma(ri, ri, v[0]);
  }
  double tot[1];
  if (grid_sum<1>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    const double b2 = sc->bnorm2;
    sc->rnorm2 = tot[0];
    const int zero = b2 == 0.0;
    const int go = !zero && tot[0] > tol2 * b2 && maxit > 0;
    sc->conv = !go;
    if (use_handle) cudaGraphSetConditional(h, go ? 1u : 0u);
    if (relres_out) *relres_out = zero ? 0.0 : sqrt(tot[0] / b2);
    if (kept_out) *kept_out = a != 0.0;
  }
}

// z0 = x0 + alpha d (the corrected start alone).
__global__ void k_axpy_alpha(int nf, const double* __restrict__ x0, const double* __restrict__ d,
                             const double* __restrict__ alpha, double* __restrict__ z0) {
  const int64_t i = gtid();
  if (i < nf) z0[i] = fma(*alpha, d[i], x0[i]);
}

// Per recorded solve k >= 1 of the SPE-correction mode: the input scale
// s_k = RMS(d0) with d0 = x0_k - z_{k-1} = (z_k - z_{k-1}) - e_k, and the
// target scale RMS(e_k), from the stored solutions z and distances
// e = z - x0 (block k; 0 for k = 0).
__global__ void k_store_rms_spe(int nf, const float* __restrict__ store, const float* __restrict__ store_e,
                                float* __restrict__ rms, float* __restrict__ rms_e) {
  const int k = blockIdx.x;
  if (k == 0) {
    if (threadIdx.x == 0) rms[0] = rms_e[0] = 0.f;
    return;
  }
  const float* z = store + (size_t)k * nf;
  const float* zp = store + (size_t)(k - 1) * nf;
  const float* e = store_e + (size_t)k * nf;
  double acc[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < nf; i += blockDim.x) {
    const double d = ((double)z[i] - (double)zp[i]) - (double)e[i];
    acc[0] += d * d;
    acc[1] += (double)e[i] * (double)e[i];
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    rms[k] = (float)sqrt(acc[0] / nf);
    rms_e[k] = (float)sqrt(acc[1] / nf);
  }
}

// Per-block RMS of each recorded solution: rms[k] = sqrt(mean(store[k]^2)).
__global__ void k_store_rms(int nf, const float* __restrict__ store, float* __restrict__ rms) {
  const float* v = store + (size_t)blockIdx.x * nf;
  double acc[1] = {0.0};
  for (int i = threadIdx.x; i < nf; i += blockDim.x) acc[0] += (double)v[i] * v[i];
  block_sum<1>(acc);
  if (threadIdx.x == 0) rms[blockIdx.x] = (float)sqrt(acc[0] / nf);
}

// One training mini-batch: forward, MSE loss, backward; per-block sums of
// the parameter gradients are added to grad.  Samples are either drawn
// (solve k in [4, count), node i) from splitmix64 stream `seed`, values
// 2 (step B + b) and 2 (step B + b) + 1, or given as X (B x 8) / T (B).
// With store_e (the SPE-correction mode) a drawn sample has the increment
// inputs of k_mlp_dir_spe (scale s_k = rms[k]), x0_k = z_k - e_k, and target
// e_k / RMS(e_k) (rms_e[k]); otherwise the previous-solution mode's inputs
// and target.
__global__ void __launch_bounds__(kTrainBlock) k_mlp_train(
    int nf, const float* __restrict__ store, const float* __restrict__ rms, int count,
    const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj_col,
    const float* __restrict__ inv_deg, const __nv_bfloat16* __restrict__ wb, float* __restrict__ grad,
    float* __restrict__ loss, unsigned long long seed, long long step, int B,
    const float* __restrict__ Xin, const float* __restrict__ Tin, const float* __restrict__ store_e,
    const float* __restrict__ rms_e) {
  extern __shared__ float sm[];
  float* sw = sm;
  const int S = kTrainBlock + 1;  // padded stride of the per-sample arrays
  float* sx = sm + kNP + 3;       // 8 x S
  float* sg1 = sx + 8 * S;        // 32 x S
  float* sd1 = sg1 + 32 * S;      // 32 x S  (dL/da1)
  float* sd2 = sd1 + 32 * S;      // 32 x S  (dL/da2)
  float* sg2 = sd2 + 32 * S;      // 32 x S  (g2 * dL/do)
  float* sdo = sg2 + 32 * S;      // S       (dL/do)
  load_weights(wb, sw);
  const int tl = threadIdx.x;
  const int b = blockIdx.x * blockDim.x + tl;
  float x[8], t = 0.f;
  bool valid = b < B;
  if (valid) {
    if (Xin) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = Xin[(size_t)b * 8 + k];
      t = Tin[b];
    } else {
      const uint64_t ctr = 2ull * ((uint64_t)step * (uint64_t)B + (uint64_t)b);
      const int k = 4 + (int)(smix64(seed, ctr) % (uint64_t)(count - 4));
      const int i = (int)(smix64(seed, ctr + 1) % (uint64_t)nf);
      const float s_h = store_e ? rms[k] : rms[k - 1];
      if (store_e && s_h > 0.f && rms_e[k] > 0.f) {
        // z_k, z_{k-1} .. z_{k-4}: d0 = (z_k - z_{k-1}) - e_k, d_l = z_{k-l} - z_{k-l-1}
        const float* z[5];  // z_k, z_{k-1}, ..., z_{k-4}
#pragma unroll
        for (int l = 0; l < 5; ++l) z[l] = store + (size_t)(k - l) * nf;
        const float* ek = store_e + (size_t)k * nf;
        const float inv_s = 1.0f / s_h;
        float dd[4], mm[4] = {0.f, 0.f, 0.f, 0.f};
        dd[0] = (z[0][i] - z[1][i]) - ek[i];
#pragma unroll
        for (int l = 1; l < 4; ++l) dd[l] = z[l][i] - z[l + 1][i];
        const int e = adj_ptr[i + 1];
        for (int q = adj_ptr[i]; q < e; ++q) {
          const int jn = adj_col[q];
          mm[0] += (z[0][jn] - z[1][jn]) - ek[jn];
#pragma unroll
          for (int l = 1; l < 4; ++l) mm[l] += z[l][jn] - z[l + 1][jn];
        }
        const float w = inv_deg[i] * inv_s;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          x[l] = dd[l] * inv_s;
          x[4 + l] = mm[l] * w;
        }
        t = ek[i] / rms_e[k];
      } else if (!store_e && s_h > 0.f) {
        const float* h0 = store + (size_t)(k - 1) * nf;
        node_features(i, h0, h0 - nf, h0 - 2 * (size_t)nf, h0 - 3 * (size_t)nf, adj_ptr, adj_col, inv_deg,
                      1.0f / s_h, x);
        t = (store[(size_t)k * nf + i] - h0[i]) / s_h;
      } else {
        valid = false;
      }
    }
  }
  if (!valid)
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 0.f;
  // forward
  const float* W1 = sw;
  const float* b1 = sw + 256;
  const float* W2 = sw + 288;
  const float* b2 = sw + 1312;
  const float* w3 = sw + 1344;
  float a1[32], g1[32], d2[32];
#pragma unroll
  for (int o = 0; o < 32; ++o) {
    float a = b1[o];
#pragma unroll
    for (int k = 0; k < 8; ++k) a = fmaf(W1[o * 8 + k], x[k], a);
    a1[o] = a;
    g1[o] = gelu_f(a);
  }
  float out = sw[1376];
#pragma unroll 4
  for (int o = 0; o < 32; ++o) {
    float a = b2[o];
#pragma unroll
    for (int k = 0; k < 32; ++k) a = fmaf(W2[o * 32 + k], g1[k], a);
    const float g2 = gelu_f(a);
    out = fmaf(w3[o], g2, out);
    d2[o] = a;   // a2 kept for the backward pass
    sg2[o * S + tl] = g2;
  }
  const float e = valid ? out - t : 0.f;
  const float dout = 2.f * e / (float)B;
  if (valid) atomicAdd(loss, e * e / (float)B);
  // backward
#pragma unroll
  for (int o = 0; o < 32; ++o) {
    const float da2 = dout * w3[o] * gelu_df(d2[o]);
    d2[o] = da2;
    sd2[o * S + tl] = da2;
    sg2[o * S + tl] *= dout;
  }
#pragma unroll 4
  for (int k = 0; k < 32; ++k) {
    float dg = 0.f;
#pragma unroll
    for (int o = 0; o < 32; ++o) dg = fmaf(W2[o * 32 + k], d2[o], dg);
    sd1[k * S + tl] = dg * gelu_df(a1[k]);
    sg1[k * S + tl] = g1[k];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) sx[k * S + tl] = x[k];
  sdo[tl] = dout;
  __syncthreads();
  // per-block reduction over the samples: one parameter per thread pass
  for (int p = tl; p < kNP; p += blockDim.x) {
    const float *ua, *ub;  // gradient = sum_b ua[b] * (ub ? ub[b] : 1)
    if (p < 256) {
      ua = sd1 + (p / 8) * S;
      ub = sx + (p % 8) * S;
    } else if (p < 288) {
      ua = sd1 + (p - 256) * S;
      ub = nullptr;
    } else if (p < 1312) {
      ua = sd2 + ((p - 288) / 32) * S;
      ub = sg1 + ((p - 288) % 32) * S;
    } else if (p < 1344) {
      ua = sd2 + (p - 1312) * S;
      ub = nullptr;
    } else if (p < 1376) {
      ua = sg2 + (p - 1344) * S;
      ub = nullptr;
    } else {
      ua = sdo;
      ub = nullptr;
    }
    float acc = 0.f;
    if (ub)
      for (int q = 0; q < (int)blockDim.x; ++q) acc = fmaf(ua[q], ub[q], acc);
    else
      for (int q = 0; q < (int)blockDim.x; ++q) acc += ua[q];
    atomicAdd(grad + p, acc);
  }
}

// Adam on the FP32 master parameters (Kingma & Ba 2015), then the BF16
// copy; the gradient accumulator is cleared.
__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       float* __restrict__ grad, __nv_bfloat16* __restrict__ wb, float lr, float bc1,
                       float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNP) return;
  const float g = grad[p];
  const float mm = 0.9f * m[p] + 0.1f * g;
  const float vv = 0.999f * v[p] + 0.001f * g * g;
  m[p] = mm;
  v[p] = vv;
  const float th = theta[p] - lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
  theta[p] = th;
  wb[p] = __float2bfloat16_rn(th);
  grad[p] = 0.f;
}

__global__ void k_to_bf16(int n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) b[p] = __float2bfloat16_rn(a[p]);
}

// History ring slot / recorded copy of one solution (FP32).
__global__ void k_push_solution(int nf, const double* __restrict__ F, float* __restrict__ dst) {
  const int64_t i = gtid();
  if (i < nf) dst[i] = (float)F[i];
}

}  // namespace eqs
