// Ensemble of kEnsW = 4 trajectories on one mesh (the same M, AMG hierarchy
// and materials; each column has its own drive amplitude).  Every stage
// solves its four right-hand sides together: the multiple right-hand-side
// problem of Section IV with the constant M read once per four columns.
//
// Layout: every ensemble vector is row-interleaved, element (i, c) at
// 4 i + c, so a row's four columns are one 16-byte (FP32) or 32-byte (FP64)
// load and the matrix entry of a row is read once for all four columns
// (SpMM).  Mixed precision only: FP32 element kernel and V-cycle, FP64
// recurrence, CG residuals and dot products; the CG operator product uses
// the split-M FP32-pair form (df_acc); the coarsest level applies the dense
// inverse in split FP32 parts with FP32-pair sums.
//
// CG runs per column with its own alpha, beta and convergence flag; a
// converged column is frozen (its x and r no longer change) while the
// others iterate.  The loop runs while any column is active.
#pragma once

#include "spe_kernels.cuh"

namespace eqs {

constexpr int kEnsW = 4;
constexpr int kEnsSpe = 6;  // SPE history length of the ensemble (48 sums per Gram pass)

// ------------------------------------------------------------ float4 ops
__device__ __forceinline__ float4 operator+(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 operator-(float4 a, float4 b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 operator*(float a, float4 b) {
  return make_float4(a * b.x, a * b.y, a * b.z, a * b.w);
}
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 acc) {
  return make_float4(fmaf(a, x.x, acc.x), fmaf(a, x.y, acc.y), fmaf(a, x.z, acc.z), fmaf(a, x.w, acc.w));
}
__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 shfl_xor4(float4 v, int o) {
  return make_float4(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o),
                     __shfl_xor_sync(0xffffffffu, v.z, o), __shfl_xor_sync(0xffffffffu, v.w, o));
}
__device__ __forceinline__ float comp(const float4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

template <bool ADD>
__device__ __forceinline__ float4 xv4(const float4* __restrict__ x, const float4* __restrict__ xadd, int j) {
  return ADD ? __ldg(x + j) + __ldg(xadd + j) : __ldg(x + j);
}

// (A X)_row for four interleaved columns (A in FP32, any of the three
// layouts); same lane conventions as mat_row_impl.
template <bool ADD>
__device__ __forceinline__ float4 mat_row4_impl(const DevSell<float>& A, int64_t tid, int n,
                                                const float4* __restrict__ x, const float4* __restrict__ xadd) {
  const int row = (int)(tid >> A.logG);
  float4 acc = zero4();
  if (A.G == 0) {  // DIA, chunks of loads issued before use (as mat_row_impl)
    if (row >= n) return acc;
    const float* __restrict__ v = A.val + row;
    float4 acc1 = zero4();
    constexpr int C = kDiaChunk / 2;
    for (int d0 = 0; d0 < A.ndiag; d0 += C) {
      float a[C];
      float4 xs[C];
#pragma unroll
      for (int u = 0; u < C; ++u) {
        const int d = d0 + u;
        const int j = row + A.off[d < kMaxDiag ? d : 0];
        const bool ok = d < A.ndiag && (unsigned)j < (unsigned)A.n_cols;
        a[u] = ok ? __ldg(v + (int64_t)d * n) : 0.f;
        xs[u] = ok ? xv4<ADD>(x, xadd, j) : zero4();
      }
#pragma unroll
      for (int u = 0; u < C; u += 2) {
        acc = fma4(a[u], xs[u], acc);
        acc1 = fma4(a[u + 1], xs[u + 1], acc1);
      }
    }
    return acc + acc1;
  }
  if (A.G == 1) {  // SELL-32
    if (row >= n) return acc;
    const int s = row >> 5, lane = row & 31;
    const int64_t end = A.slice_ptr[s + 1];
    for (int64_t k = A.slice_ptr[s] + lane; k < end; k += 32 * 4) {
      int c[4];
      float a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t kk = k + 32 * u;
        c[u] = kk < end ? __ldg(A.col + kk) : 0;
        a[u] = kk < end ? __ldg(A.val + kk) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = fma4(a[u], xv4<ADD>(x, xadd, c[u]), acc);
    }
    return acc;
  }
  const int g = (int)(tid & (A.G - 1));
  int64_t k = 0, end = 0;
  if (row < n) {
    k = A.slice_ptr[row] + g;
    end = A.slice_ptr[row + 1];
  }
  // four entries per lane and round: the float4 gathers of long rows (AMG
  // coarse operators, restriction) are latency bound
  for (; k < end; k += (int64_t)A.G * 4) {
    int c[4];
    float a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t kk = k + (int64_t)A.G * u;
      c[u] = kk < end ? __ldg(A.col + kk) : 0;
      a[u] = kk < end ? __ldg(A.val + kk) : 0.f;
    }
    float4 xs[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) xs[u] = xv4<ADD>(x, xadd, c[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) acc = fma4(a[u], xs[u], acc);
  }
  for (int o = A.G >> 1; o > 0; o >>= 1) acc = acc + shfl_xor4(acc, o);
  return acc;
}

__device__ __forceinline__ float4 mat_row4(const DevSell<float>& A, int64_t tid, int n, const float4* x) {
  return mat_row4_impl<false>(A, tid, n, x, nullptr);
}

// ------------------------------------------------------- V-cycle (4 cols)
__global__ void __launch_bounds__(kBlock, 4)
k4_cheb_step(DevSell<float> A, int n, const float4* r_in, const float4* __restrict__ d_in,
             const float* __restrict__ dinv, float c1, float c2, float4* r_out, float4* __restrict__ d_out,
             float4* __restrict__ x, int add_pending) {
  pdl_enter();
  EQS_ROWS2(A, n, {
    const float4 a0 = mat_row4(A, t0, n, d_in);
    const float4 a1 = mat_row4(A, t1, n, d_in);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = h ? t1 : t0;
      if (!row_leader(A, t, n)) continue;
      const int i = (int)(t >> A.logG);
      const float4 di = d_in[i];
      const float4 r = r_in[i] - (h ? a1 : a0);
      const float4 dn = c1 * di + (c2 * dinv[i]) * r;
      r_out[i] = r;
      d_out[i] = dn;
      x[i] = x[i] + (add_pending ? dn + di : dn);
    }
  })
}

__global__ void __launch_bounds__(kBlock, 4) k4_resid_update(DevSell<float> A, int n, float4* r,
                                                             const float4* __restrict__ d) {
  pdl_enter();
  EQS_ROWS2(A, n, {
    const float4 a0 = mat_row4(A, t0, n, d);
    const float4 a1 = mat_row4(A, t1, n, d);
    if (row_leader(A, t0, n)) r[t0 >> A.logG] = r[t0 >> A.logG] - a0;
    if (row_leader(A, t1, n)) r[t1 >> A.logG] = r[t1 >> A.logG] - a1;
  })
}

__global__ void __launch_bounds__(kBlock, 4) k4_resid(DevSell<float> A, int n, const float4* __restrict__ b,
                                                      const float4* __restrict__ x, float4* __restrict__ out) {
  pdl_enter();
  EQS_ROWS2(A, n, {
    const float4 a0 = mat_row4(A, t0, n, x);
    const float4 a1 = mat_row4(A, t1, n, x);
    if (row_leader(A, t0, n)) out[t0 >> A.logG] = b[t0 >> A.logG] - a0;
    if (row_leader(A, t1, n)) out[t1 >> A.logG] = b[t1 >> A.logG] - a1;
  })
}

__global__ void __launch_bounds__(kBlock, 4) k4_restrict(DevSell<float> R, int nc, const float4* __restrict__ rf,
                                                         float4* __restrict__ bc, const float* __restrict__ dinv_c,
                                                         float inv_theta_c, float4* __restrict__ xc,
                                                         float4* __restrict__ dc, int first_step) {
  pdl_enter();
  EQS_ROWS2(R, nc, {
    const float4 b0 = mat_row4(R, t0, nc, rf);
    const float4 b1 = mat_row4(R, t1, nc, rf);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = h ? t1 : t0;
      if (!row_leader(R, t, nc)) continue;
      const int i = (int)(t >> R.logG);
      const float4 b = h ? b1 : b0;
      bc[i] = b;
      if (first_step) {
        const float4 d = (dinv_c[i] * inv_theta_c) * b;
        xc[i] = d;
        if (dc) dc[i] = d;  // first Chebyshev direction (degree >= 2)
      }
    }
  })
}

__global__ void __launch_bounds__(kBlock, 4) k4_prolong(DevSell<float> P, int nf, const float4* __restrict__ xc,
                                                        const float4* __restrict__ dc, float4* __restrict__ xf) {
  pdl_enter();
  EQS_ROWS2(P, nf, {
    const float4 p0 = dc ? mat_row4_impl<true>(P, t0, nf, xc, dc) : mat_row4(P, t0, nf, xc);
    const float4 p1 = dc ? mat_row4_impl<true>(P, t1, nf, xc, dc) : mat_row4(P, t1, nf, xc);
    if (row_leader(P, t0, nf)) xf[t0 >> P.logG] = xf[t0 >> P.logG] + p0;
    if (row_leader(P, t1, nf)) xf[t1 >> P.logG] = xf[t1 >> P.logG] + p1;
  })
}

// First post-smoothing step: d = D^-1 (b - A x) / theta into d_out, or with
// write_iterate (degree-1 smoothing, nothing follows) the smoothed iterate
// x + d, so the prolongation above gathers one vector instead of two.
__global__ void __launch_bounds__(kBlock, 4) k4_post_first(DevSell<float> A, int n, const float4* __restrict__ b,
                                                           const float4* __restrict__ x, const float* __restrict__ dinv,
                                                           float inv_theta, float4* __restrict__ r_out,
                                                           float4* __restrict__ d_out, int write_iterate) {
  pdl_enter();
  EQS_ROWS2(A, n, {
    const float4 a0 = mat_row4(A, t0, n, x);
    const float4 a1 = mat_row4(A, t1, n, x);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = h ? t1 : t0;
      if (!row_leader(A, t, n)) continue;
      const int i = (int)(t >> A.logG);
      const float4 r = b[i] - (h ? a1 : a0);
      if (r_out) r_out[i] = r;  // read by the Chebyshev steps of degree >= 2
      const float4 d = (dinv[i] * inv_theta) * r;
      d_out[i] = write_iterate ? x[i] + d : d;
    }
  })
}

__global__ void k4_axpy1(int n, float4* __restrict__ x, const float4* __restrict__ d) {
  pdl_enter();
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = x[i] + d[i];
}

// Error-free sum of two FP32 pairs into (S, s).
__device__ __forceinline__ void df_add(float& S, float& s, float S2, float s2) {
  const float S1 = __fadd_rn(S, S2);
  const float bv = __fsub_rn(S1, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(S1, bv)), __fsub_rn(S2, bv));
  S = S1;
  s = __fadd_rn(s, __fadd_rn(s2, err));
}

// Coarsest level, W interleaved columns: x = A_c^-1 b with the dense inverse
// held as two FP32 parts (hi + lo) and FP32-pair row sums (df_acc), one warp
// per row; b (FP32) is staged once per block in shared memory (W = 4: one
// 16-byte element per row, conflict-free).
template <int W>
__global__ void k_coarse_solve_df(int n, const float* __restrict__ ihi, const float* __restrict__ ilo,
                                  const float* __restrict__ b, float* __restrict__ x) {
  extern __shared__ float4 sb4[];
  float* sbf = reinterpret_cast<float*>(sb4);
  pdl_enter();
  for (int j = threadIdx.x; j < n * W; j += blockDim.x) sbf[j] = b[j];
  __syncthreads();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const float* __restrict__ rh = ihi + (int64_t)warp * n;
  const float* __restrict__ rl = ilo + (int64_t)warp * n;
  float S[W], s[W];
#pragma unroll
  for (int c = 0; c < W; ++c) S[c] = s[c] = 0.f;
  for (int j = lane; j < n; j += 32) {
    const float ah = __ldg(rh + j), al = __ldg(rl + j);
    if constexpr (W == 4) {
      const float4 bj = sb4[j];
      df_acc(S[0], s[0], ah, al, bj.x);
      df_acc(S[1], s[1], ah, al, bj.y);
      df_acc(S[2], s[2], ah, al, bj.z);
      df_acc(S[3], s[3], ah, al, bj.w);
    } else {
#pragma unroll
      for (int c = 0; c < W; ++c) df_acc(S[c], s[c], ah, al, sbf[j * W + c]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < W; ++c) {
      const float S2 = __shfl_xor_sync(0xffffffffu, S[c], o);
      const float s2 = __shfl_xor_sync(0xffffffffu, s[c], o);
      df_add(S[c], s[c], S2, s2);
    }
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < W; ++c) x[(int64_t)warp * W + c] = (float)((double)S[c] + (double)s[c]);
}

// Coarsest level, W interleaved columns: x = A_c^-1 b with the FP32 rounding
// of the dense inverse and FP32 row sums (the V-cycle around it is FP32, so
// the FP32-pair form above buys no accuracy the preconditioner keeps).  Rows
// are padded to ld floats (a multiple of 4, zeros beyond n) so that every
// row starts on a 16-byte boundary; one warp per row, b staged once per
// block in shared memory, zero-padded to ld.  W = 1 reads the row as float4
// (four columns per load, b as the matching float4); W = 4 reads one
// column per lane and load (b rows are one float4 each: conflict-free).
template <int W>
__global__ void k_coarse_solve32(int n, int ld, const float* __restrict__ inv, const float* __restrict__ b,
                                 float* __restrict__ x) {
  static_assert(W == 1 || W == 4, "one or four interleaved columns");
  extern __shared__ float4 sb4[];
  float* sbf = reinterpret_cast<float*>(sb4);
  pdl_enter();
  for (int j = threadIdx.x; j < ld * W; j += blockDim.x) sbf[j] = j < n * W ? b[j] : 0.f;
  __syncthreads();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  float S[W];
#pragma unroll
  for (int c = 0; c < W; ++c) S[c] = 0.f;
  // The row's loads are issued in batches of U per lane before any of them
  // is used, so that each warp keeps U loads in flight (the kernel is bound
  // by load latency: a few warps per SM, one row each).
  if constexpr (W == 1) {
    constexpr int U = 16;
    const float4* __restrict__ r4 = reinterpret_cast<const float4*>(inv + (int64_t)warp * ld);
    const int n4 = ld >> 2;
    int q = lane;
    for (; q + 32 * (U - 1) < n4; q += 32 * U) {  // full batches
      float4 a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) a[u] = __ldg(r4 + q + 32 * u);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float4 bq = sb4[q + 32 * u];
        S[0] = fmaf(a[u].x, bq.x, S[0]);
        S[0] = fmaf(a[u].y, bq.y, S[0]);
        S[0] = fmaf(a[u].z, bq.z, S[0]);
        S[0] = fmaf(a[u].w, bq.w, S[0]);
      }
    }
    for (; q < n4; q += 32) {  // the rest of the row
      const float4 a = __ldg(r4 + q);
      const float4 bq = sb4[q];
      S[0] = fmaf(a.x, bq.x, S[0]);
      S[0] = fmaf(a.y, bq.y, S[0]);
      S[0] = fmaf(a.z, bq.z, S[0]);
      S[0] = fmaf(a.w, bq.w, S[0]);
    }
  } else {
    constexpr int U = 16;
    const float* __restrict__ r = inv + (int64_t)warp * ld;
    int j = lane;
    for (; j + 32 * (U - 1) < n; j += 32 * U) {  // full batches
      float a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) a[u] = __ldg(r + j + 32 * u);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float4 bj = sb4[j + 32 * u];
        S[0] = fmaf(a[u], bj.x, S[0]);
        S[1] = fmaf(a[u], bj.y, S[1]);
        S[2] = fmaf(a[u], bj.z, S[2]);
        S[3] = fmaf(a[u], bj.w, S[3]);
      }
    }
    for (; j < n; j += 32) {  // the rest of the row
      const float a = __ldg(r + j);
      const float4 bj = sb4[j];
      S[0] = fmaf(a, bj.x, S[0]);
      S[1] = fmaf(a, bj.y, S[1]);
      S[2] = fmaf(a, bj.z, S[2]);
      S[3] = fmaf(a, bj.w, S[3]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < W; ++c) S[c] += __shfl_xor_sync(0xffffffffu, S[c], o);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < W; ++c) x[(int64_t)warp * W + c] = S[c];
}

// Interleave four column-major FP64 columns (column c at src + c n) into
// rows of four, and back.
__global__ void k4_interleave(int n, const double* __restrict__ src, double4_32a* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double4_32a v;
  v.x = src[i];
  v.y = src[(int64_t)n + i];
  v.z = src[2 * (int64_t)n + i];
  v.w = src[3 * (int64_t)n + i];
  dst[i] = v;
}

__global__ void k4_deinterleave(int n, const double4_32a* __restrict__ src, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double4_32a v = src[i];
  dst[i] = v.x;
  dst[(int64_t)n + i] = v.y;
  dst[2 * (int64_t)n + i] = v.z;
  dst[3 * (int64_t)n + i] = v.w;
}

// ------------------------------------------------------------- CG (4 cols)
// Per-column solve state; conv = 1 freezes the column.
struct EnsScalars {
  double bnorm2[kEnsW], rnorm2[kEnsW], rz[kEnsW], rz_old[kEnsW], alpha[kEnsW], beta[kEnsW];
  int it[kEnsW], conv[kEnsW];
  int pass;  // CG loop passes of the current solve
};

__device__ __forceinline__ float4 to_f4(const double4_32a& v) {
  return make_float4((float)v.x, (float)v.y, (float)v.z, (float)v.w);
}
__device__ __forceinline__ double dc4(const double4_32a& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set4(double4_32a& v, int c, double a) {
  if (c == 0) v.x = a; else if (c == 1) v.y = a; else if (c == 2) v.z = a; else v.w = a;
}

// (M X)_row in FP64 for four interleaved FP64 columns (one thread per row).
__device__ __forceinline__ double4_32a mat_row_d4(const DevSell<double>& A, int64_t row, int n,
                                                  const double4_32a* __restrict__ x) {
  double4_32a acc = {0.0, 0.0, 0.0, 0.0};
  if (row >= n) return acc;
  if (A.G == 0) {
#pragma unroll 5
    for (int d = 0; d < A.ndiag; ++d) {
      const int j = (int)row + A.off[d];
      if ((unsigned)j >= (unsigned)A.n_cols) continue;
      const double a = __ldg(A.val + (int64_t)d * n + row);
      const double4_32a v = x[j];
      acc.x = fma(a, v.x, acc.x);
      acc.y = fma(a, v.y, acc.y);
      acc.z = fma(a, v.z, acc.z);
      acc.w = fma(a, v.w, acc.w);
    }
    return acc;
  }
  const int64_t sl = row >> 5, lane = row & 31;
  const int64_t end = A.slice_ptr[sl + 1];
  for (int64_t k = A.slice_ptr[sl] + lane; k < end; k += 32) {
    const double a = __ldg(A.val + k);
    const double4_32a v = x[__ldg(A.col + k)];
    acc.x = fma(a, v.x, acc.x);
    acc.y = fma(a, v.y, acc.y);
    acc.z = fma(a, v.z, acc.z);
    acc.w = fma(a, v.w, acc.w);
  }
  return acc;
}

// The V-cycle input of a row from its four FP64 residuals.
__device__ __forceinline__ float4 vc_f4(const double4_32a& v) {
  return make_float4(vc_narrow(v.x), vc_narrow(v.y), vc_narrow(v.z), vc_narrow(v.w));
}

__device__ __forceinline__ void vc_input4(int64_t i, const double4_32a& r, const float* __restrict__ dinv0,
                                          float inv_theta0, float4* __restrict__ b0, float4* __restrict__ x0,
                                          float4* __restrict__ d0) {
  const float4 bi = vc_f4(r);
  b0[i] = bi;
  const float4 d = (dinv0[i] * inv_theta0) * bi;
  x0[i] = d;
  if (d0) d0[i] = d;  // the first Chebyshev direction (degree >= 2 only)
}

// Last block of a CG start: per-column norms (tot: ||R_c||^2, then ||r_c||^2),
// flags and the loop condition (any column active).
__device__ __forceinline__ void ens_init_tail(const double* tot, EnsScalars* sc, double tol2, int maxit,
                                              cudaGraphConditionalHandle h, int use_handle, int* iters_out,
                                              double* relres_out, int* zero_out) {
  int go = 0;
  for (int c = 0; c < kEnsW; ++c) {
    sc->bnorm2[c] = tot[c];
    sc->rnorm2[c] = tot[kEnsW + c];
    sc->it[c] = 0;
    sc->rz_old[c] = 0.0;
    sc->beta[c] = 0.0;
    sc->alpha[c] = 0.0;
    const int zero = tot[c] == 0.0;
    const int gc = !zero && tot[kEnsW + c] > tol2 * tot[c] && maxit > 0;
    sc->conv[c] = !gc;
    go |= gc;
    if (iters_out) iters_out[c] = 0;
    if (relres_out) relres_out[c] = zero ? 0.0 : sqrt(tot[kEnsW + c] / tot[c]);
    if (zero_out) zero_out[c] = zero;
  }
  sc->pass = 0;
  if (use_handle) cudaGraphSetConditional(h, go ? 1u : 0u);
}

// r = R - M x for the four columns (FP64), norms of R and r per column, the
// first V-cycle input; the last block sets the per-column flags and the
// loop condition (any column active).
__global__ void k4_pcg_init(DevSell<double> M, int n, const double4_32a* __restrict__ R,
                            const double4_32a* __restrict__ x, double4_32a* __restrict__ r,
                            const float* __restrict__ dinv0, float inv_theta0, float4* __restrict__ b0,
                            float4* __restrict__ x0, float4* __restrict__ d0, EnsScalars* sc,
                            double* partials, unsigned int* counter, int max_blocks, double tol2, int maxit,
                            cudaGraphConditionalHandle h, int use_handle, int* iters_out,
                            double* relres_out, int* zero_out) {
  pdl_enter();
  double v[2 * kEnsW];
#pragma unroll
  for (int k = 0; k < 2 * kEnsW; ++k) v[k] = 0.0;
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double4_32a Ri = R[i];
    const double4_32a mx = mat_row_d4(M, i, n, x);
    double4_32a ri;
    ri.x = Ri.x - mx.x;
    ri.y = Ri.y - mx.y;
    ri.z = Ri.z - mx.z;
    ri.w = Ri.w - mx.w;
    r[i] = ri;
    vc_input4(i, ri, dinv0, inv_theta0, b0, x0, d0);
#pragma unroll
    for (int c = 0; c < kEnsW; ++c) {
      v[c] = fma(dc4(Ri, c), dc4(Ri, c), v[c]);
      v[kEnsW + c] = fma(dc4(ri, c), dc4(ri, c), v[kEnsW + c]);
    }
  }
  double tot[2 * kEnsW];
  if (grid_sum<2 * kEnsW>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0)
    ens_init_tail(tot, sc, tol2, maxit, h, use_handle, iters_out, relres_out, zero_out);
}

// Last block of the dot-product pass: beta per active column
// (Polak-Ribiere or Fletcher-Reeves) from r.z (tot[0..4)) and q.z, q the
// operator product of the last update (r_new = r_old - alpha q), so the
// Polak-Ribiere numerator z.(r_new - r_old) is -alpha z.q: no copy of the
// previous residual is kept.
__device__ __forceinline__ void ens_beta_tail(const double* tot, EnsScalars* sc, int flexible) {
  for (int c = 0; c < kEnsW; ++c) {
    if (sc->conv[c]) {
      sc->beta[c] = 0.0;
      continue;
    }
    const double rz = tot[c];
    double beta = 0.0;
    if (sc->it[c] > 0 && sc->rz_old[c] != 0.0)
      beta = flexible ? -sc->alpha[c] * tot[kEnsW + c] / sc->rz_old[c] : rz / sc->rz_old[c];
    sc->beta[c] = beta;
    sc->rz[c] = rz;
    sc->rz_old[c] = rz;
  }
}

// z = V-cycle output (+ pending direction) kept in FP32; r.z and q.z per
// column; the last block forms beta per active column (Polak-Ribiere or
// Fletcher-Reeves).
__global__ void k4_pcg_dots(int n, const double4_32a* __restrict__ r, const double4_32a* __restrict__ q,
                            const float4* __restrict__ z, const float4* __restrict__ zpend,
                            float4* __restrict__ z32, EnsScalars* sc, double* partials, unsigned int* counter,
                            int max_blocks, int flexible) {
  pdl_enter();
  double v[2 * kEnsW];
#pragma unroll
  for (int k = 0; k < 2 * kEnsW; ++k) v[k] = 0.0;
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 zt = zpend ? z[i] + zpend[i] : z[i];
    z32[i] = zt;
    const double4_32a ri = r[i], qi = q[i];
#pragma unroll
    for (int c = 0; c < kEnsW; ++c) {
      const double zc = f2d(comp(zt, c));
      v[c] = fma(dc4(ri, c), zc, v[c]);
      v[kEnsW + c] = fma(dc4(qi, c), zc, v[kEnsW + c]);
    }
  }
  double tot[2 * kEnsW];
  if (grid_sum<2 * kEnsW>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0)
    ens_beta_tail(tot, sc, flexible);
}

// Level-0 post-smoothing step of a degree-1 V-cycle fused with the dot
// products (as k_post_first_dots, four columns): z = x + D^-1 (b - A x)/theta.
__global__ void __launch_bounds__(kBlock, 4)
k4_post_first_dots(DevSell<float> A, int n, const float4* __restrict__ b, const float4* __restrict__ x,
                   const float* __restrict__ dinv, float inv_theta, const double4_32a* __restrict__ rcg,
                   const double4_32a* __restrict__ q, float4* __restrict__ z32, EnsScalars* sc,
                   double* partials, unsigned int* counter, int max_blocks, int flexible) {
  pdl_enter();
  double v[2 * kEnsW];
#pragma unroll
  for (int k = 0; k < 2 * kEnsW; ++k) v[k] = 0.0;
  EQS_ROWS2(A, n, {
    const float4 a0 = mat_row4(A, t0, n, x);
    const float4 a1 = mat_row4(A, t1, n, x);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = h ? t1 : t0;
      if (!row_leader(A, t, n)) continue;
      const int i = (int)(t >> A.logG);
      const float4 r = b[i] - (h ? a1 : a0);
      const float4 zt = x[i] + (dinv[i] * inv_theta) * r;
      z32[i] = zt;
      const double4_32a ri = rcg[i];
      const double4_32a qi = q[i];
#pragma unroll
      for (int c = 0; c < kEnsW; ++c) {
        const double zc = f2d(comp(zt, c));
        v[c] = fma(dc4(ri, c), zc, v[c]);
        v[kEnsW + c] = fma(dc4(qi, c), zc, v[kEnsW + c]);
      }
    }
  })
  double tot[2 * kEnsW];
  if (grid_sum<2 * kEnsW>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0)
    ens_beta_tail(tot, sc, flexible);
}

// q = M z + beta q, p = z + beta p per active column (split-M product of the
// FP32 z: four columns per matrix entry), p.q and alpha.
__global__ void k4_pcg_pq(DevSell<double> M, const float* __restrict__ Mhi, const float* __restrict__ Mlo, int n,
                          const float4* __restrict__ z32, double4_32a* __restrict__ p, double4_32a* __restrict__ q,
                          EnsScalars* sc, double* partials, unsigned int* counter, int max_blocks) {
  pdl_enter();
  double beta[kEnsW];
  int act[kEnsW];
#pragma unroll
  for (int c = 0; c < kEnsW; ++c) {
    beta[c] = sc->beta[c];
    act[c] = !sc->conv[c];
  }
  double v[kEnsW];
#pragma unroll
  for (int c = 0; c < kEnsW; ++c) v[c] = 0.0;
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float S[kEnsW] = {0.f, 0.f, 0.f, 0.f}, s[kEnsW] = {0.f, 0.f, 0.f, 0.f};
    if (M.G == 0) {
      constexpr int C = kDiaChunk / 2;
      for (int d0 = 0; d0 < M.ndiag; d0 += C) {
        float ah[C], al[C];
        float4 zz[C];
#pragma unroll
        for (int u = 0; u < C; ++u) {
          const int d = d0 + u;
          const int j = (int)i + M.off[d < kMaxDiag ? d : 0];
          const bool ok = d < M.ndiag && (unsigned)j < (unsigned)M.n_cols;
          const int64_t k = (int64_t)d * n + i;
          ah[u] = ok ? __ldg(Mhi + k) : 0.f;
          al[u] = ok ? __ldg(Mlo + k) : 0.f;
          zz[u] = ok ? __ldg(z32 + j) : zero4();
        }
#pragma unroll
        for (int u = 0; u < C; ++u) {
          df_acc(S[0], s[0], ah[u], al[u], zz[u].x);
          df_acc(S[1], s[1], ah[u], al[u], zz[u].y);
          df_acc(S[2], s[2], ah[u], al[u], zz[u].z);
          df_acc(S[3], s[3], ah[u], al[u], zz[u].w);
        }
      }
    } else {
      const int64_t sl = i >> 5, lane = i & 31;
      const int64_t end = M.slice_ptr[sl + 1];
      for (int64_t k = M.slice_ptr[sl] + lane; k < end; k += 32) {
        const float ah = __ldg(Mhi + k), al = __ldg(Mlo + k);
        const float4 zj = __ldg(z32 + __ldg(M.col + k));
        df_acc(S[0], s[0], ah, al, zj.x);
        df_acc(S[1], s[1], ah, al, zj.y);
        df_acc(S[2], s[2], ah, al, zj.z);
        df_acc(S[3], s[3], ah, al, zj.w);
      }
    }
    const float4 zi = z32[i];
    double4_32a pi = p[i], qi = q[i];
#pragma unroll
    for (int c = 0; c < kEnsW; ++c) {
      if (!act[c]) continue;
      const double w = f2d(S[c]) + f2d(s[c]);
      const double zc = f2d(comp(zi, c));
      const double qn = fma(beta[c], dc4(qi, c), w);
      const double pn = fma(beta[c], dc4(pi, c), zc);
      set4(qi, c, qn);
      set4(pi, c, pn);
      v[c] = fma(pn, qn, v[c]);
    }
    p[i] = pi;
    q[i] = qi;
  }
  double tot[kEnsW];
  if (grid_sum<kEnsW>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    for (int c = 0; c < kEnsW; ++c)
      sc->alpha[c] = (!sc->conv[c] && tot[c] != 0.0) ? sc->rz[c] / tot[c] : 0.0;
  }
}

// x += alpha p ; r -= alpha q (active columns), ||r||^2 per column, the
// next V-cycle input; the last block updates the flags, the per-column
// iteration counts and the loop condition.
__global__ void k4_pcg_update(int n, double4_32a* __restrict__ x, double4_32a* __restrict__ r,
                              const double4_32a* __restrict__ p,
                              const double4_32a* __restrict__ q, const float* __restrict__ dinv0,
                              float inv_theta0, float4* __restrict__ b0, float4* __restrict__ x0,
                              float4* __restrict__ d0, EnsScalars* sc, double* partials,
                              unsigned int* counter, int max_blocks, double tol2, int maxit,
                              cudaGraphConditionalHandle h, int use_handle, int* iters_out,
                              double* relres_out) {
  pdl_enter();
  double a[kEnsW];
  int act[kEnsW];
#pragma unroll
  for (int c = 0; c < kEnsW; ++c) {
    act[c] = !sc->conv[c];
    a[c] = sc->alpha[c];
  }
  double v[kEnsW];
#pragma unroll
  for (int c = 0; c < kEnsW; ++c) v[c] = 0.0;
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double4_32a xi = x[i], ri = r[i];
    const double4_32a pi = p[i], qi = q[i];
#pragma unroll
    for (int c = 0; c < kEnsW; ++c) {
      if (act[c]) {
        set4(xi, c, fma(a[c], dc4(pi, c), dc4(xi, c)));
        set4(ri, c, fma(-a[c], dc4(qi, c), dc4(ri, c)));
      }
      v[c] = fma(dc4(ri, c), dc4(ri, c), v[c]);
    }
    x[i] = xi;
    r[i] = ri;
    vc_input4(i, ri, dinv0, inv_theta0, b0, x0, d0);
  }
  double tot[kEnsW];
  if (grid_sum<kEnsW>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    const int pass = sc->pass + 1;
    sc->pass = pass;
    int go = 0;
    int act[kEnsW];
    for (int c = 0; c < kEnsW; ++c) {
      act[c] = !sc->conv[c];
      if (!act[c]) continue;
      sc->rnorm2[c] = tot[c];
      sc->it[c] += 1;
      const int conv = tot[c] <= tol2 * sc->bnorm2[c];
      sc->conv[c] = conv;
      go |= !conv;
      if (iters_out) iters_out[c] = sc->it[c];
    }
    const int more = go && pass < maxit;
    if (use_handle) cudaGraphSetConditional(h, more ? 1u : 0u);
    // final relative residuals only for columns that stop now (a division
    // and a square root are long FP64 chains in this one-thread tail)
    if (relres_out)
      for (int c = 0; c < kEnsW; ++c)
        if (act[c] && (sc->conv[c] || !more)) relres_out[c] = sqrt(tot[c] / sc->bnorm2[c]);
  }
}

// ------------------------------------------------------- SPE (4 cols)
// Section IV, Eq. 4-5 per column: the rings hold the last NH solutions of
// all four columns (row-interleaved) and W = M X; column c has its own Gram
// matrix G[c] and coefficients.  One pass: w = M x_newest (four columns per
// matrix entry), the Gram column and c_k = x_k . b of every column; the last
// block solves the four small systems (k4_spe_gram_df below).  coef: per
// column kSpeMax + 1 doubles (coefficients by slot, then the slots in use).
// Double-float (FP32 pair) arithmetic on the FP32 pipe (Dekker's exact
// product by FMA and Knuth's two-sum): S + s += (ah + al)(zh + zl), the
// al zl term (below 2^-48 of the product) dropped; the pair keeps about 44
// bits of the running sum.
__device__ __forceinline__ void df_acc2(float& S, float& s, float ah, float al, float zh, float zl) {
  const float p = __fmul_rn(ah, zh);
  float t = __fmaf_rn(ah, zh, -p);  // ah zh = p + t exactly
  t = __fmaf_rn(al, zh, t);
  t = __fmaf_rn(ah, zl, t);
  const float S1 = __fadd_rn(S, p);
  const float bv = __fsub_rn(S1, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(S1, bv)), __fsub_rn(p, bv));  // S + p = S1 + err
  S = S1;
  s = __fadd_rn(s, __fadd_rn(err, t));
}

// a - b = d + err exactly (two-sum of a and -b).
__device__ __forceinline__ float two_diff(float a, float b, float& err) {
  const float d = __fsub_rn(a, b);
  const float bb = __fsub_rn(d, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(d, bb)), __fsub_rn(-b, bb));
  return d;
}

// S + s += (ah + al)((zh + zl) - (xh + xl)): a matrix entry times the
// difference of two pair values, the difference formed without rounding
// of its leading part.
__device__ __forceinline__ void df_acc_diff(float& S, float& s, float ah, float al, float zh, float zl, float xh,
                                            float xl) {
  float err;
  const float dh = two_diff(zh, xh, err);
  const float dl = __fadd_rn(__fsub_rn(zl, xl), err);
  df_acc2(S, s, ah, al, dh, dl);
}

// Renormalised pair (hi, lo) of S + s.
__device__ __forceinline__ float2 df_norm(float S, float s) {
  const float h = __fadd_rn(S, s);
  return make_float2(h, __fsub_rn(s, __fsub_rn(h, S)));
}

// The (hi, lo) FP32 pair of an FP64 value: hi truncated to FP32 by integer
// operations, lo the truncated remainder (one FP64 subtraction; the pair
// carries about 47 bits: the truncated tail of lo is below 2^-47 of the
// value).  Magnitudes below the FP32 normal range pair to 0 (there below
// 1e-38 in absolute terms).
__device__ __forceinline__ float2 split_pair(double v) {
  const float h = vc_narrow(v);
  return make_float2(h, vc_narrow(v - f2d(h)));
}

// W_new = M x_new of the four columns (the first launch of the split Gram
// pass): one thread per row, the matrix entry loaded once for the four
// columns, the same double-float difference form as k4_spe_gram_df (below),
// stored in FP64 into ring slot g - 1.  No dot-product state, so more rows
// are in flight than in the fused pass.
template <int NH>
__global__ void __launch_bounds__(kBlock, 3)
k4_spe_w(DevSell<double> M, const float* __restrict__ Mhi, const float* __restrict__ Mlo,
         const float2* __restrict__ rs, int nf, const float4* __restrict__ X2, double4_32a* __restrict__ W,
         const long long* __restrict__ stepcount, int j) {
  pdl_enter();
  const long long g = stepcount[0] + j;
  if (g == 0) return;
  const int sn = spe_slot(g - 1, NH);
  const float4* __restrict__ xn = X2 + (size_t)sn * 2 * nf;
  double4_32a* __restrict__ wn = W + (size_t)sn * nf;
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 xa = __ldg(xn + 2 * i), xb = __ldg(xn + 2 * i + 1);  // columns 0, 1 and 2, 3 as (hi, lo)
    const float2 ri = __ldg(rs + i);
    float S0 = 0.f, s0 = 0.f, S1 = 0.f, s1 = 0.f, S2 = 0.f, s2 = 0.f, S3 = 0.f, s3 = 0.f;
    df_acc2(S0, s0, ri.x, ri.y, xa.x, xa.y);
    df_acc2(S1, s1, ri.x, ri.y, xa.z, xa.w);
    df_acc2(S2, s2, ri.x, ri.y, xb.x, xb.y);
    df_acc2(S3, s3, ri.x, ri.y, xb.z, xb.w);
    if (M.G == 0) {
      constexpr int C = kDiaChunk / 2;
      for (int d0 = 0; d0 < M.ndiag; d0 += C) {
        float mh[C], ml[C];
        float4 ya[C], yb[C];
#pragma unroll
        for (int q = 0; q < C; ++q) {
          const int d = d0 + q;
          const int jj = (int)i + M.off[d < kMaxDiag ? d : 0];
          const bool ok = d < M.ndiag && (unsigned)jj < (unsigned)M.n_cols;
          const int64_t k = (int64_t)d * nf + i;
          mh[q] = ok ? __ldg(Mhi + k) : 0.f;
          ml[q] = ok ? __ldg(Mlo + k) : 0.f;
          ya[q] = ok ? __ldg(xn + 2 * (int64_t)jj) : xa;  // outside: a zero difference
          yb[q] = ok ? __ldg(xn + 2 * (int64_t)jj + 1) : xb;
        }
#pragma unroll
        for (int q = 0; q < C; ++q) {
          df_acc_diff(S0, s0, mh[q], ml[q], ya[q].x, ya[q].y, xa.x, xa.y);
          df_acc_diff(S1, s1, mh[q], ml[q], ya[q].z, ya[q].w, xa.z, xa.w);
          df_acc_diff(S2, s2, mh[q], ml[q], yb[q].x, yb[q].y, xb.x, xb.y);
          df_acc_diff(S3, s3, mh[q], ml[q], yb[q].z, yb[q].w, xb.z, xb.w);
        }
      }
    } else {
      const int64_t sl = i >> 5, lane = i & 31;
      const int64_t end = M.slice_ptr[sl + 1];
      for (int64_t k = M.slice_ptr[sl] + lane; k < end; k += 32) {
        const float mh = __ldg(Mhi + k), ml = __ldg(Mlo + k);
        const int64_t jj = __ldg(M.col + k);
        const float4 ya = __ldg(xn + 2 * jj), yb = __ldg(xn + 2 * jj + 1);
        df_acc_diff(S0, s0, mh, ml, ya.x, ya.y, xa.x, xa.y);
        df_acc_diff(S1, s1, mh, ml, ya.z, ya.w, xa.z, xa.w);
        df_acc_diff(S2, s2, mh, ml, yb.x, yb.y, xb.x, xb.y);
        df_acc_diff(S3, s3, mh, ml, yb.z, yb.w, xb.z, xb.w);
      }
    }
    const float2 w0 = df_norm(S0, s0), w1 = df_norm(S1, s1), w2 = df_norm(S2, s2), w3 = df_norm(S3, s3);
    double4_32a w;
    w.x = f2d(w0.x) + f2d(w0.y);
    w.y = f2d(w1.x) + f2d(w1.y);
    w.z = f2d(w2.x) + f2d(w2.y);
    w.w = f2d(w3.x) + f2d(w3.y);
    wn[i] = w;
  }
}

// The SPE Gram pass of the four columns in double-float on the FP32 pipe
// (GB300 runs FP64 at about 1/64 of the FP32 rate, which bound an FP64 pass
// at 0.15 of HBM bandwidth).  Two threads per row, thread h taking columns
// 2h and 2h+1, whose (hi, lo) pairs are float4 h of the row in the pair
// layout (store_split4):
//   W_new = M x_new with M as two FP32 parts (Mhi + Mlo) and x_new from the
//           pair ring X2, in difference form
//             (M x)_i = sum_j m_ij (x_j - x_i) + r_i x_i,
//           r_i the row sum of the split M (rs, formed in FP64 at setup):
//           M is Laplace-type, so sum_j m_ij x_j cancels to a small part of
//           sum_j |m_ij x_j| for a smooth x, while the differences carry no
//           such cancellation -- the pair arithmetic (about 2^-45 of the sum
//           of magnitudes) then gives W to FP64-class accuracy; stored in
//           FP64 into the ring W;
//   c_k = x_k . W_new and d_k = x_k . b with x_k from X2, b from the pair
//           copy b2 of the right-hand side;
// the sums are widened to FP64, added over the lanes of one parity within a
// warp, then over warps and blocks; the last block runs the four small
// solves.  (Four threads per row, one column each, measured slower: the
// matrix and index work repeats per thread.)  With STORED_W, W_new comes
// from the ring (written by k4_spe_w) and is split back into pairs: the
// pass then carries only the dot products and the solves.
template <int NH, bool STORED_W>
__global__ void __launch_bounds__(kBlock, 2)
k4_spe_gram_df(DevSell<double> M, const float* __restrict__ Mhi, const float* __restrict__ Mlo,
               const float2* __restrict__ rs, int nf, const float4* __restrict__ X2, double4_32a* __restrict__ W,
               const float4* __restrict__ b2, const long long* __restrict__ stepcount, int s, int j,
               double* __restrict__ G, double* partials, unsigned int* counter, int max_blocks, double drop2,
               double* __restrict__ coef) {
  pdl_enter();
  const long long g = stepcount[0] + j;
  if (g == 0) {
    if (blockIdx.x == 0 && threadIdx.x < kEnsW)
      reinterpret_cast<int*>(coef + threadIdx.x * (kSpeMax + 1) + kSpeMax)[0] = 0;
    return;
  }
  const int m = (int)(g < NH ? g : NH);
  const int sn = spe_slot(g - 1, NH);
  const int h = threadIdx.x & 1;  // column pair of this thread
  constexpr int NP = 2 * NH * 2;  // per column of the pair: Gram column (NH), projections (NH)
  float S[NP], e[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) S[k] = e[k] = 0.f;
  const float4* xs[NH];
#pragma unroll
  for (int k = 0; k < NH; ++k) xs[k] = X2 + (size_t)spe_slot(g - 1 - k, NH) * 2 * nf;
  const float4* __restrict__ xn = X2 + (size_t)sn * 2 * nf;
  double* __restrict__ wn = reinterpret_cast<double*>(W + (size_t)sn * nf);
  const int64_t n2 = 2 * (int64_t)nf;
  for (int64_t u = gtid(); u < n2; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = u >> 1;
    // the row's ring and right-hand-side loads go out before the SpMV rounds
    float4 xpre[NH];
#pragma unroll
    for (int k = 0; k < NH; ++k) xpre[k] = __ldg(xs[k] + u);
    const float4 bi = __ldg(b2 + u);
    float2 w0, w1;
    if constexpr (STORED_W) {  // W_new from the ring, split into pairs
      const double2 wv = __ldcs(reinterpret_cast<const double2*>(wn + 4 * i + 2 * h));
      w0 = split_pair(wv.x);
      w1 = split_pair(wv.y);
    } else {
    const float4 xi = __ldg(xn + u);
    const float2 ri = __ldg(rs + i);
    float A0 = 0.f, a0 = 0.f, A1 = 0.f, a1 = 0.f;  // (M x_new) of the two columns, as pairs
    df_acc2(A0, a0, ri.x, ri.y, xi.x, xi.y);
    df_acc2(A1, a1, ri.x, ri.y, xi.z, xi.w);
    if (M.G == 0) {
      constexpr int C = kDiaChunk / 2;
      for (int d0 = 0; d0 < M.ndiag; d0 += C) {
        float mh[C], ml[C];
        float4 xx[C];
#pragma unroll
        for (int q = 0; q < C; ++q) {
          const int d = d0 + q;
          const int jj = (int)i + M.off[d < kMaxDiag ? d : 0];
          const bool ok = d < M.ndiag && (unsigned)jj < (unsigned)M.n_cols;
          const int64_t k = (int64_t)d * nf + i;
          mh[q] = ok ? __ldg(Mhi + k) : 0.f;
          ml[q] = ok ? __ldg(Mlo + k) : 0.f;
          xx[q] = ok ? __ldg(xn + 2 * (int64_t)jj + h) : xi;  // outside: a zero difference
        }
#pragma unroll
        for (int q = 0; q < C; ++q) {
          df_acc_diff(A0, a0, mh[q], ml[q], xx[q].x, xx[q].y, xi.x, xi.y);
          df_acc_diff(A1, a1, mh[q], ml[q], xx[q].z, xx[q].w, xi.z, xi.w);
        }
      }
    } else {
      const int64_t sl = i >> 5, lane = i & 31;
      const int64_t end = M.slice_ptr[sl + 1];
      for (int64_t k = M.slice_ptr[sl] + lane; k < end; k += 32) {
        const float mh = __ldg(Mhi + k), ml = __ldg(Mlo + k);
        const float4 xj = __ldg(xn + 2 * (int64_t)__ldg(M.col + k) + h);
        df_acc_diff(A0, a0, mh, ml, xj.x, xj.y, xi.x, xi.y);
        df_acc_diff(A1, a1, mh, ml, xj.z, xj.w, xi.z, xi.w);
      }
    }
    w0 = df_norm(A0, a0);
    w1 = df_norm(A1, a1);
    *reinterpret_cast<double2*>(wn + 4 * i + 2 * h) =
        make_double2(f2d(w0.x) + f2d(w0.y), f2d(w1.x) + f2d(w1.y));
    }
#pragma unroll
    for (int k = 0; k < NH; ++k) {
      if (k >= m) break;
      const float4 xk = xpre[k];
      df_acc2(S[k], e[k], xk.x, xk.y, w0.x, w0.y);
      df_acc2(S[NH + k], e[NH + k], xk.x, xk.y, bi.x, bi.y);
      df_acc2(S[2 * NH + k], e[2 * NH + k], xk.z, xk.w, w1.x, w1.y);
      df_acc2(S[3 * NH + k], e[3 * NH + k], xk.z, xk.w, bi.z, bi.w);
    }
  }
  // Sums widened to FP64, slot h NP + k (column c at c 2 NH: NH Gram entries,
  // then NH projections): lanes of one parity add over the warp, then the
  // warps of the block in shared memory, one partial per slot and block.
  constexpr int NS = 2 * NH * kEnsW;
  __shared__ double wsum[kBlock / 32][NS];
  __shared__ double stot[NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    double t = f2d(S[k]) + f2d(e[k]);
#pragma unroll
    for (int o = 16; o >= 2; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane < 2) wsum[warp][lane * NP + k] = t;
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w][threadIdx.x];
    partials[threadIdx.x * max_blocks + blockIdx.x] = t;
    __threadfence();  // every writer publishes its partial before the ticket
  }
  __syncthreads();
  if (!grid_ticket(counter)) return;
  __threadfence();
  if (threadIdx.x < NS) {  // the last block: totals per slot, then the four small solves
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(partials + threadIdx.x * max_blocks + b);
    stot[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
  if (threadIdx.x < kEnsW)
    spe_solve<NH>(stot + threadIdx.x * 2 * NH, g, m, sn, G + threadIdx.x * kSpeMax * kSpeMax, drop2,
                  coef + threadIdx.x * (kSpeMax + 1));
}

// Row sums of the split M (hi + lo) in FP64, kept as FP32 pairs: the r_i of
// the difference-form products (one thread per row; setup).
__global__ void k_rowsum_split(DevSell<double> M, const float* __restrict__ Mhi, const float* __restrict__ Mlo,
                               int n, float2* __restrict__ rs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = 0.0;
  if (M.G == 0) {
    for (int d = 0; d < M.ndiag; ++d) {
      const int j = (int)i + M.off[d];
      if ((unsigned)j >= (unsigned)M.n_cols) continue;
      const int64_t k = (int64_t)d * n + i;
      t += (double)Mhi[k] + (double)Mlo[k];
    }
  } else {
    const int64_t sl = i >> 5, lane = i & 31;
    for (int64_t k = M.slice_ptr[sl] + lane; k < M.slice_ptr[sl + 1]; k += 32) t += (double)Mhi[k] + (double)Mlo[k];
  }
  const float h = (float)t;
  rs[i] = make_float2(h, (float)(t - (double)h));
}

// CG start of the four columns from their SPE vectors: x0 = X a_c,
// r0 = R - W a_c (no SpMV), norms, V-cycle input and flags (as
// k4_pcg_init); without history r0 = R - M x.
template <int NH>
__global__ void k4_spe_start(DevSell<double> M, int nf, const double4_32a* __restrict__ X,
                             const double4_32a* __restrict__ W, const double* __restrict__ coef,
                             const double4_32a* __restrict__ R, double4_32a* __restrict__ x,
                             double4_32a* __restrict__ r, const float* __restrict__ dinv0, float inv_theta0,
                             float4* __restrict__ b0, float4* __restrict__ x0, float4* __restrict__ d0,
                             EnsScalars* sc, double* partials, unsigned int* counter, int max_blocks,
                             double tol2, int maxit, cudaGraphConditionalHandle h, int use_handle,
                             int* iters_out, double* relres_out, int* zero_out) {
  pdl_enter();
  const int m = reinterpret_cast<const int*>(coef + kSpeMax)[0];  // same for every column
  double y[kEnsW][NH];
#pragma unroll
  for (int c = 0; c < kEnsW; ++c)
#pragma unroll
    for (int k = 0; k < NH; ++k) y[c][k] = k < m ? coef[c * (kSpeMax + 1) + k] : 0.0;
  double v[2 * kEnsW];
#pragma unroll
  for (int k = 0; k < 2 * kEnsW; ++k) v[k] = 0.0;
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    double4_32a mx;
    if (m > 0) {
      double4_32a xi = {0.0, 0.0, 0.0, 0.0};
      mx = xi;
#pragma unroll
      for (int k = 0; k < NH; ++k) {
        if (k >= m) break;
        const double4_32a xk = X[(size_t)k * nf + i], wk = W[(size_t)k * nf + i];
#pragma unroll
        for (int c = 0; c < kEnsW; ++c) {
          set4(xi, c, fma(y[c][k], dc4(xk, c), dc4(xi, c)));
          set4(mx, c, fma(y[c][k], dc4(wk, c), dc4(mx, c)));
        }
      }
      x[i] = xi;
    } else {
      mx = mat_row_d4(M, i, nf, x);
    }
    const double4_32a Ri = R[i];
    double4_32a ri;
#pragma unroll
    for (int c = 0; c < kEnsW; ++c) {
      set4(ri, c, dc4(Ri, c) - dc4(mx, c));
      v[c] = fma(dc4(Ri, c), dc4(Ri, c), v[c]);
      v[kEnsW + c] = fma(dc4(ri, c), dc4(ri, c), v[kEnsW + c]);
    }
    r[i] = ri;
    vc_input4(i, ri, dinv0, inv_theta0, b0, x0, d0);
  }
  double tot[2 * kEnsW];
  if (grid_sum<2 * kEnsW>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0)
    ens_init_tail(tot, sc, tol2, maxit, h, use_handle, iters_out, relres_out, zero_out);
}

// --------------------------------------------------- element and stages
// K(x)x for four columns: the tet's geometry once, four gradients, kappas
// and local residuals, scattered with one 16-byte vector atomic per vertex.
// Y2: per node the four columns as (hi, lo) FP32 pairs (two float4).
__global__ void k4_elem32(int64_t nt, const int4* __restrict__ conn, const uint8_t* __restrict__ mat,
                          const MaterialDev* __restrict__ mats, const float4* __restrict__ xh,
                          const float4* __restrict__ xl, const float4* __restrict__ Y2, int n_limit,
                          float4* __restrict__ y) {
  pdl_enter();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  const int4 t = conn[e];
  const float4 h0 = xh[t.x], h1 = xh[t.y], h2 = xh[t.z], h3 = xh[t.w];
  const float4 l0 = xl[t.x], l1 = xl[t.y], l2 = xl[t.z], l3 = xl[t.w];
  const float e1x = (h1.x - h0.x) + (l1.x - l0.x), e1y = (h1.y - h0.y) + (l1.y - l0.y),
              e1z = (h1.z - h0.z) + (l1.z - l0.z);
  const float e2x = (h2.x - h0.x) + (l2.x - l0.x), e2y = (h2.y - h0.y) + (l2.y - l0.y),
              e2z = (h2.z - h0.z) + (l2.z - l0.z);
  const float e3x = (h3.x - h0.x) + (l3.x - l0.x), e3y = (h3.y - h0.y) + (l3.y - l0.y),
              e3z = (h3.z - h0.z) + (l3.z - l0.z);
  const float c1x = e2y * e3z - e2z * e3y, c1y = e2z * e3x - e2x * e3z, c1z = e2x * e3y - e2y * e3x;
  const float c2x = e3y * e1z - e3z * e1y, c2y = e3z * e1x - e3x * e1z, c2z = e3x * e1y - e3y * e1x;
  const float c3x = e1y * e2z - e1z * e2y, c3y = e1z * e2x - e1x * e2z, c3z = e1x * e2y - e1y * e2x;
  const float invD = 1.0f / (e1x * c1x + e1y * c1y + e1z * c1z);  // one division for the four columns
  const MaterialDev m = mats[mat[e]];
  // potentials: node v holds columns 0,1 in Y2[2v] and 2,3 in Y2[2v+1]
  const float4 a0 = Y2[2 * (int64_t)t.x], b0 = Y2[2 * (int64_t)t.x + 1];
  const float4 a1 = Y2[2 * (int64_t)t.y], b1 = Y2[2 * (int64_t)t.y + 1];
  const float4 a2 = Y2[2 * (int64_t)t.z], b2 = Y2[2 * (int64_t)t.z + 1];
  const float4 a3 = Y2[2 * (int64_t)t.w], b3 = Y2[2 * (int64_t)t.w + 1];
  float r0[kEnsW], r1[kEnsW], r2[kEnsW], r3[kEnsW];
#pragma unroll
  for (int c = 0; c < kEnsW; ++c) {
    // (hi, lo) of column c at the four vertices
    const float2 f0 = c == 0 ? make_float2(a0.x, a0.y) : c == 1 ? make_float2(a0.z, a0.w)
                    : c == 2 ? make_float2(b0.x, b0.y) : make_float2(b0.z, b0.w);
    const float2 f1 = c == 0 ? make_float2(a1.x, a1.y) : c == 1 ? make_float2(a1.z, a1.w)
                    : c == 2 ? make_float2(b1.x, b1.y) : make_float2(b1.z, b1.w);
    const float2 f2 = c == 0 ? make_float2(a2.x, a2.y) : c == 1 ? make_float2(a2.z, a2.w)
                    : c == 2 ? make_float2(b2.x, b2.y) : make_float2(b2.z, b2.w);
    const float2 f3 = c == 0 ? make_float2(a3.x, a3.y) : c == 1 ? make_float2(a3.z, a3.w)
                    : c == 2 ? make_float2(b3.x, b3.y) : make_float2(b3.z, b3.w);
    const float d1 = (f1.x - f0.x) + (f1.y - f0.y);
    const float d2 = (f2.x - f0.x) + (f2.y - f0.y);
    const float d3 = (f3.x - f0.x) + (f3.y - f0.y);
    const float gx = d1 * c1x + d2 * c2x + d3 * c3x;
    const float gy = d1 * c1y + d2 * c2y + d3 * c3y;
    const float gz = d1 * c1z + d2 * c2z + d3 * c3z;
    float kap;
    if (m.is_const) {
      kap = m.klo_f;
    } else {
      const float E = sqrtf(gx * gx + gy * gy + gz * gz) * invD;
      kap = kappa32(m, E);
    }
    const float sc = kap * (invD * (1.0f / 6.0f));
    r1[c] = sc * (c1x * gx + c1y * gy + c1z * gz);
    r2[c] = sc * (c2x * gx + c2y * gy + c2z * gz);
    r3[c] = sc * (c3x * gx + c3y * gy + c3z * gz);
    r0[c] = -(r1[c] + r2[c] + r3[c]);
  }
  if (t.x < n_limit) atomicAdd(y + t.x, make_float4(r0[0], r0[1], r0[2], r0[3]));
  if (t.y < n_limit) atomicAdd(y + t.y, make_float4(r1[0], r1[1], r1[2], r1[3]));
  if (t.z < n_limit) atomicAdd(y + t.z, make_float4(r2[0], r2[1], r2[2], r2[3]));
  if (t.w < n_limit) atomicAdd(y + t.w, make_float4(r3[0], r3[1], r3[2], r3[3]));
}

// K(x)x for four columns on Kuhn cells (as k_elem32_cell): the cell's
// corners, coordinates and four potentials loaded once, the six tets'
// residuals summed per corner, one 16-byte atomic add per corner.  Columns
// (0, 1) and (2, 3) travel as packed FP32 pairs: one f32x2 instruction
// (__ffma2_rn, __fadd2_rn, __fmul2_rn; per component the same rounding as
// the scalar operation) does the work of two columns.
constexpr int kElemBlock4 = 128;  // threads per block of k4_elem32_cell (4 blocks per SM at 128 registers)

__device__ __forceinline__ float2 bcast2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float4 cat2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// One tet (corners 0, B, C, D of the cell) into the corner sums; pa/pb hold
// the corners' potential offsets to corner 0 of columns (0, 1) and (2, 3).
// With d_l the offsets at B, C, D and c_k the cofactors, r_k = s c_k . g,
// g = sum_l d_l c_l, s = kappa / (6 D), and r_0 = -(r_1 + r_2 + r_3).  For a
// constant kappa this is r_k = sum_l G_kl d_l with G_kl = s c_k . c_l: the
// 3x3 Gram matrix is formed once for the four columns; a field-dependent
// kappa needs |g| per column, so there g is formed as written.
template <int B, int C, int D>
__device__ __forceinline__ void cell_tet32x4(const float (&dx)[8][3], const float2 (&pa)[8], const float2 (&pb)[8],
                                             const MaterialDev& m, float2 (&aa)[8], float2 (&ab)[8]) {
  const float e[3][3] = {{dx[B][0], dx[B][1], dx[B][2]}, {dx[C][0], dx[C][1], dx[C][2]},
                         {dx[D][0], dx[D][1], dx[D][2]}};
  const TetGeom<float> g = tet_geom<float>(e);  // one division for the four columns
  float2 u1a, u2a, u3a, u1b, u2b, u3b;
  if (m.is_const) {
    const float s = m.klo_f * (g.invD * (1.0f / 6.0f));
    const float2 G11 = bcast2(s * (g.c[0][0] * g.c[0][0] + g.c[0][1] * g.c[0][1] + g.c[0][2] * g.c[0][2]));
    const float2 G12 = bcast2(s * (g.c[0][0] * g.c[1][0] + g.c[0][1] * g.c[1][1] + g.c[0][2] * g.c[1][2]));
    const float2 G13 = bcast2(s * (g.c[0][0] * g.c[2][0] + g.c[0][1] * g.c[2][1] + g.c[0][2] * g.c[2][2]));
    const float2 G22 = bcast2(s * (g.c[1][0] * g.c[1][0] + g.c[1][1] * g.c[1][1] + g.c[1][2] * g.c[1][2]));
    const float2 G23 = bcast2(s * (g.c[1][0] * g.c[2][0] + g.c[1][1] * g.c[2][1] + g.c[1][2] * g.c[2][2]));
    const float2 G33 = bcast2(s * (g.c[2][0] * g.c[2][0] + g.c[2][1] * g.c[2][1] + g.c[2][2] * g.c[2][2]));
    u1a = __ffma2_rn(G11, pa[B], __ffma2_rn(G12, pa[C], __fmul2_rn(G13, pa[D])));
    u2a = __ffma2_rn(G12, pa[B], __ffma2_rn(G22, pa[C], __fmul2_rn(G23, pa[D])));
    u3a = __ffma2_rn(G13, pa[B], __ffma2_rn(G23, pa[C], __fmul2_rn(G33, pa[D])));
    u1b = __ffma2_rn(G11, pb[B], __ffma2_rn(G12, pb[C], __fmul2_rn(G13, pb[D])));
    u2b = __ffma2_rn(G12, pb[B], __ffma2_rn(G22, pb[C], __fmul2_rn(G23, pb[D])));
    u3b = __ffma2_rn(G13, pb[B], __ffma2_rn(G23, pb[C], __fmul2_rn(G33, pb[D])));
  } else {
    const float2 C00 = bcast2(g.c[0][0]), C01 = bcast2(g.c[0][1]), C02 = bcast2(g.c[0][2]);
    const float2 C10 = bcast2(g.c[1][0]), C11 = bcast2(g.c[1][1]), C12 = bcast2(g.c[1][2]);
    const float2 C20 = bcast2(g.c[2][0]), C21 = bcast2(g.c[2][1]), C22 = bcast2(g.c[2][2]);
    const float2 gxa = __ffma2_rn(pa[B], C00, __ffma2_rn(pa[C], C10, __fmul2_rn(pa[D], C20)));
    const float2 gya = __ffma2_rn(pa[B], C01, __ffma2_rn(pa[C], C11, __fmul2_rn(pa[D], C21)));
    const float2 gza = __ffma2_rn(pa[B], C02, __ffma2_rn(pa[C], C12, __fmul2_rn(pa[D], C22)));
    const float2 gxb = __ffma2_rn(pb[B], C00, __ffma2_rn(pb[C], C10, __fmul2_rn(pb[D], C20)));
    const float2 gyb = __ffma2_rn(pb[B], C01, __ffma2_rn(pb[C], C11, __fmul2_rn(pb[D], C21)));
    const float2 gzb = __ffma2_rn(pb[B], C02, __ffma2_rn(pb[C], C12, __fmul2_rn(pb[D], C22)));
    // |E| = |g| / D per column, kappa(|E|), s = kappa / (6 D)
    const float2 na = __ffma2_rn(gxa, gxa, __ffma2_rn(gya, gya, __fmul2_rn(gza, gza)));
    const float2 nb = __ffma2_rn(gxb, gxb, __ffma2_rn(gyb, gyb, __fmul2_rn(gzb, gzb)));
    const float q = g.invD * (1.0f / 6.0f);
    const float2 sa = make_float2(kappa32(m, sqrtf(na.x) * g.invD) * q, kappa32(m, sqrtf(na.y) * g.invD) * q);
    const float2 sb = make_float2(kappa32(m, sqrtf(nb.x) * g.invD) * q, kappa32(m, sqrtf(nb.y) * g.invD) * q);
    u1a = __fmul2_rn(sa, __ffma2_rn(C00, gxa, __ffma2_rn(C01, gya, __fmul2_rn(C02, gza))));
    u2a = __fmul2_rn(sa, __ffma2_rn(C10, gxa, __ffma2_rn(C11, gya, __fmul2_rn(C12, gza))));
    u3a = __fmul2_rn(sa, __ffma2_rn(C20, gxa, __ffma2_rn(C21, gya, __fmul2_rn(C22, gza))));
    u1b = __fmul2_rn(sb, __ffma2_rn(C00, gxb, __ffma2_rn(C01, gyb, __fmul2_rn(C02, gzb))));
    u2b = __fmul2_rn(sb, __ffma2_rn(C10, gxb, __ffma2_rn(C11, gyb, __fmul2_rn(C12, gzb))));
    u3b = __fmul2_rn(sb, __ffma2_rn(C20, gxb, __ffma2_rn(C21, gyb, __fmul2_rn(C22, gzb))));
  }
  aa[B] = __fadd2_rn(aa[B], u1a);
  aa[C] = __fadd2_rn(aa[C], u2a);
  aa[D] = __fadd2_rn(aa[D], u3a);
  aa[0] = __fadd2_rn(aa[0], neg2(__fadd2_rn(__fadd2_rn(u1a, u2a), u3a)));
  ab[B] = __fadd2_rn(ab[B], u1b);
  ab[C] = __fadd2_rn(ab[C], u2b);
  ab[D] = __fadd2_rn(ab[D], u3b);
  ab[0] = __fadd2_rn(ab[0], neg2(__fadd2_rn(__fadd2_rn(u1b, u2b), u3b)));
}

// Only the corners' offsets to corner 0 stay live across the six tets (all
// share the diagonal 0-7): positions dx[k] and the potential pairs pa[k],
// pb[k], each formed from the (hi, lo) FP32 pairs as (hi_k - hi_0) +
// (lo_k - lo_0).
__global__ void __launch_bounds__(kElemBlock4, 4)
k4_elem32_cell(int64_t ncell, const int32_t* __restrict__ corner, const uint8_t* __restrict__ mat,
               const MaterialDev* __restrict__ mats, const float4* __restrict__ xh, const float4* __restrict__ xl,
               const float4* __restrict__ Y2, int n_limit, float4* __restrict__ y) {
  pdl_enter();
  const int64_t cidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cidx >= ncell) return;
  int v[8];
  float dx[8][3];
  float2 pa[8], pb[8], aa[8], ab[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __ldg(corner + (int64_t)k * ncell + cidx);
  const float4 h0 = xh[v[0]], l0 = xl[v[0]], a0 = Y2[2 * (int64_t)v[0]], b0 = Y2[2 * (int64_t)v[0] + 1];
  const float2 nh0 = make_float2(-h0.x, -h0.y), nl0 = make_float2(-l0.x, -l0.y);
  const float2 na0 = make_float2(-a0.x, -a0.y), na1 = make_float2(-a0.z, -a0.w);
  const float2 nb0 = make_float2(-b0.x, -b0.y), nb1 = make_float2(-b0.z, -b0.w);
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    const float4 h = xh[v[k]], l = xl[v[k]];
    const float4 a = Y2[2 * (int64_t)v[k]], b = Y2[2 * (int64_t)v[k] + 1];
    const float2 dxy = __fadd2_rn(__fadd2_rn(make_float2(h.x, h.y), nh0), __fadd2_rn(make_float2(l.x, l.y), nl0));
    dx[k][0] = dxy.x;
    dx[k][1] = dxy.y;
    dx[k][2] = (h.z - h0.z) + (l.z - l0.z);
    // columns 0, 1 in a as (hi, lo, hi, lo), columns 2, 3 in b: the (hi, lo)
    // differences of one column as a pair, then their sum
    const float2 t0 = __fadd2_rn(make_float2(a.x, a.y), na0), t1 = __fadd2_rn(make_float2(a.z, a.w), na1);
    const float2 t2 = __fadd2_rn(make_float2(b.x, b.y), nb0), t3 = __fadd2_rn(make_float2(b.z, b.w), nb1);
    pa[k] = make_float2(t0.x + t0.y, t1.x + t1.y);
    pb[k] = make_float2(t2.x + t2.y, t3.x + t3.y);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) aa[k] = ab[k] = make_float2(0.f, 0.f);
  const uint8_t* mt = mat + 6 * cidx;
  // tets ordered so that corners retire early: each corner's atomic add
  // goes out after the last tet that touches it
  cell_tet32x4<1, 3, 7>(dx, pa, pb, mats[mt[0]], aa, ab);
  cell_tet32x4<1, 7, 5>(dx, pa, pb, mats[mt[1]], aa, ab);
  if (v[1] < n_limit) atomicAdd(y + v[1], cat2(aa[1], ab[1]));
  cell_tet32x4<2, 7, 3>(dx, pa, pb, mats[mt[2]], aa, ab);
  if (v[3] < n_limit) atomicAdd(y + v[3], cat2(aa[3], ab[3]));
  cell_tet32x4<4, 5, 7>(dx, pa, pb, mats[mt[4]], aa, ab);
  if (v[5] < n_limit) atomicAdd(y + v[5], cat2(aa[5], ab[5]));
  cell_tet32x4<4, 7, 6>(dx, pa, pb, mats[mt[5]], aa, ab);
  if (v[4] < n_limit) atomicAdd(y + v[4], cat2(aa[4], ab[4]));
  cell_tet32x4<2, 6, 7>(dx, pa, pb, mats[mt[3]], aa, ab);
  if (v[0] < n_limit) atomicAdd(y + v[0], cat2(aa[0], ab[0]));
  if (v[2] < n_limit) atomicAdd(y + v[2], cat2(aa[2], ab[2]));
  if (v[6] < n_limit) atomicAdd(y + v[6], cat2(aa[6], ab[6]));
  if (v[7] < n_limit) atomicAdd(y + v[7], cat2(aa[7], ab[7]));
}

__device__ __forceinline__ void store_split4(float4* __restrict__ Y2, int64_t i, const double4_32a& v) {
  const float2 x = split_pair(v.x), y = split_pair(v.y), z = split_pair(v.z), w = split_pair(v.w);
  Y2[2 * i] = make_float4(x.x, x.y, y.x, y.y);
  Y2[2 * i + 1] = make_float4(z.x, z.y, w.x, w.y);
}

// Four column-major mesh-order columns (src + c n) into the FP32-pair layout
// in internal order (internal node i is mesh node perm[i]).
__global__ void k4_gather_pair_perm(int n, const double* __restrict__ src, const int32_t* __restrict__ perm,
                                    float4* __restrict__ dst2) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t m = perm[i];
  double4_32a v;
  v.x = src[m];
  v.y = src[(int64_t)n + m];
  v.z = src[2 * (int64_t)n + m];
  v.w = src[3 * (int64_t)n + m];
  store_split4(dst2, i, v);
}

// Four FP32 columns (internal order, one float4 per node) widened into
// column-major FP64 columns in mesh order.
__global__ void k4_scatter_perm(int n, const float4* __restrict__ y, const int32_t* __restrict__ perm,
                                double* __restrict__ dst) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 v = y[i];
  const int64_t m = perm[i];
  dst[m] = (double)v.x;
  dst[(int64_t)n + m] = (double)v.y;
  dst[2 * (int64_t)n + m] = (double)v.z;
  dst[3 * (int64_t)n + m] = (double)v.w;
}

// Four column-major columns (src + c n) into the interleaved FP64 layout and
// the FP32-pair layout.
__global__ void k4_interleave_pair(int n, const double* __restrict__ src, double4_32a* __restrict__ dst,
                                   float4* __restrict__ dst2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double4_32a v;
  v.x = src[i];
  v.y = src[(int64_t)n + i];
  v.z = src[2 * (int64_t)n + i];
  v.w = src[3 * (int64_t)n + i];
  dst[i] = v;
  store_split4(dst2, i, v);
}

// Y0 (interleaved, internal order) from the caller's column-major mesh-order
// X = prm->x (column c at X + c n), Dirichlet rows = g(t) times the column's
// drive scale; the start vector of the first solve (previous solution).
__global__ void k4_gather_state(int n, int nf, const StepParams* prm, const int32_t* __restrict__ noi,
                                const double* __restrict__ dir_scale, const double* __restrict__ g,
                                const double* __restrict__ colv, double4_32a* __restrict__ Y0,
                                float4* __restrict__ Y2, const double4_32a* __restrict__ Fsrc,
                                double4_32a* __restrict__ Fdst) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double4_32a v;
  if (i < nf) {
    const double* __restrict__ X = prm->x;
    const int64_t m = noi[i];
    v.x = X[m];
    v.y = X[(int64_t)n + m];
    v.z = X[2 * (int64_t)n + m];
    v.w = X[3 * (int64_t)n + m];
    Fdst[i] = Fsrc[i];
  } else {
    const double gd = dir_scale[i - nf] * g[0];
    v.x = gd * colv[0];
    v.y = gd * colv[1];
    v.z = gd * colv[2];
    v.w = gd * colv[3];
  }
  Y0[i] = v;
  store_split4(Y2, i, v);
}

// Stage recurrence for the four columns (same coefficients; a column whose
// right-hand side was zero contributes F = 0), the next start vector and,
// after the last stage (write_x), x(t + dt) back to the caller's column-major
// layout at prm->x.
__global__ void k4_recurrence(int n, int nf, double c0, double mu, double nu, double mut, double gt,
                              const StepParams* prm, const double4_32a* __restrict__ Y0,
                              const double4_32a* __restrict__ Yjm1, const double4_32a* __restrict__ Yjm2,
                              const double4_32a* __restrict__ Fjm1, const double4_32a* __restrict__ F0,
                              const int* __restrict__ zero_flags, int jm1, const double* __restrict__ dir_scale,
                              const double* __restrict__ gj, const double* __restrict__ colv,
                              double4_32a* __restrict__ Yj, float4* __restrict__ Y2,
                              double4_32a* __restrict__ Fguess, int write_x,
                              const int32_t* __restrict__ noi, const long long* __restrict__ stepcount, int s,
                              double4_32a* __restrict__ ring, float4* __restrict__ ring2, int nh) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double4_32a v;
  if (i < nf) {
    const double dt = prm->dt;
    const double4_32a y0 = Y0[i], y1 = Yjm1[i], y2 = Yjm2[i], f1 = Fjm1[i], f0 = F0[i];
    if (ring) {  // SPE history, in FP64 and as FP32 pairs
      const size_t slot = (size_t)((stepcount[0] + jm1) % nh);
      ring[slot * nf + i] = f1;
      store_split4(ring2 + slot * 2 * nf, i, f1);
    }
#pragma unroll
    for (int c = 0; c < kEnsW; ++c) {
      const double fj = zero_flags[jm1 * kEnsW + c] ? 0.0 : dc4(f1, c);
      const double ff = zero_flags[c] ? 0.0 : dc4(f0, c);
      set4(v, c, c0 * dc4(y0, c) + mu * dc4(y1, c) + nu * dc4(y2, c) + (mut * dt) * fj + (gt * dt) * ff);
    }
    if (Fguess) Fguess[i] = f1;
  } else {
    const double gd = dir_scale[i - nf] * (*gj);
    v.x = gd * colv[0];
    v.y = gd * colv[1];
    v.z = gd * colv[2];
    v.w = gd * colv[3];
  }
  Yj[i] = v;
  if (Y2) store_split4(Y2, i, v);
  if (write_x) {
    double* __restrict__ X = prm->x;
    const int64_t m = noi[i];
    X[m] = v.x;
    X[(int64_t)n + m] = v.y;
    X[2 * (int64_t)n + m] = v.z;
    X[3 * (int64_t)n + m] = v.w;
  }
}

// R = -y - g'(t_j) v_c M_fd 1_top per column in FP64 (and as FP32 pairs
// into R2 when given), and clear y.
__global__ void k4_rhs(int nf, float4* __restrict__ y32, const double* __restrict__ gpj,
                       const double* __restrict__ colv, const double* __restrict__ mtop,
                       double4_32a* __restrict__ R, float4* __restrict__ R2) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  const float4 y = y32[i];
  const double gm = (*gpj) * mtop[i];
  double4_32a r;
  r.x = -f2d(y.x) - gm * colv[0];
  r.y = -f2d(y.y) - gm * colv[1];
  r.z = -f2d(y.z) - gm * colv[2];
  r.w = -f2d(y.w) - gm * colv[3];
  R[i] = r;
  if (R2) store_split4(R2, i, r);
  y32[i] = zero4();
}

}  // namespace eqs
