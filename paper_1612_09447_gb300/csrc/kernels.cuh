// Device kernels of the EQS RKC library (sm_103a).
//
// Vector kernels run one thread per row; matrices are SELL-32 (slices of 32
// rows stored column-major), so the 32 lanes of a warp read 32 consecutive
// values/column indices per step (coalesced) and no shuffles are needed.
#pragma once

#include <cuda_runtime.h>

#include "eqs_internal.h"

namespace eqs {

constexpr int kBlock = 256;
// DIA diagonals whose loads are issued together (8: a batch of 16 loads per
// row; 16 measured no faster on GB300).
constexpr int kDiaChunk = 8;

// Programmatic dependent launch: wait until the preceding kernel of the
// stream has completed (its writes visible), then allow the next kernel to
// start launching.  A no-op for kernels launched without the attribute.
__device__ __forceinline__ void pdl_enter() {
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
}

// FP32 -> FP64 widening by integer operations, exact (the same value as
// (double)f, subnormal inputs normalised, infinities and NaN kept): GB300
// executes the hardware conversion on its FP64 pipe (about 1/64 of the FP32
// rate), which bounds the FP64-accumulating CG kernels; this runs on the
// integer pipe with no hardware-conversion path to predicate in.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  const unsigned sh = m ? __clz(m) - 8u : 0u;  // subnormal: bring the leading one to bit 23
  const unsigned ed = e == 0u ? (m ? 897u - sh : 0u) : (e == 0xFFu ? 0x7FFu : e + 896u);
  const unsigned md = e == 0u ? ((m << sh) & 0x7FFFFFu) : m;
  const unsigned hi = (u & 0x80000000u) | (ed << 20) | (md >> 3);
  return __hiloint2double((int)hi, (int)(md << 29));
}

// FP64 -> FP32 for a V-cycle input by integer operations: the mantissa is
// truncated (not rounded), magnitudes below the FP32 normal range become
// zero and those above it the largest FP32 value.  Only the preconditioner
// sees these values (the flexible CG keeps r, x and the dot products in
// FP64), so the truncation costs nothing in accuracy, and it keeps the
// conversion off GB300's FP64 pipe.
__device__ __forceinline__ float vc_narrow(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned mag = e <= 896u ? 0u : (e >= 1151u ? 0x7F7FFFFFu : ((e - 896u) << 23) | m);
  return __uint_as_float((hi & 0x80000000u) | mag);
}
template <typename T>
__device__ __forceinline__ T vc_in(double d);
template <>
__device__ __forceinline__ float vc_in<float>(double d) { return vc_narrow(d); }
template <>
__device__ __forceinline__ double vc_in<double>(double d) { return d; }

// Widening for the precision T of a V-cycle (float: f2d; double: as is).
__device__ __forceinline__ double widen(float f) { return f2d(f); }
__device__ __forceinline__ double widen(double d) { return d; }

// Both conversions over arrays (for checking f2d against (double)f).
__global__ void k_convert_check(int n, const float* __restrict__ f, double* __restrict__ f_wide) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f_wide[i] = f2d(f[i]);
}

__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }

// (A x)_row, accumulation in T.  Thread `tid` serves row tid >> A.logG; with
// G > 1 every lane of the row's group returns the full sum (all lanes of a
// warp must call this, also those past the last row).
// x_j (+ xadd_j when ADD: a pending update not yet added to x).
template <typename T, bool ADD>
__device__ __forceinline__ T xv(const T* __restrict__ x, const T* __restrict__ xadd, int j) {
  return ADD ? __ldg(x + j) + __ldg(xadd + j) : __ldg(x + j);
}

template <typename T, bool ADD>
__device__ __forceinline__ T mat_row_impl(const DevSell<T>& A, int64_t tid, int n, const T* __restrict__ x,
                                          const T* __restrict__ xadd) {
  const int row = (int)(tid >> A.logG);
  T acc = T(0);
  if (A.G == 0) {  // DIA: coalesced loads, no indices; chunks of kDiaChunk
    // diagonals whose loads are all issued before the first use (memory-level
    // parallelism for these latency-bound row kernels), two accumulation chains
    if (row >= n) return acc;
    const T* __restrict__ v = A.val + row;
    T acc1 = T(0);
    constexpr int CH = kDiaChunk;
    for (int d0 = 0; d0 < A.ndiag; d0 += CH) {
      T a[CH], xs[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int d = d0 + u;
        const int j = row + A.off[d < kMaxDiag ? d : 0];
        const bool ok = d < A.ndiag && (unsigned)j < (unsigned)A.n_cols;
        a[u] = ok ? __ldg(v + (int64_t)d * n) : T(0);
        xs[u] = ok ? xv<T, ADD>(x, xadd, j) : T(0);
      }
#pragma unroll
      for (int u = 0; u < CH; u += 2) {
        acc = fmadd(a[u], xs[u], acc);
        acc1 = fmadd(a[u + 1], xs[u + 1], acc1);
      }
    }
    return acc + acc1;
  }
  if (A.G == 1) {  // SELL-32: load a batch of indices, then the gathers
    if (row >= n) return acc;
    const int s = row >> 5, lane = row & 31;
    int64_t k = A.slice_ptr[s] + lane;
    const int64_t end = A.slice_ptr[s + 1];
    for (; k < end; k += 32 * 8) {
      int c[8];
      T a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t kk = k + 32 * u;
        c[u] = kk < end ? __ldg(A.col + kk) : 0;
        a[u] = kk < end ? __ldg(A.val + kk) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) acc = fmadd(a[u], xv<T, ADD>(x, xadd, c[u]), acc);
    }
    return acc;
  }
  const int g = (int)(tid & (A.G - 1));
  int64_t k = 0, end = 0;
  if (row < n) {
    k = A.slice_ptr[row] + g;
    end = A.slice_ptr[row + 1];
  }
  for (; k < end; k += (int64_t)A.G * 4) {
    int c[4];
    T a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t kk = k + (int64_t)A.G * u;
      c[u] = kk < end ? __ldg(A.col + kk) : 0;
      a[u] = kk < end ? __ldg(A.val + kk) : T(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) acc = fmadd(a[u], xv<T, ADD>(x, xadd, c[u]), acc);
  }
  for (int o = A.G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

template <typename T>
__device__ __forceinline__ T mat_row(const DevSell<T>& A, int64_t tid, int n, const T* __restrict__ x) {
  return mat_row_impl<T, false>(A, tid, n, x, nullptr);
}

// (A (x + xadd))_row
template <typename T>
__device__ __forceinline__ T mat_row_add(const DevSell<T>& A, int64_t tid, int n, const T* __restrict__ x,
                                         const T* __restrict__ xadd) {
  return mat_row_impl<T, true>(A, tid, n, x, xadd);
}

// (A (x1 + beta x2))_row for a one-thread-per-row matrix (DIA or SELL-32).
__device__ __forceinline__ double mat_row_axpy(const DevSell<double>& A, int row, int n,
                                               const double* __restrict__ x1,
                                               const double* __restrict__ x2, double beta) {
  double acc = 0.0;
  if (row >= n) return acc;
  if (A.G == 0) {
    const double* __restrict__ v = A.val + row;
#pragma unroll 8
    for (int d = 0; d < A.ndiag; ++d) {
      const int j = row + A.off[d];
      const double a = __ldg(v + (int64_t)d * n);
      if ((unsigned)j < (unsigned)A.n_cols) acc = fma(a, fma(beta, __ldg(x2 + j), __ldg(x1 + j)), acc);
    }
    return acc;
  }
  const int s = row >> 5, lane = row & 31;
  const int64_t end = A.slice_ptr[s + 1];
  for (int64_t k = A.slice_ptr[s] + lane; k < end; k += 32) {
    const int c = __ldg(A.col + k);
    acc = fma(__ldg(A.val + k), fma(beta, __ldg(x2 + c), __ldg(x1 + c)), acc);
  }
  return acc;
}

// True for the one thread that writes row `row` (lane 0 of its group).
template <typename T>
__device__ __forceinline__ bool row_leader(const DevSell<T>& A, int64_t tid, int n) {
  return (int)(tid >> A.logG) < n && (A.G <= 1 || (tid & (A.G - 1)) == 0);
}

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }

// ------------------------------------------------------------ V-cycle pieces
// Row kernels use resident-sized grids: a grid-stride loop in which every
// thread keeps two rows (t and t + stride) in flight, loading both before
// any store.  Loop bounds are multiples of 32, so warps stay converged for
// the G-lane shuffles.
#define EQS_ROWS2(A_, n_, BODY2)                                              \
  const int64_t lim_ = round32((int64_t)(n_) << (A_).logG);                   \
  const int64_t st_ = (int64_t)gridDim.x * blockDim.x;                        \
  for (int64_t t0 = gtid(); t0 < lim_; t0 += 2 * st_) {                       \
    const int64_t t1 = t0 + st_;                                               \
    BODY2                                                                      \
  }

__device__ __forceinline__ int64_t round32(int64_t v) { return (v + 31) & ~(int64_t)31; }

// One Chebyshev step:  r_out = r_in - A d_in ;  d_out = c1 d_in + c2 D^-1 r_out ;
// x += d_out (+ d_in when the previous direction was not yet added to x).
template <typename T>
__global__ void __launch_bounds__(kBlock, 4)
k_cheb_step(DevSell<T> A, int n, const T* r_in, const T* __restrict__ d_in,
            const T* __restrict__ dinv, T c1, T c2, T* r_out, T* __restrict__ d_out,
            T* __restrict__ x, int add_pending) {
  pdl_enter();
  EQS_ROWS2(A, n, {
    const T a0 = mat_row(A, t0, n, d_in);
    const T a1 = mat_row(A, t1, n, d_in);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = h ? t1 : t0;
      if (!row_leader(A, t, n)) continue;
      const int i = (int)(t >> A.logG);
      const T di = d_in[i];
      const T r = r_in[i] - (h ? a1 : a0);
      const T dn = c1 * di + c2 * dinv[i] * r;
      r_out[i] = r;
      d_out[i] = dn;
      x[i] += add_pending ? dn + di : dn;
    }
  })
}

// r -= A d  (in place; r is row-local)
template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_resid_update(DevSell<T> A, int n, T* r, const T* __restrict__ d) {
  pdl_enter();
  EQS_ROWS2(A, n, {
    const T a0 = mat_row(A, t0, n, d);
    const T a1 = mat_row(A, t1, n, d);
    if (row_leader(A, t0, n)) r[t0 >> A.logG] -= a0;
    if (row_leader(A, t1, n)) r[t1 >> A.logG] -= a1;
  })
}

// out = b - A x
template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_resid(DevSell<T> A, int n, const T* __restrict__ b, const T* __restrict__ x,
                        T* __restrict__ out) {
  pdl_enter();
  EQS_ROWS2(A, n, {
    const T a0 = mat_row(A, t0, n, x);
    const T a1 = mat_row(A, t1, n, x);
    if (row_leader(A, t0, n)) out[t0 >> A.logG] = b[t0 >> A.logG] - a0;
    if (row_leader(A, t1, n)) out[t1 >> A.logG] = b[t1 >> A.logG] - a1;
  })
}

// b_c = R r_f ; when first_step: x_c = d_c = D_c^-1 b_c / theta_c (the first
// Chebyshev step of the coarse level from a zero initial guess).
template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_restrict(DevSell<T> R, int nc, const T* __restrict__ rf, T* __restrict__ bc,
                           const T* __restrict__ dinv_c, T inv_theta_c, T* __restrict__ xc,
                           T* __restrict__ dc, int first_step) {
  pdl_enter();
  EQS_ROWS2(R, nc, {
    const T b0 = mat_row(R, t0, nc, rf);
    const T b1 = mat_row(R, t1, nc, rf);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = h ? t1 : t0;
      if (!row_leader(R, t, nc)) continue;
      const int i = (int)(t >> R.logG);
      const T b = h ? b1 : b0;
      bc[i] = b;
      if (first_step) {
        const T d = dinv_c[i] * b * inv_theta_c;
        xc[i] = d;
        dc[i] = d;
      }
    }
  })
}

// x_f += P x_c, or P (x_c + d_c) when the coarse level's last Chebyshev
// direction d_c is still pending
template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_prolong(DevSell<T> P, int nf, const T* __restrict__ xc,
                                                       const T* __restrict__ dc, T* __restrict__ xf) {
  pdl_enter();
  EQS_ROWS2(P, nf, {
    const T p0 = dc ? mat_row_add(P, t0, nf, xc, dc) : mat_row(P, t0, nf, xc);
    const T p1 = dc ? mat_row_add(P, t1, nf, xc, dc) : mat_row(P, t1, nf, xc);
    if (row_leader(P, t0, nf)) xf[t0 >> P.logG] += p0;
    if (row_leader(P, t1, nf)) xf[t1 >> P.logG] += p1;
  })
}

// First post-smoothing step from the current x: r = b - A x ; d = D^-1 r / theta.
// x is not updated here (other rows still read it); the next step adds d.
template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_post_first(DevSell<T> A, int n, const T* __restrict__ b,
                             const T* __restrict__ x, const T* __restrict__ dinv, T inv_theta,
                             T* __restrict__ r_out, T* __restrict__ d_out, int write_iterate) {
  pdl_enter();
  EQS_ROWS2(A, n, {
    const T a0 = mat_row(A, t0, n, x);
    const T a1 = mat_row(A, t1, n, x);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = h ? t1 : t0;
      if (!row_leader(A, t, n)) continue;
      const int i = (int)(t >> A.logG);
      const T r = b[i] - (h ? a1 : a0);
      if (r_out) r_out[i] = r;  // read by the Chebyshev steps of degree >= 2
      const T d = dinv[i] * r * inv_theta;
      d_out[i] = write_iterate ? x[i] + d : d;  // degree 1: the smoothed iterate
    }
  })
}

template <typename T>
__global__ void k_axpy1(int n, T* __restrict__ x, const T* __restrict__ d) {
  pdl_enter();
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] += d[i];
}

// Coarsest level: x = A_c^-1 b with the dense FP64 inverse; one warp per
// row.  b is staged once per block in shared memory as FP64 (dynamic shared
// memory of n doubles), so the inner loop has no conversions; two
// accumulation chains per lane.
template <typename T>
__global__ void k_coarse_solve(int n, const double* __restrict__ inv, const T* __restrict__ b,
                               T* __restrict__ x) {
  extern __shared__ double sb[];
  pdl_enter();
  for (int j = threadIdx.x; j < n; j += blockDim.x) sb[j] = (double)b[j];
  __syncthreads();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* __restrict__ row = inv + (int64_t)warp * n;
  double a0 = 0.0, a1 = 0.0;
  int j = lane;
  for (; j + 32 < n; j += 64) {
    a0 = fma(__ldg(row + j), sb[j], a0);
    a1 = fma(__ldg(row + j + 32), sb[j + 32], a1);
  }
  if (j < n) a0 = fma(__ldg(row + j), sb[j], a0);
  double acc = a0 + a1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[warp] = (T)acc;
}

// ---------------------------------------------------------------- reductions
// Warp sum of NV doubles by recursive halving: at offset o every lane keeps
// half of its remaining values (the upper half when bit o of its lane is
// set) and adds the partner's copy of that half, so the warp spends about
// NV shuffles and adds instead of 5 NV.  Afterwards every lane holds full
// sums of a run of values and stores them to out[] (lanes that hold the same
// values store the same sums).
__host__ __device__ constexpr int pow2_at_least(int v) { return v <= 1 ? 1 : 2 * pow2_at_least((v + 1) / 2); }

template <int NV>
__device__ __forceinline__ void warp_sum_scatter(const double (&v)[NV], double* out) {
  constexpr int P = pow2_at_least(NV);
  static_assert(NV <= 64, "warp_sum_scatter handles up to 64 values");
  const int lane = threadIdx.x & 31;
  double w[P];
#pragma unroll
  for (int k = 0; k < P; ++k) w[k] = k < NV ? v[k] : 0.0;
  int cnt = P, base = 0;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    if (cnt > 1) {
      const int half = cnt / 2;
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int k = 0; k < P / 2; ++k) {
        if (k >= half) break;
        const double send = up ? w[k] : w[k + half];
        const double keep = up ? w[k + half] : w[k];
        w[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
      if (up) base += half;
      cnt = half;
    } else {
      w[0] += __shfl_xor_sync(0xffffffffu, w[0], o);
    }
  }
  // each lane now holds the full sums of values base .. base + cnt - 1
#pragma unroll
  for (int k = 0; k < (P > 32 ? P / 32 : 1); ++k)
    if (base + k < NV) out[base + k] = w[k];  // lanes of a group write the same value
}

// Block sum of NV doubles (any block size up to 1024 threads, a multiple of
// 32); result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  __shared__ double tot_s[NV];
  const int nw = (int)(blockDim.x >> 5);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (NV >= 4) {
    __shared__ double part[32][NV];
    warp_sum_scatter<NV>(v, part[w]);
    __syncthreads();
    if (w == 0) {
      double t[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) t[k] = lane < nw ? part[lane][k] : 0.0;
      warp_sum_scatter<NV>(t, tot_s);
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k] = tot_s[k];
    __syncthreads();
    return;
  }
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][w] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < nw ? sh[k][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      v[k] = t;
    }
  }
  __syncthreads();
}

// Grid-wide deterministic sum: every block stores its partials; the last
// block to finish (atomic ticket) sums them in block order and returns true
// in all of its threads with the totals in `tot` (thread 0).
// Arrival of this block after its partials are written (thread 0 has
// written them): true in every thread of the last block to arrive.
__device__ __forceinline__ bool grid_ticket(unsigned int* counter) {
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    __threadfence();
    // two-level ticket: blocks arrive on one of 8 group counters (counter[1..8]);
    // the last block of each group arrives on counter[0]
    const unsigned int grp = blockIdx.x & 7u;
    const unsigned int in_grp = (gridDim.x - grp + 7u) / 8u;  // blocks with this residue
    bool last = false;
    if (atomicAdd(counter + 1 + grp, 1u) == in_grp - 1u) {
      counter[1 + grp] = 0u;
      __threadfence();  // order the group's arrivals before the main ticket
      const unsigned int groups = gridDim.x < 8u ? gridDim.x : 8u;
      last = atomicAdd(counter, 1u) == groups - 1u;
    }
    am_last = last;
  }
  __syncthreads();
  return am_last;
}

template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials, unsigned int* counter,
                                         int max_blocks, double (&tot)[NV]) {
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[k * max_blocks + blockIdx.x] = v[k];
  }
  if (!grid_ticket(counter)) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(partials + k * max_blocks + b);
    tot[k] = t;
  }
  block_sum<NV>(tot);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// Deferred sums (the CG's consumer-side reductions): a producer kernel ends
// with its block sums in part[k * cap + block] and no grid-wide step; every
// block of the consuming kernel adds the nb partials itself, in a fixed
// order, so all blocks hold the same totals -- no atomic ticket, no fence
// and no serial last block between the two kernels.
template <int NV>
__device__ __forceinline__ void write_partials(double (&v)[NV], double* __restrict__ part, int cap) {
  block_sum<NV>(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) part[k * cap + blockIdx.x] = v[k];
}

template <int NV>
__device__ __forceinline__ void sum_partials(const double* __restrict__ part, int nb, int cap, double (&tot)[NV]) {
  __shared__ double bc[NV];
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += __ldcg(part + k * cap + b);
  block_sum<NV>(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) bc[k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = bc[k];
}

// ------------------------------------------------------------------ PCG
// CG kernels run grid-stride over rows with a capped grid (fewer blocks take
// part in the atomic ticket of each grid reduction).
//
// Initial residual r = R - M x, norms of R and r, and the first V-cycle
// input (b0 = r in T, x0 = d0 = D0^-1 b0 / theta0).  The last block decides
// whether the CG loop runs (condition handle).
template <typename T>
__global__ void k_pcg_init(DevSell<double> M, int n, const double* __restrict__ R,
                           const double* __restrict__ x, double* __restrict__ r,
                           const T* __restrict__ dinv0, T inv_theta0, T* __restrict__ b0,
                           T* __restrict__ x0, T* __restrict__ d0, PcgScalars* sc,
                           double* partials, unsigned int* counter, int max_blocks, double tol2,
                           int maxit, cudaGraphConditionalHandle h, int use_handle,
                           int* iters_out, double* relres_out, int* zero_out) {
  pdl_enter();
  double v[2] = {0.0, 0.0};
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double Ri = R[i];
    const double ri = Ri - mat_row<double>(M, i, n, x);
    r[i] = ri;
    const T bi = vc_in<T>(ri);
    b0[i] = bi;
    const T d = dinv0[i] * bi * inv_theta0;
    x0[i] = d;
    d0[i] = d;
    v[0] += Ri * Ri;
    v[1] += ri * ri;
  }
  double tot[2];
  if (grid_sum<2>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    sc->bnorm2 = tot[0];
    sc->rnorm2 = tot[1];
    sc->it = 0;
    sc->parity = 0;
    const int zero = tot[0] == 0.0;
    const int go = !zero && tot[1] > tol2 * tot[0] && maxit > 0;
    sc->conv = !go;
    if (use_handle) cudaGraphSetConditional(h, go ? 1u : 0u);
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = zero ? 0.0 : sqrt(tot[1] / tot[0]);
    if (zero_out) *zero_out = zero;
  }
}

// Start from the learned guess x unless the previous solution h1 has the
// smaller residual: r = R - M x, rtmp = R - M h1, norms of R, r, rtmp; the
// last block records the choice (sc->use_prev) and sets the loop condition.
template <typename T>
__global__ void k_pcg_init_dual(DevSell<double> M, int n, const double* __restrict__ R,
                                const double* __restrict__ x, const double* __restrict__ h1,
                                double* __restrict__ r, double* __restrict__ rtmp,
                                const T* __restrict__ dinv0, T inv_theta0, T* __restrict__ b0,
                                T* __restrict__ x0, T* __restrict__ d0, PcgScalars* sc,
                                double* partials, unsigned int* counter, int max_blocks, double tol2,
                                int maxit, cudaGraphConditionalHandle h, int use_handle,
                                int* iters_out, double* relres_out, int* zero_out, int* kept_out) {
  pdl_enter();
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double Ri = R[i];
    const double r1 = Ri - mat_row<double>(M, i, n, x);
    const double r2 = Ri - mat_row<double>(M, i, n, h1);
    r[i] = r1;
    rtmp[i] = r2;
    const T bi = vc_in<T>(r1);
    b0[i] = bi;
    const T d = dinv0[i] * bi * inv_theta0;
    x0[i] = d;
    d0[i] = d;
    v[0] += Ri * Ri;
    v[1] += r1 * r1;
    v[2] += r2 * r2;
  }
  double tot[3];
  if (grid_sum<3>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    const int prev = tot[2] < tot[1];
    const double rn = prev ? tot[2] : tot[1];
    sc->bnorm2 = tot[0];
    sc->rnorm2 = rn;
    sc->it = 0;
    sc->parity = 0;
    sc->use_prev = prev;
    const int zero = tot[0] == 0.0;
    const int go = !zero && rn > tol2 * tot[0] && maxit > 0;
    sc->conv = !go;
    if (use_handle) cudaGraphSetConditional(h, go ? 1u : 0u);
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = zero ? 0.0 : sqrt(rn / tot[0]);
    if (zero_out) *zero_out = zero;
    if (kept_out) *kept_out = !prev;
  }
}

// Fallback of k_pcg_init_dual: x = h1, r = rtmp and the V-cycle input.
template <typename T>
__global__ void k_pcg_select(int n, double* __restrict__ x, const double* __restrict__ h1,
                             double* __restrict__ r, const double* __restrict__ rtmp,
                             const T* __restrict__ dinv0, T inv_theta0, T* __restrict__ b0,
                             T* __restrict__ x0, T* __restrict__ d0, const PcgScalars* sc) {
  pdl_enter();
  if (!sc->use_prev) return;
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = h1[i];
    const double ri = rtmp[i];
    r[i] = ri;
    const T bi = vc_in<T>(ri);
    b0[i] = bi;
    const T d = dinv0[i] * bi * inv_theta0;
    x0[i] = d;
    d0[i] = d;
  }
}

// z (from the V-cycle, in T) to FP64 (zd) or, for the split-M operator
// pass, kept in FP32 (z32); r.z and r_prev.z; the last block forms beta
// (Fletcher-Reeves, or Polak-Ribiere when flexible).
template <typename T>
__global__ void k_pcg_dots(int n, const double* __restrict__ r, const double* __restrict__ rprev,
                           const T* __restrict__ z, const T* __restrict__ zpend, double* __restrict__ zd,
                           float* __restrict__ z32, PcgScalars* sc, double* partials, unsigned int* counter,
                           int max_blocks, int flexible) {
  pdl_enter();
  double v[2] = {0.0, 0.0};
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T zt = zpend ? z[i] + zpend[i] : z[i];
    const double zi = widen(zt);
    if (z32)
      z32[i] = (float)zt;
    else
      zd[i] = zi;
    v[0] += r[i] * zi;
    v[1] += rprev[i] * zi;
  }
  double tot[2];
  if (grid_sum<2>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    const double rz = tot[0];
    double beta = 0.0;
    if (sc->it > 0) beta = flexible ? (rz - tot[1]) / sc->rz_old : rz / sc->rz_old;
    sc->beta = beta;
    sc->rz = rz;
    sc->rz_old = rz;
  }
}

// Level-0 post-smoothing step of a degree-1 V-cycle fused with the CG dot
// products: r = b - A x, d = D^-1 r / theta, and the preconditioned residual
// z = x + d (FP32 z32 for the split-M operator pass, else FP64 zd); sums
// r_cg.z and r_prev.z; the last block forms beta (as k_pcg_dots).  Saves
// one kernel per CG iteration: every value it needs is row-local.
// DEFER: the two sums are left as per-block partials in dpart (the split-M
// operator pass adds them and forms beta).
template <typename T, bool DEFER>
__global__ void __launch_bounds__(kBlock, 4)
k_post_first_dots(DevSell<T> A, int n, const T* __restrict__ b, const T* __restrict__ x,
                  const T* __restrict__ dinv, T inv_theta, const double* __restrict__ rcg,
                  const double* __restrict__ rprev, double* __restrict__ zd, float* __restrict__ z32,
                  PcgScalars* sc, double* partials, unsigned int* counter, int max_blocks, int flexible,
                  double* __restrict__ dpart) {
  pdl_enter();
  double v[2] = {0.0, 0.0};
  EQS_ROWS2(A, n, {
    const T a0 = mat_row(A, t0, n, x);
    const T a1 = mat_row(A, t1, n, x);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = h ? t1 : t0;
      if (!row_leader(A, t, n)) continue;
      const int i = (int)(t >> A.logG);
      const T r = b[i] - (h ? a1 : a0);
      const T zt = x[i] + dinv[i] * r * inv_theta;
      const double zi = widen(zt);
      if (z32)
        z32[i] = (float)zt;
      else
        zd[i] = zi;
      v[0] += rcg[i] * zi;
      v[1] += rprev[i] * zi;
    }
  })
  if constexpr (DEFER) {
    write_partials<2>(v, dpart, max_blocks);
    return;
  }
  double tot[2];
  if (grid_sum<2>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    const double rz = tot[0];
    double beta = 0.0;
    if (sc->it > 0) beta = flexible ? (rz - tot[1]) / sc->rz_old : rz / sc->rz_old;
    sc->beta = beta;
    sc->rz = rz;
    sc->rz_old = rz;
  }
}

// p = z + beta p and q = M p through q = M z + beta q (M p_old = q_old), so
// p and q stay row-local and M costs one FMA per non-zero; p.q and alpha.
__global__ void k_pcg_pq(DevSell<double> M, int n, const double* __restrict__ zd, double* __restrict__ p,
                         double* __restrict__ q, PcgScalars* sc, double* partials,
                         unsigned int* counter, int max_blocks) {
  pdl_enter();
  const double beta = sc->beta;
  double v[1] = {0.0};
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = gtid(); i0 < n; i0 += 2 * st) {  // two rows in flight per thread
    const int64_t i1 = i0 + st;
    const double w0 = mat_row<double>(M, i0, n, zd);
    const double w1 = mat_row<double>(M, i1, n, zd);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t i = h ? i1 : i0;
      if (i >= n) continue;
      const double w = h ? w1 : w0;
      const double qi = beta == 0.0 ? w : fma(beta, q[i], w);
      const double pi = beta == 0.0 ? zd[i] : fma(beta, p[i], zd[i]);
      p[i] = pi;
      q[i] = qi;
      v[0] += pi * qi;
    }
  }
  double tot[1];
  if (grid_sum<1>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    sc->pq = tot[0];
    sc->alpha = sc->rz / tot[0];
  }
}

// ------------------------------------------------ split-M operator pass
// M z with M stored as two FP32 parts (M = M_hi + M_lo to about 2^-48) and z
// exactly FP32 (the V-cycle output of the mixed path): every product M_hi z
// is split exactly into p + e by an FMA, M_lo z is rounded to FP32 (it is
// 2^-24 smaller), and the row sum is carried as an unevaluated FP32 pair
// (S, s) with an error-free two-sum per term.  The result is accurate to a
// few units of 2^-48 of sum |m_ij z_j| -- FP64-class for the CG operator --
// but uses the FP32 pipe, 62x faster than FP64 on GB300.  The __f*_rn forms
// keep the compiler from contracting the error-free steps.
__device__ __forceinline__ void df_acc(float& S, float& s, float ah, float al, float z) {
  const float p = __fmul_rn(ah, z);
  const float e = __fmaf_rn(ah, z, -p);  // ah z = p + e exactly
  const float t = __fmaf_rn(al, z, e);
  const float S1 = __fadd_rn(S, p);
  const float bv = __fsub_rn(S1, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(S1, bv)), __fsub_rn(p, bv));  // S + p = S1 + err
  S = S1;
  s = __fadd_rn(s, __fadd_rn(err, t));
}

__device__ __forceinline__ double mat_row_split(const DevSell<double>& A, const float* __restrict__ hi,
                                                const float* __restrict__ lo, int64_t row, int n,
                                                const float* __restrict__ z) {
  float S = 0.0f, s = 0.0f;
  if (row >= n) return 0.0;
  if (A.G == 0) {  // chunks of diagonals: all loads before the sums
    constexpr int CH = kDiaChunk;
    for (int d0 = 0; d0 < A.ndiag; d0 += CH) {
      float ah[CH], al[CH], zz[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int d = d0 + u;
        const int j = (int)row + A.off[d < kMaxDiag ? d : 0];
        const bool ok = d < A.ndiag && (unsigned)j < (unsigned)A.n_cols;
        const int64_t k = (int64_t)d * n + row;
        ah[u] = ok ? __ldg(hi + k) : 0.0f;
        al[u] = ok ? __ldg(lo + k) : 0.0f;
        zz[u] = ok ? __ldg(z + j) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) df_acc(S, s, ah[u], al[u], zz[u]);
    }
  } else {
    const int64_t sl = row >> 5, lane = row & 31;
    const int64_t end = A.slice_ptr[sl + 1];
    for (int64_t k = A.slice_ptr[sl] + lane; k < end; k += 32)
      df_acc(S, s, __ldg(hi + k), __ldg(lo + k), __ldg(z + __ldg(A.col + k)));
  }
  return f2d(S) + f2d(s);
}

// k_pcg_pq with the split-M product: q = M z + beta q_old, p = z + beta p,
// p.q and alpha (z in FP32).  DEFER: every block first adds the nb_in
// partials of r.z and r_prev.z left by k_post_first_dots (dpart) and forms
// beta itself (block 0 records r.z by iteration parity in sc->rz_hist), and
// p.q is left as per-block partials (dpart + 2 cap) for k_pcg_update.
template <bool DEFER>
__global__ void k_pcg_pq_split(DevSell<double> M, const float* __restrict__ Mhi,
                               const float* __restrict__ Mlo, int n, const float* __restrict__ z32,
                               double* __restrict__ p, double* __restrict__ q, PcgScalars* sc,
                               double* partials, unsigned int* counter, int max_blocks,
                               double* __restrict__ dpart, int nb_in, int flexible) {
  pdl_enter();
  double beta;
  if constexpr (DEFER) {
    double d[2];
    sum_partials<2>(dpart, nb_in, max_blocks, d);
    const int it = sc->it;
    beta = 0.0;
    if (it > 0) beta = (flexible ? d[0] - d[1] : d[0]) / sc->rz_hist[(it + 1) & 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->rz_hist[it & 1] = d[0];
  } else {
    beta = sc->beta;
  }
  double v[1] = {0.0};
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = gtid(); i0 < n; i0 += 2 * st) {  // two rows in flight per thread
    const int64_t i1 = i0 + st;
    const double w0 = mat_row_split(M, Mhi, Mlo, i0, n, z32);
    const double w1 = mat_row_split(M, Mhi, Mlo, i1, n, z32);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t i = h ? i1 : i0;
      if (i >= n) continue;
      const double w = h ? w1 : w0;
      const double zi = f2d(z32[i]);
      const double qi = beta == 0.0 ? w : fma(beta, q[i], w);
      const double pi = beta == 0.0 ? zi : fma(beta, p[i], zi);
      p[i] = pi;
      q[i] = qi;
      v[0] += pi * qi;
    }
  }
  if constexpr (DEFER) {
    write_partials<1>(v, dpart + 2 * (size_t)max_blocks, max_blocks);
    return;
  }
  double tot[1];
  if (grid_sum<1>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    sc->pq = tot[0];
    sc->alpha = sc->rz / tot[0];
  }
}

// x += alpha p ; r_prev = r ; r -= alpha q ; ||r||^2 ; next V-cycle input;
// the last block updates the loop condition and the statistics.  DEFER:
// every block adds the nb_in partials of p.q (dpart + 2 cap) and forms
// alpha = r.z / p.q itself.
template <typename T, bool DEFER>
__global__ void k_pcg_update(int n, double* __restrict__ x, double* __restrict__ r,
                             double* __restrict__ rprev, const double* __restrict__ p,
                             const double* __restrict__ q, const T* __restrict__ dinv0,
                             T inv_theta0, T* __restrict__ b0, T* __restrict__ x0,
                             T* __restrict__ d0, PcgScalars* sc, double* partials,
                             unsigned int* counter, int max_blocks, double tol2, int maxit,
                             cudaGraphConditionalHandle h, int use_handle, int* iters_out,
                             double* relres_out, const double* __restrict__ dpart, int nb_in) {
  pdl_enter();
  double a;
  if constexpr (DEFER) {
    double pq[1];
    sum_partials<1>(dpart + 2 * (size_t)max_blocks, nb_in, max_blocks, pq);
    a = sc->rz_hist[sc->it & 1] / pq[0];
  } else {
    a = sc->alpha;
  }
  double v[1] = {0.0};
  for (int64_t i = gtid(); i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    const double ro = r[i];
    rprev[i] = ro;
    const double rn = fma(-a, q[i], ro);
    r[i] = rn;
    v[0] += rn * rn;
    const T bi = vc_in<T>(rn);
    b0[i] = bi;
    const T d = dinv0[i] * bi * inv_theta0;
    x0[i] = d;
    d0[i] = d;
  }
  double tot[1];
  if (grid_sum<1>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    sc->rnorm2 = tot[0];
    const int it = sc->it + 1;
    sc->it = it;
    const int conv = tot[0] <= tol2 * sc->bnorm2;
    sc->conv = conv;
    const int go = !conv && it < maxit;
    if (use_handle) cudaGraphSetConditional(h, go ? 1u : 0u);
    if (iters_out) *iters_out = it;
    // the final relative residual only when the loop ends (a division and a
    // square root are long FP64 chains in this one-thread tail)
    if (relres_out && !go) *relres_out = sqrt(tot[0] / sc->bnorm2);
  }
}

// ---------------------------------------------------------- element kernels
// One thread per tet (Section III): gather the 4 vertices and potentials,
// form the gradient and kappa(|E|), and add r_e = kappa V G (G^T phi_e) to y
// (only rows < n_limit).  With e_k = p_k - p_0 and c_1 = e_2 x e_3,
// c_2 = e_3 x e_1, c_3 = e_1 x e_2, D = e_1 . c_1 = det J = 6V:
//   grad(lambda_k) = c_k / D,  grad phi = g / D,  g = sum_k (phi_k - phi_0) c_k
//   r_k = kappa V grad(lambda_k) . grad phi = kappa (c_k . g) / (6 D),
//   r_0 = -(r_1 + r_2 + r_3).
__device__ __forceinline__ double kappa64(const MaterialDev& m, double E) {
  if (m.is_const) return m.klo;
  const double u = (E - m.E0) * m.inv_w;
  double s;
  if (u >= 0.0) {
    s = 1.0 / (1.0 + exp(-u));
  } else {
    const double e = exp(u);
    s = e / (1.0 + e);
  }
  return m.klo + (m.khi - m.klo) * s;
}

// FP32 conductivity from the table's FP32 copies (no FP64 conversions:
// they run on GB300's slow FP64 pipe).
__device__ __forceinline__ float kappa32(const MaterialDev& m, float E) {
  if (m.is_const) return m.klo_f;
  const float u = (E - m.E0_f) * m.inv_w_f;
  float s;
  if (u >= 0.0f) {
    s = 1.0f / (1.0f + expf(-u));
  } else {
    const float e = expf(u);
    s = e / (1.0f + e);
  }
  return m.klo_f + m.dk_f * s;
}

__global__ void k_elem64(int64_t nt, const int4* __restrict__ conn, const uint8_t* __restrict__ mat,
                         const MaterialDev* __restrict__ mats, const double4* __restrict__ xyz,
                         const double* __restrict__ x, int n_limit, double sign,
                         double* __restrict__ y) {
  pdl_enter();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  const int4 t = conn[e];
  const double4 p0 = xyz[t.x], p1 = xyz[t.y], p2 = xyz[t.z], p3 = xyz[t.w];
  const double f0 = __ldg(x + t.x);
  const double d1 = __ldg(x + t.y) - f0, d2 = __ldg(x + t.z) - f0, d3 = __ldg(x + t.w) - f0;
  const double e1x = p1.x - p0.x, e1y = p1.y - p0.y, e1z = p1.z - p0.z;
  const double e2x = p2.x - p0.x, e2y = p2.y - p0.y, e2z = p2.z - p0.z;
  const double e3x = p3.x - p0.x, e3y = p3.y - p0.y, e3z = p3.z - p0.z;
  const double c1x = e2y * e3z - e2z * e3y, c1y = e2z * e3x - e2x * e3z, c1z = e2x * e3y - e2y * e3x;
  const double c2x = e3y * e1z - e3z * e1y, c2y = e3z * e1x - e3x * e1z, c2z = e3x * e1y - e3y * e1x;
  const double c3x = e1y * e2z - e1z * e2y, c3y = e1z * e2x - e1x * e2z, c3z = e1x * e2y - e1y * e2x;
  const double invD = 1.0 / (e1x * c1x + e1y * c1y + e1z * c1z);
  const double gx = d1 * c1x + d2 * c2x + d3 * c3x;
  const double gy = d1 * c1y + d2 * c2y + d3 * c3y;
  const double gz = d1 * c1z + d2 * c2z + d3 * c3z;
  const MaterialDev m = mats[mat[e]];
  double kap;
  if (m.is_const) {
    kap = m.klo;
  } else {
    const double E = sqrt(gx * gx + gy * gy + gz * gz) * invD;
    kap = kappa64(m, E);
  }
  const double s = sign * kap * (invD * (1.0 / 6.0));
  const double r1 = s * (c1x * gx + c1y * gy + c1z * gz);
  const double r2 = s * (c2x * gx + c2y * gy + c2z * gz);
  const double r3 = s * (c3x * gx + c3y * gy + c3z * gz);
  const double r0 = -(r1 + r2 + r3);
  if (t.x < n_limit) atomicAdd(y + t.x, r0);
  if (t.y < n_limit) atomicAdd(y + t.y, r1);
  if (t.z < n_limit) atomicAdd(y + t.z, r2);
  if (t.w < n_limit) atomicAdd(y + t.w, r3);
}

// Mixed precision: coordinates and potentials are stored as FP32 (hi, lo)
// pairs, so edge vectors and potential differences are formed as
// (hi_a - hi_b) + (lo_a - lo_b) with FP32 relative accuracy; everything else
// is FP32 with FP32 accumulation.  r_0 = -(r_1 + r_2 + r_3) keeps the
// local residual's zero sum exactly.
__device__ __forceinline__ void elem32_tet(int64_t e, const int4* __restrict__ conn,
                                           const uint8_t* __restrict__ mat,
                                           const MaterialDev* __restrict__ mats,
                                           const float4* __restrict__ xh, const float4* __restrict__ xl,
                                           const float2* __restrict__ x, int n_limit, float* __restrict__ y) {
  const int4 t = conn[e];
  const float4 h0 = xh[t.x], h1 = xh[t.y], h2 = xh[t.z], h3 = xh[t.w];
  const float4 l0 = xl[t.x], l1 = xl[t.y], l2 = xl[t.z], l3 = xl[t.w];
  const float2 f0 = x[t.x], f1 = x[t.y], f2 = x[t.z], f3 = x[t.w];
  const float d1 = (f1.x - f0.x) + (f1.y - f0.y);
  const float d2 = (f2.x - f0.x) + (f2.y - f0.y);
  const float d3 = (f3.x - f0.x) + (f3.y - f0.y);
  const float e1x = (h1.x - h0.x) + (l1.x - l0.x), e1y = (h1.y - h0.y) + (l1.y - l0.y),
              e1z = (h1.z - h0.z) + (l1.z - l0.z);
  const float e2x = (h2.x - h0.x) + (l2.x - l0.x), e2y = (h2.y - h0.y) + (l2.y - l0.y),
              e2z = (h2.z - h0.z) + (l2.z - l0.z);
  const float e3x = (h3.x - h0.x) + (l3.x - l0.x), e3y = (h3.y - h0.y) + (l3.y - l0.y),
              e3z = (h3.z - h0.z) + (l3.z - l0.z);
  const float c1x = e2y * e3z - e2z * e3y, c1y = e2z * e3x - e2x * e3z, c1z = e2x * e3y - e2y * e3x;
  const float c2x = e3y * e1z - e3z * e1y, c2y = e3z * e1x - e3x * e1z, c2z = e3x * e1y - e3y * e1x;
  const float c3x = e1y * e2z - e1z * e2y, c3y = e1z * e2x - e1x * e2z, c3z = e1x * e2y - e1y * e2x;
  const float invD = 1.0f / (e1x * c1x + e1y * c1y + e1z * c1z);
  const float gx = d1 * c1x + d2 * c2x + d3 * c3x;
  const float gy = d1 * c1y + d2 * c2y + d3 * c3y;
  const float gz = d1 * c1z + d2 * c2z + d3 * c3z;
  const MaterialDev m = mats[mat[e]];
  float kap;
  if (m.is_const) {
    kap = m.klo_f;
  } else {
    const float E = sqrtf(gx * gx + gy * gy + gz * gz) * invD;
    kap = kappa32(m, E);
  }
  const float s = kap * (invD * (1.0f / 6.0f));
  const float r1 = s * (c1x * gx + c1y * gy + c1z * gz);
  const float r2 = s * (c2x * gx + c2y * gy + c2z * gz);
  const float r3 = s * (c3x * gx + c3y * gy + c3z * gz);
  const float r0 = -(r1 + r2 + r3);
  if (t.x < n_limit) atomicAdd(y + t.x, r0);
  if (t.y < n_limit) atomicAdd(y + t.y, r1);
  if (t.z < n_limit) atomicAdd(y + t.z, r2);
  if (t.w < n_limit) atomicAdd(y + t.w, r3);
}

__global__ void k_elem32(int64_t nt, const int4* __restrict__ conn, const uint8_t* __restrict__ mat,
                         const MaterialDev* __restrict__ mats, const float4* __restrict__ xh,
                         const float4* __restrict__ xl, const float2* __restrict__ x,
                         int n_limit, float* __restrict__ y) {
  pdl_enter();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  elem32_tet(e, conn, mat, mats, xh, xl, x, n_limit, y);
}

// kappa(|E|) in the element's working precision.
template <typename R>
__device__ __forceinline__ R kappa_of(const MaterialDev& m, R E);
template <>
__device__ __forceinline__ double kappa_of<double>(const MaterialDev& m, double E) { return kappa64(m, E); }
template <>
__device__ __forceinline__ float kappa_of<float>(const MaterialDev& m, float E) { return kappa32(m, E); }
template <typename R>
__device__ __forceinline__ R kappa_lo(const MaterialDev& m);
template <>
__device__ __forceinline__ double kappa_lo<double>(const MaterialDev& m) { return m.klo; }
template <>
__device__ __forceinline__ float kappa_lo<float>(const MaterialDev& m) { return m.klo_f; }

// ------------------------------------------------ Kuhn-cell element kernels
// Meshes whose tets come in groups of six forming one Kuhn-split hexahedron
// (detected at setup): one thread per cell loads the cell's 8 corners and
// potentials once, forms the six tets' residuals (the same arithmetic as
// the per-tet kernels) into 8 corner sums and issues 8 atomic adds instead
// of 24.  Corner c = bx + 2 by + 4 bz; the six tets of a cell have the
// corners (0,1,3,7), (0,1,7,5), (0,2,7,3), (0,2,6,7), (0,4,5,7), (0,4,7,6)
// (the vertex order of the mesh: positive orientation).

// The tet's cofactor vectors c_k = e_l x e_m (k = 1..3; grad lambda_k =
// c_k / D with D = e_1 . c_1 = 6 V) and 1/D: formed once per tet and shared
// by every potential column it carries, so a tet pays one division.
template <typename R>
struct TetGeom {
  R c[3][3];
  R invD;
};

template <typename R>
__device__ __forceinline__ TetGeom<R> tet_geom(const R (&e)[3][3]) {
  TetGeom<R> g;
  g.c[0][0] = e[1][1] * e[2][2] - e[1][2] * e[2][1];
  g.c[0][1] = e[1][2] * e[2][0] - e[1][0] * e[2][2];
  g.c[0][2] = e[1][0] * e[2][1] - e[1][1] * e[2][0];
  g.c[1][0] = e[2][1] * e[0][2] - e[2][2] * e[0][1];
  g.c[1][1] = e[2][2] * e[0][0] - e[2][0] * e[0][2];
  g.c[1][2] = e[2][0] * e[0][1] - e[2][1] * e[0][0];
  g.c[2][0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
  g.c[2][1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
  g.c[2][2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
  g.invD = R(1) / (e[0][0] * g.c[0][0] + e[0][1] * g.c[0][1] + e[0][2] * g.c[0][2]);
  return g;
}

// One potential column of a tet: D grad u = sum_k d_k c_k (d_k = u_k - u_0),
// |E| = |D grad u| / D, and r_k = V kappa grad lambda_k . grad u =
// kappa / (6 D) c_k . (D grad u); r_0 = -(r_1 + r_2 + r_3).
template <typename R>
__device__ __forceinline__ void tet_column(const TetGeom<R>& g, R d1, R d2, R d3, const MaterialDev& m, R sign,
                                           R (&r)[4]) {
  const R gx = d1 * g.c[0][0] + d2 * g.c[1][0] + d3 * g.c[2][0];
  const R gy = d1 * g.c[0][1] + d2 * g.c[1][1] + d3 * g.c[2][1];
  const R gz = d1 * g.c[0][2] + d2 * g.c[1][2] + d3 * g.c[2][2];
  R kap;
  if (m.is_const) {
    kap = kappa_lo<R>(m);
  } else {
    const R E = sqrt(gx * gx + gy * gy + gz * gz) * g.invD;
    kap = kappa_of<R>(m, E);
  }
  const R sc = sign * kap * (g.invD * (R(1) / R(6)));
  r[1] = sc * (g.c[0][0] * gx + g.c[0][1] * gy + g.c[0][2] * gz);
  r[2] = sc * (g.c[1][0] * gx + g.c[1][1] * gy + g.c[1][2] * gz);
  r[3] = sc * (g.c[2][0] * gx + g.c[2][1] * gy + g.c[2][2] * gz);
  r[0] = -(r[1] + r[2] + r[3]);
}

template <typename R>
__device__ __forceinline__ void tet_residual(const R (&e)[3][3], R d1, R d2, R d3, const MaterialDev& m,
                                             R sign, R (&r)[4]) {
  tet_column<R>(tet_geom<R>(e), d1, d2, d3, m, sign, r);
}

// One tet (corners A, B, C, D of the cell; compile-time indices keep the
// corner arrays in registers) into the cell's corner sums.
template <int A, int B, int C, int D>
__device__ __forceinline__ void cell_tet64(const double (&px)[8][3], const double (&f)[8], const MaterialDev& m,
                                           double sign, double (&acc)[8]) {
  double e[3][3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    e[0][q] = px[B][q] - px[A][q];
    e[1][q] = px[C][q] - px[A][q];
    e[2][q] = px[D][q] - px[A][q];
  }
  double r[4];
  tet_residual<double>(e, f[B] - f[A], f[C] - f[A], f[D] - f[A], m, sign, r);
  acc[A] += r[0];
  acc[B] += r[1];
  acc[C] += r[2];
  acc[D] += r[3];
}

// One tet (0, B, C, D) of a Kuhn cell (all six share the diagonal 0-7) from
// the corners' offsets to corner 0: dx[k] = position, df[k] = potential,
// each formed from the (hi, lo) FP32 pairs as (hi_k - hi_0) + (lo_k - lo_0),
// so only these 4 floats per corner stay live across the six tets.
template <int B, int C, int D>
__device__ __forceinline__ void cell_tet32(const float (&dx)[8][3], const float (&df)[8], const MaterialDev& m,
                                           float (&acc)[8]) {
  const float e[3][3] = {{dx[B][0], dx[B][1], dx[B][2]}, {dx[C][0], dx[C][1], dx[C][2]},
                         {dx[D][0], dx[D][1], dx[D][2]}};
  float r[4];
  tet_residual<float>(e, df[B], df[C], df[D], m, 1.0f, r);
  acc[0] += r[0];
  acc[B] += r[1];
  acc[C] += r[2];
  acc[D] += r[3];
}

__global__ void k_elem64_cell(int64_t ncell, const int32_t* __restrict__ corner, const uint8_t* __restrict__ mat,
                              const MaterialDev* __restrict__ mats, const double4* __restrict__ xyz,
                              const double* __restrict__ x, int n_limit, double sign, double* __restrict__ y) {
  pdl_enter();
  const int64_t cidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cidx >= ncell) return;
  int v[8];
  double px[8][3], f[8], acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = __ldg(corner + (int64_t)k * ncell + cidx);
    const double4 p = xyz[v[k]];
    px[k][0] = p.x;
    px[k][1] = p.y;
    px[k][2] = p.z;
    f[k] = __ldg(x + v[k]);
    acc[k] = 0.0;
  }
  const uint8_t* mt = mat + 6 * cidx;
  cell_tet64<0, 1, 3, 7>(px, f, mats[mt[0]], sign, acc);
  cell_tet64<0, 1, 7, 5>(px, f, mats[mt[1]], sign, acc);
  cell_tet64<0, 2, 7, 3>(px, f, mats[mt[2]], sign, acc);
  cell_tet64<0, 2, 6, 7>(px, f, mats[mt[3]], sign, acc);
  cell_tet64<0, 4, 5, 7>(px, f, mats[mt[4]], sign, acc);
  cell_tet64<0, 4, 7, 6>(px, f, mats[mt[5]], sign, acc);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (v[k] < n_limit) atomicAdd(y + v[k], acc[k]);
}

__global__ void __launch_bounds__(kBlock, 3)
k_elem32_cell(int64_t ncell, const int32_t* __restrict__ corner, const uint8_t* __restrict__ mat,
              const MaterialDev* __restrict__ mats, const float4* __restrict__ xh, const float4* __restrict__ xl,
              const float2* __restrict__ x, int n_limit, float* __restrict__ y) {
  pdl_enter();
  const int64_t cidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cidx >= ncell) return;
  int v[8];
  float dx[8][3], df[8], acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __ldg(corner + (int64_t)k * ncell + cidx);
  const float4 h0 = xh[v[0]], l0 = xl[v[0]];
  const float2 f0 = x[v[0]];
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    const float4 h = xh[v[k]], l = xl[v[k]];
    const float2 f = x[v[k]];
    dx[k][0] = (h.x - h0.x) + (l.x - l0.x);
    dx[k][1] = (h.y - h0.y) + (l.y - l0.y);
    dx[k][2] = (h.z - h0.z) + (l.z - l0.z);
    df[k] = (f.x - f0.x) + (f.y - f0.y);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.f;
  const uint8_t* mt = mat + 6 * cidx;
  cell_tet32<1, 3, 7>(dx, df, mats[mt[0]], acc);
  cell_tet32<1, 7, 5>(dx, df, mats[mt[1]], acc);
  cell_tet32<2, 7, 3>(dx, df, mats[mt[2]], acc);
  cell_tet32<2, 6, 7>(dx, df, mats[mt[3]], acc);
  cell_tet32<4, 5, 7>(dx, df, mats[mt[4]], acc);
  cell_tet32<4, 7, 6>(dx, df, mats[mt[5]], acc);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (v[k] < n_limit) atomicAdd(y + v[k], acc[k]);
}

// ---------------------------------------------------- P2 element kernels
// Quadratic tets (Section V's 2nd order ansatz functions): 10 nodes, the
// vertices then the midpoints of the edges (0,1) (0,2) (0,3) (1,2) (1,3)
// (2,3); straight edges, so the barycentric gradients are those of the
// vertices: grad lambda_k = c_k / D (k = 1..3), grad lambda_0 = -sum.  At each
// point of the symmetric 4-point rule of degree 2 (weights V/4)
//   grad phi = sum_k a_k grad lambda_k,
//   a_k = (4 lambda_k - 1) phi_k + 4 sum_{edges (k,l)} lambda_l phi_kl,
//   s_k = grad lambda_k . grad phi,
//   vertex k:     r_k  += (V/4) kappa(|grad phi|) (4 lambda_k - 1) s_k,
//   edge (k, l):  r_kl += (V/4) kappa 4 (lambda_k s_l + lambda_l s_k).
// Potentials enter as differences to phi_0 (a constant shift moves every a_k
// by the same amount and sum_k grad lambda_k = 0), and r_0 = -(r_1 + ... +
// r_9) keeps the local residual's zero sum exactly.

template <typename R>
__device__ __forceinline__ void p2_residual(const R (&gl)[4][3], R D, const R (&d)[10], const MaterialDev& m,
                                            R (&r)[10]) {
  const R QA = (R)0.5854101966249684544613760503096914353161, QB = (R)0.1381966011250105151795413165634361882280;
  const R invD = R(1) / D;  // one division per tet
#pragma unroll
  for (int i = 0; i < 10; ++i) r[i] = R(0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    R l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) l[k] = k == q ? QA : QB;
    R a[4];
    a[0] = (R(4) * l[0] - R(1)) * d[0] + R(4) * (l[1] * d[4] + l[2] * d[5] + l[3] * d[6]);
    a[1] = (R(4) * l[1] - R(1)) * d[1] + R(4) * (l[0] * d[4] + l[2] * d[7] + l[3] * d[8]);
    a[2] = (R(4) * l[2] - R(1)) * d[2] + R(4) * (l[0] * d[5] + l[1] * d[7] + l[3] * d[9]);
    a[3] = (R(4) * l[3] - R(1)) * d[3] + R(4) * (l[0] * d[6] + l[1] * d[8] + l[2] * d[9]);
    R g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c] = a[0] * gl[0][c] + a[1] * gl[1][c] + a[2] * gl[2][c] + a[3] * gl[3][c];
    R kap;
    if (m.is_const) {
      kap = kappa_lo<R>(m);
    } else {
      const R E = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) * invD;
      kap = kappa_of<R>(m, E);
    }
    R sk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) sk[k] = gl[k][0] * g[0] + gl[k][1] * g[1] + gl[k][2] * g[2];
    const R sc = kap * (invD * (R(1) / R(24)));  // (V/4) / D^2 with V = D/6
#pragma unroll
    for (int k = 1; k < 4; ++k) r[k] += sc * (R(4) * l[k] - R(1)) * sk[k];
    r[4] += sc * R(4) * (l[0] * sk[1] + l[1] * sk[0]);
    r[5] += sc * R(4) * (l[0] * sk[2] + l[2] * sk[0]);
    r[6] += sc * R(4) * (l[0] * sk[3] + l[3] * sk[0]);
    r[7] += sc * R(4) * (l[1] * sk[2] + l[2] * sk[1]);
    r[8] += sc * R(4) * (l[1] * sk[3] + l[3] * sk[1]);
    r[9] += sc * R(4) * (l[2] * sk[3] + l[3] * sk[2]);
  }
  R s0 = R(0);
#pragma unroll
  for (int i = 1; i < 10; ++i) s0 += r[i];
  r[0] = -s0;
}

template <typename R>
__device__ __forceinline__ void p2_gradients(const R (&e)[3][3], R (&gl)[4][3], R& D) {
  // c_1 = e_2 x e_3, c_2 = e_3 x e_1, c_3 = e_1 x e_2; D = e_1 . c_1
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R* a = e[(k + 1) % 3];
    const R* b = e[(k + 2) % 3];
    gl[k + 1][0] = a[1] * b[2] - a[2] * b[1];
    gl[k + 1][1] = a[2] * b[0] - a[0] * b[2];
    gl[k + 1][2] = a[0] * b[1] - a[1] * b[0];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) gl[0][c] = -(gl[1][c] + gl[2][c] + gl[3][c]);
  D = e[0][0] * gl[1][0] + e[0][1] * gl[1][1] + e[0][2] * gl[1][2];
}

__global__ void k_elem64_p2(int64_t nt, const int32_t* __restrict__ conn10, const uint8_t* __restrict__ mat,
                            const MaterialDev* __restrict__ mats, const double4* __restrict__ xyz,
                            const double* __restrict__ x, int n_limit, double sign, double* __restrict__ y) {
  pdl_enter();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  int t[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) t[k] = __ldg(conn10 + (int64_t)k * nt + e);
  const double4 p0 = xyz[t[0]];
  double ed[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double4 pk = xyz[t[k + 1]];
    ed[k][0] = pk.x - p0.x;
    ed[k][1] = pk.y - p0.y;
    ed[k][2] = pk.z - p0.z;
  }
  double gl[4][3], D;
  p2_gradients<double>(ed, gl, D);
  const double f0 = __ldg(x + t[0]);
  double d[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) d[k] = k == 0 ? 0.0 : __ldg(x + t[k]) - f0;
  double r[10];
  p2_residual<double>(gl, D, d, mats[mat[e]], r);
#pragma unroll
  for (int k = 0; k < 10; ++k)
    if (t[k] < n_limit) atomicAdd(y + t[k], sign * r[k]);
}

// Mixed precision: coordinates and potentials as FP32 (hi, lo) pairs,
// differences formed as (hi_a - hi_b) + (lo_a - lo_b), the rest in FP32.
__global__ void k_elem32_p2(int64_t nt, const int32_t* __restrict__ conn10, const uint8_t* __restrict__ mat,
                            const MaterialDev* __restrict__ mats, const float4* __restrict__ xh,
                            const float4* __restrict__ xl, const float2* __restrict__ x, int n_limit,
                            float* __restrict__ y) {
  pdl_enter();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  int t[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) t[k] = __ldg(conn10 + (int64_t)k * nt + e);
  const float4 h0 = xh[t[0]], l0 = xl[t[0]];
  float ed[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 hk = xh[t[k + 1]], lk = xl[t[k + 1]];
    ed[k][0] = (hk.x - h0.x) + (lk.x - l0.x);
    ed[k][1] = (hk.y - h0.y) + (lk.y - l0.y);
    ed[k][2] = (hk.z - h0.z) + (lk.z - l0.z);
  }
  float gl[4][3], D;
  p2_gradients<float>(ed, gl, D);
  const float2 f0 = x[t[0]];
  float d[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const float2 fk = x[t[k]];
    d[k] = k == 0 ? 0.f : (fk.x - f0.x) + (fk.y - f0.y);
  }
  float r[10];
  p2_residual<float>(gl, D, d, mats[mat[e]], r);
#pragma unroll
  for (int k = 0; k < 10; ++k)
    if (t[k] < n_limit) atomicAdd(y + t[k], r[k]);
}

// ------------------------------------------------------------- RKC pieces
__device__ __forceinline__ float2 split2(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// Drive values at the stage times: g[j] = V0 sin(w t_j + phase),
// gp[j] = V0 w cos(w t_j + phase), t_j = t + c_j dt, j = 0..s.
__global__ void k_stage_scalars(int s1, const double* __restrict__ cj, const StepParams* prm,
                                double V0, double w, double phase, double* __restrict__ g,
                                double* __restrict__ gp, long long* stepcount) {
  pdl_enter();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) {  // [0]: solves before this step (history index of its first
    stepcount[0] = stepcount[1];  // solve), [1]: after it; steps may differ in s
    stepcount[1] += s1 - 1;
  }
  if (j >= s1) return;
  const double tj = prm->t + cj[j] * prm->dt;
  const double a = w * tj + phase;
  g[j] = V0 * sin(a);
  gp[j] = V0 * w * cos(a);
}

// Y0 (internal order) from the caller's mesh-order x (prm->x), Dirichlet
// rows = g(t); the start vector of the first solve (previous solution) and,
// in FP64 mode, R = -g'(t) M_fd 1_top (the element kernel then subtracts
// K(Y0)Y0).
__global__ void k_gather_state(int n, int nf, const StepParams* prm,
                               const int32_t* __restrict__ node_of_internal,
                               const double* __restrict__ dir_scale, const double* __restrict__ g,
                               const double* __restrict__ gp, const double* __restrict__ mtop,
                               double* __restrict__ Y0, float2* __restrict__ Y32,
                               const double* __restrict__ Fsrc, double* __restrict__ Fdst,
                               double* __restrict__ R) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v;
  if (i < nf) {
    v = prm->x[node_of_internal[i]];
    if (Fdst) Fdst[i] = Fsrc[i];
    if (R) R[i] = -gp[0] * mtop[i];
  } else {
    v = dir_scale[i - nf] * g[0];
  }
  Y0[i] = v;
  if (Y32) Y32[i] = split2(v);
}

// Stage recurrence (Section II; ref. [9]):
//   Y_j = c0 Y0 + mu Y_{j-1} + nu Y_{j-2} + mut dt F_{j-1} + gt dt F_0
// on free rows, g(t_j) on Dirichlet rows.  Also the next solve's start vector
// (F_j <- F_{j-1}), the FP64 right-hand side start R = -g'(t_j) M_fd 1_top,
// and, after the last stage (write_x), x(t + dt) in mesh order into prm->x.
__global__ void k_recurrence(int n, int nf, double c0, double mu, double nu, double mut, double gt,
                             const StepParams* prm, const double* __restrict__ Y0,
                             const double* __restrict__ Yjm1, const double* __restrict__ Yjm2,
                             const double* __restrict__ Fjm1, const double* __restrict__ F0,
                             const int* __restrict__ zero_flags, int jm1,
                             const double* __restrict__ dir_scale, const double* __restrict__ gj,
                             const double* __restrict__ gpj, const double* __restrict__ mtop,
                             double* __restrict__ Yj, float2* __restrict__ Y32,
                             double* __restrict__ Fguess, double* __restrict__ R,
                             int write_x, const int32_t* __restrict__ node_of_internal,
                             float* __restrict__ ring, const long long* __restrict__ stepcount, int s,
                             float* __restrict__ store, long long store_cap, double* __restrict__ spe_ring,
                             int spe_n, float* __restrict__ store_e, const double* __restrict__ x0save) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v;
  if (i < nf) {
    // F_{j-1} enters the solution history (ring slot g % 4; recorded copy)
    const long long gidx = stepcount[0] + jm1;
    const float f32 = (float)Fjm1[i];
    ring[(size_t)(gidx & 3) * nf + i] = f32;
    if (store && gidx < store_cap) {
      store[(size_t)gidx * nf + i] = f32;
      // the solve's distance from its SPE start, z - x0 (FP64 difference)
      if (store_e) store_e[(size_t)gidx * nf + i] = (float)(Fjm1[i] - x0save[i]);
    }
    if (spe_ring) spe_ring[(size_t)(gidx % spe_n) * nf + i] = Fjm1[i];
    const double dt = prm->dt;
    const double fj = zero_flags[jm1] ? 0.0 : Fjm1[i];
    const double f0 = zero_flags[0] ? 0.0 : F0[i];
    v = c0 * Y0[i] + mu * Yjm1[i] + nu * Yjm2[i] + (mut * dt) * fj + (gt * dt) * f0;
    if (Fguess) Fguess[i] = Fjm1[i];
    if (R) R[i] = -(*gpj) * mtop[i];
  } else {
    v = dir_scale[i - nf] * (*gj);
  }
  Yj[i] = v;
  if (Y32) Y32[i] = split2(v);
  if (write_x) prm->x[node_of_internal[i]] = v;
}

// Mixed precision: R = -y32 - g'(t_j) M_fd 1_top in FP64, and clear y32.
__global__ void k_rhs_from_y32(int nf, float* __restrict__ y32, const double* __restrict__ gpj,
                               const double* __restrict__ mtop, double* __restrict__ R) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  R[i] = -(double)y32[i] - (*gpj) * mtop[i];
  y32[i] = 0.0f;
}

// Weighted RMS norm of the local error estimate of the RKC scheme (ref. [9]),
// Est_i = (12 (y_n,i - y_n+1,i) + 6 h (F_n,i + F_n+1,i)) / 15 with weights
// atol + rtol max(|y_n,i|, |y_n+1,i|) over the free rows; the last block
// writes sqrt(mean((Est / w)^2)) to *out.  y in mesh order, F internal.
__global__ void k_rkc_errnorm(int nf, const double* __restrict__ y0, const double* __restrict__ y1,
                              const int32_t* __restrict__ node_of_internal, const double* __restrict__ F0,
                              const double* __restrict__ F1, double h, double atol, double rtol,
                              double* partials, unsigned int* counter, int max_blocks, double* out) {
  pdl_enter();
  double v[1] = {0.0};
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const int m = node_of_internal[i];
    const double a = y0[m], b = y1[m];
    const double est = (12.0 * (a - b) + 6.0 * h * (F0[i] + F1[i])) * (1.0 / 15.0);
    const double w = atol + rtol * fmax(fabs(a), fabs(b));
    const double q = est / w;
    v[0] = fma(q, q, v[0]);
  }
  double tot[1];
  if (grid_sum<1>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) *out = sqrt(tot[0] / nf);
}

// ------------------------------------------------------- small utilities
__global__ void k_gather_perm(int n, const double* __restrict__ src, const int32_t* __restrict__ perm,
                              double* __restrict__ dst, float2* __restrict__ dst32) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = src[perm[i]];
  dst[i] = v;
  if (dst32) dst32[i] = split2(v);
}

__global__ void k_scatter_perm(int n, const double* __restrict__ src, const float* __restrict__ src32,
                               const int32_t* __restrict__ perm, double* __restrict__ dst) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[perm[i]] = src32 ? (double)src32[i] : src[i];
}

template <typename T>
__global__ void k_to_T(int n, const double* __restrict__ a, T* __restrict__ b) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)a[i];
}

template <typename T>
__global__ void k_from_T(int n, const T* __restrict__ a, double* __restrict__ b) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

template <typename T>
__global__ void k_first_step(int n, const T* __restrict__ b, const T* __restrict__ dinv, T inv_theta,
                             T* __restrict__ x, T* __restrict__ d) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T v = dinv[i] * b[i] * inv_theta;
  x[i] = v;
  d[i] = v;
}

// y = M x for FP32 x through the split-M product (the CG operator pass of
// the mixed path without its vector updates).
__global__ void k_spmv_split(DevSell<double> A, const float* __restrict__ hi, const float* __restrict__ lo,
                             int n, const float* __restrict__ x, double* __restrict__ y) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = mat_row_split(A, hi, lo, i, n, x);
}

__global__ void k_spmv64(DevSell<double> A, int n, const double* __restrict__ x, double* __restrict__ y) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double v = mat_row<double>(A, i, n, x);
  if (i < n) y[i] = v;
}

}  // namespace eqs

// ===================================================== persistent M-solve
// One cooperative launch runs a whole CG solve (Section IV): every CTA
// loops over the CG iterations; the V-cycle and CG phases are grid-stride
// loops over rows separated by grid barriers.  Each barrier wait is bounded:
// on time-out the CTA raises an error flag and every CTA returns.
namespace eqs {

constexpr int kMaxLevels = 12;
constexpr int kPBlock = 512;
constexpr long long kMaxSpins = 1LL << 22;

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int err;   // 1: a barrier wait timed out
  int pad;
};

template <typename T>
struct PLevel {
  DevSell<T> A, P, R;
  T *dinv, *b, *x, *r, *dA, *dB;
  int n;
  T inv_theta;
  T c1[5], c2[5];
};

template <typename T>
struct PPlan {
  int nl, deg, nf, maxit, flexible, pad;
  long long max_spins;  // wait budget of one grid barrier (polls)
  const double* coarse_inv;
  DevSell<double> M;
  double *r, *rprev, *pA, *pB, *q, *zd;
  double* partials;  // 16 slots x gridDim
  GridBarrier* bar;
  PLevel<T> lev[kMaxLevels];
};

// A group of CTAs working on one solve: the whole grid (single instance) or
// the CTAs of one instance of a batch.
struct GridCtx {
  int64_t tid, stride;      // group-relative thread id, threads in the group
  unsigned int nblocks;     // CTAs in the group
  unsigned int rank;        // this CTA's index in the group
  GridBarrier* bar;         // the group's barrier
  double* partials;         // the group's reduction slots (16 x nblocks)
  long long max_spins;      // wait budget of one barrier (polls)
};

__device__ __forceinline__ bool grid_barrier(GridBarrier* b, unsigned int nblocks,
                                             long long max_spins = kMaxSpins) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &b->gen;
    const unsigned int g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&b->count, 1u) + 1u == nblocks) {
      b->count = 0u;
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (*(volatile int*)&b->err || ++spins > max_spins) {
          atomicExch(&b->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    if (*(volatile int*)&b->err) ok = 0;
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Block partial of NV values into partials[(slot + k) * nblocks + rank].
template <int NV>
__device__ __forceinline__ void put_partials(double (&v)[NV], double* partials, int slot, unsigned nb,
                                             unsigned rank) {
  block_sum<NV>(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(slot + k) * nb + rank] = v[k];
}

// Sum of the block partials of one slot, in fixed order (same value in every
// CTA); must follow a grid barrier.
__device__ __forceinline__ double get_total(const double* partials, int slot, unsigned nb) {
  __shared__ double s_tot;
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < nb; b += 32) t += __ldcg(partials + slot * nb + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) s_tot = t;
  }
  __syncthreads();
  const double r = s_tot;
  __syncthreads();
  return r;
}

// ---- V-cycle phases (group-stride; loops are warp-uniform).  Every thread
// keeps two rows (t and t + stride) in flight, loading both before storing.
#define EQS_GROUP_ROWS2(MAT, n_, g_, BODY2)                                    \
  const int64_t lim_ = round32((int64_t)(n_) << (MAT).logG);                  \
  for (int64_t t0 = (g_).tid; t0 < lim_; t0 += 2 * (g_).stride) {             \
    const int64_t t1 = t0 + (g_).stride;                                       \
    BODY2                                                                      \
  }

template <typename T>
__device__ __forceinline__ void ph_cheb(const PLevel<T>& L, const T* r_in, const T* d_in, T* r_out,
                                        T* d_out, T c1, T c2, int pending, const GridCtx& g) {
  const int n = L.n;
  EQS_GROUP_ROWS2(L.A, n, g, {
    const T a0 = mat_row(L.A, t0, n, d_in);
    const T a1 = mat_row(L.A, t1, n, d_in);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = h ? t1 : t0;
      if (!row_leader(L.A, t, n)) continue;
      const int i = (int)(t >> L.A.logG);
      const T di = d_in[i];
      const T r = r_in[i] - (h ? a1 : a0);
      const T dn = c1 * di + c2 * L.dinv[i] * r;
      r_out[i] = r;
      d_out[i] = dn;
      L.x[i] += pending ? dn + di : dn;
    }
  })
}

template <typename T>
__device__ __forceinline__ void ph_resid_update(const PLevel<T>& L, const T* d, const GridCtx& g) {
  const int n = L.n;
  EQS_GROUP_ROWS2(L.A, n, g, {
    const T a0 = mat_row(L.A, t0, n, d);
    const T a1 = mat_row(L.A, t1, n, d);
    if (row_leader(L.A, t0, n)) L.r[t0 >> L.A.logG] -= a0;
    if (row_leader(L.A, t1, n)) L.r[t1 >> L.A.logG] -= a1;
  })
}

template <typename T>
__device__ __forceinline__ void ph_resid(const PLevel<T>& L, const GridCtx& g) {
  const int n = L.n;
  EQS_GROUP_ROWS2(L.A, n, g, {
    const T a0 = mat_row(L.A, t0, n, L.x);
    const T a1 = mat_row(L.A, t1, n, L.x);
    if (row_leader(L.A, t0, n)) L.r[t0 >> L.A.logG] = L.b[t0 >> L.A.logG] - a0;
    if (row_leader(L.A, t1, n)) L.r[t1 >> L.A.logG] = L.b[t1 >> L.A.logG] - a1;
  })
}

template <typename T>
__device__ __forceinline__ void ph_restrict(const PLevel<T>& F, const PLevel<T>& C, int first,
                                            const GridCtx& g) {
  const int nc = C.n;
  EQS_GROUP_ROWS2(F.R, nc, g, {
    const T b0 = mat_row(F.R, t0, nc, F.r);
    const T b1 = mat_row(F.R, t1, nc, F.r);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = h ? t1 : t0;
      if (!row_leader(F.R, t, nc)) continue;
      const int i = (int)(t >> F.R.logG);
      const T b = h ? b1 : b0;
      C.b[i] = b;
      if (first) {
        const T d = C.dinv[i] * b * C.inv_theta;
        C.x[i] = d;
        C.dA[i] = d;
      }
    }
  })
}

template <typename T>
__device__ __forceinline__ void ph_prolong(const PLevel<T>& F, const PLevel<T>& C, const GridCtx& g) {
  const int n = F.n;
  EQS_GROUP_ROWS2(F.P, n, g, {
    const T p0 = mat_row(F.P, t0, n, C.x);
    const T p1 = mat_row(F.P, t1, n, C.x);
    if (row_leader(F.P, t0, n)) F.x[t0 >> F.P.logG] += p0;
    if (row_leader(F.P, t1, n)) F.x[t1 >> F.P.logG] += p1;
  })
}

template <typename T>
__device__ __forceinline__ void ph_post_first(const PLevel<T>& L, const GridCtx& g) {
  const int n = L.n;
  EQS_GROUP_ROWS2(L.A, n, g, {
    const T a0 = mat_row(L.A, t0, n, L.x);
    const T a1 = mat_row(L.A, t1, n, L.x);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = h ? t1 : t0;
      if (!row_leader(L.A, t, n)) continue;
      const int i = (int)(t >> L.A.logG);
      const T r = L.b[i] - (h ? a1 : a0);
      L.r[i] = r;
      L.dA[i] = L.dinv[i] * r * L.inv_theta;
    }
  })
}

template <typename T>
__device__ __forceinline__ void ph_coarse(const PLevel<T>& L, const double* inv, const GridCtx& g) {
  const int n = L.n;
  const int64_t lim = (int64_t)n * 32;
  for (int64_t t = g.tid; t < round32(lim); t += g.stride) {
    const int row = (int)(t >> 5), lane = (int)(t & 31);
    double acc = 0.0;
    if (row < n)
      for (int j = lane; j < n; j += 32) acc = fma(inv[(int64_t)row * n + j], (double)L.b[j], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (row < n && lane == 0) L.x[row] = (T)acc;
  }
}

// Whole V-cycle from level 0 (its b, x = dA = first step already set).
template <typename T>
__device__ bool vcycle_persistent(const PPlan<T>& P, const GridCtx& g) {
  const int nl = P.nl, deg = P.deg;
  for (int l = 0; l < nl - 1; ++l) {
    const PLevel<T>& L = P.lev[l];
    T* din = L.dA;
    T* dout = L.dB;
    const T* rin = L.b;
    for (int k = 2; k <= deg; ++k) {
      ph_cheb(L, rin, din, L.r, dout, L.c1[k], L.c2[k], 0, g);
      if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return false;
      rin = L.r;
      T* tmp = din;
      din = dout;
      dout = tmp;
    }
    if (deg >= 2)
      ph_resid_update(L, din, g);
    else
      ph_resid(L, g);
    if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return false;
    ph_restrict(L, P.lev[l + 1], l + 1 < nl - 1, g);
    if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return false;
  }
  ph_coarse(P.lev[nl - 1], P.coarse_inv, g);
  if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return false;
  for (int l = nl - 2; l >= 0; --l) {
    const PLevel<T>& L = P.lev[l];
    ph_prolong(L, P.lev[l + 1], g);
    if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return false;
    ph_post_first(L, g);
    if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return false;
    T* din = L.dA;
    T* dout = L.dB;
    for (int k = 2; k <= deg; ++k) {
      ph_cheb(L, L.r, din, L.r, dout, L.c1[k], L.c2[k], k == 2, g);
      if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return false;
      T* tmp = din;
      din = dout;
      dout = tmp;
    }
    if (deg == 1) {
      for (int64_t i = g.tid; i < L.n; i += g.stride) L.x[i] += L.dA[i];
      if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return false;
    }
  }
  return true;
}

// Preconditioned CG for M_ff x = R from the start vector in x, run by the
// CTAs of group g.  Slots of the partial sums: 0-1 init, 2-3 dots, 4 p.q,
// 5 update.  Returns false if a barrier wait timed out.
template <typename T>
__device__ bool pcg_group_solve(const PPlan<T>& P, const GridCtx& g, const double* __restrict__ R,
                                double* __restrict__ x, double tol2, int* iters_out, double* relres_out,
                                int* zero_out) {
  const unsigned nb = g.nblocks;
  const int n = P.nf;
  const PLevel<T>& L0 = P.lev[0];
  const bool single = (P.nl == 1);
  {
    double v[2] = {0.0, 0.0};
    for (int64_t i = g.tid; i < n; i += g.stride) {
      const double Ri = R[i];
      const double ri = Ri - mat_row<double>(P.M, i, n, x);
      P.r[i] = ri;
      const T bi = vc_in<T>(ri);
      L0.b[i] = bi;
      if (!single) {
        const T d = L0.dinv[i] * bi * L0.inv_theta;
        L0.x[i] = d;
        L0.dA[i] = d;
      }
      v[0] += Ri * Ri;
      v[1] += ri * ri;
    }
    put_partials<2>(v, g.partials, 0, nb, g.rank);
  }
  if (!grid_barrier(g.bar, nb, g.max_spins)) return false;
  const double bnorm2 = get_total(g.partials, 0, nb);
  double rnorm2 = get_total(g.partials, 1, nb);
  const int zero = bnorm2 == 0.0;
  int conv = zero || !(rnorm2 > tol2 * bnorm2);
  int it = 0;
  double rz_old = 1.0;
  while (!conv && it < P.maxit) {
    if (!vcycle_persistent(P, g)) return false;
    {
      double v[2] = {0.0, 0.0};
      for (int64_t i = g.tid; i < n; i += g.stride) {
        const double zi = (double)L0.x[i];
        P.zd[i] = zi;
        v[0] += P.r[i] * zi;
        v[1] += P.rprev[i] * zi;
      }
      put_partials<2>(v, g.partials, 2, nb, g.rank);
    }
    if (!grid_barrier(g.bar, nb, g.max_spins)) return false;
    const double rz = get_total(g.partials, 2, nb);
    const double zrp = get_total(g.partials, 3, nb);
    const double beta = it == 0 ? 0.0 : (P.flexible ? (rz - zrp) / rz_old : rz / rz_old);
    rz_old = rz;
    // p = z + beta p ; q = M z + beta q (q_old = M p_old), row-local
    {
      double v[1] = {0.0};
      for (int64_t i0 = g.tid; i0 < n; i0 += 2 * g.stride) {
        const int64_t i1 = i0 + g.stride;
        const double w0 = mat_row<double>(P.M, i0, n, P.zd);
        const double w1 = mat_row<double>(P.M, i1, n, P.zd);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t i = h ? i1 : i0;
          if (i >= n) continue;
          const double w = h ? w1 : w0;
          const double qi = beta == 0.0 ? w : fma(beta, P.q[i], w);
          const double pi = beta == 0.0 ? P.zd[i] : fma(beta, P.pA[i], P.zd[i]);
          P.pA[i] = pi;
          P.q[i] = qi;
          v[0] += pi * qi;
        }
      }
      put_partials<1>(v, g.partials, 4, nb, g.rank);
    }
    if (!grid_barrier(g.bar, nb, g.max_spins)) return false;
    const double alpha = rz / get_total(g.partials, 4, nb);
    {
      double v[1] = {0.0};
      for (int64_t i = g.tid; i < n; i += g.stride) {
        x[i] = fma(alpha, P.pA[i], x[i]);
        const double ro = P.r[i];
        P.rprev[i] = ro;
        const double rn = fma(-alpha, P.q[i], ro);
        P.r[i] = rn;
        v[0] += rn * rn;
        const T bi = vc_in<T>(rn);
        L0.b[i] = bi;
        if (!single) {
          const T d = L0.dinv[i] * bi * L0.inv_theta;
          L0.x[i] = d;
          L0.dA[i] = d;
        }
      }
      put_partials<1>(v, g.partials, 5, nb, g.rank);
    }
    if (!grid_barrier(g.bar, nb, g.max_spins)) return false;
    rnorm2 = get_total(g.partials, 5, nb);
    ++it;
    conv = !(rnorm2 > tol2 * bnorm2);
  }
  if (g.rank == 0 && threadIdx.x == 0) {
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = zero ? 0.0 : sqrt(rnorm2 / bnorm2);
    if (zero_out) *zero_out = zero;
  }
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kPBlock) k_pcg_persistent(const PPlan<T>* __restrict__ plan,
                                                             const double* __restrict__ R,
                                                             double* __restrict__ x,
                                                             int* iters_out, double* relres_out,
                                                             int* zero_out, double tol2) {
  const PPlan<T>& P = *plan;
  GridCtx g;
  g.tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  g.stride = (int64_t)gridDim.x * blockDim.x;
  g.nblocks = gridDim.x;
  g.rank = blockIdx.x;
  g.bar = P.bar;
  g.partials = P.partials;
  g.max_spins = P.max_spins;
  pcg_group_solve(P, g, R, x, tol2, iters_out, relres_out, zero_out);
}

}  // namespace eqs
