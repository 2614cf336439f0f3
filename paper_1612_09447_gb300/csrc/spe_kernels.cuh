// Subspace projection extrapolation (SPE) start vector, Section IV, Eq. 4-5:
// x0 = V (V^T M V)^-1 V^T b with V spanning the last n solutions.
//
// The history rings hold the last n solutions X (FP64, solution q in ring
// slot q % n) and W = M X.  The Gram matrix G[a][b] = x_a . w_b (by slot) is
// kept on the device and updated incrementally: when solution q becomes the
// newest, one pass computes w_q = M x_q, the new Gram column x_k . w_q for
// every stored solution k and the projections c_k = x_k . b of the current
// right-hand side (2n sums instead of n(n+1)/2 + n).  The basis is formed in
// the M inner product by a Cholesky factorisation of the Gram matrix that
// skips a column whose remaining M-norm is below sqrt(drop2) of its own (a
// nearly dependent history vector) -- the projection of Eq. 5 over the same
// span that Euclidean Gram-Schmidt would keep.
//
// Because M x0 = W y, the initial CG residual r0 = b - W y needs no SpMV:
// k_proj_start forms x0, r0 and the first V-cycle input in one row-local pass.
#pragma once

#include "kernels.cuh"

namespace eqs {

constexpr int kSpeMax = 6;
constexpr int kSpeSums = 2 * kSpeMax;  // Gram column + projections of b

__device__ __forceinline__ int spe_slot(long long q, int NH) { return (int)(((q % NH) + NH) % NH); }

// The SPE coefficients of solve g: with m = min(g, NH) slots in use and the
// newest solution in slot sn = slot(g - 1), solve (L L^T) y = c for the Gram
// matrix A (row and column of the newest slot from tot[0..m), every other
// entry from the stored G, which is not read at the newest slot) and
// c = tot[NH..NH+m), by Cholesky with column dropping (most recent first);
// y_out[k] is the coefficient of solution g - 1 - k (ring slot
// slot(g - 1 - k)).  One
// thread; every loop runs over the compile-time NH (rows k >= m are zero and
// never kept), so the small matrices stay in registers instead of local
// memory.  On GB300 every FP64 instruction of this serial code occupies the
// slow FP64 pipe of its SM sub-partition for a whole warp's worth of lanes,
// so the factor keeps the reciprocal of each pivot (one rsqrt per column)
// and multiplies by it instead of dividing (an IEEE division is a chain of
// about ten FP64 operations).
template <int NH>
__device__ void spe_coeffs(const double* tot, long long g, int m, const double* G, double drop2,
                           double (&y_out)[NH]) {
  int slot[NH];
#pragma unroll
  for (int k = 0; k < NH; ++k) slot[k] = spe_slot(g - 1 - k, NH);
  double A[NH][NH], L[NH][NH], c[NH], z[NH], y[NH], inv[NH];
  bool keep[NH];
#pragma unroll
  for (int k = 0; k < NH; ++k) {
    c[k] = tot[NH + k];
    keep[k] = false;
    inv[k] = 0.0;
    z[k] = 0.0;
    y[k] = 0.0;
#pragma unroll
    for (int l = 0; l < NH; ++l) {
      double a = 0.0;
      if (k < m && l < m) a = k == 0 ? tot[l] : (l == 0 ? tot[k] : G[slot[k] * kSpeMax + slot[l]]);
      A[k][l] = a;
      L[k][l] = 0.0;
    }
  }
#pragma unroll
  for (int k = 0; k < NH; ++k) {
    double d = A[k][k];
#pragma unroll
    for (int p = 0; p < k; ++p)
      if (keep[p]) d -= L[k][p] * L[k][p];
    keep[k] = A[k][k] > 0.0 && d > drop2 * A[k][k];
    if (!keep[k]) continue;
    inv[k] = rsqrt(d);  // 1 / L[k][k]
#pragma unroll
    for (int r = k + 1; r < NH; ++r) {
      double e = A[r][k];
#pragma unroll
      for (int p = 0; p < k; ++p)
        if (keep[p]) e -= L[r][p] * L[k][p];
      L[r][k] = e * inv[k];
    }
  }
#pragma unroll
  for (int k = 0; k < NH; ++k) {  // L z = c (kept rows)
    if (!keep[k]) continue;
    double e = c[k];
#pragma unroll
    for (int p = 0; p < k; ++p)
      if (keep[p]) e -= L[k][p] * z[p];
    z[k] = e * inv[k];
  }
#pragma unroll
  for (int k = NH - 1; k >= 0; --k) {  // L^T y = z
    if (!keep[k]) continue;
    double e = z[k];
#pragma unroll
    for (int r = k + 1; r < NH; ++r)
      if (keep[r]) e -= L[r][k] * y[r];
    y[k] = e * inv[k];
  }
#pragma unroll
  for (int k = 0; k < NH; ++k) y_out[k] = k < m ? y[k] : 0.0;
}

// Store the new Gram column and row of the newest slot sn (tot[0..m)).
template <int NH>
__device__ __forceinline__ void spe_store_column(const double* tot, long long g, int m, int sn,
                                                 double* __restrict__ G) {
#pragma unroll
  for (int k = 0; k < NH; ++k)
    if (k < m) {
      const int sk = spe_slot(g - 1 - k, NH);
      G[sk * kSpeMax + sn] = tot[k];
      G[sn * kSpeMax + sk] = tot[k];
    }
}

// Last block of a Gram pass: store the new Gram column, solve for the
// coefficients and write them by ring slot plus the slots in use.
template <int NH>
__device__ void spe_solve(const double* tot, long long g, int m, int sn, double* __restrict__ G, double drop2,
                          double* __restrict__ y_out) {
  double y[NH];
  spe_coeffs<NH>(tot, g, m, G, drop2, y);
  spe_store_column<NH>(tot, g, m, sn, G);
#pragma unroll
  for (int k = 0; k < NH; ++k) y_out[k] = 0.0;
#pragma unroll
  for (int k = 0; k < NH; ++k)
    if (k < m) y_out[spe_slot(g - 1 - k, NH)] = y[k];
  reinterpret_cast<int*>(y_out + kSpeMax)[0] = m;
}

// Solve index g = stepcount[0] + j: solutions 0..g-1 exist, the newest
// m = min(g, NH) of them are in the rings.  One pass: w_{g-1} = M x_{g-1},
// the Gram column G[k][g-1] over the stored solutions k and c_k = x_k . b.
// The last block updates G and solves (L L^T) y = c with column dropping;
// y_out[slot] is the coefficient of the solution in that ring slot and
// y_out[kSpeMax] (as int) the number of slots in use.  DEFER: the 2 NH sums
// are left as per-block partials (partials[k * max_blocks + block]) for
// k_spe_solve.
template <int NH, bool DEFER>
__global__ void k_spe_gram(DevSell<double> M, int nf, const double* __restrict__ X, double* __restrict__ W,
                           const double* __restrict__ b, const long long* __restrict__ stepcount, int s,
                           int j, double* __restrict__ G, double* partials, unsigned int* counter,
                           int max_blocks, double drop2, double* __restrict__ y_out) {
  pdl_enter();
  const long long g = stepcount[0] + j;
  if (g == 0) {  // uniform over the grid: no history, no reduction
    if (!DEFER && blockIdx.x == 0 && threadIdx.x == 0) reinterpret_cast<int*>(y_out + kSpeMax)[0] = 0;
    return;
  }
  const int m = (int)(g < NH ? g : NH);
  const int sn = spe_slot(g - 1, NH);
  constexpr int NS = 2 * NH;
  double v[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) v[k] = 0.0;
  const double* xs[NH];
#pragma unroll
  for (int k = 0; k < NH; ++k) xs[k] = X + (size_t)spe_slot(g - 1 - k, NH) * nf;
  const double* __restrict__ xn = X + (size_t)sn * nf;
  double* __restrict__ wn = W + (size_t)sn * nf;
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const double w = mat_row<double>(M, i, nf, xn);
    wn[i] = w;
    const double bi = b[i];
#pragma unroll
    for (int k = 0; k < NH; ++k) {
      const double xk = k < m ? xs[k][i] : 0.0;
      v[k] = fma(xk, w, v[k]);
      v[NH + k] = fma(xk, bi, v[NH + k]);
    }
  }
  if constexpr (DEFER) {
    write_partials<NS>(v, partials, max_blocks);
    return;
  }
  double tot[NS];
  if (grid_sum<NS>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0)
    spe_solve<NH>(tot, g, m, sn, G, drop2, y_out);
}

// The deferred form's small solve: one block adds the Gram pass's nb
// per-block partials (in a fixed order), then thread 0 updates G and writes
// the coefficients as the last block of the undeferred pass does -- without
// the pass's atomic ticket, fences and serial last block.
template <int NH>
__global__ void k_spe_solve(const long long* __restrict__ stepcount, int j, double* __restrict__ G, double drop2,
                            const double* __restrict__ part, int nb, int cap, double* __restrict__ y_out) {
  pdl_enter();
  const long long g = stepcount[0] + j;
  if (g == 0) {
    if (threadIdx.x == 0) reinterpret_cast<int*>(y_out + kSpeMax)[0] = 0;
    return;
  }
  const int m = (int)(g < NH ? g : NH);
  double tot[2 * NH];
  sum_partials<2 * NH>(part, nb, cap, tot);
  if (threadIdx.x == 0) spe_solve<NH>(tot, g, m, spe_slot(g - 1, NH), G, drop2, y_out);
}

// Start of the CG solve from a projection start vector (SPE or POD): with
// coefficients a (by ring slot, *nuse > 0 slots in use) x0 = X a and
// r0 = R - W a (= R - M x0: W = M X, so no SpMV), the norms of R and r0, and
// the first V-cycle input (b0 = r0 in T, x = d = D0^-1 b0 / theta0); the
// last block decides whether the CG loop runs.  With *nuse == 0 (no
// history or no basis yet) x keeps the caller's start vector and
// r0 = R - M x.  With r == nullptr only x0 is written (no reduction).
template <typename T, int NH>
__global__ void k_proj_start(DevSell<double> M, int nf, const double* __restrict__ X,
                             const double* __restrict__ W, const double* __restrict__ coef,
                             const int* __restrict__ nuse, const double* __restrict__ R,
                             double* __restrict__ x, double* __restrict__ r, const T* __restrict__ dinv0,
                             T inv_theta0, T* __restrict__ b0, T* __restrict__ x0, T* __restrict__ d0,
                             PcgScalars* sc, double* partials, unsigned int* counter, int max_blocks,
                             double tol2, int maxit, cudaGraphConditionalHandle h, int use_handle,
                             int* iters_out, double* relres_out, int* zero_out, double* __restrict__ x_copy) {
  pdl_enter();
  const int m = *nuse;
  double y[NH];
#pragma unroll
  for (int k = 0; k < NH; ++k) y[k] = k < m ? coef[k] : 0.0;
  double v[2] = {0.0, 0.0};
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    double xi, mx;
    if (m > 0) {
      xi = 0.0;
      mx = 0.0;
#pragma unroll
      for (int k = 0; k < NH; ++k)
        if (k < m) {
          xi = fma(y[k], X[(size_t)k * nf + i], xi);
          mx = fma(y[k], W[(size_t)k * nf + i], mx);
        }
      x[i] = xi;
      if (x_copy) x_copy[i] = xi;
    } else {
      mx = r ? mat_row<double>(M, i, nf, x) : 0.0;
      if (x_copy) x_copy[i] = x[i];
    }
    if (!r) continue;
    const double Ri = R[i];
    const double ri = Ri - mx;
    r[i] = ri;
    const T bi = vc_in<T>(ri);
    b0[i] = bi;
    const T d = dinv0[i] * bi * inv_theta0;
    x0[i] = d;
    d0[i] = d;
    v[0] += Ri * Ri;
    v[1] += ri * ri;
  }
  if (!r) return;
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

}  // namespace eqs
