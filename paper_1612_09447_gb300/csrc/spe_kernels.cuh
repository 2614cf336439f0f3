// Subspace projection extrapolation (SPE) start vector, Section IV, Eq. 4-5:
// x0 = V (V^T M V)^-1 V^T b with V spanning the last n solutions.
//
// The history rings hold the last n solutions X (FP64) and W = M X; each
// solve adds one product (M times the newest solution), so V^T M V costs one
// SpMV per solve: A = X^T W (upper triangle, mirrored).  The basis is formed in the M
// inner product by a Cholesky factorisation of A that skips a column whose
// remaining M-norm is below sqrt(drop2) of its own (a nearly dependent
// history vector) -- the projection of Eq. 5 over the same span that
// Euclidean Gram-Schmidt would keep.  Solution k of the sequence is stored in
// ring slot k % n.
#pragma once

#include "kernels.cuh"

namespace eqs {

constexpr int kSpeMax = 6;
constexpr int kSpeSums = kSpeMax * (kSpeMax + 1) / 2 + kSpeMax;  // 27

// W slot of the newest solution x_{g-1}: w = M x_{g-1}.
template <int NH>
__global__ void k_spe_mx(DevSell<double> M, int nf, const double* __restrict__ X, double* __restrict__ W,
                         const long long* __restrict__ stepcount, int s, int j) {
  pdl_enter();
  const long long g = stepcount[0] * (long long)s + j;
  if (g == 0) return;
  const size_t slot = (size_t)((g - 1) % NH) * nf;
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x)
    W[slot + i] = mat_row<double>(M, i, nf, X + slot);
}

// Sums A_kl (k <= l) = x_{g-1-k} . w_{g-1-l} and c_k = x_{g-1-k} . b over the
// rows; the last block solves for y (y_out[0..n)).
template <int NH>
__global__ void k_spe_gram(int nf, const double* __restrict__ X, const double* __restrict__ Rr,
                           const double* __restrict__ b,
                           const long long* __restrict__ stepcount, int s, int j, double* partials,
                           unsigned int* counter, int max_blocks, double drop2, double* y_out) {
  pdl_enter();
  const long long g = stepcount[0] * (long long)s + j;
  const int m = (int)(g < NH ? g : NH);
  constexpr int NS = NH * (NH + 1) / 2 + NH;
  double v[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) v[k] = 0.0;
  const double* xs[NH];
  const double* ws[NH];
#pragma unroll
  for (int k = 0; k < NH; ++k) {
    const long long slot = ((g - 1 - k) % NH + NH) % NH;
    xs[k] = X + (size_t)slot * nf;
    ws[k] = Rr + (size_t)slot * nf;
  }
  // few blocks with many rows each: the block reductions of NS values cost
  // FP64 adds in every lane, so they must stay rare next to the row work
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    double xv[NH], wv[NH];
#pragma unroll
    for (int k = 0; k < NH; ++k) {
      xv[k] = k < m ? xs[k][i] : 0.0;
      wv[k] = k < m ? ws[k][i] : 0.0;
    }
    const double bi = b[i];
    int q = 0;
#pragma unroll
    for (int k = 0; k < NH; ++k) {
#pragma unroll
      for (int l = k; l < NH; ++l) v[q] = fma(xv[k], wv[l], v[q]), ++q;
    }
#pragma unroll
    for (int k = 0; k < NH; ++k) v[q] = fma(xv[k], bi, v[q]), ++q;
  }
  double tot[NS];
  if (grid_sum<NS>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    double A[NH][NH], c[NH], L[NH][NH], y[NH];
    int q = 0;
    for (int k = 0; k < NH; ++k)
      for (int l = k; l < NH; ++l) {
        A[k][l] = tot[q];
        A[l][k] = tot[q];
        ++q;
      }
    for (int k = 0; k < NH; ++k) c[k] = tot[q++];
    bool keep[NH];
    for (int k = 0; k < NH; ++k) {
      keep[k] = false;
      y[k] = 0.0;
      for (int l = 0; l < NH; ++l) L[k][l] = 0.0;
    }
    // Cholesky with column dropping, most recent solution first
    for (int k = 0; k < m; ++k) {
      double d = A[k][k];
      for (int p = 0; p < k; ++p)
        if (keep[p]) d -= L[k][p] * L[k][p];
      if (!(A[k][k] > 0.0) || !(d > drop2 * A[k][k])) continue;
      keep[k] = true;
      L[k][k] = sqrt(d);
      for (int r = k + 1; r < m; ++r) {
        double e = A[r][k];
        for (int p = 0; p < k; ++p)
          if (keep[p]) e -= L[r][p] * L[k][p];
        L[r][k] = e / L[k][k];
      }
    }
    double z[NH];
    for (int k = 0; k < m; ++k) {  // L z = c (kept rows)
      z[k] = 0.0;
      if (!keep[k]) continue;
      double e = c[k];
      for (int p = 0; p < k; ++p)
        if (keep[p]) e -= L[k][p] * z[p];
      z[k] = e / L[k][k];
    }
    for (int k = m - 1; k >= 0; --k) {  // L^T y = z
      if (!keep[k]) continue;
      double e = z[k];
      for (int r = k + 1; r < m; ++r)
        if (keep[r]) e -= L[r][k] * y[r];
      y[k] = e / L[k][k];
    }
    for (int k = 0; k < NH; ++k) y_out[k] = y[k];
  }
}

// x0 = sum_k y_k x_{g-1-k} (x0 is left as it is when there is no history).
template <int NH>
__global__ void k_spe_combine(int nf, const double* __restrict__ X, const double* __restrict__ y,
                              const long long* __restrict__ stepcount, int s, int j, double* __restrict__ x0) {
  pdl_enter();
  const long long g = stepcount[0] * (long long)s + j;
  const int m = (int)(g < NH ? g : NH);
  if (m == 0) return;  // no history yet: keep the previous-solution start vector
  double yc[NH];
  const double* xs[NH];
#pragma unroll
  for (int k = 0; k < NH; ++k) {
    yc[k] = k < m ? y[k] : 0.0;
    xs[k] = X + (size_t)(((g - 1 - k) % NH + NH) % NH) * nf;
  }
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NH; ++k)
      if (k < m) acc = fma(yc[k], xs[k][i], acc);
    x0[i] = acc;
  }
}

}  // namespace eqs
