// POD-MOR start vectors, Section IV: a proper orthogonal decomposition of
// earlier solutions ("snapshots") gives the basis of the projection of Eq. 5.
//
// The snapshots X (up to K, FP64, by slot) and their products W = M X are
// stored; the Euclidean Gram matrix G_E = X^T X and the M-Gram matrix
// G_M = X^T M X are kept up to date one row per added snapshot.  The POD
// of the snapshot matrix comes from the eigendecomposition G_E = U Lambda U^T
// (the left singular vectors are X U Lambda^-1/2), so with the kept modes
// U_m the projection of Eq. 5 onto span(X U_m) is
//     x0 = X a,  a = U_m (U_m^T G_M U_m)^-1 U_m^T (X^T b),
// and M x0 = W a needs no SpMV (k_proj_start).  The eigendecomposition is a
// parallel cyclic Jacobi iteration (round-robin pairing, disjoint rotations
// applied together) in one thread block.
//
// Two snapshot rules (Section IV): MOR takes the first K solutions and
// computes the basis once; MOR2 adds a solution whose solve needed more than
// min_iters CG iterations, overwriting the oldest when full, and recomputes
// the basis after every addition.
#pragma once

#include "spe_kernels.cuh"

namespace eqs {

constexpr int kPodMax = 16;
constexpr int kJacobiSweeps = 12;
// A mode is kept while its eigenvalue of G_E exceeds kPodDrop2 times the
// largest (singular value above 1e-7 of the largest); a reduced-system
// pivot must exceed kPodDrop2 of its diagonal.
constexpr double kPodDrop2 = 1e-14;

struct PodState {
  int count;     // snapshots stored (slots 0..count-1)
  int next;      // slot of the next snapshot
  int rebuild;   // 1: the basis must be recomputed
  int nuse;      // slots used by the current coefficients (0: no basis yet)
  int m_used;    // POD modes kept
  int rebuilds;  // bases computed so far
  int adds;      // snapshots added so far
  int pad;
  double U[kPodMax * kPodMax];  // kept modes: U[k * kPodMax + a], slot k, mode a
  double L[kPodMax * kPodMax];  // Cholesky factor of U_m^T G_M U_m
  double lam[kPodMax];          // eigenvalues of G_E, descending
};

// Add the newest solution xnew as a snapshot when the rule says so:
// MOR (mode 0) while fewer than cap (<= K) are stored; MOR2 (mode 1) when
// the solve that produced it needed more than min_iters iterations (ring of
// cap slots).  One pass stores it, forms w = M xnew and the new rows of G_E
// and G_M.
template <int K>
__global__ void k_pod_add(DevSell<double> M, int nf, double* __restrict__ X, double* __restrict__ W,
                          double* __restrict__ GE, double* __restrict__ GM, const double* __restrict__ xnew,
                          const int* __restrict__ prev_iters, const int* __restrict__ prev_zero,
                          const long long* __restrict__ stepcount, int s, int j, int mode, int cap,
                          int min_iters, PodState* st, double* partials, unsigned int* counter,
                          int max_blocks) {
  pdl_enter();
  const long long g = stepcount[0] + j;
  if (g == 0 || *prev_zero) return;  // no solution yet / a zero solve is not a snapshot
  const int add = mode == 0 ? st->count < cap : *prev_iters > min_iters;
  if (!add) return;  // uniform over the grid
  const int slot = st->next;
  const int cnt = st->count + 1 < cap ? st->count + 1 : cap;
  double v[2 * K];
#pragma unroll
  for (int k = 0; k < 2 * K; ++k) v[k] = 0.0;
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = xnew[i];
    const double w = mat_row<double>(M, i, nf, xnew);
    X[(size_t)slot * nf + i] = x;
    W[(size_t)slot * nf + i] = w;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const double xk = k >= cnt ? 0.0 : (k == slot ? x : X[(size_t)k * nf + i]);
      v[k] = fma(xk, x, v[k]);
      v[K + k] = fma(xk, w, v[K + k]);
    }
  }
  double tot[2 * K];
  if (grid_sum<2 * K>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    for (int k = 0; k < cnt; ++k) {
      GE[k * kPodMax + slot] = GE[slot * kPodMax + k] = tot[k];
      GM[k * kPodMax + slot] = GM[slot * kPodMax + k] = tot[K + k];
    }
    st->count = cnt;
    st->next = (slot + 1) % cap;
    st->adds += 1;
    st->rebuild = mode == 0 ? (cnt == cap) : 1;
  }
}

// Eigendecomposition of G_E (count x count) by parallel cyclic Jacobi, the
// kept modes (eigenvalue above drop2 times the largest, at most m_max), the
// reduced matrix B = U_m^T G_M U_m and its Cholesky factor (a mode whose
// pivot falls below drop2 of its diagonal is dropped).  One block.
template <int K>
__global__ void k_pod_rebuild(const double* __restrict__ GE, const double* __restrict__ GM, int m_max,
                              double drop2, PodState* st) {
  __shared__ double A[K][K + 1], V[K][K + 1], B[K][K + 1];
  __shared__ double rc[K / 2 + 1], rs[K / 2 + 1];
  __shared__ int rp[K / 2 + 1], rq[K / 2 + 1], sel[K];
  __shared__ int n_s, m_s;
  pdl_enter();
  if (!st->rebuild) return;  // uniform over the block
  const int n = st->count;
  const int t = threadIdx.x;
  for (int e = t; e < K * K; e += blockDim.x) {
    const int a = e / K, b = e % K;
    A[a][b] = (a < n && b < n) ? GE[a * kPodMax + b] : 0.0;
    V[a][b] = a == b ? 1.0 : 0.0;
  }
  __syncthreads();
  const int n2 = (n + 1) & ~1;  // even player count (index n is a bye when n is odd)
  const int np = n2 / 2;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    for (int r = 0; r + 1 < n2; ++r) {
      if (t < np) {  // round-robin pairing: player 0 fixed, the others rotate
        const int i0 = t, i1 = n2 - 1 - t;
        const int p = i0 == 0 ? 0 : (i0 - 1 + r) % (n2 - 1) + 1;
        const int q = (i1 - 1 + r) % (n2 - 1) + 1;
        double c = 1.0, s = 0.0;
        if (p < n && q < n) {
          const double apq = A[p][q];
          if (apq != 0.0) {
            const double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
          }
        }
        rp[t] = p;
        rq[t] = q;
        rc[t] = c;
        rs[t] = s;
      }
      __syncthreads();
      for (int e = t; e < np * n; e += blockDim.x) {  // rows: A <- J^T A
        const int k = e / n, col = e % n;
        const int p = rp[k], q = rq[k];
        if (p >= n || q >= n) continue;
        const double c = rc[k], s = rs[k];
        const double ap = A[p][col], aq = A[q][col];
        A[p][col] = c * ap - s * aq;
        A[q][col] = s * ap + c * aq;
      }
      __syncthreads();
      for (int e = t; e < np * n; e += blockDim.x) {  // columns: A <- A J, V <- V J
        const int k = e / n, row = e % n;
        const int p = rp[k], q = rq[k];
        if (p >= n || q >= n) continue;
        const double c = rc[k], s = rs[k];
        const double ap = A[row][p], aq = A[row][q];
        A[row][p] = c * ap - s * aq;
        A[row][q] = s * ap + c * aq;
        const double vp = V[row][p], vq = V[row][q];
        V[row][p] = c * vp - s * vq;
        V[row][q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  if (t == 0) {  // modes by decreasing eigenvalue
    bool used[K];
    double lmax = 0.0;
    for (int k = 0; k < n; ++k) {
      used[k] = false;
      lmax = fmax(lmax, A[k][k]);
    }
    int m = 0;
    for (int a = 0; a < n && m < m_max; ++a) {
      int best = -1;
      for (int k = 0; k < n; ++k)
        if (!used[k] && (best < 0 || A[k][k] > A[best][best])) best = k;
      used[best] = true;
      st->lam[a] = A[best][best];
      if (!(A[best][best] > drop2 * lmax)) break;
      sel[m++] = best;
    }
    m_s = m;
    n_s = n;
  }
  __syncthreads();
  const int m = m_s;
  for (int e = t; e < m * m; e += blockDim.x) {  // B = U_m^T G_M U_m
    const int a = e / m, b = e % m;
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      double row = 0.0;
      for (int k = 0; k < n; ++k) row = fma(GM[i * kPodMax + k], V[k][sel[b]], row);
      acc = fma(V[i][sel[a]], row, acc);
    }
    B[a][b] = acc;
  }
  __syncthreads();
  if (t == 0) {
    // Cholesky with mode dropping; kept modes are compacted into U and L
    double Lf[K][K];
    int keep[K], mk = 0;
    for (int a = 0; a < m; ++a) {
      double d = B[a][a];
      for (int p = 0; p < mk; ++p) d -= Lf[a][p] * Lf[a][p];
      // Lf[a][p] for kept p is filled below before use
      if (!(B[a][a] > 0.0) || !(d > drop2 * B[a][a])) continue;
      keep[mk] = a;
      Lf[a][mk] = sqrt(d);
      for (int r2 = a + 1; r2 < m; ++r2) {
        double e2 = B[r2][a];
        for (int p = 0; p < mk; ++p) e2 -= Lf[r2][p] * Lf[a][p];
        Lf[r2][mk] = e2 / Lf[a][mk];
      }
      ++mk;
    }
    for (int k = 0; k < kPodMax * kPodMax; ++k) {
      st->U[k] = 0.0;
      st->L[k] = 0.0;
    }
    for (int a = 0; a < mk; ++a) {
      for (int k = 0; k < n; ++k) st->U[k * kPodMax + a] = V[k][sel[keep[a]]];
      for (int b = 0; b <= a; ++b) st->L[a * kPodMax + b] = Lf[keep[a]][b];
    }
    st->m_used = mk;
    st->rebuild = 0;
    st->rebuilds += 1;
  }
}

// Per solve: c = X^T b over the stored snapshots, then (last block)
// a = U_m L^-T L^-1 U_m^T c by slot for k_proj_start, and the slots in use
// (0 while there is no basis: the start vector stays the previous solution).
template <int K>
__global__ void k_pod_gram(int nf, const double* __restrict__ X, const double* __restrict__ b, PodState* st,
                           double* __restrict__ coef, double* partials, unsigned int* counter,
                           int max_blocks) {
  pdl_enter();
  const int n = st->count, m = st->m_used;
  if (m == 0) {  // uniform over the grid
    if (blockIdx.x == 0 && threadIdx.x == 0) st->nuse = 0;
    return;
  }
  double v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0.0;
  for (int64_t i = gtid(); i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (k < n) v[k] = fma(X[(size_t)k * nf + i], bi, v[k]);
  }
  double tot[K];
  if (grid_sum<K>(v, partials, counter, max_blocks, tot) && threadIdx.x == 0) {
    double d[K], z[K], y[K];
    for (int a = 0; a < m; ++a) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc = fma(st->U[k * kPodMax + a], tot[k], acc);
      d[a] = acc;
    }
    for (int a = 0; a < m; ++a) {  // L z = d
      double e = d[a];
      for (int p = 0; p < a; ++p) e -= st->L[a * kPodMax + p] * z[p];
      z[a] = e / st->L[a * kPodMax + a];
    }
    for (int a = m - 1; a >= 0; --a) {  // L^T y = z
      double e = z[a];
      for (int r = a + 1; r < m; ++r) e -= st->L[r * kPodMax + a] * y[r];
      y[a] = e / st->L[a * kPodMax + a];
    }
    for (int k = 0; k < K; ++k) {
      double acc = 0.0;
      if (k < n)
        for (int a = 0; a < m; ++a) acc = fma(st->U[k * kPodMax + a], y[a], acc);
      coef[k] = acc;
    }
    st->nuse = n;
  }
}

}  // namespace eqs
