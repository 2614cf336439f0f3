// Host-side, run-once setup of the EQS RKC library:
//  - mesh validation and the internal node numbering (free nodes first);
//  - assembly of the constant matrix M of Eq. 2 (eps-weighted Laplacian of
//    the P1 or P2 elements)
//    restricted to free nodes, and M_fd 1_top (the Dirichlet coupling that
//    carries the drive into the right-hand side b of Eq. 2);
//  - the smoothed-aggregation AMG hierarchy of M_ff, built once and reused
//    by every stage solve (Section II: "once the preconditioner is set up,
//    it can be reused in every time-step");
//  - the RKC coefficients of the scheme cited in Section II (ref. [9]) and
//    the a-priori stability bound of the step size.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "eqs_internal.h"

namespace eqs {

static const double kEps0 = 8.8541878128e-12;  // F/m (CODATA 2018)

eqs_status validate_and_orient(eqs_ctx* c) {
  const int64_t n = c->n_nodes;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(c->xyz[i])) {
      c->err = "non-finite node coordinate";
      return EQS_ERR_MESH;
    }
  int64_t n_free = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (c->tag[i] > 2) {
      c->err = "node tag > 2 at node " + std::to_string(i);
      return EQS_ERR_MESH;
    }
    n_free += (c->tag[i] == 0);
  }
  if (n_free == 0) {
    c->err = "mesh has no free node";
    return EQS_ERR_MESH;
  }
  c->n_free = n_free;
  const int npe = c->npe;
  for (int64_t e = 0; e < c->n_tets; ++e) {
    const int32_t* t = &c->tets[(int64_t)npe * e];
    for (int k = 0; k < npe; ++k)
      if (t[k] < 0 || t[k] >= n) {
        c->err = "tet " + std::to_string(e) + " has node index out of range";
        return EQS_ERR_MESH;
      }
    const double* p0 = &c->xyz[3 * (int64_t)t[0]];
    double ed[3][3];
    for (int k = 0; k < 3; ++k) {
      const double* pk = &c->xyz[3 * (int64_t)t[k + 1]];
      for (int d = 0; d < 3; ++d) ed[k][d] = pk[d] - p0[d];
    }
    const double det = ed[0][0] * (ed[1][1] * ed[2][2] - ed[1][2] * ed[2][1]) -
                       ed[0][1] * (ed[1][0] * ed[2][2] - ed[1][2] * ed[2][0]) +
                       ed[0][2] * (ed[1][0] * ed[2][1] - ed[1][1] * ed[2][0]);
    if (!(det > 0.0)) {
      c->err = "tet " + std::to_string(e) + " is inverted or degenerate (det J <= 0)";
      return EQS_ERR_MESH;
    }
  }
  return EQS_OK;
}

void build_internal_numbering(eqs_ctx* c) {
  const int64_t n = c->n_nodes;
  c->internal_of_node.assign(n, -1);
  c->node_of_internal.assign(n, -1);
  int32_t next = 0;
  for (int64_t i = 0; i < n; ++i)
    if (c->tag[i] == 0) {
      c->internal_of_node[i] = next;
      c->node_of_internal[next++] = (int32_t)i;
    }
  for (int64_t i = 0; i < n; ++i)
    if (c->tag[i] != 0) {
      c->internal_of_node[i] = next;
      c->node_of_internal[next++] = (int32_t)i;
    }
}

// Gradients of the barycentric functions (rows of J^-1) and the volume.
static void tet_gradients(const double* xyz, const int32_t* t, double G[4][3], double& V) {
  const double* p0 = &xyz[3 * (int64_t)t[0]];
  double e[3][3];
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) e[k][d] = xyz[3 * (int64_t)t[k + 1] + d] - p0[d];
  // rows of J^-1 = (e2 x e3, e3 x e1, e1 x e2) / det
  double cr[3][3];
  for (int k = 0; k < 3; ++k) {
    const double* a = e[(k + 1) % 3];
    const double* b = e[(k + 2) % 3];
    cr[k][0] = a[1] * b[2] - a[2] * b[1];
    cr[k][1] = a[2] * b[0] - a[0] * b[2];
    cr[k][2] = a[0] * b[1] - a[1] * b[0];
  }
  const double det = e[0][0] * cr[0][0] + e[0][1] * cr[0][1] + e[0][2] * cr[0][2];
  for (int d = 0; d < 3; ++d) {
    G[1][d] = cr[0][d] / det;
    G[2][d] = cr[1][d] / det;
    G[3][d] = cr[2][d] / det;
    G[0][d] = -(G[1][d] + G[2][d] + G[3][d]);
  }
  V = det / 6.0;
}

// Row a of the local matrix integral of grad N_a . grad N_b over a P2 tet
// (vertices first, then the edges (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)),
// times w: the symmetric 4-point rule of degree 2 (exact: the integrand is
// quadratic).  grad N of vertex k = (4 l_k - 1) grad l_k, of edge (k, l) =
// 4 (l_k grad l_l + l_l grad l_k).
static const int kP2Edge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

static void p2_grad(const double G[4][3], const double lam[4], int i, double g[3]) {
  if (i < 4) {
    for (int d = 0; d < 3; ++d) g[d] = (4.0 * lam[i] - 1.0) * G[i][d];
  } else {
    const int k = kP2Edge[i - 4][0], l = kP2Edge[i - 4][1];
    for (int d = 0; d < 3; ++d) g[d] = 4.0 * (lam[k] * G[l][d] + lam[l] * G[k][d]);
  }
}

static void p2_row(const double G[4][3], double wV, int a, double row[10]) {
  const double qa = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, qb = (5.0 - std::sqrt(5.0)) / 20.0;
  for (int b = 0; b < 10; ++b) row[b] = 0.0;
  for (int q = 0; q < 4; ++q) {
    double lam[4] = {qb, qb, qb, qb};
    lam[q] = qa;
    double ga[3];
    p2_grad(G, lam, a, ga);
    for (int b = 0; b < 10; ++b) {
      double gb[3];
      p2_grad(G, lam, b, gb);
      row[b] += 0.25 * wV * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
    }
  }
}

// M = sum_e eps_e (integral of grad N_a . grad N_b): P1 eps_e V_e G_e G_e^T,
// P2 by quadrature; rows/cols of free nodes in internal numbering
// (= ascending mesh order); mtop = M_fd 1_top.
void assemble_M(const eqs_ctx* c, HostCSR& Mff, std::vector<double>& mtop) {
  const int64_t n = c->n_nodes, nf = c->n_free, nt = c->n_tets;
  const int npe = c->npe;
  // node -> tets incidence
  std::vector<int64_t> nptr(n + 1, 0);
  for (int64_t e = 0; e < nt; ++e)
    for (int k = 0; k < npe; ++k) nptr[c->tets[(int64_t)npe * e + k] + 1]++;
  for (int64_t i = 0; i < n; ++i) nptr[i + 1] += nptr[i];
  std::vector<int64_t> ntet(nptr[n]);
  {
    std::vector<int64_t> fill(nptr.begin(), nptr.end() - 1);
    for (int64_t e = 0; e < nt; ++e)
      for (int k = 0; k < npe; ++k) ntet[fill[c->tets[(int64_t)npe * e + k]]++] = e;
  }
  std::vector<double> eps(c->mats.size());
  for (size_t m = 0; m < c->mats.size(); ++m) eps[m] = kEps0 * c->mats[m].eps_r;

  Mff.n_rows = Mff.n_cols = nf;
  Mff.ptr.assign(nf + 1, 0);
  Mff.col.clear();
  Mff.val.clear();
  Mff.col.reserve(nf * 16);
  Mff.val.reserve(nf * 16);
  mtop.assign(nf, 0.0);
  std::vector<int64_t> pos(nf, -1);
  std::vector<int32_t> cols;
  std::vector<double> vals;
  for (int64_t r = 0; r < nf; ++r) {
    const int32_t node = c->node_of_internal[r];
    cols.clear();
    vals.clear();
    double top = 0.0;
    for (int64_t q = nptr[node]; q < nptr[node + 1]; ++q) {
      const int64_t e = ntet[q];
      const int32_t* t = &c->tets[(int64_t)npe * e];
      double G[4][3], V;
      tet_gradients(c->xyz.data(), t, G, V);
      int a = 0;
      while (t[a] != node) ++a;
      const double w = eps[c->tet_mat[e]] * V;
      double row[10];
      if (npe == 10)
        p2_row(G, w, a, row);
      else
        for (int b = 0; b < 4; ++b) row[b] = w * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
      for (int b = 0; b < npe; ++b) {
        const double v = row[b];
        const int32_t cn = c->internal_of_node[t[b]];
        if (cn >= nf) {
          if (c->tag[t[b]] == 2) top += v;
          continue;
        }
        if (pos[cn] < 0) {
          pos[cn] = (int64_t)cols.size();
          cols.push_back(cn);
          vals.push_back(v);
        } else {
          vals[pos[cn]] += v;
        }
      }
    }
    std::vector<int32_t> order(cols.size());
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return cols[x] < cols[y]; });
    for (int32_t o : order) {
      Mff.col.push_back(cols[o]);
      Mff.val.push_back(vals[o]);
      pos[cols[o]] = -1;
    }
    Mff.ptr[r + 1] = (int64_t)Mff.col.size();
    mtop[r] = top;
  }
}

// ------------------------------------------------------------ sparse tools
static HostCSR transpose(const HostCSR& A) {
  HostCSR T;
  T.n_rows = A.n_cols;
  T.n_cols = A.n_rows;
  T.ptr.assign(T.n_rows + 1, 0);
  for (int64_t k = 0; k < A.nnz(); ++k) T.ptr[A.col[k] + 1]++;
  for (int64_t i = 0; i < T.n_rows; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(A.nnz());
  T.val.resize(A.nnz());
  std::vector<int64_t> fill(T.ptr.begin(), T.ptr.end() - 1);
  for (int64_t i = 0; i < A.n_rows; ++i)
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const int64_t d = fill[A.col[k]]++;
      T.col[d] = (int32_t)i;
      T.val[d] = A.val[k];
    }
  return T;  // rows visited in order => columns sorted
}

static HostCSR spgemm(const HostCSR& A, const HostCSR& B) {
  HostCSR C;
  C.n_rows = A.n_rows;
  C.n_cols = B.n_cols;
  C.ptr.assign(C.n_rows + 1, 0);
  std::vector<int64_t> marker(B.n_cols, -1);
  std::vector<double> acc(B.n_cols, 0.0);
  std::vector<int32_t> cols;
  for (int64_t i = 0; i < A.n_rows; ++i) {
    cols.clear();
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const int32_t j = A.col[k];
      const double a = A.val[k];
      for (int64_t l = B.ptr[j]; l < B.ptr[j + 1]; ++l) {
        const int32_t cc = B.col[l];
        if (marker[cc] != i) {
          marker[cc] = i;
          cols.push_back(cc);
          acc[cc] = a * B.val[l];
        } else {
          acc[cc] += a * B.val[l];
        }
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t cc : cols) {
      C.col.push_back(cc);
      C.val.push_back(acc[cc]);
    }
    C.ptr[i + 1] = (int64_t)C.col.size();
  }
  return C;
}

static double diag_of(const HostCSR& A, int64_t i) {
  for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
    if (A.col[k] == i) return A.val[k];
  return 0.0;
}

// Smoothed aggregation (Vanek, Mandel, Brezina): level-scaled strength
// threshold, two-pass greedy aggregation in index order, column-normalised
// constant tentative prolongator, one damped-Jacobi smoothing step with
// omega = (4/3)/lambda (Gershgorin bound of rho(D^-1 A)), Galerkin P^T A P.
void build_hierarchy(const HostCSR& A0, const eqs_opts& o, std::vector<HostLevel>& lev) {
  lev.clear();
  lev.emplace_back();
  lev[0].A = A0;
  double theta = o.theta;
  while ((int)lev.size() < o.max_levels && lev.back().A.n_rows > o.coarse_max) {
    HostLevel& L = lev.back();
    const HostCSR& A = L.A;
    const int64_t n = A.n_rows;
    std::vector<double> d(n);
    for (int64_t i = 0; i < n; ++i) d[i] = diag_of(A, i);
    // strength graph
    std::vector<int64_t> sptr(n + 1, 0);
    std::vector<int32_t> scol;
    scol.reserve(A.nnz());
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
        const int32_t j = A.col[k];
        const double a = A.val[k];
        if (j != i && a != 0.0 && a * a >= theta * theta * std::fabs(d[i] * d[j])) scol.push_back(j);
      }
      sptr[i + 1] = (int64_t)scol.size();
    }
    // aggregation
    std::vector<int32_t> agg(n, -1);
    int32_t na = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (agg[i] >= 0) continue;
      bool free_nb = true;
      for (int64_t k = sptr[i]; k < sptr[i + 1] && free_nb; ++k) free_nb = agg[scol[k]] < 0;
      if (!free_nb) continue;
      agg[i] = na;
      for (int64_t k = sptr[i]; k < sptr[i + 1]; ++k) agg[scol[k]] = na;
      ++na;
    }
    std::vector<int32_t> agg1(agg);
    for (int64_t i = 0; i < n; ++i) {
      if (agg[i] >= 0) continue;
      int32_t pick = -1;
      for (int64_t k = sptr[i]; k < sptr[i + 1]; ++k)
        if (agg1[scol[k]] >= 0) {
          pick = agg1[scol[k]];
          break;
        }
      agg[i] = pick >= 0 ? pick : na++;
    }
    if (na >= n) break;
    // tentative prolongator
    std::vector<double> cnt(na, 0.0);
    for (int64_t i = 0; i < n; ++i) cnt[agg[i]] += 1.0;
    HostCSR P0;
    P0.n_rows = n;
    P0.n_cols = na;
    P0.ptr.resize(n + 1);
    P0.col.resize(n);
    P0.val.resize(n);
    for (int64_t i = 0; i < n; ++i) {
      P0.ptr[i] = i;
      P0.col[i] = agg[i];
      P0.val[i] = 1.0 / std::sqrt(cnt[agg[i]]);
    }
    P0.ptr[n] = n;
    // omega from the Gershgorin bound
    double lam = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) s += std::fabs(A.val[k]);
      lam = std::max(lam, s / d[i]);
    }
    const double omega = (4.0 / 3.0) / lam;
    HostCSR AP = spgemm(A, P0);
    // P = P0 - omega D^-1 A P0 (pattern of P0 is contained in that of A P0)
    HostCSR P = AP;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k) {
        double v = -omega * AP.val[k] / d[i];
        if (P.col[k] == agg[i]) v += P0.val[i];
        P.val[k] = v;
      }
    HostCSR Pt = transpose(P);
    HostCSR Ac = spgemm(Pt, spgemm(A, P));
    L.P = std::move(P);
    L.agg = std::move(agg);
    L.n_agg = na;
    L.omega = omega;
    lev.emplace_back();
    lev.back().A = std::move(Ac);
    theta *= 0.5;
  }
  for (auto& L : lev) {
    double lam = 0.0;
    for (int64_t i = 0; i < L.A.n_rows; ++i) {
      double s = 0.0;
      for (int64_t k = L.A.ptr[i]; k < L.A.ptr[i + 1]; ++k) s += std::fabs(L.A.val[k]);
      lam = std::max(lam, s / diag_of(L.A, i));
    }
    L.lam_max = lam;
  }
}

// Dense inverse of the (small) coarsest matrix by Cholesky.
bool dense_spd_inverse(const HostCSR& A, std::vector<double>& inv) {
  const int64_t n = A.n_rows;
  std::vector<double> L(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) L[i * n + A.col[k]] = A.val[k];
  for (int64_t j = 0; j < n; ++j) {
    double s = L[j * n + j];
    for (int64_t k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) return false;
    const double ljj = std::sqrt(s);
    L[j * n + j] = ljj;
    for (int64_t i = j + 1; i < n; ++i) {
      double t = L[i * n + j];
      for (int64_t k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / ljj;
    }
    for (int64_t i = 0; i < j; ++i) L[i * n + j] = 0.0;
  }
  inv.assign(n * n, 0.0);
  std::vector<double> y(n);
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = 0; i < n; ++i) {  // L y = e_c
      double t = (i == c) ? 1.0 : 0.0;
      for (int64_t k = 0; k < i; ++k) t -= L[i * n + k] * y[k];
      y[i] = t / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {  // L^T x = y
      double t = y[i];
      for (int64_t k = i + 1; k < n; ++k) t -= L[k * n + i] * inv[k * n + c];
      inv[i * n + c] = t / L[i * n + i];
    }
  }
  return true;
}

// RKC coefficients (damping 2/13): Chebyshev values T_j(w0), T_j', T_j''
// from their three-term recurrences; mu/nu/mu~/gamma~ for j = 1..s, stage
// abscissae c_0..c_s and the stability boundary beta = (1 + w0)/w1.
void rkc_coefficients(int s, std::vector<double>& mu, std::vector<double>& nu,
                      std::vector<double>& mut, std::vector<double>& gt, std::vector<double>& c,
                      double& beta) {
  const double eps = 2.0 / 13.0;
  const double w0 = 1.0 + eps / ((double)s * s);
  std::vector<double> T(s + 1, 0.0), dT(s + 1, 0.0), d2T(s + 1, 0.0);
  T[0] = 1.0;
  T[1] = w0;
  dT[1] = 1.0;
  for (int j = 2; j <= s; ++j) {
    T[j] = 2.0 * w0 * T[j - 1] - T[j - 2];
    dT[j] = 2.0 * T[j - 1] + 2.0 * w0 * dT[j - 1] - dT[j - 2];
    d2T[j] = 4.0 * dT[j - 1] + 2.0 * w0 * d2T[j - 1] - d2T[j - 2];
  }
  const double w1 = dT[s] / d2T[s];
  std::vector<double> b(s + 1, 0.0), a(s + 1, 0.0);
  for (int j = 2; j <= s; ++j) b[j] = d2T[j] / (dT[j] * dT[j]);
  b[0] = b[1] = b[2];
  for (int j = 0; j <= s; ++j) a[j] = 1.0 - b[j] * T[j];
  mu.assign(s + 1, 0.0);
  nu.assign(s + 1, 0.0);
  mut.assign(s + 1, 0.0);
  gt.assign(s + 1, 0.0);
  c.assign(s + 1, 0.0);
  mut[1] = b[1] * w1;
  for (int j = 2; j <= s; ++j) {
    mu[j] = 2.0 * b[j] * w0 / b[j - 1];
    nu[j] = -b[j] / b[j - 2];
    mut[j] = 2.0 * b[j] * w1 / b[j - 1];
    gt[j] = -a[j - 1] * mut[j];
    c[j] = w1 * d2T[j] / dT[j];
  }
  c[1] = c[2] / dT[2];
  beta = (1.0 + w0) / w1;
}

static double logistic(double u) {
  if (u >= 0) return 1.0 / (1.0 + std::exp(-u));
  const double e = std::exp(u);
  return e / (1.0 + e);
}

// sigma_d(E) = d(kappa E)/dE for the logistic law.
static double dkE(const eqs_material& m, double E) {
  const double s = logistic((E - m.E0) / m.w);
  return m.kappa_lo + (m.kappa_hi - m.kappa_lo) * (s + (E / m.w) * s * (1.0 - s));
}

double rho_bound(const std::vector<eqs_material>& mats) {
  double rho = 0.0;
  for (const auto& m : mats) {
    double kmax = std::max(m.kappa_lo, m.kappa_hi);
    if (m.kappa_hi != m.kappa_lo && m.w > 0) {
      // scan u = (E - E0)/w, then refine the bump's maximum by golden section
      double best = -1.0, bu = 0.0;
      for (double u = -m.E0 / m.w; u <= 60.0; u += 0.01) {
        const double v = dkE(m, m.E0 + u * m.w);
        if (v > best) best = v, bu = u;
      }
      double lo = bu - 0.02, hi = bu + 0.02;
      const double g = 0.5 * (std::sqrt(5.0) - 1.0);
      for (int it = 0; it < 200; ++it) {
        const double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
        if (dkE(m, m.E0 + x1 * m.w) > dkE(m, m.E0 + x2 * m.w))
          hi = x2;
        else
          lo = x1;
      }
      kmax = std::max(std::max(best, kmax), dkE(m, m.E0 + 0.5 * (lo + hi) * m.w));
    }
    rho = std::max(rho, kmax / (kEps0 * m.eps_r));
  }
  return rho;
}

}  // namespace eqs
