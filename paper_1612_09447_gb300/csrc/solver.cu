// Device orchestration and the C ABI of the EQS RKC library.
//
// One RKC step (Section II) is one CUDA graph: for every stage the element
// kernel (Section III) forms the right-hand side, and the M-solve (Section
// IV) runs as a device-side while-loop (conditional graph node) around the
// AMG V-cycle and the CG updates, so no host round trip happens inside a
// step.  Graphs are cached per (stages, output pointer).
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "kernels.cuh"
#include "mlp_kernels.cuh"
#include "batch_kernels.cuh"
#include <type_traits>

#include "spe_kernels.cuh"
#include "pod_kernels.cuh"
#include "ens_kernels.cuh"

using namespace eqs;

static thread_local std::string g_create_err = "no error";

static eqs_status fail(eqs_ctx* c, eqs_status st, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_err = msg;
  return st;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(c, EQS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

static inline int nblk(int64_t n, int b = kBlock) { return (int)((n + b - 1) / b); }

// Grid of a two-rows-per-thread row kernel: enough blocks for the work, at
// most the resident capacity (4 blocks of kBlock threads per SM).
static inline int rows_grid(const eqs_ctx* c, int64_t lanes) {
  return std::max(1, std::min(nblk((lanes + 1) / 2), 4 * c->sms));
}
// Grid of a row kernel on matrix A (rows_grid over its lanes).
template <typename T>
static inline int mat_grid(const eqs_ctx* c, const DevSell<T>& A, int64_t rows) {
  return rows_grid(c, rows * std::max(A.G, 1));
}
// Grid of a CG vector kernel (grid-stride, one reduction ticket per block).
static inline int vec_grid(const eqs_ctx* c, int64_t n) { return std::max(1, std::min(nblk(n), 4 * c->sms)); }

// Launch with programmatic dependent launch allowed (the kernels call
// pdl_enter() before touching memory), so consecutive kernels of a stream or
// graph overlap launch latency with the predecessor's tail.
static thread_local int64_t g_launches = 0;  // kernels enqueued by launch() (host-loop steps)

template <typename... KArgs, typename... Args>
static void launch(void (*k)(KArgs...), int grid, int block, cudaStream_t st, Args... args) {
  ++g_launches;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = st;
  cudaLaunchAttribute a[1];
  a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  a[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = a;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, ((KArgs)args)...);
}

// launch() with dynamic shared memory.
template <typename... KArgs, typename... Args>
static void launch_smem(void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args... args) {
  ++g_launches;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute a[1];
  a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  a[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = a;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, ((KArgs)args)...);
}


// ---------------------------------------------------------- device memory
static void free_all(eqs_ctx* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
}

template <typename T>
static cudaError_t dalloc(eqs_ctx* c, T** p, size_t n, bool zero = true) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) return e;
  c->allocs.push_back((void*)*p);
  if (zero) e = cudaMemset(*p, 0, n * sizeof(T));
  return e;
}

template <typename T>
static cudaError_t upload(eqs_ctx* c, T** p, const T* h, size_t n) {
  cudaError_t e = dalloc(c, p, n, false);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*p, h, n * sizeof(T), cudaMemcpyHostToDevice);
}

// Device buffer owned by one call (the checking / evaluation entry points
// that need a few bytes of their own); freed on every return path.
template <typename T>
struct TmpBuf {
  T* p = nullptr;
  TmpBuf() = default;
  TmpBuf(const TmpBuf&) = delete;
  TmpBuf& operator=(const TmpBuf&) = delete;
  ~TmpBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t n) { return cudaMalloc((void**)&p, n * sizeof(T)); }
};

// Puts a swapped pointer member back on every return path.
template <typename T>
struct PtrRestore {
  T** slot;
  T* saved;
  ~PtrRestore() { *slot = saved; }
};

// Lanes per row for a mean row length: 1 selects SELL-32 (thread per row).
static int lanes_for(double mean_row) {
  if (mean_row <= 16.0) return 1;
  if (mean_row <= 40.0) return 4;
  if (mean_row <= 80.0) return 8;
  if (mean_row <= 160.0) return 16;
  return 32;
}

template <typename T>
static cudaError_t upload_sell(eqs_ctx* c, const HostCSR& A, DevSell<T>& S, bool allow_groups = true) {
  S.n_rows = (int)A.n_rows;
  S.n_cols = (int)A.n_cols;
  S.n_slices = (int)((A.n_rows + 31) / 32);
  S.nnz = A.nnz();
  // DIA when the non-zeros lie on few diagonals with little padding
  {
    std::map<int64_t, int64_t> diag;
    bool ok = A.n_rows == A.n_cols && A.n_rows > 0;
    for (int64_t i = 0; ok && i < A.n_rows; ++i)
      for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
        diag[(int64_t)A.col[k] - i]++;
        if ((int)diag.size() > kMaxDiag) {
          ok = false;
          break;
        }
      }
    if (ok && (double)A.nnz() >= 0.6 * (double)A.n_rows * (double)diag.size()) {
      S.G = 0;
      S.logG = 0;
      S.ndiag = (int)diag.size();
      int d = 0;
      std::map<int64_t, int> slot;
      for (auto& kv : diag) {
        S.off[d] = (int)kv.first;
        slot[kv.first] = d++;
      }
      const int64_t n = A.n_rows;
      std::vector<T> val((size_t)n * S.ndiag, T(0));
      for (int64_t i = 0; i < n; ++i)
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
          val[(size_t)slot[(int64_t)A.col[k] - i] * n + i] = (T)A.val[k];
      S.stored = (int64_t)val.size();
      return upload(c, &S.val, val.data(), val.size());
    }
  }
  const double mean_row = A.n_rows ? (double)A.nnz() / (double)A.n_rows : 0.0;
  S.G = allow_groups ? lanes_for(mean_row) : 1;
  // small levels: more lanes per row until the rows fill the resident
  // threads (latency of long rows shared by a lane group, not serialised)
  if (allow_groups && c->opts.fill_lanes) {
    const int64_t resident = (int64_t)std::max(c->sms, 1) * 2048;
    while (S.G < 32 && S.G < mean_row && A.n_rows * (int64_t)S.G * 2 <= resident) S.G *= 2;
  }
  S.logG = 0;
  while ((1 << S.logG) < S.G) ++S.logG;
  if (S.G > 1) {  // CSR, G lanes per row
    std::vector<T> val(A.nnz());
    for (int64_t k = 0; k < A.nnz(); ++k) val[k] = (T)A.val[k];
    S.stored = A.nnz();
    cudaError_t e = upload(c, &S.slice_ptr, A.ptr.data(), A.ptr.size());
    if (e == cudaSuccess) e = upload(c, &S.col, A.col.data(), std::max<size_t>(A.col.size(), 1));
    if (e == cudaSuccess) e = upload(c, &S.val, val.data(), std::max<size_t>(val.size(), 1));
    return e;
  }
  std::vector<int64_t> sp(S.n_slices + 1, 0);
  for (int s = 0; s < S.n_slices; ++s) {
    int64_t w = 0;
    for (int l = 0; l < 32; ++l) {
      const int64_t r = (int64_t)s * 32 + l;
      if (r < A.n_rows) w = std::max<int64_t>(w, A.ptr[r + 1] - A.ptr[r]);
    }
    sp[s + 1] = sp[s] + 32 * w;
  }
  S.stored = sp[S.n_slices];
  std::vector<int32_t> col(std::max<int64_t>(S.stored, 1), 0);
  std::vector<T> val(std::max<int64_t>(S.stored, 1), T(0));
  for (int s = 0; s < S.n_slices; ++s) {
    const int64_t w = (sp[s + 1] - sp[s]) / 32;
    for (int l = 0; l < 32; ++l) {
      const int64_t r = (int64_t)s * 32 + l;
      if (r >= A.n_rows) continue;
      const int64_t len = A.ptr[r + 1] - A.ptr[r];
      for (int64_t k = 0; k < w; ++k) {
        const int64_t d = sp[s] + 32 * k + l;
        if (k < len) {
          col[d] = A.col[A.ptr[r] + k];
          val[d] = (T)A.val[A.ptr[r] + k];
        }
      }
    }
  }
  cudaError_t e = upload(c, &S.slice_ptr, sp.data(), sp.size());
  if (e == cudaSuccess) e = upload(c, &S.col, col.data(), col.size());
  if (e == cudaSuccess) e = upload(c, &S.val, val.data(), val.size());
  return e;
}

// Chebyshev coefficients of step k (2..deg): c1 = rho_k rho_{k-1},
// c2 = 2 rho_k / delta, rho_1 = 1/sigma, rho_k = 1/(2 sigma - rho_{k-1}).
static void cheb_coeffs(double sigma, double delta, int deg, std::vector<double>& c1,
                        std::vector<double>& c2) {
  c1.assign(deg + 1, 0.0);
  c2.assign(deg + 1, 0.0);
  double rho_old = 1.0 / sigma;
  for (int k = 2; k <= deg; ++k) {
    const double rho = 1.0 / (2.0 * sigma - rho_old);
    c1[k] = rho * rho_old;
    c2[k] = 2.0 * rho / delta;
    rho_old = rho;
  }
}

template <typename T>
static cudaError_t upload_levels(eqs_ctx* c, std::vector<DevLevel<T>>& L) {
  const int nl = (int)c->hlev.size();
  L.assign(nl, DevLevel<T>());
  for (int l = 0; l < nl; ++l) {
    const HostLevel& H = c->hlev[l];
    DevLevel<T>& D = L[l];
    D.n = (int)H.A.n_rows;
    D.lam_max = H.lam_max;
    const double lmin = H.lam_max / c->opts.cheb_alpha;
    const double theta = 0.5 * (H.lam_max + lmin);
    D.delta = 0.5 * (H.lam_max - lmin);
    D.sigma = theta / D.delta;
    D.inv_theta = 1.0 / theta;
    cudaError_t e = upload_sell(c, H.A, D.A);
    if (e != cudaSuccess) return e;
    if (l + 1 < nl) {
      if ((e = upload_sell(c, H.P, D.P)) != cudaSuccess) return e;
      HostCSR Pt;
      {  // transpose P for the restriction
        const HostCSR& P = H.P;
        Pt.n_rows = P.n_cols;
        Pt.n_cols = P.n_rows;
        Pt.ptr.assign(Pt.n_rows + 1, 0);
        for (int64_t k = 0; k < P.nnz(); ++k) Pt.ptr[P.col[k] + 1]++;
        for (int64_t i = 0; i < Pt.n_rows; ++i) Pt.ptr[i + 1] += Pt.ptr[i];
        Pt.col.resize(P.nnz());
        Pt.val.resize(P.nnz());
        std::vector<int64_t> fill(Pt.ptr.begin(), Pt.ptr.end() - 1);
        for (int64_t i = 0; i < P.n_rows; ++i)
          for (int64_t k = P.ptr[i]; k < P.ptr[i + 1]; ++k) {
            const int64_t d = fill[P.col[k]]++;
            Pt.col[d] = (int32_t)i;
            Pt.val[d] = P.val[k];
          }
      }
      if ((e = upload_sell(c, Pt, D.R)) != cudaSuccess) return e;
    }
    std::vector<T> dinv(D.n);
    for (int64_t i = 0; i < D.n; ++i) {
      double d = 0.0;
      for (int64_t k = H.A.ptr[i]; k < H.A.ptr[i + 1]; ++k)
        if (H.A.col[k] == i) d = H.A.val[k];
      dinv[i] = (T)(1.0 / d);
    }
    if ((e = upload(c, &D.dinv, dinv.data(), dinv.size())) != cudaSuccess) return e;
    for (T** v : {&D.b, &D.x, &D.r, &D.dA, &D.dB})
      if ((e = dalloc(c, v, D.n)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------ V-cycle
// Returns where the level's result lives: V.x, or V.dA after degree-1
// post-smoothing (the smoother writes the smoothed iterate there instead of
// updating x in place, so the prolongation above gathers one vector);
// nullptr when the fine level's last pass went into the CG dot products.
template <typename T>
static T* vcycle_level(eqs_ctx* c, std::vector<DevLevel<T>>& L, int l, cudaStream_t st,
                       bool fuse_dots = false, bool defer = false) {
  const int nl = (int)L.size();
  DevLevel<T>& V = L[l];
  if (l == nl - 1) {
    if constexpr (std::is_same<T, float>::value) {
      if (c->d_cinv32) {  // FP32 inverse, FP32 row sums
        launch_smem(k_coarse_solve32<1>, nblk((int64_t)V.n * 32), kBlock, (size_t)c->cinv_ld * sizeof(float), st,
                    V.n, c->cinv_ld, (const float*)c->d_cinv32, (const float*)V.b, (float*)V.x);
        return V.x;
      }
      if (c->d_cinv_hi) {  // FP32-pair application of the split inverse
        launch_smem(k_coarse_solve_df<1>, nblk((int64_t)V.n * 32), kBlock, (size_t)V.n * sizeof(float), st, V.n,
                    (const float*)c->d_cinv_hi, (const float*)c->d_cinv_lo, (const float*)V.b, (float*)V.x);
        return V.x;
      }
    }
    launch_smem(k_coarse_solve<T>, nblk((int64_t)V.n * 32), kBlock, (size_t)V.n * sizeof(double), st, V.n,
                c->d_coarse_inv, (const T*)V.b, V.x);
    return V.x;
  }
  const int deg = c->opts.cheb_degree;
  std::vector<double> c1, c2;
  cheb_coeffs(V.sigma, V.delta, deg, c1, c2);
  const int g = mat_grid(c, V.A, V.n);
  // pre-smoothing: x = d = D^-1 b / theta was set by the producer of b
  T* din = V.dA;
  T* dout = V.dB;
  const T* rin = V.b;
  for (int k = 2; k <= deg; ++k) {
    launch(k_cheb_step<T>, g, kBlock, st, V.A, V.n, rin, din, V.dinv, (T)c1[k], (T)c2[k], V.r, dout, V.x, 0);
    rin = V.r;
    std::swap(din, dout);
  }
  if (deg >= 2)
    launch(k_resid_update<T>, g, kBlock, st, V.A, V.n, V.r, din);
  else
    launch(k_resid<T>, g, kBlock, st, V.A, V.n, V.b, V.x, V.r);
  DevLevel<T>& C = L[l + 1];
  const int first = (l + 1 < nl - 1) ? 1 : 0;
  launch(k_restrict<T>, mat_grid(c, V.R, C.n), kBlock, st, V.R, C.n, V.r, C.b,
         C.dinv, (T)C.inv_theta, C.x, C.dA, first);
  const T* xc = vcycle_level(c, L, l + 1, st);
  launch(k_prolong<T>, mat_grid(c, V.P, V.n), kBlock, st, V.P, V.n, xc, (const T*)nullptr, V.x);
  if (fuse_dots && l == 0 && deg == 1) {  // the CG dot products ride on the last smoothing pass
    if (defer)
      launch(k_post_first_dots<T, true>, g, kBlock, st, V.A, V.n, (const T*)V.b, (const T*)V.x,
             (const T*)V.dinv, (T)V.inv_theta, (const double*)c->d_r, (const double*)c->d_rprev, c->d_zd,
             c->d_z32, c->d_sc, c->red.partials, c->red.counter, c->red.max_blocks, c->opts.flexible,
             c->d_dpart);
    else
      launch(k_post_first_dots<T, false>, g, kBlock, st, V.A, V.n, (const T*)V.b, (const T*)V.x,
             (const T*)V.dinv, (T)V.inv_theta, (const double*)c->d_r, (const double*)c->d_rprev, c->d_zd,
             c->d_z32, c->d_sc, c->red.partials, c->red.counter, c->red.max_blocks, c->opts.flexible,
             (double*)nullptr);
    return nullptr;
  }
  launch(k_post_first<T>, g, kBlock, st, V.A, V.n, V.b, V.x, V.dinv, (T)V.inv_theta, deg >= 2 ? V.r : nullptr,
         V.dA, deg == 1 ? 1 : 0);
  din = V.dA;
  dout = V.dB;
  for (int k = 2; k <= deg; ++k) {
    launch(k_cheb_step<T>, g, kBlock, st, V.A, V.n, V.r, din, V.dinv, (T)c1[k], (T)c2[k], V.r, dout, V.x,
           k == 2 ? 1 : 0);
    std::swap(din, dout);
  }
  return deg == 1 ? V.dA : V.x;
}

// ------------------------------------------------------------- PCG
struct SolveSlots {
  int* iters;
  double* relres;
  int* zero;
};

// A solve that starts from a projection start vector: SPE (stage j of an
// s-stage step) or POD (coefficients of the current basis).
struct SpeAt {
  int s, j;
  bool pod;
  bool learned;  // SPE start corrected along the network's direction
};

// Steps record each solution's distance from its SPE start (z - x0).
static bool recording_e(const eqs_ctx* c) {
  return c->recording && c->d_store_e &&
         (c->opts.guess == EQS_GUESS_SPE || c->opts.guess == EQS_GUESS_SPE_MLP);
}

// SPE projection of solve j (templated on the history length): the newest
// solution's product with M, the Gram column and the coefficients y.
// Two blocks per SM where they fit: the pass is bound by FP64 latency with
// 8 warps per SM; more blocks than are resident would run in a second wave.
template <int NH>
static int spe_gram_grid(eqs_ctx* c, int nf) {
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spe_gram<NH, false>, kBlock, 0) != cudaSuccess) occ = 1;
  const int bps = std::max(1, std::min(occ, 2));
  return std::max(1, std::min(nblk(nf), c->sms * bps));
}

// defer: leave the sums as per-block partials, added by one block of
// k_spe_solve (not launched when solve is false).
template <int NH>
static void spe_gram_n(eqs_ctx* c, cudaStream_t st, int s, int j, bool defer, bool solve = true) {
  const int nf = (int)c->n_free;
  const int grid = spe_gram_grid<NH>(c, nf);
  if (defer) {
    launch(k_spe_gram<NH, true>, grid, kBlock, st, c->M64, nf, (const double*)c->d_spe_X, c->d_spe_W,
           (const double*)c->d_R, (const long long*)c->d_stepcount, s, j, c->d_spe_G, c->d_spe_partials,
           c->red.counter, c->red.max_blocks, 1e-12, c->d_spe_y);
    if (solve)
      launch(k_spe_solve<NH>, 1, kBlock, st, (const long long*)c->d_stepcount, j, c->d_spe_G, 1e-12,
           (const double*)c->d_spe_partials, grid, c->red.max_blocks, c->d_spe_y);
  } else
    launch(k_spe_gram<NH, false>, grid, kBlock, st, c->M64, nf, (const double*)c->d_spe_X, c->d_spe_W,
           (const double*)c->d_R, (const long long*)c->d_stepcount, s, j, c->d_spe_G, c->d_spe_partials,
           c->red.counter, c->red.max_blocks, 1e-12, c->d_spe_y);
}

static void spe_gram(eqs_ctx* c, cudaStream_t st, int s, int j, bool defer, bool solve = true) {
  switch (c->opts.spe_n) {
    case 1: spe_gram_n<1>(c, st, s, j, defer, solve); break;
    case 2: spe_gram_n<2>(c, st, s, j, defer, solve); break;
    case 3: spe_gram_n<3>(c, st, s, j, defer, solve); break;
    case 4: spe_gram_n<4>(c, st, s, j, defer, solve); break;
    case 5: spe_gram_n<5>(c, st, s, j, defer, solve); break;
    default: spe_gram_n<6>(c, st, s, j, defer, solve); break;
  }
}

// x0 = X y and, unless R is null, r0 = R - W y with the first V-cycle input
// and the loop condition (the CG start of an SPE solve).
template <typename T, int NH>
static void spe_start_n(eqs_ctx* c, std::vector<DevLevel<T>>& L, cudaStream_t st, int s, int j,
                        const double* R, double* x, double tol2, cudaGraphConditionalHandle h,
                        int use_handle, SolveSlots sl, double* x_copy) {
  DevLevel<T>& V = L[0];
  const int nf = (int)c->n_free;
  launch(k_proj_start<T, NH>, vec_grid(c, nf), kBlock, st, c->M64, nf, (const double*)c->d_spe_X,
         (const double*)c->d_spe_W, (const double*)c->d_spe_y, (const int*)(c->d_spe_y + kSpeMax), R, x,
         R ? c->d_r : nullptr, V.dinv, (T)V.inv_theta, V.b, V.x, V.dA, c->d_sc, c->red.partials,
         c->red.counter, c->red.max_blocks, tol2, c->opts.max_iter, h, use_handle, sl.iters, sl.relres,
         sl.zero, x_copy);
}

// x_copy (nullable) also receives x0 (recording the distance of the
// solution from its SPE start).
template <typename T>
static void spe_start(eqs_ctx* c, std::vector<DevLevel<T>>& L, cudaStream_t st, int s, int j,
                      const double* R, double* x, double tol2, cudaGraphConditionalHandle h,
                      int use_handle, SolveSlots sl, double* x_copy = nullptr) {
  switch (c->opts.spe_n) {
    case 1: spe_start_n<T, 1>(c, L, st, s, j, R, x, tol2, h, use_handle, sl, x_copy); break;
    case 2: spe_start_n<T, 2>(c, L, st, s, j, R, x, tol2, h, use_handle, sl, x_copy); break;
    case 3: spe_start_n<T, 3>(c, L, st, s, j, R, x, tol2, h, use_handle, sl, x_copy); break;
    case 4: spe_start_n<T, 4>(c, L, st, s, j, R, x, tol2, h, use_handle, sl, x_copy); break;
    case 5: spe_start_n<T, 5>(c, L, st, s, j, R, x, tol2, h, use_handle, sl, x_copy); break;
    default: spe_start_n<T, 6>(c, L, st, s, j, R, x, tol2, h, use_handle, sl, x_copy); break;
  }
}


// POD start vector (Section IV): snapshot rule, basis rebuild when flagged,
// projection coefficients of the current right-hand side.  xnew is the
// newest solution, prev_iters / prev_zero the counters of its solve.
static void pod_prepare(eqs_ctx* c, cudaStream_t st, int s, int j, const double* xnew, const int* prev_iters,
                        const int* prev_zero, const long long* stepcount) {
  const int nf = (int)c->n_free;
  PodState* ps = (PodState*)c->d_pod_state;
  const int mode = c->opts.guess == EQS_GUESS_POD2 ? 1 : 0;
  launch(k_pod_add<kPodMax>, vec_grid(c, nf), kBlock, st, c->M64, nf, c->d_pod_X, c->d_pod_W, c->d_pod_GE,
         c->d_pod_GM, xnew, prev_iters, prev_zero, stepcount, s, j, mode, c->opts.pod_k, c->opts.pod_min_iters,
         ps, c->d_pod_partials, c->red.counter, c->red.max_blocks);
  launch(k_pod_rebuild<kPodMax>, 1, kBlock, st, (const double*)c->d_pod_GE, (const double*)c->d_pod_GM,
         c->opts.pod_m, kPodDrop2, ps);
  launch(k_pod_gram<kPodMax>, std::max(1, std::min(nblk(nf), c->sms)), kBlock, st, nf,
         (const double*)c->d_pod_X, (const double*)c->d_R, ps, c->d_pod_a, c->d_pod_partials, c->red.counter,
         c->red.max_blocks);
}

template <typename T>
static void pod_start(eqs_ctx* c, std::vector<DevLevel<T>>& L, cudaStream_t st, const double* R, double* x,
                      double tol2, cudaGraphConditionalHandle h, int use_handle, SolveSlots sl) {
  DevLevel<T>& V = L[0];
  const int nf = (int)c->n_free;
  PodState* ps = (PodState*)c->d_pod_state;
  launch(k_proj_start<T, kPodMax>, vec_grid(c, nf), kBlock, st, c->M64, nf, (const double*)c->d_pod_X,
         (const double*)c->d_pod_W, (const double*)c->d_pod_a, (const int*)&ps->nuse, R, x,
         R ? c->d_r : nullptr, V.dinv, (T)V.inv_theta, V.b, V.x, V.dA, c->d_sc, c->red.partials,
         c->red.counter, c->red.max_blocks, tol2, c->opts.max_iter, h, use_handle, sl.iters, sl.relres,
         sl.zero, (double*)nullptr);
}

// Stage vectors of a step: Y_j and the stage solutions F_j (rotating buffers).
static double* Ybuf(eqs_ctx* c, int j) { return j == 0 ? c->d_Y[0] : c->d_Y[1 + (j - 1) % 3]; }
static double* Fbuf(eqs_ctx* c, int j) { return j == 0 ? c->d_F[0] : c->d_F[1 + (j - 1) % 2]; }

// The learned correction of an SPE start (EQS_GUESS_SPE_MLP): the network's
// direction d from the increments around x0 (kept in d_x0), q = M d, the
// M-norm optimal step alpha, then x = x0 + alpha d and r = r0 - alpha q with
// the CG start redone on them.  d goes to d_rtmp, q to the CG vector q
// (its first pass does not read it).
template <typename T>
static void learned_correction(eqs_ctx* c, std::vector<DevLevel<T>>& L, cudaStream_t st, int s, int j, double* x,
                               double tol2, cudaGraphConditionalHandle h, int use_handle, SolveSlots sl,
                               int* kept) {
  DevLevel<T>& V = L[0];
  const int nf = (int)c->n_free;
  const double* h1 = Fbuf(c, j == 0 ? s - 1 : j - 1);
  const int* nuse = (const int*)(c->d_spe_y + kSpeMax);
  launch(k_rms_diff, vec_grid(c, nf), kBlock, st, nf, (const double*)c->d_x0, h1, nuse, c->d_sh,
         c->red.partials, c->red.counter, c->red.max_blocks);
  launch(k_mlp_dir_spe, std::max(1, std::min(nblk(nf), 4 * c->sms)), kBlock, st, nf, (const double*)c->d_x0, h1,
         (const float*)c->d_ring, (const long long*)c->d_stepcount, j, nuse, (const int32_t*)c->d_adj_ptr,
         (const int32_t*)c->d_adj_col, (const float*)c->d_inv_deg, (const __nv_bfloat16*)c->d_theta_bf16,
         (const double*)c->d_sh, c->d_rtmp);
  launch(k_dir_alpha, vec_grid(c, nf), kBlock, st, c->M64, nf, (const double*)c->d_rtmp, (const double*)c->d_r,
         (const double*)nullptr, (const double*)nullptr, c->d_q, c->d_alpha, c->red.partials, c->red.counter,
         c->red.max_blocks);
  launch(k_dir_apply<T>, vec_grid(c, nf), kBlock, st, nf, x, c->d_r, (const double*)c->d_rtmp,
         (const double*)c->d_q, (const double*)c->d_alpha, (const T*)V.dinv, (T)V.inv_theta, V.b, V.x, V.dA,
         c->d_sc, c->red.partials, c->red.counter, c->red.max_blocks, tol2, c->opts.max_iter, h, use_handle,
         sl.relres, kept);
}

template <typename T>
static void pcg_init_launch(eqs_ctx* c, std::vector<DevLevel<T>>& L, cudaStream_t st,
                            const double* R, double* x, double tol2, cudaGraphConditionalHandle h,
                            int use_handle, SolveSlots sl, const double* h1 = nullptr,
                            int* kept = nullptr, const SpeAt* spe = nullptr) {
  DevLevel<T>& V = L[0];
  const int n = (int)c->n_free;
  if (spe) {  // projection start vector: x0 = X y, r0 = R - W y (no SpMV)
    if (spe->pod)
      pod_start<T>(c, L, st, R, x, tol2, h, use_handle, sl);
    else
      spe_start<T>(c, L, st, spe->s, spe->j, R, x, tol2, h, use_handle, sl,
                   (recording_e(c) || spe->learned) ? c->d_x0 : nullptr);
    if (spe->learned) learned_correction<T>(c, L, st, spe->s, spe->j, x, tol2, h, use_handle, sl, kept);
    return;
  }
  if (h1) {  // learned start vector with the previous solution as fallback
    launch(k_pcg_init_dual<T>, vec_grid(c, n), kBlock, st, c->M64, n, R, x, h1, c->d_r, c->d_rtmp, V.dinv,
           (T)V.inv_theta, V.b, V.x, V.dA, c->d_sc, c->red.partials, c->red.counter,
           c->red.max_blocks, tol2, c->opts.max_iter, h, use_handle, sl.iters, sl.relres, sl.zero, kept);
    launch(k_pcg_select<T>, vec_grid(c, n), kBlock, st, n, x, h1, c->d_r, c->d_rtmp, V.dinv,
           (T)V.inv_theta, V.b, V.x, V.dA, (const PcgScalars*)c->d_sc);
    return;
  }
  launch(k_pcg_init<T>, vec_grid(c, n), kBlock, st, c->M64, n, R, x, c->d_r, V.dinv, (T)V.inv_theta, V.b, V.x,
         V.dA, c->d_sc, c->red.partials, c->red.counter, c->red.max_blocks, tol2, c->opts.max_iter, h,
         use_handle, sl.iters, sl.relres, sl.zero);
}

template <typename T>
static void pcg_body_launch(eqs_ctx* c, std::vector<DevLevel<T>>& L, cudaStream_t st, double* x,
                            double tol2, cudaGraphConditionalHandle h, int use_handle,
                            SolveSlots sl) {
  DevLevel<T>& V = L[0];
  const int n = (int)c->n_free;
  const int g = vec_grid(c, n);
  const bool fuse = c->opts.cheb_degree == 1 && L.size() > 1;
  // deferred sums: the dot products of the fused smoothing pass and of the
  // operator pass are added by the kernel that consumes them
  const bool defer = fuse && c->d_z32 && (c->opts.defer_sums & 1);
  const T* z = vcycle_level(c, L, 0, st, fuse, defer);
  if (!fuse)
    launch(k_pcg_dots<T>, g, kBlock, st, n, c->d_r, c->d_rprev, z, (const T*)nullptr, c->d_zd, c->d_z32,
           c->d_sc, c->red.partials, c->red.counter, c->red.max_blocks, c->opts.flexible);
  if (defer) {
    const int g_dots = mat_grid(c, V.A, V.n);  // the grid of k_post_first_dots
    launch(k_pcg_pq_split<true>, g, kBlock, st, c->M64, (const float*)c->d_M_hi, (const float*)c->d_M_lo, n,
           (const float*)c->d_z32, c->d_p, c->d_q, c->d_sc, c->red.partials, c->red.counter, c->red.max_blocks,
           c->d_dpart, g_dots, c->opts.flexible);
    launch(k_pcg_update<T, true>, g, kBlock, st, n, x, c->d_r, c->d_rprev, c->d_p, c->d_q, V.dinv,
           (T)V.inv_theta, V.b, V.x, V.dA, c->d_sc, c->red.partials, c->red.counter,
           c->red.max_blocks, tol2, c->opts.max_iter, h, use_handle, sl.iters, sl.relres,
           (const double*)c->d_dpart, g);
    return;
  }
  if (c->d_z32)  // mixed path: FP32 z, split-M operator pass
    launch(k_pcg_pq_split<false>, g, kBlock, st, c->M64, (const float*)c->d_M_hi, (const float*)c->d_M_lo, n,
           (const float*)c->d_z32, c->d_p, c->d_q, c->d_sc, c->red.partials, c->red.counter, c->red.max_blocks,
           (double*)nullptr, 0, c->opts.flexible);
  else
    launch(k_pcg_pq, g, kBlock, st, c->M64, n, c->d_zd, c->d_p, c->d_q, c->d_sc, c->red.partials,
           c->red.counter, c->red.max_blocks);
  launch(k_pcg_update<T, false>, g, kBlock, st, n, x, c->d_r, c->d_rprev, c->d_p, c->d_q, V.dinv,
         (T)V.inv_theta, V.b, V.x, V.dA, c->d_sc, c->red.partials, c->red.counter,
         c->red.max_blocks, tol2, c->opts.max_iter, h, use_handle, sl.iters, sl.relres,
         (const double*)nullptr, 0);
}

// Kernel nodes at the top level of graph g (loop bodies are not entered).
static int64_t count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
  int64_t k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess) return -1;
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// Append "init; while (not converged) body" to the graph being captured on
// c->cap_stream; the loop body is captured on c->cap_stream2.
template <typename T>
static eqs_status pcg_capture(eqs_ctx* c, std::vector<DevLevel<T>>& L, const double* R, double* x,
                              double tol2, SolveSlots sl, const double* h1 = nullptr, int* kept = nullptr,
                              const SpeAt* spe = nullptr) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(c->cap_stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  pcg_init_launch<T>(c, L, c->cap_stream, R, x, tol2, h, 1, sl, h1, kept, spe);
  CK(cudaGetLastError());
  CK(cudaStreamGetCaptureInfo(c->cap_stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(c->cap_stream2, body, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeRelaxed));
  pcg_body_launch<T>(c, L, c->cap_stream2, x, tol2, h, 1, sl);
  cudaError_t le = cudaGetLastError();
  cudaGraph_t body_out = nullptr;
  CK(cudaStreamEndCapture(c->cap_stream2, &body_out));
  CK(le);
  c->body_kernels = count_kernel_nodes(body_out);
  CK(cudaStreamUpdateCaptureDependencies(c->cap_stream, &node, nullptr, 1,
                                         cudaStreamSetCaptureDependencies));
  return EQS_OK;
}

// ------------------------------------------------------ persistent solve
template <typename T>
static eqs_status build_plan(eqs_ctx* c, std::vector<DevLevel<T>>& L) {
  if ((int)L.size() > kMaxLevels) return fail(c, EQS_ERR_ARG, "too many AMG levels for the persistent solve");
  PPlan<T> P{};
  P.nl = (int)L.size();
  P.deg = c->opts.cheb_degree;
  P.nf = (int)c->n_free;
  P.maxit = c->opts.max_iter;
  P.flexible = c->opts.flexible;
  P.max_spins = c->opts.barrier_polls > 0 ? (long long)c->opts.barrier_polls
                                          : (c->opts.barrier_polls == 0 ? kMaxSpins : 0);
  P.coarse_inv = c->d_coarse_inv;
  P.M = c->M64;
  P.r = c->d_r;
  P.rprev = c->d_rprev;
  P.pA = c->d_p;
  P.pB = c->d_p2;
  P.q = c->d_q;
  P.zd = c->d_zd;
  int dev = 0, sms = 0, occ = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg_persistent<T>, kPBlock, 0));
  if (occ < 1) return fail(c, EQS_ERR_CUDA, "persistent solve kernel cannot be resident");
  const int bps = std::min(occ, std::max(1, c->opts.blocks_per_sm));
  c->pblocks = sms * bps;
  CK(dalloc(c, &c->d_ppartials, 16 * (size_t)c->pblocks));
  GridBarrier* bar = nullptr;
  CK(dalloc(c, &bar, 1));
  c->d_bar = bar;
  P.partials = c->d_ppartials;
  P.bar = bar;
  for (int l = 0; l < P.nl; ++l) {
    DevLevel<T>& D = L[l];
    PLevel<T>& Q = P.lev[l];
    Q.A = D.A;
    Q.P = D.P;
    Q.R = D.R;
    Q.dinv = D.dinv;
    Q.b = D.b;
    Q.x = D.x;
    Q.r = D.r;
    Q.dA = D.dA;
    Q.dB = D.dB;
    Q.n = D.n;
    Q.inv_theta = (T)D.inv_theta;
    std::vector<double> c1, c2;
    cheb_coeffs(D.sigma, D.delta, P.deg, c1, c2);
    for (int k = 0; k <= P.deg && k < 5; ++k) {
      Q.c1[k] = (T)c1[k];
      Q.c2[k] = (T)c2[k];
    }
  }
  PPlan<T>* dp = nullptr;
  CK(upload(c, &dp, &P, 1));
  c->d_plan = dp;
  return EQS_OK;
}

template <typename T>
static eqs_status persistent_launch(eqs_ctx* c, cudaStream_t st, const double* R, double* x,
                                    double tol2, SolveSlots sl) {
  CK(cudaMemsetAsync(c->d_bar, 0, sizeof(GridBarrier), st));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->pblocks);
  cfg.blockDim = dim3(kPBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CK(cudaLaunchKernelEx(&cfg, k_pcg_persistent<T>, (const PPlan<T>*)c->d_plan, R, x, sl.iters,
                        sl.relres, sl.zero, tol2));
  return EQS_OK;
}

// CG loop driven from the host (same kernels; the convergence flag is read
// back after every iteration).  Used by the host-loop execution mode.
template <typename T>
static eqs_status pcg_direct(eqs_ctx* c, std::vector<DevLevel<T>>& L, const double* R, double* x,
                             double tol2, SolveSlots sl, const double* h1, int* kept, const SpeAt* spe) {
  cudaStream_t st = c->stream;
  pcg_init_launch<T>(c, L, st, R, x, tol2, 0, 0, sl, h1, kept, spe);
  for (int it = 0; it < c->opts.max_iter; ++it) {
    int conv = 0;
    CK(cudaMemcpyAsync(&conv, &c->d_sc->conv, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (conv) break;
    pcg_body_launch<T>(c, L, st, x, tol2, 0, 0, sl);
  }
  CK(cudaGetLastError());
  return EQS_OK;
}

template <typename T>
static eqs_status solve_launch(eqs_ctx* c, std::vector<DevLevel<T>>& L, const double* R, double* x,
                               double tol2, SolveSlots sl, const double* h1 = nullptr, int* kept = nullptr,
                               const SpeAt* spe = nullptr) {
  if (c->direct) return pcg_direct<T>(c, L, R, x, tol2, sl, h1, kept, spe);
  if (c->opts.persistent && !h1 && !(spe && spe->learned)) {
    // the persistent kernel forms its own initial residual: only x0 here
    if (spe && spe->pod) pod_start<T>(c, L, c->cap_stream, nullptr, x, tol2, 0, 0, sl);
    else if (spe) spe_start<T>(c, L, c->cap_stream, spe->s, spe->j, nullptr, x, tol2, 0, 0, sl);
    return persistent_launch<T>(c, c->cap_stream, R, x, tol2, sl);
  }
  return pcg_capture<T>(c, L, R, x, tol2, sl, h1, kept, spe);
}

static bool mixed(const eqs_ctx* c) { return c->opts.precision == EQS_PREC_MIXED; }

// ------------------------------------------------------------ element
// Mixed precision reads the two-float potential Y2 (default: c->d_Y32).
static void elem_launch(eqs_ctx* c, cudaStream_t st, const double* Y, int n_limit, double* y64,
                        float* y32, const float2* Y2 = nullptr) {
  const float2* y2in = Y2 ? Y2 : c->d_Y32;
  if (c->npe == 10) {  // quadratic tets
    if (mixed(c))
      launch(k_elem32_p2, nblk(c->n_tets), kBlock, st, c->n_tets, (const int32_t*)c->d_conn10,
             (const uint8_t*)c->d_mat, (const MaterialDev*)c->d_mats, (const float4*)c->d_xyz_hi,
             (const float4*)c->d_xyz_lo, y2in, n_limit, y32);
    else
      launch(k_elem64_p2, nblk(c->n_tets), kBlock, st, c->n_tets, (const int32_t*)c->d_conn10,
             (const uint8_t*)c->d_mat, (const MaterialDev*)c->d_mats, (const double4*)c->d_xyz, Y, n_limit,
             y64 == c->d_R ? -1.0 : 1.0, y64);
    return;
  }
  if (c->n_cells > 0) {  // Kuhn cells: 8 atomic adds per six tets
    if (mixed(c))
      launch(k_elem32_cell, nblk(c->n_cells), kBlock, st, c->n_cells, (const int32_t*)c->d_corner,
             (const uint8_t*)c->d_mat, (const MaterialDev*)c->d_mats, (const float4*)c->d_xyz_hi,
             (const float4*)c->d_xyz_lo, y2in, n_limit, y32);
    else
      launch(k_elem64_cell, nblk(c->n_cells), kBlock, st, c->n_cells, (const int32_t*)c->d_corner,
             (const uint8_t*)c->d_mat, (const MaterialDev*)c->d_mats, (const double4*)c->d_xyz, Y, n_limit,
             y64 == c->d_R ? -1.0 : 1.0, y64);
    return;
  }
  if (mixed(c))
    launch(k_elem32, nblk(c->n_tets), kBlock, st, c->n_tets, c->d_conn, c->d_mat, c->d_mats,
                                                 c->d_xyz_hi, c->d_xyz_lo, y2in, n_limit, y32);
  else
    launch(k_elem64, nblk(c->n_tets), kBlock, st, c->n_tets, c->d_conn, c->d_mat, c->d_mats, c->d_xyz,
                                                 Y, n_limit, y64 == c->d_R ? -1.0 : 1.0, y64);
}

// -------------------------------------------------------- step graph


// Enqueue one RKC step on st: captured into a graph (c->direct false) or
// launched directly with a host-driven CG loop (c->direct true).  The
// caller's x is read and written through the parameter block
// (c->d_params->x), so a captured step does not depend on it.
template <typename T>
static eqs_status enqueue_step(eqs_ctx* c, std::vector<DevLevel<T>>& L, int s, const double* d_cj,
                               cudaStream_t st) {
  std::vector<double> mu, nu, mut, gt, cj;
  double beta;
  rkc_coefficients(s, mu, nu, mut, gt, cj, beta);
  const int n = (int)c->n_nodes, nf = (int)c->n_free;
  const double tol2 = c->opts.rtol * c->opts.rtol;
  const double w = 2.0 * M_PI * c->freq;
  launch(k_stage_scalars, 1, 64, st, s + 1, d_cj, c->d_params, c->V0, w, c->phase, c->d_g, c->d_gp,
         c->d_stepcount);
  const bool mx = mixed(c);
  launch(k_gather_state, nblk(n), kBlock, st, n, nf, (const StepParams*)c->d_params, c->d_node_of_internal,
         c->d_dir_scale, c->d_g,
                                             c->d_gp, c->d_mtop, Ybuf(c, 0), mx ? c->d_Y32 : nullptr,
                                             Fbuf(c, s - 1), Fbuf(c, 0), mx ? nullptr : c->d_R);
  eqs_status stt = EQS_OK;
  for (int j = 0; j <= s && stt == EQS_OK; ++j) {
    if (j >= 1) {
      const bool first = (j == 1);
      const double c0 = first ? 1.0 : 1.0 - mu[j] - nu[j];
      const bool last = (j == s);
      launch(k_recurrence, nblk(n), kBlock, st, 
          n, nf, c0, first ? 0.0 : mu[j], first ? 0.0 : nu[j], mut[j], first ? 0.0 : gt[j], c->d_params,
          Ybuf(c, 0), Ybuf(c, j - 1), Ybuf(c, j >= 2 ? j - 2 : 0), Fbuf(c, j - 1), Fbuf(c, 0), c->d_zero,
          j - 1, c->d_dir_scale, c->d_g + j, c->d_gp + j, c->d_mtop, Ybuf(c, j),
          (mx && !last) ? c->d_Y32 : nullptr, last ? nullptr : Fbuf(c, j),
          (mx || last) ? nullptr : c->d_R, last ? 1 : 0, c->d_node_of_internal, c->d_ring,
          (const long long*)c->d_stepcount, s, c->recording ? c->d_store : nullptr, (long long)c->store_cap,
          c->d_spe_X, c->opts.spe_n, recording_e(c) ? c->d_store_e : nullptr, (const double*)c->d_x0);
      if (last) break;
    }
    if (mx) {
      elem_launch(c, st, nullptr, nf, nullptr, c->d_y32);
      launch(k_rhs_from_y32, nblk(nf), kBlock, st, nf, c->d_y32, c->d_gp + j, c->d_mtop, c->d_R);
    } else {
      elem_launch(c, st, Ybuf(c, j), nf, c->d_R, nullptr);
    }
    SolveSlots sl{c->d_iters + j, c->d_relres + j, c->d_zero + j};
    if (c->opts.guess == EQS_GUESS_MLP) {
      const double* h1 = Fbuf(c, j == 0 ? s - 1 : j - 1);
      launch(k_rms, vec_grid(c, nf), kBlock, st, nf, h1, c->d_sh, c->red.partials, c->red.counter,
             c->red.max_blocks);
      launch(k_mlp_guess, std::max(1, std::min(nblk(nf), 4 * c->sms)), kBlock, st, nf, h1,
             (const float*)c->d_ring, (const long long*)c->d_stepcount, s, j, (const int32_t*)c->d_adj_ptr,
             (const int32_t*)c->d_adj_col, (const float*)c->d_inv_deg,
             (const __nv_bfloat16*)c->d_theta_bf16, (const double*)c->d_sh, Fbuf(c, j));
      stt = solve_launch<T>(c, L, c->d_R, Fbuf(c, j), tol2, sl, h1, c->d_mlp_used + j);
    } else if (c->opts.guess == EQS_GUESS_SPE) {
      spe_gram(c, st, s, j, (c->opts.defer_sums & 2) != 0);
      const SpeAt at{s, j, false, false};
      stt = solve_launch<T>(c, L, c->d_R, Fbuf(c, j), tol2, sl, nullptr, nullptr, &at);
    } else if (c->opts.guess == EQS_GUESS_SPE_MLP) {
      // the SPE start, corrected along the network's direction (line search in the M-norm)
      spe_gram(c, st, s, j, (c->opts.defer_sums & 2) != 0);
      const SpeAt at{s, j, false, true};
      stt = solve_launch<T>(c, L, c->d_R, Fbuf(c, j), tol2, sl, nullptr, c->d_mlp_used + j, &at);
    } else if (c->opts.guess == EQS_GUESS_POD || c->opts.guess == EQS_GUESS_POD2) {
      const int jp = j == 0 ? s - 1 : j - 1;  // the solve that produced the newest solution
      pod_prepare(c, st, s, j, Fbuf(c, jp), c->d_iters + jp, c->d_zero + jp, (const long long*)c->d_stepcount);
      const SpeAt at{s, j, true, false};
      stt = solve_launch<T>(c, L, c->d_R, Fbuf(c, j), tol2, sl, nullptr, nullptr, &at);
    } else {
      if (c->opts.guess == EQS_GUESS_ZERO && cudaMemsetAsync(Fbuf(c, j), 0, nf * sizeof(double), st) != cudaSuccess)
        stt = fail(c, EQS_ERR_CUDA, "cudaMemsetAsync failed during capture");
      stt = solve_launch<T>(c, L, c->d_R, Fbuf(c, j), tol2, sl);
    }
  }
  return stt;
}

template <typename T>
static eqs_status capture_step(eqs_ctx* c, std::vector<DevLevel<T>>& L, int s, GraphEntry& ge) {
  std::vector<double> mu, nu, mut, gt, cj;
  double beta;
  rkc_coefficients(s, mu, nu, mut, gt, cj, beta);
  CK(upload(c, &ge.d_cj, cj.data(), cj.size()));
  cudaStream_t st = c->cap_stream;
  c->direct = false;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  eqs_status stt = enqueue_step<T>(c, L, s, ge.d_cj, st);
  cudaError_t le = cudaGetLastError();
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  if (stt != EQS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return stt;
  }
  CK(le);
  CK(ee);
  ge.graph = graph;
  ge.s = s;
  ge.fixed_kernels = count_kernel_nodes(graph);
  ge.per_iter_kernels = c->body_kernels;
  CK(cudaGraphInstantiate(&ge.exec, graph, 0));
  return EQS_OK;
}

// F(t, x) = M_ff^-1 (-[K(x~)x~]_f - g'(t) M_fd 1_top) into Fout (internal
// order; its content is the CG start vector): the stage evaluation of a step
// as a graph of its own (time from the device parameters).
template <typename T>
static eqs_status enqueue_eval_F(eqs_ctx* c, std::vector<DevLevel<T>>& L, double* Fout, cudaStream_t st) {
  const int n = (int)c->n_nodes, nf = (int)c->n_free;
  const bool mx = mixed(c);
  const double w = 2.0 * M_PI * c->freq;
  launch(k_stage_scalars, 1, 64, st, 1, (const double*)c->d_cj0, (const StepParams*)c->d_params, c->V0, w,
         c->phase, c->d_g, c->d_gp, c->d_evalcount);
  launch(k_gather_state, nblk(n), kBlock, st, n, nf, (const StepParams*)c->d_params,
         (const int32_t*)c->d_node_of_internal,
         (const double*)c->d_dir_scale, (const double*)c->d_g, (const double*)c->d_gp, (const double*)c->d_mtop,
         c->d_tmpn, mx ? c->d_Y32 : nullptr, (const double*)nullptr, (double*)nullptr, mx ? nullptr : c->d_R);
  if (mx) {
    elem_launch(c, st, nullptr, nf, nullptr, c->d_y32);
    launch(k_rhs_from_y32, nblk(nf), kBlock, st, nf, c->d_y32, (const double*)c->d_gp, (const double*)c->d_mtop,
           c->d_R);
  } else {
    elem_launch(c, st, c->d_tmpn, nf, c->d_R, nullptr);
  }
  SolveSlots sl{c->d_iters + EQS_MAX_STAGES, c->d_relres + EQS_MAX_STAGES, c->d_zero + EQS_MAX_STAGES};
  const double tol2 = c->opts.rtol * c->opts.rtol;
  return solve_launch<T>(c, L, c->d_R, Fout, tol2, sl);
}

template <typename T>
static eqs_status capture_eval_F(eqs_ctx* c, std::vector<DevLevel<T>>& L, double* Fout, GraphEntry& ge) {
  cudaStream_t st = c->cap_stream;
  c->direct = false;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  const eqs_status stt = enqueue_eval_F<T>(c, L, Fout, st);
  cudaError_t le = cudaGetLastError();
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  if (stt != EQS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return stt;
  }
  CK(le);
  CK(ee);
  ge.graph = graph;
  CK(cudaGraphInstantiate(&ge.exec, graph, 0));
  return EQS_OK;
}

template <typename T>
static eqs_status capture_solve(eqs_ctx* c, std::vector<DevLevel<T>>& L, double rtol, GraphEntry& ge) {
  cudaStream_t st = c->cap_stream;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  SolveSlots sl{c->d_iters, c->d_relres, c->d_zero};
  eqs_status stt = solve_launch<T>(c, L, c->d_R, c->d_sol, rtol * rtol, sl);
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  if (stt != EQS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return stt;
  }
  CK(ee);
  ge.graph = graph;
  CK(cudaGraphInstantiate(&ge.exec, graph, 0));
  return EQS_OK;
}

static void destroy_graph(GraphEntry& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  g.exec = nullptr;
  g.graph = nullptr;
}

static void destroy_graphs(eqs_ctx* c) {
  c->last_step = nullptr;
  for (auto& kv : c->step_graphs) destroy_graph(kv.second);
  c->step_graphs.clear();
  for (auto& kv : c->solve_graphs) destroy_graph(kv.second);
  c->solve_graphs.clear();
  destroy_graph(c->eval_graph);
  c->ens_last = nullptr;
  for (auto& kv : c->ens_graphs) destroy_graph(kv.second);
  c->ens_graphs.clear();
  destroy_graph(c->ens_solve_graph);
  c->ens_solve_tol = -1.0;
}

template <typename T>
static eqs_status vcycle_impl(eqs_ctx* c, std::vector<DevLevel<T>>& L, const double* r, double* z) {
  const int nf = (int)c->n_free;
  cudaStream_t st = c->stream;
  DevLevel<T>& V = L[0];
  launch(k_to_T<T>, nblk(nf), kBlock, st, nf, r, V.b);
  if (L.size() > 1) launch(k_first_step<T>, nblk(nf), kBlock, st, nf, V.b, V.dinv, (T)V.inv_theta, V.x, V.dA);
  const T* res = vcycle_level(c, L, 0, st);
  launch(k_from_T<T>, nblk(nf), kBlock, st, nf, res, z);
  CK(cudaGetLastError());
  return EQS_OK;
}

// ------------------------------------------------------------ ensemble
// Four trajectories on one context (row-interleaved vectors); mixed
// precision with the previous-solution start vector.
static eqs_status ens_alloc(eqs_ctx* c) {
  if (c->ens_ready) return EQS_OK;
  if (!mixed(c) || !c->d_M_hi || !(c->d_cinv_hi || c->d_cinv32))
    return fail(c, EQS_ERR_STATE, "the ensemble needs a context set up in EQS_PREC_MIXED with split_m 1");
  if (c->npe != 4) return fail(c, EQS_ERR_STATE, "the ensemble runs linear (4-node) tets");
  if (c->opts.guess != EQS_GUESS_PREV && c->opts.guess != EQS_GUESS_SPE)
    return fail(c, EQS_ERR_STATE, "the ensemble starts from EQS_GUESS_PREV or EQS_GUESS_SPE");
  const int64_t n = c->n_nodes, nf = c->n_free;
  c->elev.assign(c->lev32.size(), eqs_ctx::EnsLevel());
  for (size_t l = 0; l < c->lev32.size(); ++l) {
    const int nl = c->lev32[l].n;
    eqs_ctx::EnsLevel& E = c->elev[l];
    for (float4** v : {&E.b, &E.x, &E.r, &E.dA, &E.dB}) CK(dalloc(c, v, nl));
  }
  for (auto& y : c->d_eY) CK(dalloc(c, &y, n));
  CK(dalloc(c, &c->d_eY2, 2 * n));
  for (auto& f : c->d_eF) CK(dalloc(c, &f, nf));
  for (double4_32a** v : {&c->d_eR, &c->d_er, &c->d_ep, &c->d_eq, &c->d_esol}) CK(dalloc(c, v, nf));
  CK(dalloc(c, &c->d_ey32, n));
  CK(dalloc(c, &c->d_ez32, nf));
  EnsScalars* sc = nullptr;
  CK(dalloc(c, &sc, 1));
  c->d_esc = sc;
  CK(dalloc(c, &c->d_epart, 2 * kEnsW * (size_t)c->red.max_blocks));
  CK(dalloc(c, &c->d_eiters, (EQS_MAX_STAGES + 1) * kEnsW));
  CK(dalloc(c, &c->d_erelres, (EQS_MAX_STAGES + 1) * kEnsW));
  CK(dalloc(c, &c->d_ezero, (EQS_MAX_STAGES + 1) * kEnsW));
  CK(dalloc(c, &c->d_ecolv, kEnsW));
  CK(dalloc(c, &c->d_eX, (size_t)kEnsSpe * nf));
  CK(dalloc(c, &c->d_eW, (size_t)kEnsSpe * nf));
  CK(dalloc(c, &c->d_eX2, (size_t)kEnsSpe * 2 * nf));
  CK(dalloc(c, &c->d_eR2, (size_t)2 * nf));
  CK(dalloc(c, &c->d_eG, (size_t)kEnsW * kSpeMax * kSpeMax));
  CK(dalloc(c, &c->d_ecoef, (size_t)kEnsW * (kSpeMax + 1)));
  CK(dalloc(c, &c->d_espart, 2 * (size_t)kEnsSpe * kEnsW * c->red.max_blocks));
  CK(dalloc(c, &c->d_estepcount, 2));
  c->ens_ready = true;
  return EQS_OK;
}

// The fine level's first Chebyshev direction, written with the V-cycle input
// only when a degree >= 2 smoother reads it.
static float4* ens_d0(eqs_ctx* c) { return c->opts.cheb_degree >= 2 ? c->elev[0].dA : nullptr; }

// V-cycle of the four columns from level l; returns where the level's
// result lives (E.x, or E.dA after degree-1 post-smoothing, which writes the
// smoothed iterate there instead of updating E.x in place), nullptr when the
// fine level's last pass went into the CG dot products.
static const float4* ens_vcycle_level(eqs_ctx* c, int l, cudaStream_t st, bool fuse_dots = false) {
  std::vector<DevLevel<float>>& L = c->lev32;
  const int nl = (int)L.size();
  DevLevel<float>& V = L[l];
  eqs_ctx::EnsLevel& E = c->elev[l];
  if (l == nl - 1) {
    if (c->d_cinv32)
      launch_smem(k_coarse_solve32<4>, nblk((int64_t)V.n * 32), kBlock, (size_t)c->cinv_ld * sizeof(float4), st,
                  V.n, c->cinv_ld, (const float*)c->d_cinv32, (const float*)E.b, (float*)E.x);
    else
      launch_smem(k_coarse_solve_df<4>, nblk((int64_t)V.n * 32), kBlock, (size_t)V.n * sizeof(float4), st, V.n,
                  (const float*)c->d_cinv_hi, (const float*)c->d_cinv_lo, (const float*)E.b, (float*)E.x);
    return E.x;
  }
  const int deg = c->opts.cheb_degree;
  std::vector<double> c1, c2;
  cheb_coeffs(V.sigma, V.delta, deg, c1, c2);
  const int g = mat_grid(c, V.A, V.n);
  float4* din = E.dA;
  float4* dout = E.dB;
  const float4* rin = E.b;
  for (int k = 2; k <= deg; ++k) {
    launch(k4_cheb_step, g, kBlock, st, V.A, V.n, rin, (const float4*)din, (const float*)V.dinv, (float)c1[k],
           (float)c2[k], E.r, dout, E.x, 0);
    rin = E.r;
    std::swap(din, dout);
  }
  if (deg >= 2)
    launch(k4_resid_update, g, kBlock, st, V.A, V.n, E.r, (const float4*)din);
  else
    launch(k4_resid, g, kBlock, st, V.A, V.n, (const float4*)E.b, (const float4*)E.x, E.r);
  DevLevel<float>& C = L[l + 1];
  eqs_ctx::EnsLevel& EC = c->elev[l + 1];
  const int first = (l + 1 < nl - 1) ? 1 : 0;
  launch(k4_restrict, mat_grid(c, V.R, C.n), kBlock, st, V.R, C.n, (const float4*)E.r,
         EC.b, (const float*)C.dinv, (float)C.inv_theta, EC.x, deg >= 2 ? EC.dA : nullptr, first);
  const float4* xc = ens_vcycle_level(c, l + 1, st);
  launch(k4_prolong, mat_grid(c, V.P, V.n), kBlock, st, V.P, V.n, xc, (const float4*)nullptr, E.x);
  if (fuse_dots && l == 0 && deg == 1) {  // the CG dot products ride on the last smoothing pass
    launch(k4_post_first_dots, g, kBlock, st, V.A, V.n, (const float4*)E.b, (const float4*)E.x,
           (const float*)V.dinv, (float)V.inv_theta, (const double4_32a*)c->d_er,
           (const double4_32a*)c->d_eq, c->d_ez32, (EnsScalars*)c->d_esc, c->d_epart, c->red.counter,
           c->red.max_blocks, c->opts.flexible);
    return nullptr;
  }
  launch(k4_post_first, g, kBlock, st, V.A, V.n, (const float4*)E.b, (const float4*)E.x, (const float*)V.dinv,
         (float)V.inv_theta, deg >= 2 ? E.r : nullptr, E.dA, deg == 1 ? 1 : 0);
  din = E.dA;
  dout = E.dB;
  for (int k = 2; k <= deg; ++k) {
    launch(k4_cheb_step, g, kBlock, st, V.A, V.n, (const float4*)E.r, (const float4*)din, (const float*)V.dinv,
           (float)c1[k], (float)c2[k], E.r, dout, E.x, k == 2 ? 1 : 0);
    std::swap(din, dout);
  }
  return deg == 1 ? E.dA : E.x;
}

struct EnsSlots {
  int* iters;      // 4 per stage
  double* relres;  // 4 per stage
  int* zero;       // 4 per stage
};

static void ens_init_launch(eqs_ctx* c, cudaStream_t st, const double4_32a* R, double4_32a* x, double tol2,
                            cudaGraphConditionalHandle h, int use_handle, EnsSlots sl, bool spe = false) {
  DevLevel<float>& V = c->lev32[0];
  eqs_ctx::EnsLevel& E = c->elev[0];
  const int n = (int)c->n_free;
  if (spe) {  // SPE start: x0 = X a_c, r0 = R - W a_c
    launch(k4_spe_start<kEnsSpe>, vec_grid(c, n), kBlock, st, c->M64, n, (const double4_32a*)c->d_eX,
           (const double4_32a*)c->d_eW, (const double*)c->d_ecoef, R, x, c->d_er, (const float*)V.dinv,
           (float)V.inv_theta, E.b, E.x, ens_d0(c), (EnsScalars*)c->d_esc, c->d_epart, c->red.counter,
           c->red.max_blocks, tol2, c->opts.max_iter, h, use_handle, sl.iters, sl.relres, sl.zero);
    return;
  }
  launch(k4_pcg_init, vec_grid(c, n), kBlock, st, c->M64, n, R, (const double4_32a*)x, c->d_er,
         (const float*)V.dinv, (float)V.inv_theta, E.b, E.x, ens_d0(c), (EnsScalars*)c->d_esc, c->d_epart,
         c->red.counter, c->red.max_blocks, tol2, c->opts.max_iter, h, use_handle, sl.iters, sl.relres, sl.zero);
}

static void ens_body_launch(eqs_ctx* c, cudaStream_t st, double4_32a* x, double tol2,
                            cudaGraphConditionalHandle h, int use_handle, EnsSlots sl) {
  DevLevel<float>& V = c->lev32[0];
  eqs_ctx::EnsLevel& E = c->elev[0];
  const int n = (int)c->n_free;
  const int g = vec_grid(c, n);
  EnsScalars* sc = (EnsScalars*)c->d_esc;
  const bool fuse = c->opts.cheb_degree == 1 && c->lev32.size() > 1;
  const float4* z = ens_vcycle_level(c, 0, st, fuse);
  if (!fuse)
    launch(k4_pcg_dots, g, kBlock, st, n, (const double4_32a*)c->d_er, (const double4_32a*)c->d_eq,
           z, (const float4*)nullptr, c->d_ez32, sc, c->d_epart, c->red.counter,
           c->red.max_blocks, c->opts.flexible);
  launch(k4_pcg_pq, g, kBlock, st, c->M64, (const float*)c->d_M_hi, (const float*)c->d_M_lo, n,
         (const float4*)c->d_ez32, c->d_ep, c->d_eq, sc, c->d_epart, c->red.counter, c->red.max_blocks);
  launch(k4_pcg_update, g, kBlock, st, n, x, c->d_er, (const double4_32a*)c->d_ep,
         (const double4_32a*)c->d_eq, (const float*)V.dinv, (float)V.inv_theta, E.b, E.x, ens_d0(c), sc, c->d_epart,
         c->red.counter, c->red.max_blocks, tol2, c->opts.max_iter, h, use_handle, sl.iters, sl.relres);
}

// "init; while (any column active) body" captured into the graph of c->cap_stream.
static eqs_status ens_pcg_capture(eqs_ctx* c, const double4_32a* R, double4_32a* x, double tol2, EnsSlots sl,
                                  bool spe = false) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(c->cap_stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  ens_init_launch(c, c->cap_stream, R, x, tol2, h, 1, sl, spe);
  CK(cudaGetLastError());
  CK(cudaStreamGetCaptureInfo(c->cap_stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(c->cap_stream2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  ens_body_launch(c, c->cap_stream2, x, tol2, h, 1, sl);
  cudaError_t le = cudaGetLastError();
  cudaGraph_t body_out = nullptr;
  CK(cudaStreamEndCapture(c->cap_stream2, &body_out));
  CK(le);
  c->ens_body_kernels = count_kernel_nodes(body_out);
  CK(cudaStreamUpdateCaptureDependencies(c->cap_stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return EQS_OK;
}

// Host-driven loop (host_loop option): same kernels, the flags are read back
// after every pass.
static eqs_status ens_pcg_direct(eqs_ctx* c, const double4_32a* R, double4_32a* x, double tol2, EnsSlots sl,
                                 bool spe = false) {
  cudaStream_t st = c->stream;
  ens_init_launch(c, st, R, x, tol2, 0, 0, sl, spe);
  EnsScalars* sc = (EnsScalars*)c->d_esc;
  for (int it = 0; it < c->opts.max_iter; ++it) {
    int conv[kEnsW];
    CK(cudaMemcpyAsync(conv, sc->conv, sizeof(conv), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool any = false;
    for (int k = 0; k < kEnsW; ++k) any |= !conv[k];
    if (!any) break;
    ens_body_launch(c, st, x, tol2, 0, 0, sl);
  }
  CK(cudaGetLastError());
  return EQS_OK;
}

// SPE Gram pass of the four columns (double-float on the FP32 pipe), two
// threads per row, as many CTAs as are resident at once.
// The Gram pass as two launches: W_new = M x_new alone (k4_spe_w: one
// thread per row, no dot-product state), then the dot products from the
// stored W_new and the small solves (kGramSplit); or both in one launch.
constexpr bool kGramSplit = true;

template <typename K>
static int occupancy_of(K kern) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBlock, 0) != cudaSuccess) occ = 1;
  return std::max(1, occ);
}

static void ens_spe_gram(eqs_ctx* c, cudaStream_t st, int s, int j) {
  const int nf = (int)c->n_free;
  static const int occ_w = occupancy_of(k4_spe_w<kEnsSpe>);
  static const int occ_split = occupancy_of(k4_spe_gram_df<kEnsSpe, true>);
  static const int occ_fused = occupancy_of(k4_spe_gram_df<kEnsSpe, false>);
  auto gram = [&](auto kern, int occ) {
    const int grid = std::max(1, std::min(std::min(nblk(2 * (int64_t)nf), c->sms * occ), c->red.max_blocks));
    launch(kern, grid, kBlock, st, c->M64, (const float*)c->d_M_hi, (const float*)c->d_M_lo,
           (const float2*)c->d_M_rs, nf, (const float4*)c->d_eX2, c->d_eW, (const float4*)c->d_eR2,
           (const long long*)c->d_estepcount, s, j, c->d_eG, c->d_espart, c->red.counter, c->red.max_blocks, 1e-12,
           c->d_ecoef);
  };
  if (kGramSplit) {
    launch(k4_spe_w<kEnsSpe>, std::max(1, std::min(nblk(nf), c->sms * occ_w)), kBlock, st, c->M64,
           (const float*)c->d_M_hi, (const float*)c->d_M_lo, (const float2*)c->d_M_rs, nf, (const float4*)c->d_eX2,
           c->d_eW, (const long long*)c->d_estepcount, j);
    gram(k4_spe_gram_df<kEnsSpe, true>, occ_split);
  } else {
    gram(k4_spe_gram_df<kEnsSpe, false>, occ_fused);
  }
}

static double4_32a* eYbuf(eqs_ctx* c, int j) { return j == 0 ? c->d_eY[0] : c->d_eY[1 + (j - 1) % 3]; }
static double4_32a* eFbuf(eqs_ctx* c, int j) { return j == 0 ? c->d_eF[0] : c->d_eF[1 + (j - 1) % 2]; }

// The caller's X is read and written through the parameter block
// (c->d_params->x), so the captured graph does not depend on it.
static eqs_status ens_enqueue_step(eqs_ctx* c, int s, const double* d_cj, cudaStream_t st) {
  std::vector<double> mu, nu, mut, gt, cj;
  double beta;
  rkc_coefficients(s, mu, nu, mut, gt, cj, beta);
  const int n = (int)c->n_nodes, nf = (int)c->n_free;
  const double tol2 = c->opts.rtol * c->opts.rtol;
  const double w = 2.0 * M_PI * c->freq;
  const bool spe = c->opts.guess == EQS_GUESS_SPE;
  launch(k_stage_scalars, 1, 64, st, s + 1, d_cj, c->d_params, c->V0, w, c->phase, c->d_g, c->d_gp,
         c->d_estepcount);
  launch(k4_gather_state, nblk(n), kBlock, st, n, nf, (const StepParams*)c->d_params,
         (const int32_t*)c->d_node_of_internal,
         (const double*)c->d_dir_scale, (const double*)c->d_g, (const double*)c->d_ecolv, eYbuf(c, 0), c->d_eY2,
         (const double4_32a*)eFbuf(c, s - 1), eFbuf(c, 0));
  eqs_status stt = EQS_OK;
  for (int j = 0; j <= s && stt == EQS_OK; ++j) {
    if (j >= 1) {
      const bool first = (j == 1);
      const bool last = (j == s);
      const double c0 = first ? 1.0 : 1.0 - mu[j] - nu[j];
      launch(k4_recurrence, nblk(n), kBlock, st, n, nf, c0, first ? 0.0 : mu[j], first ? 0.0 : nu[j], mut[j],
             first ? 0.0 : gt[j], (const StepParams*)c->d_params, (const double4_32a*)eYbuf(c, 0),
             (const double4_32a*)eYbuf(c, j - 1), (const double4_32a*)eYbuf(c, j >= 2 ? j - 2 : 0),
             (const double4_32a*)eFbuf(c, j - 1), (const double4_32a*)eFbuf(c, 0), (const int*)c->d_ezero, j - 1,
             (const double*)c->d_dir_scale, (const double*)(c->d_g + j), (const double*)c->d_ecolv, eYbuf(c, j),
             last ? nullptr : c->d_eY2, last ? nullptr : eFbuf(c, j), last ? 1 : 0,
             (const int32_t*)c->d_node_of_internal, (const long long*)c->d_estepcount, s,
             spe ? c->d_eX : nullptr, c->d_eX2, kEnsSpe);
      if (last) break;
    }
    if (c->n_cells > 0)  // Kuhn cells: one 16-byte atomic per corner, 8 per six tets
      launch(k4_elem32_cell, (int)((c->n_cells + kElemBlock4 - 1) / kElemBlock4), kElemBlock4, st, c->n_cells,
             (const int32_t*)c->d_corner, (const uint8_t*)c->d_mat, (const MaterialDev*)c->d_mats,
             (const float4*)c->d_xyz_hi, (const float4*)c->d_xyz_lo, (const float4*)c->d_eY2, nf, c->d_ey32);
    else
      launch(k4_elem32, nblk(c->n_tets), kBlock, st, c->n_tets, (const int4*)c->d_conn, (const uint8_t*)c->d_mat,
             (const MaterialDev*)c->d_mats, (const float4*)c->d_xyz_hi, (const float4*)c->d_xyz_lo,
             (const float4*)c->d_eY2, nf, c->d_ey32);
    launch(k4_rhs, nblk(nf), kBlock, st, nf, c->d_ey32, (const double*)(c->d_gp + j), (const double*)c->d_ecolv,
           (const double*)c->d_mtop, c->d_eR, spe ? c->d_eR2 : nullptr);
    EnsSlots sl{c->d_eiters + kEnsW * j, c->d_erelres + kEnsW * j, c->d_ezero + kEnsW * j};
    if (spe) ens_spe_gram(c, st, s, j);
    if (c->direct)
      stt = ens_pcg_direct(c, c->d_eR, eFbuf(c, j), tol2, sl, spe);
    else
      stt = ens_pcg_capture(c, c->d_eR, eFbuf(c, j), tol2, sl, spe);
  }
  return stt;
}

static eqs_status ens_capture_step(eqs_ctx* c, int s, GraphEntry& ge) {
  std::vector<double> mu, nu, mut, gt, cj;
  double beta;
  rkc_coefficients(s, mu, nu, mut, gt, cj, beta);
  CK(upload(c, &ge.d_cj, cj.data(), cj.size()));
  cudaStream_t st = c->cap_stream;
  c->direct = false;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  eqs_status stt = ens_enqueue_step(c, s, ge.d_cj, st);
  cudaError_t le = cudaGetLastError();
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  if (stt != EQS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return stt;
  }
  CK(le);
  CK(ee);
  ge.graph = graph;
  ge.s = s;
  ge.fixed_kernels = count_kernel_nodes(graph);
  ge.per_iter_kernels = c->ens_body_kernels;
  CK(cudaGraphInstantiate(&ge.exec, graph, 0));
  return EQS_OK;
}

// ----------------------------------------------- allocation-free K(x)x
// Scratch of eqs_apply_K_static: three regions of 8 bytes per node (the
// gathered potential, its two-float copy, the accumulated result), for at most
// kStaticMaxNodes nodes.  It lives in the module's static device memory, so
// every GPU that loads the library holds these 12 MiB until the process exits.
constexpr int64_t kStaticMaxNodes = 524288;
static __device__ __align__(256) unsigned char g_static_scratch[3 * 8 * kStaticMaxNodes];

namespace {
std::mutex g_static_mu;
void* g_static_ptr[256] = {};  // device address of g_static_scratch, per device
}  // namespace

// Host code cannot use g_static_scratch's address directly (in host code the
// name is a host-side stand-in); look up the device address once per device,
// with that device current.
static eqs_status static_scratch(eqs_ctx* c, int dev, unsigned char** out) {
  if (dev < 0 || dev >= 256) return fail(c, EQS_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess)
      return fail(c, EQS_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  *out = (unsigned char*)g_static_ptr[dev];
  return EQS_OK;
}

// ================================================================ C ABI
extern "C" {

void eqs_opts_default(eqs_opts* o) {
  if (!o) return;
  o->precision = EQS_PREC_FP64;
  o->theta = 0.08;
  o->coarse_max = 500;
  o->max_levels = 10;
  o->cheb_degree = 2;
  o->cheb_alpha = 30.0;
  o->rtol = 1e-8;
  o->max_iter = 500;
  o->guess = EQS_GUESS_PREV;
  o->flexible = 1;
  o->persistent = 0;
  o->blocks_per_sm = 1;
  o->spe_n = 4;
  o->host_loop = 0;
  o->barrier_polls = 0;
  o->split_m = 1;
  o->pod_k = 12;
  o->pod_m = 6;
  o->pod_min_iters = 3;
  o->fill_lanes = 1;
  o->coarse_split = 0;
  o->defer_sums = 2;
}

static eqs_status mesh_create(const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                              int npe, const uint8_t* node_tag, eqs_ctx** out);

eqs_status eqs_mesh_create(const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                           const uint8_t* node_tag, eqs_ctx** out) {
  return mesh_create(xyz, n_nodes, tets, n_tets, 4, node_tag, out);
}

eqs_status eqs_mesh_create_p2(const double* xyz, int64_t n_nodes, const int32_t* tets10, int64_t n_tets,
                              const uint8_t* node_tag, eqs_ctx** out) {
  return mesh_create(xyz, n_nodes, tets10, n_tets, 10, node_tag, out);
}

static eqs_status mesh_create(const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                              int npe, const uint8_t* node_tag, eqs_ctx** out) {
  if (!out) return fail(nullptr, EQS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!xyz || !tets || !node_tag || n_nodes <= 0 || n_tets <= 0)
    return fail(nullptr, EQS_ERR_ARG, "null pointer or non-positive size");
  if (n_nodes > (int64_t)INT32_MAX / 2 || n_tets > (int64_t)INT32_MAX * 16)
    return fail(nullptr, EQS_ERR_ARG, "mesh too large for 32-bit node indices");
  eqs_ctx* c = new eqs_ctx();
  c->n_nodes = n_nodes;
  c->n_tets = n_tets;
  c->xyz.assign(xyz, xyz + 3 * n_nodes);
  c->npe = npe;
  c->tets.assign(tets, tets + (int64_t)npe * n_tets);
  c->tag.assign(node_tag, node_tag + n_nodes);
  eqs_opts_default(&c->opts);
  eqs_status st = validate_and_orient(c);
  if (st != EQS_OK) {
    g_create_err = c->err;
    delete c;
    return st;
  }
  build_internal_numbering(c);
  *out = c;
  return EQS_OK;
}

eqs_status eqs_set_materials(eqs_ctx* c, const uint8_t* tet_mat, int n_mat, const eqs_material* mats) {
  if (!c) return fail(nullptr, EQS_ERR_ARG, "ctx is NULL");
  if (!tet_mat || !mats || n_mat < 1 || n_mat > 255) return fail(c, EQS_ERR_ARG, "bad material arguments");
  for (int m = 0; m < n_mat; ++m) {
    const eqs_material& q = mats[m];
    if (!(q.eps_r > 0) || !(q.kappa_lo >= 0) || !(q.kappa_hi >= 0) ||
        (q.kappa_hi != q.kappa_lo && !(q.w > 0)))
      return fail(c, EQS_ERR_ARG, "material " + std::to_string(m) + " has invalid parameters");
  }
  for (int64_t e = 0; e < c->n_tets; ++e)
    if (tet_mat[e] >= n_mat) return fail(c, EQS_ERR_MESH, "tet material id out of range");
  c->tet_mat.assign(tet_mat, tet_mat + c->n_tets);
  c->mats.assign(mats, mats + n_mat);
  c->have_materials = true;
  c->setup_done = false;
  return EQS_OK;
}

eqs_status eqs_set_dirichlet(eqs_ctx* c, double V0, double freq_hz, double phase) {
  if (!c) return fail(nullptr, EQS_ERR_ARG, "ctx is NULL");
  if (!std::isfinite(V0) || !std::isfinite(freq_hz) || !std::isfinite(phase))
    return fail(c, EQS_ERR_ARG, "non-finite drive parameter");
  c->V0 = V0;
  c->freq = freq_hz;
  c->phase = phase;
  destroy_graphs(c);  // drive parameters are baked into the step graphs
  return EQS_OK;
}

eqs_status eqs_amg_setup(eqs_ctx* c, const eqs_opts* opts) {
  if (!c) return fail(nullptr, EQS_ERR_ARG, "ctx is NULL");
  if (!c->have_materials) return fail(c, EQS_ERR_STATE, "eqs_set_materials must come first");
  eqs_opts o;
  if (opts)
    o = *opts;
  else
    eqs_opts_default(&o);
  if (o.cheb_degree < 1 || o.cheb_degree > 4 || o.blocks_per_sm < 0 || o.spe_n < 1 || o.spe_n > kSpeMax || o.max_levels < 1 || o.coarse_max < 1 ||
      o.pod_k < 1 || o.pod_k > kPodMax || o.pod_m < 1 || o.pod_m > o.pod_k || o.pod_min_iters < 0 ||
      (o.coarse_split != 0 && o.coarse_split != 1) || o.defer_sums < 0 || o.defer_sums > 3 ||
      !(o.theta >= 0) || !(o.cheb_alpha > 1) || !(o.rtol > 0) || o.max_iter < 1 ||
      (o.precision != EQS_PREC_FP64 && o.precision != EQS_PREC_MIXED))
    return fail(c, EQS_ERR_ARG, "invalid eqs_opts");
  // release an earlier setup
  destroy_graphs(c);
  free_all(c);
  c->setup_done = false;
  c->ens_ready = false;
  c->elev.clear();
  c->opts = o;
  c->hier_ready = false;

  // host part: M, M_fd 1_top and the AMG hierarchy (inspectable without a GPU)
  HostCSR Mff;
  std::vector<double> mtop;
  assemble_M(c, Mff, mtop);
  build_hierarchy(Mff, o, c->hlev);
  if (c->hlev.back().A.n_rows > 4096)
    return fail(c, EQS_ERR_ARG, "coarsest AMG level has more than 4096 rows: raise max_levels");
  std::vector<double> inv;
  if (!dense_spd_inverse(c->hlev.back().A, inv))
    return fail(c, EQS_ERR_MESH, "coarsest AMG matrix is not SPD");
  c->coarse_n = (int)c->hlev.back().A.n_rows;
  c->hier_ready = true;

  // device part
  if (!c->own_stream) {
    CK(cudaGetDevice(&c->device));
    CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking));
  }
  CK(cudaSetDevice(c->device));
  CK(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device));

  const int64_t n = c->n_nodes, nf = c->n_free;
  // mesh data in internal numbering
  std::vector<int4> conn(c->n_tets);
  const int npe = c->npe;
  for (int64_t e = 0; e < c->n_tets; ++e) {
    const int32_t* t = &c->tets[(int64_t)npe * e];
    conn[e] = make_int4(c->internal_of_node[t[0]], c->internal_of_node[t[1]], c->internal_of_node[t[2]],
                        c->internal_of_node[t[3]]);
  }
  // Kuhn cells: every group of six consecutive tets is the split of one
  // hexahedron (corner c = bx + 2 by + 4 bz, tet p with corners
  // kKuhnTetHost[p]); then the element kernel works per cell
  static const int kKuhnTetHost[6][4] = {{0, 1, 3, 7}, {0, 1, 7, 5}, {0, 2, 7, 3},
                                         {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 7, 6}};
  std::vector<int32_t> corner;
  c->n_cells = 0;
  if (npe == 4 && c->n_tets % 6 == 0) {
    const int64_t nc = c->n_tets / 6;
    corner.resize((size_t)8 * nc);
    bool ok = true;
    for (int64_t q = 0; q < nc && ok; ++q) {
      const int32_t* t = &c->tets[24 * q];
      int32_t cn[8];
      cn[0] = t[0];
      cn[1] = t[1];
      cn[3] = t[2];
      cn[7] = t[3];
      cn[5] = t[4 + 3];
      cn[2] = t[8 + 1];
      cn[6] = t[12 + 2];
      cn[4] = t[16 + 1];
      for (int p = 0; p < 6 && ok; ++p)
        for (int k = 0; k < 4 && ok; ++k) ok = t[4 * p + k] == cn[kKuhnTetHost[p][k]];
      for (int k = 0; k < 8; ++k) corner[(size_t)k * nc + q] = c->internal_of_node[cn[k]];
    }
    if (ok) c->n_cells = nc;
  }
  std::vector<int32_t> conn10;
  if (npe == 10) {  // node-major: entry k of tet e at k * n_tets + e (coalesced per k)
    conn10.resize((size_t)10 * c->n_tets);
    for (int64_t e = 0; e < c->n_tets; ++e)
      for (int k = 0; k < 10; ++k) conn10[(size_t)k * c->n_tets + e] = c->internal_of_node[c->tets[10 * e + k]];
  }
  std::vector<double4> xyz(n);
  std::vector<float4> xh(n), xl(n);
  for (int64_t i = 0; i < n; ++i) {
    const double* p = &c->xyz[3 * (int64_t)c->node_of_internal[i]];
    xyz[i] = make_double4(p[0], p[1], p[2], 0.0);
    float h[3], l[3];
    for (int d = 0; d < 3; ++d) {
      h[d] = (float)p[d];
      l[d] = (float)(p[d] - (double)h[d]);
    }
    xh[i] = make_float4(h[0], h[1], h[2], 0.f);
    xl[i] = make_float4(l[0], l[1], l[2], 0.f);
  }
  std::vector<double> dir_scale(n - nf);
  for (int64_t i = nf; i < n; ++i) dir_scale[i - nf] = c->tag[c->node_of_internal[i]] == 2 ? 1.0 : 0.0;
  std::vector<MaterialDev> md(c->mats.size());
  for (size_t m = 0; m < c->mats.size(); ++m) {
    const eqs_material& q = c->mats[m];
    md[m].eps = 8.8541878128e-12 * q.eps_r;
    md[m].klo = q.kappa_lo;
    md[m].khi = q.kappa_hi;
    md[m].E0 = q.E0;
    md[m].inv_w = q.kappa_hi != q.kappa_lo ? 1.0 / q.w : 0.0;
    md[m].is_const = q.kappa_hi == q.kappa_lo;
    md[m].pad = 0;
    md[m].klo_f = (float)md[m].klo;
    md[m].dk_f = (float)(md[m].khi - md[m].klo);
    md[m].E0_f = (float)md[m].E0;
    md[m].inv_w_f = (float)md[m].inv_w;
  }
  CK(upload(c, &c->d_conn, conn.data(), conn.size()));
  c->d_conn10 = nullptr;
  if (npe == 10) CK(upload(c, &c->d_conn10, conn10.data(), conn10.size()));
  c->d_corner = nullptr;
  if (c->n_cells > 0) CK(upload(c, &c->d_corner, corner.data(), corner.size()));
  CK(upload(c, &c->d_mat, c->tet_mat.data(), c->tet_mat.size()));
  CK(upload(c, &c->d_mats, md.data(), md.size()));
  CK(upload(c, &c->d_xyz, xyz.data(), xyz.size()));
  CK(upload(c, &c->d_xyz_hi, xh.data(), xh.size()));
  CK(upload(c, &c->d_xyz_lo, xl.data(), xl.size()));
  CK(upload(c, &c->d_node_of_internal, c->node_of_internal.data(), c->node_of_internal.size()));
  CK(upload(c, &c->d_dir_scale, dir_scale.data(), dir_scale.size()));
  CK(upload(c, &c->d_mtop, mtop.data(), mtop.size()));
  CK(upload_sell(c, Mff, c->M64, false));  // CG kernels use one thread per row (DIA or SELL)
  c->d_M_hi = c->d_M_lo = nullptr;
  c->d_M_rs = nullptr;
  c->d_z32 = nullptr;
  if (mixed(c) && c->opts.split_m) {  // M_ff = hi + lo in FP32 parts, same layout
    std::vector<double> mv((size_t)c->M64.stored);
    CK(cudaMemcpy(mv.data(), c->M64.val, mv.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<float> mh(mv.size()), ml(mv.size());
    for (size_t k = 0; k < mv.size(); ++k) {
      mh[k] = (float)mv[k];
      ml[k] = (float)(mv[k] - (double)mh[k]);
    }
    CK(upload(c, &c->d_M_hi, mh.data(), mh.size()));
    CK(upload(c, &c->d_M_lo, ml.data(), ml.size()));
    CK(dalloc(c, &c->d_z32, std::max<int64_t>(nf, 1)));
    CK(dalloc(c, &c->d_M_rs, std::max<int64_t>(nf, 1)));
    if (nf > 0) {
      k_rowsum_split<<<nblk(nf), kBlock>>>(c->M64, c->d_M_hi, c->d_M_lo, (int)nf, c->d_M_rs);
      CK(cudaGetLastError());
    }
  }
  CK(upload(c, &c->d_coarse_inv, inv.data(), inv.size()));
  c->d_cinv_hi = c->d_cinv_lo = c->d_cinv32 = nullptr;
  c->cinv_ld = 0;
  if (mixed(c)) {  // the FP32 (or FP32-pair) coarse solve of the mixed V-cycle
    const int nc = c->coarse_n;
    const int ld = (nc + 3) & ~3;
    const size_t smem = (size_t)ld * 4 * sizeof(float);
    if (smem > 227 * 1024) return fail(c, EQS_ERR_ARG, "coarsest level too large for the shared-memory coarse solve");
    const int smem_attr = (int)std::max<size_t>(smem, 48 * 1024);
    if (c->opts.coarse_split) {
      std::vector<float> ih(inv.size()), il(inv.size());
      for (size_t k = 0; k < inv.size(); ++k) {
        ih[k] = (float)inv[k];
        il[k] = (float)(inv[k] - (double)ih[k]);
      }
      CK(upload(c, &c->d_cinv_hi, ih.data(), ih.size()));
      CK(upload(c, &c->d_cinv_lo, il.data(), il.size()));
      CK(cudaFuncSetAttribute(k_coarse_solve_df<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_attr));
      CK(cudaFuncSetAttribute(k_coarse_solve_df<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_attr));
    } else {
      std::vector<float> i32((size_t)nc * ld, 0.f);
      for (int r = 0; r < nc; ++r)
        for (int k = 0; k < nc; ++k) i32[(size_t)r * ld + k] = (float)inv[(size_t)r * nc + k];
      CK(upload(c, &c->d_cinv32, i32.data(), i32.size()));
      c->cinv_ld = ld;
      CK(cudaFuncSetAttribute(k_coarse_solve32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_attr));
      CK(cudaFuncSetAttribute(k_coarse_solve32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_attr));
    }
  }
  c->lev64.clear();
  c->lev32.clear();
  if (mixed(c))
    CK(upload_levels(c, c->lev32));
  else
    CK(upload_levels(c, c->lev64));
  for (int k = 0; k < 4; ++k) CK(dalloc(c, &c->d_Y[k], n));
  for (int k = 0; k < 3; ++k) CK(dalloc(c, &c->d_F[k], nf));
  CK(dalloc(c, &c->d_Y32, n));
  CK(dalloc(c, &c->d_y32, n));
  for (double** v : {&c->d_R, &c->d_r, &c->d_rprev, &c->d_p, &c->d_p2, &c->d_q, &c->d_zd, &c->d_sol})
    CK(dalloc(c, v, nf));
  CK(dalloc(c, &c->d_tmpn, n));
  CK(dalloc(c, &c->d_tmpn2, n));
  CK(dalloc(c, &c->d_sc, 1));
  CK(dalloc(c, &c->d_params, 1));
  CK(dalloc(c, &c->d_iters, EQS_MAX_STAGES + 1));
  CK(dalloc(c, &c->d_relres, EQS_MAX_STAGES + 1));
  CK(dalloc(c, &c->d_zero, EQS_MAX_STAGES + 1));
  CK(dalloc(c, &c->d_g, EQS_MAX_STAGES + 1));
  CK(dalloc(c, &c->d_gp, EQS_MAX_STAGES + 1));
  // room for the partial sums of every reducing grid: row kernels on lane
  // groups can launch more blocks than nblk(nf), never more than 4 per SM
  c->red.max_blocks = std::max(nblk(std::max<int64_t>(nf, 1)), 4 * c->sms);
  CK(dalloc(c, &c->red.partials, 4 * (size_t)c->red.max_blocks));
  CK(dalloc(c, &c->d_dpart, 3 * (size_t)c->red.max_blocks));  // deferred CG sums: r.z, r_prev.z; p.q
  CK(dalloc(c, &c->red.counter, 9));  // main + 8 group tickets
  {
    const eqs_status ps = mixed(c) ? build_plan(c, c->lev32) : build_plan(c, c->lev64);
    if (ps != EQS_OK) return ps;
  }
  // learned start vector: free-node graph from the pattern of M_ff, network
  // state (zero parameters = previous-solution guess), history ring
  {
    std::vector<int32_t> aptr(nf + 1, 0), acol;
    std::vector<float> ideg(nf, 0.f);
    acol.reserve(Mff.nnz());
    for (int64_t i = 0; i < nf; ++i) {
      for (int64_t k = Mff.ptr[i]; k < Mff.ptr[i + 1]; ++k)
        if (Mff.col[k] != i) acol.push_back(Mff.col[k]);
      aptr[i + 1] = (int32_t)acol.size();
      const int deg = aptr[i + 1] - aptr[i];
      ideg[i] = deg > 0 ? 1.0f / (float)deg : 0.0f;
    }
    CK(upload(c, &c->d_adj_ptr, aptr.data(), aptr.size()));
    CK(upload(c, &c->d_adj_col, acol.data(), std::max<size_t>(acol.size(), 1)));
    CK(upload(c, &c->d_inv_deg, ideg.data(), ideg.size()));
    CK(dalloc(c, &c->d_theta, kNP));
    __nv_bfloat16* wb = nullptr;
    CK(dalloc(c, &wb, kNP));
    c->d_theta_bf16 = wb;
    CK(dalloc(c, &c->d_adam_m, kNP));
    CK(dalloc(c, &c->d_adam_v, kNP));
    CK(dalloc(c, &c->d_grad, kNP));
    CK(dalloc(c, &c->d_loss, 1));
    CK(dalloc(c, &c->d_ring, 4 * (size_t)nf));
    CK(dalloc(c, &c->d_stepcount, 2));
    CK(dalloc(c, &c->d_sh, 1));
    CK(dalloc(c, &c->d_mlp_used, EQS_MAX_STAGES + 1));
    CK(dalloc(c, &c->d_x0, nf));
    CK(dalloc(c, &c->d_alpha, 1));
    CK(dalloc(c, &c->d_rtmp, nf));
    CK(dalloc(c, &c->d_xsave, n));
    CK(dalloc(c, &c->d_Fnew, nf));
    CK(dalloc(c, &c->d_err, 1));
    CK(dalloc(c, &c->d_evalcount, 2));
    CK(dalloc(c, &c->d_cj0, 1));
    CK(dalloc(c, &c->d_spe_X, (size_t)kSpeMax * nf));
    CK(dalloc(c, &c->d_spe_W, (size_t)kSpeMax * nf));
    CK(dalloc(c, &c->d_spe_y, kSpeMax + 1));  // coefficients + slots in use
    CK(dalloc(c, &c->d_spe_G, (size_t)kSpeMax * kSpeMax));
    CK(dalloc(c, &c->d_spe_partials, (size_t)kSpeSums * c->red.max_blocks));
    CK(dalloc(c, &c->d_pod_X, (size_t)c->opts.pod_k * nf));
    CK(dalloc(c, &c->d_pod_W, (size_t)c->opts.pod_k * nf));
    CK(dalloc(c, &c->d_pod_GE, (size_t)kPodMax * kPodMax));
    CK(dalloc(c, &c->d_pod_GM, (size_t)kPodMax * kPodMax));
    CK(dalloc(c, &c->d_pod_a, kPodMax));
    CK(dalloc(c, &c->d_pod_partials, 2 * (size_t)kPodMax * c->red.max_blocks));
    PodState* ps = nullptr;
    CK(dalloc(c, &ps, 1));
    c->d_pod_state = ps;
    c->adam_t = 0;
    c->d_store = nullptr;
    c->d_store_rms = nullptr;
    c->store_cap = 0;
    c->recorded = 0;
    c->recording = false;
  }
  CK(cudaDeviceSynchronize());
  c->setup_done = true;
  return EQS_OK;
}

#define REQUIRE_SETUP(c)                                                   \
  do {                                                                     \
    if (!(c)) return fail(nullptr, EQS_ERR_ARG, "ctx is NULL");            \
    if (!(c)->setup_done) return fail((c), EQS_ERR_STATE, "call eqs_amg_setup first"); \
  } while (0)

eqs_status eqs_apply_K(eqs_ctx* c, const double* x, double* y) {
  REQUIRE_SETUP(c);
  if (!x || !y) return fail(c, EQS_ERR_ARG, "null vector");
  const int n = (int)c->n_nodes;
  cudaStream_t st = c->stream;
  const bool mx = mixed(c);
  launch(k_gather_perm, nblk(n), kBlock, st, n, x, c->d_node_of_internal, c->d_tmpn, mx ? c->d_Y32 : nullptr);
  if (mx) {
    CK(cudaMemsetAsync(c->d_y32, 0, n * sizeof(float), st));
    elem_launch(c, st, nullptr, n, nullptr, c->d_y32);
    launch(k_scatter_perm, nblk(n), kBlock, st, n, nullptr, c->d_y32, c->d_node_of_internal, y);
    CK(cudaMemsetAsync(c->d_y32, 0, n * sizeof(float), st));
  } else {
    CK(cudaMemsetAsync(c->d_tmpn2, 0, n * sizeof(double), st));
    elem_launch(c, st, c->d_tmpn, n, c->d_tmpn2, nullptr);
    launch(k_scatter_perm, nblk(n), kBlock, st, n, c->d_tmpn2, nullptr, c->d_node_of_internal, y);
  }
  CK(cudaGetLastError());
  return EQS_OK;
}

eqs_status eqs_apply_K_static(eqs_ctx* c, const double* x, double* y) {
  if (!c) return fail(nullptr, EQS_ERR_ARG, "ctx is NULL");
  if (!x || !y) return fail(c, EQS_ERR_ARG, "null vector");
  if (c->n_nodes > kStaticMaxNodes)
    return fail(c, EQS_ERR_ARG, "eqs_apply_K_static: mesh has " + std::to_string(c->n_nodes) +
                                    " nodes, the static scratch holds at most " +
                                    std::to_string(kStaticMaxNodes) + "; use eqs_apply_K");
  if (!c->setup_done) return fail(c, EQS_ERR_STATE, "call eqs_amg_setup first");
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != c->device) return fail(c, EQS_ERR_ARG, "make the context's device current");
  unsigned char* base = nullptr;
  const eqs_status ss = static_scratch(c, dev, &base);
  if (ss != EQS_OK) return ss;
  const int n = (int)c->n_nodes;
  double* xg = (double*)base;                            // region 0: gathered potential
  float2* x2 = (float2*)(base + 8 * kStaticMaxNodes);    // region 1: two-float copy
  unsigned char* yacc = base + 16 * kStaticMaxNodes;     // region 2: accumulated K(x)x
  cudaStream_t st = c->stream;
  const bool mx = mixed(c);
  k_gather_perm<<<nblk(n), kBlock, 0, st>>>(n, x, c->d_node_of_internal, xg, mx ? x2 : nullptr);
  // the accumulator keeps the previous call's contents: clear it
  CK(cudaMemsetAsync(yacc, 0, (size_t)n * (mx ? sizeof(float) : sizeof(double)), st));
  // the element kernel eqs_apply_K takes (cell, tet or P2), on the static regions
  if (mx) {
    elem_launch(c, st, nullptr, n, nullptr, (float*)yacc, x2);
    k_scatter_perm<<<nblk(n), kBlock, 0, st>>>(n, nullptr, (const float*)yacc, c->d_node_of_internal, y);
  } else {
    elem_launch(c, st, xg, n, (double*)yacc, nullptr);
    k_scatter_perm<<<nblk(n), kBlock, 0, st>>>(n, (const double*)yacc, nullptr, c->d_node_of_internal, y);
  }
  CK(cudaGetLastError());
  return EQS_OK;
}

eqs_status eqs_spmv_M(eqs_ctx* c, const double* x, double* y) {
  REQUIRE_SETUP(c);
  if (!x || !y) return fail(c, EQS_ERR_ARG, "null vector");
  const int nf = (int)c->n_free;
  k_spmv64<<<nblk(nf), kBlock, 0, c->stream>>>(c->M64, nf, x, y);
  CK(cudaGetLastError());
  return EQS_OK;
}

eqs_status eqs_spmv_M32(eqs_ctx* c, const float* x, double* y) {
  REQUIRE_SETUP(c);
  if (!x || !y) return fail(c, EQS_ERR_ARG, "null vector");
  if (!c->d_M_hi) return fail(c, EQS_ERR_STATE, "set up in EQS_PREC_MIXED with split_m 1 first");
  const int nf = (int)c->n_free;
  k_spmv_split<<<nblk(nf), kBlock, 0, c->stream>>>(c->M64, c->d_M_hi, c->d_M_lo, nf, x, y);
  CK(cudaGetLastError());
  return EQS_OK;
}

eqs_status eqs_vcycle(eqs_ctx* c, const double* r, double* z) {
  REQUIRE_SETUP(c);
  if (!r || !z) return fail(c, EQS_ERR_ARG, "null vector");
  return mixed(c) ? vcycle_impl(c, c->lev32, r, z) : vcycle_impl(c, c->lev64, r, z);
}

eqs_status eqs_solve_M(eqs_ctx* c, const double* rhs, double* z, int nrhs, double rtol, int* iters_out) {
  REQUIRE_SETUP(c);
  if (!rhs || !z || nrhs < 1) return fail(c, EQS_ERR_ARG, "bad solve arguments");
  const double tol = rtol > 0 ? rtol : c->opts.rtol;
  auto it = c->solve_graphs.find(tol);
  if (it == c->solve_graphs.end()) {
    GraphEntry ge;
    eqs_status st = mixed(c) ? capture_solve(c, c->lev32, tol, ge) : capture_solve(c, c->lev64, tol, ge);
    if (st != EQS_OK) return st;
    it = c->solve_graphs.emplace(tol, ge).first;
  }
  const int64_t nf = c->n_free;
  eqs_status res = EQS_OK;
  for (int k = 0; k < nrhs; ++k) {
    CK(cudaMemcpyAsync(c->d_R, rhs + k * nf, nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_sol, z + k * nf, nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaGraphLaunch(it->second.exec, c->stream));
    int itn = 0, zero = 0;
    double rr = 0;
    CK(cudaMemcpyAsync(&itn, c->d_iters, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&rr, c->d_relres, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&zero, c->d_zero, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (zero)
      CK(cudaMemsetAsync(z + k * nf, 0, nf * sizeof(double), c->stream));
    else
      CK(cudaMemcpyAsync(z + k * nf, c->d_sol, nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (iters_out) iters_out[k] = itn;
    if (c->d_bar) {
      GridBarrier b;
      CK(cudaMemcpy(&b, c->d_bar, sizeof(b), cudaMemcpyDeviceToHost));
      if (b.err) return fail(c, EQS_ERR_TIMEOUT, "a grid barrier of the persistent solve timed out");
    }
    if (!std::isfinite(rr)) res = fail(c, EQS_ERR_NAN, "non-finite residual in solve");
    else if (!zero && rr > tol) res = fail(c, EQS_ERR_NOCONV, "CG reached max_iter");
  }
  CK(cudaStreamSynchronize(c->stream));
  return res;
}

eqs_status eqs_rkc_step(eqs_ctx* c, double* x, double t, double dt, int s, eqs_step_stats* stats) {
  REQUIRE_SETUP(c);
  if (!x) return fail(c, EQS_ERR_ARG, "x is NULL");
  if (s < 2 || s > EQS_MAX_STAGES) return fail(c, EQS_ERR_ARG, "s out of range [2, 64]");
  if (!std::isfinite(t) || !(dt > 0) || !std::isfinite(dt)) return fail(c, EQS_ERR_ARG, "bad t or dt");
  if (c->recording && !recording_e(c)) c->store_e_valid = false;  // no SPE start to measure from
  const StepParams prm{t, dt, x};
  if (c->opts.host_loop) {  // same kernels, CG loops driven from the host
    const int dkey = -s;
    auto dit = c->step_graphs.find(dkey);
    if (dit == c->step_graphs.end()) {
      GraphEntry ge;
      std::vector<double> mu, nu, mut, gt, cj;
      double beta;
      rkc_coefficients(s, mu, nu, mut, gt, cj, beta);
      CK(upload(c, &ge.d_cj, cj.data(), cj.size()));
      ge.s = s;
      dit = c->step_graphs.emplace(dkey, ge).first;
    }
    CK(cudaMemcpyAsync(c->d_params, &prm, sizeof(prm), cudaMemcpyHostToDevice, c->stream));
    c->direct = true;
    g_launches = 0;
    eqs_status st = mixed(c) ? enqueue_step(c, c->lev32, s, dit->second.d_cj, c->stream)
                             : enqueue_step(c, c->lev64, s, dit->second.d_cj, c->stream);
    c->direct = false;
    if (st != EQS_OK) return st;
    dit->second.fixed_kernels = g_launches;
    dit->second.per_iter_kernels = 0;
    c->last_step = &dit->second;
    if (c->recording) c->recorded = std::min<int64_t>(c->recorded + s, c->store_cap);
    return stats ? eqs_get_step_stats(c, stats) : EQS_OK;
  }
  auto it = c->step_graphs.find(s);
  if (it == c->step_graphs.end()) {
    GraphEntry ge;
    eqs_status st = mixed(c) ? capture_step(c, c->lev32, s, ge) : capture_step(c, c->lev64, s, ge);
    if (st != EQS_OK) return st;
    it = c->step_graphs.emplace(s, ge).first;
  }
  CK(cudaMemcpyAsync(c->d_params, &prm, sizeof(prm), cudaMemcpyHostToDevice, c->stream));
  CK(cudaGraphLaunch(it->second.exec, c->stream));
  c->last_step = &it->second;
  if (c->recording) c->recorded = std::min<int64_t>(c->recorded + s, c->store_cap);
  if (!stats) return EQS_OK;
  return eqs_get_step_stats(c, stats);
}

eqs_status eqs_get_step_stats(eqs_ctx* c, eqs_step_stats* stats) {
  REQUIRE_SETUP(c);
  if (!stats) return fail(c, EQS_ERR_ARG, "stats is NULL");
  if (!c->last_step) return fail(c, EQS_ERR_STATE, "no step has run");
  const int s = c->last_step->s;
  int iters[EQS_MAX_STAGES];
  double rr[EQS_MAX_STAGES];
  CK(cudaMemcpyAsync(iters, c->d_iters, s * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(rr, c->d_relres, s * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::memset(stats, 0, sizeof(*stats));
  stats->s = s;
  eqs_status res = EQS_OK;
  for (int j = 0; j < s; ++j) {
    stats->iters[j] = iters[j];
    stats->total_iters += iters[j];
    stats->max_iters = std::max(stats->max_iters, iters[j]);
    stats->max_relres = std::max(stats->max_relres, rr[j]);
    if (!std::isfinite(rr[j])) res = EQS_ERR_NAN;
    else if (rr[j] > c->opts.rtol && res == EQS_OK) res = EQS_ERR_NOCONV;
  }
  stats->launches = c->last_step->fixed_kernels + c->last_step->per_iter_kernels * stats->total_iters;
  if (c->opts.guess == EQS_GUESS_MLP || c->opts.guess == EQS_GUESS_SPE_MLP) {
    int kept[EQS_MAX_STAGES];
    CK(cudaMemcpy(kept, c->d_mlp_used, s * sizeof(int), cudaMemcpyDeviceToHost));
    for (int j = 0; j < s; ++j) stats->guess_kept += kept[j];
  }
  if (c->d_bar) {
    GridBarrier b;
    CK(cudaMemcpy(&b, c->d_bar, sizeof(b), cudaMemcpyDeviceToHost));
    if (b.err) res = EQS_ERR_TIMEOUT;
  }
  stats->status = res;
  if (res == EQS_ERR_TIMEOUT) return fail(c, res, "a grid barrier of the persistent solve timed out");
  if (res == EQS_ERR_NOCONV) return fail(c, res, "a stage solve reached max_iter");
  if (res == EQS_ERR_NAN) return fail(c, res, "non-finite residual in a stage solve");
  return EQS_OK;
}

eqs_status eqs_rkc_adaptive_step(eqs_ctx* c, double* x, double t, double h_try, double atol, double rtol,
                                 int s_max, eqs_adapt_stats* out) {
  REQUIRE_SETUP(c);
  if (!x || !out) return fail(c, EQS_ERR_ARG, "x or out is NULL");
  if (!std::isfinite(t) || !(h_try > 0) || !std::isfinite(h_try) || !(atol >= 0) || !(rtol >= 0) ||
      !(atol + rtol > 0) || s_max < 2 || s_max > EQS_MAX_STAGES)
    return fail(c, EQS_ERR_ARG, "bad adaptive step arguments");
  if (c->opts.host_loop) return fail(c, EQS_ERR_STATE, "adaptive stepping runs the step graphs (host_loop 0)");
  const double rho = rho_bound(c->mats);
  std::vector<double> beta(EQS_MAX_STAGES + 1, 0.0);
  for (int s = 2; s <= s_max; ++s) {
    std::vector<double> mu, nu, mut, gt, cj;
    rkc_coefficients(s, mu, nu, mut, gt, cj, beta[s]);
  }
  const double zero = 0.0;
  CK(cudaMemcpyAsync(c->d_cj0, &zero, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_xsave, x, c->n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  std::memset(out, 0, sizeof(*out));
  double h = h_try;
  const int nf = (int)c->n_free;
  for (int tries = 1; tries <= 50; ++tries) {
    int s = 2;  // smallest s with beta_s >= h rho; cut h when s_max does not suffice
    while (s < s_max && beta[s] < h * rho) ++s;
    if (beta[s] < h * rho) h = beta[s] / rho;
    if (tries > 1)
      CK(cudaMemcpyAsync(x, c->d_xsave, c->n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    eqs_step_stats st;
    const eqs_status ss = eqs_rkc_step(c, x, t, h, s, &st);
    if (ss != EQS_OK) return ss;
    out->total_iters += st.total_iters;
    // F(t + h, x_new), started from F(t, x_old) (the step's first stage)
    CK(cudaMemcpyAsync(c->d_Fnew, c->d_F[0], nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (!c->eval_graph.exec) {
      const eqs_status es = mixed(c) ? capture_eval_F(c, c->lev32, c->d_Fnew, c->eval_graph)
                                     : capture_eval_F(c, c->lev64, c->d_Fnew, c->eval_graph);
      if (es != EQS_OK) return es;
    }
    const StepParams prm{t + h, h, x};
    CK(cudaMemcpyAsync(c->d_params, &prm, sizeof(prm), cudaMemcpyHostToDevice, c->stream));
    CK(cudaGraphLaunch(c->eval_graph.exec, c->stream));
    k_rkc_errnorm<<<vec_grid(c, nf), kBlock, 0, c->stream>>>(
        nf, c->d_xsave, x, c->d_node_of_internal, c->d_F[0], c->d_Fnew, h, atol, rtol, c->red.partials,
        c->red.counter, c->red.max_blocks, c->d_err);
    double err = 0.0;
    int eit = 0;
    double err_rr = 0.0;
    CK(cudaMemcpyAsync(&err, c->d_err, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&eit, c->d_iters + EQS_MAX_STAGES, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&err_rr, c->d_relres + EQS_MAX_STAGES, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out->total_iters += eit;
    if (!std::isfinite(err) || !std::isfinite(err_rr)) return fail(c, EQS_ERR_NAN, "non-finite error estimate");
    const double fac = err == 0.0 ? 10.0 : std::min(10.0, std::max(0.1, 0.8 * std::pow(err, -1.0 / 3.0)));
    if (err <= 1.0) {
      out->h_used = h;
      out->h_next = h * fac;
      out->err = err;
      out->s = s;
      out->tries = tries;
      return EQS_OK;
    }
    h *= fac;
  }
  CK(cudaMemcpyAsync(x, c->d_xsave, c->n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return fail(c, EQS_ERR_NOCONV, "adaptive step: 50 rejected tries");
}

// ------------------------------------------------------------- ensemble
eqs_status eqs_ens_rkc_step(eqs_ctx* c, double* x, const double* v0_scale, double t, double dt, int s,
                            eqs_ens_stats* stats) {
  REQUIRE_SETUP(c);
  if (!x || !v0_scale) return fail(c, EQS_ERR_ARG, "x or v0_scale is NULL");
  if (s < 2 || s > EQS_MAX_STAGES) return fail(c, EQS_ERR_ARG, "s out of range [2, 64]");
  if (!std::isfinite(t) || !(dt > 0) || !std::isfinite(dt)) return fail(c, EQS_ERR_ARG, "bad t or dt");
  for (int k = 0; k < EQS_ENS_W; ++k)
    if (!std::isfinite(v0_scale[k])) return fail(c, EQS_ERR_ARG, "non-finite drive scale");
  if (c->opts.guess != EQS_GUESS_PREV && c->opts.guess != EQS_GUESS_SPE)
    return fail(c, EQS_ERR_STATE, "the ensemble starts from EQS_GUESS_PREV or EQS_GUESS_SPE");
  const eqs_status as = ens_alloc(c);
  if (as != EQS_OK) return as;
  StepParams prm{t, dt, x};
  CK(cudaMemcpyAsync(c->d_params, &prm, sizeof(prm), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_ecolv, v0_scale, EQS_ENS_W * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (c->opts.host_loop) {
    const int dkey = -s;
    auto dit = c->ens_graphs.find(dkey);
    if (dit == c->ens_graphs.end()) {
      GraphEntry ge;
      std::vector<double> mu, nu, mut, gt, cj;
      double beta;
      rkc_coefficients(s, mu, nu, mut, gt, cj, beta);
      CK(upload(c, &ge.d_cj, cj.data(), cj.size()));
      ge.s = s;
      dit = c->ens_graphs.emplace(dkey, ge).first;
    }
    c->direct = true;
    g_launches = 0;
    const eqs_status st = ens_enqueue_step(c, s, dit->second.d_cj, c->stream);
    c->direct = false;
    if (st != EQS_OK) return st;
    dit->second.fixed_kernels = g_launches;
    dit->second.per_iter_kernels = 0;
    c->ens_last = &dit->second;
  } else {
    const int key = s;
    auto it = c->ens_graphs.find(key);
    if (it == c->ens_graphs.end()) {
      GraphEntry ge;
      const eqs_status st = ens_capture_step(c, s, ge);
      if (st != EQS_OK) return st;
      it = c->ens_graphs.emplace(key, ge).first;
    }
    CK(cudaGraphLaunch(it->second.exec, c->stream));
    c->ens_last = &it->second;
  }
  return stats ? eqs_ens_get_step_stats(c, stats) : EQS_OK;
}

eqs_status eqs_ens_apply_K(eqs_ctx* c, const double* x, double* y) {
  REQUIRE_SETUP(c);
  if (!x || !y) return fail(c, EQS_ERR_ARG, "null vector");
  if (!mixed(c) || c->npe != 4)
    return fail(c, EQS_ERR_STATE, "the four-column element kernel needs EQS_PREC_MIXED on linear (4-node) tets");
  const int n = (int)c->n_nodes;
  cudaStream_t st = c->stream;
  if (!c->d_ekx2) CK(dalloc(c, &c->d_ekx2, 2 * (size_t)n));
  if (!c->d_ktime) CK(dalloc(c, &c->d_ktime, (size_t)n));
  const int32_t* perm = (const int32_t*)c->d_node_of_internal;
  launch(k4_gather_pair_perm, nblk(n), kBlock, st, n, x, perm, c->d_ekx2);
  CK(cudaMemsetAsync(c->d_ktime, 0, (size_t)n * sizeof(float4), st));
  if (c->n_cells > 0)
    launch(k4_elem32_cell, (int)((c->n_cells + kElemBlock4 - 1) / kElemBlock4), kElemBlock4, st, c->n_cells,
           (const int32_t*)c->d_corner, (const uint8_t*)c->d_mat, (const MaterialDev*)c->d_mats,
           (const float4*)c->d_xyz_hi, (const float4*)c->d_xyz_lo, (const float4*)c->d_ekx2, n, c->d_ktime);
  else
    launch(k4_elem32, nblk(c->n_tets), kBlock, st, c->n_tets, (const int4*)c->d_conn, (const uint8_t*)c->d_mat,
           (const MaterialDev*)c->d_mats, (const float4*)c->d_xyz_hi, (const float4*)c->d_xyz_lo,
           (const float4*)c->d_ekx2, n, c->d_ktime);
  launch(k4_scatter_perm, nblk(n), kBlock, st, n, (const float4*)c->d_ktime, perm, y);
  CK(cudaGetLastError());
  return EQS_OK;
}

eqs_status eqs_launch_kernel(eqs_ctx* c, int kernel) {
  REQUIRE_SETUP(c);
  if (!((kernel >= EQS_KERNEL_SPE_GRAM && kernel <= EQS_KERNEL_PCG_PQ) ||
        (kernel >= EQS_KERNEL_ENS_SPE_GRAM && kernel <= EQS_KERNEL_ENS_PCG_PQ)))
    return fail(c, EQS_ERR_ARG, "unknown kernel id");
  const bool ens = kernel >= EQS_KERNEL_ENS_SPE_GRAM;
  const GraphEntry* last = ens ? c->ens_last : c->last_step;
  if (!last) return fail(c, EQS_ERR_STATE, ens ? "run an ensemble step first" : "run a step first");
  const int s = last->s, j = s - 1;  // the last solve of that step
  const int nf = (int)c->n_free;
  cudaStream_t st = c->stream;
  if ((kernel == EQS_KERNEL_ELEM || kernel == EQS_KERNEL_ENS_ELEM) && !c->d_ktime)
    CK(dalloc(c, &c->d_ktime, (size_t)c->n_nodes));
  const int g = vec_grid(c, nf);
  switch (kernel) {
    case EQS_KERNEL_SPE_GRAM:
      if (c->opts.guess != EQS_GUESS_SPE) return fail(c, EQS_ERR_STATE, "SPE start vectors are not in use");
      spe_gram(c, st, s, j, (c->opts.defer_sums & 2) != 0, false);  // the Gram pass alone
      break;
    case EQS_KERNEL_ELEM:
      if (mixed(c))
        elem_launch(c, st, nullptr, nf, nullptr, (float*)c->d_ktime);
      else
        elem_launch(c, st, Ybuf(c, 0), nf, (double*)c->d_ktime, nullptr);
      break;
    case EQS_KERNEL_PCG_PQ:
      if (c->d_z32)
        launch(k_pcg_pq_split<false>, g, kBlock, st, c->M64, (const float*)c->d_M_hi, (const float*)c->d_M_lo,
               nf, (const float*)c->d_z32, c->d_p, c->d_q, c->d_sc, c->red.partials, c->red.counter,
               c->red.max_blocks, (double*)nullptr, 0, c->opts.flexible);
      else
        launch(k_pcg_pq, g, kBlock, st, c->M64, nf, c->d_zd, c->d_p, c->d_q, c->d_sc, c->red.partials,
               c->red.counter, c->red.max_blocks);
      break;
    case EQS_KERNEL_ENS_SPE_GRAM:
      if (c->opts.guess != EQS_GUESS_SPE) return fail(c, EQS_ERR_STATE, "SPE start vectors are not in use");
      ens_spe_gram(c, st, s, j);
      break;
    case EQS_KERNEL_ENS_ELEM:
      if (c->n_cells > 0)
        launch(k4_elem32_cell, (int)((c->n_cells + kElemBlock4 - 1) / kElemBlock4), kElemBlock4, st, c->n_cells,
               (const int32_t*)c->d_corner, (const uint8_t*)c->d_mat, (const MaterialDev*)c->d_mats,
               (const float4*)c->d_xyz_hi, (const float4*)c->d_xyz_lo, (const float4*)c->d_eY2, nf, c->d_ktime);
      else
        launch(k4_elem32, nblk(c->n_tets), kBlock, st, c->n_tets, (const int4*)c->d_conn, (const uint8_t*)c->d_mat,
               (const MaterialDev*)c->d_mats, (const float4*)c->d_xyz_hi, (const float4*)c->d_xyz_lo,
               (const float4*)c->d_eY2, nf, c->d_ktime);
      break;
    case EQS_KERNEL_ENS_PCG_PQ:  // as in a pass with all four columns active
      CK(cudaMemsetAsync(((EnsScalars*)c->d_esc)->conv, 0, sizeof(int) * kEnsW, st));
      launch(k4_pcg_pq, g, kBlock, st, c->M64, (const float*)c->d_M_hi, (const float*)c->d_M_lo, nf,
             (const float4*)c->d_ez32, c->d_ep, c->d_eq, (EnsScalars*)c->d_esc, c->d_epart, c->red.counter,
             c->red.max_blocks);
      break;
    default:
      return fail(c, EQS_ERR_ARG, "unknown kernel id");
  }
  CK(cudaGetLastError());
  return EQS_OK;
}

eqs_status eqs_ens_get_step_stats(eqs_ctx* c, eqs_ens_stats* stats) {
  REQUIRE_SETUP(c);
  if (!stats) return fail(c, EQS_ERR_ARG, "stats is NULL");
  if (!c->ens_last) return fail(c, EQS_ERR_STATE, "no ensemble step has run");
  const int s = c->ens_last->s;
  std::vector<int> iters((size_t)s * kEnsW);
  std::vector<double> rr((size_t)s * kEnsW);
  CK(cudaMemcpyAsync(iters.data(), c->d_eiters, iters.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(rr.data(), c->d_erelres, rr.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::memset(stats, 0, sizeof(*stats));
  stats->s = s;
  eqs_status res = EQS_OK;
  for (int j = 0; j < s; ++j) {
    int pass = 0;
    for (int k = 0; k < kEnsW; ++k) {
      const int it = iters[(size_t)j * kEnsW + k];
      const double r = rr[(size_t)j * kEnsW + k];
      stats->total_iters[k] += it;
      pass = std::max(pass, it);
      stats->max_relres = std::max(stats->max_relres, r);
      if (!std::isfinite(r)) res = EQS_ERR_NAN;
      else if (r > c->opts.rtol && res == EQS_OK) res = EQS_ERR_NOCONV;
    }
    stats->passes += pass;
    stats->max_iters = std::max(stats->max_iters, pass);
  }
  stats->launches = c->ens_last->fixed_kernels + c->ens_last->per_iter_kernels * stats->passes;
  stats->status = res;
  if (res == EQS_ERR_NOCONV) return fail(c, res, "an ensemble stage solve reached max_iter");
  if (res == EQS_ERR_NAN) return fail(c, res, "non-finite residual in an ensemble stage solve");
  return EQS_OK;
}

eqs_status eqs_ens_solve_M(eqs_ctx* c, const double* rhs, double* z, int* iters_out) {
  REQUIRE_SETUP(c);
  if (!rhs || !z) return fail(c, EQS_ERR_ARG, "null vector");
  const eqs_status as = ens_alloc(c);
  if (as != EQS_OK) return as;
  const int nf = (int)c->n_free;
  cudaStream_t st = c->stream;
  if (!c->ens_solve_graph.exec) {
    cudaStream_t cs = c->cap_stream;
    c->direct = false;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    EnsSlots sl{c->d_eiters, c->d_erelres, c->d_ezero};
    const double tol = c->opts.rtol;
    const eqs_status stt = ens_pcg_capture(c, c->d_eR, c->d_esol, tol * tol, sl);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if (stt != EQS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return stt;
    }
    CK(ee);
    c->ens_solve_graph.graph = graph;
    CK(cudaGraphInstantiate(&c->ens_solve_graph.exec, graph, 0));
  }
  k4_interleave<<<nblk(nf), kBlock, 0, st>>>(nf, rhs, c->d_eR);
  k4_interleave<<<nblk(nf), kBlock, 0, st>>>(nf, z, c->d_esol);
  CK(cudaGraphLaunch(c->ens_solve_graph.exec, st));
  k4_deinterleave<<<nblk(nf), kBlock, 0, st>>>(nf, c->d_esol, z);
  int it[kEnsW];
  double rr[kEnsW];
  CK(cudaMemcpyAsync(it, c->d_eiters, sizeof(it), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(rr, c->d_erelres, sizeof(rr), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  eqs_status res = EQS_OK;
  for (int k = 0; k < kEnsW; ++k) {
    if (iters_out) iters_out[k] = it[k];
    if (!std::isfinite(rr[k])) res = fail(c, EQS_ERR_NAN, "non-finite residual in the ensemble solve");
    else if (rr[k] > c->opts.rtol && res == EQS_OK) res = fail(c, EQS_ERR_NOCONV, "ensemble CG reached max_iter");
  }
  return res;
}

eqs_status eqs_ens_spe_eval(eqs_ctx* c, const double* X, const double* b, double* x0, double* r0) {
  REQUIRE_SETUP(c);
  if (!X || !b || !x0 || !r0) return fail(c, EQS_ERR_ARG, "null vector");
  const eqs_status as = ens_alloc(c);
  if (as != EQS_OK) return as;
  const int nf = (int)c->n_free;
  cudaStream_t st = c->stream;
  TmpBuf<long long> tcnt;
  CK(tcnt.alloc(2));
  const long long zero2[2] = {0, 1};  // stepcount 0: solve index g = j
  CK(cudaMemcpyAsync(tcnt.p, zero2, sizeof(zero2), cudaMemcpyHostToDevice, st));
  PtrRestore<long long> restore{&c->d_estepcount, c->d_estepcount};
  c->d_estepcount = tcnt.p;
  k4_interleave_pair<<<nblk(nf), kBlock, 0, st>>>(nf, b, c->d_eR, c->d_eR2);
  // push the history oldest first (solution q into slot q), updating the
  // Gram matrices as the step does, then form the start of the solve g = NH
  for (int q = 0; q < kEnsSpe; ++q) {
    const double* col = X + (size_t)(kEnsSpe - 1 - q) * kEnsW * nf;
    k4_interleave_pair<<<nblk(nf), kBlock, 0, st>>>(nf, col, c->d_eX + (size_t)q * nf,
                                                    c->d_eX2 + (size_t)q * 2 * nf);
    ens_spe_gram(c, st, 1, q + 1);
  }
  EnsSlots sl{c->d_eiters, c->d_erelres, c->d_ezero};
  ens_init_launch(c, st, c->d_eR, c->d_esol, 0.0, 0, 0, sl, true);
  k4_deinterleave<<<nblk(nf), kBlock, 0, st>>>(nf, c->d_esol, x0);
  k4_deinterleave<<<nblk(nf), kBlock, 0, st>>>(nf, c->d_er, r0);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(c, EQS_ERR_CUDA, cudaGetErrorString(e));
  return EQS_OK;
}

double eqs_rkc_dt_bound(const eqs_ctx* c, int s) {
  if (!c || !c->have_materials || s < 2 || s > EQS_MAX_STAGES) return -1.0;
  std::vector<double> mu, nu, mut, gt, cj;
  double beta;
  rkc_coefficients(s, mu, nu, mut, gt, cj, beta);
  const double rho = rho_bound(c->mats);
  return rho > 0 ? beta / rho : -1.0;
}

eqs_status eqs_set_stream(eqs_ctx* c, void* stream) {
  if (!c) return fail(nullptr, EQS_ERR_ARG, "ctx is NULL");
  c->stream = (cudaStream_t)stream;  // NULL: the legacy default stream
  return EQS_OK;
}

eqs_status eqs_get_sizes(const eqs_ctx* c, int64_t* n_nodes, int64_t* n_free, int64_t* n_tets) {
  if (!c) return fail(nullptr, EQS_ERR_ARG, "ctx is NULL");
  if (n_nodes) *n_nodes = c->n_nodes;
  if (n_free) *n_free = c->n_free;
  if (n_tets) *n_tets = c->n_tets;
  return EQS_OK;
}

eqs_status eqs_amg_info(const eqs_ctx* c, int* n_levels, int64_t* rows, int64_t* nnz) {
  if (!c) return fail(nullptr, EQS_ERR_ARG, "ctx is NULL");
  if (!c->hier_ready) return fail(const_cast<eqs_ctx*>(c), EQS_ERR_STATE, "call eqs_amg_setup first");
  const int nl = (int)c->hlev.size();
  if (n_levels) *n_levels = nl;
  for (int l = 0; l < nl && l < 16; ++l) {
    if (rows) rows[l] = c->hlev[l].A.n_rows;
    if (nnz) nnz[l] = c->hlev[l].A.nnz();
  }
  return EQS_OK;
}

eqs_status eqs_amg_aggregates(const eqs_ctx* c, int level, int32_t* agg_out) {
  if (!c) return fail(nullptr, EQS_ERR_ARG, "ctx is NULL");
  if (!c->hier_ready) return fail(const_cast<eqs_ctx*>(c), EQS_ERR_STATE, "call eqs_amg_setup first");
  if (!agg_out || level < 0 || level + 1 >= (int)c->hlev.size())
    return fail(const_cast<eqs_ctx*>(c), EQS_ERR_ARG, "level has no aggregates");
  std::memcpy(agg_out, c->hlev[level].agg.data(), c->hlev[level].agg.size() * sizeof(int32_t));
  return EQS_OK;
}

eqs_status eqs_set_guess(eqs_ctx* c, int mode) {
  REQUIRE_SETUP(c);
  if (mode != EQS_GUESS_PREV && mode != EQS_GUESS_MLP && mode != EQS_GUESS_ZERO && mode != EQS_GUESS_SPE &&
      mode != EQS_GUESS_POD && mode != EQS_GUESS_POD2 && mode != EQS_GUESS_SPE_MLP)
    return fail(c, EQS_ERR_ARG, "unknown guess mode");
  if (mode != c->opts.guess) {
    destroy_graphs(c);
    // SPE and its learned correction share the rings: between them the history carries over
    const bool spe_new = mode == EQS_GUESS_SPE || mode == EQS_GUESS_SPE_MLP;
    const bool spe_old = c->opts.guess == EQS_GUESS_SPE || c->opts.guess == EQS_GUESS_SPE_MLP;
    if ((spe_new && !spe_old) || mode == EQS_GUESS_POD || mode == EQS_GUESS_POD2) {
      // the solution rings / snapshot set start empty: restart the history
      CK(cudaStreamSynchronize(c->stream));
      CK(cudaMemset(c->d_stepcount, 0, 2 * sizeof(long long)));
      CK(cudaMemset(c->d_pod_state, 0, sizeof(PodState)));
      if (c->d_estepcount) CK(cudaMemset(c->d_estepcount, 0, 2 * sizeof(long long)));
    }
  }
  c->opts.guess = mode;
  return EQS_OK;
}

eqs_status eqs_guess_set_params(eqs_ctx* c, const float* theta, int n) {
  REQUIRE_SETUP(c);
  if (!theta || n != kNP) return fail(c, EQS_ERR_ARG, "expected 1377 parameters");
  for (int k = 0; k < n; ++k)
    if (!std::isfinite(theta[k])) return fail(c, EQS_ERR_NAN, "non-finite network parameter");
  CK(cudaMemcpyAsync(c->d_theta, theta, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  k_to_bf16<<<nblk(kNP), kBlock, 0, c->stream>>>(kNP, c->d_theta, (__nv_bfloat16*)c->d_theta_bf16);
  CK(cudaMemsetAsync(c->d_adam_m, 0, kNP * sizeof(float), c->stream));
  CK(cudaMemsetAsync(c->d_adam_v, 0, kNP * sizeof(float), c->stream));
  CK(cudaMemsetAsync(c->d_grad, 0, kNP * sizeof(float), c->stream));
  c->adam_t = 0;
  CK(cudaStreamSynchronize(c->stream));
  return EQS_OK;
}

eqs_status eqs_guess_get_params(eqs_ctx* c, float* theta, int n) {
  REQUIRE_SETUP(c);
  if (!theta || n != kNP) return fail(c, EQS_ERR_ARG, "expected 1377 parameters");
  CK(cudaMemcpyAsync(theta, c->d_theta, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return EQS_OK;
}

eqs_status eqs_guess_record(eqs_ctx* c, int64_t capacity) {
  REQUIRE_SETUP(c);
  if (capacity < 0) return fail(c, EQS_ERR_ARG, "negative capacity");
  destroy_graphs(c);  // the record target is part of the step graphs
  CK(cudaStreamSynchronize(c->stream));
  if (c->d_store) {
    for (auto it = c->allocs.begin(); it != c->allocs.end();)
      if (*it == c->d_store || *it == c->d_store_rms || *it == c->d_store_e || *it == c->d_store_rms_e) {
        cudaFree(*it);
        it = c->allocs.erase(it);
      } else {
        ++it;
      }
    c->d_store = nullptr;
    c->d_store_rms = nullptr;
    c->d_store_e = nullptr;
    c->d_store_rms_e = nullptr;
  }
  c->store_cap = 0;
  c->recording = false;
  c->recorded = 0;
  if (capacity == 0) return EQS_OK;
  CK(dalloc(c, &c->d_store, (size_t)capacity * (size_t)c->n_free, false));
  CK(dalloc(c, &c->d_store_e, (size_t)capacity * (size_t)c->n_free, false));
  CK(dalloc(c, &c->d_store_rms, (size_t)capacity));
  CK(dalloc(c, &c->d_store_rms_e, (size_t)capacity));
  c->store_e_valid = true;
  CK(cudaMemset(c->d_stepcount, 0, 2 * sizeof(long long)));  // history index restarts at 0
  c->store_cap = capacity;
  c->recording = true;
  return EQS_OK;
}

static eqs_status train_batch(eqs_ctx* c, int count, int B, unsigned long long seed, long long step,
                              const float* X, const float* T, const float* store_e = nullptr) {
  const int S = kTrainBlock + 1;
  const size_t smem = sizeof(float) * (kNP + 3 + (size_t)S * (8 + 32 * 4 + 1));
  CK(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_mlp_train<<<nblk(B, kTrainBlock), kTrainBlock, smem, c->stream>>>(
      (int)c->n_free, c->d_store, c->d_store_rms, count, c->d_adj_ptr, c->d_adj_col, c->d_inv_deg,
      (const __nv_bfloat16*)c->d_theta_bf16, c->d_grad, c->d_loss, seed, step, B, X, T, store_e,
      (const float*)c->d_store_rms_e);
  CK(cudaGetLastError());
  return EQS_OK;
}

eqs_status eqs_guess_train(eqs_ctx* c, int iters, int batch, float lr, uint64_t seed, float* loss_first,
                           float* loss_last) {
  REQUIRE_SETUP(c);
  if (iters < 1 || batch < 1 || !(lr > 0)) return fail(c, EQS_ERR_ARG, "bad training arguments");
  if (c->recorded < 5) return fail(c, EQS_ERR_STATE, "record at least 5 solutions first");
  const bool spe = c->opts.guess == EQS_GUESS_SPE_MLP;  // train the correction of the SPE start
  if (spe && !c->store_e_valid)
    return fail(c, EQS_ERR_STATE, "the SPE correction trains on steps recorded with SPE start vectors");
  CK(cudaStreamSynchronize(c->stream));
  const int count = (int)c->recorded;
  if (spe)
    k_store_rms_spe<<<count, kBlock, 0, c->stream>>>((int)c->n_free, c->d_store, c->d_store_e, c->d_store_rms,
                                                      c->d_store_rms_e);
  else
    k_store_rms<<<count, kBlock, 0, c->stream>>>((int)c->n_free, c->d_store, c->d_store_rms);
  float lf = 0.f, ll = 0.f;
  for (int it = 0; it < iters; ++it) {
    CK(cudaMemsetAsync(c->d_loss, 0, sizeof(float), c->stream));
    const eqs_status st = train_batch(c, count, batch, seed, it, nullptr, nullptr, spe ? c->d_store_e : nullptr);
    if (st != EQS_OK) return st;
    c->adam_t += 1;
    const float bc1 = 1.0f - std::pow(0.9f, (float)c->adam_t);
    const float bc2 = 1.0f - std::pow(0.999f, (float)c->adam_t);
    k_adam<<<nblk(kNP), kBlock, 0, c->stream>>>(c->d_theta, c->d_adam_m, c->d_adam_v, c->d_grad,
                                                (__nv_bfloat16*)c->d_theta_bf16, lr, bc1, bc2);
    if (it == 0 || it == iters - 1) {
      float l = 0.f;
      CK(cudaMemcpyAsync(&l, c->d_loss, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      (it == 0 ? lf : ll) = l;
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  if (loss_first) *loss_first = lf;
  if (loss_last) *loss_last = ll;
  return EQS_OK;
}

eqs_status eqs_guess_grad(eqs_ctx* c, const float* X, const float* T, int B, float* grad, float* loss) {
  REQUIRE_SETUP(c);
  if (!X || !T || !grad || B < 1) return fail(c, EQS_ERR_ARG, "bad gradient arguments");
  TmpBuf<float> tX, tT;
  CK(tX.alloc((size_t)B * 8));
  CK(tT.alloc((size_t)B));
  float* dX = tX.p;
  float* dT = tT.p;
  CK(cudaMemcpy(dX, X, (size_t)B * 8 * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dT, T, (size_t)B * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemset(c->d_grad, 0, kNP * sizeof(float)));
  CK(cudaMemset(c->d_loss, 0, sizeof(float)));
  eqs_status st = train_batch(c, 5, B, 0ull, 0, dX, dT);
  if (st == EQS_OK) {
    cudaError_t e = cudaMemcpy(grad, c->d_grad, kNP * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && loss) e = cudaMemcpy(loss, c->d_loss, sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->d_grad, 0, kNP * sizeof(float));
    if (e != cudaSuccess) st = fail(c, EQS_ERR_CUDA, cudaGetErrorString(e));
  }
  return st;
}

eqs_status eqs_guess_train_batches(eqs_ctx* c, const float* X, const float* T, int B, int n_batches, float lr,
                                   float* losses) {
  REQUIRE_SETUP(c);
  if (!X || !T || B < 1 || n_batches < 1 || !(lr > 0)) return fail(c, EQS_ERR_ARG, "bad training arguments");
  TmpBuf<float> tX, tT;
  CK(tX.alloc((size_t)B * 8 * n_batches));
  CK(tT.alloc((size_t)B * n_batches));
  CK(cudaMemcpy(tX.p, X, (size_t)B * 8 * n_batches * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(tT.p, T, (size_t)B * n_batches * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemset(c->d_grad, 0, kNP * sizeof(float)));
  for (int k = 0; k < n_batches; ++k) {
    CK(cudaMemsetAsync(c->d_loss, 0, sizeof(float), c->stream));
    const eqs_status st = train_batch(c, 5, B, 0ull, 0, tX.p + (size_t)k * B * 8, tT.p + (size_t)k * B);
    if (st != EQS_OK) return st;
    c->adam_t += 1;  // the same update as eqs_guess_train
    const float bc1 = 1.0f - std::pow(0.9f, (float)c->adam_t);
    const float bc2 = 1.0f - std::pow(0.999f, (float)c->adam_t);
    k_adam<<<nblk(kNP), kBlock, 0, c->stream>>>(c->d_theta, c->d_adam_m, c->d_adam_v, c->d_grad,
                                                (__nv_bfloat16*)c->d_theta_bf16, lr, bc1, bc2);
    if (losses) {
      CK(cudaMemcpyAsync(losses + k, c->d_loss, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  return EQS_OK;
}

eqs_status eqs_spe_eval(eqs_ctx* c, const double* X, const double* b, int n, double* x0) {
  REQUIRE_SETUP(c);
  if (!X || !b || !x0) return fail(c, EQS_ERR_ARG, "null vector");
  if (n != c->opts.spe_n) return fail(c, EQS_ERR_ARG, "n must equal the context's spe_n");
  const int64_t nf = c->n_free;
  cudaStream_t st = c->stream;
  TmpBuf<long long> tcnt;
  CK(tcnt.alloc(2));
  long long* cnt = tcnt.p;
  const long long zero2[2] = {0, 1};  // stepcount 0: solve index g = j
  CK(cudaMemcpyAsync(cnt, zero2, sizeof(zero2), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(c->d_R, b, nf * sizeof(double), cudaMemcpyDeviceToDevice, st));
  PtrRestore<long long> restore{&c->d_stepcount, c->d_stepcount};
  c->d_stepcount = cnt;
  // push the history oldest first (solution q into slot q % n), updating the
  // Gram matrix as the step does, then form x0 for the solve g = n
  for (int q = 0; q < n; ++q) {
    const double* col = X + (size_t)(n - 1 - q) * nf;
    CK(cudaMemcpyAsync(c->d_spe_X + (size_t)(q % n) * nf, col, nf * sizeof(double), cudaMemcpyDeviceToDevice,
                       st));
    spe_gram(c, st, 1, q + 1, false);
  }
  SolveSlots sl{nullptr, nullptr, nullptr};
  if (mixed(c))
    spe_start<float>(c, c->lev32, st, 1, n, nullptr, x0, 0.0, 0, 0, sl);
  else
    spe_start<double>(c, c->lev64, st, 1, n, nullptr, x0, 0.0, 0, 0, sl);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(c, EQS_ERR_CUDA, cudaGetErrorString(e));
  return EQS_OK;
}

eqs_status eqs_pod_eval(eqs_ctx* c, const double* X, int K, const double* b, double* x0) {
  REQUIRE_SETUP(c);
  if (!X || !b || !x0) return fail(c, EQS_ERR_ARG, "null vector");
  if (K < 1 || K > c->opts.pod_k) return fail(c, EQS_ERR_ARG, "K must be in [1, pod_k]");
  const int64_t nf = c->n_free;
  cudaStream_t st = c->stream;
  TmpBuf<long long> tcnt;
  TmpBuf<int> tzero;
  CK(tcnt.alloc(2));
  CK(tzero.alloc(1));
  long long* cnt = tcnt.p;
  int* zero = tzero.p;
  const long long one2[2] = {1, 2};  // solve index g = 1: a previous solution exists
  CK(cudaMemcpyAsync(cnt, one2, sizeof(one2), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(zero, 0, sizeof(int), st));
  CK(cudaMemsetAsync(c->d_pod_state, 0, sizeof(PodState), st));
  CK(cudaMemcpyAsync(c->d_R, b, nf * sizeof(double), cudaMemcpyDeviceToDevice, st));
  PodState* ps = (PodState*)c->d_pod_state;
  const int nfi = (int)nf;
  // the K snapshots enter by the fixed-set rule with capacity K, oldest first;
  // the basis is built when the set is full
  for (int q = 0; q < K; ++q) {
    k_pod_add<kPodMax><<<vec_grid(c, nfi), kBlock, 0, st>>>(c->M64, nfi, c->d_pod_X, c->d_pod_W, c->d_pod_GE,
                                                            c->d_pod_GM, X + (size_t)q * nf, zero, zero, cnt, 1,
                                                            0, 0, K, 0, ps, c->d_pod_partials, c->red.counter,
                                                            c->red.max_blocks);
    k_pod_rebuild<kPodMax><<<1, kBlock, 0, st>>>(c->d_pod_GE, c->d_pod_GM, c->opts.pod_m, kPodDrop2, ps);
  }
  k_pod_gram<kPodMax><<<std::max(1, std::min(nblk(nf), c->sms)), kBlock, 0, st>>>(
      nfi, c->d_pod_X, c->d_R, ps, c->d_pod_a, c->d_pod_partials, c->red.counter, c->red.max_blocks);
  SolveSlots sl{nullptr, nullptr, nullptr};
  if (mixed(c))
    pod_start<float>(c, c->lev32, st, nullptr, x0, 0.0, 0, 0, sl);
  else
    pod_start<double>(c, c->lev64, st, nullptr, x0, 0.0, 0, 0, sl);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(c, EQS_ERR_CUDA, cudaGetErrorString(e));
  return EQS_OK;
}

eqs_status eqs_pod_info(eqs_ctx* c, int* count, int* modes, int* rebuilds, int* adds, double* lam) {
  REQUIRE_SETUP(c);
  PodState ps;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(&ps, c->d_pod_state, sizeof(ps), cudaMemcpyDeviceToHost));
  if (count) *count = ps.count;
  if (modes) *modes = ps.m_used;
  if (rebuilds) *rebuilds = ps.rebuilds;
  if (adds) *adds = ps.adds;
  if (lam)
    for (int k = 0; k < kPodMax; ++k) lam[k] = k < ps.count ? ps.lam[k] : 0.0;
  return EQS_OK;
}

eqs_status eqs_guess_eval(eqs_ctx* c, const double* H, double* z0) {
  REQUIRE_SETUP(c);
  if (!H || !z0) return fail(c, EQS_ERR_ARG, "null vector");
  const int nf = (int)c->n_free;
  cudaStream_t st = c->stream;
  TmpBuf<float> tring;
  TmpBuf<long long> tcnt;
  CK(tring.alloc(4 * (size_t)nf));
  CK(tcnt.alloc(2));
  float* ring = tring.p;
  long long* cnt = tcnt.p;
  // solve index g = 4: h_l (l = 1..4) goes to slot (4 - l) % 4
  for (int l = 0; l < 4; ++l)
    k_push_solution<<<nblk(nf), kBlock, 0, st>>>(nf, H + (size_t)l * nf, ring + (size_t)((3 - l) & 3) * nf);
  const long long four[2] = {4, 5};
  CK(cudaMemcpyAsync(cnt, four, sizeof(four), cudaMemcpyHostToDevice, st));
  k_rms<<<vec_grid(c, nf), kBlock, 0, st>>>(nf, H, c->d_sh, c->red.partials, c->red.counter,
                                           c->red.max_blocks);
  k_mlp_guess<<<nblk(nf), kBlock, 0, st>>>(nf, H, ring, cnt, 1, 0, c->d_adj_ptr, c->d_adj_col, c->d_inv_deg,
                                         (const __nv_bfloat16*)c->d_theta_bf16, c->d_sh, z0);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(c, EQS_ERR_CUDA, cudaGetErrorString(e));
  return EQS_OK;
}

eqs_status eqs_guess_eval_spe(eqs_ctx* c, const double* x0, const double* H, const double* R, double* z0) {
  REQUIRE_SETUP(c);
  if (!x0 || !H || !R || !z0) return fail(c, EQS_ERR_ARG, "null vector");
  const int nf = (int)c->n_free;
  cudaStream_t st = c->stream;
  TmpBuf<float> tring;
  TmpBuf<long long> tcnt;
  TmpBuf<double> td, tq;
  TmpBuf<int> tuse;
  CK(tring.alloc(4 * (size_t)nf));
  CK(tcnt.alloc(2));
  CK(td.alloc(nf));
  CK(tq.alloc(nf));
  CK(tuse.alloc(1));
  for (int l = 0; l < 4; ++l)  // solve index g = 4: h_l (l = 1..4) goes to slot (4 - l) % 4
    k_push_solution<<<nblk(nf), kBlock, 0, st>>>(nf, H + (size_t)l * nf, tring.p + (size_t)((3 - l) & 3) * nf);
  const long long four[2] = {4, 5};
  const int one = 1;
  CK(cudaMemcpyAsync(tcnt.p, four, sizeof(four), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(tuse.p, &one, sizeof(one), cudaMemcpyHostToDevice, st));
  k_rms_diff<<<vec_grid(c, nf), kBlock, 0, st>>>(nf, x0, H, tuse.p, c->d_sh, c->red.partials, c->red.counter,
                                                 c->red.max_blocks);
  k_mlp_dir_spe<<<nblk(nf), kBlock, 0, st>>>(nf, x0, H, tring.p, tcnt.p, 0, tuse.p, c->d_adj_ptr, c->d_adj_col,
                                             c->d_inv_deg, (const __nv_bfloat16*)c->d_theta_bf16, c->d_sh, td.p);
  k_dir_alpha<<<vec_grid(c, nf), kBlock, 0, st>>>(c->M64, nf, td.p, nullptr, R, x0, tq.p, c->d_alpha,
                                                  c->red.partials, c->red.counter, c->red.max_blocks);
  k_axpy_alpha<<<nblk(nf), kBlock, 0, st>>>(nf, x0, td.p, c->d_alpha, z0);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(c, EQS_ERR_CUDA, cudaGetErrorString(e));
  return EQS_OK;
}

// ------------------------------------------------------------- batches
}  // extern "C"

struct eqs_batch {
  std::vector<eqs_ctx*> ctx;
  int device = 0, sms = 0, total_blocks = 0, rows_per_block = 0;
  std::vector<int> first, nblk, blk2inst;
  BatchInst* d_insts = nullptr;
  int *d_blk2inst = nullptr, *d_first = nullptr, *d_nblk = nullptr;
  GridBarrier* d_bars = nullptr;
  double *d_gtab = nullptr, *d_gptab = nullptr;
  double** d_x = nullptr;
  StepParams* d_params = nullptr;
  long long* d_count = nullptr;       // solves before / after the current step (SPE history index)
  long long max_spins = kMaxSpins;    // wait budget of one group barrier (polls)
  cudaStream_t stream = nullptr, cap = nullptr;
  std::map<int, GraphEntry> graphs;
  std::vector<void*> allocs;
  std::string err;
  int last_s = 0;
};

static eqs_status bfail(eqs_batch* b, eqs_status st, const std::string& m) {
  if (b)
    b->err = m;
  else
    g_create_err = m;
  return st;
}

#define BCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return bfail(b, EQS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

template <typename T>
static cudaError_t balloc(eqs_batch* b, T** p, size_t n) {
  cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
  if (e == cudaSuccess) {
    b->allocs.push_back(*p);
    e = cudaMemset(*p, 0, std::max<size_t>(n, 1) * sizeof(T));
  }
  return e;
}

static void batch_free(eqs_batch* b) {
  for (auto& kv : b->graphs) destroy_graph(kv.second);
  b->graphs.clear();
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
}

static eqs_status batch_capture(eqs_batch* b, int s, GraphEntry& ge) {
  std::vector<double> mu, nu, mut, gt, cj;
  double beta;
  rkc_coefficients(s, mu, nu, mut, gt, cj, beta);
  double* d_cj = nullptr;
  BCK(balloc(b, &d_cj, cj.size()));
  BCK(cudaMemcpy(d_cj, cj.data(), cj.size() * sizeof(double), cudaMemcpyHostToDevice));
  ge.d_cj = d_cj;
  const int ninst = (int)b->ctx.size();
  const double tol2 = b->ctx[0]->opts.rtol * b->ctx[0]->opts.rtol;
  cudaStream_t st = b->cap;
  BCK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  cudaMemsetAsync(b->d_bars, 0, ninst * sizeof(GridBarrier), st);
  k_batch_drive<<<nblk((int64_t)ninst * (s + 1)), kBlock, 0, st>>>(ninst, s + 1, b->d_insts, d_cj, b->d_params,
                                                                    b->d_gtab, b->d_gptab, b->d_count);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->total_blocks);
  cfg.blockDim = dim3(kPBlock);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  for (int j = 0; j < s; ++j) {
    const bool first = (j <= 1);
    const double c0 = j == 0 ? 0.0 : (j == 1 ? 1.0 : 1.0 - mu[j] - nu[j]);
    cudaLaunchKernelEx(&cfg, k_batch_stage, (const BatchInst*)b->d_insts, (const int*)b->d_blk2inst,
                       (const int*)b->d_first, (const int*)b->d_nblk, j, s, c0, first ? 0.0 : mu[j],
                       first ? 0.0 : nu[j], j == 0 ? 0.0 : mut[j], first ? 0.0 : gt[j],
                       (const StepParams*)b->d_params, (const double*)b->d_gtab, (const double*)b->d_gptab,
                       (double* const*)b->d_x, tol2, (const long long*)b->d_count, b->max_spins);
  }
  k_batch_final<<<b->total_blocks, kPBlock, 0, st>>>(b->d_insts, b->d_blk2inst, b->d_first, b->d_nblk, s,
                                                    1.0 - mu[s] - nu[s], mu[s], nu[s], mut[s], gt[s],
                                                    b->d_params, b->d_gtab, b->d_x);
  cudaError_t le = cudaGetLastError();
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  BCK(le);
  BCK(ee);
  ge.graph = graph;
  ge.s = s;
  ge.fixed_kernels = count_kernel_nodes(graph);
  ge.per_iter_kernels = 0;
  BCK(cudaGraphInstantiate(&ge.exec, graph, 0));
  return EQS_OK;
}

extern "C" {

eqs_status eqs_batch_create(eqs_ctx* const* ctxs, int n, int rows_per_block, eqs_batch** out) {
  if (!out) return bfail(nullptr, EQS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1 || rows_per_block < 32) return bfail(nullptr, EQS_ERR_ARG, "bad batch arguments");
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k] || !ctxs[k]->setup_done) return bfail(nullptr, EQS_ERR_STATE, "every context must be set up");
    if (ctxs[k]->opts.precision != EQS_PREC_MIXED)
      return bfail(nullptr, EQS_ERR_ARG, "batched stages run in mixed precision");
    if (ctxs[k]->npe != 4) return bfail(nullptr, EQS_ERR_ARG, "batched stages run linear (4-node) tets");
    if (ctxs[k]->device != ctxs[0]->device) return bfail(nullptr, EQS_ERR_ARG, "contexts on different devices");
    if (ctxs[k]->opts.rtol != ctxs[0]->opts.rtol) return bfail(nullptr, EQS_ERR_ARG, "contexts differ in rtol");
  }
  eqs_batch* b = new eqs_batch();
  b->ctx.assign(ctxs, ctxs + n);
  b->device = ctxs[0]->device;
  b->sms = ctxs[0]->sms;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_stage, kPBlock, 0) != cudaSuccess || occ < 1) {
    delete b;
    return bfail(nullptr, EQS_ERR_CUDA, "batched stage kernel cannot be resident");
  }
  const int cap_blocks = occ * b->sms;
  // CTAs per instance proportional to its free rows; scale until co-resident
  int r = rows_per_block;
  for (;;) {
    b->first.assign(n, 0);
    b->nblk.assign(n, 0);
    int tot = 0;
    for (int k = 0; k < n; ++k) {
      const int64_t nf = ctxs[k]->n_free;
      b->nblk[k] = (int)std::min<int64_t>(std::max<int64_t>(1, (nf + r - 1) / r), ctxs[k]->pblocks);
      b->first[k] = tot;
      tot += b->nblk[k];
    }
    if (tot <= cap_blocks) {
      b->total_blocks = tot;
      break;
    }
    if (n > cap_blocks) {
      delete b;
      return bfail(nullptr, EQS_ERR_ARG, "more instances than co-resident CTAs");
    }
    r += r / 4 + 1;
  }
  b->rows_per_block = r;
  // SPE start vectors when every instance's context selects them
  bool spe = true;
  for (int k = 0; k < n; ++k) spe = spe && ctxs[k]->opts.guess == EQS_GUESS_SPE;
  b->blk2inst.resize(b->total_blocks);
  for (int k = 0; k < n; ++k)
    for (int q = 0; q < b->nblk[k]; ++q) b->blk2inst[b->first[k] + q] = k;
  std::vector<BatchInst> hi(n);
  for (int k = 0; k < n; ++k) {
    eqs_ctx* c = ctxs[k];
    BatchInst& I = hi[k];
    I.plan = (const PPlan<float>*)c->d_plan;
    I.partials = c->d_ppartials;
    I.n = (int)c->n_nodes;
    I.nf = (int)c->n_free;
    I.nt = c->n_tets;
    I.conn = c->d_conn;
    I.mat = c->d_mat;
    I.mats = c->d_mats;
    I.xh = c->d_xyz_hi;
    I.xl = c->d_xyz_lo;
    I.node_of_internal = c->d_node_of_internal;
    I.dir_scale = c->d_dir_scale;
    I.mtop = c->d_mtop;
    for (int q = 0; q < 4; ++q) I.Y[q] = c->d_Y[q];
    I.Y32 = c->d_Y32;
    for (int q = 0; q < 3; ++q) I.F[q] = c->d_F[q];
    I.R = c->d_R;
    I.y32 = c->d_y32;
    I.iters = c->d_iters;
    I.relres = c->d_relres;
    I.zero = c->d_zero;
    I.V0 = c->V0;
    I.w = 2.0 * M_PI * c->freq;
    I.phase = c->phase;
    I.X = spe ? c->d_spe_X : nullptr;
    I.G = spe ? c->d_spe_G : nullptr;
    I.coef = spe ? c->d_spe_y : nullptr;
  }
  cudaError_t e = cudaSetDevice(b->device);
  if (e == cudaSuccess) e = balloc(b, &b->d_bars, n);
  for (int k = 0; k < n && e == cudaSuccess; ++k) hi[k].bar = b->d_bars + k;
  if (e == cudaSuccess) e = balloc(b, &b->d_insts, n);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_insts, hi.data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = balloc(b, &b->d_blk2inst, b->total_blocks);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_blk2inst, b->blk2inst.data(), b->total_blocks * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = balloc(b, &b->d_first, n);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_first, b->first.data(), n * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = balloc(b, &b->d_nblk, n);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_nblk, b->nblk.data(), n * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = balloc(b, &b->d_gtab, (size_t)n * (EQS_MAX_STAGES + 1));
  if (e == cudaSuccess) e = balloc(b, &b->d_gptab, (size_t)n * (EQS_MAX_STAGES + 1));
  if (e == cudaSuccess) e = balloc(b, &b->d_x, n);
  if (e == cudaSuccess) e = balloc(b, &b->d_params, 1);
  if (e == cudaSuccess) e = balloc(b, &b->d_count, 2);
  if (e == cudaSuccess) e = cudaMemset(b->d_count, 0, 2 * sizeof(long long));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    g_create_err = std::string("batch setup: ") + cudaGetErrorString(e);
    batch_free(b);
    delete b;
    return EQS_ERR_CUDA;
  }
  b->stream = ctxs[0]->stream;
  *out = b;
  return EQS_OK;
}

eqs_status eqs_batch_rkc_step(eqs_batch* b, double* const* x, double t, double dt, int s,
                              eqs_batch_stats* stats) {
  if (!b) return bfail(nullptr, EQS_ERR_ARG, "batch is NULL");
  if (!x) return bfail(b, EQS_ERR_ARG, "x is NULL");
  if (s < 2 || s > EQS_MAX_STAGES) return bfail(b, EQS_ERR_ARG, "s out of range [2, 64]");
  if (!std::isfinite(t) || !(dt > 0) || !std::isfinite(dt)) return bfail(b, EQS_ERR_ARG, "bad t or dt");
  const int n = (int)b->ctx.size();
  for (int k = 0; k < n; ++k)
    if (!x[k]) return bfail(b, EQS_ERR_ARG, "null instance vector");
  auto it = b->graphs.find(s);
  if (it == b->graphs.end()) {
    GraphEntry ge;
    const eqs_status st = batch_capture(b, s, ge);
    if (st != EQS_OK) return st;
    it = b->graphs.emplace(s, ge).first;
  }
  const StepParams prm{t, dt};
  BCK(cudaMemcpyAsync(b->d_params, &prm, sizeof(prm), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_x, x, n * sizeof(double*), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaGraphLaunch(it->second.exec, b->stream));
  b->last_s = s;
  if (!stats) return EQS_OK;
  return eqs_batch_get_stats(b, stats, nullptr);
}

eqs_status eqs_batch_get_stats(eqs_batch* b, eqs_batch_stats* stats, int64_t* inst_iters) {
  if (!b || !stats) return bfail(b, EQS_ERR_ARG, "null argument");
  if (!b->last_s) return bfail(b, EQS_ERR_STATE, "no batched step has run");
  const int s = b->last_s, n = (int)b->ctx.size();
  BCK(cudaStreamSynchronize(b->stream));
  std::memset(stats, 0, sizeof(*stats));
  stats->n_inst = n;
  stats->s = s;
  stats->launches = b->graphs[s].fixed_kernels;
  eqs_status res = EQS_OK;
  for (int k = 0; k < n; ++k) {
    int iters[EQS_MAX_STAGES];
    double rr[EQS_MAX_STAGES];
    BCK(cudaMemcpy(iters, b->ctx[k]->d_iters, s * sizeof(int), cudaMemcpyDeviceToHost));
    BCK(cudaMemcpy(rr, b->ctx[k]->d_relres, s * sizeof(double), cudaMemcpyDeviceToHost));
    int64_t tot = 0;
    for (int j = 0; j < s; ++j) {
      tot += iters[j];
      stats->max_iters = std::max(stats->max_iters, iters[j]);
      stats->max_relres = std::max(stats->max_relres, rr[j]);
      if (!std::isfinite(rr[j])) res = EQS_ERR_NAN;
      else if (rr[j] > b->ctx[k]->opts.rtol && res == EQS_OK) res = EQS_ERR_NOCONV;
    }
    stats->total_iters += tot;
    if (inst_iters) inst_iters[k] = tot;
  }
  std::vector<GridBarrier> bars(n);
  BCK(cudaMemcpy(bars.data(), b->d_bars, n * sizeof(GridBarrier), cudaMemcpyDeviceToHost));
  for (int k = 0; k < n; ++k)
    if (bars[k].err) res = EQS_ERR_TIMEOUT;
  stats->status = res;
  if (res == EQS_ERR_TIMEOUT) return bfail(b, res, "a group barrier of the batched step timed out");
  if (res == EQS_ERR_NOCONV) return bfail(b, res, "a stage solve reached max_iter");
  if (res == EQS_ERR_NAN) return bfail(b, res, "non-finite residual in a stage solve");
  return EQS_OK;
}

eqs_status eqs_batch_info(const eqs_batch* b, int* total_blocks, int* rows_per_block) {
  if (!b) return bfail(nullptr, EQS_ERR_ARG, "batch is NULL");
  if (total_blocks) *total_blocks = b->total_blocks;
  if (rows_per_block) *rows_per_block = b->rows_per_block;
  return EQS_OK;
}

eqs_status eqs_convert_check(const float* f, int n, double* f_wide) {
  if (!f || !f_wide || n < 0) return fail(nullptr, EQS_ERR_ARG, "bad conversion check arguments");
  if (n == 0) return EQS_OK;
  k_convert_check<<<nblk(n), kBlock>>>(n, f, f_wide);
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(nullptr, EQS_ERR_CUDA, cudaGetErrorString(e));
  return EQS_OK;
}

eqs_status eqs_batch_set_barrier_polls(eqs_batch* b, long long polls) {
  if (!b) return bfail(nullptr, EQS_ERR_ARG, "batch is NULL");
  if (polls < 0) return bfail(b, EQS_ERR_ARG, "polls must be >= 0");
  const long long v = polls == 0 ? kMaxSpins : polls;
  if (v != b->max_spins) {  // the budget is an argument of the captured launches
    BCK(cudaStreamSynchronize(b->stream));
    for (auto& kv : b->graphs) destroy_graph(kv.second);
    b->graphs.clear();
    b->max_spins = v;
  }
  return EQS_OK;
}

eqs_status eqs_batch_destroy(eqs_batch* b) {
  if (!b) return EQS_OK;
  if (b->stream || !b->allocs.empty()) cudaStreamSynchronize(b->stream);
  batch_free(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return EQS_OK;
}

const char* eqs_batch_last_error(const eqs_batch* b) { return b ? b->err.c_str() : g_create_err.c_str(); }

eqs_status eqs_destroy(eqs_ctx* c) {
  if (!c) return EQS_OK;
  if (c->setup_done) cudaStreamSynchronize(c->stream);
  destroy_graphs(c);
  free_all(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->cap_stream2) cudaStreamDestroy(c->cap_stream2);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
  return EQS_OK;
}

const char* eqs_last_error(const eqs_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
