// Internal structures of the EQS RKC library (host side).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "eqs.h"

namespace eqs {

// ---------------------------------------------------------------- host CSR
struct HostCSR {
  int64_t n_rows = 0, n_cols = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

// ------------------------------------------------------- device matrix
// Two layouts, chosen by the mean row length:
//  G == 1 (short rows): SELL-32.  Rows are grouped in slices of 32; slice s
//    stores width[s] columns, element k of row 32 s + lane at
//    ptr[s] + 32 k + lane (coalesced per warp, one thread per row).
//    Padding entries have value 0 and a valid column index.
//  G  > 1 (long rows): CSR with a group of G lanes per row (ptr = row
//    pointer); the group strides over the row and reduces with shuffles.
//  G == 0 (few diagonals): DIA.  Value of diagonal d, row i at
//    val[d * n_rows + i], column i + off[d] (zero where out of range);
//    reads of val and x are coalesced and no index is loaded.
constexpr int kMaxDiag = 32;
template <typename T>
struct DevSell {
  int n_rows = 0, n_cols = 0, n_slices = 0;
  int G = 1, logG = 0;
  int ndiag = 0;
  int off[kMaxDiag] = {};
  int64_t stored = 0, nnz = 0;
  int64_t* slice_ptr = nullptr;
  int32_t* col = nullptr;
  T* val = nullptr;
};

template <typename T>
struct DevLevel {
  int n = 0;
  double lam_max = 0, inv_theta = 0, sigma = 0, delta = 0;
  DevSell<T> A;     // level operator
  DevSell<T> P;     // prolongation to this level from level+1 (n x n_c)
  DevSell<T> R;     // restriction P^T (n_c x n)
  T* dinv = nullptr;
  T* b = nullptr;   // right-hand side of the level
  T* x = nullptr;   // iterate
  T* r = nullptr;   // residual work vector
  T* dA = nullptr;  // Chebyshev directions (ping-pong)
  T* dB = nullptr;
};

struct HostLevel {
  HostCSR A, P;
  std::vector<int32_t> agg;
  int n_agg = 0;
  double lam_max = 0, omega = 0;
};

// Per-solve reduction scalars (device).
struct PcgScalars {
  double bnorm2, rnorm2, rz, rz_old, zr_prev, pq, alpha, beta;
  double rz_hist[2];  // deferred sums: r.z of iteration it in slot it & 1
  int it, conv, parity, use_prev;  // use_prev: the previous solution replaced the learned guess
};

struct StepParams {  // device-resident per-call parameters
  double t, dt;
  double* x;  // the caller's node vector(s) of this call (step graphs do not depend on it)
};

// All scratch used by the reduction kernels of one solve.
struct ReduceScratch {
  double* partials = nullptr;   // per block partial sums (up to 4 per block)
  unsigned int* counter = nullptr;
  int max_blocks = 0;
};

struct MaterialDev {  // one row of the material table
  double eps, klo, khi, E0, inv_w;
  int is_const, pad;
  float klo_f, dk_f, E0_f, inv_w_f;  // FP32 copies (klo, khi - klo, E0, 1/w) for the FP32 kernels
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  double* d_cj = nullptr;  // stage abscissae c_0..c_s of this graph
  int64_t fixed_kernels = 0;     // kernel nodes outside the CG loops
  int64_t per_iter_kernels = 0;  // kernel nodes of one CG loop body
  int s = 0;
};

}  // namespace eqs

struct eqs_ctx {
  std::string err;
  cudaStream_t stream = nullptr;      // stream of all work (NULL: legacy default stream)
  cudaStream_t own_stream = nullptr;  // created at setup (marks that streams exist)
  cudaStream_t cap_stream = nullptr;  // capture of step / solve graphs
  cudaStream_t cap_stream2 = nullptr; // capture of while-loop bodies
  int device = 0;
  int sms = 0;                        // SM count of the device
  std::vector<void*> allocs;          // every device allocation of the context

  // ---- mesh (host copies)
  int64_t n_nodes = 0, n_tets = 0, n_free = 0;
  std::vector<double> xyz;          // mesh order, n x 3
  std::vector<int32_t> tets;        // mesh order, npe nodes per tet (vertices first)
  int npe = 4;                       // nodes per tet: 4 (P1) or 10 (P2: + edge midpoints)
  int32_t* d_conn10 = nullptr;       // P2: 10 x n_tets internal node ids (node-major)
  int64_t n_cells = 0;               // > 0: the tets form Kuhn cells (6 per cell, in order)
  int32_t* d_corner = nullptr;       // 8 x n_cells internal corner ids (corner-major)
  std::vector<uint8_t> tag;         // mesh order
  std::vector<int32_t> internal_of_node, node_of_internal;  // free first
  std::vector<uint8_t> tet_mat;
  std::vector<eqs_material> mats;
  bool have_materials = false;
  double V0 = 0, freq = 0, phase = 0;

  // ---- options / state
  eqs_opts opts{};
  bool setup_done = false;   // device data ready
  bool hier_ready = false;   // host AMG hierarchy built

  // ---- host AMG (kept for inspection)
  std::vector<eqs::HostLevel> hlev;
  int coarse_n = 0;

  // ---- device mesh
  int4* d_conn = nullptr;            // internal node ids, oriented
  uint8_t* d_mat = nullptr;
  double4* d_xyz = nullptr;          // internal order (x, y, z, 0)
  float4* d_xyz_hi = nullptr;        // two-float split (mixed precision)
  float4* d_xyz_lo = nullptr;
  int32_t* d_node_of_internal = nullptr;
  double* d_dir_scale = nullptr;     // per Dirichlet node: 1 driven, 0 grounded
  double* d_mtop = nullptr;          // M_fd 1_top (n_free)
  eqs::MaterialDev* d_mats = nullptr;

  // ---- device matrices
  eqs::DevSell<double> M64;          // M_ff in FP64 (CG operator)
  float* d_M_hi = nullptr;           // split M_ff = hi + lo (FP32 parts, M64's layout;
  float* d_M_lo = nullptr;           //   mixed path with split_m)
  float* d_z32 = nullptr;            // FP32 preconditioned residual (split operator pass)
  std::vector<eqs::DevLevel<double>> lev64;
  std::vector<eqs::DevLevel<float>> lev32;
  double* d_coarse_inv = nullptr;    // dense inverse of the coarsest matrix

  // ---- device vectors (FP64 unless noted)
  double* d_Y[4] = {nullptr, nullptr, nullptr, nullptr};  // Y0 + 3 rotating, n_nodes
  float2* d_Y32 = nullptr;           // two-float copy of the current stage vector
  double* d_F[3] = {nullptr, nullptr, nullptr};  // F0, Fa, Fb (n_free)
  double* d_R = nullptr;             // stage right-hand side (n_free)
  float* d_y32 = nullptr;            // FP32 accumulation of K(x)x (n_nodes)
  double* d_r = nullptr;
  double* d_rprev = nullptr;
  double* d_p = nullptr;
  double* d_q = nullptr;
  double* d_sol = nullptr;           // solve_M work solution
  double* d_zd = nullptr;            // preconditioned residual in FP64
  double* d_p2 = nullptr;            // second search-direction buffer (persistent solve)
  void* d_plan = nullptr;            // device PPlan<T> of the persistent solve
  void* d_bar = nullptr;             // grid barrier state
  double* d_ppartials = nullptr;     // 8 slots x persistent grid
  int pblocks = 0;                   // CTAs of the persistent solve
  double* d_tmpn = nullptr;          // n_nodes scratch (apply_K)
  double* d_tmpn2 = nullptr;
  eqs::PcgScalars* d_sc = nullptr;
  eqs::StepParams* d_params = nullptr;
  int* d_iters = nullptr;            // per stage iteration counts
  double* d_relres = nullptr;        // per stage final relative residuals
  int* d_zero = nullptr;             // per stage: right-hand side was zero
  double* d_g = nullptr;             // drive g(t_j) at the stage times
  double* d_gp = nullptr;            // drive derivative g'(t_j)
  eqs::ReduceScratch red;

  // ---- learned start vector (mlp.cu)
  int32_t* d_adj_ptr = nullptr;      // free-node graph (mesh edges), CSR
  int32_t* d_adj_col = nullptr;
  float* d_inv_deg = nullptr;
  float* d_theta = nullptr;          // FP32 master parameters (1377)
  void* d_theta_bf16 = nullptr;      // BF16 copy used by the kernels
  float* d_adam_m = nullptr;
  float* d_adam_v = nullptr;
  float* d_grad = nullptr;
  float* d_loss = nullptr;
  int64_t adam_t = 0;
  float* d_ring = nullptr;           // 4 x n_free history of solutions (FP32)
  long long* d_stepcount = nullptr;  // steps since the history was reset
  double* d_sh = nullptr;            // RMS of h1 (scale of the features)
  int* d_mlp_used = nullptr;         // per stage: 1 if the network's guess was kept
  float* d_store = nullptr;          // recorded solutions (capacity x n_free)
  float* d_store_e = nullptr;        // recorded distances z - x0 from the SPE starts (capacity x n_free)
  bool store_e_valid = false;        // every recorded step ran with SPE start vectors
  double* d_x0 = nullptr;            // SPE start of the current solve (learned correction, recording)
  double* d_alpha = nullptr;         // step along the learned direction
  float* d_store_rms_e = nullptr;    // per recorded solve: RMS(z - x0) (training target scale)
  float* d_store_rms = nullptr;
  int64_t store_cap = 0, recorded = 0;
  bool recording = false;
  double* d_rtmp = nullptr;          // residual of the fallback start vector
  double* d_spe_X = nullptr;         // SPE: last solutions (spe_max x n_free)
  double* d_spe_W = nullptr;         // SPE: W = M X of the stored solutions
  double* d_spe_G = nullptr;         // SPE: Gram matrix x_a . w_b by ring slot (6 x 6)
  double* d_spe_y = nullptr;         // SPE: projection coefficients
  double* d_spe_partials = nullptr;  // SPE: reduction slots
  double* d_pod_X = nullptr;         // POD: snapshots (pod_k x n_free)
  double* d_pod_W = nullptr;         // POD: W = M X
  double* d_pod_GE = nullptr;        // POD: X^T X by slot (16 x 16)
  double* d_pod_GM = nullptr;        // POD: X^T M X by slot
  double* d_pod_a = nullptr;         // POD: projection coefficients by slot
  double* d_pod_partials = nullptr;  // POD: reduction slots
  void* d_pod_state = nullptr;       // POD: snapshot count, kept modes, reduced factor
  bool mlp_ready = false;
  bool direct = false;               // enqueue_step launches directly (host-driven CG loop)

  // ---- split coarse inverse (mixed precision): inv = hi + lo, FP32 parts
  float* d_cinv_hi = nullptr;
  float* d_cinv_lo = nullptr;
  float* d_cinv32 = nullptr;  // FP32 inverse, rows padded to cinv_ld floats
  double* d_dpart = nullptr;  // deferred CG sums (3 x red.max_blocks)
  int cinv_ld = 0;

  // ---- ensemble of 4 trajectories (allocated by the first ensemble call;
  // every vector row-interleaved, 4 columns per row)
  bool ens_ready = false;
  struct EnsLevel {
    float4 *b = nullptr, *x = nullptr, *r = nullptr, *dA = nullptr, *dB = nullptr;
  };
  std::vector<EnsLevel> elev;
  double4_32a* d_eY[4] = {nullptr, nullptr, nullptr, nullptr};  // Y0 + 3 rotating (n_nodes)
  float4* d_eY2 = nullptr;           // (hi, lo) FP32 pairs of the current stage (2 per node)
  double4_32a* d_eF[3] = {nullptr, nullptr, nullptr};  // stage solutions (n_free)
  double4_32a* d_eR = nullptr;       // stage right-hand sides
  float4* d_ey32 = nullptr;          // FP32 accumulation of K(x)x (n_nodes)
  double4_32a *d_er = nullptr, *d_ep = nullptr, *d_eq = nullptr;
  double4_32a* d_esol = nullptr;     // eqs_ens_solve_M work solution
  float4* d_ez32 = nullptr;          // FP32 preconditioned residual
  void* d_esc = nullptr;             // per-column CG scalars
  double* d_epart = nullptr;         // reduction slots (8 per block)
  int* d_eiters = nullptr;           // per stage and column: CG iterations
  double* d_erelres = nullptr;       // per stage and column: final relative residual
  int* d_ezero = nullptr;            // per stage and column: zero right-hand side
  double* d_ecolv = nullptr;         // drive scale of each column
  double4_32a* d_eX = nullptr;       // SPE history of the four columns (row-interleaved rings)
  double4_32a* d_eW = nullptr;       // W = M X
  float4* d_eX2 = nullptr;           // the rings X as FP32 pairs (two float4 per row; Gram pass)
  float4* d_eR2 = nullptr;           // the stage right-hand side as FP32 pairs (Gram pass)
  float2* d_M_rs = nullptr;          // row sums of the split M (FP32 pairs; difference-form products)
  double* d_eG = nullptr;            // per-column Gram matrices (4 x 6 x 6)
  double* d_ecoef = nullptr;         // per-column coefficients (+ slots in use)
  double* d_espart = nullptr;        // reduction slots of the ensemble Gram pass
  long long* d_estepcount = nullptr; // ensemble step counter (history index)
  int64_t ens_body_kernels = 0;
  std::map<int, eqs::GraphEntry> ens_graphs;   // key: s (graph), -s (host-loop entry)
  const eqs::GraphEntry* ens_last = nullptr;
  float4* d_ktime = nullptr;  // private K(x)x target of eqs_launch_kernel and eqs_ens_apply_K (n_nodes float4)
  float4* d_ekx2 = nullptr;   // eqs_ens_apply_K: the four input columns as FP32 pairs (2 n_nodes float4)
  eqs::GraphEntry ens_solve_graph;   // eqs_ens_solve_M (rtol of the setup)
  double ens_solve_tol = -1.0;

  // ---- adaptive stepping: F(t, x) evaluation graphs (key: x) and scratch
  eqs::GraphEntry eval_graph;  // F(t, x) of the adaptive step (x through d_params)
  double* d_xsave = nullptr;         // x(t_n) of the step being tried (n_nodes, mesh order)
  double* d_Fnew = nullptr;          // F(t_n+1, x_n+1) (n_free, internal order)
  double* d_err = nullptr;           // error norm of the last try
  long long* d_evalcount = nullptr;  // dummy history counter of the evaluations
  double* d_cj0 = nullptr;           // {0}: stage abscissa of an evaluation

  std::map<int, eqs::GraphEntry> step_graphs;  // key: s (graph), -s (host-loop entry)
  const eqs::GraphEntry* last_step = nullptr;                       // graph of the last step
  int64_t body_kernels = 0;  // kernel nodes of the last captured CG loop body
  std::map<double, eqs::GraphEntry> solve_graphs;                   // key: rtol
};

namespace eqs {

// host_setup.cpp
eqs_status validate_and_orient(eqs_ctx* c);
void build_internal_numbering(eqs_ctx* c);
void assemble_M(const eqs_ctx* c, HostCSR& Mff, std::vector<double>& mtop);
void build_hierarchy(const HostCSR& A, const eqs_opts& o, std::vector<HostLevel>& lev);
bool dense_spd_inverse(const HostCSR& A, std::vector<double>& inv);
void rkc_coefficients(int s, std::vector<double>& mu, std::vector<double>& nu,
                      std::vector<double>& mut, std::vector<double>& gt, std::vector<double>& c,
                      double& beta);
double rho_bound(const std::vector<eqs_material>& mats);

}  // namespace eqs
