// Batched RKC stages: many independent EQS instances advance together, one
// cooperative launch per stage.  Each instance owns a group of CTAs sized to
// its row count; the group runs the instance's stage (recurrence, element
// kernel, right-hand side, whole CG solve) with its own bounded group
// barrier, so instances of different sizes and iteration counts share the
// GPU without host round trips.  Mixed precision (FP32 element kernel and
// V-cycle, FP64 CG and recurrence).
#pragma once

#include "kernels.cuh"
#include "spe_kernels.cuh"

namespace eqs {

constexpr int kBatchSpe = 6;  // SPE history of a batched instance (2 x 6 sums in the group's 16 slots)

struct BatchInst {
  const PPlan<float>* plan;
  GridBarrier* bar;
  double* partials;
  int n, nf;
  int64_t nt;
  const int4* conn;
  const uint8_t* mat;
  const MaterialDev* mats;
  const float4* xh;
  const float4* xl;
  const int32_t* node_of_internal;
  const double* dir_scale;
  const double* mtop;
  double* Y[4];
  float2* Y32;
  double* F[3];
  double* R;
  float* y32;
  int* iters;
  double* relres;
  int* zero;
  double V0, w, phase;
  // SPE start vectors (Sec. IV, Eq. 4-5; null X: previous solution): the
  // instance context's solution ring, Gram matrix and coefficients
  double* X;
  double* G;
  double* coef;
};

__device__ __forceinline__ double* bY(const BatchInst& I, int j) { return j == 0 ? I.Y[0] : I.Y[1 + (j - 1) % 3]; }
__device__ __forceinline__ double* bF(const BatchInst& I, int j) { return j == 0 ? I.F[0] : I.F[1 + (j - 1) % 2]; }

__device__ __forceinline__ float2 split2d(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// g(t_j), g'(t_j) of every instance at the stage times t + c_j dt; the
// solve counter (count[0]: solves before this step, count[1]: after it).
__global__ void k_batch_drive(int ninst, int s1, const BatchInst* __restrict__ insts,
                              const double* __restrict__ cj, const StepParams* prm, double* gtab,
                              double* gptab, long long* count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    count[0] = count[1];
    count[1] += s1 - 1;
  }
  if (k >= ninst * s1) return;
  const int b = k / s1, j = k % s1;
  const BatchInst& I = insts[b];
  const double a = I.w * (prm->t + cj[j] * prm->dt) + I.phase;
  gtab[k] = I.V0 * sin(a);
  gptab[k] = I.V0 * I.w * cos(a);
}

__device__ __forceinline__ GridCtx batch_group(const BatchInst* insts, const int* blk2inst,
                                               const int* first, const int* nblk, long long max_spins, int& b) {
  b = blk2inst[blockIdx.x];
  GridCtx g;
  g.rank = blockIdx.x - first[b];
  g.nblocks = nblk[b];
  g.tid = (int64_t)g.rank * blockDim.x + threadIdx.x;
  g.stride = (int64_t)g.nblocks * blockDim.x;
  g.bar = insts[b].bar;
  g.partials = insts[b].partials;
  g.max_spins = max_spins;
  return g;
}

// SPE start of solve g of instance I inside its CTA group: the newest
// solution (in x, the solve's start buffer) enters ring slot g - 1, then
// w = M x_new, the Gram column x_k . w and the projections x_k . R are
// reduced over the group, one thread updates G and solves for the
// coefficients (spe_solve, as the single-instance pass), and every row gets
// x0 = X y.  False when a group barrier gave up.
__device__ bool batch_spe_start(const BatchInst& I, const GridCtx& g, long long gi, double* __restrict__ x) {
  constexpr int NH = kBatchSpe;
  const int nf = I.nf;
  const DevSell<double>& M = I.plan->M;
  if (gi == 0) return true;  // no history: the previous solution stays the start
  const int m = (int)(gi < NH ? gi : NH);
  const int sn = spe_slot(gi - 1, NH);
  double* __restrict__ xn = I.X + (size_t)sn * nf;
  for (int64_t i = g.tid; i < nf; i += g.stride) xn[i] = x[i];
  double v[2 * NH];
#pragma unroll
  for (int k = 0; k < 2 * NH; ++k) v[k] = 0.0;
  for (int64_t i = g.tid; i < nf; i += g.stride) {
    const double w = mat_row<double>(M, i, nf, x);
    const double bi = I.R[i];
#pragma unroll
    for (int k = 0; k < NH; ++k) {
      const double xk = k < m ? I.X[(size_t)spe_slot(gi - 1 - k, NH) * nf + i] : 0.0;
      v[k] = fma(xk, w, v[k]);
      v[NH + k] = fma(xk, bi, v[NH + k]);
    }
  }
  put_partials<2 * NH>(v, g.partials, 0, g.nblocks, g.rank);
  if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return false;
  __shared__ double stot[2 * NH];
  if (g.rank == 0) {
#pragma unroll
    for (int k = 0; k < 2 * NH; ++k) {
      const double t = get_total(g.partials, k, g.nblocks);
      if (threadIdx.x == 0) stot[k] = t;
    }
    if (threadIdx.x == 0) spe_solve<NH>(stot, gi, m, sn, I.G, 1e-12, I.coef);
  }
  if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return false;
  const int mu = reinterpret_cast<const int*>(I.coef + kSpeMax)[0];
  double y[NH];
#pragma unroll
  for (int k = 0; k < NH; ++k) y[k] = k < mu ? __ldcg(I.coef + spe_slot(gi - 1 - k, NH)) : 0.0;
  if (mu > 0)
    for (int64_t i = g.tid; i < nf; i += g.stride) {
      double xi = 0.0;
#pragma unroll
      for (int k = 0; k < NH; ++k)
        if (k < mu) xi = fma(y[k], I.X[(size_t)spe_slot(gi - 1 - k, NH) * nf + i], xi);
      x[i] = xi;
    }
  return grid_barrier(g.bar, g.nblocks, g.max_spins);
}

// Stage vector Y_j of instance I: gather (j = 0) or recurrence (j >= 1), the
// Dirichlet rows g(t_j), its two-float copy, and the start vector of solve j.
__device__ __forceinline__ void batch_stage_vector(const BatchInst& I, const GridCtx& g, int j, int s,
                                                   double c0, double mu, double nu, double mut, double gt,
                                                   double dt, double gj, const double* xmesh,
                                                   double* xout) {
  const int n = I.n, nf = I.nf;
  double* Yj = bY(I, j);
  for (int64_t i = g.tid; i < n; i += g.stride) {
    double v;
    if (i < nf) {
      if (j == 0) {
        v = xmesh[I.node_of_internal[i]];
        bF(I, 0)[i] = bF(I, s - 1)[i];
      } else {
        const double fj = I.zero[j - 1] ? 0.0 : bF(I, j - 1)[i];
        const double f0 = I.zero[0] ? 0.0 : bF(I, 0)[i];
        v = c0 * I.Y[0][i] + mu * bY(I, j - 1)[i] + nu * bY(I, j >= 2 ? j - 2 : 0)[i] + (mut * dt) * fj +
            (gt * dt) * f0;
        if (j < s) bF(I, j)[i] = bF(I, j - 1)[i];
      }
    } else {
      v = I.dir_scale[i - nf] * gj;
    }
    Yj[i] = v;
    if (j < s) I.Y32[i] = split2d(v);
    if (xout) xout[I.node_of_internal[i]] = v;
  }
}

// One stage j (0 <= j < s) of every instance.
__global__ void __launch_bounds__(kPBlock) k_batch_stage(
    const BatchInst* __restrict__ insts, const int* __restrict__ blk2inst, const int* __restrict__ first,
    const int* __restrict__ nblk, int j, int s, double c0, double mu, double nu, double mut, double gt,
    const StepParams* prm, const double* __restrict__ gtab, const double* __restrict__ gptab,
    double* const* __restrict__ xmesh, double tol2, const long long* __restrict__ count, long long max_spins) {
  int b;
  const GridCtx g = batch_group(insts, blk2inst, first, nblk, max_spins, b);
  const BatchInst& I = insts[b];
  const double gj = gtab[b * (s + 1) + j], gpj = gptab[b * (s + 1) + j];
  batch_stage_vector(I, g, j, s, c0, mu, nu, mut, gt, prm->dt, gj, xmesh[b], nullptr);
  if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return;
  for (int64_t e = g.tid; e < I.nt; e += g.stride)
    elem32_tet(e, I.conn, I.mat, I.mats, I.xh, I.xl, I.Y32, I.nf, I.y32);
  if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return;
  for (int64_t i = g.tid; i < I.nf; i += g.stride) {
    I.R[i] = -(double)I.y32[i] - gpj * I.mtop[i];
    I.y32[i] = 0.0f;
  }
  if (!grid_barrier(g.bar, g.nblocks, g.max_spins)) return;
  if (I.X && !batch_spe_start(I, g, count[0] + j, bF(I, j))) return;
  pcg_group_solve(*I.plan, g, I.R, bF(I, j), tol2, I.iters + j, I.relres + j, I.zero + j);
}

// Last recurrence Y_s and x(t + dt) in mesh order (no barrier needed).
__global__ void k_batch_final(const BatchInst* __restrict__ insts, const int* __restrict__ blk2inst,
                              const int* __restrict__ first, const int* __restrict__ nblk, int s, double c0,
                              double mu, double nu, double mut, double gt, const StepParams* prm,
                              const double* __restrict__ gtab, double* const* __restrict__ xmesh) {
  int b;
  const GridCtx g = batch_group(insts, blk2inst, first, nblk, kMaxSpins, b);
  const BatchInst& I = insts[b];
  batch_stage_vector(I, g, s, s, c0, mu, nu, mut, gt, prm->dt, gtab[b * (s + 1) + s], xmesh[b], xmesh[b]);
}

}  // namespace eqs
