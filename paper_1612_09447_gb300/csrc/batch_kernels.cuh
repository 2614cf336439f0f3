// Batched RKC stages: many independent EQS instances advance together, one
// cooperative launch per stage.  Each instance owns a group of CTAs sized to
// its row count; the group runs the instance's stage (recurrence, element
// kernel, right-hand side, whole CG solve) with its own bounded group
// barrier, so instances of different sizes and iteration counts share the
// GPU without host round trips.  Mixed precision (FP32 element kernel and
// V-cycle, FP64 CG and recurrence).
#pragma once

#include "kernels.cuh"

namespace eqs {

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
};

__device__ __forceinline__ double* bY(const BatchInst& I, int j) { return j == 0 ? I.Y[0] : I.Y[1 + (j - 1) % 3]; }
__device__ __forceinline__ double* bF(const BatchInst& I, int j) { return j == 0 ? I.F[0] : I.F[1 + (j - 1) % 2]; }

__device__ __forceinline__ float2 split2d(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// g(t_j), g'(t_j) of every instance at the stage times t + c_j dt.
__global__ void k_batch_drive(int ninst, int s1, const BatchInst* __restrict__ insts,
                              const double* __restrict__ cj, const StepParams* prm, double* gtab,
                              double* gptab) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ninst * s1) return;
  const int b = k / s1, j = k % s1;
  const BatchInst& I = insts[b];
  const double a = I.w * (prm->t + cj[j] * prm->dt) + I.phase;
  gtab[k] = I.V0 * sin(a);
  gptab[k] = I.V0 * I.w * cos(a);
}

__device__ __forceinline__ GridCtx batch_group(const BatchInst* insts, const int* blk2inst,
                                               const int* first, const int* nblk, int& b) {
  b = blk2inst[blockIdx.x];
  GridCtx g;
  g.rank = blockIdx.x - first[b];
  g.nblocks = nblk[b];
  g.tid = (int64_t)g.rank * blockDim.x + threadIdx.x;
  g.stride = (int64_t)g.nblocks * blockDim.x;
  g.bar = insts[b].bar;
  g.partials = insts[b].partials;
  g.max_spins = kMaxSpins;
  return g;
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
    double* const* __restrict__ xmesh, double tol2) {
  int b;
  const GridCtx g = batch_group(insts, blk2inst, first, nblk, b);
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
  pcg_group_solve(*I.plan, g, I.R, bF(I, j), tol2, I.iters + j, I.relres + j, I.zero + j);
}

// Last recurrence Y_s and x(t + dt) in mesh order (no barrier needed).
__global__ void k_batch_final(const BatchInst* __restrict__ insts, const int* __restrict__ blk2inst,
                              const int* __restrict__ first, const int* __restrict__ nblk, int s, double c0,
                              double mu, double nu, double mut, double gt, const StepParams* prm,
                              const double* __restrict__ gtab, double* const* __restrict__ xmesh) {
  int b;
  const GridCtx g = batch_group(insts, blk2inst, first, nblk, b);
  const BatchInst& I = insts[b];
  batch_stage_vector(I, g, s, s, c0, mu, nu, mut, gt, prm->dt, gtab[b * (s + 1) + s], xmesh[b], xmesh[b]);
}

}  // namespace eqs
