// Batched streaming PCG over many domains in mixed precision (the batched
// growth line of the project, not a passage of the paper): the Jacobi PCG of
// k_cgs_start / k_cgs_hvp_tile / k_cgs_alpha / k_cgs_beta run for a set of
// independent Newton systems at once.  A work list of tiles, (instance,
// item range) over particles or over DOFs and grouped by instance, is dealt
// to the blocks of each launch; every instance keeps its own scalars (its
// domain's DevScalars) and stops on its own.  Per-instance sums use the
// instance's arrival counter: each tile stores its partial, and the last
// tile of an instance to arrive adds that instance's partials in tile order
// (so the sums do not depend on scheduling) and updates the scalars.
//
// Included by osmpm_kernels.cuh.
#pragma once

#include "osmpm_tile.cuh"

namespace osmpm {

// Per-instance sum of NV values over the instance's tiles: returns true in
// the block that arrived last, where tot holds the sums.
template <int NV>
__device__ __forceinline__ bool inst_sum(double (&v)[NV], double* part, int stride, int tile,
                                         int t0, int nt, unsigned* counter, double (&tot)[NV]) {
  __shared__ bool last;
  __shared__ double tsh[NV];
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[k * stride + tile] = v[k];
    __threadfence();
    last = atomicAdd(counter, 1u) == (unsigned)(nt - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int j = threadIdx.x; j < nt; j += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(&part[k * stride + t0 + j]);
  block_sum<NV>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) tsh[k] = acc[k];
    *counter = 0u;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = tsh[k];
  return true;
}

// Start: q = 0, the mass part of p.Ap (r, z = D^-1 r, p = z and x = 0 come
// from each instance's gradient kernel).
template <int D>
__global__ void __launch_bounds__(kThreads) k_m_start(MultiArgs m) {
  for (int t = blockIdx.x; t < m.n_dt; t += gridDim.x) {
    const MultiTile T = m.dtl[t];
    if (!m.info[T.inst].fresh) continue;  // already iterating
    const PcgArgsT<float>& a = m.inst[T.inst];
    const int64_t nn = a.g.nn;
    double acc[1] = {0.0};
    for (int64_t idx = T.lo + threadIdx.x; idx < T.hi; idx += blockDim.x) {
      const int c = (int)(idx / nn);
      const int64_t i = idx - (int64_t)c * nn;
      a.w[0][idx] = 0.0;
      if ((a.dofmask[i] >> c) & 1u) {
        const double pi = a.s[0][idx];
        acc[0] += a.m[i] * a.inv_dt2 * pi * pi;
      }
    }
    const MultiInfo in = m.info[T.inst];
    double tot[1];
    if (inst_sum<1>(acc, m.part, m.stride, t, in.dt0, in.ndt, &a.S->counter, tot) &&
        threadIdx.x == 0) {
      a.S->pq_diag = tot[0];
      a.S->cg_iter = 0;
      a.S->cg_neg = 0;
      if (a.S->cg_max <= 0) a.S->cg_done = 1;
    }
  }
}

// q = K p over the particle tiles of the running instances (the tiled
// product), p:Kp into pq.
template <int D>
__global__ void __launch_bounds__(TileCap<D>::THREADS, TileCap<D>::MIN_BLOCKS) k_m_hvp(MultiArgs m) {
  __shared__ HvpTileShared<D> sh;
  for (int t = blockIdx.x; t < m.n_pt; t += gridDim.x) {
    const MultiTile T = m.pt[t];
    const PcgArgsT<float>& a = m.inst[T.inst];
    if (__ldcg(&a.S->cg_done)) continue;  // the whole instance stopped (set by the alpha kernel)
    float accf = 0.0f;
    hvp_tile<D>(a, T.lo, T.hi, sh, accf);  // T.lo, T.hi: slots
    double acc[1] = {(double)accf};
    const MultiInfo in = m.info[T.inst];
    double tot[1];
    if (inst_sum<1>(acc, m.part, m.stride, t, in.pt0, in.npt, &a.S->counter, tot) &&
        threadIdx.x == 0)
      a.S->pq = tot[0];
  }
}

// alpha = r.z / p.Ap; x += alpha p; r -= alpha (q + M/dt^2 p); z = D^-1 r;
// the instance's last tile takes r.z, r.r, beta and the stopping tests.  On
// negative curvature the instance stops (with no direction yet, x = z_0).
template <int D>
__global__ void __launch_bounds__(kThreads) k_m_alpha(MultiArgs m) {
  for (int t = blockIdx.x; t < m.n_dt; t += gridDim.x) {
    const MultiTile T = m.dtl[t];
    const PcgArgsT<float>& a = m.inst[T.inst];
    DevScalars* S = a.S;
    if (__ldcg(&S->cg_done)) continue;
    const int64_t nn = a.g.nn;
    const double pAp = __ldcg(&S->pq) + __ldcg(&S->pq_diag);
    const double rz = __ldcg(&S->rz);
    const int it = __ldcg(&S->cg_iter);
    const bool neg = !(pAp > 0.0);
    const double alpha = neg ? 0.0 : rz / pAp;
    double acc[2] = {0.0, 0.0};
    for (int64_t idx = T.lo + threadIdx.x; idx < T.hi; idx += blockDim.x) {
      const int c = (int)(idx / nn);
      const int64_t i = idx - (int64_t)c * nn;
      if (!((a.dofmask[i] >> c) & 1u)) continue;
      const double pi = a.s[0][idx];
      if (neg) {
        if (it == 0) a.x[idx] = pi;
        continue;
      }
      a.x[idx] += alpha * pi;
      const double ap = a.w[0][idx] + a.m[i] * a.inv_dt2 * pi;
      const double ri = a.r[0][idx] - alpha * ap;
      a.r[0][idx] = ri;
      const double zi = ri * a.diag[idx];
      a.r[1][idx] = zi;
      acc[0] += ri * zi;
      acc[1] += ri * ri;
    }
    const MultiInfo in = m.info[T.inst];
    double tot[2];
    if (inst_sum<2>(acc, m.part, m.stride, t, in.dt0, in.ndt, &S->counter, tot) &&
        threadIdx.x == 0) {
      if (neg) {
        S->cg_neg = 1;
        S->cg_done = 1;
      } else {
        const int itn = it + 1;
        S->cg_iter = itn;
        S->beta = tot[0] / rz;
        S->rz = tot[0];
        S->rr = tot[1];
        if (tot[1] <= S->tol2 || itn >= S->cg_max) S->cg_done = 1;
      }
    }
  }
}

// p = z + beta p, q = 0, the mass part of the next p.Ap.
template <int D>
__global__ void __launch_bounds__(kThreads) k_m_beta(MultiArgs m) {
  for (int t = blockIdx.x; t < m.n_dt; t += gridDim.x) {
    const MultiTile T = m.dtl[t];
    const PcgArgsT<float>& a = m.inst[T.inst];
    DevScalars* S = a.S;
    if (__ldcg(&S->cg_done)) continue;
    const int64_t nn = a.g.nn;
    const double beta = __ldcg(&S->beta);
    double acc[1] = {0.0};
    for (int64_t idx = T.lo + threadIdx.x; idx < T.hi; idx += blockDim.x) {
      const int c = (int)(idx / nn);
      const int64_t i = idx - (int64_t)c * nn;
      a.w[0][idx] = 0.0;
      if ((a.dofmask[i] >> c) & 1u) {
        const double pi = a.r[1][idx] + beta * a.s[0][idx];
        a.s[0][idx] = pi;
        acc[0] += a.m[i] * a.inv_dt2 * pi * pi;
      }
    }
    const MultiInfo in = m.info[T.inst];
    double tot[1];
    if (inst_sum<1>(acc, m.part, m.stride, t, in.dt0, in.ndt, &S->counter, tot) &&
        threadIdx.x == 0)
      S->pq_diag = tot[0];
  }
}

// The number of systems still iterating into pending[0], every system's
// stop flag and iteration count into pending[1 + 2i], pending[2 + 2i] (one
// block).
template <int D>
__global__ void k_m_pending(MultiArgs m) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < m.n_inst; i += blockDim.x) {
    const DevScalars* S = m.inst[i].S;
    const int done = __ldcg(&S->cg_done);
    if (!done) atomicAdd(&cnt, 1);
    m.pending[1 + 2 * i] = done;
    m.pending[2 + 2 * i] = __ldcg(&S->cg_iter);
  }
  __syncthreads();
  if (threadIdx.x == 0) *m.pending = cnt;
}

}  // namespace osmpm
