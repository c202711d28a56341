// Batched streaming PCG over many domains in mixed precision (a service for
// many independent instances, not a passage of the paper): the Jacobi PCG
// of the streaming kernels, with the tiled Hessian-vector product of
// k_cgs_hvp_tile, run for a set of independent Newton systems at once.  A
// work list of tiles, (instance, item range) over particles or over DOFs
// and grouped by instance, is dealt to the blocks of each launch (fixed
// grids, grid stride; the kernels read the work list from a device
// argument block, so a captured graph serves every work list); every
// instance keeps its own scalars (its domain's DevScalars) and stops on its
// own.  Per-instance sums use the
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
  if (nt == 1) {
    // the instance's only tile: its block sum is the total (no partials,
    // fence or arrival count)
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) tsh[k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = tsh[k];
    __syncthreads();  // tsh is reused by the next call
    return true;
  }
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

// The batched solver is the Jacobi PCG in Chronopoulos-Gear form: one
// Hessian-vector product and one vector update per iteration, each ending
// in one per-instance reduction (the standard form needs a third kernel and
// reduction for the search direction).  With u = D^-1 r and w = A u:
//   gamma = r.u, delta = u.Au;  beta = gamma / gamma_prev,
//   alpha = gamma / (delta - beta gamma / alpha_prev)  (beta = 0 at first);
//   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s,
// the same iterates as the standard form in exact arithmetic.  Vectors:
// r = a.r[0], u = a.r[1], p = a.s[0], s = a.s[1], w = a.w[0] (K u, the mass
// part M/dt^2 u added where w is used).

// Start: w = 0, p = s = 0, the mass part of u.Au (r, u = D^-1 r, gamma =
// r.u and x = 0 come from each instance's gradient kernel).
template <int D>
__global__ void __launch_bounds__(kThreads) k_m_start(const MultiArgs* __restrict__ mp) {
  const MultiArgs m = *mp;
  for (int t = blockIdx.x; t < m.n_dt; t += gridDim.x) {
    const MultiTile T = m.dtl[t];
    if (!m.info[T.inst].fresh) continue;  // already iterating
    const PcgArgsT<float>& a = m.inst[T.inst];
    const int64_t nn = a.g.nn;
    double acc[1] = {0.0};
    int64_t idx = T.lo + threadIdx.x;
    int c = (int)(idx / nn);  // component and node of idx, then stepped
    int64_t i = idx - (int64_t)c * nn;
    for (; idx < T.hi; idx += blockDim.x) {
      a.w[0][idx] = 0.0;
      a.s[0][idx] = 0.0;
      a.s[1][idx] = 0.0;
      if ((a.dofmask[i] >> c) & 1u) {
        const double ui = a.r[1][idx];
        acc[0] += a.m[i] * a.inv_dt2 * ui * ui;
      }
      i += blockDim.x;
      while (i >= nn) {
        i -= nn;
        ++c;
      }
    }
    const MultiInfo in = m.info[T.inst];
    double tot[1];
    if (inst_sum<1>(acc, m.part, m.stride, t, in.dt0, in.ndt, &a.S->counter, tot) &&
        threadIdx.x == 0) {
      a.S->pq_diag = tot[0];
      a.S->cg_iter = 0;
      a.S->cg_neg = 0;
      a.S->neg0 = 0;
      if (a.S->cg_max <= 0) a.S->cg_done = 1;
    }
  }
}

// w = K u over the particle tiles of the running instances (the tiled
// product); the instance's last tile forms delta = u.Ku + u.Mu/dt^2 and
// the step's alpha and beta, or stops the instance on negative curvature.
template <int D>
__global__ void __launch_bounds__(TileCap<D>::THREADS, TileCap<D>::MIN_BLOCKS) k_m_hvp(const MultiArgs* __restrict__ mp) {
  const MultiArgs m = *mp;
  __shared__ HvpTileShared<D> sh;
  for (int t = blockIdx.x; t < m.n_pt; t += gridDim.x) {
    const MultiTile T = m.pt[t];
    const PcgArgsT<float>& a = m.inst[T.inst];
    DevScalars* S = a.S;
    if (__ldcg(&S->cg_done)) continue;  // the whole instance stopped (set by a last tile)
    // T.lo, T.hi: slots, one or more tiles of blockDim.x (a block works
    // through them with one sum for the item); each thread reads its slot
    // of the next tile before working on the current one
    float accf = 0.0f;
    auto slot_of = [&](int64_t s0) -> int64_t {
      const int64_t sl = s0 + threadIdx.x;
      return sl < T.hi ? (int64_t)a.slot2p[sl] : -1;
    };
    int64_t pi_next = slot_of(T.lo);
    for (int64_t s0 = T.lo; s0 < T.hi; s0 += blockDim.x) {
      const int64_t pi = pi_next;
      pi_next = slot_of(s0 + blockDim.x);
      hvp_tile<D>(a, a.r[1], pi, sh, accf);
    }
    double acc[1] = {(double)accf};
    const MultiInfo in = m.info[T.inst];
    double tot[1];
    if (inst_sum<1>(acc, m.part, m.stride, t, in.pt0, in.npt, &S->counter, tot) &&
        threadIdx.x == 0) {
      const double delta = tot[0] + S->pq_diag;
      const double gamma = S->rz;
      const int it = S->cg_iter;
      const double beta = it == 0 ? 0.0 : gamma / S->rz_prev;
      const double den = it == 0 ? delta : delta - beta * gamma / S->alpha_prev;
      if (!(den > 0.0)) {
        // negative curvature: stop (with no step yet, x = u_0 = D^-1 r_0)
        S->cg_neg = 1;
        S->cg_done = 1;
        S->neg0 = it == 0 ? 1 : 0;
      } else {
        S->alpha = gamma / den;
        S->beta = beta;
      }
    }
  }
}

// p = u + beta p, s = (w + M/dt^2 u) + beta s, x += alpha p, r -= alpha s,
// u = D^-1 r, w = 0; the instance's last tile takes gamma = r.u, r.r, the
// mass part of the next delta and the stopping tests.
template <int D>
__global__ void __launch_bounds__(kThreads) k_m_update(const MultiArgs* __restrict__ mp) {
  const MultiArgs m = *mp;
  for (int t = blockIdx.x; t < m.n_dt; t += gridDim.x) {
    const MultiTile T = m.dtl[t];
    const PcgArgsT<float>& a = m.inst[T.inst];
    DevScalars* S = a.S;
    const int64_t nn = a.g.nn;
    if (__ldcg(&S->cg_done)) {
      if (__ldcg(&S->neg0)) {
        // the instance stopped before its first step: x = u_0 (every tile
        // writes its DOFs; the flag is left for the next start to clear)
        for (int64_t idx = T.lo + threadIdx.x; idx < T.hi; idx += blockDim.x) {
          const int c = (int)(idx / nn);
          const int64_t i = idx - (int64_t)c * nn;
          if ((a.dofmask[i] >> c) & 1u) a.x[idx] = a.r[1][idx];
        }
      }
      continue;
    }
    const double alpha = __ldcg(&S->alpha), beta = __ldcg(&S->beta);
    const int it = __ldcg(&S->cg_iter);
    // the instance's vectors, distinct arrays (loads may pass the stores)
    const double* __restrict__ mass = a.m;
    const uint8_t* __restrict__ mask = a.dofmask;
    const double* __restrict__ dg = a.diag;
    double* __restrict__ w = a.w[0];
    double* __restrict__ u = a.r[1];
    double* __restrict__ r = a.r[0];
    double* __restrict__ p = a.s[0];
    double* __restrict__ sv = a.s[1];
    double* __restrict__ x = a.x;
    const double idt2 = a.inv_dt2;
    double acc[3] = {0.0, 0.0, 0.0};
    int64_t idx = T.lo + threadIdx.x;
    int c = (int)(idx / nn);  // component and node of idx, then stepped
    int64_t i = idx - (int64_t)c * nn;
    for (; idx < T.hi; idx += blockDim.x) {
      const double wi = w[idx];
      w[idx] = 0.0;
      if ((mask[i] >> c) & 1u) {
        const double mi = mass[i] * idt2;
        const double ui = u[idx];
        const double pi = ui + beta * p[idx];
        const double si = (wi + mi * ui) + beta * sv[idx];
        p[idx] = pi;
        sv[idx] = si;
        x[idx] += alpha * pi;
        const double ri = r[idx] - alpha * si;
        r[idx] = ri;
        const double un = ri * dg[idx];
        u[idx] = un;
        acc[0] += ri * un;
        acc[1] += ri * ri;
        acc[2] += mi * un * un;
      }
      i += blockDim.x;
      while (i >= nn) {
        i -= nn;
        ++c;
      }
    }
    const MultiInfo in = m.info[T.inst];
    double tot[3];
    if (inst_sum<3>(acc, m.part, m.stride, t, in.dt0, in.ndt, &S->counter, tot) &&
        threadIdx.x == 0) {
      const int itn = it + 1;
      S->cg_iter = itn;
      S->rz_prev = S->rz;
      S->alpha_prev = alpha;
      S->rz = tot[0];
      S->rr = tot[1];
      S->pq_diag = tot[2];
      if (tot[1] <= S->tol2 || itn >= S->cg_max) S->cg_done = 1;
    }
  }
}

// The number of systems still iterating into pending[0], every system's
// stop flag and iteration count into pending[1 + 2i], pending[2 + 2i] (one
// block).
template <int D>
__global__ void k_m_pending(const MultiArgs* __restrict__ mp) {
  const MultiArgs m = *mp;
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
