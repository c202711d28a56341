// Persistent Jacobi-preconditioned CG for the Newton system
// (M/dt^2 + K) delta = -g of Sec. 2.2.5, one cooperative launch per solve.
//
// Each iteration has two phases separated by grid barriers:
//  1. p_new = z + beta p_old on the free DOFs owned by this thread (double-
//     buffered p), q += (m/dt^2) p_new, and the particle Hessian-vector
//     product: every particle gathers p at its stencil as z + beta p_old
//     (so no barrier is needed between the p update and the gather), forms
//     Y = L G and scatters Y grad N_i into q.  Partial sums of p.Hp.
//  2. alpha = r.z / p.Hp, x += alpha p, r -= alpha q, z = r/diag, q = 0;
//     partial sums of r.z and r.r.
// Every block sums the partials of the previous phase itself, in block
// order, so all blocks take the same branch and the result is
// deterministic.  Arrays that other blocks write during the launch are
// read with __ldcg (L2, not the non-coherent L1).
#pragma once

#include "osmpm_device.cuh"

namespace osmpm {

constexpr unsigned long long kBarrierSpinLimit = 1ull << 22;

// Sense-reversing grid barrier over `expected` (= gridDim.x) co-resident
// blocks.  The spin gives up after kBarrierSpinLimit polls (about two
// seconds) and reports kErrBarrierTimeout.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, int* err,
                                             unsigned expected) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g0 = *((volatile unsigned*)gen);
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u);
    if (arrived == expected - 1) {
      *((volatile unsigned*)count) = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned long long spins = 0;
      while (*((volatile unsigned*)gen) == g0) {
        if (++spins > kBarrierSpinLimit) {
          atomicOr(err, kErrBarrierTimeout);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Deterministic sum of NV partial rows (row k at partials[k*G .. k*G+G-1]),
// result in every thread.
template <int NV>
__device__ __forceinline__ void sum_partials(const double* partials, double (&out)[NV]) {
  __shared__ double tot[NV];
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(&partials[k * gridDim.x + b]);
  block_sum<NV>(acc);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = acc[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = tot[k];
  __syncthreads();
}

template <int NV>
__device__ __forceinline__ void publish_partials(double (&v)[NV], double* partials, int row0) {
  block_sum<NV>(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(row0 + k) * gridDim.x + blockIdx.x] = v[k];
}

// Diagnostic: a barrier that waits for one block more than the launch has,
// so its bounded spin can only run out.
template <int D>
__global__ void k_barrier_timeout_check(unsigned* words, int* err) {
  grid_barrier(&words[0], &words[1], err, gridDim.x + 1);
}

// Flat offset of stencil node k (x fastest) from the base node.
template <int D>
__device__ __forceinline__ int64_t stencil_offset(const GridGeo& g, int k) {
  const int64_t ox = k % 3, oy = (k / 3) % 3, oz = k / 9;
  return D == 2 ? ox + oy * g.res[0] : ox + (oy + oz * g.res[1]) * (int64_t)g.res[0];
}

template <int D>
__global__ void __launch_bounds__(kThreads) k_pcg(PcgArgs a) {
  constexpr int DD = D * D;
  constexpr int K = (D == 2) ? 9 : 27;
  const GridGeo& g = a.g;
  const int64_t ndof = g.nn * D;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  DevScalars* S = a.S;
  const int max_it = S->cg_max;
  const double tol2 = S->tol2;
  double rz = S->rz;
  int done = S->cg_done;
  int neg = 0;
  double beta = 0.0;
  int it = 0;
  for (; it < max_it && !done; ++it) {
    const double* pold = (it & 1) ? a.p1 : a.p0;
    double* pnew = (it & 1) ? a.p0 : a.p1;
    // ---- phase 1: p update, diagonal term, particle HVP
    double acc1[1] = {0.0};
    for (int64_t idx = tid; idx < ndof; idx += stride) {
      const int c = (int)(idx / g.nn);
      const int64_t i = idx - (int64_t)c * g.nn;
      if ((a.dofmask[i] >> c) & 1u) {
        const double pn = __ldcg(&a.z[idx]) + beta * __ldcg(&pold[idx]);
        pnew[idx] = pn;
        const double md = a.m[i] * a.inv_dt2;
        atomicAdd(&a.q[idx], md * pn);
        acc1[0] += md * pn * pn;
      }
    }
    for (int64_t pi = tid; pi < a.P.n; pi += stride) {
      const int64_t base = a.sbase[pi];
      double dN[K][D];
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int c = 0; c < D; ++c) dN[k][c] = a.sdn[(int64_t)(c * K + k) * a.P.n + pi];
      double G[DD];
#pragma unroll
      for (int e = 0; e < DD; ++e) G[e] = 0.0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int64_t node = base + stencil_offset<D>(g, k);
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const int64_t j = c * g.nn + node;
          const double pv = __ldcg(&a.z[j]) + beta * __ldcg(&pold[j]);
#pragma unroll
          for (int b = 0; b < D; ++b) G[c * D + b] += pv * dN[k][b];
        }
      }
      double Y[DD];
#pragma unroll
      for (int i = 0; i < DD; ++i) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < DD; ++j) t += a.L[(int64_t)Sym<D>::idx(i, j) * a.P.n + pi] * G[j];
        Y[i] = t;
      }
#pragma unroll
      for (int i = 0; i < DD; ++i) acc1[0] += G[i] * Y[i];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int64_t node = base + stencil_offset<D>(g, k);
        const unsigned fm = a.dofmask[node];
        if (!fm) continue;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          if (!((fm >> c) & 1u)) continue;
          double f = 0.0;
#pragma unroll
          for (int b = 0; b < D; ++b) f += Y[c * D + b] * dN[k][b];
          atomicAdd(&a.q[c * g.nn + node], f);
        }
      }
    }
    publish_partials<1>(acc1, a.partials, 0);
    if (!grid_barrier(&S->bar_count, &S->bar_gen, a.err, gridDim.x)) return;
    double pq[1];
    sum_partials<1>(a.partials, pq);
    if (!(pq[0] > 0.0)) {
      // negative curvature: keep the current iterate, or take the
      // preconditioned steepest-descent direction if there is none yet
      neg = 1;
      if (it == 0)
        for (int64_t idx = tid; idx < ndof; idx += stride) a.x[idx] = __ldcg(&pnew[idx]);
      break;
    }
    const double alpha = rz / pq[0];
    // ---- phase 2: updates
    double acc2[2] = {0.0, 0.0};
    for (int64_t idx = tid; idx < ndof; idx += stride) {
      const int c = (int)(idx / g.nn);
      const int64_t i = idx - (int64_t)c * g.nn;
      if ((a.dofmask[i] >> c) & 1u) {
        a.x[idx] += alpha * __ldcg(&pnew[idx]);
        const double ri = __ldcg(&a.r[idx]) - alpha * __ldcg(&a.q[idx]);
        a.r[idx] = ri;
        const double zi = ri / a.diag[idx];
        a.z[idx] = zi;
        acc2[0] += ri * zi;
        acc2[1] += ri * ri;
      }
      a.q[idx] = 0.0;
    }
    publish_partials<2>(acc2, a.partials, 1);
    if (!grid_barrier(&S->bar_count, &S->bar_gen, a.err, gridDim.x)) return;
    double rr[2];
    sum_partials<2>(a.partials + gridDim.x, rr);
    beta = rr[0] / rz;
    rz = rr[0];
    done = (rr[1] <= tol2) ? 1 : 0;
    if (done) {
      ++it;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->cg_iter = it;
    S->cg_done = 1;
    S->cg_neg = neg;
    S->rz = rz;
  }
}

}  // namespace osmpm
