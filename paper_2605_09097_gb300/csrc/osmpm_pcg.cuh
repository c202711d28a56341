// Persistent Jacobi-preconditioned CG for the Newton system
// (M/dt^2 + K) delta = -g of Sec. 2.2.5, one cooperative launch per solve,
// in the Chronopoulos-Gear arrangement: one fused reduction, hence one grid
// barrier, per iteration.  With u = D^-1 r and w = A u:
//   gamma = r.u, delta = u.w, beta = gamma/gamma_old,
//   alpha = gamma / (delta - beta gamma / alpha_old),
//   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s.
// Phase k (after barrier k) does the owner updates above and, in the same
// phase, the particle Hessian-vector product w_{k+1} = A u_{k+1}: each
// particle gathers u_{k+1} at its stencil as (r_k - alpha (w_k + beta
// s_{k-1})) D^-1 from buffers that were complete at barrier k (r and s
// double-buffered, w triple-buffered), and delta_{k+1} = u.Au is the
// particle quadratic form sum_p G:LG plus sum m/dt^2 u^2, so it does not
// wait for the scatter.  Every block sums the partials itself, in block
// order, so all blocks take the same branch and the result is
// deterministic.  Arrays that other blocks write during the launch are
// read with __ldcg (L2, not the non-coherent L1).
#pragma once

#include "osmpm_device.cuh"

namespace osmpm {

constexpr unsigned long long kBarrierSpinLimit = 1ull << 22;

// Grid barrier over `expected` co-resident blocks on a monotonic counter:
// each block adds 1 with release semantics and waits (acquire loads) until
// the counter reaches its running target, which grows by `expected` per
// barrier (kept per block in *target).  One round trip to L2 per barrier;
// the spin gives up after kBarrierSpinLimit polls (about a second) and
// reports kErrBarrierTimeout.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* target, int* err,
                                             unsigned expected) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned goal = *target + expected;
    *target = goal;
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
    unsigned long long spins = 0;
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if ((int)(v - goal) >= 0) break;
      if (++spins > kBarrierSpinLimit) {
        atomicOr(err, kErrBarrierTimeout);
        ok = 0;
        break;
      }
    }
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
template <int D, typename R>
__global__ void k_barrier_timeout_check(unsigned* words, int* err) {
  __shared__ unsigned goal;
  if (threadIdx.x == 0) goal = 0u;
  grid_barrier(&words[0], &goal, err, gridDim.x + 1);
}

// Flat offset of stencil node k (x fastest) from the base node.
template <int D>
__device__ __forceinline__ int64_t stencil_offset(const GridGeo& g, int k) {
  const int64_t ox = k % 3, oy = (k / 3) % 3, oz = k / 9;
  return D == 2 ? ox + oy * g.res[0] : ox + (oy + oz * g.res[1]) * (int64_t)g.res[0];
}

// Particle Hessian-vector product in arithmetic type R: gathers u at the
// stencil through `ufun(j)` (j = flat DOF index), scatters (L G) grad N_i
// into w on the free DOFs and returns the quadratic form G : L G.
template <int D, typename R, class UF>
__device__ __forceinline__ double particle_hvp(const PcgArgsT<R>& a, int64_t pi, UF ufun, double* w) {
  constexpr int DD = D * D;
  constexpr int K = (D == 2) ? 9 : 27;
  const GridGeo& g = a.g;
  const int64_t base = a.sbase[pi];
  R dN[K][D];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < D; ++c) dN[k][c] = a.sdn[(int64_t)(c * K + k) * a.P.n + pi];
  R G[DD];
#pragma unroll
  for (int e = 0; e < DD; ++e) G[e] = R(0);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t node = base + stencil_offset<D>(g, k);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const R uv = (R)ufun(c * g.nn + node);
#pragma unroll
      for (int b = 0; b < D; ++b) G[c * D + b] += uv * dN[k][b];
    }
  }
  R Y[DD];
#pragma unroll
  for (int i = 0; i < DD; ++i) {
    R t = R(0);
#pragma unroll
    for (int j = 0; j < DD; ++j) t += a.L[(int64_t)Sym<D>::idx(i, j) * a.P.n + pi] * G[j];
    Y[i] = t;
  }
  double qf = 0.0;
#pragma unroll
  for (int i = 0; i < DD; ++i) qf += (double)G[i] * (double)Y[i];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t node = base + stencil_offset<D>(g, k);
    const unsigned fm = a.dofmask[node];
    if (!fm) continue;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (!((fm >> c) & 1u)) continue;
      R f = R(0);
#pragma unroll
      for (int b = 0; b < D; ++b) f += Y[c * D + b] * dN[k][b];
      atomicAdd(&w[c * g.nn + node], (double)f);
    }
  }
  return qf;
}

template <int D, typename R>
__global__ void __launch_bounds__(kThreads) k_pcg(PcgArgsT<R> a) {
  const GridGeo& g = a.g;
  const int64_t ndof = g.nn * D;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  DevScalars* S = a.S;
  const int max_it = S->cg_max;
  const double tol2 = S->tol2;
  const double* idiag = a.diag;  // inverse Jacobi diagonal
  __shared__ unsigned bar_target;  // this block's running barrier goal (count starts at 0)
  if (threadIdx.x == 0) bar_target = 0u;
  int it = 0, neg = 0;
  double sums[3];

  // ---- phase 0: w_0 = A u_0, gamma_0 = r0.u0, delta_0 = u0.w0
  {
    double acc[3] = {0.0, 0.0, 0.0};
    const double* r0 = a.r[0];
    for (int64_t idx = tid; idx < ndof; idx += stride) {
      const int c = (int)(idx / g.nn);
      const int64_t i = idx - (int64_t)c * g.nn;
      if ((a.dofmask[i] >> c) & 1u) {
        const double ri = r0[idx];
        const double ui = ri * idiag[idx];
        acc[0] += ri * ui;
        acc[2] += a.m[i] * a.inv_dt2 * ui * ui;
        atomicAdd(&a.w[0][idx], a.m[i] * a.inv_dt2 * ui);
      }
    }
    for (int64_t pi = tid; pi < a.P.n; pi += stride)
      acc[2] += particle_hvp<D, R>(a, pi, [&](int64_t j) { return __ldcg(&r0[j]) * idiag[j]; }, a.w[0]);
    publish_partials<3>(acc, a.partials, 0);
    if (!grid_barrier(&S->bar_count, &bar_target, a.err, gridDim.x)) return;
    sum_partials<3>(a.partials, sums);
  }
  double gamma = sums[0], delta = sums[2];
  double alpha_old = 1.0, gamma_old = 1.0;
  int done = (gamma == 0.0) || (S->cg_done != 0);
  for (; it < max_it && !done; ++it) {
    double beta, alpha;
    if (it == 0) {
      beta = 0.0;
      if (!(delta > 0.0)) {
        neg = 1;
        break;
      }
      alpha = gamma / delta;
    } else {
      beta = gamma / gamma_old;
      const double den = delta - beta * gamma / alpha_old;
      if (!(den > 0.0)) {
        neg = 1;
        break;
      }
      alpha = gamma / den;
    }
    const double* rk = a.r[it & 1];
    double* rn = a.r[(it + 1) & 1];
    double* sk = a.s[it & 1];
    const double* sp = a.s[(it + 1) & 1];
    const double* wk = a.w[it % 3];
    double* wn = a.w[(it + 1) % 3];
    double* wz = a.w[(it + 2) % 3];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t idx = tid; idx < ndof; idx += stride) {
      const int c = (int)(idx / g.nn);
      const int64_t i = idx - (int64_t)c * g.nn;
      if ((a.dofmask[i] >> c) & 1u) {
        const double id = idiag[idx];
        const double rki = __ldcg(&rk[idx]);
        const double ski = __ldcg(&wk[idx]) + beta * __ldcg(&sp[idx]);
        sk[idx] = ski;
        const double pk = rki * id + beta * a.p[idx];
        a.p[idx] = pk;
        a.x[idx] += alpha * pk;
        const double rni = rki - alpha * ski;
        rn[idx] = rni;
        const double ui = rni * id;
        acc[0] += rni * ui;
        acc[1] += rni * rni;
        const double md = a.m[i] * a.inv_dt2;
        acc[2] += md * ui * ui;
        atomicAdd(&wn[idx], md * ui);
      }
      wz[idx] = 0.0;
    }
    for (int64_t pi = tid; pi < a.P.n; pi += stride)
      acc[2] += particle_hvp<D, R>(
          a, pi,
          [&](int64_t j) {
            return (__ldcg(&rk[j]) - alpha * (__ldcg(&wk[j]) + beta * __ldcg(&sp[j]))) * idiag[j];
          },
          wn);
    publish_partials<3>(acc, a.partials, 0);
    if (!grid_barrier(&S->bar_count, &bar_target, a.err, gridDim.x)) return;
    sum_partials<3>(a.partials, sums);
    gamma_old = gamma;
    alpha_old = alpha;
    gamma = sums[0];
    delta = sums[2];
    if (sums[1] <= tol2) {
      done = 1;
      ++it;
      break;
    }
  }
  if (neg && it == 0) {
    // no direction yet: take the preconditioned steepest descent u_0
    const double* r0 = a.r[0];
    for (int64_t idx = tid; idx < ndof; idx += stride) {
      const int c = (int)(idx / g.nn);
      const int64_t i = idx - (int64_t)c * g.nn;
      if ((a.dofmask[i] >> c) & 1u) a.x[idx] = r0[idx] * idiag[idx];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->cg_iter = it;
    S->cg_done = 1;
    S->cg_neg = neg;
    S->rz = gamma;
  }
}

}  // namespace osmpm
