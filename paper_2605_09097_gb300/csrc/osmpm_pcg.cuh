// Persistent Jacobi-preconditioned CG for the Newton system
// (M/dt^2 + K) delta = -g of Sec. 2.2.5, one cooperative launch per solve,
// in the Chronopoulos-Gear arrangement: one fused reduction, hence one grid
// barrier, per iteration.  With u = D^-1 r and w = A u:
//   gamma = r.u, delta = u.w, beta = gamma/gamma_old,
//   alpha = gamma / (delta - beta gamma / alpha_old),
//   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s.
// Phase k (after barrier k) does the owner updates above and, in the same
// phase, the particle Hessian-vector product w_{k+1} = A u_{k+1}: each
// particle (a group of lanes, one per stencil row) gathers u_{k+1} at its
// stencil as (r_k - alpha (w_k + beta s_{k-1})) D^-1 from buffers that were
// complete at barrier k (r and s double-buffered, w triple-buffered; the
// single-pass variant forms it once per node of a block-local table), and
// delta_{k+1} = u.Au is the particle quadratic form sum_p G:LG plus
// sum m/dt^2 u^2, so it does not wait for the scatter.  Every block sums
// the partials itself, in an order fixed by the launch shape, so all
// blocks take the same branch (the scatter's FP64 atomics still let the
// last bits of a solve vary between runs).  Arrays that other blocks write
// during the launch are read with __ldcg (L2, not the non-coherent L1).
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

// Particle Hessian-vector product in arithmetic type R, spread over a group
// of LPP lanes per particle: lane q owns the stencil row of nodes
// k = 3q .. 3q+2 (x fastest).  Each lane gathers u at its nodes through
// `ufun(f, j, c)` (f = flat DOF index of component c at the lane's node j)
// into a partial G = sum u grad N^T; the
// group sums the partials in lane order (every lane gets the same G), lane q
// forms the rows i = q, q + LPP, ... of Y = L G, the rows are broadcast, and
// each lane scatters (Y grad N_k) onto the free DOFs of its nodes.  Returns
// this lane's share of the quadratic form G : L G (its rows).  All lanes of
// the warp must call it together (it shuffles); lanes with valid = false
// take part without loading or writing.
template <int D>
struct HvpGroup {
  static constexpr int LPP = (D == 2) ? 3 : 9;  // lanes per particle (stencil rows)
  static constexpr int GP = 32 / LPP;           // particles per warp
};

// One lane's share of a particle: the nodes of its stencil row, their grad N
// and its rows i = q, q + LPP, ... of the particle's Hessian block L.
template <int D, typename R>
struct LaneData {
  static constexpr int DD = D * D;
  static constexpr int ROWS = (DD + HvpGroup<D>::LPP - 1) / HvpGroup<D>::LPP;
  int64_t node[3];
  R dN[3][D];
  R L[ROWS][DD];
};

template <int D, typename R>
__device__ __forceinline__ void load_lane(const PcgArgsT<R>& a, int64_t pi, bool valid, int q,
                                          LaneData<D, R>& ld) {
  constexpr int DD = D * D;
  constexpr int K = (D == 2) ? 9 : 27;
  constexpr int LPP = HvpGroup<D>::LPP;
  if (!valid) return;
  const int64_t base = a.sbase[pi];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int k = 3 * q + j;
    ld.node[j] = base + stencil_offset<D>(a.g, k);
#pragma unroll
    for (int c = 0; c < D; ++c) ld.dN[j][c] = a.sdn[(int64_t)(c * K + k) * a.P.n + pi];
  }
#pragma unroll
  for (int r = 0; r < LaneData<D, R>::ROWS; ++r) {
    const int i = q + r * LPP;
#pragma unroll
    for (int j = 0; j < DD; ++j)
      ld.L[r][j] = i < DD ? a.L[(int64_t)Sym<D>::idx(i, j) * a.P.n + pi] : R(0);
  }
}

template <int D, typename R, class UF>
__device__ __forceinline__ double group_hvp_lane(const PcgArgsT<R>& a, const LaneData<D, R>& ld,
                                                 bool valid, int q, int leader, UF ufun, double* w) {
  constexpr int DD = D * D;
  constexpr int LPP = HvpGroup<D>::LPP;
  const GridGeo& g = a.g;
  R G[DD];
#pragma unroll
  for (int e = 0; e < DD; ++e) G[e] = R(0);
  if (valid) {
    R uv[3][D];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c) uv[j][c] = (R)ufun(c * g.nn + ld.node[j], j, c);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int b = 0; b < D; ++b) G[c * D + b] += uv[j][c] * ld.dN[j][b];
  }
  // the group's G, summed in lane order
#pragma unroll
  for (int e = 0; e < DD; ++e) {
    R t = __shfl_sync(kFull, G[e], leader);
#pragma unroll
    for (int l = 1; l < LPP; ++l) t += __shfl_sync(kFull, G[e], leader + l);
    G[e] = t;
  }
  // this lane's rows of Y = L G, then every row from its owner lane
  R Ymine[DD];
  double qf = 0.0;
#pragma unroll
  for (int i = 0; i < DD; ++i) Ymine[i] = R(0);
  if (valid) {
#pragma unroll
    for (int r = 0; r < LaneData<D, R>::ROWS; ++r) {
      const int i = q + r * LPP;
      if (i < DD) {
        R t = R(0);
#pragma unroll
        for (int j = 0; j < DD; ++j) t += ld.L[r][j] * G[j];
        // i depends on the lane: select with static indices (keeps G and
        // Ymine in registers)
        R Gi = R(0);
#pragma unroll
        for (int ii = 0; ii < DD; ++ii)
          if (ii == i) {
            Gi = G[ii];
            Ymine[ii] = t;
          }
        qf += (double)Gi * (double)t;
      }
    }
  }
  R Y[DD];
#pragma unroll
  for (int i = 0; i < DD; ++i) Y[i] = __shfl_sync(kFull, Ymine[i], leader + i % LPP);
  if (valid) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const unsigned fm = a.dofmask[ld.node[j]];
      if (!fm) continue;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        if (!((fm >> c) & 1u)) continue;
        R f = R(0);
#pragma unroll
        for (int b = 0; b < D; ++b) f += Y[c * D + b] * ld.dN[j][b];
        atomicAdd(&w[c * g.nn + ld.node[j]], (double)f);
      }
    }
  }
  return qf;
}

template <int D, typename R, class UF>
__device__ __forceinline__ double group_hvp(const PcgArgsT<R>& a, int64_t pi, bool valid, int q,
                                            int leader, UF ufun, double* w) {
  LaneData<D, R> ld;
  load_lane<D, R>(a, pi, valid, q, ld);
  return group_hvp_lane<D, R>(a, ld, valid, q, leader, ufun, w);
}

// FP64 instructions are scarce on this part (one warp-wide FP64 instruction
// per SMSP every ~64 clocks), and every FP64 instruction on the serial path
// between two grid barriers costs that much latency.  So the per-iteration
// control avoids redundant and serial FP64 work: the block sums and the
// grid totals of the three recurrence values run on three warps at once
// (different SMSPs), thread 0 evaluates beta and the stopping tests while
// thread 32 evaluates alpha, both handing them to the block through shared
// memory (the launch has at least 64 threads), and the DOFs are dealt to
// the blocks in equal contiguous chunks.

// This block's sums of NV values per thread, stored as its partials
// (partials[k * gridDim.x + blockIdx.x]): the threads park their values in
// shared memory, then warp k alone sums value k (lane-strided over the
// threads, then a warp shuffle).  The order depends only on the block size.
template <int NV>
__device__ __forceinline__ void pcg_block_partials(const double (&v)[NV], double* partials) {
  __shared__ double sh[NV][kThreads];
#pragma unroll
  for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  for (int k = warp; k < NV; k += nw) {
    double t = 0.0;
    for (unsigned j = lane; j < blockDim.x; j += 32) t += sh[k][j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(kFull, t, off);
    if (lane == 0) partials[k * gridDim.x + blockIdx.x] = t;
  }
}

// The NV totals of the grid's partial rows into tot[] (shared): warp k forms
// total k, lane-strided over the blocks, then a warp shuffle (the order
// depends only on the launch shape).  The caller synchronises the block
// before reading tot.
template <int NV>
__device__ __forceinline__ void pcg_grid_totals(const double* partials, double* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  for (int k = warp; k < NV; k += nw) {
    double t = 0.0;
    for (unsigned b = lane; b < gridDim.x; b += 32) t += __ldcg(&partials[k * gridDim.x + b]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(kFull, t, off);
    if (lane == 0) tot[k] = t;
  }
}

// Block-local node table of the single-pass variant: the distinct nodes of
// the block's particle stencils (open addressing on the node index, bounded
// probes).  Each iteration then forms u_{k+1} once per table node into
// shared memory and the gathers read it there, instead of every (particle,
// stencil node) pair forming it again from three L2 loads (a node sits in
// the stencils of ~9 x particles-per-cell particles).  A block whose nodes do
// not fit keeps the L2 gather.
constexpr int kLocNodes = 512;  // table slots, a power of two; local ids < 1024

struct LocTable {
  unsigned long long key[kLocNodes];  // node index, or kLocEmpty
  int id[kLocNodes];                  // dense local id of the slot's node
  long long node[kLocNodes];          // dense local id -> node index
  int count, over;
};
constexpr unsigned long long kLocEmpty = ~0ull;

__device__ __forceinline__ unsigned loc_hash(unsigned long long key) {
  return (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 55) & (kLocNodes - 1);
}

// ONE: the launch covers the problem in a single pass (every thread owns at
// most one DOF, every lane at most one particle); then each lane keeps its
// particle's stencil, grad N and Hessian rows in registers for the whole
// solve, and each DOF owner its inverse diagonal, m/dt^2, p and x, so an
// iteration reads only r, s and w.
template <int D, typename R, bool ONE>
__global__ void __launch_bounds__(kThreads) k_pcg(PcgArgsT<R> a) {
  const GridGeo& g = a.g;
  const int64_t ndof = g.nn * D;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  DevScalars* S = a.S;
  const double* idiag = a.diag;  // inverse Jacobi diagonal
  __shared__ unsigned bar_target;  // this block's running barrier goal (count starts at 0)
  __shared__ double sh_alpha, sh_beta;
  __shared__ int sh_stop;          // tolerance or iteration cap reached
  __shared__ int sh_neg;           // the curvature test failed
  __shared__ double sh_tot[3];     // the grid totals after a barrier
  if (threadIdx.x == 0) bar_target = 0u;
  // DOFs: block b owns the contiguous chunk [b c, (b+1) c)
  const int64_t chunk = (ndof + gridDim.x - 1) / gridDim.x;
  const int64_t d_lo = (int64_t)blockIdx.x * chunk;
  const int64_t d_hi = d_lo + chunk < ndof ? d_lo + chunk : ndof;
  // particle work: groups of LPP lanes, GP particles per warp (blockDim is a
  // multiple of 32); the loops over particles run warp-uniformly
  constexpr int LPP = HvpGroup<D>::LPP, GP = HvpGroup<D>::GP;
  const int lane = threadIdx.x & 31;
  const int grp = lane / LPP;
  const int q = lane - grp * LPP;
  const int leader = grp * LPP;
  const bool in_group = grp < GP;
  const int64_t warp0 = (tid >> 5) * GP;
  const int64_t wstride = (stride >> 5) * GP;
  // single-pass residents
  const int64_t my_idx = d_lo + threadIdx.x;
  bool my_free = false;
  double my_id = 0.0, my_md = 0.0, my_p = 0.0, my_x = 0.0;
  const int64_t my_pi = warp0 + grp;
  const bool my_valid = in_group && my_pi < a.P.n;
  LaneData<D, R> ld;
  __shared__ LocTable loc;
  __shared__ double loc_u[D * kLocNodes];  // u at the table's nodes, component-major
  bool loc_ok = false;
  unsigned my_slots = 0u;  // local ids of the lane's 3 nodes, 10 bits each
  // u for the gathers: from the table when the block has one, else from L2
  auto loc_gather = [&](auto ufun) {
    return [&, ufun](int64_t f, int j, int c) {
      return loc_ok ? loc_u[c * kLocNodes + ((my_slots >> (10 * j)) & 1023u)] : ufun(f, j, c);
    };
  };
  auto loc_fill = [&](auto ufun) {
    if (loc_ok) {
      const int nl = loc.count;
      for (int t = threadIdx.x; t < nl * D; t += blockDim.x) {
        const int c = t / nl, i = t - c * nl;
        loc_u[c * kLocNodes + i] = ufun(c * g.nn + loc.node[i], 0, c);
      }
    }
    __syncthreads();
  };
  if constexpr (ONE) {
    if (my_idx < d_hi) {
      const int c = (int)(my_idx / g.nn);
      const int64_t i = my_idx - (int64_t)c * g.nn;
      my_free = (a.dofmask[i] >> c) & 1u;
      if (my_free) {
        my_id = idiag[my_idx];
        my_md = a.m[i] * a.inv_dt2;
      }
    }
    load_lane<D, R>(a, my_pi, my_valid, q, ld);
    for (int i = threadIdx.x; i < kLocNodes; i += blockDim.x) loc.key[i] = kLocEmpty;
    if (threadIdx.x == 0) {
      loc.count = 0;
      loc.over = 0;
    }
    __syncthreads();
    if (my_valid)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const unsigned long long key = (unsigned long long)ld.node[j];
        unsigned h = loc_hash(key);
        bool done = false;
        for (int probe = 0; probe < kLocNodes && !done; ++probe, h = (h + 1) & (kLocNodes - 1)) {
          const unsigned long long prev = atomicCAS(&loc.key[h], kLocEmpty, key);
          if (prev == kLocEmpty) {
            const int id = atomicAdd(&loc.count, 1);
            loc.node[id] = (long long)key;
            loc.id[h] = id;
            done = true;
          } else if (prev == key) {
            done = true;
          }
        }
        if (!done) loc.over = 1;
      }
    __syncthreads();
    loc_ok = loc.over == 0;
    if (my_valid && loc_ok)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const unsigned long long key = (unsigned long long)ld.node[j];
        unsigned h = loc_hash(key);
        for (int probe = 0; probe < kLocNodes; ++probe, h = (h + 1) & (kLocNodes - 1))
          if (loc.key[h] == key) {
            my_slots |= (unsigned)loc.id[h] << (10 * j);
            break;
          }
      }
  }
  // scalar state: thread 0 of every block keeps gamma for beta and the
  // stopping tests, thread 32 its own copy for alpha (all blocks see the
  // same totals, so they take the same decisions); every thread counts the
  // iterations and keeps the curvature-failure flag
  int it = 0, neg = 0;
  double gamma = 0.0;
  const int max_it = S->cg_max;
  const double tol2 = S->tol2;

  // ---- phase 0: w_0 = A u_0, gamma_0 = r0.u0, delta_0 = u0.w0
  {
    double acc[3] = {0.0, 0.0, 0.0};
    const double* r0 = a.r[0];
    auto u0 = [=](int64_t f, int, int) { return __ldcg(&r0[f]) * idiag[f]; };
    if constexpr (ONE) {
      if (my_free) {
        const double ri = r0[my_idx];
        const double ui = ri * my_id;
        const double mu = my_md * ui;
        acc[0] += ri * ui;
        acc[2] += mu * ui;
        atomicAdd(&a.w[0][my_idx], mu);
      }
      loc_fill(u0);
      acc[2] += group_hvp_lane<D, R>(a, ld, my_valid, q, leader, loc_gather(u0), a.w[0]);
    } else {
      for (int64_t idx = d_lo + threadIdx.x; idx < d_hi; idx += blockDim.x) {
        const int c = (int)(idx / g.nn);
        const int64_t i = idx - (int64_t)c * g.nn;
        if ((a.dofmask[i] >> c) & 1u) {
          const double ri = r0[idx];
          const double ui = ri * idiag[idx];
          const double mu = a.m[i] * a.inv_dt2 * ui;
          acc[0] += ri * ui;
          acc[2] += mu * ui;
          atomicAdd(&a.w[0][idx], mu);
        }
      }
      for (int64_t b0 = warp0; b0 < a.P.n; b0 += wstride) {
        const int64_t pi = b0 + grp;
        acc[2] += group_hvp<D, R>(a, pi, in_group && pi < a.P.n, q, leader, u0, a.w[0]);
      }
    }
    pcg_block_partials<3>(acc, a.partials);
    if (!grid_barrier(&S->bar_count, &bar_target, a.err, gridDim.x)) return;
    pcg_grid_totals<3>(a.partials, sh_tot);
    __syncthreads();
    if (threadIdx.x == 0) {
      const double delta = sh_tot[2];
      int stop = (sh_tot[0] == 0.0) || (S->cg_done != 0) || max_it <= 0;
      const int bad = !stop && !(delta > 0.0);
      sh_alpha = stop || bad ? 0.0 : sh_tot[0] / delta;
      sh_beta = 0.0;
      sh_stop = stop;
      sh_neg = bad;
    }
    gamma = sh_tot[0];
    __syncthreads();
    neg = sh_neg;
  }
  bool halt = sh_stop || sh_neg;
  while (!halt) {
    const double alpha = sh_alpha, beta = sh_beta;
    const double* rk = a.r[it & 1];
    double* rn = a.r[(it + 1) & 1];
    double* sk = a.s[it & 1];
    const double* sp = a.s[(it + 1) & 1];
    const double* wk = a.w[it % 3];
    double* wn = a.w[(it + 1) % 3];
    double* wz = a.w[(it + 2) % 3];
    double acc[3] = {0.0, 0.0, 0.0};
    auto uk = [=](int64_t f, int, int) {
      return (__ldcg(&rk[f]) - alpha * (__ldcg(&wk[f]) + beta * __ldcg(&sp[f]))) * idiag[f];
    };
    if constexpr (ONE) {
      if (my_free) {
        const double rki = __ldcg(&rk[my_idx]);
        const double ski = __ldcg(&wk[my_idx]) + beta * __ldcg(&sp[my_idx]);
        sk[my_idx] = ski;
        my_p = rki * my_id + beta * my_p;
        my_x += alpha * my_p;
        const double rni = rki - alpha * ski;
        rn[my_idx] = rni;
        const double ui = rni * my_id;
        const double mu = my_md * ui;
        acc[0] += rni * ui;
        acc[1] += rni * rni;
        acc[2] += mu * ui;
        atomicAdd(&wn[my_idx], mu);
      }
      if (my_idx < d_hi) wz[my_idx] = 0.0;
      loc_fill(uk);
      acc[2] += group_hvp_lane<D, R>(a, ld, my_valid, q, leader, loc_gather(uk), wn);
    } else {
      for (int64_t idx = d_lo + threadIdx.x; idx < d_hi; idx += blockDim.x) {
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
          const double mu = a.m[i] * a.inv_dt2 * ui;
          acc[0] += rni * ui;
          acc[1] += rni * rni;
          acc[2] += mu * ui;
          atomicAdd(&wn[idx], mu);
        }
        wz[idx] = 0.0;
      }
      for (int64_t b0 = warp0; b0 < a.P.n; b0 += wstride) {
        const int64_t pi = b0 + grp;
        acc[2] += group_hvp<D, R>(a, pi, in_group && pi < a.P.n, q, leader, uk, wn);
      }
    }
    pcg_block_partials<3>(acc, a.partials);
    if (!grid_barrier(&S->bar_count, &bar_target, a.err, gridDim.x)) return;
    ++it;
    pcg_grid_totals<3>(a.partials, sh_tot);
    __syncthreads();
    // beta = gamma / gamma_old, and alpha = gamma / (delta - beta gamma /
    // alpha_old) as gamma P / Q with P = gamma_old alpha_old > 0 and
    // Q = delta P - gamma^2 (the sign of the curvature term), so the two
    // divisions (each a long serial FP64 sequence) run at once on two warps
    if (threadIdx.x == 0) {
      const double gamma_old = gamma;
      gamma = sh_tot[0];
      const int stop = sh_tot[1] <= tol2 || it >= max_it;
      sh_beta = stop ? 0.0 : gamma / gamma_old;
      sh_stop = stop;
    } else if (threadIdx.x == 32) {
      const double gamma_new = sh_tot[0];
      const double P = gamma * alpha;
      const double Q = fma(sh_tot[2], P, -gamma_new * gamma_new);
      const int ok = Q > 0.0;
      sh_alpha = ok ? gamma_new * P / Q : 0.0;
      sh_neg = !ok;
      gamma = gamma_new;
    }
    __syncthreads();
    if (!sh_stop && sh_neg) neg = 1;
    halt = sh_stop || sh_neg;
  }
  // thread 0 of each block knows whether the first direction failed
  __shared__ int sh_fallback;
  if (threadIdx.x == 0) sh_fallback = (neg && it == 0);
  __syncthreads();
  const double* r0 = a.r[0];
  if constexpr (ONE) {
    // no direction yet: the preconditioned steepest descent u_0
    if (my_free) a.x[my_idx] = sh_fallback ? r0[my_idx] * my_id : my_x;
  } else if (sh_fallback) {
    for (int64_t idx = d_lo + threadIdx.x; idx < d_hi; idx += blockDim.x) {
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

// ---------------------------------------------------------------------------
// Streaming PCG for problems that one co-resident pass does not cover: the
// same Jacobi PCG as three small kernels per iteration at full occupancy,
// the kernel boundaries standing in for the grid barrier.  The scalars stay
// on the device; a kernel launched after convergence returns at once, so
// the host enqueues iterations in chunks and looks at the flag between them.
//   k_cgs_start: q = 0 and the mass part of p.Ap (r, z = D^-1 r, p = z,
//                x = 0 and r.z come from the gradient kernel); vectors x = a.x,
//                r = a.r[0], z = a.r[1], p = a.s[0], q = a.w[0]
//   k_cgs_hvp:   q = K p by the particle gather-scatter (lane groups) and
//                the particle part p:Kp = sum_p G : L G
//   k_cgs_alpha: alpha = r.z / p.Ap; x += alpha p; r -= alpha (q + M/dt^2 p);
//                z = D^-1 r; the last block takes r.z, r.r, beta and the
//                stopping tests
//   k_cgs_beta:  p = z + beta p, q = 0, the mass part of the next p.Ap
// Deterministic: every sum is taken in block order by the last block.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t cgs_tid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t cgs_stride() { return (int64_t)gridDim.x * blockDim.x; }
// Steps the (component, node) pair of a flat DOF index idx = c nn + i by
// `step` DOFs without a 64-bit division per DOF.
__device__ __forceinline__ void dof_step(int& c, int64_t& i, int64_t step, int64_t nn) {
  i += step;
  while (i >= nn) {
    i -= nn;
    ++c;
  }
}

template <int D, typename R>
__global__ void __launch_bounds__(kThreads) k_cgs_start(PcgArgsT<R> a) {
  const GridGeo& g = a.g;
  double acc[1] = {0.0};
  int64_t idx = cgs_tid();
  int c = (int)(idx / g.nn);
  int64_t i = idx - (int64_t)c * g.nn;
  for (const int64_t step = cgs_stride(); idx < g.nn * D; idx += step, dof_step(c, i, step, g.nn)) {
    a.w[0][idx] = 0.0;
    if ((a.dofmask[i] >> c) & 1u) {
      const double pi = a.s[0][idx];
      acc[0] += a.m[i] * a.inv_dt2 * pi * pi;
    }
  }
  double tot[1];
  if (grid_sum<1>(acc, a.partials, &a.S->counter, tot) && threadIdx.x == 0) {
    a.S->pq_diag = tot[0];
    a.S->cg_iter = 0;
    a.S->cg_neg = 0;
    if (a.S->cg_max <= 0) a.S->cg_done = 1;
  }
}

template <int D, typename R>
__global__ void __launch_bounds__(kThreads) k_cgs_hvp(PcgArgsT<R> a) {
  if (__ldcg(&a.S->cg_done)) return;
  constexpr int LPP = HvpGroup<D>::LPP, GP = HvpGroup<D>::GP;
  const int64_t tid = cgs_tid(), stride = cgs_stride();
  const int lane = threadIdx.x & 31;
  const int grp = lane / LPP;
  const int q = lane - grp * LPP;
  const int leader = grp * LPP;
  const bool in_group = grp < GP;
  const double* p = a.s[0];
  double acc[1] = {0.0};
  for (int64_t b0 = (tid >> 5) * GP; b0 < a.P.n; b0 += (stride >> 5) * GP) {
    const int64_t pi = b0 + grp;
    acc[0] += group_hvp<D, R>(a, pi, in_group && pi < a.P.n, q, leader,
                              [=](int64_t f, int, int) { return __ldcg(&p[f]); }, a.w[0]);
  }
  double tot[1];
  if (grid_sum<1>(acc, a.partials, &a.S->counter, tot) && threadIdx.x == 0) a.S->pq = tot[0];
}

template <int D, typename R>
__global__ void __launch_bounds__(kThreads) k_cgs_alpha(PcgArgsT<R> a) {
  DevScalars* S = a.S;
  if (__ldcg(&S->cg_done)) return;
  const GridGeo& g = a.g;
  const double pAp = __ldcg(&S->pq) + __ldcg(&S->pq_diag);
  const double rz = __ldcg(&S->rz);
  const int it = __ldcg(&S->cg_iter);
  if (!(pAp > 0.0)) {
    // negative curvature: stop; with no direction yet take z_0 = D^-1 r_0
    if (it == 0) {
      int64_t idx = cgs_tid();
      int c = (int)(idx / g.nn);
      int64_t i = idx - (int64_t)c * g.nn;
      for (const int64_t step = cgs_stride(); idx < g.nn * D; idx += step, dof_step(c, i, step, g.nn)) {
        if ((a.dofmask[i] >> c) & 1u) a.x[idx] = a.s[0][idx];
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->cg_neg = 1;
      S->cg_done = 1;
    }
    return;
  }
  const double alpha = rz / pAp;
  double* r = a.r[0];
  double* z = a.r[1];
  double acc[2] = {0.0, 0.0};
  int64_t idx = cgs_tid();
  int c = (int)(idx / g.nn);
  int64_t i = idx - (int64_t)c * g.nn;
  for (const int64_t step = cgs_stride(); idx < g.nn * D; idx += step, dof_step(c, i, step, g.nn)) {
    if ((a.dofmask[i] >> c) & 1u) {
      const double pi = a.s[0][idx];
      a.x[idx] += alpha * pi;
      const double ap = a.w[0][idx] + a.m[i] * a.inv_dt2 * pi;
      const double ri = r[idx] - alpha * ap;
      r[idx] = ri;
      const double zi = ri * a.diag[idx];
      z[idx] = zi;
      acc[0] += ri * zi;
      acc[1] += ri * ri;
    }
  }
  double tot[2];
  if (grid_sum<2>(acc, a.partials, &S->counter, tot) && threadIdx.x == 0) {
    const int itn = it + 1;
    S->cg_iter = itn;
    S->beta = tot[0] / rz;
    S->rz = tot[0];
    S->rr = tot[1];
    if (tot[1] <= S->tol2 || itn >= S->cg_max) S->cg_done = 1;
  }
}

template <int D, typename R>
__global__ void __launch_bounds__(kThreads) k_cgs_beta(PcgArgsT<R> a) {
  DevScalars* S = a.S;
  if (__ldcg(&S->cg_done)) return;
  const GridGeo& g = a.g;
  const double beta = __ldcg(&S->beta);
  const double* z = a.r[1];
  double acc[1] = {0.0};
  int64_t idx = cgs_tid();
  int c = (int)(idx / g.nn);
  int64_t i = idx - (int64_t)c * g.nn;
  for (const int64_t step = cgs_stride(); idx < g.nn * D; idx += step, dof_step(c, i, step, g.nn)) {
    a.w[0][idx] = 0.0;
    if ((a.dofmask[i] >> c) & 1u) {
      const double pi = z[idx] + beta * a.s[0][idx];
      a.s[0][idx] = pi;
      acc[0] += a.m[i] * a.inv_dt2 * pi * pi;
    }
  }
  double tot[1];
  if (grid_sum<1>(acc, a.partials, &S->counter, tot) && threadIdx.x == 0) S->pq_diag = tot[0];
}

}  // namespace osmpm
