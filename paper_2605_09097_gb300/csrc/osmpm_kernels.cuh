// Kernels of the OS-MPM hot path, templated on the dimension D.  Included
// by kernels_d2.cu and kernels_d3.cu, which instantiate Kernels<2>/<3>.
//
// Layouts: particle fields component-major (x[a*n + p]); grid fields
// component-major over the dense node box (u[a*nn + i]); per-particle
// Hessian blocks L packed symmetric, entry-major (L[e*n + p]).
#pragma once

#include "osmpm_device.cuh"
#include "osmpm_internal.h"
#include "osmpm_pcg.cuh"
#include "osmpm_tile.cuh"
#include "osmpm_contact.cuh"
#include "osmpm_multi.cuh"

namespace osmpm {

template <int D>
struct Pow3 {
  static constexpr int K = (D == 2) ? 9 : 27;
};

__device__ __forceinline__ int64_t gtid() {
  return (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

template <int D, class PP>
__device__ __forceinline__ void load_x(const PP& P, int64_t p, double* x) {
#pragma unroll
  for (int a = 0; a < D; ++a) x[a] = P.x[a * P.n + p];
}
template <int D, class PP>
__device__ __forceinline__ void load_F(const PP& P, int64_t p, double* F) {
#pragma unroll
  for (int e = 0; e < D * D; ++e) F[e] = P.F[e * P.n + p];
}

// F(u) = (I + G) F^n with G = sum_i u_i grad N_i^T (Eq. F_update).
template <int D>
__device__ __forceinline__ void deform(const double* G, const double* Fn, double* F) {
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double t = Fn[a * D + b];
#pragma unroll
      for (int c = 0; c < D; ++c) t += G[a * D + c] * Fn[c * D + b];
      F[a * D + b] = t;
    }
}

// G = sum over the stencil of w_i grad N_i^T for a grid vector field w.
template <int D>
__device__ __forceinline__ void gather_grad(const Stencil<D>& s, const GridGeo& g,
                                            const double* w, double* G) {
#pragma unroll
  for (int e = 0; e < D * D; ++e) G[e] = 0.0;
#pragma unroll 3
  for (int k = 0; k < Pow3<D>::K; ++k) {
    double N, dN[D];
    const int64_t node = stencil_node<D>(s, g, k, N, dN);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double wa = w[a * g.nn + node];
#pragma unroll
      for (int b = 0; b < D; ++b) G[a * D + b] += wa * dN[b];
    }
  }
}

// ---------------------------------------------------------------------------
// Particle bookkeeping
// ---------------------------------------------------------------------------
template <int D, typename R>
__global__ void k_morton_keys(const double* x, int64_t n, GridGeo g, uint64_t* keys,
                              uint32_t* vals, int* err) {
  const int64_t p = gtid();
  if (p >= n) return;
  double xp[D];
#pragma unroll
  for (int a = 0; a < D; ++a) xp[a] = x[a * n + p];
  Stencil<D> s;
  uint64_t code = 0;
  if (!make_stencil<D>(xp, g, s)) {
    atomicOr(err, kErrOutOfGrid);
  } else {
    for (int bit = 0; bit < 21; ++bit)
#pragma unroll
      for (int a = 0; a < D; ++a)
        code |= (uint64_t)(((unsigned)s.base[a] >> bit) & 1u) << (bit * D + a);
  }
  keys[p] = code;
  vals[p] = (uint32_t)p;
}

template <int D, typename R>
__global__ void k_permute(PartPtrsT<R> src, PartPtrsT<R> dst, const uint32_t* perm) {
  const int64_t s = gtid();
  const int64_t n = src.n;
  if (s >= n) return;
  const int64_t q = perm[s];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    dst.x[a * n + s] = src.x[a * n + q];
    dst.v[a * n + s] = src.v[a * n + q];
  }
#pragma unroll
  for (int e = 0; e < D * D; ++e) {
    dst.B[e * n + s] = src.B[e * n + q];
    dst.F[e * n + s] = src.F[e * n + q];
  }
  dst.vol0[s] = src.vol0[q];
  dst.mass[s] = src.mass[q];
  dst.mu[s] = src.mu[q];
  dst.lam[s] = src.lam[q];
  dst.flags[s] = src.flags[q];
  dst.id[s] = src.id[q];
}

template <int D, typename R>
__global__ void k_scatter_by_id(PartPtrsT<R> src, PartPtrsT<R> dst) {
  const int64_t s = gtid();
  const int64_t n = src.n;
  if (s >= n) return;
  const int64_t q = src.id[s];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    dst.x[a * n + q] = src.x[a * n + s];
    dst.v[a * n + q] = src.v[a * n + s];
  }
#pragma unroll
  for (int e = 0; e < D * D; ++e) {
    dst.B[e * n + q] = src.B[e * n + s];
    dst.F[e * n + q] = src.F[e * n + s];
  }
  dst.vol0[q] = src.vol0[s];
  dst.mass[q] = src.mass[s];
  dst.mu[q] = src.mu[s];
  dst.lam[q] = src.lam[s];
  dst.flags[q] = src.flags[s];
  dst.id[q] = (uint32_t)q;
}

template <int D, typename R>
__global__ void k_lame(const double* E, const double* nu, PartPtrsT<R> P) {
  const int64_t p = gtid();
  if (p >= P.n) return;
  const double e = E[p], v = nu[p];
  P.mu[p] = e / (2.0 * (1.0 + v));
  P.lam[p] = e * v / ((1.0 + v) * (1.0 - 2.0 * v));
}

// Sorted component-major state -> id-ordered particle-major host layout.
template <int D, typename R>
__global__ void k_pack_out(PartPtrsT<R> P, double* x, double* v, double* B, double* F) {
  const int64_t s = gtid();
  const int64_t n = P.n;
  if (s >= n) return;
  const int64_t q = P.id[s];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    x[q * D + a] = P.x[a * n + s];
    v[q * D + a] = P.v[a * n + s];
  }
#pragma unroll
  for (int e = 0; e < D * D; ++e) {
    B[q * D * D + e] = P.B[e * n + s];
    F[q * D * D + e] = P.F[e * n + s];
  }
}

template <int D, typename R>
__global__ void k_unpack_in(const double* x, const double* v, const double* B, const double* F,
                            PartPtrsT<R> dst) {
  const int64_t q = gtid();
  const int64_t n = dst.n;
  if (q >= n) return;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    dst.x[a * n + q] = x[q * D + a];
    dst.v[a * n + q] = (R)v[q * D + a];
  }
#pragma unroll
  for (int e = 0; e < D * D; ++e) {
    dst.B[e * n + q] = (R)B[q * D * D + e];
    dst.F[e * n + q] = (R)F[q * D * D + e];
  }
}

template <int D, typename R>
__global__ void k_normalize(GridGeo g, const double* m, const double* mv, double* vn) {
  for (int64_t i = gtid(); i < g.nn; i += gstride()) {
    const double mi = m[i];
#pragma unroll
    for (int a = 0; a < D; ++a) vn[a * g.nn + i] = mi > g.mass_eps ? mv[a * g.nn + i] / mi : 0.0;
  }
}

// ---------------------------------------------------------------------------
// Grid preparation: Dirichlet data (physical rules, then Schwarz receivers
// with temporally interpolated values, Eq. temporal_interp), the free-DOF
// mask and the initial guess x_hat^(0) = x^n + dt v^n on free DOFs.
// ---------------------------------------------------------------------------
template <int D, typename R>
__global__ void k_grid_prep(GridGeo g, const double* m, const double* vn, PrepArgs A, double dt,
                            uint8_t* dofmask, double* u) {
  const unsigned all = (1u << D) - 1u;
  for (int64_t i = gtid(); i < g.nn; i += gstride()) {
    const bool active = m[i] > g.mass_eps;
    double xi[D];
#pragma unroll
    for (int a = 0; a < D; ++a) xi[a] = node_pos(g, i, a);
    unsigned fixed = 0u;
    double vel[D];
#pragma unroll
    for (int a = 0; a < D; ++a) vel[a] = 0.0;
    for (int r = 0; r < A.n_rules; ++r) {
      const DevRule& rule = A.rules[r];
      bool in = true;
#pragma unroll
      for (int a = 0; a < D; ++a) in = in && (xi[a] >= rule.lo[a]) && (xi[a] <= rule.hi[a]);
      if (!in) continue;
      if (rule.kind == 0) {
#pragma unroll
        for (int a = 0; a < D; ++a)
          if ((rule.comp_mask >> a) & 1u) {
            fixed |= 1u << a;
            vel[a] = rule.vel[a];
          }
      } else {
        double rel[D];
#pragma unroll
        for (int a = 0; a < D; ++a) rel[a] = xi[a] - rule.center[a];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          double t = 0.0;
#pragma unroll
          for (int b = 0; b < D; ++b) t += rule.R[a * 3 + b] * rel[b];
          vel[a] = (t - rel[a]) / dt;
        }
        fixed = all;
      }
    }
    if (A.physmask) A.physmask[i] = (uint8_t)fixed;
    if (A.hold && A.hold[i]) {  // rigid-plane contact: the held normal component
      fixed |= 2u;
      vel[1] = A.hold_v[i];
    }
    if (A.recv && A.recv[i] && fixed == 0u) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        vel[a] = (1.0 - A.a_m) * A.bc0[a * g.nn + i] + A.a_m * A.bc1[a * g.nn + i];
        if (A.bc_applied) A.bc_applied[a * g.nn + i] = vel[a];
      }
      fixed = all;
    } else if (A.bc_applied) {
#pragma unroll
      for (int a = 0; a < D; ++a) A.bc_applied[a * g.nn + i] = 0.0;
    }
    dofmask[i] = active ? (uint8_t)(~fixed & all) : (uint8_t)0;
#pragma unroll
    for (int a = 0; a < D; ++a)
      u[a * g.nn + i] = !active ? 0.0 : (((fixed >> a) & 1u) ? dt * vel[a] : dt * vn[a * g.nn + i]);
  }
}

// ---------------------------------------------------------------------------
// Gradient of E_h (Eq. grid_residual with the energy-consistent internal
// force sum_p V0 P F^nT grad N_i), Jacobi diagonal, and the per-particle
// Hessian block L(G) = V0 dP[G F^n] F^nT used by every HVP of the Newton
// iteration (K = Hessian of sum_p V0 Psi(F_p(u)), Sec. 2.2.5).
// ---------------------------------------------------------------------------
template <int D, typename R>
__global__ void __launch_bounds__(kThreads) k_grad(PartPtrsT<R> P, GridGeo g, const double* u,
                                                   const uint8_t* dofmask, double* grad,
                                                   double* diag, R* L, int* err, int lmode) {
  constexpr int DD = D * D;
  const int64_t p = gtid();
  if (p >= P.n) return;
  double xp[D], Fn[DD], G[DD], F[DD];
  load_x<D>(P, p, xp);
  load_F<D>(P, p, Fn);
  Stencil<D> s;
  if (!make_stencil<D>(xp, g, s)) {
    atomicOr(err, kErrOutOfGrid);
    return;
  }
  gather_grad<D>(s, g, u, G);
  deform<D>(G, Fn, F);
  const double mu = P.mu[p], lam = P.lam[p], V0 = P.vol0[p];
  NeoHookean<D> nh;
  if (!neo_hookean<D>(F, mu, lam, nh)) {
    atomicOr(err, kErrNonFinite);
    return;
  }
  double Pk[DD], Y[DD];
  pk1<D>(F, mu, lam, nh, Pk);
  // Y = V0 P F^nT
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double t = 0.0;
#pragma unroll
      for (int b = 0; b < D; ++b) t += Pk[a * D + b] * Fn[c * D + b];
      Y[a * D + c] = V0 * t;
    }
  // L columns: basis G = e_a e_b^T -> dF = e_a (row b of F^n); its diagonal
  // blocks give the Jacobi diagonal, the packed blocks are stored when asked
  double Lfull[DD * DD];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double dF[DD], dP[DD];
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int d = 0; d < D; ++d) dF[c * D + d] = (c == a) ? Fn[b * D + d] : 0.0;
      dpdf_apply<D>(dF, mu, lam, nh, dP);
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int e = 0; e < D; ++e) {
          double t = 0.0;
#pragma unroll
          for (int d = 0; d < D; ++d) t += dP[c * D + d] * Fn[e * D + d];
          Lfull[(c * D + e) * DD + (a * D + b)] = V0 * t;
        }
    }
  if (lmode & 1)
#pragma unroll
    for (int i = 0; i < DD; ++i)
#pragma unroll
      for (int j = i; j < DD; ++j)
        L[(int64_t)Sym<D>::idx(i, j) * P.n + p] = (R)(0.5 * (Lfull[i * DD + j] + Lfull[j * DD + i]));
  if constexpr (std::is_same<R, float>::value) {
    if (lmode & 2) {
      // the tiled product's data at this iterate (TileX): F^-T, the
      // coefficients of dP with V0 folded in, the offsets from the base
      R* X = L + (int64_t)Sym<D>::packed * P.n;
#pragma unroll
      for (int e = 0; e < DD; ++e) X[(int64_t)(TileX<D>::A + e) * P.n + p] = (R)nh.FiT[e];
      X[(int64_t)TileX<D>::C1 * P.n + p] = (R)(V0 * (mu - lam * nh.lnJ));
      X[(int64_t)TileX<D>::MU * P.n + p] = (R)(V0 * mu);
      X[(int64_t)TileX<D>::LAM * P.n + p] = (R)(V0 * lam);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const double t = __dmul_rn(__dsub_rn(xp[a], g.o[a]), g.inv_dx);  // as make_stencil
        X[(int64_t)(TileX<D>::FX + a) * P.n + p] = (R)(t - (double)s.base[a]);
      }
    }
  }
  // scatter gradient and diagonal
#pragma unroll 3
  for (int k = 0; k < Pow3<D>::K; ++k) {
    double N, dN[D];
    const int64_t node = stencil_node<D>(s, g, k, N, dN);
    const unsigned fm = dofmask[node];
    if (!fm) continue;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      if (!((fm >> a) & 1u)) continue;
      double f = 0.0, dg = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) f += Y[a * D + c] * dN[c];
#pragma unroll
      for (int b = 0; b < D; ++b)
#pragma unroll
        for (int c = 0; c < D; ++c) dg += Lfull[(a * D + b) * DD + (a * D + c)] * dN[b] * dN[c];
      atomicAdd(&grad[a * g.nn + node], f);
      atomicAdd(&diag[a * g.nn + node], dg);
    }
  }
}

// Completes the gradient on the free DOFs (inertia and external force),
// adds m/dt^2 to the diagonal and stores its inverse, and starts PCG from
// x = 0: r = -g, z = D^-1 r, p = z; reduces r.z and r.r.
template <int D, typename R>
__global__ void k_grad_finish(GridGeo g, const double* m, const double* vn, const double* u,
                              const uint8_t* dofmask, double gx, double gy, double gz, double dt,
                              double cg_rtol, double eta_max, int first, int cg_max, double* grad,
                              double* diag, double* x, double* r, double* z, double* p,
                              DevScalars* S, double* partials) {
  const double inv_dt2 = 1.0 / (dt * dt);
  const double gv[3] = {gx, gy, gz};
  double acc[2] = {0.0, 0.0};
  const int64_t total = g.nn * D;
  for (int64_t idx = gtid(); idx < total; idx += gstride()) {
    const int a = (int)(idx / g.nn);
    const int64_t i = idx - (int64_t)a * g.nn;
    const double mi = m[i];
    const bool active = mi > g.mass_eps;
    const bool fr = (dofmask[i] >> a) & 1u;
    double gi = 0.0;
    if (active) gi = grad[idx] + mi * inv_dt2 * (u[idx] - dt * vn[idx]) - mi * gv[a];
    grad[idx] = gi;
    x[idx] = 0.0;
    if (fr) {
      const double dg = 1.0 / (diag[idx] + mi * inv_dt2);  // stored inverted
      diag[idx] = dg;
      const double ri = -gi;
      const double zi = ri * dg;
      r[idx] = ri;
      z[idx] = zi;
      p[idx] = zi;
      acc[0] += ri * zi;
      acc[1] += ri * ri;
    } else {
      diag[idx] = 1.0;
      r[idx] = 0.0;
      z[idx] = 0.0;
      p[idx] = 0.0;
    }
  }
  double tot[2];
  if (grid_sum<2>(acc, partials, &S->counter, tot) && threadIdx.x == 0) {
    S->rz = tot[0];
    S->rr = tot[1];
    S->rr0 = tot[1];
    // inexact Newton: PCG stops at eta |r0| with eta = |g_k|/|g_0| clamped
    // to [cg_rtol, eta_max] (the Newton stop test decides convergence)
    if (first) S->g0sq = tot[1];
    double eta2 = S->g0sq > 0.0 ? tot[1] / S->g0sq : 0.0;
    const double lo = cg_rtol * cg_rtol, hi = eta_max * eta_max;
    eta2 = eta2 < lo ? lo : (eta2 > hi ? hi : eta2);
    if (hi < lo) eta2 = lo;
    S->tol2 = eta2 * tot[1];
    S->cg_iter = 0;
    S->cg_max = cg_max;
    S->cg_neg = 0;
    S->cg_done = (tot[1] == 0.0) ? 1 : 0;
    S->beta = 0.0;
  }
}

// PCG step A: p = z + beta p (after the first iteration); q = (m/dt^2) p on
// free DOFs; reduces the diagonal part of p.Hp.
template <int D, typename R>
__global__ void k_cg_a(GridGeo g, const double* m, const uint8_t* dofmask, double inv_dt2,
                       const double* z, double* p, double* q, DevScalars* S, double* partials) {
  if (*((volatile int*)&S->cg_done)) return;
  const int it = S->cg_iter;
  const double beta = S->beta;
  double acc[1] = {0.0};
  const int64_t total = g.nn * D;
  for (int64_t idx = gtid(); idx < total; idx += gstride()) {
    const int a = (int)(idx / g.nn);
    const int64_t i = idx - (int64_t)a * g.nn;
    if ((dofmask[i] >> a) & 1u) {
      double pv = p[idx];
      if (it > 0) {
        pv = z[idx] + beta * pv;
        p[idx] = pv;
      }
      const double md = m[i] * inv_dt2;
      q[idx] = md * pv;
      acc[0] += md * pv * pv;
    } else {
      q[idx] = 0.0;
    }
  }
  double tot[1];
  if (grid_sum<1>(acc, partials, &S->counter, tot) && threadIdx.x == 0) S->pq_diag = tot[0];
}

// PCG step B: the matrix-free Hessian-vector product, a particle gather of
// p (G = sum_j p_j grad N_j^T), Y = L G, scatter q_i += Y grad N_i, and the
// particle part of p.Hp = sum_p G : L G.  The last block forms alpha.
template <int D, typename R>
__global__ void __launch_bounds__(kThreads) k_cg_b(PartPtrsT<R> P, GridGeo g, const uint8_t* dofmask,
                                                   const R* L, const double* p, double* q,
                                                   DevScalars* S, double* partials) {
  constexpr int DD = D * D;
  if (*((volatile int*)&S->cg_done)) return;
  double acc[1] = {0.0};
  for (int64_t pi = gtid(); pi < P.n; pi += gstride()) {
    double xp[D];
    load_x<D>(P, pi, xp);
    Stencil<D> s;
    make_stencil<D>(xp, g, s);
    double G[DD], Y[DD];
    gather_grad<D>(s, g, p, G);
#pragma unroll
    for (int i = 0; i < DD; ++i) {
      double t = 0.0;
#pragma unroll
      for (int j = 0; j < DD; ++j) t += (double)L[(int64_t)Sym<D>::idx(i, j) * P.n + pi] * G[j];
      Y[i] = t;
    }
    double qf = 0.0;
#pragma unroll
    for (int i = 0; i < DD; ++i) qf += G[i] * Y[i];
    acc[0] += qf;
#pragma unroll 3
    for (int k = 0; k < Pow3<D>::K; ++k) {
      double N, dN[D];
      const int64_t node = stencil_node<D>(s, g, k, N, dN);
      const unsigned fm = dofmask[node];
      if (!fm) continue;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        if (!((fm >> a) & 1u)) continue;
        double f = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) f += Y[a * D + c] * dN[c];
        atomicAdd(&q[a * g.nn + node], f);
      }
    }
  }
  double tot[1];
  if (grid_sum<1>(acc, partials, &S->counter, tot) && threadIdx.x == 0) {
    const double pq = S->pq_diag + tot[0];
    S->pq = pq;
    if (!(pq > 0.0)) {
      S->cg_neg = 1;
      S->cg_done = 1;
    } else {
      S->alpha = S->rz / pq;
    }
  }
}

// PCG step C: x += alpha p, r -= alpha q, z = r/diag; the last block forms
// beta and the stopping test |r| <= rtol |r0| or the iteration cap.
template <int D, typename R>
__global__ void k_cg_c(GridGeo g, const uint8_t* dofmask, const double* diag, const double* p,
                       const double* q, double* x, double* r, double* z, DevScalars* S,
                       double* partials) {
  if (*((volatile int*)&S->cg_done)) return;
  const double alpha = S->alpha;
  double acc[2] = {0.0, 0.0};
  const int64_t total = g.nn * D;
  for (int64_t idx = gtid(); idx < total; idx += gstride()) {
    const int a = (int)(idx / g.nn);
    const int64_t i = idx - (int64_t)a * g.nn;
    if ((dofmask[i] >> a) & 1u) {
      x[idx] += alpha * p[idx];
      const double ri = r[idx] - alpha * q[idx];
      r[idx] = ri;
      const double zi = ri * diag[idx];  // diag holds the inverse
      z[idx] = zi;
      acc[0] += ri * zi;
      acc[1] += ri * ri;
    }
  }
  double tot[2];
  if (grid_sum<2>(acc, partials, &S->counter, tot) && threadIdx.x == 0) {
    S->beta = tot[0] / S->rz;
    S->rz = tot[0];
    S->rr = tot[1];
    const int it = S->cg_iter + 1;
    S->cg_iter = it;
    S->cg_done = (tot[1] <= S->tol2 || it >= S->cg_max) ? 1 : 0;
  }
}

template <int D, typename R>
__global__ void k_copy_if_neg(GridGeo g, const double* p, double* x, const DevScalars* S) {
  if (!(S->cg_neg && S->cg_iter == 0)) return;
  for (int64_t idx = gtid(); idx < g.nn * D; idx += gstride()) x[idx] = p[idx];
}

template <int D, typename R>
__global__ void k_set_cg_state(DevScalars* S, int iter, int done) {
  S->cg_iter = iter;
  S->cg_done = done;
  S->cg_neg = 0;
}

template <int D, typename R>
__global__ void k_maxabs(GridGeo g, const uint8_t* dofmask, const double* x, DevScalars* S,
                         double* partials) {
  double v = 0.0;
  for (int64_t idx = gtid(); idx < g.nn * D; idx += gstride()) {
    const int a = (int)(idx / g.nn);
    const int64_t i = idx - (int64_t)a * g.nn;
    if ((dofmask[i] >> a) & 1u) v = fmax(v, fabs(x[idx]));
  }
  double tot;
  if (grid_max(v, partials, &S->counter, tot) && threadIdx.x == 0) S->maxabs = tot;
}

// E_h(u + alpha x) - E_h(u) summed term by term (the line-search test of
// Sec. 2.2.5): per particle V0 (Psi(F(u + alpha x)) - Psi(F(u))), per node
// m/(2dt^2) s.(2(u - dt v^n) + s) - s.f_ext with s = alpha x.  +inf when a
// trial inverts an element; NaN, with kErrOutOfGrid in S->err, when a
// particle's support leaves the grid box.
template <int D, typename R>
__global__ void __launch_bounds__(kThreads) k_energy_change(PartPtrsT<R> P, GridGeo g, const double* m,
                                                            const double* vn, const double* u,
                                                            const double* x, double gx, double gy,
                                                            double gz, double dt, double alpha,
                                                            DevScalars* S, double* partials) {
  constexpr int DD = D * D;
  double acc[1] = {0.0};
  for (int64_t pi = gtid(); pi < P.n; pi += gstride()) {
    double xp[D], Fn[DD], Gu[DD], Gs[DD], F0[DD], dF[DD];
    load_x<D>(P, pi, xp);
    load_F<D>(P, pi, Fn);
    Stencil<D> s;
    if (!make_stencil<D>(xp, g, s)) {
      // a support leaving the grid box has no energy term: the sum becomes
      // NaN and the scalars' error word says why
      atomicOr(&S->err, kErrOutOfGrid);
      acc[0] += NAN;
      continue;
    }
    gather_grad<D>(s, g, u, Gu);
    gather_grad<D>(s, g, x, Gs);
    deform<D>(Gu, Fn, F0);
    // dF = alpha Gs F^n
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) {
        double t = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) t += Gs[a * D + c] * Fn[c * D + b];
        dF[a * D + b] = alpha * t;
      }
    double dpsi;
    if (!psi_change<D>(F0, dF, P.mu[pi], P.lam[pi], dpsi)) {
      acc[0] += INFINITY;
    } else {
      acc[0] += P.vol0[pi] * dpsi;
    }
  }
  const double inv_2dt2 = 0.5 / (dt * dt);
  const double gv[3] = {gx, gy, gz};
  for (int64_t idx = gtid(); idx < g.nn * D; idx += gstride()) {
    const int a = (int)(idx / g.nn);
    const int64_t i = idx - (int64_t)a * g.nn;
    const double mi = m[i];
    if (!(mi > g.mass_eps)) continue;
    const double sv = alpha * x[idx];
    acc[0] += mi * inv_2dt2 * sv * (2.0 * (u[idx] - dt * vn[idx]) + sv) - sv * mi * gv[a];
  }
  double tot[1];
  if (grid_sum<1>(acc, partials, &S->counter, tot) && threadIdx.x == 0) S->dE = tot[0];
}

// Warm start: free DOFs take a previous solution, fixed DOFs keep the
// prepared Dirichlet values.
template <int D, typename R>
__global__ void k_warm_start(GridGeo g, const uint8_t* dofmask, const double* src, double* u) {
  for (int64_t idx = gtid(); idx < g.nn * D; idx += gstride()) {
    const int a = (int)(idx / g.nn);
    const int64_t i = idx - (int64_t)a * g.nn;
    if ((dofmask[i] >> a) & 1u) u[idx] = src[idx];
  }
}

// Moves the free-DOF part of u into x (u keeps its fixed DOFs, x is zero
// on them): u becomes the x_hat = x^n candidate, u + x the prepared one.
template <int D, typename R>
__global__ void k_split_free(GridGeo g, const uint8_t* dofmask, double* u, double* x) {
  for (int64_t idx = gtid(); idx < g.nn * D; idx += gstride()) {
    const int a = (int)(idx / g.nn);
    const int64_t i = idx - (int64_t)a * g.nn;
    if ((dofmask[i] >> a) & 1u) {
      x[idx] = u[idx];
      u[idx] = 0.0;
    } else {
      x[idx] = 0.0;
    }
  }
}

template <int D, typename R>
__global__ void k_axpy(GridGeo g, double* u, const double* x, double alpha) {
  for (int64_t idx = gtid(); idx < g.nn * D; idx += gstride()) u[idx] += alpha * x[idx];
}

// ---------------------------------------------------------------------------
// APIC grid-to-particle transfer with v_i = u_i/dt (Eqs. g2p_v, g2p_B), the
// F update (Eq. F_update) and advection (Eq. advection).
// ---------------------------------------------------------------------------
template <int D, typename R>
__global__ void __launch_bounds__(kThreads) k_g2p(PartPtrsT<R> P, GridGeo g, const double* u,
                                                  double dt) {
  constexpr int DD = D * D;
  const int64_t p = gtid();
  if (p >= P.n) return;
  double xp[D], Fn[DD];
  load_x<D>(P, p, xp);
  load_F<D>(P, p, Fn);
  Stencil<D> s;
  make_stencil<D>(xp, g, s);
  double vnew[D], Bnew[DD], G[DD];
#pragma unroll
  for (int a = 0; a < D; ++a) vnew[a] = 0.0;
#pragma unroll
  for (int e = 0; e < DD; ++e) {
    Bnew[e] = 0.0;
    G[e] = 0.0;
  }
#pragma unroll 3
  for (int k = 0; k < Pow3<D>::K; ++k) {
    double N, dN[D], r[D], vi[D];
    const int64_t node = stencil_node<D>(s, g, k, N, dN);
#pragma unroll
    for (int a = 0; a < D; ++a) r[a] = stencil_node_pos<D>(s, g, k, a) - xp[a];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double ua = u[a * g.nn + node];
      vi[a] = ua / dt;
      vnew[a] += N * vi[a];
#pragma unroll
      for (int b = 0; b < D; ++b) {
        Bnew[a * D + b] += N * vi[a] * r[b];
        G[a * D + b] += ua * dN[b];
      }
    }
  }
  double F[DD];
  deform<D>(G, Fn, F);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    P.v[a * P.n + p] = (R)vnew[a];
    P.x[a * P.n + p] = xp[a] + dt * vnew[a];
  }
#pragma unroll
  for (int e = 0; e < DD; ++e) {
    P.B[e * P.n + p] = (R)Bnew[e];
    P.F[e * P.n + p] = (R)F[e];
  }
}

// ---------------------------------------------------------------------------
// Schwarz interface operators (Sec. 3.2)
// ---------------------------------------------------------------------------
template <int D, typename R>
__global__ void k_gamma(int64_t nn, double mass_eps, const double* m, const double* bm, double tau,
                        uint8_t* gam) {
  for (int64_t i = gtid(); i < nn; i += gstride())
    gam[i] = (m[i] > mass_eps && bm[i] > tau) ? 1 : 0;
}

// Eq. overlap_donor on coincident boundary nodes (|x_B - x_S|_inf <= 1e-9
// dx_S): the larger grid mass donates, ties (within 1e-12 relative) to B.
template <int D, typename R>
__global__ void k_arbitrate(GridGeo gB, GridGeo gS, const uint8_t* gamB, const uint8_t* gamS,
                            const double* mB, const double* mS, uint8_t* recvB, uint8_t* recvS) {
  for (int64_t I = gtid(); I < gB.nn; I += gstride()) {
    if (!gamB[I]) continue;
    bool ok = true;
    int64_t j = 0, stride = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double xb = node_pos(gB, I, a);
      const double jf = rint(__ddiv_rn(__dsub_rn(xb, gS.o[a]), gS.dx));
      const bool inside = jf >= 0.0 && jf < (double)gS.res[a];
      const double xs = __dadd_rn(gS.o[a], __dmul_rn(jf, gS.dx));
      ok = ok && inside && (fabs(xs - xb) <= 1e-9 * gS.dx);
      j += (int64_t)(inside ? jf : 0.0) * stride;
      stride *= gS.res[a];
    }
    if (!ok || !gamS[j]) continue;
    if (mS[j] > mB[I] * (1.0 + 1e-12))
      recvS[j] = 0;
    else
      recvB[I] = 0;
  }
}

// Numerator and denominator of Eq. spatial_projection: every active fine
// node j scatters m_Sj N_BI(x_Sj) (times v_Sj) to its coarse support.
template <int D, typename R>
__global__ void k_proj_scatter(GridGeo gB, GridGeo gS, const double* mS, const double* vS,
                               double* num, double* den) {
  for (int64_t j = gtid(); j < gS.nn; j += gstride()) {
    const double mj = mS[j];
    if (!(mj > gS.mass_eps)) continue;
    double xs[D], vj[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      xs[a] = node_pos(gS, j, a);
      vj[a] = vS[a * gS.nn + j];
    }
    int base[D];
    double w[D][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double t = __dmul_rn(__dsub_rn(xs[a], gB.o[a]), gB.inv_dx);
      const double b = floor(__dsub_rn(t, 0.5));
      base[a] = (int)b;
      const double fx = t - b;
      const double e0 = 1.5 - fx, e1 = fx - 1.0, e2 = fx - 0.5;
      w[a][0] = 0.5 * e0 * e0;
      w[a][1] = 0.75 - e1 * e1;
      w[a][2] = 0.5 * e2 * e2;
    }
    for (int k = 0; k < Pow3<D>::K; ++k) {
      const int off[3] = {k % 3, (k / 3) % 3, k / 9};
      bool in = true;
      int64_t node = 0, stride = 1;
      double N = mj;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int c = base[a] + off[a];
        in = in && c >= 0 && c < gB.res[a];
        node += (int64_t)c * stride;
        stride *= gB.res[a];
        N *= w[a][off[a]];
      }
      if (!in) continue;
      atomicAdd(&den[node], N);
#pragma unroll
      for (int a = 0; a < D; ++a) atomicAdd(&num[a * gB.nn + node], N * vj[a]);
    }
  }
}

template <int D, typename R>
__global__ void k_recvB_filter(int64_t nn, const double* den, double tau, const uint8_t* physB,
                               uint8_t* recvB) {
  for (int64_t I = gtid(); I < nn; I += gstride())
    if (recvB[I] && (!(den[I] > tau) || physB[I])) recvB[I] = 0;
}

// Gamma_hat_S keeps fine nodes whose coarse support lies in the box and is
// all active; no receiver carries a physical rule.
template <int D, typename R>
__global__ void k_recvS_filter(GridGeo gB, GridGeo gS, const double* mB, const uint8_t* physS,
                               uint8_t* recvS) {
  for (int64_t j = gtid(); j < gS.nn; j += gstride()) {
    if (!recvS[j]) continue;
    if (physS[j]) {
      recvS[j] = 0;
      continue;
    }
    int base[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double xs = node_pos(gS, j, a);
      const double t = __dmul_rn(__dsub_rn(xs, gB.o[a]), gB.inv_dx);
      base[a] = (int)floor(__dsub_rn(t, 0.5));
    }
    bool all = true;
    for (int k = 0; k < Pow3<D>::K && all; ++k) {
      const int off[3] = {k % 3, (k / 3) % 3, k / 9};
      int64_t node = 0, stride = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int c = base[a] + off[a];
        all = all && c >= 0 && c < gB.res[a];
        node += (int64_t)c * stride;
        stride *= gB.res[a];
      }
      all = all && (mB[node] > gB.mass_eps);
    }
    if (!all) recvS[j] = 0;
  }
}

template <int D, typename R>
__global__ void k_proj_finish(GridGeo gB, const uint8_t* recvB, const double* num,
                              const double* den, double eps_tol, double* out) {
  for (int64_t I = gtid(); I < gB.nn; I += gstride()) {
    const bool r = recvB[I];
#pragma unroll
    for (int a = 0; a < D; ++a)
      out[a * gB.nn + I] = r ? num[a * gB.nn + I] / (den[I] + eps_tol) : 0.0;
  }
}

// I_{B->S} of Eq. interp_BtoS on the fine receivers.
template <int D, typename R>
__global__ void k_interp(GridGeo gB, GridGeo gS, const double* vB, const uint8_t* recvS,
                         double* out) {
  for (int64_t j = gtid(); j < gS.nn; j += gstride()) {
    double acc[D];
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] = 0.0;
    if (recvS[j]) {
      double xs[D];
#pragma unroll
      for (int a = 0; a < D; ++a) xs[a] = node_pos(gS, j, a);
      Stencil<D> s;
      make_stencil<D>(xs, gB, s);
      for (int k = 0; k < Pow3<D>::K; ++k) {
        double N, dN[D];
        const int64_t node = stencil_node<D>(s, gB, k, N, dN);
#pragma unroll
        for (int a = 0; a < D; ++a) acc[a] += N * vB[a * gB.nn + node];
      }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) out[a * gS.nn + j] = acc[a];
  }
}

template <int D, typename R>
__global__ void k_vel_from_u(GridGeo g, const double* m, const double* u, double dt, double* v) {
  for (int64_t idx = gtid(); idx < g.nn * D; idx += gstride()) {
    const int64_t i = idx % g.nn;
    v[idx] = m[i] > g.mass_eps ? u[idx] / dt : 0.0;
  }
}

// Sums of |new - old|^2 and |new|^2 over a receiver set (Eq.
// convergence_residuals), written to slot `slot` of the scalars.
template <int D, typename R>
__global__ void k_rel_change(GridGeo g, const double* vnew, const double* vold,
                             const uint8_t* recv, int slot, DevScalars* S, double* partials) {
  double acc[2] = {0.0, 0.0};
  for (int64_t idx = gtid(); idx < g.nn * D; idx += gstride()) {
    const int64_t i = idx % g.nn;
    if (!recv[i]) continue;
    const double a = vnew[idx], b = vold[idx];
    acc[0] += (a - b) * (a - b);
    acc[1] += a * a;
  }
  double tot[2];
  if (grid_sum<2>(acc, partials, &S->counter, tot) && threadIdx.x == 0) {
    S->res_num[slot] = tot[0];
    S->res_den[slot] = tot[1];
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
#define OSMPM_NB(n) (g_launch_count += 1, blocks_for(n)), kThreads, 0, s
#define OSMPM_RB(n) (g_launch_count += 1, red_blocks_for(n)), kThreads, 0, s

template <int D, typename R>
void Kernels<D, R>::morton_keys(const double* x, int64_t n, const GridGeo& g, uint64_t* keys,
                             uint32_t* vals, int* err, cudaStream_t s) {
  k_morton_keys<D, R><<<OSMPM_NB(n)>>>(x, n, g, keys, vals, err);
}
template <int D, typename R>
void Kernels<D, R>::permute(const PartPtrsT<R>& src, const PartPtrsT<R>& dst, const uint32_t* perm,
                         cudaStream_t s) {
  k_permute<D, R><<<OSMPM_NB(src.n)>>>(src, dst, perm);
}
template <int D, typename R>
void Kernels<D, R>::scatter_by_id(const PartPtrsT<R>& src, const PartPtrsT<R>& dst, cudaStream_t s) {
  k_scatter_by_id<D, R><<<OSMPM_NB(src.n)>>>(src, dst);
}
template <int D, typename R>
void Kernels<D, R>::lame(const double* E, const double* nu, PartPtrsT<R> P, cudaStream_t s) {
  k_lame<D, R><<<OSMPM_NB(P.n)>>>(E, nu, P);
}
template <int D, typename R>
void Kernels<D, R>::pack_out(const PartPtrsT<R>& P, double* x, double* v, double* B, double* F,
                          cudaStream_t s) {
  k_pack_out<D, R><<<OSMPM_NB(P.n)>>>(P, x, v, B, F);
}
template <int D, typename R>
void Kernels<D, R>::unpack_in(const double* x, const double* v, const double* B, const double* F,
                           PartPtrsT<R> dst, cudaStream_t s) {
  k_unpack_in<D, R><<<OSMPM_NB(dst.n)>>>(x, v, B, F, dst);
}
template <int D, typename R>
void Kernels<D, R>::p2g(const PartPtrsT<R>& P, const GridGeo& g, double* m, double* mv, double* bm,
                     int* err, int* sbase, R* sdn, cudaStream_t s) {
  const int64_t tiles = (P.n + TileCap<D>::THREADS - 1) / TileCap<D>::THREADS;
  g_launch_count += 1;
  k_p2g_tile<D, R><<<(int)std::min<int64_t>(std::max<int64_t>(tiles, 1), 4096), TileCap<D>::THREADS,
                     0, s>>>(P, g, m, mv, bm, err, sbase, sdn);
}
template <int D, typename R>
void Kernels<D, R>::normalize(const GridGeo& g, const double* m, const double* mv, double* vn,
                           cudaStream_t s) {
  k_normalize<D, R><<<OSMPM_RB(g.nn)>>>(g, m, mv, vn);
}
template <int D, typename R>
void Kernels<D, R>::grid_prep(const GridGeo& g, const double* m, const double* vn,
                           const PrepArgs& a, double dt, uint8_t* dofmask, double* u,
                           cudaStream_t s) {
  k_grid_prep<D, R><<<OSMPM_RB(g.nn)>>>(g, m, vn, a, dt, dofmask, u);
}
template <int D, typename R>
void Kernels<D, R>::grad(const PartPtrsT<R>& P, const GridGeo& g, const double* u,
                      const uint8_t* dofmask, double* grad, double* diag, R* L, int* err,
                      cudaStream_t s, int lmode) {
  if (lmode < 0) lmode = std::is_same<R, float>::value ? 3 : 1;
  k_grad<D, R><<<OSMPM_NB(P.n)>>>(P, g, u, dofmask, grad, diag, L, err, lmode);
}
template <int D, typename R>
void Kernels<D, R>::grad_finish(const GridGeo& g, const double* m, const double* vn,
                                const double* u, const uint8_t* dofmask, const double* gravity,
                                double dt, double cg_rtol, double eta_max, int first, int cg_max,
                                double* grad, double* diag, double* x, double* r, double* z,
                                double* p, DevScalars* S, double* partials, cudaStream_t s) {
  k_grad_finish<D, R><<<OSMPM_RB(g.nn * D)>>>(g, m, vn, u, dofmask, gravity[0], gravity[1],
                                              gravity[2], dt, cg_rtol, eta_max, first, cg_max,
                                              grad, diag, x, r, z, p, S, partials);
}
template <int D, typename R>
void Kernels<D, R>::cg_a(const GridGeo& g, const double* m, const uint8_t* dofmask, double dt,
                      const double* z, double* p, double* q, DevScalars* S, double* partials,
                      cudaStream_t s) {
  k_cg_a<D, R><<<OSMPM_RB(g.nn * D)>>>(g, m, dofmask, 1.0 / (dt * dt), z, p, q, S, partials);
}
template <int D, typename R>
void Kernels<D, R>::cg_b(const PartPtrsT<R>& P, const GridGeo& g, const uint8_t* dofmask,
                      const R* L, const double* p, double* q, DevScalars* S,
                      double* partials, cudaStream_t s) {
  k_cg_b<D, R><<<OSMPM_RB(P.n)>>>(P, g, dofmask, L, p, q, S, partials);
}
template <int D, typename R>
void Kernels<D, R>::cg_c(const GridGeo& g, const uint8_t* dofmask, const double* diag,
                      const double* p, const double* q, double* x, double* r, double* z,
                      DevScalars* S, double* partials, cudaStream_t s) {
  k_cg_c<D, R><<<OSMPM_RB(g.nn * D)>>>(g, dofmask, diag, p, q, x, r, z, S, partials);
}
template <int D, typename R>
void Kernels<D, R>::hvp_only(const PartPtrsT<R>& P, const GridGeo& g, const double* m,
                          const uint8_t* dofmask, const R* L, double dt, double* p,
                          double* q, DevScalars* S, double* partials, cudaStream_t s) {
  const double inv_dt2 = 1.0 / (dt * dt);
  k_cg_a<D, R><<<OSMPM_RB(g.nn * D)>>>(g, m, dofmask, inv_dt2, p, p, q, S, partials);
  k_cg_b<D, R><<<OSMPM_RB(P.n)>>>(P, g, dofmask, L, p, q, S, partials);
}
template <int D, typename R>
void Kernels<D, R>::maxabs(const GridGeo& g, const uint8_t* dofmask, const double* x,
                        DevScalars* S, double* partials, cudaStream_t s) {
  k_maxabs<D, R><<<OSMPM_RB(g.nn * D)>>>(g, dofmask, x, S, partials);
}
template <int D, typename R>
void Kernels<D, R>::energy_change(const PartPtrsT<R>& P, const GridGeo& g, const double* m,
                               const double* vn, const double* u, const double* x,
                               const double* gravity, double dt, double alpha, DevScalars* S,
                               double* partials, cudaStream_t s) {
  const int64_t work = P.n > g.nn * D ? P.n : g.nn * D;
  k_energy_change<D, R><<<OSMPM_RB(work)>>>(P, g, m, vn, u, x, gravity[0], gravity[1], gravity[2],
                                         dt, alpha, S, partials);
}
template <int D, typename R>
void Kernels<D, R>::energy_change_blocks(const PartPtrsT<R>& P, const GridGeo& g, const double* m,
                                      const double* vn, const double* u, const double* x,
                                      const double* gravity, double dt, double alpha,
                                      DevScalars* S, double* partials, int blocks,
                                      cudaStream_t s) {
  g_launch_count += 1;
  k_energy_change<D, R><<<blocks, kThreads, 0, s>>>(P, g, m, vn, u, x, gravity[0], gravity[1],
                                                gravity[2], dt, alpha, S, partials);
}
template <int D, typename R>
void Kernels<D, R>::split_free(const GridGeo& g, const uint8_t* dofmask, double* u, double* x,
                               cudaStream_t s) {
  k_split_free<D, R><<<OSMPM_RB(g.nn * D)>>>(g, dofmask, u, x);
}
template <int D, typename R>
void Kernels<D, R>::warm_start(const GridGeo& g, const uint8_t* dofmask, const double* src, double* u,
                            cudaStream_t s) {
  k_warm_start<D, R><<<OSMPM_RB(g.nn * D)>>>(g, dofmask, src, u);
}
template <int D, typename R>
void Kernels<D, R>::axpy(const GridGeo& g, double* u, const double* x, double alpha,
                      cudaStream_t s) {
  k_axpy<D, R><<<OSMPM_RB(g.nn * D)>>>(g, u, x, alpha);
}
template <int D, typename R>
void Kernels<D, R>::g2p(const PartPtrsT<R>& P, const GridGeo& g, const double* u, double dt,
                     cudaStream_t s) {
  k_g2p<D, R><<<OSMPM_NB(P.n)>>>(P, g, u, dt);
}
template <int D, typename R>
void Kernels<D, R>::gamma(const GridGeo& g, const double* m, const double* bm, double tau,
                       uint8_t* gam, cudaStream_t s) {
  k_gamma<D, R><<<OSMPM_RB(g.nn)>>>(g.nn, g.mass_eps, m, bm, tau, gam);
}
template <int D, typename R>
void Kernels<D, R>::arbitrate(const GridGeo& gB, const GridGeo& gS, const uint8_t* gamB,
                           const uint8_t* gamS, const double* mB, const double* mS,
                           uint8_t* recvB, uint8_t* recvS, cudaStream_t s) {
  k_arbitrate<D, R><<<OSMPM_RB(gB.nn)>>>(gB, gS, gamB, gamS, mB, mS, recvB, recvS);
}
template <int D, typename R>
void Kernels<D, R>::proj_scatter(const GridGeo& gB, const GridGeo& gS, const double* mS,
                              const double* vS, double* num, double* den, cudaStream_t s) {
  k_proj_scatter<D, R><<<OSMPM_RB(gS.nn)>>>(gB, gS, mS, vS, num, den);
}
template <int D, typename R>
void Kernels<D, R>::recvB_filter(const GridGeo& gB, const double* den, double tau,
                              const uint8_t* physB, uint8_t* recvB, cudaStream_t s) {
  k_recvB_filter<D, R><<<OSMPM_RB(gB.nn)>>>(gB.nn, den, tau, physB, recvB);
}
template <int D, typename R>
void Kernels<D, R>::recvS_filter(const GridGeo& gB, const GridGeo& gS, const double* mB,
                              const uint8_t* physS, uint8_t* recvS, cudaStream_t s) {
  k_recvS_filter<D, R><<<OSMPM_RB(gS.nn)>>>(gB, gS, mB, physS, recvS);
}
template <int D, typename R>
void Kernels<D, R>::proj_finish(const GridGeo& gB, const uint8_t* recvB, const double* num,
                             const double* den, double eps_tol, double* out, cudaStream_t s) {
  k_proj_finish<D, R><<<OSMPM_RB(gB.nn)>>>(gB, recvB, num, den, eps_tol, out);
}
template <int D, typename R>
void Kernels<D, R>::interp(const GridGeo& gB, const GridGeo& gS, const double* vB,
                        const uint8_t* recvS, double* out, cudaStream_t s) {
  k_interp<D, R><<<OSMPM_RB(gS.nn)>>>(gB, gS, vB, recvS, out);
}
template <int D, typename R>
void Kernels<D, R>::vel_from_u(const GridGeo& g, const double* m, const double* u, double dt,
                            double* v, cudaStream_t s) {
  k_vel_from_u<D, R><<<OSMPM_RB(g.nn * D)>>>(g, m, u, dt, v);
}
template <int D, typename R>
void Kernels<D, R>::rel_change(const GridGeo& g, const double* vnew, const double* vold,
                            const uint8_t* recv, int slot, DevScalars* S, double* partials,
                            cudaStream_t s) {
  k_rel_change<D, R><<<OSMPM_RB(g.nn * D)>>>(g, vnew, vold, recv, slot, S, partials);
}
template <int D, typename R>
void Kernels<D, R>::copy_if_neg(const GridGeo& g, const double* p, double* x, const DevScalars* S,
                             cudaStream_t s) {
  k_copy_if_neg<D, R><<<OSMPM_RB(g.nn * D)>>>(g, p, x, S);
}
template <int D, typename R>
void Kernels<D, R>::set_cg_state(DevScalars* S, int iter, int done, cudaStream_t s) {
  g_launch_count += 1;
  k_set_cg_state<D, R><<<1, 1, 0, s>>>(S, iter, done);
}

template <int D, typename R>
void Kernels<D, R>::pcg_shape(int64_t work, int share, int* blocks, int* threads) {
  // One block per SM while the work fits (the FP64 pipe of every SM is used
  // and each grid barrier spans as few blocks as possible); threads per
  // block sized to the work, a multiple of 32 in [64, 256]; larger problems
  // use grid-stride loops.  The grid never exceeds 1/share of the device's
  // co-resident capacity (counted in 256-thread blocks): when `share`
  // cooperative grids run concurrently they can then all be resident at
  // once, so none of their grid barriers can wait on a block that another
  // grid keeps out.  Concurrent grids (share > 1) together take at most 3/4
  // of that capacity, so a block launched late still finds room beside the
  // other pairs' ordinary kernels (at the full capacity a 256-instance batch
  // with four concurrent grids let a grid barrier run out its bounded wait).
  struct Info {
    int sms = 0, per_sm256 = 1;
  };
  static const Info info = [] {  // thread-safe one-time query (first device used)
    Info i;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&i.sms, cudaDevAttrMultiProcessorCount, dev);
    int one = 1, many = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&one, k_pcg<D, R, true>, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&many, k_pcg<D, R, false>, 256, 0);
    i.per_sm256 = one < many ? one : many;
    if (i.per_sm256 < 1) i.per_sm256 = 1;
    if (i.sms < 1) i.sms = 1;
    return i;
  }();
  if (share < 1) share = 1;
  int64_t cap = (int64_t)info.sms * info.per_sm256 / share;
  if (share > 1) cap = cap * 3 / 4;
  if (cap < 1) cap = 1;
  const int64_t sms_share = info.sms / share > 0 ? info.sms / share : 1;
  int64_t t = (work + sms_share - 1) / sms_share;
  t = ((t + 31) / 32) * 32;
  if (t < 64) t = 64;
  if (t > 256) t = 256;
  int64_t b = (work + t - 1) / t;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  *blocks = (int)b;
  *threads = (int)t;
}
template <int D, typename R>
cudaError_t Kernels<D, R>::pcg(const PcgArgsT<R>& a, int blocks, int threads, cudaStream_t s) {
  PcgArgsT<R> copy = a;
  void* args[] = {(void*)&copy};
  g_launch_count += 1;
  // the single-pass variant when every thread owns at most one DOF and every
  // lane at most one particle
  return cudaLaunchCooperativeKernel(pcg_kernel(a, blocks, threads), dim3(blocks), dim3(threads),
                                     args, 0, s);
}
template <int D, typename R>
const void* Kernels<D, R>::pcg_kernel(const PcgArgsT<R>& a, int blocks, int threads) {
  return pcg_one_pass(a, blocks, threads) ? (const void*)k_pcg<D, R, true>
                                          : (const void*)k_pcg<D, R, false>;
}
template <int D, typename R>
bool Kernels<D, R>::pcg_one_pass(const PcgArgsT<R>& a, int blocks, int threads) {
  const int64_t ndof = a.g.nn * D;
  const int64_t chunk = (ndof + blocks - 1) / blocks;
  const int64_t groups = (a.P.n + HvpGroup<D>::GP - 1) / HvpGroup<D>::GP;
  return chunk <= threads && groups <= (int64_t)blocks * threads / 32;
}
template <int D, typename R>
int64_t Kernels<D, R>::pcg_passes(const PcgArgsT<R>& a, int blocks, int threads) {
  const int64_t ndof = a.g.nn * D;
  const int64_t dpass = (ndof + (int64_t)blocks * threads - 1) / ((int64_t)blocks * threads);
  const int64_t warps = (int64_t)blocks * threads / 32;
  const int64_t groups = (a.P.n + HvpGroup<D>::GP - 1) / HvpGroup<D>::GP;
  const int64_t ppass = (groups + warps - 1) / warps;
  return dpass > ppass ? dpass : ppass;
}
template <int D, typename R>
void Kernels<D, R>::cgs_start(const PcgArgsT<R>& a, cudaStream_t s) {
  k_cgs_start<D, R><<<OSMPM_RB(a.g.nn * D)>>>(a);
}
template <int D, typename R>
void Kernels<D, R>::cgs_iteration(const PcgArgsT<R>& a, int hvp_mode, cudaStream_t s,
                                  cudaEvent_t e0, cudaEvent_t e1) {
  if (e0) cudaEventRecord(e0, s);
  cgs_hvp(a, hvp_mode, s);
  if (e1) cudaEventRecord(e1, s);
  k_cgs_alpha<D, R><<<OSMPM_RB(a.g.nn * D)>>>(a);
  k_cgs_beta<D, R><<<OSMPM_RB(a.g.nn * D)>>>(a);
}
template <int D, typename R>
void Kernels<D, R>::cgs_hvp(const PcgArgsT<R>& a, int hvp_mode, cudaStream_t s) {
  bool tiled = false;
  if constexpr (std::is_same<R, float>::value) {
    if (hvp_mode != 1) {
      // tiles over the slot capacity; the kernel reads the slot count
      const int64_t tiles = ((int64_t)(1 << D) * a.P.n + TileCap<D>::THREADS - 1) / TileCap<D>::THREADS;
      const int blocks = (int)std::min<int64_t>(std::max<int64_t>(tiles, 1), kRedBlocksMax);
      g_launch_count += 1;
      k_cgs_hvp_tile<D><<<blocks, TileCap<D>::THREADS, 0, s>>>(a);
      tiled = true;
    }
  }
  if (!tiled) {
    const int64_t lanes = (a.P.n + HvpGroup<D>::GP - 1) / HvpGroup<D>::GP * 32;
    k_cgs_hvp<D, R><<<OSMPM_RB(lanes)>>>(a);
  }
}

template <int D, typename R>
void Kernels<D, R>::plane_colmin(const PartPtrsT<R>& P, const GridGeo& g, double spacing,
                                 unsigned long long* colmin, cudaStream_t s) {
  k_plane_colmin<D, R><<<OSMPM_NB(P.n)>>>(P, g, spacing, colmin);
}
template <int D, typename R>
void Kernels<D, R>::plane_init(const GridGeo& g, const double* m, const uint8_t* physmask,
                               const unsigned long long* colmin, double level, double cand_hi,
                               double spacing, double dt, double* gap, double* hold_v,
                               uint8_t* cand, uint8_t* act, cudaStream_t s) {
  k_plane_init<D, R><<<OSMPM_RB(g.nn)>>>(g, m, physmask, colmin, level, cand_hi, spacing, dt, gap,
                                         hold_v, cand, act);
}
template <int D, typename R>
void Kernels<D, R>::mask_all(const GridGeo& g, const double* m, uint8_t* mask, cudaStream_t s) {
  k_mask_all<D, R><<<OSMPM_RB(g.nn)>>>(g, m, mask);
}
template <int D, typename R>
void Kernels<D, R>::plane_update(const GridGeo& g, const uint8_t* cand, const double* grad,
                                 const double* u, const double* gap, uint8_t* act, double* lam,
                                 int* changes, cudaStream_t s) {
  k_plane_update<D, R><<<OSMPM_RB(g.nn)>>>(g, cand, grad, u, gap, act, lam, changes);
}
template <int D, typename R>
void Kernels<D, R>::barrier_timeout_check(unsigned* words, int* err, cudaStream_t s) {
  g_launch_count += 1;
  k_barrier_timeout_check<D, R><<<2, 32, 0, s>>>(words, err);
}

template <int D, typename R>
void Kernels<D, R>::build_slots(const int* sbase, int64_t n, int* rs, int* flag, int* gsum,
                                int* bsum, int* slot2p, int64_t slot_cap, int* n_slots,
                                cudaStream_t s) {
  constexpr int GL = 1 << D;
  cudaMemsetAsync(slot2p, 0xFF, sizeof(int) * slot_cap, s);
  cudaMemsetAsync(n_slots, 0, sizeof(int), s);
  if (n <= 0) return;
  const int nb = (int)((n + kScanItems - 1) / kScanItems);
  const int blocks = blocks_for(n);
  g_launch_count += 9;
  k_slot_starts<GL><<<blocks, kThreads, 0, s>>>(sbase, n, rs);
  k_scan_block<true><<<nb, 256, 0, s>>>(rs, rs, n, bsum);
  k_scan_top<true><<<1, 256, 0, s>>>(bsum, nb);
  k_scan_add<true><<<blocks, kThreads, 0, s>>>(rs, n, bsum);
  k_slot_flags<GL><<<blocks, kThreads, 0, s>>>(rs, n, flag);
  k_scan_block<false><<<nb, 256, 0, s>>>(flag, gsum, n, bsum);
  k_scan_top<false><<<1, 256, 0, s>>>(bsum, nb);
  k_scan_add<false><<<blocks, kThreads, 0, s>>>(gsum, n, bsum);
  k_slot_fill<GL><<<blocks, kThreads, 0, s>>>(rs, gsum, flag, n, slot2p, n_slots);
}

template <int D>
void MultiKernels<D>::start(const MultiArgs* mp, int grid_dt, cudaStream_t s) {
  g_launch_count += 1;
  k_m_start<D><<<grid_dt, kThreads, 0, s>>>(mp);
}
template <int D>
void MultiKernels<D>::iteration(const MultiArgs* mp, int grid_pt, int grid_dt, cudaStream_t s,
                                cudaEvent_t e0, cudaEvent_t e1, bool capturing) {
  g_launch_count += 2;
  const unsigned flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (e0) cudaEventRecordWithFlags(e0, s, flags);
  k_m_hvp<D><<<grid_pt, TileCap<D>::THREADS, 0, s>>>(mp);
  if (e1) cudaEventRecordWithFlags(e1, s, flags);
  k_m_update<D><<<grid_dt, kThreads, 0, s>>>(mp);
}
template <int D>
void MultiKernels<D>::pending(const MultiArgs* mp, cudaStream_t s) {
  g_launch_count += 1;
  k_m_pending<D><<<1, kThreads, 0, s>>>(mp);
}
template <int D>
int MultiKernels<D>::particle_tile() {
  return TileCap<D>::THREADS;
}
template <int D>
int MultiKernels<D>::hvp_blocks_per_sm() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_m_hvp<D>, TileCap<D>::THREADS, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return TileCap<D>::MIN_BLOCKS;
  }
  return b;
}

#undef OSMPM_NB
#undef OSMPM_RB

}  // namespace osmpm
