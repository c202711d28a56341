// Unilateral frictionless contact with a rigid plane y = level (the rigid
// plane of Sec. 4.2; the paper gives no treatment, the reading is a
// gap-aware Signorini condition on the normal motion of the grid nodes at or
// below the plane): over one implicit step u_iy >= -gap_i on the candidate
// nodes, with gap_i the height of the body's lowest particle over node i's
// column (within one particle spacing in x) minus half a spacing above the
// plane.  The host solves it by a primal-dual active set: held nodes get
// u_iy = -gap_i as Dirichlet data, their multipliers lambda_i = dE_h/du_iy
// come from the gradient with every active DOF free, and the set changes by
// releasing held nodes with lambda_i < 0 and holding free nodes that moved
// past -gap_i.  Two-dimensional.  Included by osmpm_kernels.cuh.
#pragma once

#include "osmpm_device.cuh"

namespace osmpm {

// Order-preserving map of a double onto unsigned 64-bit integers (for
// atomicMin over positions of either sign).
__device__ __forceinline__ unsigned long long order_key(double y) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double order_value(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}
constexpr unsigned long long kNoParticle = ~0ull;

// Per grid column i (x fastest): the lowest particle height among the
// particles with |x_p - x_i| <= spacing (x_i = o_x + i dx, rounded as on the
// host); colmin starts at kNoParticle.
template <int D, typename R>
__global__ void k_plane_colmin(PartPtrsT<R> P, GridGeo g, double spacing,
                               unsigned long long* colmin) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const double x = P.x[p], y = P.x[P.n + p];
  const double t = (x - g.o[0]) * g.inv_dx;
  const double w = spacing * g.inv_dx;
  int lo = (int)floor(t - w) - 1, hi = (int)ceil(t + w) + 1;
  lo = lo < 0 ? 0 : lo;
  hi = hi > g.res[0] - 1 ? g.res[0] - 1 : hi;
  const unsigned long long key = order_key(y);
  for (int i = lo; i <= hi; ++i) {
    const double xi = __dadd_rn(g.o[0], __dmul_rn((double)i, g.dx));
    if (fabs(__dsub_rn(x, xi)) <= spacing) atomicMin(&colmin[i], key);
  }
}

// Candidates (nodes with y_i <= cand_hi, active, without a physical rule on
// y, with a particle over their column), their gaps
// max(0, (y_min - spacing/2) - level), the prescribed y velocity -gap/dt of a
// held node, and the initial active set (the closed gaps).
template <int D, typename R>
__global__ void k_plane_init(GridGeo g, const double* m, const uint8_t* physmask,
                             const unsigned long long* colmin, double level, double cand_hi,
                             double spacing, double dt, double* gap, double* hold_v,
                             uint8_t* cand, uint8_t* act) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.nn;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % g.res[0]);
    const int iy = (int)((i / g.res[0]) % g.res[1]);
    const double yi = __dadd_rn(g.o[1], __dmul_rn((double)iy, g.dx));
    bool c = yi <= cand_hi && m[i] > g.mass_eps && !(physmask[i] & 2u);
    double gp = INFINITY;
    const unsigned long long k = colmin[ix];
    if (k != kNoParticle) gp = fmax(0.0, __dsub_rn(__dsub_rn(order_value(k), 0.5 * spacing), level));
    c = c && isfinite(gp);
    gap[i] = c ? gp : INFINITY;
    hold_v[i] = c ? -gp / dt : 0.0;
    cand[i] = c ? 1 : 0;
    act[i] = (c && gp <= 0.0) ? 1 : 0;
  }
}

// Every active node's DOFs free (the multipliers need the gradient on the
// held ones too).
template <int D, typename R>
__global__ void k_mask_all(GridGeo g, const double* m, uint8_t* mask) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.nn;
       i += (int64_t)gridDim.x * blockDim.x)
    mask[i] = m[i] > g.mass_eps ? (uint8_t)((1u << D) - 1u) : (uint8_t)0;
}

// Multipliers lambda_i = dE_h/du_iy on the held nodes (0 elsewhere) from the
// full gradient, and the active-set update: release held nodes with
// lambda_i < 0, hold free candidates with u_iy < -gap_i; counts the changes.
template <int D, typename R>
__global__ void k_plane_update(GridGeo g, const uint8_t* cand, const double* grad,
                               const double* u, const double* gap, uint8_t* act, double* lam,
                               int* changes) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.nn;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!cand[i]) {
      lam[i] = 0.0;
      continue;
    }
    const bool held = act[i] != 0;
    const double l = held ? grad[g.nn + i] : 0.0;
    lam[i] = l;
    const bool release = held && l < 0.0;
    const bool enter = !held && u[g.nn + i] < -gap[i];
    if (release || enter) {
      act[i] = held ? 0 : 1;
      atomicAdd(changes, 1);
    }
  }
}

}  // namespace osmpm
