// Device building blocks of the OS-MPM hot path (sm_103a): grid geometry,
// the quadratic B-spline stencil, the neo-Hookean law and deterministic
// block reductions.  Everything is FP64.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "osmpm_types.h"

namespace osmpm {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Quadratic B-spline stencil (Sec. 2.2.2).  base = floor((x - o)/dx - 1/2)
// is formed with explicitly rounded FP64 operations (no fused multiply-add),
// so the node indexing is reproducible bit for bit on any IEEE host.  With
// fx = t - base in [1/2, 3/2) the three weights along an axis are
// (3/2 - fx)^2/2, 3/4 - (fx - 1)^2, (fx - 1/2)^2/2.
// ---------------------------------------------------------------------------
template <int D>
struct Stencil {
  int base[D];
  double w[D][3];
  double dw[D][3];  // d w / d x (includes 1/dx)
};

template <int D>
__device__ __forceinline__ bool make_stencil(const double* xp, const GridGeo& g, Stencil<D>& s) {
  bool ok = true;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const double t = __dmul_rn(__dsub_rn(xp[a], g.o[a]), g.inv_dx);
    const double b = floor(__dsub_rn(t, 0.5));
    ok = ok && (b >= 0.0) && (b + 2.0 < (double)g.res[a]);
    const int bi = ok ? (int)b : 0;
    s.base[a] = bi;
    const double fx = t - b;
    const double e0 = 1.5 - fx, e1 = fx - 1.0, e2 = fx - 0.5;
    s.w[a][0] = 0.5 * e0 * e0;
    s.w[a][1] = 0.75 - e1 * e1;
    s.w[a][2] = 0.5 * e2 * e2;
    s.dw[a][0] = -e0 * g.inv_dx;
    s.dw[a][1] = -2.0 * e1 * g.inv_dx;
    s.dw[a][2] = e2 * g.inv_dx;
  }
  return ok;
}

// Stencil node k (0 <= k < 3^D, x fastest): flat node index, weight N and
// gradient dN.
template <int D>
__device__ __forceinline__ int64_t stencil_node(const Stencil<D>& s, const GridGeo& g, int k,
                                                double& N, double* dN) {
  int off[3];
  off[0] = k % 3;
  off[1] = (k / 3) % 3;
  off[2] = k / 9;
  int64_t flat = 0, stride = 1;
  N = 1.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    flat += (int64_t)(s.base[a] + off[a]) * stride;
    stride *= g.res[a];
    N *= s.w[a][off[a]];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double v = s.dw[a][off[a]];
#pragma unroll
    for (int b = 0; b < D; ++b)
      if (b != a) v *= s.w[b][off[b]];
    dN[a] = v;
  }
  return flat;
}

// Position of stencil node k along axis a: o + (base + off) dx, rounded as
// o + (i dx) without contraction.
template <int D>
__device__ __forceinline__ double stencil_node_pos(const Stencil<D>& s, const GridGeo& g, int k,
                                                   int a) {
  const int off = (a == 0) ? (k % 3) : (a == 1 ? (k / 3) % 3 : k / 9);
  return __dadd_rn(g.o[a], __dmul_rn((double)(s.base[a] + off), g.dx));
}

__device__ __forceinline__ double node_pos(const GridGeo& g, int64_t i, int a) {
  int64_t idx = i;
  int c = 0;
  for (int b = 0; b <= a; ++b) {
    c = (int)(idx % g.res[b]);
    idx /= g.res[b];
  }
  return __dadd_rn(g.o[a], __dmul_rn((double)c, g.dx));
}

// ---------------------------------------------------------------------------
// Small dense algebra, row-major D x D.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ double det_minus_one(const double* H) {
  // det(I + H) - 1 expanded in H, so that small strains do not cancel
  if (D == 2) {
    return (H[0] + H[3]) + (H[0] * H[3] - H[1] * H[2]);
  } else {
    const double tr = H[0] + H[4] + H[8];
    const double m2 = (H[0] * H[4] - H[1] * H[3]) + (H[0] * H[8] - H[2] * H[6]) +
                      (H[4] * H[8] - H[5] * H[7]);
    const double dH = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                      H[2] * (H[3] * H[7] - H[4] * H[6]);
    return tr + m2 + dH;
  }
}

// Inverse transpose of F given J = det F.
template <int D>
__device__ __forceinline__ void inv_transpose(const double* F, double J, double* FiT) {
  const double r = 1.0 / J;
  if (D == 2) {
    FiT[0] = F[3] * r;
    FiT[1] = -F[2] * r;
    FiT[2] = -F[1] * r;
    FiT[3] = F[0] * r;
  } else {
    // cofactor matrix / J
    FiT[0] = (F[4] * F[8] - F[5] * F[7]) * r;
    FiT[1] = (F[5] * F[6] - F[3] * F[8]) * r;
    FiT[2] = (F[3] * F[7] - F[4] * F[6]) * r;
    FiT[3] = (F[2] * F[7] - F[1] * F[8]) * r;
    FiT[4] = (F[0] * F[8] - F[2] * F[6]) * r;
    FiT[5] = (F[1] * F[6] - F[0] * F[7]) * r;
    FiT[6] = (F[1] * F[5] - F[2] * F[4]) * r;
    FiT[7] = (F[2] * F[3] - F[0] * F[5]) * r;
    FiT[8] = (F[0] * F[4] - F[1] * F[3]) * r;
  }
}

// Neo-Hookean state at F: Psi, ln J and F^-T.  Returns false when J <= 0
// (the energy is +inf there).
template <int D>
struct NeoHookean {
  double lnJ;
  double FiT[D * D];
  double psi;
};

template <int D>
__device__ __forceinline__ bool neo_hookean(const double* F, double mu, double lam,
                                            NeoHookean<D>& s) {
  double H[D * D];
#pragma unroll
  for (int i = 0; i < D * D; ++i) H[i] = F[i] - ((i % (D + 1)) == 0 ? 1.0 : 0.0);
  const double jm1 = det_minus_one<D>(H);
  if (!(jm1 > -1.0)) return false;
  s.lnJ = log1p(jm1);
  double trH = 0.0, hh = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) trH += H[a * (D + 1)];
#pragma unroll
  for (int i = 0; i < D * D; ++i) hh += H[i] * H[i];
  s.psi = 0.5 * mu * (2.0 * trH + hh) - mu * s.lnJ + 0.5 * lam * s.lnJ * s.lnJ;
  inv_transpose<D>(F, 1.0 + jm1, s.FiT);
  return true;
}

// det(F0 + dF) - det(F0) as a polynomial in dF (exact identity).
template <int D>
__device__ __forceinline__ double det_change(const double* A, const double* B) {
  if (D == 2) {
    return A[0] * B[3] + B[0] * A[3] - A[1] * B[2] - B[1] * A[2] + (B[0] * B[3] - B[1] * B[2]);
  } else {
    // cof(A):B + A:cof(B) + det B, cof rows = cross products of the other rows
    double cA[9], cB[9];
    const int r1[3] = {1, 2, 0}, r2[3] = {2, 0, 1};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double* a1 = A + 3 * r1[i];
      const double* a2 = A + 3 * r2[i];
      const double* b1 = B + 3 * r1[i];
      const double* b2 = B + 3 * r2[i];
      cA[3 * i + 0] = a1[1] * a2[2] - a1[2] * a2[1];
      cA[3 * i + 1] = a1[2] * a2[0] - a1[0] * a2[2];
      cA[3 * i + 2] = a1[0] * a2[1] - a1[1] * a2[0];
      cB[3 * i + 0] = b1[1] * b2[2] - b1[2] * b2[1];
      cB[3 * i + 1] = b1[2] * b2[0] - b1[0] * b2[2];
      cB[3 * i + 2] = b1[0] * b2[1] - b1[1] * b2[0];
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) s += cA[i] * B[i] + A[i] * cB[i];
    const double detB = B[0] * cB[0] + B[1] * cB[1] + B[2] * cB[2];
    return s + detB;
  }
}

// Psi(F0 + dF) - Psi(F0) through exact difference identities, so that its
// rounding error scales with dF:  mu (F0:dF + |dF|^2/2) - mu dl
// + lam/2 dl (2 ln J0 + dl), dl = log1p(dJ / J0).  False when J0 <= 0 or
// J0 + dJ <= 0 (the energy change is +inf).
template <int D>
__device__ __forceinline__ bool psi_change(const double* F0, const double* dF, double mu,
                                           double lam, double& out) {
  double H[D * D];
#pragma unroll
  for (int i = 0; i < D * D; ++i) H[i] = F0[i] - ((i % (D + 1)) == 0 ? 1.0 : 0.0);
  const double jm1 = det_minus_one<D>(H);
  const double J0 = 1.0 + jm1;
  const double dJ = det_change<D>(F0, dF);
  if (!(J0 > 0.0) || !(J0 + dJ > 0.0)) return false;
  const double dl = log1p(dJ / J0);
  const double lnJ0 = log1p(jm1);
  double fd = 0.0, dd = 0.0;
#pragma unroll
  for (int i = 0; i < D * D; ++i) {
    fd += F0[i] * dF[i];
    dd += dF[i] * dF[i];
  }
  out = mu * (fd + 0.5 * dd) - mu * dl + 0.5 * lam * dl * (2.0 * lnJ0 + dl);
  return true;
}

// First Piola-Kirchhoff stress P = mu (F - F^-T) + lam ln J F^-T.
template <int D>
__device__ __forceinline__ void pk1(const double* F, double mu, double lam, const NeoHookean<D>& s,
                                    double* P) {
#pragma unroll
  for (int i = 0; i < D * D; ++i) P[i] = mu * (F[i] - s.FiT[i]) + lam * s.lnJ * s.FiT[i];
}

// dP[dF] = mu dF + (mu - lam ln J) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T.
template <int D>
__device__ __forceinline__ void dpdf_apply(const double* dF, double mu, double lam,
                                           const NeoHookean<D>& s, double* out) {
  const double* A = s.FiT;
  // tr(F^-1 dF) = F^-T : dF
  double tr = 0.0;
#pragma unroll
  for (int i = 0; i < D * D; ++i) tr += A[i] * dF[i];
  const double c1 = mu - lam * s.lnJ;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      // (A dF^T A)_ac = sum_e,f A_ae dF_fe A_fc
      double t = 0.0;
#pragma unroll
      for (int e = 0; e < D; ++e)
#pragma unroll
        for (int f = 0; f < D; ++f) t += A[a * D + e] * dF[f * D + e] * A[f * D + c];
      out[a * D + c] = mu * dF[a * D + c] + c1 * t + lam * tr * A[a * D + c];
    }
}

// Packed upper triangle of a symmetric (D*D) x (D*D) matrix.
template <int D>
struct Sym {
  static constexpr int n = D * D;
  static constexpr int packed = n * (n + 1) / 2;
  __host__ __device__ static constexpr int idx(int i, int j) {
    return i <= j ? i * n - i * (i - 1) / 2 + (j - i) : j * n - j * (j - 1) / 2 + (i - j);
  }
};

// ---------------------------------------------------------------------------
// Deterministic reductions.  Every block reduces its values, writes them to
// a partials array and bumps a counter; the last block to arrive sums the
// partials in block order, writes the totals and resets the counter.  The
// result depends only on the launch shape, not on scheduling.
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(kFull, v[k], off);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = lane < (int)(blockDim.x >> 5) ? sh[k][lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(kFull, v[k], off);
    }
  }
}

__device__ __forceinline__ double block_max(double v) {
  __shared__ double sh[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(kFull, v, off));
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(kFull, v, off));
  }
  return v;
}

// Sum reduction across the grid; returns true in the last block, where
// `total` holds the grid-wide sums (valid in every thread of that block).
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials, unsigned* counter,
                                         double (&total)[NV]) {
  __shared__ bool is_last;
  __shared__ double tot_sh[NV];
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[k * gridDim.x + blockIdx.x] = v[k];
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(&partials[k * gridDim.x + b]);
  block_sum<NV>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) tot_sh[k] = acc[k];
    *counter = 0u;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) total[k] = tot_sh[k];
  return true;
}

__device__ __forceinline__ bool grid_max(double v, double* partials, unsigned* counter,
                                         double& total) {
  __shared__ bool is_last;
  __shared__ double tot_sh;
  v = block_max(v);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v;
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double acc = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
    acc = fmax(acc, __ldcg(&partials[b]));
  acc = block_max(acc);
  if (threadIdx.x == 0) {
    tot_sh = acc;
    *counter = 0u;
  }
  __syncthreads();
  total = tot_sh;
  return true;
}

}  // namespace osmpm
