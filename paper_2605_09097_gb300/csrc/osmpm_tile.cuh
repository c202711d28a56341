// Block-tiled particle kernels: each block takes a run of Morton-sorted
// particles, finds the bounding box of their stencils (a few hundred grid
// nodes) and stages that box of the grid in shared memory.  Gathers then read
// shared memory, and the scatter accumulates into a shared tile that is
// flushed with one global atomic per (tile node, component) instead of one
// per (particle, stencil node, component).  A block whose box is larger than
// the tile capacity (a Morton run that jumps across a high-level boundary)
// works on global memory directly, with the same arithmetic.
//
// Included by osmpm_kernels.cuh.
#pragma once

#include <climits>
#include <type_traits>

#include "osmpm_device.cuh"

namespace osmpm {

// Tile shape per dimension: threads per block (one slot or particle each),
// shared tile capacity in nodes, and resident blocks per SM the register
// budget is set for (2D: 64 registers, 8 blocks of 4 warps; 3D: 96
// registers, 5 blocks).  Several small tiles per SM keep independent
// load chains in flight: a tile's particle data depend on its slot map,
// and its node box on those.
template <int D>
struct TileCap {
  static constexpr int NODES = (D == 2) ? 512 : 768;
  static constexpr int THREADS = 128;
  static constexpr int MIN_BLOCKS = (D == 2) ? 8 : 5;
};

// Geometry of one block's tile: the box [lo, lo + ext) of grid nodes.
template <int D>
struct TileBox {
  int lo[3];
  int ext[3];
  int nodes;  // ext product, or 0 when the box exceeds the capacity
};

// Flat index of a tile-local node (x fastest).
template <int D>
__device__ __forceinline__ int tile_local(const TileBox<D>& t, int i0, int i1, int i2) {
  if constexpr (D == 2) return i0 + t.ext[0] * i1;
  return i0 + t.ext[0] * (i1 + t.ext[1] * i2);
}

// Global flat node index of tile-local node `l`.
template <int D>
__device__ __forceinline__ int64_t tile_global(const TileBox<D>& t, const GridGeo& g, int l) {
  const int i0 = l % t.ext[0];
  const int r = l / t.ext[0];
  if constexpr (D == 2) return (int64_t)(t.lo[0] + i0) + (int64_t)g.res[0] * (t.lo[1] + r);
  const int i1 = r % t.ext[1];
  const int i2 = r / t.ext[1];
  return (int64_t)(t.lo[0] + i0) +
         (int64_t)g.res[0] * ((int64_t)(t.lo[1] + i1) + (int64_t)g.res[1] * (t.lo[2] + i2));
}

// The block's tile box from its particles' base nodes (valid lanes only);
// every thread gets the same box in `out` (shared).  nodes = 0 when the box
// needs more than `cap` nodes or the block has no valid particle.
template <int D>
__device__ __forceinline__ void tile_box(const int (&base)[D], bool valid, int cap,
                                         TileBox<D>& out) {
  __shared__ int smin[3][32], smax[3][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int mn = valid ? base[a] : INT_MAX;
    int mx = valid ? base[a] : INT_MIN;
    mn = __reduce_min_sync(kFull, mn);
    mx = __reduce_max_sync(kFull, mx);
    if (lane == 0) {
      smin[a][warp] = mn;
      smax[a][warp] = mx;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long nodes = 1;
    bool any = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      int mn = INT_MAX, mx = INT_MIN;
      for (int w = 0; w < nw; ++w) {
        mn = min(mn, smin[a][w]);
        mx = max(mx, smax[a][w]);
      }
      any = any && (mx >= mn);
      out.lo[a] = mn;
      out.ext[a] = any ? mx - mn + 3 : 0;
      nodes *= any ? (long long)(mx - mn + 3) : 0ll;
    }
    for (int a = D; a < 3; ++a) {
      out.lo[a] = 0;
      out.ext[a] = 1;
    }
    out.nodes = (any && nodes <= cap) ? (int)nodes : 0;
  }
  __syncthreads();
}

// Per-particle data of the tiled product, written by the gradient kernel at
// each Newton iterate (FP32, entry e of particle p at [(off + e) n + p] past
// the packed Hessian blocks): A = F_hat^-T (D*D), c1 = V0 (mu - lam ln J),
// V0 mu, V0 lam, and the particle's offset from its stencil base in cells
// (D values, t - base with t = (x - o)/dx), so that the product reads no
// FP64 particle data.
template <int D>
struct TileX {
  static constexpr int A = 0;
  static constexpr int C1 = D * D;
  static constexpr int MU = D * D + 1;
  static constexpr int LAM = D * D + 2;
  static constexpr int FX = D * D + 3;
  static constexpr int N = D * D + 3 + D;
  static_assert(N == tile_x_count(D), "TileX layout");
};

// Conversions between FP32 and FP64 on the integer pipes, from the IEEE-754
// fields (the GB300's FP64 pipe issues one warp instruction per 16 SM
// cycles, so a conversion there costs as much as a few dozen integer
// operations).  float -> double is exact for normal numbers and zero;
// subnormal floats become signed zero; inf and NaN keep their class.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned m = u & 0x7FFFFFu;
  const unsigned eh = e == 0u ? 0u : (e == 0xFFu ? 0x7FFu : e + 896u);  // rebias 127 -> 1023
  const unsigned hi = (u & 0x80000000u) | (eh << 20) | (e == 0u ? 0u : m >> 3);
  const unsigned lo = e == 0u ? 0u : m << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// double -> float rounded to nearest even; magnitudes below the smallest
// normal float become signed zero, above the largest inf; NaN stays NaN.
__device__ __forceinline__ float d2f_bits(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned s = hi & 0x80000000u;
  const unsigned ef = (hi >> 20) & 0x7FFu;
  const int e = (int)ef - 896;
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // the top 23 mantissa bits
  const unsigned rest = lo & 0x1FFFFFFFu;                  // the 29 bits rounded off
  const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  unsigned r;
  if (e <= 0) r = s;
  else if (e >= 0xFF) r = s | ((ef == 0x7FFu && ((hi & 0xFFFFFu) | lo)) ? 0x7FC00000u : 0x7F800000u);
  else r = s | (((unsigned)e << 23) + m + up);  // a carry out of m rounds into the exponent
  return __uint_as_float(r);
}

// Quadratic B-spline weights of one particle in FP32 from its offsets fx
// (t - base per axis, in [0.5, 1.5)).
template <int D>
__device__ __forceinline__ void stencil_fx(const float (&fx)[D], float inv_dx, float (&w)[D][3],
                                           float (&dw)[D][3]) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const float e0 = 1.5f - fx[a], e1 = fx[a] - 1.0f, e2 = fx[a] - 0.5f;
    w[a][0] = 0.5f * e0 * e0;
    w[a][1] = 0.75f - e1 * e1;
    w[a][2] = 0.5f * e2 * e2;
    dw[a][0] = -e0 * inv_dx;
    dw[a][1] = -2.0f * e1 * inv_dx;
    dw[a][2] = e2 * inv_dx;
  }
}

// Per-axis base node from the flat index b0 + res0 (b1 + res1 b2).
template <int D>
__device__ __forceinline__ void unflatten_base(int sb, const GridGeo& g, int (&base)[D]) {
  const unsigned u = (unsigned)sb;
  if constexpr (D == 2) {
    base[1] = (int)(u / (unsigned)g.res[0]);
    base[0] = (int)(u - (unsigned)base[1] * (unsigned)g.res[0]);
  } else {
    const unsigned r = u / (unsigned)g.res[0];
    base[0] = (int)(u - r * (unsigned)g.res[0]);
    base[2] = (int)(r / (unsigned)g.res[1]);
    base[1] = (int)(r - (unsigned)base[2] * (unsigned)g.res[1]);
  }
}

// The weights of stencil layer o2 (the z offset; 1 and 0 in 2D) by
// selects, so that a loop over the layers need not index the register
// arrays with a run-time value.
template <int D>
__device__ __forceinline__ void layer_weights(const float (&w)[D][3], const float (&dw)[D][3], int o2,
                                              float& wz, float& dwz) {
  if constexpr (D == 2) {
    wz = 1.0f;
    dwz = 0.0f;
  } else {
    wz = o2 == 0 ? w[2][0] : (o2 == 1 ? w[2][1] : w[2][2]);
    dwz = o2 == 0 ? dw[2][0] : (o2 == 1 ? dw[2][1] : dw[2][2]);
  }
}

// grad N of stencil node (o0, o1) of a layer with weights wz, dwz
// (products left to right: the x factor, the y factor, the layer's).
template <int D>
__device__ __forceinline__ void grad_n_layer(const float (&w)[D][3], const float (&dw)[D][3], int o0,
                                             int o1, float wz, float dwz, float (&dN)[D]) {
  if constexpr (D == 2) {
    dN[0] = dw[0][o0] * w[1][o1];
    dN[1] = w[0][o0] * dw[1][o1];
  } else {
    dN[0] = dw[0][o0] * w[1][o1] * wz;
    dN[1] = w[0][o0] * dw[1][o1] * wz;
    dN[2] = w[0][o0] * w[1][o1] * dwz;
  }
}

// Reduce-scatter over an aligned group of L lanes (L a power of two, NV a
// multiple of L): afterwards lane r of the group holds, in v[0 .. NV/L), the
// group's sums of the values r NV/L .. (r + 1) NV/L - 1.  Recursive halving:
// at distance h a lane keeps the half of its current segment selected by
// (r & h), sends the other half to lane r ^ h and adds what it receives.
template <int L, int NV>
__device__ __forceinline__ void group_reduce_scatter(float (&v)[NV], int r) {
  static_assert(NV % L == 0, "NV must be a multiple of L");
#pragma unroll
  for (int h = L / 2, seg = NV; h >= 1; h >>= 1, seg >>= 1) {
    const bool upper = (r & h) != 0;
#pragma unroll
    for (int i = 0; i < seg / 2; ++i) {
      const float send = upper ? v[i] : v[i + seg / 2];
      const float keep = upper ? v[i + seg / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, h);
    }
  }
}

// The particle Hessian in FP32 at the Newton iterate's deformation
// gradient F_hat, from the data the gradient kernel stored there (computed
// in FP64): dF = G_d F^n and Y = V0 dP[F_hat; dF] F^nT with
//   V0 dP[dF] = V0 mu dF + c1 A dF^T A + V0 lam tr(A^T dF) A,
//   A = F_hat^-T,  c1 = V0 (mu - lam ln J)
// (the operator of the cached block L(G) = V0 dP[G F^n] F^nT of the
// gradient kernel).  Returns G_d : Y, the particle's share of d.Kd.
template <int D>
__device__ __forceinline__ float hessian_apply_x(const float (&A)[D * D], float c1, float vmu,
                                                 float vlam, const float (&Gd)[D * D],
                                                 const float (&Fn)[D * D], float (&Y)[D * D]) {
  constexpr int DD = D * D;
  float dF[DD];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      float t = 0.0f;
#pragma unroll
      for (int c = 0; c < D; ++c) t = fmaf(Gd[a * D + c], Fn[c * D + b], t);
      dF[a * D + b] = t;
    }
  float tr = 0.0f;
#pragma unroll
  for (int i = 0; i < DD; ++i) tr = fmaf(A[i], dF[i], tr);
  const float c2 = vlam * tr;
  float Bm[DD];  // dF^T A
#pragma unroll
  for (int e = 0; e < D; ++e)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float t = 0.0f;
#pragma unroll
      for (int f = 0; f < D; ++f) t = fmaf(dF[f * D + e], A[f * D + c], t);
      Bm[e * D + c] = t;
    }
  float dP[DD];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float t = 0.0f;
#pragma unroll
      for (int e = 0; e < D; ++e) t = fmaf(A[a * D + e], Bm[e * D + c], t);
      dP[a * D + c] = fmaf(vmu, dF[a * D + c], fmaf(c1, t, c2 * A[a * D + c]));
    }
  float qf = 0.0f;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float t = 0.0f;
#pragma unroll
      for (int b = 0; b < D; ++b) t = fmaf(dP[a * D + b], Fn[c * D + b], t);
      Y[a * D + c] = t;
      qf = fmaf(Gd[a * D + c], t, qf);
    }
  return qf;
}

// Shared memory of one block of the tiled Hessian-vector product.
template <int D>
struct HvpTileShared {
  static constexpr int CAP = TileCap<D>::NODES;
  using Vec = typename std::conditional<D == 2, float2, float4>::type;
  Vec sd[CAP];        // direction p at the tile nodes (one vector load per node)
  // K p accumulators in FP64: a node sums the contributions of up to 27
  // cells; for smooth directions they nearly cancel, and an FP32 sum loses
  // the small remainder (the plate-bending modes of a thin body)
  double sq[D][CAP];
  TileBox<D> box;
};

// The tiled Hessian-vector product of one tile of slots (one slot per
// thread, the tile starting at a multiple of 2^D; the whole block calls it
// with each thread's particle pi, -1 for a padding slot or a thread past
// the last slot): q = a.w[0] += K p on the free DOFs with p = pv (a grid
// vector), and acc += this run's share of p.Kp = sum_p G:Y.  Per particle
// it reads its slot, its stencil base (flat), F^n and the FP32 data of
// TileX; no FP64 arithmetic runs per particle.  The block stages the node
// box of its particles' stencils in shared memory, gathers from it, and
// scatters into FP64 shared accumulators flushed with one global atomic per
// tile node and component.  The slots come in aligned groups of 2^D whose
// particles share a stencil base, so each group first reduce-scatters its
// contributions among its lanes (FP32, 2^D terms) and every lane adds a few
// group sums to the tile.  A run whose node box exceeds the tile adds the
// group sums to global memory instead.
template <int D>
__device__ __forceinline__ void hvp_tile(const PcgArgsT<float>& a, const double* pv, int64_t pi,
                                         HvpTileShared<D>& sh, float& acc) {
  constexpr int DD = D * D;
  constexpr int CAP = TileCap<D>::NODES;
  constexpr int GL = 1 << D;                 // lanes per slot group
  constexpr int KC = 9;                      // stencil nodes per scatter chunk
  constexpr int NVP = ((KC * D + GL - 1) / GL) * GL;
  using X = TileX<D>;
  auto& sd = sh.sd;
  auto& sq = sh.sq;
  auto& box = sh.box;
  const GridGeo& g = a.g;
  const int64_t n = a.P.n;
  double* q = a.w[0];
  const int gr = threadIdx.x & (GL - 1);
  const int sb = pi >= 0 ? a.sbase[pi] : -1;  // -1: outside the grid box
  const bool valid = sb >= 0;
  int base[D];
  float w[D][3], dw[D][3];
  if (valid) {
    unflatten_base<D>(sb, g, base);
    float fx[D];
#pragma unroll
    for (int c = 0; c < D; ++c) fx[c] = a.tx[(int64_t)(X::FX + c) * n + pi];
    stencil_fx<D>(fx, (float)g.inv_dx, w, dw);
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) base[c] = 0;
  }
  tile_box<D>(base, valid, CAP, box);
  const bool tiled = box.nodes > 0;
  if (tiled) {
    for (int l = threadIdx.x; l < box.nodes; l += blockDim.x) {
      const int64_t gi = tile_global<D>(box, g, l);
      float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int c = 0; c < D; ++c) {
        t[c] = d2f_bits(__ldcg(&pv[c * g.nn + gi]));
        sq[c][l] = 0.0;
      }
      if constexpr (D == 2) sd[l] = make_float2(t[0], t[1]);
      else sd[l] = make_float4(t[0], t[1], t[2], 0.0f);
    }
    __syncthreads();
  }
  const int lb = (tiled && valid) ? tile_local<D>(box, base[0] - box.lo[0], base[1] - box.lo[1],
                                                  base[D - 1] - box.lo[D - 1])
                                  : 0;
  float Y[DD];
#pragma unroll
  for (int e = 0; e < DD; ++e) Y[e] = 0.0f;
  if (valid) {
    float Gd[DD];
#pragma unroll
    for (int e = 0; e < DD; ++e) Gd[e] = 0.0f;
    // one layer of 9 stencil nodes per pass (a rolled loop in 3D keeps the
    // code within the instruction cache)
#pragma unroll 1
    for (int o2 = 0; o2 < (D == 3 ? 3 : 1); ++o2) {
      float wz, dwz;
      layer_weights<D>(w, dw, o2, wz, dwz);
#pragma unroll
      for (int kk = 0; kk < 9; ++kk) {
        const int o0 = kk % 3, o1 = kk / 3;
        float dN[D];
        grad_n_layer<D>(w, dw, o0, o1, wz, dwz, dN);
        float dk[D];
        if (tiled) {
          const int l = lb + tile_local<D>(box, o0, o1, o2);
          const auto v = sd[l];
          dk[0] = v.x;
          dk[1] = v.y;
          if constexpr (D == 3) dk[D - 1] = v.z;
        } else {
          const int64_t gi = (int64_t)sb + (D == 2 ? o0 + o1 * g.res[0]
                                                  : o0 + (o1 + o2 * g.res[1]) * g.res[0]);
#pragma unroll
          for (int c = 0; c < D; ++c) dk[c] = d2f_bits(__ldcg(&pv[c * g.nn + gi]));
        }
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
          for (int b = 0; b < D; ++b) Gd[c * D + b] = fmaf(dk[c], dN[b], Gd[c * D + b]);
      }
    }
    float Fn[DD], A[DD];
#pragma unroll
    for (int e = 0; e < DD; ++e) {
      Fn[e] = a.P.F[e * n + pi];
      A[e] = a.tx[(int64_t)(X::A + e) * n + pi];
    }
    acc += hessian_apply_x<D>(A, a.tx[(int64_t)X::C1 * n + pi], a.tx[(int64_t)X::MU * n + pi],
                              a.tx[(int64_t)X::LAM * n + pi], Gd, Fn, Y);
  }
  // Scatter: every lane of the warp takes part in its group's
  // reduce-scatter (a padding slot adds zeros), in chunks of KC stencil
  // nodes (one layer); each lane then adds its share of the group sums to
  // the shared tile, or to global memory when the box exceeds the tile.
#pragma unroll 1
  for (int o2c = 0; o2c < (D == 3 ? 3 : 1); ++o2c) {
    float v[NVP];
#pragma unroll
    for (int j = 0; j < NVP; ++j) v[j] = 0.0f;
    if (valid) {
      float wz, dwz;
      layer_weights<D>(w, dw, o2c, wz, dwz);
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        float dN[D];
        grad_n_layer<D>(w, dw, kk % 3, kk / 3, wz, dwz, dN);
#pragma unroll
        for (int c = 0; c < D; ++c) {
          float t = 0.0f;
#pragma unroll
          for (int b = 0; b < D; ++b) t = fmaf(Y[c * D + b], dN[b], t);
          v[kk * D + c] = t;
        }
      }
    }
    group_reduce_scatter<GL, NVP>(v, gr);
    // the group's base from any valid lane of the group (lane gr holds the
    // sums of values gr NVP/GL .. (gr + 1) NVP/GL - 1).  The shuffle runs in
    // every lane: a group with no particle reads its own lane, so no lane of
    // a partly filled warp skips it.
    const unsigned gmask = ((1u << GL) - 1u) << ((threadIdx.x & 31) & ~(GL - 1));
    const unsigned vmask = __ballot_sync(kFull, valid) & gmask;
    const int gbase = __shfl_sync(kFull, tiled ? lb : sb,
                                  vmask ? __ffs(vmask) - 1 : (int)(threadIdx.x & 31));
    if (vmask) {
#pragma unroll
      for (int j = 0; j < NVP / GL; ++j) {
        const int idx = gr * (NVP / GL) + j;
        if (idx < KC * D) {
          const int kk = idx / D, c = idx - kk * D;
          const int o0 = kk % 3, o1 = kk / 3, o2 = o2c;
          if (tiled) {
            atomicAdd(&sq[c][gbase + tile_local<D>(box, o0, o1, o2)], f2d_bits(v[j]));
          } else {
            const int64_t gi = (int64_t)gbase + (D == 2 ? o0 + o1 * g.res[0]
                                                        : o0 + (o1 + o2 * g.res[1]) * g.res[0]);
            if ((a.dofmask[gi] >> c) & 1u) atomicAdd(&q[c * g.nn + gi], f2d_bits(v[j]));
          }
        }
      }
    }
  }
  if (tiled) {
    __syncthreads();
    for (int l = threadIdx.x; l < box.nodes; l += blockDim.x) {
      const int64_t gi = tile_global<D>(box, g, l);
      const unsigned fm = a.dofmask[gi];
      if (!fm) continue;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const double t = sq[c][l];
        // (a zero test on the bits: no FP64 instruction)
        if (((fm >> c) & 1u) && (__double_as_longlong(t) << 1) != 0) atomicAdd(&q[c * g.nn + gi], t);
      }
    }
  }
  __syncthreads();  // the tile arrays are reused by the next run
}

// Streaming-PCG Hessian-vector product, mixed precision, block tiles over
// the cell-aligned slots (hvp_tile, grid stride); p.Kp into S->pq.
template <int D>
__global__ void __launch_bounds__(TileCap<D>::THREADS, TileCap<D>::MIN_BLOCKS)
    k_cgs_hvp_tile(PcgArgsT<float> a) {
  if (__ldcg(&a.S->cg_done)) return;
  __shared__ HvpTileShared<D> sh;
  const int64_t ns = __ldcg(a.n_slots);
  float accf = 0.0f;  // this thread's particles' share of p.Kp (a few tiles)
  const int64_t tiles = (ns + blockDim.x - 1) / blockDim.x;
  // each thread's slot of the block's next tile is read one tile ahead, so
  // the slot map's latency overlaps the current tile
  auto slot_of = [&](int64_t t) -> int64_t {
    const int64_t sl = t * blockDim.x + threadIdx.x;
    return (t < tiles && sl < ns) ? (int64_t)a.slot2p[sl] : -1;
  };
  int64_t pi_next = slot_of(blockIdx.x);
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t pi = pi_next;
    pi_next = slot_of(t + gridDim.x);
    hvp_tile<D>(a, a.s[0], pi, sh, accf);
  }
  double acc[1] = {(double)accf};
  double tot[1];
  if (grid_sum<1>(acc, a.partials, &a.S->counter, tot) && threadIdx.x == 0) a.S->pq = tot[0];
}

// Warp-aggregated add into a shared tile: lanes whose particles share a
// stencil base (a run of equal keys, contiguous in Morton order) target the
// same node for every stencil offset, so each run is summed with shuffles
// and its first lane adds the run's total.  `first` and `last` bound the
// lane's run; `steps` = ceil(log2(longest run in the warp)).  Every lane of
// the warp calls it (shuffles); lanes with `active` false add nothing.
template <int NV>
__device__ __forceinline__ void warp_run_add(double (&v)[NV], int lane, int first, int last,
                                             int steps, bool active, double* const (&dst)[NV]) {
  for (int s = 0, off = 1; s < steps; ++s, off <<= 1) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const double t = __shfl_down_sync(kFull, v[c], off);
      if (lane + off <= last) v[c] += t;
    }
  }
  if (active && lane == first)
#pragma unroll
    for (int c = 0; c < NV; ++c)
      if (v[c] != 0.0) atomicAdd(dst[c], v[c]);
}

// APIC particle-to-grid transfer (Eq. p2g_transfer, Eq. p2g_substep), with
// bm != nullptr also the boundary-particle mass of Eq. boundary_grid_set,
// block-tiled: each block accumulates m, mv (and bm) of its Morton run of
// particles in a shared node tile (warp-aggregated over runs of particles
// that share a stencil base), then flushes each tile node with one global
// atomic per field.  Same per-particle arithmetic as the one-thread-per-
// particle transfer; with sbase/sdn also caches each particle's stencil.
template <int D, typename R>
__global__ void __launch_bounds__(TileCap<D>::THREADS)
    k_p2g_tile(PartPtrsT<R> P, GridGeo g, double* m, double* mv, double* bm, int* err,
               int* sbase, R* sdn) {
  constexpr int K = (D == 2) ? 9 : 27;
  constexpr int NV = D + 2;           // m, mv (D), bm
  constexpr int CAP = TileCap<D>::NODES;
  __shared__ double acc[NV][CAP];
  __shared__ TileBox<D> box;
  const int64_t n = P.n;
  const int lane = threadIdx.x & 31;
  const double Dinv = 4.0 * g.inv_dx * g.inv_dx;  // D_p^-1 of the quadratic B-spline
  const int64_t tiles = (n + blockDim.x - 1) / blockDim.x;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t p = t * blockDim.x + threadIdx.x;
    double xp[D];
    Stencil<D> s;
    bool valid = false;
    if (p < n) {
#pragma unroll
      for (int a = 0; a < D; ++a) xp[a] = P.x[a * n + p];
      valid = make_stencil<D>(xp, g, s);
      if (!valid) {
        atomicOr(err, kErrOutOfGrid);
        if (sbase) sbase[p] = -1;  // no stencil (the slots and the tiled product skip it)
      }
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) s.base[a] = 0;
    }
    tile_box<D>(s.base, valid, CAP, box);
    const bool tiled = box.nodes > 0;
    if (tiled) {
      for (int l = threadIdx.x; l < box.nodes; l += blockDim.x)
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c][l] = 0.0;
      __syncthreads();
    }
    double vp[D], Bp[D * D], mp = 0.0;
    bool isb = false;
    int lb = 0;
    if (valid) {
#pragma unroll
      for (int a = 0; a < D; ++a) vp[a] = (double)P.v[a * n + p];
#pragma unroll
      for (int e = 0; e < D * D; ++e) Bp[e] = (double)P.B[e * n + p];
      mp = P.mass[p];
      isb = (bm != nullptr) && (P.flags[p] & 1u);
      if (sbase) {
        int64_t b = 0, stride = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          b += (int64_t)s.base[a] * stride;
          stride *= g.res[a];
        }
        sbase[p] = (int)b;
      }
      if (tiled)
        lb = tile_local<D>(box, s.base[0] - box.lo[0], s.base[1] - box.lo[1],
                           s.base[D - 1] - box.lo[D - 1]);
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) vp[a] = 0.0;
#pragma unroll
      for (int e = 0; e < D * D; ++e) Bp[e] = 0.0;
    }
    // runs of lanes with the same stencil base (tile-local base index; an
    // invalid lane forms a run of its own)
    const int key = (tiled && valid) ? lb : -1 - lane;
    const unsigned run = __match_any_sync(kFull, key);
    const int first = __ffs(run) - 1, last = 31 - __clz(run);
    const bool contiguous = (run >> first) == ((1u << (last - first)) << 1) - 1u;
    const bool warp_ok = __all_sync(kFull, contiguous);
    int longest = __reduce_max_sync(kFull, (unsigned)(last - first + 1));
    int steps = 0;
    while ((1 << steps) < longest) ++steps;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double N = 0.0, dN[D];
      int64_t node = 0;
      double vals[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) vals[c] = 0.0;
      if (valid) {
        node = stencil_node<D>(s, g, k, N, dN);
        if (sdn)
#pragma unroll
          for (int a = 0; a < D; ++a) sdn[(int64_t)(a * K + k) * n + p] = (R)dN[a];
        double r[D];
#pragma unroll
        for (int a = 0; a < D; ++a) r[a] = stencil_node_pos<D>(s, g, k, a) - xp[a];
        const double wm = mp * N;
        vals[0] = wm;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          double va = 0.0;
#pragma unroll
          for (int b = 0; b < D; ++b) va += Bp[a * D + b] * r[b];
          vals[1 + a] = wm * (vp[a] + Dinv * va);
        }
        vals[D + 1] = isb ? wm : 0.0;
      }
      if (tiled) {
        const int l = valid ? lb + tile_local<D>(box, k % 3, (k / 3) % 3, k / 9) : 0;
        double* dst[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) dst[c] = &acc[c][l];
        if (warp_ok) {
          warp_run_add<NV>(vals, lane, first, last, steps, valid, dst);
        } else if (valid) {
#pragma unroll
          for (int c = 0; c < NV; ++c)
            if (vals[c] != 0.0) atomicAdd(dst[c], vals[c]);
        }
      } else if (valid) {
        atomicAdd(&m[node], vals[0]);
#pragma unroll
        for (int a = 0; a < D; ++a) atomicAdd(&mv[a * g.nn + node], vals[1 + a]);
        if (isb) atomicAdd(&bm[node], vals[D + 1]);
      }
    }
    if (tiled) {
      __syncthreads();
      for (int l = threadIdx.x; l < box.nodes; l += blockDim.x) {
        if (acc[0][l] == 0.0) continue;  // no particle reached this node
        const int64_t gi = tile_global<D>(box, g, l);
        atomicAdd(&m[gi], acc[0][l]);
#pragma unroll
        for (int a = 0; a < D; ++a) atomicAdd(&mv[a * g.nn + gi], acc[1 + a][l]);
        if (bm && acc[D + 1][l] != 0.0) atomicAdd(&bm[gi], acc[D + 1][l]);
      }
    }
    __syncthreads();  // the tile is reused by the next run of particles
  }
}

// ---------------------------------------------------------------------------
// Cell-aligned slots.  The tiled Hessian-vector product works on groups of
// 2^D lanes whose particles share a stencil base (they scatter to the same
// 3^D nodes, so a group reduces its contributions among its lanes before
// touching shared memory).  Runs of equal base in Morton order are not
// aligned to such groups (a body's boundary cells hold fewer particles), so
// after each P2G the particles are dealt to slots: every run starts a new
// group of 2^D slots and longer runs take several groups; unused slots hold
// -1.  slot2p[slot] = particle.
// ---------------------------------------------------------------------------
constexpr int kScanItems = 1024;  // items per block of the device-wide scans

// Inclusive scan (sum or max, non-negative ints) of one block's items; the
// block's total into bsum.
template <bool MAX>
__global__ void __launch_bounds__(256) k_scan_block(const int* in, int* out, int64_t n,
                                                     int* bsum) {
  __shared__ int sh[kScanItems];
  const int64_t base = (int64_t)blockIdx.x * kScanItems;
  for (int i = threadIdx.x; i < kScanItems; i += blockDim.x)
    sh[i] = base + i < n ? in[base + i] : 0;
  __syncthreads();
  for (int off = 1; off < kScanItems; off <<= 1) {
    int v[kScanItems / 256];
#pragma unroll
    for (int r = 0; r < kScanItems / 256; ++r) {
      const int i = threadIdx.x + r * 256;
      v[r] = i >= off ? (MAX ? max(sh[i], sh[i - off]) : sh[i] + sh[i - off]) : sh[i];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kScanItems / 256; ++r) sh[threadIdx.x + r * 256] = v[r];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kScanItems; i += blockDim.x)
    if (base + i < n) out[base + i] = sh[i];
  if (threadIdx.x == 0) bsum[blockIdx.x] = sh[kScanItems - 1];
}

// Inclusive scan of the block totals in place (one block, serial chunks).
template <bool MAX>
__global__ void k_scan_top(int* bsum, int nb) {
  __shared__ int carry;
  __shared__ int sh[256];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += 256) {
    const int i = b0 + threadIdx.x;
    sh[threadIdx.x] = i < nb ? bsum[i] : 0;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
      const int v = threadIdx.x >= off ? (MAX ? max(sh[threadIdx.x], sh[threadIdx.x - off])
                                              : sh[threadIdx.x] + sh[threadIdx.x - off])
                                       : sh[threadIdx.x];
      __syncthreads();
      sh[threadIdx.x] = v;
      __syncthreads();
    }
    const int c = carry;
    if (i < nb) bsum[i] = MAX ? max(c, sh[threadIdx.x]) : c + sh[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) carry = MAX ? max(c, sh[255]) : c + sh[255];
    __syncthreads();
  }
}

template <bool MAX>
__global__ void k_scan_add(int* out, int64_t n, const int* bsum) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = (int)(i / kScanItems);
  if (b == 0) return;
  const int c = bsum[b - 1];
  out[i] = MAX ? max(out[i], c) : out[i] + c;
}

// rs[p] = p at a run start (p = 0 or a new stencil base), else 0.
__device__ __forceinline__ bool run_start(const int* sbase, int64_t p) {
  return p == 0 || sbase[p] != sbase[p - 1];
}
template <int GL>
__global__ void k_slot_starts(const int* sbase, int64_t n, int* rs) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) rs[p] = run_start(sbase, p) ? (int)p : 0;
}
// flag[p] = 1 where a group of GL slots starts (rank in the run a multiple of GL)
template <int GL>
__global__ void k_slot_flags(const int* rs, int64_t n, int* flag) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) flag[p] = ((p - rs[p]) % GL) == 0 ? 1 : 0;
}
// slot2p[GL (groups before p's group) + lane] = p; the slot count into *n_slots
template <int GL>
__global__ void k_slot_fill(const int* rs, const int* gsum, const int* flag, int64_t n,
                            int* slot2p, int* n_slots) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int lane = (int)((p - rs[p]) % GL);
  const int64_t g0 = p - lane;                      // the group's first particle
  const int group = gsum[g0] - 1;                   // inclusive sum of flags - 1
  slot2p[(int64_t)GL * group + lane] = (int)p;
  if (p == n - 1) *n_slots = GL * gsum[p];
}

}  // namespace osmpm
