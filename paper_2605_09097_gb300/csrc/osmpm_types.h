// Plain structures shared by the host drivers and the kernels.
#pragma once

#include <stdint.h>

namespace osmpm {

// Structured background grid (Sec. 2.2.2): node (i,j,k) at o + dx (i,j,k),
// flat index i + res0 (j + res1 k).
struct GridGeo {
  double o[3];
  double dx, inv_dx;
  int res[3];
  int64_t nn;
  double mass_eps;  // active nodes: m_i > mass_eps
};

// Particle state, structure of arrays, component-major (x[a*n + p]).  R is
// the storage type of v, B and F: double in FP64 mode, float in mixed mode
// (positions, masses and material constants stay double).
template <typename R>
struct PartPtrsT {
  int64_t n;
  double* x;      // D
  R* v;           // D
  R* B;           // D*D (row-major entry e at B[e*n + p])
  R* F;           // D*D
  double* vol0;
  double* mass;
  double* mu;
  double* lam;
  uint8_t* flags;
  uint32_t* id;
};
using PartPtrs = PartPtrsT<double>;

// Device-side Dirichlet rule (mirrors osmpm_dirichlet; for kind 1 the
// rotation matrix R of the step is precomputed on the host).
struct DevRule {
  int kind;
  unsigned comp_mask;
  double lo[3], hi[3];
  double vel[3];
  double center[3];
  double R[9];
};

constexpr int kMaxRules = 16;

// Scalars of the solver loop, kept on the device so that PCG iterations run
// back to back without host round trips.
struct DevScalars {
  double rz, pq, alpha, beta, rr, rr0, tol2;
  double pq_diag;
  double maxabs;
  double dE;
  double res_num[2], res_den[2];
  double g0sq;  // |g|^2 at the first Newton iteration of the current solve
  int cg_iter, cg_done, cg_neg, cg_max;
  int err;
  unsigned counter;
  unsigned bar_count, bar_spare;  // grid-barrier counter of the persistent PCG kernel
  int n_slots;                     // cell-aligned slots of the last P2G (tiled product)
  int neg0;                        // batched PCG: negative curvature before the first step
  double rz_prev, alpha_prev;      // batched PCG (Chronopoulos-Gear): gamma, alpha of the last step
};

enum : int {
  kErrOutOfGrid = 1,
  kErrNonFinite = 2,
  kErrBarrierTimeout = 4,
};

// Arguments of the persistent PCG kernel (R: storage and arithmetic type of
// the Hessian-vector product).
template <typename R>
struct PcgArgsT {
  PartPtrsT<R> P;
  GridGeo g;
  const double* m;
  const uint8_t* dofmask;
  const R* L;
  const double* diag;   // inverse Jacobi diagonal
  double inv_dt2;
  double* x;
  double* r[2];      // residual, double-buffered (r[0] holds -g at launch)
  double* s[2];      // s = A p, double-buffered
  double* w[3];      // w = A u, triple-buffered (w[0], w[1] zero at launch)
  double* p;
  DevScalars* S;
  double* partials;  // 3 * gridDim.x doubles
  int* err;
  const int* sbase;     // per particle: flat index of the stencil's base node
  const R* sdn;         // per particle: grad N of the 3^D stencil nodes, [(c*K + k)*n + p]
  const double* u;      // the Newton iterate
  // the tiled product (mixed precision): cell-aligned slots of the last P2G
  // (slot2p[slot] = particle or -1, *n_slots of them, device) and the
  // per-particle data the gradient kernel stores for it at each Newton
  // iterate, [e*n + p] (TileX layout)
  const int* slot2p;
  const int* n_slots;
  const R* tx;
};

// FP32 values per particle that the gradient kernel stores for the tiled
// product (TileX in osmpm_tile.cuh): F_hat^-T, c1, V0 mu, V0 lam, the
// offsets from the stencil base.
constexpr int tile_x_count(int D) { return D * D + 3 + D; }

// Batched PCG over many domains (osmpm_multi.cuh): items [lo, hi)
// (particles or DOFs) of instance `inst`.
struct MultiTile {
  int inst;
  int lo, hi;
};

// Where an instance's tiles sit in the two work lists.
struct MultiInfo {
  int pt0, npt;  // slot tiles
  int dt0, ndt;  // DOF tiles
  int fresh;     // 1: the system joins with this launch (its PCG start runs)
  int pad_;
};

struct MultiArgs {
  const PcgArgsT<float>* inst;  // the instances' PCG arguments (domain buffers, scalars)
  const MultiInfo* info;
  const MultiTile* pt;
  int n_pt;
  const MultiTile* dtl;
  int n_dt;
  int n_inst;
  double* part;   // tile partials, row k at part[k * stride + tile]
  int stride;
  int* pending;   // [0]: systems still iterating; [1 + 2i], [2 + 2i]: stop flag, iterations
};

}  // namespace osmpm
