// Host-side interface between the C ABI / drivers and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/osmpm.h"
#include "osmpm_types.h"

namespace osmpm {

// Kernels launched by the library in this process (every launcher adds the
// number of kernels it enqueues).
extern std::atomic<long long> g_launch_count;

// Launch shape helpers shared by drivers and launchers.
constexpr int kRedBlocksMax = 1216;  // 152 SMs x 8 resident 256-thread blocks
inline int blocks_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : b);
}
inline int red_blocks_for(int64_t n) {
  int b = blocks_for(n);
  return b < kRedBlocksMax ? b : kRedBlocksMax;
}

// Arguments of the grid-preparation kernel (Dirichlet data, Schwarz
// receivers and the initial Newton guess).
struct PrepArgs {
  const DevRule* rules;
  int n_rules;
  const uint8_t* recv;  // Schwarz receiver mask or nullptr
  const double* bc0;    // receiver velocity at the start of the window
  const double* bc1;    // receiver velocity at the end of the window
  double a_m;           // temporal weight: v = (1 - a_m) bc0 + a_m bc1
  double* bc_applied;   // receiver velocity applied (written), may be null
  uint8_t* physmask;    // the components a physical rule fixes, bit a (written), may be null
  const uint8_t* hold;  // rigid-plane contact: nodes whose y component is held, or nullptr
  const double* hold_v; // their prescribed y velocity
};

// Launchers of the reverse-mode kernels (FP64 only; osmpm_adjoint.cuh).
template <int D>
struct AdjointKernels {
  static void g2p(int64_t n, const double* x, const double* F, const GridGeo& g, const double* u,
                  double dt, const double* xb, const double* vb, const double* Bb,
                  const double* Fb, double* ubar, double* xb_out, double* Fb_out, cudaStream_t s);
  static void rhs(const GridGeo& g, const double* m, const uint8_t* dofmask, double dt,
                  double cg_rtol, int cg_max, const double* ubar, double* diag, double* x,
                  double* r, double* z, double* p, DevScalars* S, double* partials,
                  cudaStream_t s);
  static void solve(int64_t n, const double* x, const double* F, const double* mu,
                    const double* lam, const double* vol0, const GridGeo& g, const double* u,
                    const double* lamg, const uint8_t* dofmask, double* xb, double* Fb,
                    double* Eb, double* klam, int* err, cudaStream_t s);
  static void nodes(const GridGeo& g, const double* m, const double* vn, const double* u,
                    const double* lamg, const double* gravity, double dt, const double* mextra,
                    double* qbar, double* mbar, cudaStream_t s);
  // coupled step in reverse
  static void bc(const GridGeo& g, const uint8_t* recv, const double* m, const double* ubar,
                 const double* klam, double s0, double s1, double* v0bar, double* v1bar,
                 cudaStream_t s);
  static void interp_t(const GridGeo& gB, const GridGeo& gS, const uint8_t* recvS,
                       const double* vbar, double* out, cudaStream_t s);
  static void proj_coarse(const GridGeo& gB, const uint8_t* recvB, const double* num,
                          const double* den, double eps, const double* vbar, double* nbar,
                          double* dbar, cudaStream_t s);
  static void proj_fine(const GridGeo& gB, const GridGeo& gS, const double* nbar,
                        const double* dbar, double* G, double* H, cudaStream_t s);
  static void inject(const GridGeo& g, const double* m, const double* u, double dt, const double* G,
                     const double* H, double* ubar, double* mextra, cudaStream_t s);
  static void grid_acc(const GridGeo& g, const double* m, const double* vn, const double* G,
                       const double* H, const double* vbar, double* qbar, double* mbar,
                       cudaStream_t s);
  static void axpy_active(const GridGeo& g, const double* m, double scale, const double* v,
                          double* out, cudaStream_t s);
  static void add(int64_t cnt, const double* src, double* dst, cudaStream_t s);
  static void p2g(int64_t n, const double* x, const double* v, const double* B,
                  const double* mass, const GridGeo& g, const double* qbar, const double* mbar,
                  double* vb_out, double* Bb_out, double* xb, cudaStream_t s);
  static void from_ids(int64_t n, int w, const uint32_t* id, const double* src, double* dst,
                       cudaStream_t s);
  static void to_ids(int64_t n, int w, const uint32_t* id, const double* src, double* dst,
                     cudaStream_t s);
};

// Launchers of the batched streaming PCG over many domains (mixed
// precision; osmpm_multi.cuh).
template <int D>
struct MultiKernels {
  // mp: the device argument block; grids fixed by the caller (grid stride
  // over the tiles)
  static void start(const MultiArgs* mp, int grid_dt, cudaStream_t s);
  // one PCG iteration of every instance still running; with e0, e1 the
  // Hessian-vector product is bracketed by event records (external event
  // nodes when the stream is being captured)
  static void iteration(const MultiArgs* mp, int grid_pt, int grid_dt, cudaStream_t s,
                        cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr, bool capturing = false);
  static void pending(const MultiArgs* mp, cudaStream_t s);
  static int particle_tile();      // slots per slot tile (one per thread of a block)
  static int hvp_blocks_per_sm();  // co-resident blocks of the product per SM
};

template <int D, typename R>
struct Kernels {
  static void morton_keys(const double* x, int64_t n, const GridGeo& g, uint64_t* keys,
                          uint32_t* vals, int* err, cudaStream_t s);
  static void permute(const PartPtrsT<R>& src, const PartPtrsT<R>& dst, const uint32_t* perm,
                      cudaStream_t s);
  static void scatter_by_id(const PartPtrsT<R>& src, const PartPtrsT<R>& dst, cudaStream_t s);
  static void lame(const double* E, const double* nu, PartPtrsT<R> P, cudaStream_t s);
  static void pack_out(const PartPtrsT<R>& P, double* x, double* v, double* B, double* F,
                       cudaStream_t s);
  static void unpack_in(const double* x, const double* v, const double* B, const double* F,
                        PartPtrsT<R> dst, cudaStream_t s);
  // P2G; with sbase/sdn also caches each particle's stencil (base node and
  // grad N) for the PCG of the step
  static void p2g(const PartPtrsT<R>& P, const GridGeo& g, double* m, double* mv, double* bm,
                  int* err, int* sbase, R* sdn, cudaStream_t s);
  static void normalize(const GridGeo& g, const double* m, const double* mv, double* vn,
                        cudaStream_t s);
  static void grid_prep(const GridGeo& g, const double* m, const double* vn, const PrepArgs& a,
                        double dt, uint8_t* dofmask, double* u, cudaStream_t s);
  // lmode: bit 1 the packed Hessian blocks L, bit 2 the tiled product's
  // per-particle data (mixed precision); -1: every part the precision uses
  static void grad(const PartPtrsT<R>& P, const GridGeo& g, const double* u, const uint8_t* dofmask,
                   double* grad, double* diag, R* L, int* err, cudaStream_t s, int lmode = -1);
  // completes the gradient, inverts the Jacobi diagonal and starts PCG; the
  // PCG tolerance is eta |r0|, eta = |g|/|g_0| clamped to [cg_rtol, eta_max]
  // (g_0: the gradient of the solve's first Newton iteration, `first` = 1)
  static void grad_finish(const GridGeo& g, const double* m, const double* vn, const double* u,
                          const uint8_t* dofmask, const double* gravity, double dt, double cg_rtol,
                          double eta_max, int first, int cg_max, double* grad, double* diag,
                          double* x, double* r, double* z, double* p, DevScalars* S,
                          double* partials, cudaStream_t s);
  // one PCG iteration = cg_a (p update, diagonal part), cg_b (HVP), cg_c (updates)
  static void cg_a(const GridGeo& g, const double* m, const uint8_t* dofmask, double dt,
                   const double* z, double* p, double* q, DevScalars* S, double* partials,
                   cudaStream_t s);
  static void cg_b(const PartPtrsT<R>& P, const GridGeo& g, const uint8_t* dofmask, const R* L,
                   const double* p, double* q, DevScalars* S, double* partials, cudaStream_t s);
  static void cg_c(const GridGeo& g, const uint8_t* dofmask, const double* diag,
                   const double* p, const double* q, double* x, double* r, double* z,
                   DevScalars* S, double* partials, cudaStream_t s);
  // persistent cooperative PCG (whole solve in one launch)
  static void pcg_shape(int64_t work, int share, int* blocks, int* threads);
  static cudaError_t pcg(const PcgArgsT<R>& a, int blocks, int threads, cudaStream_t s);
  // the k_pcg variant pcg() launches for this shape (for a graph kernel node)
  static const void* pcg_kernel(const PcgArgsT<R>& a, int blocks, int threads);
  // does one co-resident pass of the persistent PCG cover the problem, and
  // how many passes does it need?
  static bool pcg_one_pass(const PcgArgsT<R>& a, int blocks, int threads);
  static int64_t pcg_passes(const PcgArgsT<R>& a, int blocks, int threads);
  // streaming PCG: start, then per iteration hvp, alpha, beta
  static void cgs_start(const PcgArgsT<R>& a, cudaStream_t s);
  // hvp_mode (mixed precision only): 1 lane groups over the cached stencil
  // and Hessian blocks, otherwise block tiles recomputing the Hessian
  // with e0, e1 the Hessian-vector product is bracketed by event records
  static void cgs_iteration(const PcgArgsT<R>& a, int hvp_mode, cudaStream_t s,
                            cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr);
  // the streaming PCG's particle product alone: a.w[0] += K a.s[0] on the
  // free DOFs, p.Kp into S->pq
  static void cgs_hvp(const PcgArgsT<R>& a, int hvp_mode, cudaStream_t s);
  static void hvp_only(const PartPtrsT<R>& P, const GridGeo& g, const double* m,
                       const uint8_t* dofmask, const R* L, double dt, double* p, double* q,
                       DevScalars* S, double* partials, cudaStream_t s);
  static void maxabs(const GridGeo& g, const uint8_t* dofmask, const double* x, DevScalars* S,
                     double* partials, cudaStream_t s);
  static void energy_change(const PartPtrsT<R>& P, const GridGeo& g, const double* m,
                            const double* vn, const double* u, const double* x,
                            const double* gravity, double dt, double alpha, DevScalars* S,
                            double* partials, cudaStream_t s);
  // same kernel with an explicit block count (one block per 256 work items)
  static void energy_change_blocks(const PartPtrsT<R>& P, const GridGeo& g, const double* m,
                                   const double* vn, const double* u, const double* x,
                                   const double* gravity, double dt, double alpha, DevScalars* S,
                                   double* partials, int blocks, cudaStream_t s);
  static void warm_start(const GridGeo& g, const uint8_t* dofmask, const double* src, double* u,
                         cudaStream_t s);
  static void split_free(const GridGeo& g, const uint8_t* dofmask, double* u, double* x,
                         cudaStream_t s);
  static void axpy(const GridGeo& g, double* u, const double* x, double alpha, cudaStream_t s);
  static void g2p(const PartPtrsT<R>& P, const GridGeo& g, const double* u, double dt,
                  cudaStream_t s);
  // Schwarz interface operators (Sec. 3.2)
  static void gamma(const GridGeo& g, const double* m, const double* bm, double tau,
                    uint8_t* gam, cudaStream_t s);
  static void arbitrate(const GridGeo& gB, const GridGeo& gS, const uint8_t* gamB,
                        const uint8_t* gamS, const double* mB, const double* mS, uint8_t* recvB,
                        uint8_t* recvS, cudaStream_t s);
  static void proj_scatter(const GridGeo& gB, const GridGeo& gS, const double* mS,
                           const double* vS, double* num, double* den, cudaStream_t s);
  static void recvB_filter(const GridGeo& gB, const double* den, double tau,
                           const uint8_t* physB, uint8_t* recvB, cudaStream_t s);
  static void recvS_filter(const GridGeo& gB, const GridGeo& gS, const double* mB,
                           const uint8_t* physS, uint8_t* recvS, cudaStream_t s);
  static void proj_finish(const GridGeo& gB, const uint8_t* recvB, const double* num,
                          const double* den, double eps_tol, double* out, cudaStream_t s);
  static void interp(const GridGeo& gB, const GridGeo& gS, const double* vB,
                     const uint8_t* recvS, double* out, cudaStream_t s);
  static void vel_from_u(const GridGeo& g, const double* m, const double* u, double dt,
                         double* v, cudaStream_t s);
  static void rel_change(const GridGeo& g, const double* vnew, const double* vold,
                         const uint8_t* recv, int slot, DevScalars* S, double* partials,
                         cudaStream_t s);
  static void copy_if_neg(const GridGeo& g, const double* p, double* x, const DevScalars* S,
                          cudaStream_t s);
  static void set_cg_state(DevScalars* S, int iter, int done, cudaStream_t s);
  static void barrier_timeout_check(unsigned* words, int* err, cudaStream_t s);
  // cell-aligned slots of the tiled product from the stencil bases of the
  // last P2G (scratch: rs, flag, gsum n ints each, bsum n/1024 + 1 ints;
  // slot2p slot_cap = 2^D n ints; the slot count into *n_slots)
  static void build_slots(const int* sbase, int64_t n, int* rs, int* flag, int* gsum, int* bsum,
                          int* slot2p, int64_t slot_cap, int* n_slots, cudaStream_t s);
  // rigid-plane contact (2D; osmpm_contact.cuh)
  static void plane_colmin(const PartPtrsT<R>& P, const GridGeo& g, double spacing,
                           unsigned long long* colmin, cudaStream_t s);
  static void plane_init(const GridGeo& g, const double* m, const uint8_t* physmask,
                         const unsigned long long* colmin, double level, double cand_hi,
                         double spacing, double dt, double* gap, double* hold_v, uint8_t* cand,
                         uint8_t* act, cudaStream_t s);
  static void mask_all(const GridGeo& g, const double* m, uint8_t* mask, cudaStream_t s);
  static void plane_update(const GridGeo& g, const uint8_t* cand, const double* grad,
                           const double* u, const double* gap, uint8_t* act, double* lam,
                           int* changes, cudaStream_t s);
};

// Records the message returned by osmpm_last_error() and returns st.
osmpm_status set_error(osmpm_status st, const char* fmt, ...);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
// keys; result ends in (keys, vals).  hist needs 256 * radix_tiles(n) words.
int64_t radix_tiles(int64_t n);
void radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                      int64_t n, int bits, unsigned* hist, cudaStream_t s);

}  // namespace osmpm
