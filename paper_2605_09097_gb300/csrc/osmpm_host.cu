// C ABI of the OS-MPM hot path: domain lifetime, the Newton / PCG driver of
// the implicit step (Sec. 2.2.5) and the Schwarz alternating loop (Alg. 1).
// All arithmetic of the method runs in the kernels; this file launches them
// on the domain's stream and reads back the few scalars that steer the loop.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>
#include <chrono>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/osmpm.h"
#include "osmpm_internal.h"

using namespace osmpm;

std::atomic<long long> osmpm::g_launch_count{0};

namespace {

// An NVTX range over one phase of the method (P2G, Newton, PCG, G2P, a
// Schwarz iteration, a batched PCG chunk); Nsight tools show them, and
// without a tool attached a push or pop costs a few nanoseconds.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};


thread_local std::string g_last_error = "no error";

osmpm_status vfail(osmpm_status st, const char* fmt, va_list ap) {
  char buf[512];
  vsnprintf(buf, sizeof(buf), fmt, ap);
  g_last_error = buf;
  return st;
}

osmpm_status fail(osmpm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vfail(st, fmt, ap);
  va_end(ap);
  return st;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(OSMPM_E_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));         \
  } while (0)

#define OSMPM_TRY(expr)               \
  do {                                \
    osmpm_status st_ = (expr);        \
    if (st_ != OSMPM_OK) return st_;  \
  } while (0)

}  // namespace

osmpm_status osmpm::set_error(osmpm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vfail(st, fmt, ap);
  va_end(ap);
  return st;
}

// Particle memory with the storage type of v, B, F erased; typed<R>()
// gives the kernels' view.
struct PartMem {
  int64_t n;
  double* x;
  void* v;
  void* B;
  void* F;
  double* vol0;
  double* mass;
  double* mu;
  double* lam;
  uint8_t* flags;
  uint32_t* id;
};

template <class R>
PartPtrsT<R> typed(const PartMem& m) {
  PartPtrsT<R> p;
  p.n = m.n;
  p.x = m.x;
  p.v = (R*)m.v;
  p.B = (R*)m.B;
  p.F = (R*)m.F;
  p.vol0 = m.vol0;
  p.mass = m.mass;
  p.mu = m.mu;
  p.lam = m.lam;
  p.flags = m.flags;
  p.id = m.id;
  return p;
}

namespace {
struct PcgBatcher;
}

struct osmpm_domain {
  osmpm_domain_desc desc{};
  int dim = 2;
  GridGeo geo{};
  int64_t n = 0;
  cudaStream_t stream = nullptr;
  osmpm_allocator alloc{};
  bool have_alloc = false;
  std::vector<std::pair<void*, size_t>> blocks;

  int prec = 0;        // 0: FP64, 1: mixed (v, B, F, L, grad N and the HVP in FP32)
  size_t rsize = 8;    // bytes of the particle-state type
  PartMem P{}, A{};    // primary (Morton-sorted) and alternate particle sets
  double* snap_x = nullptr;
  void *snap_v = nullptr, *snap_B = nullptr, *snap_F = nullptr;
  double* stage = nullptr;  // host-layout staging for get/set_particles
  uint64_t *keys = nullptr, *keys_alt = nullptr;
  uint32_t *vals = nullptr, *vals_alt = nullptr;
  unsigned* hist = nullptr;

  // grid (component-major)
  double *m = nullptr, *mv = nullptr, *vn = nullptr, *bm = nullptr, *u = nullptr;
  double *grad = nullptr, *diag = nullptr;
  // PCG vectors: x, r (2), s (2), w (3), p; cz/cp double as r[1]/s[0]
  double *cx = nullptr, *cr = nullptr, *cz = nullptr, *cp = nullptr, *cp1 = nullptr, *cq = nullptr;
  double *cw1 = nullptr, *cw2 = nullptr, *cpp = nullptr;
  void* L = nullptr;       // per-particle Hessian blocks (particle-state type)
  int* sbase = nullptr;    // stencil cache of the last P2G (base node, grad N)
  int* slot2p = nullptr;   // mixed precision: cell-aligned slots of the last P2G
  void* sdn = nullptr;
  uint8_t *dofmask = nullptr, *physmask = nullptr, *gam = nullptr, *recv = nullptr;
  double *bc0 = nullptr, *bc1 = nullptr, *bc_prev = nullptr, *bc_applied = nullptr;
  double *vtmp = nullptr, *proj_num = nullptr, *proj_den = nullptr;
  // Schwarz warm starts: previous solutions (coarse: 1, fine: one per sub-step)
  double* u_keep = nullptr;
  int n_keep = 0;

  DevRule* rules_dev = nullptr;
  std::vector<osmpm_dirichlet> rules;
  DevScalars* S = nullptr;
  DevScalars* S_host = nullptr;  // pinned mirror
  double* partials = nullptr;
  int* err = nullptr;
  int* err_host = nullptr;

  // cooperative PCG grids that may run at once (set by the batched entry
  // point); each PCG grid uses at most 1/pcg_share of the device
  int pcg_share = 1;
  // the batched PCG service of osmpm_schwarz_couple_multi (set while a
  // multi call drives the domain): Newton systems go there instead of to
  // a PCG launch of their own
  struct PcgBatcher* batcher = nullptr;

  // reverse-mode tape (osmpm_record / osmpm_adjoint): per recorded step its
  // input particle state, the converged grid displacement and the DOF mask
  struct TapeStep {
    void* mem = nullptr;
    size_t bytes = 0;
    double dt = 0.0;
  };
  bool recording = false, tape_broken = false;
  std::vector<TapeStep> tape;
  double* adj = nullptr;  // adjoint work arrays, allocated on first use
  // coupled steps recorded on the coarse domain: per step a head block (both
  // start states, receiver masks, the k = 0 projection sums) and one block
  // per Schwarz iteration (see CoupledLayout)
  struct CoupledStep {
    TapeStep head;
    std::vector<TapeStep> iters;
    int M = 1;
    double dT = 0.0, eps_tol = 0.0;
  };
  std::vector<CoupledStep> ctape;
  osmpm_domain* partner = nullptr;  // the other domain of the recorded coupled steps
  int tape_kind = 0;                // 0 empty, 1 single-domain steps, 2 coupled (coarse), 3 coupled (fine)
  double* cadj = nullptr;           // coupled-adjoint work arrays
  // checkpointed record (osmpm_record with every >= 2): instead of the full
  // per-step record, the particle state at the start of every ckpt_every-th
  // recorded step (for coupled steps both domains', kept on the coarse
  // domain) and the controls of every recorded step; osmpm_adjoint re-runs
  // one segment of steps at a time with the full record and reverses it
  int ckpt_every = 1;
  bool replaying = false;           // osmpm_adjoint re-running a segment
  struct StepCtl {
    double dt = 0.0;                               // dt (single) or dT (coupled)
    osmpm_schwarz_desc sd{};                       // coupled steps
    std::vector<osmpm_dirichlet> rules, rules_fine;  // the rule sets in force
  };
  std::vector<StepCtl> ctl;
  std::vector<TapeStep> ckpts;      // one per segment: the state at its first step

  // CUDA graphs of one Newton iteration's device work (launch_mode 0), one
  // slot per iteration kind (first | confirming << 1 | timed << 2), each
  // valid for the dt and PCG launch shape it was captured with
  struct NewtonGraph {
    cudaGraphExec_t exec = nullptr;
    double dt = 0.0;
    int blocks = 0, threads = 0;
    int kernels = 0;  // kernel nodes, counted as launches per replay
  };
  NewtonGraph ngraph[8];
  bool graph_off = false;  // capture failed once: plain launches from then on
  bool graph_hold = false; // set while a batched call drives the domain from a worker thread
  int graph_error = 0;     // its cudaError_t
  long long graph_replays = 0;

  // rigid-plane contact (osmpm_set_plane): gaps, prescribed y velocities of
  // held nodes, multipliers per node, candidates, the active set
  osmpm_plane plane{};
  bool plane_on = false;
  bool hold_in_prep = false;  // prep applies the active set as Dirichlet data
  double *plane_gap = nullptr, *plane_hold_v = nullptr, *plane_lam = nullptr;
  unsigned long long* plane_colmin = nullptr;
  uint8_t *plane_cand = nullptr, *plane_act = nullptr, *mask_all = nullptr;
  int* plane_changes = nullptr;
  int contact_sets = 0;

  // optional CUDA-event timing of the PCG launches (osmpm_set_profiling)
  bool time_hvp = false;
  std::vector<cudaEvent_t> hev;  // streaming PCG: around each product of a chunk
  double hvp_ms = 0.0;
  int64_t hvp_launches = 0;
  std::vector<cudaEvent_t> ev;  // one start/stop pair
  double pcg_ms = 0.0;
  long long pcg_launches = 0, pcg_iters = 0;
};

namespace {

// ---------------------------------------------------------------------------
// memory
// ---------------------------------------------------------------------------
osmpm_status dalloc(osmpm_domain* d, size_t bytes, void** out) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (d->have_alloc) {
    p = d->alloc.alloc(bytes, d->alloc.ctx, (void*)d->stream);
    if (!p) return fail(OSMPM_E_NOMEM, "allocator returned NULL for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, d->stream);
    if (e != cudaSuccess) return fail(OSMPM_E_NOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
  }
  d->blocks.emplace_back(p, bytes);
  *out = p;
  return OSMPM_OK;
}

template <class T>
osmpm_status dalloc_n(osmpm_domain* d, int64_t count, T** out) {
  void* p = nullptr;
  OSMPM_TRY(dalloc(d, sizeof(T) * (size_t)count, &p));
  *out = (T*)p;
  return OSMPM_OK;
}

// Device memory outside the domain's block list (the tape, freed with it).
osmpm_status raw_alloc(osmpm_domain* d, size_t bytes, void** out) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (d->have_alloc) {
    p = d->alloc.alloc(bytes, d->alloc.ctx, (void*)d->stream);
    if (!p) return fail(OSMPM_E_NOMEM, "allocator returned NULL for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, d->stream);
    if (e != cudaSuccess) return fail(OSMPM_E_NOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
  }
  *out = p;
  return OSMPM_OK;
}

void raw_free(osmpm_domain* d, void* p, size_t bytes) {
  if (!p) return;
  bytes = (bytes + 255) & ~size_t(255);
  if (d->have_alloc)
    d->alloc.free(p, bytes, d->alloc.ctx, (void*)d->stream);
  else
    cudaFreeAsync(p, d->stream);
}

void clear_tape(osmpm_domain* d) {
  for (auto& t : d->tape) raw_free(d, t.mem, t.bytes);
  d->tape.clear();
  for (auto& c : d->ctape) {
    raw_free(d, c.head.mem, c.head.bytes);
    for (auto& t : c.iters) raw_free(d, t.mem, t.bytes);
  }
  d->ctape.clear();
  for (auto& c : d->ckpts) raw_free(d, c.mem, c.bytes);
  d->ckpts.clear();
  d->ctl.clear();
  d->partner = nullptr;
  d->tape_kind = 0;
  d->tape_broken = false;
}

// Frees a coupled record's per-step blocks, keeping the checkpoints.
void clear_ctape(osmpm_domain* d) {
  for (auto& c : d->ctape) {
    raw_free(d, c.head.mem, c.head.bytes);
    for (auto& t : c.iters) raw_free(d, t.mem, t.bytes);
  }
  d->ctape.clear();
}

void free_all(osmpm_domain* d) {
  clear_tape(d);
  for (auto& b : d->blocks) {
    if (d->have_alloc)
      d->alloc.free(b.first, b.second, d->alloc.ctx, (void*)d->stream);
    else
      cudaFreeAsync(b.first, d->stream);
  }
  d->blocks.clear();
  for (auto& gs : d->ngraph) {
    if (gs.exec) cudaGraphExecDestroy(gs.exec);
    gs = osmpm_domain::NewtonGraph{};
  }
  for (cudaEvent_t e : d->ev) cudaEventDestroy(e);
  d->ev.clear();
  for (cudaEvent_t e : d->hev) cudaEventDestroy(e);
  d->hev.clear();
  if (d->S_host) cudaFreeHost(d->S_host);
  if (d->err_host) cudaFreeHost(d->err_host);
  d->S_host = nullptr;
  d->err_host = nullptr;
}

osmpm_status alloc_parts(osmpm_domain* d, PartMem& P) {
  const int D = d->dim;
  const int64_t n = d->n;
  const size_t rs = d->rsize;
  P.n = n;
  OSMPM_TRY(dalloc_n(d, D * n, &P.x));
  OSMPM_TRY(dalloc(d, rs * D * n, &P.v));
  OSMPM_TRY(dalloc(d, rs * D * D * n, &P.B));
  OSMPM_TRY(dalloc(d, rs * D * D * n, &P.F));
  OSMPM_TRY(dalloc_n(d, n, &P.vol0));
  OSMPM_TRY(dalloc_n(d, n, &P.mass));
  OSMPM_TRY(dalloc_n(d, n, &P.mu));
  OSMPM_TRY(dalloc_n(d, n, &P.lam));
  OSMPM_TRY(dalloc_n(d, n, &P.flags));
  OSMPM_TRY(dalloc_n(d, n, &P.id));
  return OSMPM_OK;
}

// ---------------------------------------------------------------------------
// dispatch over dimension and precision: inside `call`, K is the launcher
// class, R the particle-state type, P_/A_ the typed particle sets, L_ and
// SDN_ the typed Hessian blocks and stencil gradients of domain d
// ---------------------------------------------------------------------------
#define DISPATCH_R(d, Dim, RT, call)           \
  do {                                          \
    using K = Kernels<Dim, RT>;                 \
    using R = RT;                               \
    const PartPtrsT<RT> P_ = typed<RT>((d)->P); \
    const PartPtrsT<RT> A_ = typed<RT>((d)->A); \
    RT* L_ = (RT*)(d)->L;                       \
    RT* SDN_ = (RT*)(d)->sdn;                   \
    (void)P_;                                   \
    (void)A_;                                   \
    (void)L_;                                   \
    (void)SDN_;                                 \
    call;                                       \
  } while (0)
#define DISPATCH(d, call)                                     \
  do {                                                        \
    if ((d)->prec == 0) {                                     \
      if ((d)->dim == 2) DISPATCH_R(d, 2, double, call);      \
      else DISPATCH_R(d, 3, double, call);                    \
    } else {                                                  \
      if ((d)->dim == 2) DISPATCH_R(d, 2, float, call);       \
      else DISPATCH_R(d, 3, float, call);                     \
    }                                                         \
  } while (0)

osmpm_status sync_scalars(osmpm_domain* d) {
  CUDA_TRY(cudaMemcpyAsync(d->S_host, d->S, sizeof(DevScalars), cudaMemcpyDeviceToHost, d->stream));
  CUDA_TRY(cudaMemcpyAsync(d->err_host, d->err, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  CUDA_TRY(cudaGetLastError());
  return OSMPM_OK;
}

osmpm_status check_err(osmpm_domain* d) {
  const int e = *d->err_host;
  if (e & kErrOutOfGrid) return fail(OSMPM_E_OUT_OF_GRID, "a particle's support left the grid box");
  if (e & kErrNonFinite) return fail(OSMPM_E_NONFINITE, "inverted element (J <= 0) at an accepted iterate");
  if (e & kErrBarrierTimeout) return fail(OSMPM_E_TIMEOUT, "a grid barrier of the PCG kernel gave up waiting");
  return OSMPM_OK;
}

// Morton sort of the id-ordered alternate set A into the primary set P.
osmpm_status sort_into_primary(osmpm_domain* d) {
  const int64_t n = d->n;
  DISPATCH(d, K::morton_keys(d->A.x, n, d->geo, d->keys, d->vals, d->err, d->stream));
  int maxres = d->geo.res[0];
  for (int a = 1; a < d->dim; ++a) maxres = std::max(maxres, d->geo.res[a]);
  int bits_axis = 1;
  while ((1 << bits_axis) < maxres) ++bits_axis;
  radix_sort_pairs(d->keys, d->vals, d->keys_alt, d->vals_alt, n, bits_axis * d->dim, d->hist,
                   d->stream);
  DISPATCH(d, K::permute(A_, P_, d->vals, d->stream));
  OSMPM_TRY(sync_scalars(d));
  return check_err(d);
}

osmpm_status upload_rules(osmpm_domain* d, double dt) {
  DevRule host[kMaxRules];
  const int nr = (int)d->rules.size();
  for (int r = 0; r < nr; ++r) {
    const osmpm_dirichlet& s = d->rules[r];
    DevRule& t = host[r];
    memset(&t, 0, sizeof(t));
    t.kind = s.kind;
    t.comp_mask = s.comp_mask;
    for (int a = 0; a < 3; ++a) {
      t.lo[a] = s.lo[a];
      t.hi[a] = s.hi[a];
      t.vel[a] = s.vel[a];
      t.center[a] = s.center[a];
    }
    if (s.kind == 1) {
      // Rodrigues rotation by omega*dt about the unit axis (2D: about z)
      const double th = s.omega * dt;
      const double c = cos(th), sn = sin(th);
      if (d->dim == 2) {
        t.R[0] = c;
        t.R[1] = -sn;
        t.R[3] = sn;
        t.R[4] = c;
      } else {
        double k[3] = {s.axis[0], s.axis[1], s.axis[2]};
        const double nk = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        for (int a = 0; a < 3; ++a) k[a] /= nk;
        const double Kx[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
        double K2[9];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int l = 0; l < 3; ++l) acc += Kx[i * 3 + l] * Kx[l * 3 + j];
            K2[i * 3 + j] = acc;
          }
        for (int i = 0; i < 9; ++i) t.R[i] = ((i % 4) == 0 ? 1.0 : 0.0) + sn * Kx[i] + (1 - c) * K2[i];
      }
    }
  }
  if (nr > 0)
    CUDA_TRY(cudaMemcpyAsync(d->rules_dev, host, sizeof(DevRule) * nr, cudaMemcpyHostToDevice, d->stream));
  return OSMPM_OK;
}

// ---------------------------------------------------------------------------
// grid phases
// ---------------------------------------------------------------------------
int grad_lmode(osmpm_domain* d);

osmpm_status run_p2g(osmpm_domain* d, bool boundary_mass) {
  NvtxRange nvtx_("p2g");
  const int64_t nn = d->geo.nn;
  const int D = d->dim;
  CUDA_TRY(cudaMemsetAsync(d->m, 0, sizeof(double) * nn, d->stream));
  CUDA_TRY(cudaMemsetAsync(d->mv, 0, sizeof(double) * D * nn, d->stream));
  if (boundary_mass) CUDA_TRY(cudaMemsetAsync(d->bm, 0, sizeof(double) * nn, d->stream));
  // the stencil-gradient cache feeds only the lane-group products; a
  // domain on the tiled product alone skips its write (D x 3^D values per
  // particle, most of the P2G's traffic)
  DISPATCH(d, K::p2g(P_, d->geo, d->m, d->mv, boundary_mass ? d->bm : nullptr, d->err, d->sbase,
                     grad_lmode(d) == 2 ? nullptr : SDN_, d->stream));
  DISPATCH(d, K::normalize(d->geo, d->m, d->mv, d->vn, d->stream));
  if (d->slot2p) {
    // the sort scratch (idle between sorts) holds the slot builder's scans
    int* rs = (int*)d->keys;
    int* flag = rs + d->n;
    DISPATCH(d, K::build_slots(d->sbase, d->n, rs, flag, (int*)d->vals, (int*)d->keys_alt,
                               d->slot2p, (int64_t)(1 << D) * d->n, &d->S->n_slots, d->stream));
  }
  return OSMPM_OK;
}

osmpm_status prep(osmpm_domain* d, double dt, bool with_rules, const uint8_t* recv,
                  const double* bc0, const double* bc1, double a_m, uint8_t* physmask) {
  OSMPM_TRY(upload_rules(d, dt));
  PrepArgs a{};
  a.rules = d->rules_dev;
  a.n_rules = with_rules ? (int)d->rules.size() : 0;
  a.recv = recv;
  a.bc0 = bc0;
  a.bc1 = bc1;
  a.a_m = a_m;
  a.bc_applied = d->bc_applied;
  a.physmask = physmask;
  a.hold = d->hold_in_prep ? d->plane_act : nullptr;
  a.hold_v = d->plane_hold_v;
  DISPATCH(d, K::grid_prep(d->geo, d->m, d->vn, a, dt, d->dofmask, d->u, d->stream));
  return OSMPM_OK;
}

struct SolveStats {
  int newton = 0, cg = 0, ls = 0, solves = 0;
  int contact_sets = 0;
  double last_dx = 0.0;
};

// Gradient + Hessian data at the current iterate, then PCG from x = 0 until
// |r| <= rtol |r0| (device-side control, host polls once per chunk).
// Launches the persistent PCG kernel with the domain's buffers (x, r[2],
// s[2], w[3], p) and one block per SM; records the timing events if asked.
template <class R>
PcgArgsT<R> pcg_args(osmpm_domain* d, double dt) {
  PcgArgsT<R> a{};
  a.P = typed<R>(d->P);
  a.g = d->geo;
  a.m = d->m;
  a.dofmask = d->dofmask;
  a.L = (const R*)d->L;
  a.diag = d->diag;
  a.inv_dt2 = 1.0 / (dt * dt);
  a.x = d->cx;
  a.r[0] = d->cr;
  a.r[1] = d->cz;
  a.s[0] = d->cp;
  a.s[1] = d->cp1;
  a.w[0] = d->cq;
  a.w[1] = d->cw1;
  a.w[2] = d->cw2;
  a.p = d->cpp;
  a.S = d->S;
  a.partials = d->partials;
  a.err = d->err;
  a.sbase = d->sbase;
  a.sdn = (const R*)d->sdn;
  a.u = d->u;
  a.slot2p = d->slot2p;
  a.n_slots = &d->S->n_slots;
  const int npk = (d->dim * d->dim) * (d->dim * d->dim + 1) / 2;
  a.tx = (const R*)d->L + (int64_t)npk * d->n;
  return a;
}

// Automatic PCG choice: the persistent kernel while its co-resident grid
// covers the problem in at most kMaxPasses[dim] passes, else the streaming
// kernels (measured: the register-light 2D persistent kernel stays ahead up
// to about 1M particles, the 3D one only for small problems).
constexpr int64_t kMaxPasses2D = 64, kMaxPasses3D = 4;

template <class K, class R>
bool pcg_persistent_fits(osmpm_domain* d, double dt, int64_t work) {
  int blocks = 0, threads = 0;
  K::pcg_shape(work, d->pcg_share, &blocks, &threads);
  const int64_t passes = K::pcg_passes(pcg_args<R>(d, dt), blocks, threads);
  return passes <= (d->dim == 2 ? kMaxPasses2D : kMaxPasses3D);
}

template <class K, class R>
cudaError_t launch_pcg(osmpm_domain* d, double dt, int64_t work, bool timed) {
  const PcgArgsT<R> a = pcg_args<R>(d, dt);
  int blocks = 0, threads = 0;
  K::pcg_shape(work, d->pcg_share, &blocks, &threads);
  if (timed) {
    const cudaError_t e = cudaEventRecord(d->ev[0], d->stream);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t le = K::pcg(a, blocks, threads, d->stream);
  if (le != cudaSuccess) return le;
  if (timed) return cudaEventRecord(d->ev[1], d->stream);
  return cudaSuccess;
}

// Streaming PCG: the start kernel, then chunks of kStreamChunk iterations
// (kernels launched after convergence return at once) with a look at the
// device flags between chunks.
constexpr int kStreamChunk = 16;

template <class K, class R>
cudaError_t stream_pcg_chunk(osmpm_domain* d, double dt, bool first, bool timed) {
  const PcgArgsT<R> a = pcg_args<R>(d, dt);
  if (first) K::cgs_start(a, d->stream);
  for (int i = 0; i < kStreamChunk; ++i) {
    cudaEvent_t e0 = timed ? d->hev[(size_t)2 * i] : nullptr;
    cudaEvent_t e1 = timed ? d->hev[(size_t)2 * i + 1] : nullptr;
    K::cgs_iteration(a, d->desc.hvp_mode, d->stream, e0, e1);
  }
  return cudaGetLastError();
}

// Newton forcing bound: PCG tolerance eta |r0| with eta <= cg_eta_max
// (default kEtaMax).
constexpr double kEtaMax = 1e-3;

osmpm_status run_pcg(osmpm_domain* d, double dt, bool newton, SolveStats& st);

// The confirming Newton step: once the previous step is within
// kCheckRatio x the tolerance, the next one (expected below it) is solved
// only to kCheckEta and accepted when max |delta| <= tol / 2.
constexpr double kCheckRatio = 500.0, kCheckEta = 0.1;

// Gradient, Jacobi diagonal and the PCG start (x = 0, r[0], inverted
// diagonal, tolerance and controls) of a Newton iteration.
void enqueue_gradient(osmpm_domain* d, double dt, bool first, bool check) {
  const int64_t nn = d->geo.nn;
  const int D = d->dim;
  cudaMemsetAsync(d->grad, 0, sizeof(double) * D * nn, d->stream);
  cudaMemsetAsync(d->diag, 0, sizeof(double) * D * nn, d->stream);
  DISPATCH(d, K::grad(P_, d->geo, d->u, d->dofmask, d->grad, d->diag, L_, d->err, d->stream,
                      grad_lmode(d)));
  const double eta_max = d->desc.cg_eta_max > 0.0 ? d->desc.cg_eta_max : kEtaMax;
  const double rtol = check ? std::max(kCheckEta, d->desc.cg_rtol) : d->desc.cg_rtol;
  DISPATCH(d, K::grad_finish(d->geo, d->m, d->vn, d->u, d->dofmask, d->desc.gravity, dt, rtol,
                             check ? rtol : eta_max, first ? 1 : 0, d->desc.cg_max, d->grad,
                             d->diag, d->cx, d->cr, d->cz, d->cp, d->S, d->partials, d->stream));
}

// PCG launch threads: one per DOF, and LPP lanes per particle (GP particles
// per warp).
int64_t pcg_work(const osmpm_domain* d) {
  const int GP = 32 / (d->dim == 2 ? 3 : 9);
  return std::max<int64_t>((d->n + GP - 1) / GP * 32, (int64_t)d->dim * d->geo.nn);
}

// Whether this solve takes the streaming PCG (pcg_mode 2, or 0 when the
// persistent grid would need too many passes) rather than the persistent one.
bool pcg_streaming(osmpm_domain* d, double dt, int64_t work) {
  bool streaming = d->desc.pcg_mode == 2;
  if (d->desc.pcg_mode == 0) DISPATCH(d, (streaming = !pcg_persistent_fits<K, R>(d, dt, work)));
  return streaming;
}

// What the gradient kernel stores for the PCG's products: the packed
// Hessian blocks (FP64, the persistent PCG, the lane-group product) and/or
// the tiled product's per-particle data (mixed precision).  A mixed domain
// whose solves take the streaming PCG with the tiled product, or the
// batched PCG service, needs only the latter (the P2G then also skips the
// stencil-gradient cache).
int grad_lmode(osmpm_domain* d) {
  if (d->prec != 1) return 1;
  if (d->desc.hvp_mode == 1) return 3;
  if (d->batcher || d->desc.pcg_mode == 2) return 2;
  if (d->desc.pcg_mode == 1) return 3;
  return pcg_streaming(d, 1.0, pcg_work(d)) ? 2 : 3;  // automatic (independent of dt)
}

// s[1], w[0..2], p and the barrier counter of the persistent PCG to zero.
void enqueue_pcg_reset(osmpm_domain* d) {
  const size_t vb = sizeof(double) * d->dim * d->geo.nn;
  cudaMemsetAsync(d->cp1, 0, vb, d->stream);
  cudaMemsetAsync(d->cq, 0, vb, d->stream);
  cudaMemsetAsync(d->cw1, 0, vb, d->stream);
  cudaMemsetAsync(d->cw2, 0, vb, d->stream);
  cudaMemsetAsync(d->cpp, 0, vb, d->stream);
  cudaMemsetAsync(&d->S->bar_count, 0, sizeof(unsigned), d->stream);
}

// One Newton iteration's device work up to the host's decision: gradient,
// persistent PCG, max |delta| and the scalars and error word copied to the
// pinned mirrors.  Enqueue errors come back as the first failing status.
cudaError_t enqueue_newton_iteration(osmpm_domain* d, double dt, bool first, bool check, bool timed,
                                     int64_t work) {
  enqueue_gradient(d, dt, first, check);
  enqueue_pcg_reset(d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  DISPATCH(d, (e = launch_pcg<K, R>(d, dt, work, timed)));
  if (e != cudaSuccess) return e;
  DISPATCH(d, K::maxabs(d->geo, d->dofmask, d->cx, d->S, d->partials, d->stream));
  cudaMemcpyAsync(d->S_host, d->S, sizeof(DevScalars), cudaMemcpyDeviceToHost, d->stream);
  cudaMemcpyAsync(d->err_host, d->err, sizeof(int), cudaMemcpyDeviceToHost, d->stream);
  return cudaGetLastError();
}

// Kernel nodes of a graph.
size_t graph_kernels(cudaGraph_t g) {
  size_t nodes = 0, nk = 0;
  if (cudaGraphGetNodes(g, nullptr, &nodes) != cudaSuccess || nodes == 0) return 0;
  std::vector<cudaGraphNode_t> list(nodes);
  if (cudaGraphGetNodes(g, list.data(), &nodes) != cudaSuccess) return 0;
  for (size_t i = 0; i < nodes; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(list[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
  }
  return nk;
}

// The persistent PCG as a cooperative kernel node after `dep` (stream
// capture does not record cooperative launches, graph nodes take them as
// a launch attribute).
template <class K, class R>
cudaError_t add_pcg_node(osmpm_domain* d, double dt, int64_t work, cudaGraph_t g,
                         cudaGraphNode_t dep, cudaGraphNode_t* out) {
  PcgArgsT<R> a = pcg_args<R>(d, dt);
  int blocks = 0, threads = 0;
  K::pcg_shape(work, d->pcg_share, &blocks, &threads);
  void* args[] = {(void*)&a};
  cudaKernelNodeParams kp = {};
  kp.func = const_cast<void*>(K::pcg_kernel(a, blocks, threads));
  kp.gridDim = dim3(blocks);
  kp.blockDim = dim3(threads);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  cudaError_t e = cudaGraphAddKernelNode(out, g, &dep, 1, &kp);
  if (e != cudaSuccess) return e;
  cudaLaunchAttributeValue v = {};
  v.cooperative = 1;
  return cudaGraphKernelNodeSetAttribute(*out, cudaLaunchAttributeCooperative, &v);
}

// Stream work enqueued by `body`, captured (thread-local mode, so domains
// driven by other host threads are not affected) into a new graph.
template <class F>
cudaError_t capture(osmpm_domain* d, F&& body, cudaGraph_t* out) {
  *out = nullptr;
  cudaError_t e = cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  body();
  const cudaError_t eb = cudaGetLastError();
  e = cudaStreamEndCapture(d->stream, out);
  return e != cudaSuccess ? e : eb;
}

// The graph of one Newton iteration for this key, built on first use: the
// captured gradient and PCG set-up, the cooperative PCG node (between event
// records when timed), then the captured max |delta| and scalar read-back.
// nullptr when graphs are off, the domain runs on the legacy default stream
// or building failed; the caller then enqueues the same work directly.
cudaGraphExec_t newton_graph(osmpm_domain* d, double dt, bool first, bool check, bool timed,
                             int64_t work, int* kernels) {
  // the legacy default stream cannot be captured: plain launches there
  if (d->desc.launch_mode != 0 || d->graph_off || d->graph_hold || d->stream == nullptr ||
      d->stream == cudaStreamLegacy)
    return nullptr;
  int blocks = 0, threads = 0;
  DISPATCH(d, K::pcg_shape(work, d->pcg_share, &blocks, &threads));
  osmpm_domain::NewtonGraph& slot = d->ngraph[(first ? 1 : 0) | (check ? 2 : 0) | (timed ? 4 : 0)];
  if (slot.exec && slot.dt == dt && slot.blocks == blocks && slot.threads == threads) {
    *kernels = slot.kernels;
    return slot.exec;
  }
  if (slot.exec) cudaGraphExecDestroy(slot.exec);
  slot = osmpm_domain::NewtonGraph{};
  cudaGraph_t ga = nullptr, gb = nullptr, top = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t nk = 0;
  cudaError_t e = capture(d, [&] {
    enqueue_gradient(d, dt, first, check);
    enqueue_pcg_reset(d);
  }, &ga);
  if (e == cudaSuccess)
    e = capture(d, [&] {
      DISPATCH(d, K::maxabs(d->geo, d->dofmask, d->cx, d->S, d->partials, d->stream));
      cudaMemcpyAsync(d->S_host, d->S, sizeof(DevScalars), cudaMemcpyDeviceToHost, d->stream);
      cudaMemcpyAsync(d->err_host, d->err, sizeof(int), cudaMemcpyDeviceToHost, d->stream);
    }, &gb);
  // the launchers counted the captured kernels; replays count them instead
  const size_t captured = (ga ? graph_kernels(ga) : 0) + (gb ? graph_kernels(gb) : 0);
  g_launch_count -= (long long)captured;
  if (e == cudaSuccess) e = cudaGraphCreate(&top, 0);
  cudaGraphNode_t prev = nullptr, node = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&prev, top, nullptr, 0, ga);
  if (e == cudaSuccess && timed) {
    e = cudaGraphAddEventRecordNode(&node, top, &prev, 1, d->ev[0]);
    prev = node;
  }
  if (e == cudaSuccess) {
    DISPATCH(d, (e = add_pcg_node<K, R>(d, dt, work, top, prev, &node)));
    prev = node;
  }
  if (e == cudaSuccess && timed) {
    e = cudaGraphAddEventRecordNode(&node, top, &prev, 1, d->ev[1]);
    prev = node;
  }
  if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&node, top, &prev, 1, gb);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, top, 0);
  nk = captured + 1;
  if (ga) cudaGraphDestroy(ga);
  if (gb) cudaGraphDestroy(gb);
  if (top) cudaGraphDestroy(top);
  if (e != cudaSuccess || !exec) {
    if (exec) cudaGraphExecDestroy(exec);
    cudaGetLastError();  // a failed capture or build leaves no sticky error
    d->graph_off = true;
    d->graph_error = e != cudaSuccess ? (int)e : -1;
    return nullptr;
  }
  slot.exec = exec;
  slot.dt = dt;
  slot.blocks = blocks;
  slot.threads = threads;
  slot.kernels = (int)nk;
  *kernels = slot.kernels;
  return exec;
}

// After the scalars reached the pinned mirror: the device error word, the
// iteration count and, when timed, the PCG launch's event time.
osmpm_status pcg_finish(osmpm_domain* d, bool timed, SolveStats& st) {
  OSMPM_TRY(check_err(d));
  st.cg += d->S_host->cg_iter;
  if (timed) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, d->ev[0], d->ev[1]));
    d->pcg_ms += ms;
    d->pcg_launches += 1;
    d->pcg_iters += d->S_host->cg_iter;
  }
  return OSMPM_OK;
}

// ---------------------------------------------------------------------------
// Batched PCG service (osmpm_schwarz_couple_multi, mixed precision).  The
// pairs' host threads run Alg. 1 and Newton as in osmpm_schwarz_couple;
// when a Newton iteration needs its PCG, the thread enqueues the gradient
// and PCG start on its stream, waits for it and hands the system to this
// service.  The service batches continuously: the systems in flight iterate
// together in chunks over a work list of (instance, slot tile) and
// (instance, DOF tile) with per-instance scalars and stop flags
// (osmpm_multi.cuh); after each chunk the converged systems leave and the
// systems handed in meanwhile join.  The kernels read the work list and
// their arguments from a device block that is rewritten when the set
// changes, with fixed grids, so one CUDA graph of a chunk serves every
// composition (captured again only when the block grows).
// ---------------------------------------------------------------------------
struct PcgBatcher {
  int dim = 2;
  int dof_tile = 2048;  // DOFs per DOF tile
  int chunk = 16;       // iterations between looks at the stop flags
  int slot_tiles = 1;   // slot tiles per work item of the product
  int grid_pt = 1, grid_dt = 1;  // fixed grids of the product and of the DOF kernels
  cudaStream_t stream = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  struct Req {
    osmpm_domain* d;
    double dt;
    bool done;
    osmpm_status st;
  };
  std::vector<Req*> queue;
  bool stop = false;
  std::thread th;
  // The device block: MultiArgs, then the instance table, infos, slot tiles,
  // DOF tiles (capacities cap_*), the tile partials (3 rows) and the
  // pending words; `host` mirrors it up to the partials (pinned).
  struct Layout {
    size_t inst, info, pt, dt, part, pend, bytes;
    int stride;
  };
  int cap_inst = 0, cap_pt = 0, cap_dt = 0;
  Layout lay{};
  char* dev = nullptr;
  char* host = nullptr;
  int* pending_host = nullptr;  // pending count, then per system: stop flag, iterations
  // the chunk's graph, and the same chunk with every product launch
  // bracketed by event records (replayed every kTimedEvery-th chunk: the
  // records cost ~6 % of the service's device time when in every chunk)
  static constexpr int kTimedEvery = 8;
  cudaGraphExec_t exec = nullptr, exec_timed = nullptr;
  long long per_chunk = 0;  // kernel launches in one replay
  int64_t chunk_no = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> hev;  // around each k_m_hvp of a chunk
  std::string error;
  osmpm_multi_stats stats{};

  static size_t up(size_t b) { return (b + 255) & ~size_t(255); }

  static Layout layout(int ci, int cp, int cd) {
    Layout L{};
    L.inst = up(sizeof(MultiArgs));
    L.info = L.inst + up(sizeof(PcgArgsT<float>) * (size_t)ci);
    L.pt = L.info + up(sizeof(MultiInfo) * (size_t)ci);
    L.dt = L.pt + up(sizeof(MultiTile) * (size_t)cp);
    L.part = L.dt + up(sizeof(MultiTile) * (size_t)cd);
    L.stride = std::max(cp, cd);
    L.pend = L.part + up(sizeof(double) * 3 * (size_t)L.stride);
    L.bytes = L.pend + up(sizeof(int) * (1 + 2 * (size_t)ci));
    return L;
  }

  osmpm_status open(int dim_, int dof_tile_, int chunk_, int slot_tiles_) {
    dim = dim_;
    dof_tile = dof_tile_ > 0 ? dof_tile_ : 2048;
    chunk = chunk_ > 0 ? chunk_ : 16;
    slot_tiles = slot_tiles_ > 0 ? slot_tiles_ : 1;
    int dev_id = 0, sms = 1;
    cudaGetDevice(&dev_id);
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id));
    const int occ = dim == 2 ? MultiKernels<2>::hvp_blocks_per_sm() : MultiKernels<3>::hvp_blocks_per_sm();
    grid_pt = sms * std::max(occ, 1);
    grid_dt = sms * 2;
    CUDA_TRY(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreate(&ev[0]));
    CUDA_TRY(cudaEventCreate(&ev[1]));
    hev.assign((size_t)2 * chunk, nullptr);
    for (auto& e : hev) CUDA_TRY(cudaEventCreate(&e));
    th = std::thread([this, dev_id] {
      cudaSetDevice(dev_id);
      loop();
    });
    return OSMPM_OK;
  }

  void close() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv_work.notify_all();
    if (th.joinable()) th.join();
    if (exec) cudaGraphExecDestroy(exec);
    if (exec_timed) cudaGraphExecDestroy(exec_timed);
    if (stream) cudaStreamSynchronize(stream);
    if (dev) cudaFreeAsync(dev, stream);
    if (stream) cudaStreamSynchronize(stream);
    if (host) cudaFreeHost(host);
    if (pending_host) cudaFreeHost(pending_host);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    for (auto& e : hev)
      if (e) cudaEventDestroy(e);
    if (stream) cudaStreamDestroy(stream);
  }

  // Called by a pair's thread with its system prepared on its (synchronised)
  // stream; returns when the PCG of that system has finished.
  osmpm_status solve(osmpm_domain* d, double dt) {
    Req r{d, dt, false, OSMPM_OK};
    std::unique_lock<std::mutex> lk(mu);
    queue.push_back(&r);
    cv_work.notify_one();
    cv_done.wait(lk, [&] { return r.done; });
    return r.st;
  }

  // The service loop: continuous batching.  The systems in flight ("live")
  // iterate together in chunks; after each chunk the converged ones leave
  // (their threads resume at once) and the systems handed in meanwhile join
  // (their PCG start runs before the next chunk).
  void loop() {
    std::vector<Req*> live;
    std::vector<int> iters_before;  // per live system: its iterations before the chunk
    std::vector<int> fresh_flags;
    bool dirty = false;
    for (;;) {
      std::vector<Req*> fresh;
      {
        std::unique_lock<std::mutex> lk(mu);
        if (live.empty()) cv_work.wait(lk, [&] { return stop || !queue.empty(); });
        if (live.empty() && queue.empty()) break;
        fresh.swap(queue);
      }
      osmpm_status st = OSMPM_OK;
      if (!fresh.empty() || dirty) {
        const size_t old = live.size();
        live.insert(live.end(), fresh.begin(), fresh.end());
        iters_before.resize(live.size(), 0);
        fresh_flags.assign(live.size(), 0);
        for (size_t i = old; i < live.size(); ++i) fresh_flags[i] = 1;
        st = build(live, fresh_flags);
        if (st == OSMPM_OK) {
          stats.batches += 1;
          stats.instances += (int64_t)fresh.size();
          if ((int64_t)live.size() > stats.max_batch) stats.max_batch = (int64_t)live.size();
          if (!fresh.empty()) {
            const MultiArgs* mp = (const MultiArgs*)dev;
            if (dim == 2) MultiKernels<2>::start(mp, grid_dt, stream);
            else MultiKernels<3>::start(mp, grid_dt, stream);
          }
          if (!exec) exec = capture(false);
          if (!exec_timed) exec_timed = capture(true);
        }
        dirty = false;
      }
      if (st == OSMPM_OK) st = run_chunk(live, iters_before);
      // the systems that stopped leave (all of them after a failure)
      std::vector<Req*> done;
      std::vector<Req*> keep;
      std::vector<int> keep_iters;
      for (size_t i = 0; i < live.size(); ++i) {
        const bool stopped = st != OSMPM_OK || pending_host[1 + 2 * i] != 0 ||
                             pending_host[2 + 2 * i] >= live[i]->d->desc.cg_max;
        if (stopped) {
          done.push_back(live[i]);
          if (st == OSMPM_OK) {
            const int it = pending_host[2 + 2 * i];
            stats.iterations += it;
            stats.particle_iterations += (int64_t)it * live[i]->d->n;
            stats.dof_iterations += (int64_t)it * live[i]->d->dim * live[i]->d->geo.nn;
            stats.particles += live[i]->d->n;
            stats.dofs += (int64_t)live[i]->d->dim * live[i]->d->geo.nn;
          }
        } else {
          keep.push_back(live[i]);
          keep_iters.push_back(pending_host[2 + 2 * i]);
        }
      }
      live.swap(keep);
      iters_before.swap(keep_iters);
      dirty = !done.empty();
      {
        std::lock_guard<std::mutex> lk(mu);
        for (Req* r : done) {
          r->st = st;
          r->done = true;
        }
      }
      if (!done.empty()) cv_done.notify_all();
    }
  }

  // Writes the argument block for `live` (fresh[i] = 1 for the systems
  // whose PCG start is still to run), growing it (and dropping the graph)
  // when a table outgrows its capacity.
  osmpm_status build(const std::vector<Req*>& live, const std::vector<int>& fresh) {
    const int n = (int)live.size();
    // a product work item covers slot_tiles tiles of TP slots of one instance
    const int TP = slot_tiles * (dim == 2 ? MultiKernels<2>::particle_tile()
                                          : MultiKernels<3>::particle_tile());
    std::vector<PcgArgsT<float>> inst((size_t)n);
    std::vector<MultiInfo> info((size_t)n);
    std::vector<MultiTile> pt, dtl;
    for (int i = 0; i < n; ++i) {
      osmpm_domain* d = live[(size_t)i]->d;
      inst[(size_t)i] = pcg_args<float>(d, live[(size_t)i]->dt);
      info[(size_t)i].pt0 = (int)pt.size();
      const int64_t ns = d->S_host->n_slots;  // the slots of the last P2G (read back since)
      for (int64_t s0 = 0; s0 < ns; s0 += TP)
        pt.push_back(MultiTile{i, (int)s0, (int)std::min<int64_t>(ns, s0 + TP)});
      info[(size_t)i].npt = (int)pt.size() - info[(size_t)i].pt0;
      info[(size_t)i].dt0 = (int)dtl.size();
      const int64_t ndof = (int64_t)d->dim * d->geo.nn;
      for (int64_t q0 = 0; q0 < ndof; q0 += dof_tile)
        dtl.push_back(MultiTile{i, (int)q0, (int)std::min<int64_t>(ndof, q0 + dof_tile)});
      info[(size_t)i].ndt = (int)dtl.size() - info[(size_t)i].dt0;
      info[(size_t)i].fresh = fresh[(size_t)i];
    }
    CUDA_TRY(cudaStreamSynchronize(stream));  // the block is no longer read
    if (n > cap_inst || (int)pt.size() > cap_pt || (int)dtl.size() > cap_dt || !dev) {
      cap_inst = std::max(cap_inst, n + n / 2 + 8);
      cap_pt = std::max(cap_pt, (int)pt.size() + (int)pt.size() / 2 + 64);
      cap_dt = std::max(cap_dt, (int)dtl.size() + (int)dtl.size() / 2 + 64);
      lay = layout(cap_inst, cap_pt, cap_dt);
      if (exec) cudaGraphExecDestroy(exec);
      if (exec_timed) cudaGraphExecDestroy(exec_timed);
      exec = exec_timed = nullptr;
      if (dev) cudaFreeAsync(dev, stream);
      if (host) cudaFreeHost(host);
      if (pending_host) cudaFreeHost(pending_host);
      dev = host = nullptr;
      pending_host = nullptr;
      if (cudaMallocAsync((void**)&dev, lay.bytes, stream) != cudaSuccess ||
          cudaMallocHost((void**)&host, lay.part) != cudaSuccess ||
          cudaMallocHost((void**)&pending_host, sizeof(int) * (1 + 2 * (size_t)cap_inst)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(OSMPM_E_NOMEM, "batched PCG: memory for the work list");
      }
    }
    MultiArgs m{};
    m.inst = (const PcgArgsT<float>*)(dev + lay.inst);
    m.info = (const MultiInfo*)(dev + lay.info);
    m.pt = (const MultiTile*)(dev + lay.pt);
    m.n_pt = (int)pt.size();
    m.dtl = (const MultiTile*)(dev + lay.dt);
    m.n_dt = (int)dtl.size();
    m.n_inst = n;
    m.part = (double*)(dev + lay.part);
    m.stride = lay.stride;
    m.pending = (int*)(dev + lay.pend);
    memcpy(host, &m, sizeof(m));
    memcpy(host + lay.inst, inst.data(), sizeof(PcgArgsT<float>) * n);
    memcpy(host + lay.info, info.data(), sizeof(MultiInfo) * n);
    if (!pt.empty()) memcpy(host + lay.pt, pt.data(), sizeof(MultiTile) * pt.size());
    if (!dtl.empty()) memcpy(host + lay.dt, dtl.data(), sizeof(MultiTile) * dtl.size());
    const size_t bytes = lay.dt + sizeof(MultiTile) * dtl.size();
    CUDA_TRY(cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, stream));
    return OSMPM_OK;
  }

  void enqueue_chunk(bool capturing, bool timed) {
    const MultiArgs* mp = (const MultiArgs*)dev;
    for (int c = 0; c < chunk; ++c) {
      cudaEvent_t e0 = timed ? hev[(size_t)2 * c] : nullptr;
      cudaEvent_t e1 = timed ? hev[(size_t)2 * c + 1] : nullptr;
      if (dim == 2) MultiKernels<2>::iteration(mp, grid_pt, grid_dt, stream, e0, e1, capturing);
      else MultiKernels<3>::iteration(mp, grid_pt, grid_dt, stream, e0, e1, capturing);
    }
    if (dim == 2) MultiKernels<2>::pending(mp, stream);
    else MultiKernels<3>::pending(mp, stream);
    cudaMemcpyAsync(pending_host, dev + lay.pend, sizeof(int) * (1 + 2 * (size_t)cap_inst),
                    cudaMemcpyDeviceToHost, stream);
  }

  // The chunk as a CUDA graph over the current block (nullptr: plain
  // launches); timed: with the product launches bracketed by events.
  cudaGraphExec_t capture(bool timed) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t ex = nullptr;
    const long long before = g_launch_count.load();
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      enqueue_chunk(true, timed);
      if (cudaStreamEndCapture(stream, &graph) != cudaSuccess || !graph ||
          cudaGraphInstantiate(&ex, graph, 0) != cudaSuccess)
        ex = nullptr;
    }
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    per_chunk = g_launch_count.load() - before;
    g_launch_count -= per_chunk;  // counted when replayed or launched
    return ex;
  }

  osmpm_status run_chunk(const std::vector<Req*>& live, const std::vector<int>& iters_before) {
    NvtxRange nvtx_("batched_pcg_chunk");
    const bool timed = (chunk_no++ % kTimedEvery) == 0;
    cudaGraphExec_t g = timed ? exec_timed : exec;
    cudaEventRecord(ev[0], stream);
    cudaError_t e;
    if (g) {
      e = cudaGraphLaunch(g, stream);
      g_launch_count += per_chunk;
    } else {
      enqueue_chunk(false, timed);
      e = cudaGetLastError();
    }
    cudaEventRecord(ev[1], stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return set_error(OSMPM_E_CUDA, "batched PCG: %s", cudaGetErrorString(e));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    stats.chunks += 1;
    stats.device_ms += ms;
    if (timed) {
      for (int c = 0; c < chunk; ++c) {
        float h = 0.f;
        if (cudaEventElapsedTime(&h, hev[(size_t)2 * c], hev[(size_t)2 * c + 1]) == cudaSuccess) {
          stats.hvp_ms += h;
          stats.hvp_launches += 1;
        }
      }
      cudaGetLastError();
      // the particle-iterations those launches carried: each system's
      // iterations in this chunk times its particles
      for (size_t i = 0; i < live.size(); ++i)
        stats.hvp_particle_iterations +=
            (int64_t)std::max(0, pending_host[2 + 2 * i] - iters_before[i]) * live[i]->d->n;
    }
    return OSMPM_OK;
  }
};

// One Newton iteration's gradient and PCG solve, up to the host's look at
// max |delta|: a replayed graph where launch_mode 0 allows one, else the
// same work launched directly; the streaming PCG always launches directly.
osmpm_status gradient_and_pcg(osmpm_domain* d, double dt, bool first, bool check, SolveStats& st) {
  NvtxRange nvtx_("newton_iteration");
  const int64_t work = pcg_work(d);
  const bool timed = d->time_hvp && !d->ev.empty();
  if (d->batcher) {
    // the batched PCG service solves the system with the other pairs' ones
    // (the scalars read back here carry the slot count of the last P2G)
    enqueue_gradient(d, dt, first, check);
    OSMPM_TRY(sync_scalars(d));
    OSMPM_TRY(d->batcher->solve(d, dt));
    DISPATCH(d, K::maxabs(d->geo, d->dofmask, d->cx, d->S, d->partials, d->stream));
    OSMPM_TRY(sync_scalars(d));
    return pcg_finish(d, false, st);
  }
  if (pcg_streaming(d, dt, work)) {
    enqueue_gradient(d, dt, first, check);
    CUDA_TRY(cudaGetLastError());
    return run_pcg(d, dt, true, st);
  }
  int kernels = 0;
  const cudaGraphExec_t g = newton_graph(d, dt, first, check, timed, work, &kernels);
  if (g) {
    CUDA_TRY(cudaGraphLaunch(g, d->stream));
    g_launch_count += kernels;
    d->graph_replays += 1;
  } else {
    const cudaError_t e = enqueue_newton_iteration(d, dt, first, check, timed, work);
    if (e != cudaSuccess) return fail(OSMPM_E_CUDA, "Newton iteration launch: %s", cudaGetErrorString(e));
  }
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  CUDA_TRY(cudaGetLastError());
  return pcg_finish(d, timed, st);
}

// The whole PCG in one cooperative launch on a prepared system (x = 0, r[0],
// the inverted diagonal and the controls in place): s[1], w[0..2], p and the
// barrier counter start at zero.  With `newton` also reduces max |x| for the
// Newton stop test.
osmpm_status run_pcg(osmpm_domain* d, double dt, bool newton, SolveStats& st) {
  NvtxRange nvtx_("pcg");
  enqueue_pcg_reset(d);
  CUDA_TRY(cudaGetLastError());
  const int64_t work = pcg_work(d);
  const bool timed = d->time_hvp && !d->ev.empty();
  cudaError_t le = cudaSuccess;
  if (!pcg_streaming(d, dt, work)) {
    DISPATCH(d, (le = launch_pcg<K, R>(d, dt, work, timed)));
    if (le != cudaSuccess) return fail(OSMPM_E_CUDA, "cooperative PCG launch: %s", cudaGetErrorString(le));
  } else {
    if (timed) CUDA_TRY(cudaEventRecord(d->ev[0], d->stream));
    int done_iters = 0;
    for (bool first = true;; first = false) {
      DISPATCH(d, (le = stream_pcg_chunk<K, R>(d, dt, first, timed)));
      if (le != cudaSuccess) return fail(OSMPM_E_CUDA, "streaming PCG launch: %s", cudaGetErrorString(le));
      OSMPM_TRY(sync_scalars(d));
      if (timed) {
        // the products of this chunk's iterations that ran (later ones
        // returned at once)
        const int ran = std::min(kStreamChunk, std::max(0, d->S_host->cg_iter - done_iters));
        for (int i = 0; i < ran; ++i) {
          float h = 0.f;
          CUDA_TRY(cudaEventElapsedTime(&h, d->hev[(size_t)2 * i], d->hev[(size_t)2 * i + 1]));
          d->hvp_ms += h;
          d->hvp_launches += 1;
        }
        done_iters = d->S_host->cg_iter;
      }
      if (d->S_host->cg_done || d->S_host->err) break;
    }
    if (timed) CUDA_TRY(cudaEventRecord(d->ev[1], d->stream));
  }
  if (newton) DISPATCH(d, K::maxabs(d->geo, d->dofmask, d->cx, d->S, d->partials, d->stream));
  OSMPM_TRY(sync_scalars(d));
  return pcg_finish(d, timed, st);
}

// Newton's method with backtracking line search (Sec. 2.2.5) on the
// prepared grid (P2G done, Dirichlet data and initial guess in place).
// Cold start of Newton: of the prepared x_tilde = x^n + dt v^n and x^n (free
// DOFs; fixed DOFs keep their prescribed values), keep the one with the lower
// E_h.  x^n is taken only when E_h(x_tilde) - E_h(x^n) > 0 (+inf when x_tilde
// inverts an element), so x_tilde stays the start whenever it is no worse.
osmpm_status cold_start(osmpm_domain* d, double dt) {
  DISPATCH(d, K::split_free(d->geo, d->dofmask, d->u, d->cx, d->stream));
  DISPATCH(d, K::energy_change(P_, d->geo, d->m, d->vn, d->u, d->cx, d->desc.gravity, dt, 1.0,
                               d->S, d->partials, d->stream));
  OSMPM_TRY(sync_scalars(d));
  if (!(d->S_host->dE > 0.0)) DISPATCH(d, K::axpy(d->geo, d->u, d->cx, 1.0, d->stream));
  return OSMPM_OK;
}

osmpm_status newton_solve(osmpm_domain* d, double dt, SolveStats& st) {
  NvtxRange nvtx_("newton");
  st.solves++;
  const double tol = d->desc.newton_tol * dt;
  double prev_dx = INFINITY;
  for (int it = 0; it < d->desc.newton_max; ++it) {
    st.newton++;
    const bool check = it > 0 && prev_dx <= kCheckRatio * tol;
    OSMPM_TRY(gradient_and_pcg(d, dt, it == 0, check, st));
    const double dxinf = d->S_host->maxabs;
    st.last_dx = dxinf;
    if (!std::isfinite(dxinf)) return fail(OSMPM_E_NONFINITE, "non-finite Newton step");
    if (dxinf <= (check ? 0.5 * tol : tol)) {
      DISPATCH(d, K::axpy(d->geo, d->u, d->cx, 1.0, d->stream));
      return OSMPM_OK;
    }
    double alpha = 1.0;
    bool ok = false;
    for (int s = 0; s <= d->desc.ls_max; ++s) {
      DISPATCH(d, K::energy_change(P_, d->geo, d->m, d->vn, d->u, d->cx, d->desc.gravity, dt,
                                   alpha, d->S, d->partials, d->stream));
      OSMPM_TRY(sync_scalars(d));
      if (d->S_host->dE < 0.0) {
        ok = true;
        break;
      }
      alpha *= 0.5;
      st.ls++;
    }
    if (!ok) return fail(OSMPM_E_LINESEARCH, "no decrease of E_h after %d halvings", d->desc.ls_max);
    DISPATCH(d, K::axpy(d->geo, d->u, d->cx, alpha, d->stream));
    prev_dx = alpha * dxinf;
  }
  return fail(OSMPM_E_NEWTON_MAXITER, "Newton did not reach %g in %d iterations (last |dx| %g)",
              d->desc.newton_tol, d->desc.newton_max, st.last_dx);
}

// One implicit solve with the rigid plane (the primal-dual active set of
// the unilateral contact, osmpm_contact.cuh): gaps and the initial active
// set from the prepared grid, then solve with the held nodes' y prescribed,
// multipliers from the full gradient, update the set, until it no longer
// changes.  u holds the last solve.
osmpm_status contact_solve(osmpm_domain* d, double dt, SolveStats& st) {
  cudaStream_t s = d->stream;
  const int D = d->dim;
  const int64_t nn = d->geo.nn;
  OSMPM_TRY(prep(d, dt, true, nullptr, nullptr, nullptr, 0.0, d->physmask));
  CUDA_TRY(cudaMemsetAsync(d->plane_colmin, 0xFF, sizeof(unsigned long long) * d->geo.res[0], s));
  DISPATCH(d, K::plane_colmin(P_, d->geo, d->plane.spacing, d->plane_colmin, s));
  DISPATCH(d, K::plane_init(d->geo, d->m, d->physmask, d->plane_colmin, d->plane.level,
                            d->plane.cand_hi, d->plane.spacing, dt, d->plane_gap, d->plane_hold_v,
                            d->plane_cand, d->plane_act, s));
  const int max_sets = d->plane.max_sets > 0 ? d->plane.max_sets : 50;
  for (int set = 0; set < max_sets; ++set) {
    d->hold_in_prep = true;
    const osmpm_status e = prep(d, dt, true, nullptr, nullptr, nullptr, 0.0, nullptr);
    d->hold_in_prep = false;
    OSMPM_TRY(e);
    OSMPM_TRY(cold_start(d, dt));
    OSMPM_TRY(newton_solve(d, dt, st));
    // lambda = dE_h/du_y on the held nodes: the gradient with every active DOF free
    CUDA_TRY(cudaMemsetAsync(d->grad, 0, sizeof(double) * D * nn, s));
    CUDA_TRY(cudaMemsetAsync(d->diag, 0, sizeof(double) * D * nn, s));
    DISPATCH(d, K::mask_all(d->geo, d->m, d->mask_all, s));
    DISPATCH(d, K::grad(P_, d->geo, d->u, d->mask_all, d->grad, d->diag, L_, d->err, s));
    DISPATCH(d, K::grad_finish(d->geo, d->m, d->vn, d->u, d->mask_all, d->desc.gravity, dt,
                               d->desc.cg_rtol, d->desc.cg_rtol, 1, d->desc.cg_max, d->grad,
                               d->diag, d->cx, d->cr, d->cz, d->cp, d->S, d->partials, s));
    CUDA_TRY(cudaMemsetAsync(d->plane_changes, 0, sizeof(int), s));
    DISPATCH(d, K::plane_update(d->geo, d->plane_cand, d->grad, d->u, d->plane_gap, d->plane_act,
                                d->plane_lam, d->plane_changes, s));
    int changes = 0;
    CUDA_TRY(cudaMemcpyAsync(&changes, d->plane_changes, sizeof(int), cudaMemcpyDeviceToHost, s));
    OSMPM_TRY(sync_scalars(d));
    OSMPM_TRY(check_err(d));
    st.contact_sets = set + 1;
    if (changes == 0) return OSMPM_OK;
  }
  return fail(OSMPM_E_NEWTON_MAXITER, "the contact active set did not settle in %d sets", max_sets);
}

void fill_stats(osmpm_stats* out, const SolveStats& st, int schwarz_iters, int converged, double rB,
                double rS) {
  if (!out) return;
  memset(out, 0, sizeof(*out));
  out->newton_iters = st.newton;
  out->cg_iters = st.cg;
  out->ls_halvings = st.ls;
  out->solves = st.solves;
  out->schwarz_iters = schwarz_iters;
  out->converged = converged;
  out->r_B = rB;
  out->r_S = rS;
  out->last_dx_inf = st.last_dx;
  out->contact_sets = st.contact_sets;
}

osmpm_status ensure_keep(osmpm_domain* d, int slots) {
  if (d->n_keep >= slots) return OSMPM_OK;
  OSMPM_TRY(dalloc_n(d, (int64_t)slots * d->dim * d->geo.nn, &d->u_keep));
  d->n_keep = slots;
  return OSMPM_OK;
}

double* keep_slot(osmpm_domain* d, int slot) { return d->u_keep + (int64_t)slot * d->dim * d->geo.nn; }

osmpm_status snapshot(osmpm_domain* d, bool restore) {
  const int D = d->dim;
  const int64_t n = d->n;
  const size_t rs = d->rsize;
  auto cp = [&](void* a, void* b, size_t bytes) {
    return cudaMemcpyAsync(restore ? a : b, restore ? b : a, bytes, cudaMemcpyDeviceToDevice,
                           d->stream);
  };
  CUDA_TRY(cp(d->P.x, d->snap_x, sizeof(double) * D * n));
  CUDA_TRY(cp(d->P.v, d->snap_v, rs * D * n));
  CUDA_TRY(cp(d->P.B, d->snap_B, rs * D * D * n));
  CUDA_TRY(cp(d->P.F, d->snap_F, rs * D * D * n));
  return OSMPM_OK;
}

bool finite_all(const double* a, int64_t cnt) {
  for (int64_t i = 0; i < cnt; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

osmpm_status check_domain(const osmpm_domain* d) {
  if (!d) return fail(OSMPM_E_INVALID, "null domain");
  return OSMPM_OK;
}

// Uploads host arrays (id order, particle-major) into A (component-major).
osmpm_status upload_state(osmpm_domain* d, const double* x, const double* v, const double* B,
                          const double* F) {
  const int D = d->dim;
  const int64_t n = d->n;
  double* sx = d->stage;
  double* sv = sx + D * n;
  double* sB = sv + D * n;
  double* sF = sB + D * D * n;
  CUDA_TRY(cudaMemcpyAsync(sx, x, sizeof(double) * D * n, cudaMemcpyHostToDevice, d->stream));
  CUDA_TRY(cudaMemcpyAsync(sv, v, sizeof(double) * D * n, cudaMemcpyHostToDevice, d->stream));
  CUDA_TRY(cudaMemcpyAsync(sB, B, sizeof(double) * D * D * n, cudaMemcpyHostToDevice, d->stream));
  CUDA_TRY(cudaMemcpyAsync(sF, F, sizeof(double) * D * D * n, cudaMemcpyHostToDevice, d->stream));
  DISPATCH(d, K::unpack_in(sx, sv, sB, sF, A_, d->stream));
  return OSMPM_OK;
}

// host node-major <-> device component-major grid vectors
osmpm_status upload_grid_vec(osmpm_domain* d, const double* host, double* dev) {
  const int D = d->dim;
  const int64_t nn = d->geo.nn;
  std::vector<double> tmp((size_t)(D * nn));
  for (int64_t i = 0; i < nn; ++i)
    for (int a = 0; a < D; ++a) tmp[(size_t)(a * nn + i)] = host[i * D + a];
  CUDA_TRY(cudaMemcpyAsync(dev, tmp.data(), sizeof(double) * D * nn, cudaMemcpyHostToDevice, d->stream));
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  return OSMPM_OK;
}

osmpm_status download_grid_vec(osmpm_domain* d, const double* dev, double* host, int comps) {
  const int64_t nn = d->geo.nn;
  std::vector<double> tmp((size_t)(comps * nn));
  CUDA_TRY(cudaMemcpyAsync(tmp.data(), dev, sizeof(double) * comps * nn, cudaMemcpyDeviceToHost, d->stream));
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  for (int64_t i = 0; i < nn; ++i)
    for (int a = 0; a < comps; ++a) host[i * comps + a] = tmp[(size_t)(a * nn + i)];
  return OSMPM_OK;
}

osmpm_status probe_setup(osmpm_domain* d, double dt, const double* u_host) {
  if (!(dt > 0.0)) return fail(OSMPM_E_INVALID, "dt must be > 0");
  CUDA_TRY(cudaMemsetAsync(d->err, 0, sizeof(int), d->stream));
  OSMPM_TRY(run_p2g(d, false));
  OSMPM_TRY(prep(d, dt, false, nullptr, nullptr, nullptr, 0.0, nullptr));
  OSMPM_TRY(upload_grid_vec(d, u_host, d->u));
  OSMPM_TRY(sync_scalars(d));
  return check_err(d);
}

// Tape slot layout: x, v, B, F (sorted order, component-major), u, DOF mask.
struct TapeLayout {
  size_t x, v, B, F, u, mask, bytes;
  explicit TapeLayout(const osmpm_domain* d) {
    const size_t D = d->dim, n = (size_t)d->n, nn = (size_t)d->geo.nn;
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    x = 0;
    v = x + up(8 * D * n);
    B = v + up(8 * D * n);
    F = B + up(8 * D * D * n);
    u = F + up(8 * D * D * n);
    mask = u + up(8 * D * nn);
    bytes = mask + up(nn);
  }
};

osmpm_status tape_begin(osmpm_domain* d, osmpm_domain::TapeStep& slot) {
  const TapeLayout L(d);
  const size_t D = d->dim, n = (size_t)d->n;
  OSMPM_TRY(raw_alloc(d, L.bytes, &slot.mem));
  slot.bytes = L.bytes;
  char* b = (char*)slot.mem;
  CUDA_TRY(cudaMemcpyAsync(b + L.x, d->P.x, 8 * D * n, cudaMemcpyDeviceToDevice, d->stream));
  CUDA_TRY(cudaMemcpyAsync(b + L.v, d->P.v, 8 * D * n, cudaMemcpyDeviceToDevice, d->stream));
  CUDA_TRY(cudaMemcpyAsync(b + L.B, d->P.B, 8 * D * D * n, cudaMemcpyDeviceToDevice, d->stream));
  CUDA_TRY(cudaMemcpyAsync(b + L.F, d->P.F, 8 * D * D * n, cudaMemcpyDeviceToDevice, d->stream));
  return OSMPM_OK;
}

osmpm_status tape_end(osmpm_domain* d, osmpm_domain::TapeStep& slot, double dt) {
  const TapeLayout L(d);
  const size_t D = d->dim, nn = (size_t)d->geo.nn;
  char* b = (char*)slot.mem;
  CUDA_TRY(cudaMemcpyAsync(b + L.u, d->u, 8 * D * nn, cudaMemcpyDeviceToDevice, d->stream));
  CUDA_TRY(cudaMemcpyAsync(b + L.mask, d->dofmask, nn, cudaMemcpyDeviceToDevice, d->stream));
  slot.dt = dt;
  d->tape.push_back(slot);
  slot.mem = nullptr;
  return OSMPM_OK;
}

// Coupled-step record layout (coarse domain B, fine domain S, M sub-steps).
// Head: both start states (x, v, B, F contiguous), the receiver masks and
// the k = 0 projection sums.  Per iteration: the coarse solution and DOF
// mask, per sub-step the fine state entering it (from the second sub-step
// on), its solution and DOF mask, and the iteration's projection sums.
struct CoupledLayout {
  size_t stB, stS, recvB, recvS, N0, D0, head_bytes;
  size_t uB, maskB, N, Dn, iter_bytes;
  std::vector<size_t> state, uS, maskS;
  CoupledLayout(const osmpm_domain* B, const osmpm_domain* S, int M) {
    const size_t D = B->dim, DD = D * D, nB = (size_t)B->n, nS = (size_t)S->n;
    const size_t nnB = (size_t)B->geo.nn, nnS = (size_t)S->geo.nn;
    size_t o = 0;
    auto take = [&](size_t bytes) {
      const size_t r = o;
      o += (bytes + 255) & ~size_t(255);
      return r;
    };
    stB = take(8 * (2 * D + 2 * DD) * nB);
    stS = take(8 * (2 * D + 2 * DD) * nS);
    recvB = take(nnB);
    recvS = take(nnS);
    N0 = take(8 * D * nnB);
    D0 = take(8 * nnB);
    head_bytes = o;
    o = 0;
    uB = take(8 * D * nnB);
    maskB = take(nnB);
    state.assign(M, 0);
    uS.assign(M, 0);
    maskS.assign(M, 0);
    for (int m = 0; m < M; ++m) {
      if (m > 0) state[m] = take(8 * (2 * D + 2 * DD) * nS);
      uS[m] = take(8 * D * nnS);
      maskS[m] = take(nnS);
    }
    N = take(8 * D * nnB);
    Dn = take(8 * nnB);
    iter_bytes = o;
  }
};

// Copies of an FP64 particle state (x, v, B, F) to and from a contiguous block.
osmpm_status save_state(osmpm_domain* d, char* b) {
  const size_t D = d->dim, n = (size_t)d->n;
  const size_t off[4] = {0, 8 * D * n, 16 * D * n, 8 * (2 * D + D * D) * n};
  const size_t len[4] = {8 * D * n, 8 * D * n, 8 * D * D * n, 8 * D * D * n};
  void* src[4] = {d->P.x, d->P.v, d->P.B, d->P.F};
  for (int i = 0; i < 4; ++i)
    CUDA_TRY(cudaMemcpyAsync(b + off[i], src[i], len[i], cudaMemcpyDeviceToDevice, d->stream));
  return OSMPM_OK;
}
osmpm_status load_state(osmpm_domain* d, const char* b) {
  const size_t D = d->dim, n = (size_t)d->n;
  const size_t off[4] = {0, 8 * D * n, 16 * D * n, 8 * (2 * D + D * D) * n};
  const size_t len[4] = {8 * D * n, 8 * D * n, 8 * D * D * n, 8 * D * D * n};
  void* dst[4] = {d->P.x, d->P.v, d->P.B, d->P.F};
  for (int i = 0; i < 4; ++i)
    CUDA_TRY(cudaMemcpyAsync(dst[i], b + off[i], len[i], cudaMemcpyDeviceToDevice, d->stream));
  return OSMPM_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* osmpm_last_error(void) { return g_last_error.c_str(); }

osmpm_status osmpm_create_domain(const osmpm_domain_desc* desc, const osmpm_particles_in* pin,
                                 const osmpm_allocator* allocator, void* cuda_stream,
                                 osmpm_domain** out) {
  if (!desc || !pin || !out) return fail(OSMPM_E_INVALID, "null argument");
  *out = nullptr;
  if (desc->dim != 2 && desc->dim != 3) return fail(OSMPM_E_INVALID, "dim must be 2 or 3");
  if (desc->precision != 0 && desc->precision != 1)
    return fail(OSMPM_E_INVALID, "precision must be 0 (FP64) or 1 (mixed)");
  for (int i = 0; i < 3; ++i)
    if (desc->reserved[i] != 0) return fail(OSMPM_E_INVALID, "reserved fields must be zero");
  if (desc->pcg_mode < 0 || desc->pcg_mode > 2) return fail(OSMPM_E_INVALID, "pcg_mode must be 0, 1 or 2");
  if (desc->hvp_mode < 0 || desc->hvp_mode > 2) return fail(OSMPM_E_INVALID, "hvp_mode must be 0, 1 or 2");
  if (desc->launch_mode != 0 && desc->launch_mode != 1)
    return fail(OSMPM_E_INVALID, "launch_mode must be 0 (graphs) or 1 (plain launches)");
  if (!(desc->cg_eta_max >= 0.0 && desc->cg_eta_max < 1.0))
    return fail(OSMPM_E_INVALID, "cg_eta_max must be in [0, 1)");
  if (!(desc->dx > 0.0) || !std::isfinite(desc->dx)) return fail(OSMPM_E_INVALID, "dx must be > 0");
  int64_t nn = 1;
  for (int a = 0; a < desc->dim; ++a) {
    if (desc->res[a] < 4 || desc->res[a] > (1 << 20))
      return fail(OSMPM_E_INVALID, "res[%d] = %d out of range [4, 2^20]", a, desc->res[a]);
    nn *= desc->res[a];
  }
  if (!(desc->newton_tol > 0.0) || desc->newton_max < 1 || !(desc->cg_rtol > 0.0) ||
      desc->cg_max < 1 || desc->ls_max < 0 || !(desc->mass_eps >= 0.0) || !std::isfinite(desc->mass_eps))
    return fail(OSMPM_E_INVALID, "bad solver controls");
  if (pin->n < 1 || pin->n > (int64_t)0x7fffffff) return fail(OSMPM_E_INVALID, "particle count out of range");
  if (!pin->x || !pin->v || !pin->B || !pin->F || !pin->vol0 || !pin->mass || !pin->E || !pin->nu ||
      !pin->flags)
    return fail(OSMPM_E_INVALID, "null particle array");
  const int D = desc->dim;
  const int64_t n = pin->n;
  if (!finite_all(pin->x, D * n) || !finite_all(pin->v, D * n) || !finite_all(pin->B, D * D * n) ||
      !finite_all(pin->F, D * D * n) || !finite_all(pin->vol0, n) || !finite_all(pin->mass, n) ||
      !finite_all(pin->E, n) || !finite_all(pin->nu, n))
    return fail(OSMPM_E_NONFINITE, "non-finite particle input");
  for (int64_t p = 0; p < n; ++p)
    if (!(pin->nu[p] < 0.5) || !(pin->nu[p] > -1.0) || !(pin->mass[p] > 0.0) || !(pin->vol0[p] > 0.0))
      return fail(OSMPM_E_INVALID, "particle %lld: need -1 < nu < 0.5, mass > 0, vol0 > 0", (long long)p);

  osmpm_domain* d = new osmpm_domain();
  d->desc = *desc;
  d->dim = D;
  d->n = n;
  d->prec = desc->precision;
  d->rsize = d->prec == 0 ? sizeof(double) : sizeof(float);
  d->stream = (cudaStream_t)cuda_stream;
  if (allocator && allocator->alloc && allocator->free) {
    d->alloc = *allocator;
    d->have_alloc = true;
  }
  GridGeo& g = d->geo;
  for (int a = 0; a < 3; ++a) {
    g.o[a] = a < D ? desc->origin[a] : 0.0;
    g.res[a] = a < D ? desc->res[a] : 1;
  }
  g.dx = desc->dx;
  g.inv_dx = 1.0 / desc->dx;
  g.nn = nn;
  g.mass_eps = desc->mass_eps;

  auto cleanup = [&](osmpm_status st) {
    free_all(d);
    delete d;
    return st;
  };
#define C_TRY(expr)                          \
  do {                                       \
    osmpm_status s_ = (expr);                \
    if (s_ != OSMPM_OK) return cleanup(s_);  \
  } while (0)

  C_TRY(alloc_parts(d, d->P));
  C_TRY(alloc_parts(d, d->A));
  C_TRY(dalloc_n(d, D * n, &d->snap_x));
  C_TRY(dalloc(d, d->rsize * D * n, &d->snap_v));
  C_TRY(dalloc(d, d->rsize * D * D * n, &d->snap_B));
  C_TRY(dalloc(d, d->rsize * D * D * n, &d->snap_F));
  C_TRY(dalloc_n(d, (2 * D + 2 * D * D) * n, &d->stage));
  C_TRY(dalloc_n(d, n, &d->keys));
  C_TRY(dalloc_n(d, n, &d->keys_alt));
  C_TRY(dalloc_n(d, n, &d->vals));
  C_TRY(dalloc_n(d, n, &d->vals_alt));
  C_TRY(dalloc_n(d, 256 * radix_tiles(n), &d->hist));
  C_TRY(dalloc_n(d, nn, &d->m));
  C_TRY(dalloc_n(d, D * nn, &d->mv));
  C_TRY(dalloc_n(d, D * nn, &d->vn));
  C_TRY(dalloc_n(d, nn, &d->bm));
  C_TRY(dalloc_n(d, D * nn, &d->u));
  C_TRY(dalloc_n(d, D * nn, &d->grad));
  C_TRY(dalloc_n(d, D * nn, &d->diag));
  C_TRY(dalloc_n(d, D * nn, &d->cx));
  C_TRY(dalloc_n(d, D * nn, &d->cr));
  C_TRY(dalloc_n(d, D * nn, &d->cz));
  C_TRY(dalloc_n(d, D * nn, &d->cp));
  C_TRY(dalloc_n(d, D * nn, &d->cp1));
  C_TRY(dalloc_n(d, D * nn, &d->cw1));
  C_TRY(dalloc_n(d, D * nn, &d->cw2));
  C_TRY(dalloc_n(d, D * nn, &d->cpp));
  C_TRY(dalloc_n(d, D * nn, &d->cq));
  const int npk = (D * D) * (D * D + 1) / 2;
  // mixed precision: the Hessian blocks, then the per-particle data of the
  // tiled product at the Newton iterate, and the particles' slots
  C_TRY(dalloc(d, d->rsize * (npk + (d->prec == 1 ? tile_x_count(D) : 0)) * n, &d->L));
  if (d->prec == 1) C_TRY(dalloc_n(d, (int64_t)(1 << D) * n, &d->slot2p));
  C_TRY(dalloc_n(d, n, &d->sbase));
  C_TRY(dalloc(d, d->rsize * D * (D == 2 ? 9 : 27) * n, &d->sdn));
  C_TRY(dalloc_n(d, nn, &d->dofmask));
  C_TRY(dalloc_n(d, nn, &d->physmask));
  C_TRY(dalloc_n(d, nn, &d->gam));
  C_TRY(dalloc_n(d, nn, &d->recv));
  C_TRY(dalloc_n(d, D * nn, &d->bc0));
  C_TRY(dalloc_n(d, D * nn, &d->bc1));
  C_TRY(dalloc_n(d, D * nn, &d->bc_prev));
  C_TRY(dalloc_n(d, D * nn, &d->bc_applied));
  C_TRY(dalloc_n(d, D * nn, &d->vtmp));
  C_TRY(dalloc_n(d, D * nn, &d->proj_num));
  C_TRY(dalloc_n(d, nn, &d->proj_den));
  C_TRY(dalloc_n(d, kMaxRules, &d->rules_dev));
  C_TRY(dalloc_n(d, 1, &d->S));
  const int64_t maxblk = std::max<int64_t>(red_blocks_for(std::max<int64_t>(n, D * nn)), kRedBlocksMax);
  C_TRY(dalloc_n(d, 4 * std::max<int64_t>(maxblk, 152 * 64), &d->partials));
  C_TRY(dalloc_n(d, 1, &d->err));
  if (cudaMallocHost(&d->S_host, sizeof(DevScalars)) != cudaSuccess ||
      cudaMallocHost(&d->err_host, sizeof(int)) != cudaSuccess)
    return cleanup(fail(OSMPM_E_NOMEM, "cudaMallocHost failed"));
  if (cudaMemsetAsync(d->S, 0, sizeof(DevScalars), d->stream) != cudaSuccess ||
      cudaMemsetAsync(d->err, 0, sizeof(int), d->stream) != cudaSuccess ||
      cudaMemsetAsync(d->recv, 0, nn, d->stream) != cudaSuccess ||
      cudaMemsetAsync(d->bc_applied, 0, sizeof(double) * D * nn, d->stream) != cudaSuccess ||
      cudaMemsetAsync(d->u, 0, sizeof(double) * D * nn, d->stream) != cudaSuccess ||
      cudaMemsetAsync(d->m, 0, sizeof(double) * nn, d->stream) != cudaSuccess ||
      cudaMemsetAsync(d->vn, 0, sizeof(double) * D * nn, d->stream) != cudaSuccess ||
      cudaMemsetAsync(d->bm, 0, sizeof(double) * nn, d->stream) != cudaSuccess)
    return cleanup(fail(OSMPM_E_CUDA, "initial memset failed"));

  // Upload in id order into A, material constants, then Morton sort into P.
  C_TRY(upload_state(d, pin->x, pin->v, pin->B, pin->F));
  // E and nu go through the staging area (it holds 2D + 2D^2 >= 2 values per particle)
  double* sE = d->stage;
  double* snu = d->stage + n;
  if (cudaMemcpyAsync(sE, pin->E, sizeof(double) * n, cudaMemcpyHostToDevice, d->stream) != cudaSuccess ||
      cudaMemcpyAsync(snu, pin->nu, sizeof(double) * n, cudaMemcpyHostToDevice, d->stream) != cudaSuccess ||
      cudaMemcpyAsync(d->A.vol0, pin->vol0, sizeof(double) * n, cudaMemcpyHostToDevice, d->stream) != cudaSuccess ||
      cudaMemcpyAsync(d->A.mass, pin->mass, sizeof(double) * n, cudaMemcpyHostToDevice, d->stream) != cudaSuccess ||
      cudaMemcpyAsync(d->A.flags, pin->flags, n, cudaMemcpyHostToDevice, d->stream) != cudaSuccess)
    return cleanup(fail(OSMPM_E_CUDA, "particle upload failed"));
  DISPATCH(d, K::lame(sE, snu, A_, d->stream));
  {
    std::vector<uint32_t> ids((size_t)n);
    for (int64_t p = 0; p < n; ++p) ids[(size_t)p] = (uint32_t)p;
    if (cudaMemcpyAsync(d->A.id, ids.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, d->stream) != cudaSuccess ||
        cudaStreamSynchronize(d->stream) != cudaSuccess)
      return cleanup(fail(OSMPM_E_CUDA, "id upload failed"));
  }
  C_TRY(sort_into_primary(d));
#undef C_TRY
  *out = d;
  return OSMPM_OK;
}

osmpm_status osmpm_destroy_domain(osmpm_domain* d) {
  if (!d) return OSMPM_OK;
  cudaStreamSynchronize(d->stream);
  free_all(d);
  cudaStreamSynchronize(d->stream);
  delete d;
  return OSMPM_OK;
}

osmpm_status osmpm_set_dirichlet(osmpm_domain* d, const osmpm_dirichlet* rules, int32_t n_rules) {
  OSMPM_TRY(check_domain(d));
  if (n_rules < 0 || n_rules > kMaxRules) return fail(OSMPM_E_INVALID, "n_rules must be in [0, %d]", kMaxRules);
  if (n_rules > 0 && !rules) return fail(OSMPM_E_INVALID, "null rules");
  for (int r = 0; r < n_rules; ++r) {
    if (rules[r].kind != 0 && rules[r].kind != 1) return fail(OSMPM_E_INVALID, "rule %d: unknown kind", r);
    if (rules[r].kind == 1 && d->dim == 3) {
      const double* k = rules[r].axis;
      if (!(k[0] * k[0] + k[1] * k[1] + k[2] * k[2] > 0.0)) return fail(OSMPM_E_INVALID, "rule %d: zero axis", r);
    }
  }
  d->rules.assign(rules, rules + n_rules);
  return OSMPM_OK;
}

osmpm_status osmpm_set_plane(osmpm_domain* d, const osmpm_plane* plane) {
  OSMPM_TRY(check_domain(d));
  if (!plane) return fail(OSMPM_E_INVALID, "null plane");
  if (!plane->enabled) {
    d->plane_on = false;
    return OSMPM_OK;
  }
  if (d->dim != 2) return fail(OSMPM_E_UNSUPPORTED, "the rigid plane is two-dimensional");
  if (!std::isfinite(plane->level) || !std::isfinite(plane->cand_hi) || !(plane->spacing > 0.0) ||
      !std::isfinite(plane->spacing) || plane->max_sets < 0)
    return fail(OSMPM_E_INVALID, "plane: finite level and cand_hi, spacing > 0, max_sets >= 0");
  const int64_t nn = d->geo.nn;
  if (!d->plane_gap) {
    OSMPM_TRY(dalloc_n(d, nn, &d->plane_gap));
    OSMPM_TRY(dalloc_n(d, nn, &d->plane_hold_v));
    OSMPM_TRY(dalloc_n(d, nn, &d->plane_lam));
    OSMPM_TRY(dalloc_n(d, (int64_t)d->geo.res[0], &d->plane_colmin));
    OSMPM_TRY(dalloc_n(d, nn, &d->plane_cand));
    OSMPM_TRY(dalloc_n(d, nn, &d->plane_act));
    OSMPM_TRY(dalloc_n(d, nn, &d->mask_all));
    OSMPM_TRY(dalloc_n(d, 1, &d->plane_changes));
    CUDA_TRY(cudaMemsetAsync(d->plane_lam, 0, sizeof(double) * nn, d->stream));
    CUDA_TRY(cudaMemsetAsync(d->plane_gap, 0, sizeof(double) * nn, d->stream));
    CUDA_TRY(cudaMemsetAsync(d->plane_act, 0, nn, d->stream));
    CUDA_TRY(cudaStreamSynchronize(d->stream));
  }
  d->plane = *plane;
  d->plane_on = true;
  return OSMPM_OK;
}

osmpm_status osmpm_step(osmpm_domain* d, double dt, osmpm_stats* stats) {
  NvtxRange nvtx_("osmpm_step");
  OSMPM_TRY(check_domain(d));
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(OSMPM_E_INVALID, "dt must be > 0");
  SolveStats st;
  osmpm_domain::TapeStep slot{};
  bool ck_new = false, ck_ctl = false;  // a checkpoint / step controls pushed by this call
  if (d->recording) {
    if (d->tape_kind != 0 && d->tape_kind != 1) d->tape_broken = true;
    d->tape_kind = 1;
    if (!d->tape_broken && (d->ckpt_every <= 1 || d->replaying)) {
      OSMPM_TRY(tape_begin(d, slot));
    } else if (!d->tape_broken) {
      // checkpointed record: the state at the start of every ckpt_every-th
      // step, and every step's controls
      if (d->ctl.size() % (size_t)d->ckpt_every == 0) {
        osmpm_domain::TapeStep c{};
        c.bytes = sizeof(double) * (2 * d->dim + 2 * d->dim * d->dim) * (size_t)d->n;
        OSMPM_TRY(raw_alloc(d, c.bytes, &c.mem));
        d->ckpts.push_back(c);
        ck_new = true;
        OSMPM_TRY(save_state(d, (char*)c.mem));
      }
      osmpm_domain::StepCtl c;
      c.dt = dt;
      c.rules = d->rules;
      d->ctl.push_back(std::move(c));
      ck_ctl = true;
    }
  }
  auto drop = [&](osmpm_status e) {
    raw_free(d, slot.mem, slot.bytes);
    if (ck_ctl) d->ctl.pop_back();
    if (ck_new) {
      raw_free(d, d->ckpts.back().mem, d->ckpts.back().bytes);
      d->ckpts.pop_back();
    }
    return e;
  };
#define T_TRY(expr)                       \
  do {                                    \
    osmpm_status t_ = (expr);             \
    if (t_ != OSMPM_OK) return drop(t_);  \
  } while (0)
  CUDA_TRY(cudaMemsetAsync(d->err, 0, sizeof(int), d->stream));
  T_TRY(run_p2g(d, false));
  T_TRY(sync_scalars(d));
  T_TRY(check_err(d));
  osmpm_status s = OSMPM_OK;
  if (d->plane_on) {
    s = contact_solve(d, dt, st);
  } else {
    T_TRY(prep(d, dt, true, nullptr, nullptr, nullptr, 0.0, nullptr));
    T_TRY(cold_start(d, dt));
    s = newton_solve(d, dt, st);
  }
  if (s != OSMPM_OK) {
    fill_stats(stats, st, 0, 0, 0.0, 0.0);
    return drop(s);
  }
  if (slot.mem) T_TRY(tape_end(d, slot, dt));
#undef T_TRY
  {
    NvtxRange nvtx_("g2p");
    DISPATCH(d, K::g2p(P_, d->geo, d->u, dt, d->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  CUDA_TRY(cudaGetLastError());
  fill_stats(stats, st, 0, 1, 0.0, 0.0);
  return OSMPM_OK;
}

osmpm_status osmpm_schwarz_couple(osmpm_domain* B, osmpm_domain* S, double dT,
                                  const osmpm_schwarz_desc* sd, osmpm_stats* stats) {
  OSMPM_TRY(check_domain(B));
  OSMPM_TRY(check_domain(S));
  if (!sd) return fail(OSMPM_E_INVALID, "null schwarz descriptor");
  if (B == S) return fail(OSMPM_E_INVALID, "coarse and fine must be different domains");
  if (B->dim != S->dim) return fail(OSMPM_E_INVALID, "domains differ in dim");
  if (B->stream != S->stream) return fail(OSMPM_E_INVALID, "domains must share one stream");
  if (B->prec != S->prec) return fail(OSMPM_E_INVALID, "domains differ in precision");
  if (B->plane_on || S->plane_on)
    return fail(OSMPM_E_UNSUPPORTED, "the rigid-plane contact serves osmpm_step only");
  if (!(B->geo.dx >= S->geo.dx)) return fail(OSMPM_E_INVALID, "coarse dx must be >= fine dx");
  if (sd->M < 1 || sd->k_max < 0 || !(sd->eps_conv > 0.0) || !(sd->eps_tol >= 0.0) ||
      std::isnan(sd->tau_B) || std::isnan(sd->tau_S) ||
      (sd->pi_source != OSMPM_PI_STEP_AVERAGE && sd->pi_source != OSMPM_PI_LAST_SUBSTEP))
    return fail(OSMPM_E_INVALID, "bad Schwarz controls");
  for (int i = 0; i < 7; ++i)
    if (sd->reserved[i] != 0) return fail(OSMPM_E_INVALID, "reserved fields must be zero");
  const bool pi_avg = sd->pi_source == OSMPM_PI_STEP_AVERAGE;
  if (!(dT > 0.0) || !std::isfinite(dT)) return fail(OSMPM_E_INVALID, "dT must be > 0");
  const int M = sd->M;
  const double dt = dT / M;
  const int D = B->dim;
  // reverse-mode record of this step, kept on the coarse domain (needs both
  // domains recording in FP64, the step-average projection and a record of
  // coupled steps of this pair only; anything else interrupts the record)
  const bool want_rec = B->recording || S->recording;
  const bool rec = want_rec && B->recording && S->recording && !B->tape_broken &&
                   !S->tape_broken && sd->pi_source == OSMPM_PI_STEP_AVERAGE && B->prec == 0 &&
                   S->prec == 0 && (B->tape_kind == 0 || (B->tape_kind == 2 && B->partner == S)) &&
                   (S->tape_kind == 0 || (S->tape_kind == 3 && S->partner == B));
  if (want_rec && !rec) {
    if (B->recording) B->tape_broken = true;
    if (S->recording) S->tape_broken = true;
  }
  // checkpointed record (the coarse domain's interval): controls of every
  // step, both start states at every ckpt_every-th; the full record while
  // osmpm_adjoint re-runs a segment
  const bool ck = rec && B->ckpt_every > 1 && !B->replaying;
  const bool rec_full = rec && !ck;
  osmpm_domain::CoupledStep cs{};
  const CoupledLayout CL(B, S, sd->M);
  bool ck_new = false, ck_ctl = false;
  auto drop_rec = [&]() {
    raw_free(B, cs.head.mem, cs.head.bytes);
    for (auto& t : cs.iters) raw_free(B, t.mem, t.bytes);
    cs.head.mem = nullptr;
    cs.iters.clear();
    if (ck_ctl) B->ctl.pop_back();
    if (ck_new) {
      raw_free(B, B->ckpts.back().mem, B->ckpts.back().bytes);
      B->ckpts.pop_back();
    }
    ck_ctl = ck_new = false;
    if (rec) {
      B->tape_broken = true;
      S->tape_broken = true;
    }
  };
  const GridGeo &gB = B->geo, &gS = S->geo;
  cudaStream_t s = B->stream;
  SolveStats st;
  auto bail = [&](osmpm_status e) {
    drop_rec();
    snapshot(S, true);  // the fine particles go back to t_n
    cudaStreamSynchronize(s);
    fill_stats(stats, st, 0, 0, 0.0, 0.0);
    return e;
  };
#define S_TRY(expr)                        \
  do {                                     \
    osmpm_status s_ = (expr);              \
    if (s_ != OSMPM_OK) return bail(s_);   \
  } while (0)

  // Step 0 (Eq. store_states, Alg. 1): snapshot, P2G on both grids with
  // boundary-particle mass, boundary sets and arbitration.
  CUDA_TRY(cudaMemsetAsync(B->err, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(S->err, 0, sizeof(int), s));
  OSMPM_TRY(snapshot(S, false));
  if (ck) {
    if (B->ctl.size() % (size_t)B->ckpt_every == 0) {
      const size_t sb = sizeof(double) * (2 * D + 2 * D * D) * (size_t)B->n;
      const size_t ss = sizeof(double) * (2 * D + 2 * D * D) * (size_t)S->n;
      osmpm_domain::TapeStep c{};
      c.bytes = sb + ss;
      S_TRY(raw_alloc(B, c.bytes, &c.mem));
      B->ckpts.push_back(c);
      ck_new = true;
      S_TRY(save_state(B, (char*)c.mem));
      S_TRY(save_state(S, (char*)c.mem + sb));
    }
    osmpm_domain::StepCtl c;
    c.dt = dT;
    c.sd = *sd;
    c.rules = B->rules;
    c.rules_fine = S->rules;
    B->ctl.push_back(std::move(c));
    ck_ctl = true;
  }
  S_TRY(run_p2g(B, true));
  S_TRY(run_p2g(S, true));
  S_TRY(sync_scalars(B));
  S_TRY(check_err(B));
  S_TRY(sync_scalars(S));
  S_TRY(check_err(S));
  // physical Dirichlet masks of both grids
  S_TRY(prep(B, dT, true, nullptr, nullptr, nullptr, 0.0, B->physmask));
  S_TRY(prep(S, dt, true, nullptr, nullptr, nullptr, 0.0, S->physmask));
  DISPATCH(B, K::gamma(gB, B->m, B->bm, sd->tau_B, B->gam, s));
  DISPATCH(S, K::gamma(gS, S->m, S->bm, sd->tau_S, S->gam, s));
  CUDA_TRY(cudaMemcpyAsync(B->recv, B->gam, gB.nn, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(S->recv, S->gam, gS.nn, cudaMemcpyDeviceToDevice, s));
  DISPATCH(B, K::arbitrate(gB, gS, B->gam, S->gam, B->m, S->m, B->recv, S->recv, s));
  CUDA_TRY(cudaMemsetAsync(B->proj_num, 0, sizeof(double) * D * gB.nn, s));
  CUDA_TRY(cudaMemsetAsync(B->proj_den, 0, sizeof(double) * gB.nn, s));
  DISPATCH(B, K::proj_scatter(gB, gS, S->m, S->vn, B->proj_num, B->proj_den, s));
  DISPATCH(B, K::recvB_filter(gB, B->proj_den, sd->tau_B, B->physmask, B->recv, s));
  DISPATCH(B, K::recvS_filter(gB, gS, B->m, S->physmask, S->recv, s));
  // v_GammaB^(0) = Pi(fine P2G at t_n); v_GammaS^n = I(v_B^n)
  DISPATCH(B, K::proj_finish(gB, B->recv, B->proj_num, B->proj_den, sd->eps_tol, B->bc0, s));
  DISPATCH(B, K::interp(gB, gS, B->vn, S->recv, S->bc0, s));
  CUDA_TRY(cudaMemcpyAsync(S->bc_prev, S->bc0, sizeof(double) * D * gS.nn, cudaMemcpyDeviceToDevice, s));
  if (rec_full) {
    S_TRY(raw_alloc(B, CL.head_bytes, &cs.head.mem));
    cs.head.bytes = CL.head_bytes;
    cs.M = M;
    cs.dT = dT;
    cs.eps_tol = sd->eps_tol;
    char* h = (char*)cs.head.mem;
    S_TRY(save_state(B, h + CL.stB));
    S_TRY(save_state(S, h + CL.stS));
    CUDA_TRY(cudaMemcpyAsync(h + CL.recvB, B->recv, gB.nn, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(h + CL.recvS, S->recv, gS.nn, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(h + CL.N0, B->proj_num, 8 * D * gB.nn, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(h + CL.D0, B->proj_den, 8 * gB.nn, cudaMemcpyDeviceToDevice, s));
  }

  // Newton warm starts for the re-solves of iterations k >= 1: the coarse
  // solve from its previous solution, fine sub-step m from the previous
  // iteration's sub-step m (same minimisers; the first solve is cold)
  S_TRY(ensure_keep(B, 1));
  S_TRY(ensure_keep(S, M));
  const size_t bytesB = sizeof(double) * D * gB.nn, bytesS = sizeof(double) * D * gS.nn;
  int k = 0, converged = 0;
  double rB = 0.0, rS = 0.0;
  for (k = 0; k <= sd->k_max; ++k) {
    NvtxRange nvtx_("schwarz_iteration");
    // 1. coarse solve over dT with Pi data on Gamma_hat_B (Eq. implicit_solve_coarse)
    S_TRY(prep(B, dT, true, B->recv, B->bc0, B->bc0, 1.0, nullptr));
    if (k > 0)
      DISPATCH(B, K::warm_start(gB, B->dofmask, keep_slot(B, 0), B->u, s));
    else
      S_TRY(cold_start(B, dT));
    S_TRY(newton_solve(B, dT, st));
    CUDA_TRY(cudaMemcpyAsync(keep_slot(B, 0), B->u, bytesB, cudaMemcpyDeviceToDevice, s));
    char* ib = nullptr;
    if (rec_full) {
      osmpm_domain::TapeStep it{};
      S_TRY(raw_alloc(B, CL.iter_bytes, &it.mem));
      it.bytes = CL.iter_bytes;
      cs.iters.push_back(it);
      ib = (char*)it.mem;
      CUDA_TRY(cudaMemcpyAsync(ib + CL.uB, B->u, bytesB, cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(ib + CL.maskB, B->dofmask, gB.nn, cudaMemcpyDeviceToDevice, s));
    }
    DISPATCH(B, K::vel_from_u(gB, B->m, B->u, dT, B->vtmp, s));
    // 2. fine: restore, P2G, endpoint data I(v_B^n), I(v_B^(k+1)), sub-cycle
    S_TRY(snapshot(S, true));
    S_TRY(run_p2g(S, false));
    DISPATCH(B, K::interp(gB, gS, B->vtmp, S->recv, S->bc1, s));
    // Step-average source: the projection sums collect every sub-step's
    // solved grid (its mass and u/dt)
    CUDA_TRY(cudaMemsetAsync(B->proj_num, 0, sizeof(double) * D * gB.nn, s));
    CUDA_TRY(cudaMemsetAsync(B->proj_den, 0, sizeof(double) * gB.nn, s));
    for (int m = 1; m <= M; ++m) {
      S_TRY(prep(S, dt, true, S->recv, S->bc0, S->bc1, (double)m / (double)M, nullptr));
      if (k > 0)
        DISPATCH(S, K::warm_start(gS, S->dofmask, keep_slot(S, m - 1), S->u, s));
      else
        S_TRY(cold_start(S, dt));
      if (ib && m > 1) S_TRY(save_state(S, ib + CL.state[m - 1]));
      S_TRY(newton_solve(S, dt, st));
      CUDA_TRY(cudaMemcpyAsync(keep_slot(S, m - 1), S->u, bytesS, cudaMemcpyDeviceToDevice, s));
      if (ib) {
        CUDA_TRY(cudaMemcpyAsync(ib + CL.uS[m - 1], S->u, bytesS, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(ib + CL.maskS[m - 1], S->dofmask, gS.nn, cudaMemcpyDeviceToDevice, s));
      }
      if (pi_avg) {
        DISPATCH(S, K::vel_from_u(gS, S->m, S->u, dt, S->vtmp, s));
        DISPATCH(B, K::proj_scatter(gB, gS, S->m, S->vtmp, B->proj_num, B->proj_den, s));
      }
      DISPATCH(S, K::g2p(P_, gS, S->u, dt, s));
      S_TRY(run_p2g(S, false));
      S_TRY(sync_scalars(S));
      S_TRY(check_err(S));
    }
    // 3. convergence: the new Pi vs the BC in use.  Step average: the sums
    // hold M times the time averages, so eps_tol is scaled by M to keep
    // Pi = avg num / (avg den + eps_tol).  Last sub-step: Pi of the P2G grid.
    if (!pi_avg)
      DISPATCH(B, K::proj_scatter(gB, gS, S->m, S->vn, B->proj_num, B->proj_den, s));
    if (ib) {
      CUDA_TRY(cudaMemcpyAsync(ib + CL.N, B->proj_num, 8 * D * gB.nn, cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(ib + CL.Dn, B->proj_den, 8 * gB.nn, cudaMemcpyDeviceToDevice, s));
    }
    DISPATCH(B, K::proj_finish(gB, B->recv, B->proj_num, B->proj_den,
                               pi_avg ? sd->eps_tol * M : sd->eps_tol, B->bc1, s));
    DISPATCH(B, K::rel_change(gB, B->bc1, B->bc0, B->recv, 0, B->S, B->partials, s));
    DISPATCH(S, K::rel_change(gS, S->bc1, S->bc_prev, S->recv, 1, B->S, B->partials, s));
    S_TRY(sync_scalars(B));
    {
      const double nB = sqrt(B->S_host->res_num[0]), dB = sqrt(B->S_host->res_den[0]);
      const double nS = sqrt(B->S_host->res_num[1]), dS = sqrt(B->S_host->res_den[1]);
      rB = dB < 1e-14 ? nB : nB / dB;
      rS = dS < 1e-14 ? nS : nS / dS;
    }
    std::swap(B->bc0, B->bc1);
    std::swap(S->bc_prev, S->bc1);
    if (k >= 1 && rB <= sd->eps_conv && rS <= sd->eps_conv) {
      converged = 1;
      break;
    }
  }
  const int iters = converged ? k + 1 : sd->k_max + 1;
  // 4. post-convergence coarse update (Sec. 3.5)
  DISPATCH(B, K::g2p(P_, gB, B->u, dT, s));
  if (rec) {
    if (rec_full) B->ctape.push_back(cs);
    B->tape_kind = 2;
    B->partner = S;
    S->tape_kind = 3;
    S->partner = B;
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  CUDA_TRY(cudaGetLastError());
#undef S_TRY
  fill_stats(stats, st, iters, converged, rB, rS);
  if (!converged)
    return fail(OSMPM_W_SCHWARZ_MAXITER, "Schwarz stopped at k_max = %d (r_B %g, r_S %g)", sd->k_max, rB, rS);
  return OSMPM_OK;
}

osmpm_status osmpm_set_profiling(osmpm_domain* d, int32_t enable) {
  OSMPM_TRY(check_domain(d));
  if (enable && d->ev.empty()) {
    d->ev.resize(2);
    for (auto& e : d->ev) CUDA_TRY(cudaEventCreate(&e));
    d->hev.resize((size_t)2 * kStreamChunk);
    for (auto& e : d->hev) CUDA_TRY(cudaEventCreate(&e));
  }
  d->time_hvp = enable != 0;
  d->hvp_ms = 0.0;
  d->hvp_launches = 0;
  d->pcg_ms = 0.0;
  d->pcg_launches = 0;
  d->pcg_iters = 0;
  return OSMPM_OK;
}

osmpm_status osmpm_get_counters(const osmpm_domain* d, osmpm_counters* out) {
  if (!out) return fail(OSMPM_E_INVALID, "null output");
  memset(out, 0, sizeof(*out));
  out->launches = (int64_t)g_launch_count.load();
  if (d) {
    out->pcg_launches = d->pcg_launches;
    out->pcg_ms = d->pcg_ms;
    out->pcg_iters = d->pcg_iters;
    out->particles = d->n;
    out->dofs = d->geo.nn * d->dim;
    out->graph_replays = d->graph_replays;
    out->graph_error = d->graph_error;
    out->hvp_ms = d->hvp_ms;
    out->hvp_launches = d->hvp_launches;
    for (const auto& gs : d->ngraph) out->graphs += gs.exec ? 1 : 0;
  }
  return OSMPM_OK;
}

osmpm_status osmpm_record(osmpm_domain* d, int32_t enable) {
  OSMPM_TRY(check_domain(d));
  if (enable < 0) return fail(OSMPM_E_INVALID, "enable must be >= 0");
  if (enable && d->prec != 0)
    return fail(OSMPM_E_UNSUPPORTED, "reverse mode needs a precision 0 (FP64) domain");
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  clear_tape(d);
  d->recording = enable != 0;
  d->ckpt_every = enable > 1 ? enable : 1;
  return OSMPM_OK;
}

#define ADJ(d, call)                     \
  do {                                   \
    if ((d)->dim == 2) {                 \
      using AK = AdjointKernels<2>;      \
      call;                              \
    } else {                             \
      using AK = AdjointKernels<3>;      \
      call;                              \
    }                                    \
  } while (0)

// Reverse of the recorded coupled steps (Alg. 1 differentiated through the
// iterations it ran).  Per step, last to first: the post-convergence coarse
// G2P; then for k = K .. 0 the fine sub-steps of iteration k in reverse
// (each a single-domain step adjoint, plus the adjoint of its receiver data
// through T_m and, for k < K, the share of the next coarse solve's
// projection adjoint), the transposed I_{B->S} into coarse solve k, that
// solve's adjoint, and its receiver data back through the transposed
// Pi_{S->B} (into fine iteration k-1, or for k = 0 into the fine P2G at
// t_n); finally v_S^n = I(v_B^n) and the coarse P2G at t_n.
static osmpm_status coupled_adjoint(osmpm_domain* B, osmpm_domain* S, const double* dJ_dx,
                                    const osmpm_adjoint_out* out, osmpm_stats* stats) {
  if (B->dim != S->dim || B->stream != S->stream)
    return fail(OSMPM_E_INVALID, "coarse and fine must share dim and stream");
  if (B->prec != 0 || S->prec != 0)
    return fail(OSMPM_E_UNSUPPORTED, "reverse mode needs precision 0 (FP64) domains");
  if (B->tape_broken || S->tape_broken)
    return fail(OSMPM_E_INVALID, "the record was interrupted");
  if ((B->ctape.empty() && B->ctl.empty()) || B->tape_kind != 2 || B->partner != S ||
      S->partner != B)
    return fail(OSMPM_E_INVALID, "no coupled steps of this pair recorded");
  const bool ck = !B->ctl.empty();  // checkpointed record: re-run each segment
  const int D = B->dim, DD = D * D;
  const int64_t nB = B->n, nS = S->n, nnB = B->geo.nn, nnS = S->geo.nn;
  const GridGeo &gB = B->geo, &gS = S->geo;
  cudaStream_t s = B->stream;
  for (osmpm_domain* d : {B, S}) {
    if (!d->adj)
      OSMPM_TRY(dalloc_n(d, (int64_t)(2 * (2 * D + 2 * DD) + 1) * d->n + (2 * D + 1) * d->geo.nn, &d->adj));
    if (!d->cadj) OSMPM_TRY(dalloc_n(d, (int64_t)(2 * D + 2 * DD) * d->n + (4 * D + 3) * d->geo.nn, &d->cadj));
  }
  struct Bufs {
    double *x, *v, *B, *F, *x2, *v2, *B2, *F2, *E, *ubar, *qbar, *mbar;
    double *ax, *av, *aB, *aF, *klam, *g1, *g2, *g3, *h1, *h2;
  };
  auto carve = [&](osmpm_domain* d) {
    Bufs b{};
    const int64_t n = d->n, nn = d->geo.nn;
    b.x = d->adj;
    b.v = b.x + D * n;
    b.B = b.v + D * n;
    b.F = b.B + DD * n;
    b.x2 = b.F + DD * n;
    b.v2 = b.x2 + D * n;
    b.B2 = b.v2 + D * n;
    b.F2 = b.B2 + DD * n;
    b.E = b.F2 + DD * n;
    b.ubar = b.E + n;
    b.qbar = b.ubar + D * nn;
    b.mbar = b.qbar + D * nn;
    b.ax = d->cadj;
    b.av = b.ax + D * n;
    b.aB = b.av + D * n;
    b.aF = b.aB + DD * n;
    b.klam = b.aF + DD * n;
    b.g1 = b.klam + D * nn;
    b.g2 = b.g1 + D * nn;
    b.g3 = b.g2 + D * nn;
    b.h1 = b.g3 + D * nn;
    b.h2 = b.h1 + nn;
    return b;
  };
  Bufs bb = carve(B), sb = carve(S);
  // coarse: g1 = v_GammaB bar, g2 = v_B bar, g3 = Pi's nbar, h1 = dbar
  // fine:   g1 = v_S^n bar, g2 = v_S^{n+1} bar, g3 = G, h1 = H, h2 = m_extra
  const size_t stateB = sizeof(double) * (2 * D + 2 * DD) * nB;
  const size_t stateS = sizeof(double) * (2 * D + 2 * DD) * nS;
  const size_t gvB = sizeof(double) * D * nnB, gvS = sizeof(double) * D * nnS;
  SolveStats st;
  CUDA_TRY(cudaMemsetAsync(B->err, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(S->err, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(bb.v, 0, sizeof(double) * (D + 2 * DD) * nB, s));
  CUDA_TRY(cudaMemsetAsync(sb.v, 0, sizeof(double) * (D + 2 * DD) * nS, s));
  CUDA_TRY(cudaMemsetAsync(bb.E, 0, sizeof(double) * nB, s));
  CUDA_TRY(cudaMemsetAsync(sb.E, 0, sizeof(double) * nS, s));
  ADJ(B, AK::from_ids(nB, D, B->P.id, dJ_dx, bb.x, s));
  ADJ(S, AK::from_ids(nS, D, S->P.id, dJ_dx + (int64_t)D * nB, sb.x, s));
  // the states after the last recorded step, kept aside (a re-run segment
  // moves the particles and uses the fine snapshot)
  void* keep = nullptr;
  OSMPM_TRY(raw_alloc(B, stateB + stateS, &keep));
  OSMPM_TRY(save_state(B, (char*)keep));
  OSMPM_TRY(save_state(S, (char*)keep + stateB));
  osmpm_status status = OSMPM_OK;
  // one solve's adjoint on domain d with u, dofmask in place and u_bar in
  // its ubar: lam in d->cx, particle terms into (xacc, Facc, E), K lam on
  // the fixed DOFs into klam
  auto solve_adj = [&](osmpm_domain* d, Bufs& b, double dt, double* xacc, double* Facc) {
    const int64_t nn = d->geo.nn;
    CUDA_TRY(cudaMemsetAsync(d->grad, 0, sizeof(double) * D * nn, s));
    CUDA_TRY(cudaMemsetAsync(d->diag, 0, sizeof(double) * D * nn, s));
    DISPATCH(d, K::grad(P_, d->geo, d->u, d->dofmask, d->grad, d->diag, L_, d->err, s));
    ADJ(d, AK::rhs(d->geo, d->m, d->dofmask, dt, d->desc.cg_rtol, d->desc.cg_max, b.ubar, d->diag,
                   d->cx, d->cr, d->cz, d->cp, d->S, d->partials, s));
    OSMPM_TRY(run_pcg(d, dt, false, st));
    st.solves++;
    CUDA_TRY(cudaMemsetAsync(b.klam, 0, sizeof(double) * D * nn, s));
    ADJ(d, AK::solve(d->n, d->P.x, (const double*)d->P.F, d->P.mu, d->P.lam, d->P.vol0, d->geo,
                     d->u, d->cx, d->dofmask, xacc, Facc, b.E, b.klam, d->err, s));
    return OSMPM_OK;
  };
  // the recorded steps of B->ctape, last to first
  auto reverse_record = [&]() -> osmpm_status {
  for (size_t step = B->ctape.size(); step-- > 0 && status == OSMPM_OK;) {
    const auto& cst = B->ctape[step];
    const int M = cst.M;
    const CoupledLayout CL(B, S, M);
    const char* h = (const char*)cst.head.mem;
    const int Kit = (int)cst.iters.size() - 1;
    const double dT = cst.dT, dt = dT / M;
    const uint8_t* recvB = (const uint8_t*)(h + CL.recvB);
    const uint8_t* recvS = (const uint8_t*)(h + CL.recvS);
    // accumulators of the start-state adjoints and of the coarse P2G at t_n
    CUDA_TRY(cudaMemsetAsync(bb.ax, 0, stateB, s));
    CUDA_TRY(cudaMemsetAsync(sb.ax, 0, stateS, s));
    CUDA_TRY(cudaMemsetAsync(bb.qbar, 0, sizeof(double) * (D + 1) * nnB, s));
    CUDA_TRY(cudaMemsetAsync(sb.g1, 0, gvS, s));
    // coarse state and grid at t_n (shared by every coarse solve)
    OSMPM_TRY(load_state(B, h + CL.stB));
    OSMPM_TRY(run_p2g(B, false));
    // post-convergence coarse G2P with u_B^(K)
    {
      const char* ik = (const char*)cst.iters[Kit].mem;
      CUDA_TRY(cudaMemcpyAsync(B->u, ik + CL.uB, gvB, cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaMemsetAsync(bb.ubar, 0, gvB, s));
      ADJ(B, AK::g2p(nB, B->P.x, (const double*)B->P.F, gB, B->u, dT, bb.x, bb.v, bb.B, bb.F, bb.ubar,
                     bb.x2, bb.F2, s));
      ADJ(B, AK::add(D * nB, bb.x2, bb.ax, s));
      ADJ(B, AK::add(DD * nB, bb.F2, bb.aF, s));
    }
    bool pending = false;  // G, H of the projection adjoint wait for fine iteration k
    for (int k = Kit; k >= 0 && status == OSMPM_OK; --k) {
      const char* ik = (const char*)cst.iters[k].mem;
      // ---- fine iteration k, sub-steps in reverse
      double *cx = sb.x, *cv = sb.v, *cB = sb.B, *cF = sb.F;
      double *nx = sb.x2, *nv = sb.v2, *nB_ = sb.B2, *nF = sb.F2;
      if (k < Kit) CUDA_TRY(cudaMemsetAsync(sb.x, 0, stateS, s));  // (x, v, B, F contiguous)
      CUDA_TRY(cudaMemsetAsync(sb.g2, 0, gvS, s));
      for (int m = M - 1; m >= 0; --m) {
        OSMPM_TRY(load_state(S, m == 0 ? h + CL.stS : ik + CL.state[m]));
        status = run_p2g(S, false);
        if (status != OSMPM_OK) break;
        CUDA_TRY(cudaMemcpyAsync(S->u, ik + CL.uS[m], gvS, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(S->dofmask, ik + CL.maskS[m], nnS, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemsetAsync(sb.ubar, 0, gvS, s));
        if (pending) ADJ(S, AK::inject(gS, S->m, S->u, dt, sb.g3, sb.h1, sb.ubar, sb.h2, s));
        ADJ(S, AK::g2p(nS, S->P.x, (const double*)S->P.F, gS, S->u, dt, cx, cv, cB, cF, sb.ubar, nx,
                       nF, s));
        status = solve_adj(S, sb, dt, nx, nF);
        if (status != OSMPM_OK) break;
        const double a = (double)(m + 1) / (double)M;
        ADJ(S, AK::bc(gS, recvS, S->m, sb.ubar, sb.klam, (1.0 - a) * dt, a * dt, sb.g1, sb.g2, s));
        CUDA_TRY(cudaMemsetAsync(sb.qbar, 0, sizeof(double) * (D + 1) * nnS, s));
        ADJ(S, AK::nodes(gS, S->m, S->vn, S->u, S->cx, S->desc.gravity, dt, pending ? sb.h2 : nullptr,
                         sb.qbar, sb.mbar, s));
        ADJ(S, AK::p2g(nS, S->P.x, (const double*)S->P.v, (const double*)S->P.B, S->P.mass, gS,
                       sb.qbar, sb.mbar, nv, nB_, nx, s));
        std::swap(cx, nx);
        std::swap(cv, nv);
        std::swap(cB, nB_);
        std::swap(cF, nF);
      }
      if (status != OSMPM_OK) break;
      // the snapshot fed this iteration
      ADJ(S, AK::add(D * nS, cx, sb.ax, s));
      ADJ(S, AK::add(D * nS, cv, sb.av, s));
      ADJ(S, AK::add(DD * nS, cB, sb.aB, s));
      ADJ(S, AK::add(DD * nS, cF, sb.aF, s));
      if (cx != sb.x) {  // keep the incoming-adjoint slots where the next pass expects them
        CUDA_TRY(cudaMemsetAsync(sb.x, 0, stateS, s));
      }
      // ---- v_S^{n+1} = I(v_B^(k+1)), v_B^(k+1) = u_B^(k) / dT (active coarse nodes)
      CUDA_TRY(cudaMemsetAsync(bb.g2, 0, gvB, s));
      ADJ(B, AK::interp_t(gB, gS, recvS, sb.g2, bb.g2, s));
      if (k < Kit) CUDA_TRY(cudaMemsetAsync(bb.ubar, 0, gvB, s));
      ADJ(B, AK::axpy_active(gB, B->m, 1.0 / dT, bb.g2, bb.ubar, s));
      // ---- coarse solve k
      CUDA_TRY(cudaMemcpyAsync(B->u, ik + CL.uB, gvB, cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(B->dofmask, ik + CL.maskB, nnB, cudaMemcpyDeviceToDevice, s));
      status = solve_adj(B, bb, dT, bb.ax, bb.aF);
      if (status != OSMPM_OK) break;
      ADJ(B, AK::nodes(gB, B->m, B->vn, B->u, B->cx, B->desc.gravity, dT, nullptr, bb.qbar, bb.mbar, s));
      CUDA_TRY(cudaMemsetAsync(bb.g1, 0, gvB, s));
      ADJ(B, AK::bc(gB, recvB, B->m, bb.ubar, bb.klam, dT, 0.0, bb.g1, nullptr, s));
      // ---- transposed Pi: of fine iteration k-1's step average, or of the fine P2G at t_n
      const double* num = k >= 1 ? (const double*)((const char*)cst.iters[k - 1].mem + CL.N)
                                 : (const double*)(h + CL.N0);
      const double* den = k >= 1 ? (const double*)((const char*)cst.iters[k - 1].mem + CL.Dn)
                                 : (const double*)(h + CL.D0);
      const double eps = k >= 1 ? cst.eps_tol * M : cst.eps_tol;
      ADJ(B, AK::proj_coarse(gB, recvB, num, den, eps, bb.g1, bb.g3, bb.h1, s));
      ADJ(B, AK::proj_fine(gB, gS, bb.g3, bb.h1, sb.g3, sb.h1, s));
      pending = k >= 1;
      if (k == 0) {
        OSMPM_TRY(load_state(S, h + CL.stS));
        status = run_p2g(S, false);
        if (status != OSMPM_OK) break;
        CUDA_TRY(cudaMemsetAsync(sb.qbar, 0, sizeof(double) * (D + 1) * nnS, s));
        ADJ(S, AK::grid_acc(gS, S->m, S->vn, sb.g3, sb.h1, nullptr, sb.qbar, sb.mbar, s));
        CUDA_TRY(cudaMemsetAsync(sb.x2, 0, sizeof(double) * D * nS, s));
        ADJ(S, AK::p2g(nS, S->P.x, (const double*)S->P.v, (const double*)S->P.B, S->P.mass, gS, sb.qbar,
                       sb.mbar, sb.v2, sb.B2, sb.x2, s));
        ADJ(S, AK::add(D * nS, sb.x2, sb.ax, s));
        ADJ(S, AK::add(D * nS, sb.v2, sb.av, s));
        ADJ(S, AK::add(DD * nS, sb.B2, sb.aB, s));
      }
    }
    if (status != OSMPM_OK) break;
    // ---- v_S^n = I(v_B^n), then the coarse P2G at t_n
    CUDA_TRY(cudaMemsetAsync(bb.g2, 0, gvB, s));
    ADJ(B, AK::interp_t(gB, gS, recvS, sb.g1, bb.g2, s));
    ADJ(B, AK::grid_acc(gB, B->m, B->vn, nullptr, nullptr, bb.g2, bb.qbar, bb.mbar, s));
    CUDA_TRY(cudaMemsetAsync(bb.x2, 0, sizeof(double) * D * nB, s));
    ADJ(B, AK::p2g(nB, B->P.x, (const double*)B->P.v, (const double*)B->P.B, B->P.mass, gB, bb.qbar,
                   bb.mbar, bb.v2, bb.B2, bb.x2, s));
    ADJ(B, AK::add(D * nB, bb.x2, bb.ax, s));
    ADJ(B, AK::add(D * nB, bb.v2, bb.av, s));
    ADJ(B, AK::add(DD * nB, bb.B2, bb.aB, s));
    // the start-state adjoints feed the earlier step
    CUDA_TRY(cudaMemcpyAsync(bb.x, bb.ax, stateB, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(sb.x, sb.ax, stateS, cudaMemcpyDeviceToDevice, s));
  }
  return status;
  };
  if (!ck) {
    status = reverse_record();
  } else {
    // segments last to first: from the segment's checkpoint, re-run its
    // steps with the full record (the recorded controls and rule sets), then
    // reverse them
    const std::vector<osmpm_dirichlet> rulesB = B->rules, rulesS = S->rules;
    B->replaying = S->replaying = true;
    const size_t every = (size_t)B->ckpt_every, nsteps = B->ctl.size();
    for (size_t seg = B->ckpts.size(); seg-- > 0 && status == OSMPM_OK;) {
      const char* c = (const char*)B->ckpts[seg].mem;
      status = load_state(B, c);
      if (status == OSMPM_OK) status = load_state(S, c + stateB);
      for (size_t j = seg * every; j < std::min(nsteps, (seg + 1) * every) && status == OSMPM_OK;
           ++j) {
        const auto& cj = B->ctl[j];
        B->rules = cj.rules;
        S->rules = cj.rules_fine;
        const osmpm_status f = osmpm_schwarz_couple(B, S, cj.dt, &cj.sd, nullptr);
        if (f != OSMPM_OK && f != OSMPM_W_SCHWARZ_MAXITER) status = f;
      }
      if (status == OSMPM_OK) status = reverse_record();
      clear_ctape(B);
    }
    B->replaying = S->replaying = false;
    B->rules = rulesB;
    S->rules = rulesS;
  }
  const osmpm_status rB = load_state(B, (const char*)keep);
  const osmpm_status rS = load_state(S, (const char*)keep + stateB);
  cudaStreamSynchronize(s);
  raw_free(B, keep, stateB + stateS);
  if (status != OSMPM_OK) return status;
  OSMPM_TRY(rB);
  OSMPM_TRY(rS);
  ADJ(B, AK::to_ids(nB, 1, B->P.id, bb.E, out->dJ_dE, s));
  ADJ(S, AK::to_ids(nS, 1, S->P.id, sb.E, out->dJ_dE + nB, s));
  struct O4 {
    double* dst;
    double *srcB, *srcS;
    int w;
  } o4[4] = {{out->dJ_dx0, bb.x, sb.x, D}, {out->dJ_dv0, bb.v, sb.v, D},
             {out->dJ_dB0, bb.B, sb.B, DD}, {out->dJ_dF0, bb.F, sb.F, DD}};
  for (auto& o : o4) {
    if (!o.dst) continue;
    ADJ(B, AK::to_ids(nB, o.w, B->P.id, o.srcB, o.dst, s));
    ADJ(S, AK::to_ids(nS, o.w, S->P.id, o.srcS, o.dst + (int64_t)o.w * nB, s));
  }
  OSMPM_TRY(sync_scalars(B));
  OSMPM_TRY(check_err(B));
  OSMPM_TRY(check_err(S));
  CUDA_TRY(cudaGetLastError());
  fill_stats(stats, st, 0, 1, 0.0, 0.0);
  return OSMPM_OK;
}

osmpm_status osmpm_adjoint(osmpm_domain* coarse, osmpm_domain* fine, const double* dJ_dx,
                           const osmpm_adjoint_out* out, osmpm_stats* stats) {
  NvtxRange nvtx_("osmpm_adjoint");
  OSMPM_TRY(check_domain(coarse));
  if (!dJ_dx || !out || !out->dJ_dE) return fail(OSMPM_E_INVALID, "null dJ_dx or dJ_dE");
  if (fine) return coupled_adjoint(coarse, fine, dJ_dx, out, stats);
  osmpm_domain* d = coarse;
  if (d->tape_kind > 1) return fail(OSMPM_E_INVALID, "the record holds coupled steps: pass both domains");
  if (!dJ_dx || !out || !out->dJ_dE) return fail(OSMPM_E_INVALID, "null dJ_dx or dJ_dE");
  if (d->prec != 0) return fail(OSMPM_E_UNSUPPORTED, "reverse mode needs a precision 0 (FP64) domain");
  if (d->tape_broken)
    return fail(OSMPM_E_INVALID, "the tape was interrupted (a coupled step or set_particles while recording)");
  if (d->tape.empty() && d->ctl.empty())
    return fail(OSMPM_E_INVALID, "nothing recorded (osmpm_record, then osmpm_step)");
  const bool ck = !d->ctl.empty();  // checkpointed record: re-run each segment
  const int D = d->dim, DD = D * D;
  const int64_t n = d->n, nn = d->geo.nn;
  cudaStream_t s = d->stream;
  if (!d->adj) OSMPM_TRY(dalloc_n(d, (int64_t)(2 * (2 * D + 2 * DD) + 1) * n + (2 * D + 1) * nn, &d->adj));
  double* xb = d->adj;
  double* vb = xb + D * n;
  double* Bb = vb + D * n;
  double* Fb = Bb + DD * n;
  double* xb2 = Fb + DD * n;
  double* vb2 = xb2 + D * n;
  double* Bb2 = vb2 + D * n;
  double* Fb2 = Bb2 + DD * n;
  double* Eb = Fb2 + DD * n;
  double* ubar = Eb + n;
  double* qbar = ubar + D * nn;
  double* mbar = qbar + D * nn;
  SolveStats st;
  CUDA_TRY(cudaMemsetAsync(d->err, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(vb, 0, sizeof(double) * (D + 2 * DD) * n, s));
  CUDA_TRY(cudaMemsetAsync(Eb, 0, sizeof(double) * n, s));
  ADJ(d, AK::from_ids(n, D, d->P.id, dJ_dx, xb, s));
  // the state after the last recorded step comes back at the end
  const size_t state_bytes = sizeof(double) * (2 * D + 2 * DD) * (size_t)n;
  void* keep = nullptr;
  OSMPM_TRY(raw_alloc(d, state_bytes, &keep));
  OSMPM_TRY(save_state(d, (char*)keep));
  const TapeLayout TL(d);
  osmpm_status status = OSMPM_OK;
  // the recorded steps of d->tape, last to first
  auto reverse_tape = [&]() -> osmpm_status {
  for (size_t k = d->tape.size(); k-- > 0 && status == OSMPM_OK;) {
    const auto& t = d->tape[k];
    const char* b = (const char*)t.mem;
    const double dt = t.dt;
    CUDA_TRY(cudaMemcpyAsync(d->P.x, b + TL.x, 8 * D * n, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d->P.v, b + TL.v, 8 * D * n, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d->P.B, b + TL.B, 8 * DD * n, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d->P.F, b + TL.F, 8 * DD * n, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d->u, b + TL.u, 8 * D * nn, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d->dofmask, b + TL.mask, nn, cudaMemcpyDeviceToDevice, s));
    // the step's grid (m, v^n) and stencil cache
    status = run_p2g(d, false);
    if (status != OSMPM_OK) break;
    // 1. transposed G2P, F update and advection
    CUDA_TRY(cudaMemsetAsync(ubar, 0, sizeof(double) * D * nn, s));
    ADJ(d, AK::g2p(n, d->P.x, (const double*)d->P.F, d->geo, d->u, dt, xb, vb, Bb, Fb, ubar, xb2, Fb2, s));
    // 2. K lam = u_bar with the Hessian at the converged u (implicit function theorem)
    CUDA_TRY(cudaMemsetAsync(d->grad, 0, sizeof(double) * D * nn, s));
    CUDA_TRY(cudaMemsetAsync(d->diag, 0, sizeof(double) * D * nn, s));
    DISPATCH(d, K::grad(P_, d->geo, d->u, d->dofmask, d->grad, d->diag, L_, d->err, s));
    ADJ(d, AK::rhs(d->geo, d->m, d->dofmask, dt, d->desc.cg_rtol, d->desc.cg_max, ubar, d->diag,
                   d->cx, d->cr, d->cz, d->cp, d->S, d->partials, s));
    status = run_pcg(d, dt, false, st);
    if (status != OSMPM_OK) break;
    st.solves++;
    // 3. -lam . dg/dz for the particle and node inputs of the solve
    ADJ(d, AK::solve(n, d->P.x, (const double*)d->P.F, d->P.mu, d->P.lam, d->P.vol0, d->geo, d->u,
                     d->cx, d->dofmask, xb2, Fb2, Eb, nullptr, d->err, s));
    CUDA_TRY(cudaMemsetAsync(qbar, 0, sizeof(double) * (D + 1) * nn, s));
    ADJ(d, AK::nodes(d->geo, d->m, d->vn, d->u, d->cx, d->desc.gravity, dt, nullptr, qbar, mbar, s));
    // 4. transposed P2G
    ADJ(d, AK::p2g(n, d->P.x, (const double*)d->P.v, (const double*)d->P.B, d->P.mass, d->geo, qbar,
                   mbar, vb2, Bb2, xb2, s));
    std::swap(xb, xb2);
    std::swap(vb, vb2);
    std::swap(Bb, Bb2);
    std::swap(Fb, Fb2);
  }
  return status;
  };
  if (!ck) {
    status = reverse_tape();
  } else {
    // segments last to first: re-run each from its checkpoint with the full
    // record (the recorded step sizes and rule sets), then reverse it
    const std::vector<osmpm_dirichlet> rules0 = d->rules;
    d->replaying = true;
    const size_t every = (size_t)d->ckpt_every, nsteps = d->ctl.size();
    for (size_t seg = d->ckpts.size(); seg-- > 0 && status == OSMPM_OK;) {
      status = load_state(d, (const char*)d->ckpts[seg].mem);
      for (size_t j = seg * every; j < std::min(nsteps, (seg + 1) * every) && status == OSMPM_OK;
           ++j) {
        d->rules = d->ctl[j].rules;
        status = osmpm_step(d, d->ctl[j].dt, nullptr);
      }
      if (status == OSMPM_OK) status = reverse_tape();
      for (auto& t : d->tape) raw_free(d, t.mem, t.bytes);
      d->tape.clear();
    }
    d->replaying = false;
    d->rules = rules0;
  }
  const osmpm_status restored = load_state(d, (const char*)keep);
  cudaStreamSynchronize(s);
  raw_free(d, keep, state_bytes);
  if (status != OSMPM_OK) return status;
  OSMPM_TRY(restored);
  ADJ(d, AK::to_ids(n, 1, d->P.id, Eb, out->dJ_dE, s));
  if (out->dJ_dx0) ADJ(d, AK::to_ids(n, D, d->P.id, xb, out->dJ_dx0, s));
  if (out->dJ_dv0) ADJ(d, AK::to_ids(n, D, d->P.id, vb, out->dJ_dv0, s));
  if (out->dJ_dB0) ADJ(d, AK::to_ids(n, DD, d->P.id, Bb, out->dJ_dB0, s));
  if (out->dJ_dF0) ADJ(d, AK::to_ids(n, DD, d->P.id, Fb, out->dJ_dF0, s));
  OSMPM_TRY(sync_scalars(d));
  OSMPM_TRY(check_err(d));
  CUDA_TRY(cudaGetLastError());
  fill_stats(stats, st, 0, 1, 0.0, 0.0);
  return OSMPM_OK;
}
#undef ADJ

osmpm_status osmpm_check_wait_timeout(void* cuda_stream) {
  cudaStream_t s = (cudaStream_t)cuda_stream;
  void* mem = nullptr;
  CUDA_TRY(cudaMallocAsync(&mem, 64, s));
  CUDA_TRY(cudaMemsetAsync(mem, 0, 64, s));
  unsigned* words = (unsigned*)mem;
  int* err = (int*)((char*)mem + 32);
  Kernels<2, double>::barrier_timeout_check(words, err, s);
  int host_err = 0;
  cudaError_t e = cudaMemcpyAsync(&host_err, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(mem, s);
  cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(OSMPM_E_CUDA, "timeout check: %s", cudaGetErrorString(e));
  if (host_err & kErrBarrierTimeout)
    return fail(OSMPM_E_TIMEOUT, "the device-side wait gave up as designed");
  return fail(OSMPM_E_CUDA, "the device-side wait did not report its timeout");
}

osmpm_status osmpm_schwarz_couple_batch(osmpm_domain* const* coarse, osmpm_domain* const* fine,
                                        int32_t n, double dT, const osmpm_schwarz_desc* sdesc,
                                        int32_t n_threads, osmpm_stats* stats,
                                        osmpm_status* status) {
  if (n < 0 || !coarse || !fine || !sdesc) return fail(OSMPM_E_INVALID, "null argument or n < 0");
  if (n == 0) return OSMPM_OK;
  for (int32_t i = 0; i < n; ++i) {
    if (!coarse[i] || !fine[i]) return fail(OSMPM_E_INVALID, "pair %d: null domain", i);
    for (int32_t j = 0; j < i; ++j)
      if (coarse[i] == coarse[j] || fine[i] == fine[j] || coarse[i] == fine[j] || fine[i] == coarse[j])
        return fail(OSMPM_E_INVALID, "pairs %d and %d share a domain", j, i);
  }
  int threads = n_threads > 0 ? n_threads : 8;
  if (threads > n) threads = n;
  std::vector<osmpm_status> st((size_t)n, OSMPM_OK);
  std::vector<std::string> msg((size_t)n);
  for (int32_t i = 0; i < n; ++i) coarse[i]->pcg_share = fine[i]->pcg_share = threads;
  // the worker threads launch directly: no graph capture from concurrent
  // host threads (a capture records whatever reaches its stream, and pairs
  // may share a stream)
  for (int32_t i = 0; i < n; ++i) coarse[i]->graph_hold = fine[i]->graph_hold = true;
  std::atomic<int32_t> next{0};
  int dev = 0;
  cudaGetDevice(&dev);
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int32_t i = next.fetch_add(1);
      if (i >= n) break;
      osmpm_stats s;
      st[(size_t)i] = osmpm_schwarz_couple(coarse[i], fine[i], dT, &sdesc[i], &s);
      if (st[(size_t)i] == OSMPM_E_TIMEOUT) {
        // a grid barrier of the pair's cooperative PCG gave up waiting (its
        // blocks could not all become resident beside the other pairs'
        // work); a failed coupled step leaves the pair at t_n (the fine
        // particles restored, the coarse ones not yet committed), so it is
        // run again once on half the grid
        coarse[i]->pcg_share = fine[i]->pcg_share = 2 * threads;
        st[(size_t)i] = osmpm_schwarz_couple(coarse[i], fine[i], dT, &sdesc[i], &s);
        coarse[i]->pcg_share = fine[i]->pcg_share = threads;
      }
      if (stats) stats[i] = s;
      if (st[(size_t)i] != OSMPM_OK) msg[(size_t)i] = g_last_error;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  for (int32_t i = 0; i < n; ++i) {
    coarse[i]->pcg_share = fine[i]->pcg_share = 1;
    coarse[i]->graph_hold = fine[i]->graph_hold = false;
  }
  osmpm_status worst = OSMPM_OK;
  int32_t first_bad = -1;
  for (int32_t i = 0; i < n; ++i) {
    if (status) status[i] = st[(size_t)i];
    if (st[(size_t)i] != OSMPM_OK && st[(size_t)i] != OSMPM_W_SCHWARZ_MAXITER && first_bad < 0) {
      first_bad = i;
      worst = st[(size_t)i];
    }
    if (worst == OSMPM_OK && st[(size_t)i] == OSMPM_W_SCHWARZ_MAXITER) worst = OSMPM_W_SCHWARZ_MAXITER;
  }
  if (first_bad >= 0) return fail(worst, "pair %d: %s", first_bad, msg[(size_t)first_bad].c_str());
  if (worst != OSMPM_OK) return fail(worst, "at least one pair hit k_max");
  return OSMPM_OK;
}

osmpm_status osmpm_schwarz_couple_multi(osmpm_domain* const* coarse, osmpm_domain* const* fine,
                                        int32_t n, double dT, const osmpm_schwarz_desc* sdesc,
                                        const osmpm_multi_desc* desc, osmpm_stats* stats,
                                        osmpm_status* status, osmpm_multi_stats* ms) {
  if (n < 0 || !coarse || !fine || !sdesc || !desc)
    return fail(OSMPM_E_INVALID, "null argument or n < 0");
  if (desc->n_threads < 0 || desc->dof_tile < 0 || desc->chunk < 0 || desc->slot_tiles < 0)
    return fail(OSMPM_E_INVALID, "multi descriptor: counts >= 0");
  if (ms) memset(ms, 0, sizeof(*ms));
  if (n == 0) return OSMPM_OK;
  for (int32_t i = 0; i < n; ++i) {
    if (!coarse[i] || !fine[i]) return fail(OSMPM_E_INVALID, "pair %d: null domain", i);
    if (coarse[i]->prec != 1 || fine[i]->prec != 1)
      return fail(OSMPM_E_UNSUPPORTED, "pair %d: the batched PCG serves mixed-precision domains", i);
    if (coarse[i]->dim != coarse[0]->dim || fine[i]->dim != coarse[0]->dim)
      return fail(OSMPM_E_UNSUPPORTED, "pair %d: every domain must have the same dimension", i);
    for (int32_t j = 0; j < i; ++j)
      if (coarse[i] == coarse[j] || fine[i] == fine[j] || coarse[i] == fine[j] || fine[i] == coarse[j])
        return fail(OSMPM_E_INVALID, "pairs %d and %d share a domain", j, i);
  }
  PcgBatcher b;
  OSMPM_TRY(b.open(coarse[0]->dim, desc->dof_tile, desc->chunk, desc->slot_tiles));
  int threads = desc->n_threads > 0 ? desc->n_threads : 32;
  if (threads > n) threads = n;
  std::vector<osmpm_status> st((size_t)n, OSMPM_OK);
  std::vector<std::string> msg((size_t)n);
  for (int32_t i = 0; i < n; ++i) {
    coarse[i]->batcher = fine[i]->batcher = &b;
    coarse[i]->graph_hold = fine[i]->graph_hold = true;
  }
  std::atomic<int32_t> next{0};
  int dev = 0;
  cudaGetDevice(&dev);
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int32_t i = next.fetch_add(1);
      if (i >= n) break;
      osmpm_stats s1;
      st[(size_t)i] = osmpm_schwarz_couple(coarse[i], fine[i], dT, &sdesc[i], &s1);
      if (stats) stats[i] = s1;
      if (st[(size_t)i] != OSMPM_OK) msg[(size_t)i] = g_last_error;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  for (int32_t i = 0; i < n; ++i) {
    coarse[i]->batcher = fine[i]->batcher = nullptr;
    coarse[i]->graph_hold = fine[i]->graph_hold = false;
  }
  if (ms) *ms = b.stats;
  b.close();
  osmpm_status worst = OSMPM_OK;
  int32_t first_bad = -1;
  for (int32_t i = 0; i < n; ++i) {
    if (status) status[i] = st[(size_t)i];
    if (st[(size_t)i] != OSMPM_OK && st[(size_t)i] != OSMPM_W_SCHWARZ_MAXITER && first_bad < 0) {
      first_bad = i;
      worst = st[(size_t)i];
    }
    if (worst == OSMPM_OK && st[(size_t)i] == OSMPM_W_SCHWARZ_MAXITER) worst = OSMPM_W_SCHWARZ_MAXITER;
  }
  if (first_bad >= 0) return fail(worst, "pair %d: %s", first_bad, msg[(size_t)first_bad].c_str());
  if (worst != OSMPM_OK) return fail(worst, "at least one pair hit k_max");
  return OSMPM_OK;
}

osmpm_status osmpm_autotune_multi(osmpm_domain* const* coarse, osmpm_domain* const* fine, int32_t n,
                                  double dT, const osmpm_schwarz_desc* sdesc,
                                  const osmpm_multi_desc* candidates, int32_t n_candidates,
                                  int32_t* best, double* us_per_cg_iter) {
  if (!candidates || n_candidates < 1 || !best || n < 1)
    return fail(OSMPM_E_INVALID, "need n >= 1 pairs, candidates and best");
  std::vector<osmpm_stats> stats((size_t)n);
  auto step = [&](const osmpm_multi_desc& md, double* seconds, int64_t* cg) -> osmpm_status {
    CUDA_TRY(cudaDeviceSynchronize());
    const auto t0 = std::chrono::steady_clock::now();
    const osmpm_status st = osmpm_schwarz_couple_multi(coarse, fine, n, dT, sdesc, &md, stats.data(),
                                                       nullptr, nullptr);
    CUDA_TRY(cudaDeviceSynchronize());
    if (st != OSMPM_OK && st != OSMPM_W_SCHWARZ_MAXITER) return st;
    *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *cg = 0;
    for (const auto& x : stats) *cg += x.cg_iters;
    return OSMPM_OK;
  };
  double sec = 0.0;
  int64_t cg = 0;
  OSMPM_TRY(step(candidates[0], &sec, &cg));  // warm-up: first-use allocations
  double best_score = INFINITY;
  *best = 0;
  for (int32_t c = 0; c < n_candidates; ++c) {
    OSMPM_TRY(step(candidates[c], &sec, &cg));
    const double score = 1e6 * sec / (double)std::max<int64_t>(cg, 1);
    if (us_per_cg_iter) us_per_cg_iter[c] = score;
    if (score < best_score) {
      best_score = score;
      *best = c;
    }
  }
  return OSMPM_OK;
}

osmpm_status osmpm_create_stream(void** out) {
  if (!out) return fail(OSMPM_E_INVALID, "null out");
  cudaStream_t s = nullptr;
  CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  *out = (void*)s;
  return OSMPM_OK;
}

osmpm_status osmpm_destroy_stream(void* stream) {
  if (!stream) return OSMPM_OK;
  CUDA_TRY(cudaStreamDestroy((cudaStream_t)stream));
  return OSMPM_OK;
}

osmpm_status osmpm_autotune_batch(osmpm_domain* const* coarse, osmpm_domain* const* fine, int32_t n,
                                  double dT, const osmpm_schwarz_desc* sdesc,
                                  const int32_t* candidates, int32_t n_candidates, int32_t* best,
                                  double* us_per_cg_iter) {
  if (!candidates || n_candidates < 1 || !best || n < 1)
    return fail(OSMPM_E_INVALID, "need n >= 1 pairs, candidates and best");
  for (int32_t c = 0; c < n_candidates; ++c)
    if (candidates[c] < 1) return fail(OSMPM_E_INVALID, "candidate %d is < 1", c);
  std::vector<osmpm_stats> stats((size_t)n);
  auto step = [&](int32_t threads, double* seconds, int64_t* cg) -> osmpm_status {
    CUDA_TRY(cudaDeviceSynchronize());
    const auto t0 = std::chrono::steady_clock::now();
    const osmpm_status st = osmpm_schwarz_couple_batch(coarse, fine, n, dT, sdesc, threads,
                                                       stats.data(), nullptr);
    CUDA_TRY(cudaDeviceSynchronize());
    if (st != OSMPM_OK && st != OSMPM_W_SCHWARZ_MAXITER) return st;
    *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *cg = 0;
    for (const auto& x : stats) *cg += x.cg_iters;
    return OSMPM_OK;
  };
  double sec = 0.0;
  int64_t cg = 0;
  OSMPM_TRY(step(candidates[0], &sec, &cg));  // warm-up: first-use allocations and graph captures
  double best_score = INFINITY;
  *best = candidates[0];
  for (int32_t c = 0; c < n_candidates; ++c) {
    OSMPM_TRY(step(candidates[c], &sec, &cg));
    const double score = 1e6 * sec / (double)std::max<int64_t>(cg, 1);
    if (us_per_cg_iter) us_per_cg_iter[c] = score;
    if (score < best_score) {
      best_score = score;
      *best = candidates[c];
    }
  }
  return OSMPM_OK;
}

osmpm_status osmpm_get_info(const osmpm_domain* d, int64_t* n, int32_t* dim) {
  OSMPM_TRY(check_domain(d));
  if (n) *n = d->n;
  if (dim) *dim = d->dim;
  return OSMPM_OK;
}

osmpm_status osmpm_get_particles(const osmpm_domain* dc, double* x, double* v, double* B, double* F) {
  osmpm_domain* d = const_cast<osmpm_domain*>(dc);
  OSMPM_TRY(check_domain(d));
  const int D = d->dim;
  const int64_t n = d->n;
  double* sx = d->stage;
  double* sv = sx + D * n;
  double* sB = sv + D * n;
  double* sF = sB + D * D * n;
  DISPATCH(d, K::pack_out(P_, sx, sv, sB, sF, d->stream));
  if (x) CUDA_TRY(cudaMemcpyAsync(x, sx, sizeof(double) * D * n, cudaMemcpyDeviceToHost, d->stream));
  if (v) CUDA_TRY(cudaMemcpyAsync(v, sv, sizeof(double) * D * n, cudaMemcpyDeviceToHost, d->stream));
  if (B) CUDA_TRY(cudaMemcpyAsync(B, sB, sizeof(double) * D * D * n, cudaMemcpyDeviceToHost, d->stream));
  if (F) CUDA_TRY(cudaMemcpyAsync(F, sF, sizeof(double) * D * D * n, cudaMemcpyDeviceToHost, d->stream));
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  return OSMPM_OK;
}

osmpm_status osmpm_set_particles(osmpm_domain* d, const double* x, const double* v, const double* B,
                                 const double* F) {
  OSMPM_TRY(check_domain(d));
  if (!x || !v || !B || !F) return fail(OSMPM_E_INVALID, "null array");
  const int D = d->dim;
  const int64_t n = d->n;
  if (!finite_all(x, D * n) || !finite_all(v, D * n) || !finite_all(B, D * D * n) || !finite_all(F, D * D * n))
    return fail(OSMPM_E_NONFINITE, "non-finite particle input");
  if (d->recording) d->tape_broken = true;  // the recorded steps no longer lead here
  // materials and ids back to id order in A, then the new kinematic state
  DISPATCH(d, K::scatter_by_id(P_, A_, d->stream));
  OSMPM_TRY(upload_state(d, x, v, B, F));
  CUDA_TRY(cudaMemsetAsync(d->err, 0, sizeof(int), d->stream));
  return sort_into_primary(d);
}

osmpm_status osmpm_get_order(const osmpm_domain* d, uint32_t* ids) {
  OSMPM_TRY(check_domain(d));
  if (!ids) return fail(OSMPM_E_INVALID, "null ids");
  CUDA_TRY(cudaMemcpyAsync(ids, d->P.id, sizeof(uint32_t) * d->n, cudaMemcpyDeviceToHost, d->stream));
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  return OSMPM_OK;
}

osmpm_status osmpm_get_grid(const osmpm_domain* dc, int32_t field, double* out) {
  osmpm_domain* d = const_cast<osmpm_domain*>(dc);
  OSMPM_TRY(check_domain(d));
  if (!out) return fail(OSMPM_E_INVALID, "null output");
  const int D = d->dim;
  const int64_t nn = d->geo.nn;
  switch (field) {
    case OSMPM_FIELD_MASS:
      return download_grid_vec(d, d->m, out, 1);
    case OSMPM_FIELD_BMASS:
      return download_grid_vec(d, d->bm, out, 1);
    case OSMPM_FIELD_VN:
      return download_grid_vec(d, d->vn, out, D);
    case OSMPM_FIELD_U:
      return download_grid_vec(d, d->u, out, D);
    case OSMPM_FIELD_BC:
      return download_grid_vec(d, d->bc_applied, out, D);
    case OSMPM_FIELD_PLANE_FORCE:
    case OSMPM_FIELD_PLANE_GAP:
    case OSMPM_FIELD_PLANE_ACTIVE: {
      if (!d->plane_gap) return fail(OSMPM_E_INVALID, "no rigid plane was set on this domain");
      if (field == OSMPM_FIELD_PLANE_FORCE) return download_grid_vec(d, d->plane_lam, out, 1);
      if (field == OSMPM_FIELD_PLANE_GAP) return download_grid_vec(d, d->plane_gap, out, 1);
      std::vector<uint8_t> tmp((size_t)nn);
      CUDA_TRY(cudaMemcpyAsync(tmp.data(), d->plane_act, nn, cudaMemcpyDeviceToHost, d->stream));
      CUDA_TRY(cudaStreamSynchronize(d->stream));
      for (int64_t i = 0; i < nn; ++i) out[i] = tmp[(size_t)i] ? 1.0 : 0.0;
      return OSMPM_OK;
    }
    case OSMPM_FIELD_RECEIVER: {
      std::vector<uint8_t> tmp((size_t)nn);
      CUDA_TRY(cudaMemcpyAsync(tmp.data(), d->recv, nn, cudaMemcpyDeviceToHost, d->stream));
      CUDA_TRY(cudaStreamSynchronize(d->stream));
      for (int64_t i = 0; i < nn; ++i) out[i] = tmp[(size_t)i] ? 1.0 : 0.0;
      return OSMPM_OK;
    }
    default:
      return fail(OSMPM_E_INVALID, "unknown grid field %d", field);
  }
}

osmpm_status osmpm_probe_gradient(osmpm_domain* d, double dt, const double* u, double* grad) {
  OSMPM_TRY(check_domain(d));
  if (!u || !grad) return fail(OSMPM_E_INVALID, "null array");
  OSMPM_TRY(probe_setup(d, dt, u));
  const int64_t nn = d->geo.nn;
  const int D = d->dim;
  CUDA_TRY(cudaMemsetAsync(d->grad, 0, sizeof(double) * D * nn, d->stream));
  CUDA_TRY(cudaMemsetAsync(d->diag, 0, sizeof(double) * D * nn, d->stream));
  DISPATCH(d, K::grad(P_, d->geo, d->u, d->dofmask, d->grad, d->diag, L_, d->err, d->stream));
  DISPATCH(d, K::grad_finish(d->geo, d->m, d->vn, d->u, d->dofmask, d->desc.gravity, dt,
                             d->desc.cg_rtol, d->desc.cg_rtol, 1, d->desc.cg_max, d->grad,
                             d->diag, d->cx, d->cr, d->cz, d->cp, d->S, d->partials, d->stream));
  OSMPM_TRY(sync_scalars(d));
  OSMPM_TRY(check_err(d));
  return download_grid_vec(d, d->grad, grad, D);
}

osmpm_status osmpm_probe_hvp(osmpm_domain* d, double dt, const double* u, const double* dv, double* hd) {
  OSMPM_TRY(check_domain(d));
  if (!u || !dv || !hd) return fail(OSMPM_E_INVALID, "null array");
  OSMPM_TRY(probe_setup(d, dt, u));
  const int64_t nn = d->geo.nn;
  const int D = d->dim;
  CUDA_TRY(cudaMemsetAsync(d->grad, 0, sizeof(double) * D * nn, d->stream));
  CUDA_TRY(cudaMemsetAsync(d->diag, 0, sizeof(double) * D * nn, d->stream));
  DISPATCH(d, K::grad(P_, d->geo, d->u, d->dofmask, d->grad, d->diag, L_, d->err, d->stream));
  OSMPM_TRY(upload_grid_vec(d, dv, d->cp));
  DISPATCH(d, K::set_cg_state(d->S, 0, 0, d->stream));
  if (d->desc.pcg_mode == 2) {
    // the streaming PCG's own product (lane groups, or block tiles in mixed
    // precision): the mass part, then the particle part added to it
    DISPATCH(d, K::cg_a(d->geo, d->m, d->dofmask, dt, d->cp, d->cp, d->cq, d->S, d->partials,
                        d->stream));
    DISPATCH(d, K::cgs_hvp(pcg_args<R>(d, dt), d->desc.hvp_mode, d->stream));
  } else {
    DISPATCH(d, K::hvp_only(P_, d->geo, d->m, d->dofmask, L_, dt, d->cp, d->cq, d->S,
                            d->partials, d->stream));
  }
  OSMPM_TRY(sync_scalars(d));
  OSMPM_TRY(check_err(d));
  return download_grid_vec(d, d->cq, hd, D);
}

osmpm_status osmpm_probe_energy_change(osmpm_domain* d, double dt, const double* u, const double* dv,
                                       double alpha, double* dE) {
  OSMPM_TRY(check_domain(d));
  if (!u || !dv || !dE) return fail(OSMPM_E_INVALID, "null array");
  OSMPM_TRY(probe_setup(d, dt, u));
  OSMPM_TRY(upload_grid_vec(d, dv, d->cx));
  DISPATCH(d, K::energy_change(P_, d->geo, d->m, d->vn, d->u, d->cx, d->desc.gravity, dt, alpha,
                               d->S, d->partials, d->stream));
  OSMPM_TRY(sync_scalars(d));
  *dE = d->S_host->dE;
  return OSMPM_OK;
}

}  // extern "C"
