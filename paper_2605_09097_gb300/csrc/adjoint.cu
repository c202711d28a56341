// Launchers of the reverse-mode kernels (2D and 3D, FP64).
#include "osmpm_adjoint.cuh"
#include "osmpm_internal.h"

namespace osmpm {

template <int D>
void AdjointKernels<D>::g2p(int64_t n, const double* x, const double* F, const GridGeo& g,
                            const double* u, double dt, const double* xb, const double* vb,
                            const double* Bb, const double* Fb, double* ubar, double* xb_out,
                            double* Fb_out, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_g2p<D><<<blocks_for(n), kThreads, 0, s>>>(n, x, F, g, u, dt, xb, vb, Bb, Fb, ubar, xb_out,
                                                  Fb_out);
}
template <int D>
void AdjointKernels<D>::rhs(const GridGeo& g, const double* m, const uint8_t* dofmask, double dt,
                            double cg_rtol, int cg_max, const double* ubar, double* diag,
                            double* x, double* r, double* z, double* p, DevScalars* S,
                            double* partials, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_rhs<D><<<red_blocks_for(g.nn * D), kThreads, 0, s>>>(g, m, dofmask, dt, cg_rtol, cg_max,
                                                             ubar, diag, x, r, z, p, S, partials);
}
template <int D>
void AdjointKernels<D>::solve(int64_t n, const double* x, const double* F, const double* mu,
                              const double* lam, const double* vol0, const GridGeo& g,
                              const double* u, const double* lamg, const uint8_t* dofmask,
                              double* xb, double* Fb, double* Eb, double* klam, int* err,
                              cudaStream_t s) {
  g_launch_count += 1;
  k_adj_solve<D><<<blocks_for(n), kThreads, 0, s>>>(n, x, F, mu, lam, vol0, g, u, lamg, dofmask,
                                                    xb, Fb, Eb, klam, err);
}
template <int D>
void AdjointKernels<D>::nodes(const GridGeo& g, const double* m, const double* vn, const double* u,
                              const double* lamg, const double* gravity, double dt,
                              const double* mextra, double* qbar, double* mbar, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_nodes<D><<<red_blocks_for(g.nn), kThreads, 0, s>>>(g, m, vn, u, lamg, gravity[0],
                                                           gravity[1], gravity[2], dt, mextra,
                                                           qbar, mbar);
}
template <int D>
void AdjointKernels<D>::bc(const GridGeo& g, const uint8_t* recv, const double* m, const double* ubar,
                           const double* klam, double s0, double s1, double* v0bar, double* v1bar,
                           cudaStream_t s) {
  g_launch_count += 1;
  k_adj_bc<D><<<red_blocks_for(g.nn), kThreads, 0, s>>>(g, recv, m, ubar, klam, s0, s1, v0bar, v1bar);
}
template <int D>
void AdjointKernels<D>::interp_t(const GridGeo& gB, const GridGeo& gS, const uint8_t* recvS,
                                 const double* vbar, double* out, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_interp<D><<<red_blocks_for(gS.nn), kThreads, 0, s>>>(gB, gS, recvS, vbar, out);
}
template <int D>
void AdjointKernels<D>::proj_coarse(const GridGeo& gB, const uint8_t* recvB, const double* num,
                                    const double* den, double eps, const double* vbar,
                                    double* nbar, double* dbar, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_proj_coarse<D><<<red_blocks_for(gB.nn), kThreads, 0, s>>>(gB, recvB, num, den, eps, vbar,
                                                                  nbar, dbar);
}
template <int D>
void AdjointKernels<D>::proj_fine(const GridGeo& gB, const GridGeo& gS, const double* nbar,
                                  const double* dbar, double* G, double* H, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_proj_fine<D><<<red_blocks_for(gS.nn), kThreads, 0, s>>>(gB, gS, nbar, dbar, G, H);
}
template <int D>
void AdjointKernels<D>::inject(const GridGeo& g, const double* m, const double* u, double dt,
                               const double* G, const double* H, double* ubar, double* mextra,
                               cudaStream_t s) {
  g_launch_count += 1;
  k_adj_inject<D><<<red_blocks_for(g.nn), kThreads, 0, s>>>(g, m, u, dt, G, H, ubar, mextra);
}
template <int D>
void AdjointKernels<D>::grid_acc(const GridGeo& g, const double* m, const double* vn,
                                 const double* G, const double* H, const double* vbar,
                                 double* qbar, double* mbar, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_grid_acc<D><<<red_blocks_for(g.nn), kThreads, 0, s>>>(g, m, vn, G, H, vbar, qbar, mbar);
}
template <int D>
void AdjointKernels<D>::axpy_active(const GridGeo& g, const double* m, double scale, const double* v,
                                    double* out, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_axpy_active<D><<<red_blocks_for(g.nn * D), kThreads, 0, s>>>(g, m, scale, v, out);
}
template <int D>
void AdjointKernels<D>::add(int64_t cnt, const double* src, double* dst, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_add<D><<<red_blocks_for(cnt), kThreads, 0, s>>>(cnt, src, dst);
}
template <int D>
void AdjointKernels<D>::p2g(int64_t n, const double* x, const double* v, const double* B,
                            const double* mass, const GridGeo& g, const double* qbar,
                            const double* mbar, double* vb_out, double* Bb_out, double* xb,
                            cudaStream_t s) {
  g_launch_count += 1;
  k_adj_p2g<D><<<blocks_for(n), kThreads, 0, s>>>(n, x, v, B, mass, g, qbar, mbar, vb_out, Bb_out,
                                                  xb);
}
template <int D>
void AdjointKernels<D>::from_ids(int64_t n, int w, const uint32_t* id, const double* src,
                                 double* dst, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_from_ids<D><<<red_blocks_for(n * w), kThreads, 0, s>>>(n, w, id, src, dst);
}
template <int D>
void AdjointKernels<D>::to_ids(int64_t n, int w, const uint32_t* id, const double* src,
                               double* dst, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_to_ids<D><<<red_blocks_for(n * w), kThreads, 0, s>>>(n, w, id, src, dst);
}

template struct AdjointKernels<2>;
template struct AdjointKernels<3>;

}  // namespace osmpm
