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
                              const double* u, const double* lamg, double* xb, double* Fb,
                              double* Eb, int* err, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_solve<D><<<blocks_for(n), kThreads, 0, s>>>(n, x, F, mu, lam, vol0, g, u, lamg, xb, Fb, Eb,
                                                    err);
}
template <int D>
void AdjointKernels<D>::nodes(const GridGeo& g, const double* m, const double* vn, const double* u,
                              const double* lamg, const double* gravity, double dt, double* qbar,
                              double* mbar, cudaStream_t s) {
  g_launch_count += 1;
  k_adj_nodes<D><<<red_blocks_for(g.nn), kThreads, 0, s>>>(g, m, vn, u, lamg, gravity[0],
                                                           gravity[1], gravity[2], dt, qbar, mbar);
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
