// Reverse-mode kernels of the backward-Euler MPM step (Sec. 2.2), FP64.
//
// A recorded step maps (x, v, B, F) and the moduli to the next state through
// APIC P2G, the implicit solve g(u*) = 0 and G2P with the F update and
// advection.  Walking a step backwards:
//   k_adj_g2p    transposed G2P / F update / advection: u_bar on the grid and
//                the direct x_bar, F_bar terms (N and grad N depend on x_p,
//                hence the B-spline Hessian);
//   (adjoint PCG) K lam = u_bar on the free DOFs with the step's own
//                symmetric Hessian-vector product (implicit function theorem);
//   k_adj_solve  -lam . dg/dz for z = F_p, mu_p, lam_p (-> E_p) and x_p;
//   k_adj_nodes  -lam . dg/dz for the nodal mass and velocity, then through
//                v_i = q_i / m_i;
//   k_adj_p2g    transposed APIC P2G: v_bar, B_bar and the x_bar terms.
// Particle arrays are component-major in the domain's sorted order.
#pragma once

#include "osmpm_kernels.cuh"

namespace osmpm {

// Second derivative of the 1D weight of stencil offset o with respect to
// the particle position: (1, -2, 1) / dx^2.
__device__ __forceinline__ double bspline_dd(int o, double inv_dx) {
  return (o == 1 ? -2.0 : 1.0) * inv_dx * inv_dx;
}

// Hessian of N_k(x) at the particle (stencil node k), row-major D x D.
template <int D>
__device__ __forceinline__ void stencil_hessian(const Stencil<D>& s, double inv_dx, int k, double* H) {
  int off[3];
  off[0] = k % 3;
  off[1] = (k / 3) % 3;
  off[2] = k / 9;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double f = 1.0;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        if (a == b)
          f *= (c == a) ? bspline_dd(off[c], inv_dx) : s.w[c][off[c]];
        else
          f *= (c == a || c == b) ? s.dw[c][off[c]] : s.w[c][off[c]];
      }
      H[a * D + b] = f;
    }
}

template <int D>
__device__ __forceinline__ void load_vec(const double* a, int64_t n, int64_t p, double* out, int w) {
  for (int e = 0; e < w; ++e) out[e] = a[(int64_t)e * n + p];
}

// Transposed G2P (Eqs. g2p_v, g2p_B, F_update, advection): from the adjoints
// of x', v', B', F' to u_bar (scattered), the direct x_bar and F_bar.
template <int D>
__global__ void __launch_bounds__(kThreads) k_adj_g2p(int64_t n, const double* x, const double* F,
                                                      GridGeo g, const double* u, double dt,
                                                      const double* xb, const double* vb,
                                                      const double* Bb, const double* Fb,
                                                      double* ubar, double* xb_out,
                                                      double* Fb_out) {
  constexpr int DD = D * D;
  constexpr int K = (D == 2) ? 9 : 27;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double xp[D], Fp[DD], xbp[D], vbp[D], Bbp[DD], Fbp[DD];
  load_vec<D>(x, n, p, xp, D);
  load_vec<D>(F, n, p, Fp, DD);
  load_vec<D>(xb, n, p, xbp, D);
  load_vec<D>(vb, n, p, vbp, D);
  load_vec<D>(Bb, n, p, Bbp, DD);
  load_vec<D>(Fb, n, p, Fbp, DD);
  Stencil<D> s;
  make_stencil<D>(xp, g, s);
  const double inv_dt = 1.0 / dt;
  // M1 = Fbar F^T (its transpose F Fbar^T feeds the Hessian term)
  double M1[DD];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double t = 0.0;
#pragma unroll
      for (int b = 0; b < D; ++b) t += Fbp[a * D + b] * Fp[c * D + b];
      M1[a * D + c] = t;
    }
  double xv[D], xacc[D], A[DD];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    xv[a] = xbp[a] + vbp[a] * inv_dt;
    xacc[a] = xbp[a];
  }
#pragma unroll
  for (int e = 0; e < DD; ++e) A[e] = (e % (D + 1)) == 0 ? 1.0 : 0.0;
  for (int k = 0; k < K; ++k) {
    double N, dN[D];
    const int64_t node = stencil_node<D>(s, g, k, N, dN);
    double dxi[D], uk[D], Bd[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      dxi[a] = stencil_node_pos<D>(s, g, k, a) - xp[a];
      uk[a] = u[(int64_t)a * g.nn + node];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double t = 0.0;
#pragma unroll
      for (int b = 0; b < D; ++b) t += Bbp[a * D + b] * dxi[b];
      Bd[a] = t;
    }
    double sk = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double c = N * xv[a] + N * inv_dt * Bd[a];
#pragma unroll
      for (int b = 0; b < D; ++b) c += M1[a * D + b] * dN[b];
      atomicAdd(&ubar[(int64_t)a * g.nn + node], c);
      sk += xv[a] * uk[a] + uk[a] * Bd[a] * inv_dt;
    }
    double H[DD], t[D];
    stencil_hessian<D>(s, g.inv_dx, k, H);
    // t = F Fbar^T u_k = M1^T u_k
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double v = 0.0;
#pragma unroll
      for (int d2 = 0; d2 < D; ++d2) v += M1[d2 * D + b] * uk[d2];
      t[b] = v;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double btu = 0.0, ht = 0.0;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        btu += Bbp[b * D + a] * uk[b];
        ht += H[a * D + b] * t[b];
      }
      xacc[a] += dN[a] * sk - N * inv_dt * btu + ht;
#pragma unroll
      for (int b = 0; b < D; ++b) A[a * D + b] += uk[a] * dN[b];
    }
  }
#pragma unroll
  for (int a = 0; a < D; ++a) xb_out[(int64_t)a * n + p] = xacc[a];
  // F_bar = A^T Fbar'
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double v = 0.0;
#pragma unroll
      for (int b = 0; b < D; ++b) v += A[b * D + a] * Fbp[b * D + c];
      Fb_out[(int64_t)(a * D + c) * n + p] = v;
    }
}

// Right-hand side of the adjoint system: r = u_bar on the free DOFs, x = 0,
// the inverted Jacobi diagonal, and the PCG controls (tolerance cg_rtol |r|).
template <int D>
__global__ void k_adj_rhs(GridGeo g, const double* m, const uint8_t* dofmask, double dt,
                          double cg_rtol, int cg_max, const double* ubar, double* diag, double* x,
                          double* r, double* z, double* p, DevScalars* S, double* partials) {
  const double inv_dt2 = 1.0 / (dt * dt);
  double acc[2] = {0.0, 0.0};
  const int64_t total = g.nn * D;
  for (int64_t idx = gtid(); idx < total; idx += gstride()) {
    const int a = (int)(idx / g.nn);
    const int64_t i = idx - (int64_t)a * g.nn;
    const bool fr = (dofmask[i] >> a) & 1u;
    x[idx] = 0.0;
    if (fr) {
      const double dg = 1.0 / (diag[idx] + m[i] * inv_dt2);
      diag[idx] = dg;
      const double ri = ubar[idx];
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
    S->tol2 = cg_rtol * cg_rtol * tot[1];
    S->cg_iter = 0;
    S->cg_max = cg_max;
    S->cg_neg = 0;
    S->cg_done = (tot[1] == 0.0) ? 1 : 0;
    S->beta = 0.0;
  }
}

// -lam . dg/dz for the particle inputs of g: F_p, mu_p, lam_p and x_p (the
// last through grad N in F_p(u) and in the internal force).  E_bar gets
// (mu_bar mu + lam_bar lam) / E, both moduli being proportional to E.
// With klam, also scatters (K lam)_i = sum_p V Y F^T grad N_i onto the fixed
// DOFs (the adjoint of prescribed displacements needs u_bar_D - (K lam)_D).
template <int D>
__global__ void __launch_bounds__(kThreads) k_adj_solve(int64_t n, const double* x, const double* F,
                                                        const double* mu, const double* lamb,
                                                        const double* vol0, GridGeo g,
                                                        const double* u, const double* lam,
                                                        const uint8_t* dofmask, double* xb,
                                                        double* Fb, double* Eb, double* klam,
                                                        int* err) {
  constexpr int DD = D * D;
  constexpr int K = (D == 2) ? 9 : 27;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double xp[D], Fp[DD];
  load_vec<D>(x, n, p, xp, D);
  load_vec<D>(F, n, p, Fp, DD);
  Stencil<D> s;
  make_stencil<D>(xp, g, s);
  double Gu[DD], Gl[DD];
#pragma unroll
  for (int e = 0; e < DD; ++e) Gu[e] = Gl[e] = 0.0;
  for (int k = 0; k < K; ++k) {
    double N, dN[D];
    const int64_t node = stencil_node<D>(s, g, k, N, dN);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double ua = u[(int64_t)a * g.nn + node];
      const double la = lam[(int64_t)a * g.nn + node];
#pragma unroll
      for (int b = 0; b < D; ++b) {
        Gu[a * D + b] += ua * dN[b];
        Gl[a * D + b] += la * dN[b];
      }
    }
  }
  double A[DD], Fh[DD], X[DD];
#pragma unroll
  for (int e = 0; e < DD; ++e) A[e] = Gu[e] + ((e % (D + 1)) == 0 ? 1.0 : 0.0);
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double t = 0.0, t2 = 0.0;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        t += A[a * D + b] * Fp[b * D + c];
        t2 += Gl[a * D + b] * Fp[b * D + c];
      }
      Fh[a * D + c] = t;
      X[a * D + c] = t2;
    }
  const double mup = mu[p], lp = lamb[p], V = vol0[p];
  NeoHookean<D> nh;
  if (!neo_hookean<D>(Fh, mup, lp, nh)) {
    atomicOr(err, kErrNonFinite);
    return;
  }
  double P[DD], Y[DD];
  pk1<D>(Fh, mup, lp, nh, P);
  dpdf_apply<D>(X, mup, lp, nh, Y);
  double fx = 0.0, ix = 0.0;
#pragma unroll
  for (int e = 0; e < DD; ++e) {
    fx += (Fh[e] - nh.FiT[e]) * X[e];
    ix += nh.FiT[e] * X[e];
  }
  const double mub = -V * fx, lab = -V * nh.lnJ * ix;
  const double E = mup * (3.0 * lp + 2.0 * mup) / (lp + mup);
  Eb[p] += (mub * mup + lab * lp) / E;
  // F_bar -= V (A^T Y + Gl^T P)
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double t = 0.0;
#pragma unroll
      for (int b = 0; b < D; ++b) t += A[b * D + a] * Y[b * D + c] + Gl[b * D + a] * P[b * D + c];
      Fb[(int64_t)(a * D + c) * n + p] -= V * t;
    }
  // x_bar -= V sum_k H_k F (Y^T u_k + P^T lam_k)
  double xacc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) xacc[a] = 0.0;
  for (int k = 0; k < K; ++k) {
    double N, dN[D];
    const int64_t node = stencil_node<D>(s, g, k, N, dN);
    double uk[D], lk[D], Z[D], t[D], H[DD];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      uk[a] = u[(int64_t)a * g.nn + node];
      lk[a] = lam[(int64_t)a * g.nn + node];
    }
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double v = 0.0;
#pragma unroll
      for (int a = 0; a < D; ++a) v += Y[a * D + b] * uk[a] + P[a * D + b] * lk[a];
      Z[b] = v;
    }
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) v += Fp[b * D + c] * Z[c];
      t[b] = v;
    }
    stencil_hessian<D>(s, g.inv_dx, k, H);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double v = 0.0;
#pragma unroll
      for (int b = 0; b < D; ++b) v += H[a * D + b] * t[b];
      xacc[a] += v;
    }
    if (klam) {
      const unsigned fm = dofmask[node];
      double ftn[D];  // F^T grad N_k
#pragma unroll
      for (int e = 0; e < D; ++e) {
        double v = 0.0;
#pragma unroll
        for (int b = 0; b < D; ++b) v += Fp[b * D + e] * dN[b];
        ftn[e] = v;
      }
#pragma unroll
      for (int c = 0; c < D; ++c) {
        if ((fm >> c) & 1u) continue;
        double v = 0.0;
#pragma unroll
        for (int e = 0; e < D; ++e) v += Y[c * D + e] * ftn[e];
        atomicAdd(&klam[(int64_t)c * g.nn + node], V * v);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < D; ++a) xb[(int64_t)a * n + p] -= V * xacc[a];
}

// Nodal part: -lam . dg/dz for z = v_i (m_i/dt lam_i) and m_i
// (-lam_i . ((u_i - dt v_i)/dt^2 - g)), then through v_i = q_i / m_i:
// q_bar = v_bar / m, m_bar -= v_bar . v / m.  lam vanishes off the free DOFs.
// Adds to qbar and mbar; mextra (may be null) is a further adjoint of m_i.
template <int D>
__global__ void k_adj_nodes(GridGeo g, const double* m, const double* vn, const double* u,
                            const double* lam, double gx, double gy, double gz, double dt,
                            const double* mextra, double* qbar, double* mbar) {
  const double gv[3] = {gx, gy, gz};
  for (int64_t i = gtid(); i < g.nn; i += gstride()) {
    const double mi = m[i];
    if (!(mi > g.mass_eps)) continue;
    double mb = mextra ? mextra[i] : 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int64_t idx = (int64_t)a * g.nn + i;
      const double l = lam[idx];
      const double vi = vn[idx];
      const double vba = mi / dt * l;
      mb -= l * ((u[idx] - dt * vi) / (dt * dt) - gv[a]);
      mb -= vba * vi / mi;
      qbar[idx] += vba / mi;
    }
    mbar[i] += mb;
  }
}

// Transposed APIC P2G (Eq. p2g_transfer) with D_p^-1 = 4/dx^2 I.
template <int D>
__global__ void __launch_bounds__(kThreads) k_adj_p2g(int64_t n, const double* x, const double* v,
                                                      const double* B, const double* mass,
                                                      GridGeo g, const double* qbar,
                                                      const double* mbar, double* vb_out,
                                                      double* Bb_out, double* xb) {
  constexpr int DD = D * D;
  constexpr int K = (D == 2) ? 9 : 27;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double xp[D], vp[D], Bp[DD];
  load_vec<D>(x, n, p, xp, D);
  load_vec<D>(v, n, p, vp, D);
  load_vec<D>(B, n, p, Bp, DD);
  const double mp = mass[p];
  const double Dinv = 4.0 * g.inv_dx * g.inv_dx;
  Stencil<D> s;
  make_stencil<D>(xp, g, s);
  double vb[D], Bb[DD], xacc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) vb[a] = xacc[a] = 0.0;
#pragma unroll
  for (int e = 0; e < DD; ++e) Bb[e] = 0.0;
  for (int k = 0; k < K; ++k) {
    double N, dN[D];
    const int64_t node = stencil_node<D>(s, g, k, N, dN);
    double dxi[D], qk[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      dxi[a] = stencil_node_pos<D>(s, g, k, a) - xp[a];
      qk[a] = qbar[(int64_t)a * g.nn + node];
    }
    const double mk = mbar[node];
    double qv = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double vel = vp[a];
#pragma unroll
      for (int b = 0; b < D; ++b) vel += Dinv * Bp[a * D + b] * dxi[b];
      qv += qk[a] * vel;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vb[a] += mp * N * qk[a];
      double ctq = 0.0;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        Bb[a * D + b] += Dinv * mp * N * qk[a] * dxi[b];
        ctq += Dinv * Bp[b * D + a] * qk[b];
      }
      xacc[a] += mp * (dN[a] * (qv + mk) - N * ctq);
    }
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    vb_out[(int64_t)a * n + p] = vb[a];
    xb[(int64_t)a * n + p] += xacc[a];
  }
#pragma unroll
  for (int e = 0; e < DD; ++e) Bb_out[(int64_t)e * n + p] = Bb[e];
}

// ---------------------------------------------------------------------------
// Coupled step (Alg. 1) in reverse
// ---------------------------------------------------------------------------

// Adjoint of the prescribed velocities on receiver nodes: with u_D = s v on
// an active receiver, v0bar += s0 (u_bar - K lam) and (if v1bar) v1bar +=
// s1 (u_bar - K lam) (the two end values of the temporal interpolation).
template <int D>
__global__ void k_adj_bc(GridGeo g, const uint8_t* recv, const double* m, const double* ubar,
                         const double* klam, double s0, double s1, double* v0bar, double* v1bar) {
  for (int64_t j = gtid(); j < g.nn; j += gstride()) {
    if (!recv[j] || !(m[j] > g.mass_eps)) continue;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int64_t idx = (int64_t)a * g.nn + j;
      const double ud = ubar[idx] - klam[idx];
      v0bar[idx] += s0 * ud;
      if (v1bar) v1bar[idx] += s1 * ud;
    }
  }
}

// Transposed I_{B->S} (Eq. interp_BtoS): each fine receiver scatters
// N_I(x_j) vbar_j onto its coarse support.
template <int D>
__global__ void k_adj_interp(GridGeo gB, GridGeo gS, const uint8_t* recvS, const double* vbar,
                             double* out) {
  for (int64_t j = gtid(); j < gS.nn; j += gstride()) {
    if (!recvS[j]) continue;
    double xs[D];
#pragma unroll
    for (int a = 0; a < D; ++a) xs[a] = node_pos(gS, j, a);
    Stencil<D> s;
    make_stencil<D>(xs, gB, s);
    for (int k = 0; k < Pow3<D>::K; ++k) {
      double N, dN[D];
      const int64_t node = stencil_node<D>(s, gB, k, N, dN);
#pragma unroll
      for (int a = 0; a < D; ++a) atomicAdd(&out[(int64_t)a * gB.nn + node], N * vbar[(int64_t)a * gS.nn + j]);
    }
  }
}

// Transposed Pi_{S->B} (Eq. spatial_projection), coarse part: with
// Pi_I = num_I / (den_I + eps) on the receivers, nbar = vbar / (den + eps)
// and dbar = -vbar . num / (den + eps)^2.
template <int D>
__global__ void k_adj_proj_coarse(GridGeo gB, const uint8_t* recvB, const double* num,
                                  const double* den, double eps, const double* vbar,
                                  double* nbar, double* dbar) {
  for (int64_t I = gtid(); I < gB.nn; I += gstride()) {
    double db = 0.0;
    const bool r = recvB[I];
    const double dd = den[I] + eps;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int64_t idx = (int64_t)a * gB.nn + I;
      const double vb = r ? vbar[idx] : 0.0;
      nbar[idx] = vb / dd;
      db -= vb * num[idx];
    }
    dbar[I] = r ? db / (dd * dd) : 0.0;
  }
}

// Fine part: G_j = sum_I N_I(x_j) nbar_I and H_j = sum_I N_I(x_j) dbar_I
// over the coarse support inside the coarse box (the weights of the forward
// scatter without the fine mass).
template <int D>
__global__ void k_adj_proj_fine(GridGeo gB, GridGeo gS, const double* nbar, const double* dbar,
                                double* G, double* H) {
  for (int64_t j = gtid(); j < gS.nn; j += gstride()) {
    double xs[D];
#pragma unroll
    for (int a = 0; a < D; ++a) xs[a] = node_pos(gS, j, a);
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
    double g[D], h = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) g[a] = 0.0;
    for (int k = 0; k < Pow3<D>::K; ++k) {
      const int off[3] = {k % 3, (k / 3) % 3, k / 9};
      bool in = true;
      int64_t node = 0, stride = 1;
      double N = 1.0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int c = base[a] + off[a];
        in = in && c >= 0 && c < gB.res[a];
        node += (int64_t)c * stride;
        stride *= gB.res[a];
        N *= w[a][off[a]];
      }
      if (!in) continue;
      h += N * dbar[node];
#pragma unroll
      for (int a = 0; a < D; ++a) g[a] += N * nbar[(int64_t)a * gB.nn + node];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) G[(int64_t)a * gS.nn + j] = g[a];
    H[j] = h;
  }
}

// A fine sub-step's share of the step-averaged projection: its solved grid
// (m_j, u_j / dt) entered the sums as m_j u_j / dt and m_j, so
// u_bar_j += m_j / dt G_j and the mass adjoint m_extra_j = u_j / dt . G_j + H_j
// on the sub-step's active nodes.
template <int D>
__global__ void k_adj_inject(GridGeo g, const double* m, const double* u, double dt,
                             const double* G, const double* H, double* ubar, double* mextra) {
  for (int64_t j = gtid(); j < g.nn; j += gstride()) {
    double mx = 0.0;
    const double mj = m[j];
    if (mj > g.mass_eps) {
      mx = H[j];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int64_t idx = (int64_t)a * g.nn + j;
        ubar[idx] += mj / dt * G[idx];
        mx += u[idx] / dt * G[idx];
      }
    }
    mextra[j] = mx;
  }
}

// Adjoints of a P2G grid's momentum and mass (qbar += G, mbar += H) and of
// its velocity v = q / m (qbar += vbar / m, mbar -= vbar . v / m), on the
// active nodes; either source may be null.
template <int D>
__global__ void k_adj_grid_acc(GridGeo g, const double* m, const double* vn, const double* G,
                               const double* H, const double* vbar, double* qbar, double* mbar) {
  for (int64_t j = gtid(); j < g.nn; j += gstride()) {
    const double mj = m[j];
    if (!(mj > g.mass_eps)) continue;
    double mb = H ? H[j] : 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int64_t idx = (int64_t)a * g.nn + j;
      double qb = G ? G[idx] : 0.0;
      if (vbar) {
        qb += vbar[idx] / mj;
        mb -= vbar[idx] * vn[idx] / mj;
      }
      qbar[idx] += qb;
    }
    mbar[j] += mb;
  }
}

// out += scale * v on the active nodes (D components).
template <int D>
__global__ void k_adj_axpy_active(GridGeo g, const double* m, double scale, const double* v,
                                  double* out) {
  for (int64_t idx = gtid(); idx < g.nn * D; idx += gstride()) {
    const int64_t j = idx % g.nn;
    if (m[j] > g.mass_eps) out[idx] += scale * v[idx];
  }
}

// dst += src over cnt doubles.
template <int D>
__global__ void k_adj_add(int64_t cnt, const double* src, double* dst) {
  for (int64_t t = gtid(); t < cnt; t += gstride()) dst[t] += src[t];
}

// Layout changes between the caller's id-ordered, particle-major arrays and
// the sorted component-major ones: dst[e*n + p] = src[id[p]*w + e] and back.
template <int D>
__global__ void k_adj_from_ids(int64_t n, int w, const uint32_t* id, const double* src,
                               double* dst) {
  for (int64_t t = gtid(); t < n * w; t += gstride()) {
    const int64_t p = t / w;
    const int e = (int)(t - p * w);
    dst[(int64_t)e * n + p] = src[(int64_t)id[p] * w + e];
  }
}
template <int D>
__global__ void k_adj_to_ids(int64_t n, int w, const uint32_t* id, const double* src,
                             double* dst) {
  for (int64_t t = gtid(); t < n * w; t += gstride()) {
    const int64_t p = t / w;
    const int e = (int)(t - p * w);
    dst[(int64_t)id[p] * w + e] = src[(int64_t)e * n + p];
  }
}

}  // namespace osmpm
