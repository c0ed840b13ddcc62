// Reverse-mode (vector-Jacobian) device functions of the residual's building blocks, FP64.
// Each *_vjp function adds the adjoint of its inputs, given the adjoint of its outputs, for the
// same arithmetic as the forward functions in kernels.cu (branch decisions held fixed).
#pragma once

#include "kernels.hpp"

namespace hfd {
namespace adj {

// Roe-averaged state (u, v, H, c) of two conservative states (the weights sqrt(rho) form).
struct RoeState {
  double irl, irr, ul, vl, ur, vr, pl, pr, Hl, Hr, rl, rr, fl, fr, u, v, H, c;
};

__device__ __forceinline__ void roe_state(const double* wl, const double* wr, double g1, RoeState& s) {
  s.irl = 1.0 / wl[0];
  s.irr = 1.0 / wr[0];
  s.ul = wl[1] * s.irl; s.vl = wl[2] * s.irl;
  s.ur = wr[1] * s.irr; s.vr = wr[2] * s.irr;
  s.pl = g1 * (wl[3] - 0.5 * (wl[1] * s.ul + wl[2] * s.vl));
  s.pr = g1 * (wr[3] - 0.5 * (wr[1] * s.ur + wr[2] * s.vr));
  s.Hl = (wl[3] + s.pl) * s.irl;
  s.Hr = (wr[3] + s.pr) * s.irr;
  s.rl = sqrt(wl[0]);
  s.rr = sqrt(wr[0]);
  s.fl = s.rl / (s.rl + s.rr);
  s.fr = 1.0 - s.fl;
  s.u = s.fl * s.ul + s.fr * s.ur;
  s.v = s.fl * s.vl + s.fr * s.vr;
  s.H = s.fl * s.Hl + s.fr * s.Hr;
  s.c = sqrt(g1 * (s.H - 0.5 * (s.u * s.u + s.v * s.v)));
}

// adjoint of the primitive quantities of one state: given bars of (u_k, v_k, p_k, H_k) and of
// 1/rho (ir), add to wbar.
__device__ __forceinline__ void prim_vjp(const double* w, double ir, double uk, double vk, double pk,
                                         double ub, double vb, double pb, double Hb, double irb,
                                         double g1, double* wb) {
  // H = (E + p) ir
  wb[3] += Hb * ir;
  pb += Hb * ir;
  irb += Hb * (w[3] + pk);
  // p = g1 (E - 1/2 (m u + n v))
  wb[3] += g1 * pb;
  wb[1] -= 0.5 * g1 * uk * pb;
  ub -= 0.5 * g1 * w[1] * pb;
  wb[2] -= 0.5 * g1 * vk * pb;
  vb -= 0.5 * g1 * w[2] * pb;
  // u = m ir, v = n ir
  wb[1] += ub * ir;
  irb += ub * w[1];
  wb[2] += vb * ir;
  irb += vb * w[2];
  // ir = 1 / rho
  wb[0] -= irb * ir * ir;
}

// adjoint of roe_state: given (ubar, vbar, Hbar, cbar), add to wlb, wrb.
__device__ __forceinline__ void roe_state_vjp(const double* wl, const double* wr, double g1,
                                              const RoeState& s, double ub, double vb, double Hb,
                                              double cb, double* wlb, double* wrb) {
  // c = sqrt(g1 (H - (u^2 + v^2)/2))
  double c2b = cb / (2.0 * s.c);
  Hb += g1 * c2b;
  ub -= g1 * s.u * c2b;
  vb -= g1 * s.v * c2b;
  // u = fl ul + fr ur (same for v, H)
  double flb = ub * s.ul + vb * s.vl + Hb * s.Hl;
  double frb = ub * s.ur + vb * s.vr + Hb * s.Hr;
  double ulb = s.fl * ub, urb = s.fr * ub, vlb = s.fl * vb, vrb = s.fr * vb;
  double Hlb = s.fl * Hb, Hrb = s.fr * Hb;
  flb -= frb;                                   // fr = 1 - fl
  double den = s.rl + s.rr;
  double rlb = flb * s.rr / (den * den), rrb = -flb * s.rl / (den * den);
  wlb[0] += rlb / (2.0 * s.rl);
  wrb[0] += rrb / (2.0 * s.rr);
  prim_vjp(wl, s.irl, s.ul, s.vl, s.pl, ulb, vlb, 0.0, Hlb, 0.0, g1, wlb);
  prim_vjp(wr, s.irr, s.ur, s.vr, s.pr, urb, vrb, 0.0, Hrb, 0.0, g1, wrb);
}

// adjoint of the left-eigenvector matrix L(u, v, c; n) (kernels.cu: left_ev)
__device__ __forceinline__ void left_ev_vjp(double u, double v, double c, double nx, double ny,
                                            double g1, const double (*Lb)[4], double& ub,
                                            double& vb, double& cb) {
  double ic = 1.0 / c;
  double b1 = g1 * ic * ic;
  double qn = u * nx + v * ny;
  double b1b = 0, b2b = 0, qnb = 0, qtb = 0, icb = 0;
  b2b += 0.5 * Lb[0][0]; qnb += 0.5 * ic * Lb[0][0]; icb += 0.5 * qn * Lb[0][0];
  b2b += 0.5 * Lb[3][0]; qnb -= 0.5 * ic * Lb[3][0]; icb -= 0.5 * qn * Lb[3][0];
  b2b -= Lb[1][0];
  b1b -= 0.5 * u * Lb[0][1]; ub -= 0.5 * b1 * Lb[0][1]; icb -= 0.5 * nx * Lb[0][1];
  b1b -= 0.5 * u * Lb[3][1]; ub -= 0.5 * b1 * Lb[3][1]; icb += 0.5 * nx * Lb[3][1];
  b1b -= 0.5 * v * Lb[0][2]; vb -= 0.5 * b1 * Lb[0][2]; icb -= 0.5 * ny * Lb[0][2];
  b1b -= 0.5 * v * Lb[3][2]; vb -= 0.5 * b1 * Lb[3][2]; icb += 0.5 * ny * Lb[3][2];
  b1b += 0.5 * (Lb[0][3] + Lb[3][3]) - Lb[1][3];
  b1b += u * Lb[1][1]; ub += b1 * Lb[1][1];
  b1b += v * Lb[1][2]; vb += b1 * Lb[1][2];
  qtb -= Lb[2][0];
  // b2 = b1 (u^2 + v^2) / 2
  b1b += 0.5 * (u * u + v * v) * b2b;
  ub += b1 * u * b2b;
  vb += b1 * v * b2b;
  // b1 = g1 ic^2
  icb += 2.0 * g1 * ic * b1b;
  cb -= ic * ic * icb;
  ub += nx * qnb - ny * qtb;
  vb += ny * qnb + nx * qtb;
}

// adjoint of w = R(u, v, H, c; n) C (kernels.cu: right_apply): Cbar and parameter bars
__device__ __forceinline__ void right_apply_vjp(double u, double v, double H, double c, double nx,
                                                double ny, const double* C, const double* wb,
                                                double* Cb, double& ub, double& vb, double& Hb,
                                                double& cb) {
  double qn = u * nx + v * ny, qt = -u * ny + v * nx, K = u * u + v * v;
  Cb[0] += wb[0] + (u - c * nx) * wb[1] + (v - c * ny) * wb[2] + (H - c * qn) * wb[3];
  Cb[1] += wb[0] + u * wb[1] + v * wb[2] + 0.5 * K * wb[3];
  Cb[2] += -ny * wb[1] + nx * wb[2] + qt * wb[3];
  Cb[3] += wb[0] + (u + c * nx) * wb[1] + (v + c * ny) * wb[2] + (H + c * qn) * wb[3];
  double s013 = C[0] + C[1] + C[3];
  ub += wb[1] * s013 + wb[3] * (-c * nx * C[0] + u * C[1] - ny * C[2] + c * nx * C[3]);
  vb += wb[2] * s013 + wb[3] * (-c * ny * C[0] + v * C[1] + nx * C[2] + c * ny * C[3]);
  Hb += wb[3] * (C[0] + C[3]);
  cb += (wb[1] * nx + wb[2] * ny + wb[3] * qn) * (C[3] - C[0]);
}

// adjoint of the Roe flux h(wl, wr; n) (kernels.cu: roe_flux)
__device__ void roe_flux_vjp(const double* wl, const double* wr, double nx, double ny, double g1,
                             double harten, const double* hb, double* wlb, double* wrb) {
  RoeState s;
  roe_state(wl, wr, g1, s);
  const double u = s.u, v = s.v, H = s.H, c = s.c;
  double ic = 1.0 / c, b1 = g1 * ic * ic, b2 = 0.5 * b1 * (u * u + v * v);
  double qn = u * nx + v * ny, qt = -u * ny + v * nx;
  double L[4][4] = {
      {0.5 * (b2 + qn * ic), -0.5 * (b1 * u + nx * ic), -0.5 * (b1 * v + ny * ic), 0.5 * b1},
      {1.0 - b2, b1 * u, b1 * v, -b1},
      {-qt, -ny, nx, 0.0},
      {0.5 * (b2 - qn * ic), -0.5 * (b1 * u - nx * ic), -0.5 * (b1 * v - ny * ic), 0.5 * b1}};
  double d[4] = {wr[0] - wl[0], wr[1] - wl[1], wr[2] - wl[2], wr[3] - wl[3]};
  double lam[4] = {qn - c, qn, qn, qn + c};
  double del = harten * c;
  double alpha[4], al[4], k[4];
  bool fixd[4];
  for (int i = 0; i < 4; ++i) {
    alpha[i] = L[i][0] * d[0] + L[i][1] * d[1] + L[i][2] * d[2] + L[i][3] * d[3];
    al[i] = fabs(lam[i]);
    fixd[i] = al[i] < del;
    if (fixd[i]) al[i] = (lam[i] * lam[i] + del * del) / (2.0 * del);
    k[i] = al[i] * alpha[i];
  }
  // h = 1/2 (f(wl) + f(wr)) - 1/2 R k
  double dissb[4] = {-0.5 * hb[0], -0.5 * hb[1], -0.5 * hb[2], -0.5 * hb[3]};
  double ub = 0, vb = 0, Hb = 0, cb = 0;
  double kb[4] = {0, 0, 0, 0};
  right_apply_vjp(u, v, H, c, nx, ny, k, dissb, kb, ub, vb, Hb, cb);
  double Lb[4][4];
  double db[4] = {0, 0, 0, 0};
  double qnb = 0, delb = 0;
  for (int i = 0; i < 4; ++i) {
    double ab = al[i] * kb[i], alb = alpha[i] * kb[i];
    double lamb;
    if (fixd[i]) {
      lamb = lam[i] / del * alb;
      delb += (0.5 - lam[i] * lam[i] / (2.0 * del * del)) * alb;
    } else {
      lamb = (lam[i] >= 0 ? 1.0 : -1.0) * alb;
    }
    qnb += lamb;
    if (i == 0) cb -= lamb;
    if (i == 3) cb += lamb;
    for (int j = 0; j < 4; ++j) {
      db[j] += ab * L[i][j];
      Lb[i][j] = ab * d[j];
    }
  }
  cb += harten * delb;
  ub += nx * qnb;
  vb += ny * qnb;
  left_ev_vjp(u, v, c, nx, ny, g1, Lb, ub, vb, cb);
  for (int j = 0; j < 4; ++j) {
    wrb[j] += db[j];
    wlb[j] -= db[j];
  }
  // normal fluxes of both sides (with their own primitive quantities)
  for (int side = 0; side < 2; ++side) {
    const double* w = side == 0 ? wl : wr;
    double* wbx = side == 0 ? wlb : wrb;
    double uk = side == 0 ? s.ul : s.ur, vk = side == 0 ? s.vl : s.vr;
    double pk = side == 0 ? s.pl : s.pr, ir = side == 0 ? s.irl : s.irr;
    double un = uk * nx + vk * ny;
    double f0 = 0.5 * hb[0], f1 = 0.5 * hb[1], f2 = 0.5 * hb[2], f3 = 0.5 * hb[3];
    double unb = f0 * w[0] + f1 * w[1] + f2 * w[2] + f3 * (w[3] + pk);
    wbx[0] += f0 * un;
    wbx[1] += f1 * un;
    wbx[2] += f2 * un;
    wbx[3] += f3 * un;
    double pb = f1 * nx + f2 * ny + f3 * un;
    prim_vjp(w, ir, uk, vk, pk, nx * unb, ny * unb, pb, 0.0, 0.0, g1, wbx);
  }
  roe_state_vjp(wl, wr, g1, s, ub, vb, Hb, cb, wlb, wrb);
}

// adjoint of one side of Rusanov's flux: the normal flux f(w) = (rho u_n, m u_n + p n_x,
// n u_n + p n_y, (E + p) u_n) with bar fb, and the side's speed |u_n| + c with bar sb
__device__ __forceinline__ void rusanov_side_vjp(const double* w, double nx, double ny, double g1,
                                                 const double* fb, double sb, double* wb) {
  const double ir = 1.0 / w[0], u = w[1] * ir, v = w[2] * ir;
  const double p = g1 * (w[3] - 0.5 * (w[1] * u + w[2] * v));
  const double un = u * nx + v * ny, gam = g1 + 1.0;
  const double c = sqrt(gam * p * ir);
  const double unb = fb[0] * w[0] + fb[1] * w[1] + fb[2] * w[2] + fb[3] * (w[3] + p) +
                     (un < 0.0 ? -sb : sb);
  const double pb = fb[1] * nx + fb[2] * ny + fb[3] * un + sb * gam * ir / (2.0 * c);
  const double irb = sb * gam * p / (2.0 * c);
  wb[0] += fb[0] * un;
  wb[1] += fb[1] * un;
  wb[2] += fb[2] * un;
  wb[3] += fb[3] * un;
  prim_vjp(w, ir, u, v, p, nx * unb, ny * unb, pb, 0.0, irb, g1, wb);
}

// adjoint of Rusanov's flux h = (f(wl) + f(wr)) / 2 - s (wr - wl) / 2, s = max of the two sides'
// |u_n| + c (kernels.cu: rusanov_flux; the larger side takes the bar, the left one on a tie)
__device__ __forceinline__ void rusanov_flux_vjp(const double* wl, const double* wr, double nx,
                                                 double ny, double g1, const double* hb,
                                                 double* wlb, double* wrb) {
  auto speed = [&](const double* w) {
    const double ir = 1.0 / w[0];
    const double un = (w[1] * nx + w[2] * ny) * ir;
    const double p = g1 * (w[3] - 0.5 * (w[1] * w[1] + w[2] * w[2]) * ir);
    return fabs(un) + sqrt((g1 + 1.0) * p * ir);
  };
  const double sl = speed(wl), sr = speed(wr);
  const double s = sl >= sr ? sl : sr;
  double sbar = 0.0, fb[4];
  for (int i = 0; i < 4; ++i) {
    fb[i] = 0.5 * hb[i];
    sbar -= 0.5 * hb[i] * (wr[i] - wl[i]);
    wlb[i] += 0.5 * s * hb[i];
    wrb[i] -= 0.5 * s * hb[i];
  }
  rusanov_side_vjp(wl, nx, ny, g1, fb, sl >= sr ? sbar : 0.0, wlb);
  rusanov_side_vjp(wr, nx, ny, g1, fb, sl >= sr ? 0.0 : sbar, wrb);
}

// adjoint of the edge's numerical flux with the solver the mesh was built with
__device__ __forceinline__ void riemann_flux_vjp(const double* wl, const double* wr, double nx,
                                                 double ny, const Phys& ph, const double* hb,
                                                 double* wlb, double* wrb) {
  if (ph.flux == 1)
    rusanov_flux_vjp(wl, wr, nx, ny, ph.g1, hb, wlb, wrb);
  else
    roe_flux_vjp(wl, wr, nx, ny, ph.g1, ph.harten, hb, wlb, wrb);
}

// adjoint of the Euler fluxes F(w), G(w) at a vertex: wbar += J_F^T Fb + J_G^T Gb
__device__ __forceinline__ void euler_flux_vjp(const double* w, double g1, const double* Fb,
                                               const double* Gb, double* wb) {
  double ir = 1.0 / w[0];
  double u = w[1] * ir, v = w[2] * ir;
  double p = g1 * (w[3] - 0.5 * (w[1] * u + w[2] * v));
  double ub = 0, vb = 0, pb = 0;
  wb[1] += Fb[0];
  wb[1] += Fb[1] * u; ub += Fb[1] * w[1]; pb += Fb[1];
  wb[2] += Fb[2] * u; ub += Fb[2] * w[2];
  wb[3] += Fb[3] * u; pb += Fb[3] * u; ub += Fb[3] * (w[3] + p);
  wb[2] += Gb[0];
  wb[1] += Gb[1] * v; vb += Gb[1] * w[1];
  wb[2] += Gb[2] * v; vb += Gb[2] * w[2]; pb += Gb[2];
  wb[3] += Gb[3] * v; pb += Gb[3] * v; vb += Gb[3] * (w[3] + p);
  prim_vjp(w, ir, u, v, p, ub, vb, pb, 0.0, 0.0, g1, wb);
}

// adjoint of the viscous fluxes Fv(w), Gv(w) at a vertex (the vertex_body chain: primitive
// gradients by the chain rule, Stokes stresses with constant mu, Fourier heat flux with
// p = rho R T): wbar (12 values: w, w_x, w_y) += J_Fv^T Fb + J_Gv^T Gb, in reverse order of
// the forward statements
__device__ __forceinline__ void viscous_flux_vjp(const double* w, double gm, double mu,
                                                 double kappa, double R, const double* Fb,
                                                 const double* Gb, double* wb) {
  // forward
  const double rho = w[0], ir = 1.0 / rho, u = w[1] * ir, v = w[2] * ir;
  const double ux = (w[5] - u * w[4]) * ir, vx = (w[6] - v * w[4]) * ir;
  const double uy = (w[9] - u * w[8]) * ir, vy = (w[10] - v * w[8]) * ir;
  const double q2 = u * u + v * v;
  const double pp = gm * (w[3] - 0.5 * rho * q2);
  const double px = gm * (w[7] - 0.5 * w[4] * q2 - rho * (u * ux + v * vx));
  const double py = gm * (w[11] - 0.5 * w[8] * q2 - rho * (u * uy + v * vy));
  const double txx = mu * (4.0 / 3.0 * ux - 2.0 / 3.0 * vy);
  const double tyy = mu * (4.0 / 3.0 * vy - 2.0 / 3.0 * ux);
  const double txy = mu * (uy + vx);
  // Fv = (0, txx, txy, u txx + v txy + kappa Tx), Gv = (0, txy, tyy, u txy + v tyy + kappa Ty)
  const double btxx = Fb[1] + Fb[3] * u, btyy = Gb[2] + Gb[3] * v;
  const double btxy = Fb[2] + Fb[3] * v + Gb[1] + Gb[3] * u;
  double bu = Fb[3] * txx + Gb[3] * txy, bv = Fb[3] * txy + Gb[3] * tyy;
  const double bTx = Fb[3] * kappa, bTy = Gb[3] * kappa;
  double bux = mu * (4.0 / 3.0 * btxx - 2.0 / 3.0 * btyy);
  double bvy = mu * (4.0 / 3.0 * btyy - 2.0 / 3.0 * btxx);
  double buy = mu * btxy, bvx = mu * btxy;
  // Tx = (px / rho - pp w4 / rho^2) / R, Ty likewise with py, w8
  const double iR = 1.0 / R, ir2 = ir * ir;
  const double bpx = bTx * iR * ir, bpy = bTy * iR * ir;
  const double bpp = -(bTx * w[4] + bTy * w[8]) * iR * ir2;
  double brho = bTx * iR * (-px * ir2 + 2.0 * pp * w[4] * ir2 * ir) +
                bTy * iR * (-py * ir2 + 2.0 * pp * w[8] * ir2 * ir);
  wb[4] -= bTx * pp * iR * ir2;
  wb[8] -= bTy * pp * iR * ir2;
  // px = gm (w7 - w4 q2 / 2 - rho (u ux + v vx)), py likewise
  double bq2 = -0.5 * gm * (w[4] * bpx + w[8] * bpy);
  wb[7] += gm * bpx;
  wb[11] += gm * bpy;
  wb[4] -= 0.5 * gm * q2 * bpx;
  wb[8] -= 0.5 * gm * q2 * bpy;
  brho -= gm * ((u * ux + v * vx) * bpx + (u * uy + v * vy) * bpy);
  bu -= gm * rho * (ux * bpx + uy * bpy);
  bv -= gm * rho * (vx * bpx + vy * bpy);
  bux -= gm * rho * u * bpx;
  bvx -= gm * rho * v * bpx;
  buy -= gm * rho * u * bpy;
  bvy -= gm * rho * v * bpy;
  // pp = gm (w3 - rho q2 / 2)
  wb[3] += gm * bpp;
  brho -= 0.5 * gm * q2 * bpp;
  bq2 -= 0.5 * gm * rho * bpp;
  // q2 = u^2 + v^2
  bu += 2.0 * u * bq2;
  bv += 2.0 * v * bq2;
  // ux = (w5 - u w4) / rho, vx = (w6 - v w4) / rho, uy = (w9 - u w8) / rho, vy = (w10 - v w8) / rho
  wb[5] += bux * ir;
  wb[6] += bvx * ir;
  wb[9] += buy * ir;
  wb[10] += bvy * ir;
  wb[4] -= (u * bux + v * bvx) * ir;
  wb[8] -= (u * buy + v * bvy) * ir;
  bu -= (w[4] * bux + w[8] * buy) * ir;
  bv -= (w[4] * bvx + w[8] * bvy) * ir;
  brho -= (ux * bux + vx * bvx + uy * buy + vy * bvy) * ir;
  // u = w1 / rho, v = w2 / rho
  wb[1] += bu * ir;
  wb[2] += bv * ir;
  brho -= (u * bu + v * bv) * ir;
  wb[0] += brho;
}

}  // namespace adj
}  // namespace hfd
