// Discrete adjoint of one SSP-RK3 step (hfd_adjoint): lam_n = (d step / d U_n)^T lam_{n+1}.
//
// The residual is R(U) = -D [F(U), G(U), h(U)] with the fixed least-squares rows D of
// Eq. (flux_polynomials), so its transpose product is
//   (dR/dU)^T mu = -sum_v J_(F,G)(v)^T (D^T mu)_v - sum_e J_h(e)^T (D^T mu)_e.
// D^T is applied as gathers over transposed CSR lists (every vertex and every flux edge lists
// the divergence rows that read it), and the per-edge sensitivities of the 6 stencil nodes are
// gathered per vertex over the transposed stencil lists: no atomics, deterministic.
// k_adj_edge recomputes Alg. 1 and the Roe flux of its edge (the same arithmetic and branch
// decisions as k_edge) and runs them in reverse.  The three stages of the step are recomputed
// forward from U_n, then reversed (Sec. 2.3 end: u1 = u + dt R(u), u2 = 3/4 u + 1/4 (u1 + dt
// R(u1)), u+ = 1/3 u + 2/3 (u2 + dt R(u2))).  FP64 meshes, Roe or Rusanov flux; on viscous meshes
// the residual adds Dv [Fv, Gv] (vertex-only rows), whose transpose k_adj_vertex gathers over
// the same lists as the vertex part of D.
//
// Ghost layers (R14) enter through the transpose T of the ghost refresh: a transmissive
// ghost's sensitivity goes to its donor (without the derivative rows the refresh zeroes) and
// its column becomes zero; a fixed ghost (wall band, donor -1) keeps its sensitivity, because
// every stage state holds the step input's band values.  T is applied to lambda_{n+1} (the
// step ends with a refresh) and to every residual product (each stage starts with one).  The
// stage recurrences below then hold column by column: for a band column the SSP-RK3 weights
// of each level sum to one, which gives lambda_{n+1} plus each stage's residual product.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "adjoint_kernels.cuh"
#include "kernels.hpp"
#include "mesh.hpp"
#include "prep.hpp"

namespace hfd {

// FP32 sensor of k_edge (same arithmetic, so the same branch decisions)
__device__ __forceinline__ void smooth3(float u0, float u1, float u2, float u3, float u4, float* b) {
  float a = u0 - 2.f * u1 + u2, e = u0 - 4.f * u1 + 3.f * u2;
  b[0] = (13.0f / 12.0f) * a * a + 0.25f * e * e;
  a = u1 - 2.f * u2 + u3;
  e = u1 - u3;
  b[1] = (13.0f / 12.0f) * a * a + 0.25f * e * e;
  a = u2 - 2.f * u3 + u4;
  e = 3.f * u2 - 4.f * u3 + u4;
  b[2] = (13.0f / 12.0f) * a * a + 0.25f * e * e;
}

__device__ __forceinline__ void smooth3d(double u0, double u1, double u2, double u3, double u4,
                                         double* b, double* a, double* e) {
  a[0] = u0 - 2.0 * u1 + u2; e[0] = u0 - 4.0 * u1 + 3.0 * u2;
  a[1] = u1 - 2.0 * u2 + u3; e[1] = u1 - u3;
  a[2] = u2 - 2.0 * u3 + u4; e[2] = 3.0 * u2 - 4.0 * u3 + u4;
  for (int j = 0; j < 3; ++j) b[j] = (13.0 / 12.0) * a[j] * a[j] + 0.25 * e[j] * e[j];
}

__device__ __forceinline__ void left_ev_d(double u, double v, double c, double nx, double ny,
                                          double g1, double (*L)[4]) {
  double qn = u * nx + v * ny, qt = -u * ny + v * nx;
  double ic = 1.0 / c;
  double b1 = g1 * ic * ic, b2 = 0.5 * b1 * (u * u + v * v);
  L[0][0] = 0.5 * (b2 + qn * ic); L[0][1] = -0.5 * (b1 * u + nx * ic);
  L[0][2] = -0.5 * (b1 * v + ny * ic); L[0][3] = 0.5 * b1;
  L[1][0] = 1.0 - b2; L[1][1] = b1 * u; L[1][2] = b1 * v; L[1][3] = -b1;
  L[2][0] = -qt; L[2][1] = -ny; L[2][2] = nx; L[2][3] = 0.0;
  L[3][0] = 0.5 * (b2 - qn * ic); L[3][1] = -0.5 * (b1 * u - nx * ic);
  L[3][2] = -0.5 * (b1 * v - ny * ic); L[3][3] = 0.5 * b1;
}

__device__ __forceinline__ void right_apply_d(double u, double v, double H, double c, double nx,
                                              double ny, const double* C, double* w) {
  double qn = u * nx + v * ny, qt = -u * ny + v * nx;
  w[0] = C[0] + C[1] + C[3];
  w[1] = (u - c * nx) * C[0] + u * C[1] - ny * C[2] + (u + c * nx) * C[3];
  w[2] = (v - c * ny) * C[0] + v * C[1] + nx * C[2] + (v + c * ny) * C[3];
  w[3] = (H - c * qn) * C[0] + 0.5 * (u * u + v * v) * C[1] + qt * C[2] + (H + c * qn) * C[3];
}

__device__ __forceinline__ double press(const double* w, double g1) {
  return g1 * (w[3] - 0.5 * (w[1] * w[1] + w[2] * w[2]) / w[0]);
}

// Shared front of the edge reverse pass: hbar = -(D^T mu) at the edge, the stencil, the end
// states and the FP32 sensor decisions exactly as k_edge takes them (bit side*4+q of `rough`:
// 3-node branch; of `amb`: inside the guard band, re-decided in FP64).
__device__ __forceinline__ void adj_edge_front(
    int e, int Ef, int V, const int32_t* __restrict__ sten, const double* __restrict__ nrm,
    const double* __restrict__ Ua, const int32_t* __restrict__ eptr,
    const double* __restrict__ ce, const int32_t* __restrict__ te_ptr,
    const int32_t* __restrict__ te_row, const int32_t* __restrict__ te_pos,
    const double* __restrict__ mu, const Phys& ph, double* hb, int* s, double& nx, double& ny,
    double* wi, double* wj, unsigned& rough, unsigned& amb) {
  const double g1 = ph.g1;
  // ---- hbar = -(D^T mu)_e
  for (int q = 0; q < 4; ++q) hb[q] = 0.0;
  for (int t = te_ptr[e]; t < te_ptr[e + 1]; ++t) {
    int r = te_row[t], j = te_pos[t];
    int m0 = eptr[r], M = eptr[r + 1] - m0;
    const double* d = ce + 3 * (size_t)m0;
    double d0 = d[j], dx = d[M + j], dy = d[2 * M + j];
    for (int q = 0; q < 4; ++q)
      hb[q] -= d0 * mu[(size_t)q * V + r] + dx * mu[(size_t)(4 + q) * V + r] +
               dy * mu[(size_t)(8 + q) * V + r];
  }
  for (int k = 0; k < 6; ++k) s[k] = sten[(size_t)k * Ef + e];
  nx = nrm[e];
  ny = nrm[Ef + e];
  for (int r = 0; r < 4; ++r) { wi[r] = Ua[(size_t)s[2] * 12 + r]; wj[r] = Ua[(size_t)s[3] * 12 + r]; }
  // ---- forward: FP32 sensor exactly as k_edge
  rough = 0;
  amb = 0;
  {
    float fi[4] = {(float)wi[0], (float)wi[1], (float)wi[2], (float)wi[3]};
    float fj[4] = {(float)wj[0], (float)wj[1], (float)wj[2], (float)wj[3]};
    float g1f = (float)g1;
    float rl = sqrtf(fi[0]), rr = sqrtf(fj[0]);
    float irl = 1.f / rl, irr = 1.f / rr, is = 1.f / (rl + rr);
    float pl = g1f * (fi[3] - 0.5f * (fi[1] * fi[1] + fi[2] * fi[2]) / fi[0]);
    float pr = g1f * (fj[3] - 0.5f * (fj[1] * fj[1] + fj[2] * fj[2]) / fj[0]);
    float u = (fi[1] * irl + fj[1] * irr) * is, v = (fi[2] * irl + fj[2] * irr) * is;
    float H = ((fi[3] + pl) * irl + (fj[3] + pr) * irr) * is;
    float c = sqrtf(g1f * (H - 0.5f * (u * u + v * v)));
    float fnx = (float)nx, fny = (float)ny;
    float qn = u * fnx + v * fny, qt = -u * fny + v * fnx;
    float ic = 1.f / c, b1 = g1f * ic * ic, b2 = 0.5f * b1 * (u * u + v * v);
    float Lf[4][4] = {
        {0.5f * (b2 + qn * ic), -0.5f * (b1 * u + fnx * ic), -0.5f * (b1 * v + fny * ic), 0.5f * b1},
        {1.f - b2, b1 * u, b1 * v, -b1},
        {-qt, -fny, fnx, 0.f},
        {0.5f * (b2 - qn * ic), -0.5f * (b1 * u - fnx * ic), -0.5f * (b1 * v - fny * ic), 0.5f * b1}};
    float cf[6][4];
    for (int k = 0; k < 6; ++k) {
      float d[4];
      for (int r = 0; r < 4; ++r) d[r] = (float)(Ua[(size_t)s[k] * 12 + r] - wi[r]);
      for (int q = 0; q < 4; ++q)
        cf[k][q] = Lf[q][0] * d[0] + Lf[q][1] * d[1] + Lf[q][2] * d[2] + Lf[q][3] * d[3];
    }
    for (int side = 0; side < 2; ++side)
      for (int q = 0; q < 4; ++q) {
        float uu[5];
        for (int j = 0; j < 5; ++j) uu[j] = cf[side == 0 ? j : 5 - j][q];
        float b[3];
        smooth3(uu[0], uu[1], uu[2], uu[3], uu[4], b);
        float eps = ph.epsf;
        float s0 = eps + b[0], s1 = eps + b[1], s2 = eps + b[2];
        s0 *= s0; s1 *= s1; s2 *= s2;
        float t0 = 0.0625f * s1 * s2, t1 = 0.625f * s0 * s2, t2 = 0.3125f * s0 * s1;
        float S = t0 + t1 + t2;
        float mlo = t0 - ph.sens_lof * S, mhi = ph.sens_hif * S - t0;
        unsigned bit = 1u << (side * 4 + q);
        if (!(mlo > 0.f && mhi > 0.f)) rough |= bit;
        if (!(fabsf(mlo) > 1e-3f * S && fabsf(mhi) > 1e-3f * S)) amb |= bit;
      }
  }
}

// FP64 5-node sums of both sides in conservative variables (the forward interpolation).
__device__ __forceinline__ void adj_edge_w5(int e, int Ef, const int* s, const double* __restrict__ w5,
                                            const double* __restrict__ Ua, double (*W5)[4]) {
  // ---- forward in FP64: 5-node conservative sums, sides with re-decided / 3-node components
  for (int side = 0; side < 2; ++side)
    for (int r = 0; r < 4; ++r) W5[side][r] = 0.0;
  for (int k = 0; k < 6; ++k) {
    const double* a = Ua + (size_t)s[k] * 12;
    for (int side = 0; side < 2; ++side) {
      int j = k - side;
      if (j < 0 || j > 4) continue;
      double wv = w5[(size_t)(15 * side + 3 * j) * Ef + e];
      double wx = w5[(size_t)(15 * side + 3 * j + 1) * Ef + e];
      double wy = w5[(size_t)(15 * side + 3 * j + 2) * Ef + e];
      for (int r = 0; r < 4; ++r) W5[side][r] += wv * a[r] + wx * a[4 + r] + wy * a[8 + r];
    }
  }
}

// One thread per flux edge, edges whose sides both took the 5-node branch: the reverse of the
// Roe flux and of the 5-node sums; each node's 12 sensitivities are formed in registers and
// stored once to Ge[e][72].  Edges with a 3-node or re-decided component are appended to
// `list` for k_adj_edge_full (the order of the list does not matter: each edge writes only
// its own Ge row).
__global__ void __launch_bounds__(128, 3) k_adj_edge(
    int Ef, int V, const int32_t* __restrict__ sten, const double* __restrict__ nrm,
    const double* __restrict__ w5, const double* __restrict__ w3, const double* __restrict__ Ua,
    const int32_t* __restrict__ eptr, const double* __restrict__ ce,
    const int32_t* __restrict__ te_ptr, const int32_t* __restrict__ te_row,
    const int32_t* __restrict__ te_pos, const double* __restrict__ mu, double* __restrict__ Ge,
    Phys ph, int32_t* __restrict__ list, int32_t* __restrict__ count) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Ef) return;
  double hb[4], nx, ny, wi[4], wj[4];
  int s[6];
  unsigned rough, amb;
  adj_edge_front(e, Ef, V, sten, nrm, Ua, eptr, ce, te_ptr, te_row, te_pos, mu, ph, hb, s, nx, ny,
                 wi, wj, rough, amb);
  if (rough | amb) {
    list[atomicAdd(count, 1)] = e;
    return;
  }
  double* ge = Ge + (size_t)e * 72;
  const double g1 = ph.g1;
  double W5[2][4];
  adj_edge_w5(e, Ef, s, w5, Ua, W5);
  bool fb0 = !(W5[0][0] > 0.0) || !(press(W5[0], g1) > 0.0);
  bool fb1 = !(W5[1][0] > 0.0) || !(press(W5[1], g1) > 0.0);
  double wl[4], wr[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    wl[r] = fb0 ? wi[r] : W5[0][r];
    wr[r] = fb1 ? wj[r] : W5[1][r];
  }
  double b0[4] = {0, 0, 0, 0}, b1[4] = {0, 0, 0, 0};
  adj::riemann_flux_vjp(wl, wr, nx, ny, ph, hb, b0, b1);
  double wib[4] = {0, 0, 0, 0}, wjb[4] = {0, 0, 0, 0};
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if (fb0) { wib[r] = b0[r]; b0[r] = 0.0; }
    if (fb1) { wjb[r] = b1[r]; b1[r] = 0.0; }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double g[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) g[i] = 0.0;
    if (k <= 4) {
      double wv = w5[(size_t)(3 * k) * Ef + e], wx = w5[(size_t)(3 * k + 1) * Ef + e];
      double wy = w5[(size_t)(3 * k + 2) * Ef + e];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        g[r] += wv * b0[r];
        g[4 + r] += wx * b0[r];
        g[8 + r] += wy * b0[r];
      }
    }
    if (k >= 1) {
      double wv = w5[(size_t)(15 + 3 * (k - 1)) * Ef + e];
      double wx = w5[(size_t)(16 + 3 * (k - 1)) * Ef + e];
      double wy = w5[(size_t)(17 + 3 * (k - 1)) * Ef + e];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        g[r] += wv * b1[r];
        g[4 + r] += wx * b1[r];
        g[8 + r] += wy * b1[r];
      }
    }
    if (k == 2)
#pragma unroll
      for (int r = 0; r < 4; ++r) g[r] += wib[r];
    if (k == 3)
#pragma unroll
      for (int r = 0; r < 4; ++r) g[r] += wjb[r];
    double2* o = reinterpret_cast<double2*>(ge + 12 * k);
#pragma unroll
    for (int i = 0; i < 6; ++i) o[i] = make_double2(g[2 * i], g[2 * i + 1]);
  }
}

// One thread per listed flux edge (a 3-node or re-decided component on some side): the full
// reverse of Alg. 1 and the Roe flux; writes the sensitivities of the 12 values of the 6
// stencil nodes to Ge[e][72].
__global__ void __launch_bounds__(128) k_adj_edge_full(
    int Ef, int V, const int32_t* __restrict__ sten, const double* __restrict__ nrm,
    const double* __restrict__ w5, const double* __restrict__ w3, const double* __restrict__ Ua,
    const int32_t* __restrict__ eptr, const double* __restrict__ ce,
    const int32_t* __restrict__ te_ptr, const int32_t* __restrict__ te_row,
    const int32_t* __restrict__ te_pos, const double* __restrict__ mu, double* __restrict__ Ge,
    Phys ph, const int32_t* __restrict__ list, const int32_t* __restrict__ count) {
  int li = blockIdx.x * blockDim.x + threadIdx.x;
  if (li >= *count) return;
  int e = list[li];
  double hb[4], nx, ny, wi[4], wj[4];
  int s[6];
  unsigned rough, amb;
  adj_edge_front(e, Ef, V, sten, nrm, Ua, eptr, ce, te_ptr, te_row, te_pos, mu, ph, hb, s, nx, ny,
                 wi, wj, rough, amb);
  double* ge = Ge + (size_t)e * 72;
  const double g1 = ph.g1;
  double W5[2][4];
  adj_edge_w5(e, Ef, s, w5, Ua, W5);
  for (int i = 0; i < 72; ++i) ge[i] = 0.0;
  adj::RoeState rs;
  double L[4][4];
  adj::roe_state(wi, wj, g1, rs);
  left_ev_d(rs.u, rs.v, rs.c, nx, ny, g1, L);
  double wside[2][4], C[2][4];
  bool rough_q[2][4];
  double cq[2][4][5], tt[2][4][3], SS[2][4];
  for (int side = 0; side < 2; ++side) {
    unsigned mine = ((rough | amb) >> (side * 4)) & 15u;
    for (int r = 0; r < 4; ++r) wside[side][r] = W5[side][r];
    for (int q = 0; q < 4; ++q) rough_q[side][q] = false;
    if (!mine) continue;
    for (int q = 0; q < 4; ++q) {
      C[side][q] = L[q][0] * W5[side][0] + L[q][1] * W5[side][1] + L[q][2] * W5[side][2] +
                   L[q][3] * W5[side][3];
      if (!((mine >> q) & 1u)) continue;
      for (int j = 0; j < 5; ++j) {
        const double* a = Ua + (size_t)s[side == 0 ? j : 5 - j] * 12;
        cq[side][q][j] = L[q][0] * a[0] + L[q][1] * a[1] + L[q][2] * a[2] + L[q][3] * a[3];
      }
      double b[3], aa[3], ee[3];
      smooth3d(cq[side][q][0], cq[side][q][1], cq[side][q][2], cq[side][q][3], cq[side][q][4], b,
               aa, ee);
      double s0 = ph.eps + b[0], s1 = ph.eps + b[1], s2 = ph.eps + b[2];
      s0 *= s0; s1 *= s1; s2 *= s2;
      tt[side][q][0] = (1.0 / 16.0) * s1 * s2;
      tt[side][q][1] = (10.0 / 16.0) * s0 * s2;
      tt[side][q][2] = (5.0 / 16.0) * s0 * s1;
      SS[side][q] = tt[side][q][0] + tt[side][q][1] + tt[side][q][2];
      bool smooth = tt[side][q][0] > ph.sens_lo * SS[side][q] && tt[side][q][0] < ph.sens_hi * SS[side][q];
      if (smooth) continue;
      rough_q[side][q] = true;
      const double* w = w3 + (size_t)(9 * side) * Ef + e;
      const double* c = cq[side][q];
      double c1 = w[0] * c[0] + w[Ef] * c[1] + w[2 * (size_t)Ef] * c[2];
      double c2 = w[3 * (size_t)Ef] * c[1] + w[4 * (size_t)Ef] * c[2] + w[5 * (size_t)Ef] * c[3];
      double c3 = w[6 * (size_t)Ef] * c[2] + w[7 * (size_t)Ef] * c[3] + w[8 * (size_t)Ef] * c[4];
      C[side][q] = (tt[side][q][0] * c1 + tt[side][q][1] * c2 + tt[side][q][2] * c3) / SS[side][q];
    }
    right_apply_d(rs.u, rs.v, rs.H, rs.c, nx, ny, C[side], wside[side]);
  }
  bool fb[2];
  fb[0] = !(wside[0][0] > 0.0) || !(press(wside[0], g1) > 0.0);
  fb[1] = !(wside[1][0] > 0.0) || !(press(wside[1], g1) > 0.0);
  if (fb[0]) for (int r = 0; r < 4; ++r) wside[0][r] = wi[r];
  if (fb[1]) for (int r = 0; r < 4; ++r) wside[1][r] = wj[r];
  // ---- reverse
  double wsb[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  double wib[4] = {0, 0, 0, 0}, wjb[4] = {0, 0, 0, 0};
  adj::riemann_flux_vjp(wside[0], wside[1], nx, ny, ph, hb, wsb[0], wsb[1]);
  if (fb[0]) { for (int r = 0; r < 4; ++r) { wib[r] += wsb[0][r]; wsb[0][r] = 0; } }
  if (fb[1]) { for (int r = 0; r < 4; ++r) { wjb[r] += wsb[1][r]; wsb[1][r] = 0; } }
  double ub = 0, vb = 0, Hb = 0, cb = 0;
  double Lb[4][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
  for (int side = 0; side < 2; ++side) {
    unsigned mine = ((rough | amb) >> (side * 4)) & 15u;
    double W5b[4] = {0, 0, 0, 0};
    if (!mine || fb[side]) {
      if (!fb[side]) for (int r = 0; r < 4; ++r) W5b[r] = wsb[side][r];
    } else {
      double Cb[4] = {0, 0, 0, 0};
      adj::right_apply_vjp(rs.u, rs.v, rs.H, rs.c, nx, ny, C[side], wsb[side], Cb, ub, vb, Hb, cb);
      for (int q = 0; q < 4; ++q) {
        if (!rough_q[side][q]) {
          for (int r = 0; r < 4; ++r) {
            W5b[r] += Cb[q] * L[q][r];
            Lb[q][r] += Cb[q] * W5[side][r];
          }
          continue;
        }
        const double* w = w3 + (size_t)(9 * side) * Ef + e;
        const double* c = cq[side][q];
        double c3v[3] = {w[0] * c[0] + w[Ef] * c[1] + w[2 * (size_t)Ef] * c[2],
                         w[3 * (size_t)Ef] * c[1] + w[4 * (size_t)Ef] * c[2] + w[5 * (size_t)Ef] * c[3],
                         w[6 * (size_t)Ef] * c[2] + w[7 * (size_t)Ef] * c[3] + w[8 * (size_t)Ef] * c[4]};
        double S = SS[side][q];
        double om[3] = {tt[side][q][0] / S, tt[side][q][1] / S, tt[side][q][2] / S};
        double cqb[5] = {0, 0, 0, 0, 0};
        double omb[3];
        for (int j = 0; j < 3; ++j) {
          double c3b = om[j] * Cb[q];
          omb[j] = c3v[j] * Cb[q];
          for (int kk = 0; kk < 3; ++kk) cqb[j + kk] += w[(size_t)(3 * j + kk) * Ef] * c3b;
        }
        // omega_j = alpha_j / sum(alpha), alpha_j = d_j / (eps + beta_j)^2
        double b[3], aa[3], ee[3];
        smooth3d(c[0], c[1], c[2], c[3], c[4], b, aa, ee);
        const double dj[3] = {1.0 / 16.0, 10.0 / 16.0, 5.0 / 16.0};
        double al[3], asum = 0;
        for (int j = 0; j < 3; ++j) {
          double sj = ph.eps + b[j];
          al[j] = dj[j] / (sj * sj);
          asum += al[j];
        }
        double dot = omb[0] * om[0] + omb[1] * om[1] + omb[2] * om[2];
        double ab[3], bb[3];
        for (int j = 0; j < 3; ++j) {
          ab[j] = (omb[j] - dot) / asum;
          bb[j] = -2.0 * al[j] / (ph.eps + b[j]) * ab[j];
        }
        // beta_j = 13/12 a_j^2 + 1/4 e_j^2 with the linear combinations a_j, e_j
        double a0b = 13.0 / 6.0 * aa[0] * bb[0], e0b = 0.5 * ee[0] * bb[0];
        double a1b = 13.0 / 6.0 * aa[1] * bb[1], e1b = 0.5 * ee[1] * bb[1];
        double a2b = 13.0 / 6.0 * aa[2] * bb[2], e2b = 0.5 * ee[2] * bb[2];
        cqb[0] += a0b + e0b;
        cqb[1] += -2.0 * a0b - 4.0 * e0b + a1b + e1b;
        cqb[2] += a0b + 3.0 * e0b - 2.0 * a1b + a2b + 3.0 * e2b;
        cqb[3] += a1b - e1b - 2.0 * a2b - 4.0 * e2b;
        cqb[4] += a2b + e2b;
        // cq_j = L_q . w(node j)
        for (int j = 0; j < 5; ++j) {
          int node = side == 0 ? j : 5 - j;
          const double* a = Ua + (size_t)s[node] * 12;
          for (int r = 0; r < 4; ++r) {
            ge[12 * node + r] += cqb[j] * L[q][r];
            Lb[q][r] += cqb[j] * a[r];
          }
        }
      }
    }
    // W5 = sum_k (w5v a_k + w5x a_k,x + w5y a_k,y)
    for (int j = 0; j < 5; ++j) {
      int node = j + side;
      double wv = w5[(size_t)(15 * side + 3 * j) * Ef + e];
      double wx = w5[(size_t)(15 * side + 3 * j + 1) * Ef + e];
      double wy = w5[(size_t)(15 * side + 3 * j + 2) * Ef + e];
      for (int r = 0; r < 4; ++r) {
        ge[12 * node + r] += wv * W5b[r];
        ge[12 * node + 4 + r] += wx * W5b[r];
        ge[12 * node + 8 + r] += wy * W5b[r];
      }
    }
  }
  adj::left_ev_vjp(rs.u, rs.v, rs.c, nx, ny, g1, Lb, ub, vb, cb);
  adj::roe_state_vjp(wi, wj, g1, rs, ub, vb, Hb, cb, wib, wjb);
  for (int r = 0; r < 4; ++r) {
    ge[24 + r] += wib[r];
    ge[36 + r] += wjb[r];
  }
}

// One thread per vertex: vertex-flux part of (dR/dU)^T mu, the edge sensitivities of the
// stencils this vertex belongs to, then out = cx X + cy Y + cz Z + cg g.
__global__ void __launch_bounds__(128) k_adj_vertex(
    int V, const double* __restrict__ Us, const int32_t* __restrict__ vptr,
    const double* __restrict__ cv, const double* __restrict__ cvis,
    const int32_t* __restrict__ tv_ptr,
    const int32_t* __restrict__ tv_row, const int32_t* __restrict__ tv_pos,
    const int32_t* __restrict__ ts_ptr, const int32_t* __restrict__ ts_ent,
    const double* __restrict__ mu, const double* __restrict__ Ge, double* out, double cx,
    const double* X, double cy, const double* Y, double cz, const double* Z, double cg,
    Phys ph) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= V) return;
  // R = -D [F, G, h] + Dv [Fv, Gv]: the Euler fluxes take -D^T mu, the viscous ones +Dv^T mu
  double Fb[4] = {0, 0, 0, 0}, Gb[4] = {0, 0, 0, 0};
  double Fvb[4] = {0, 0, 0, 0}, Gvb[4] = {0, 0, 0, 0};
  for (int t = tv_ptr[u]; t < tv_ptr[u + 1]; ++t) {
    int r = tv_row[t], j = tv_pos[t];
    int n0 = vptr[r], N = vptr[r + 1] - n0;
    const double* c = cv + 6 * (size_t)n0;
    double d0f = c[j], d0g = c[N + j], dxf = c[2 * N + j], dxg = c[3 * N + j];
    double dyf = c[4 * N + j], dyg = c[5 * N + j];
    for (int q = 0; q < 4; ++q) {
      double m0 = mu[(size_t)q * V + r], mx = mu[(size_t)(4 + q) * V + r];
      double my = mu[(size_t)(8 + q) * V + r];
      Fb[q] -= d0f * m0 + dxf * mx + dyf * my;
      Gb[q] -= d0g * m0 + dxg * mx + dyg * my;
    }
    if (cvis) {
      const double* z = cvis + 6 * (size_t)n0;
      double e0f = z[j], e0g = z[N + j], exf = z[2 * N + j], exg = z[3 * N + j];
      double eyf = z[4 * N + j], eyg = z[5 * N + j];
      for (int q = 0; q < 4; ++q) {
        double m0 = mu[(size_t)q * V + r], mx = mu[(size_t)(4 + q) * V + r];
        double my = mu[(size_t)(8 + q) * V + r];
        Fvb[q] += e0f * m0 + exf * mx + eyf * my;
        Gvb[q] += e0g * m0 + exg * mx + eyg * my;
      }
    }
  }
  double w[12], g[12];
  for (int r = 0; r < 12; ++r) w[r] = Us[(size_t)r * V + u];
  for (int r = 0; r < 12; ++r) g[r] = 0.0;
  adj::euler_flux_vjp(w, ph.gamma - 1.0, Fb, Gb, g);
  if (cvis) adj::viscous_flux_vjp(w, ph.gamma - 1.0, ph.mu, ph.kappa, ph.R_gas, Fvb, Gvb, g);
  for (int t = ts_ptr[u]; t < ts_ptr[u + 1]; ++t) {
    int ent = ts_ent[t];
    const double* ge = Ge + (size_t)(ent / 6) * 72 + 12 * (ent % 6);
    for (int r = 0; r < 12; ++r) g[r] += ge[r];
  }
  for (int r = 0; r < 12; ++r) {
    size_t i = (size_t)r * V + u;
    double o = cg * g[r];
    if (X) o += cx * X[i];
    if (Y) o += cy * Y[i];
    if (Z) o += cz * Z[i];
    out[i] = o;
  }
}

// Transpose of the transmissive ghost refresh, in place (see the header comment): one thread
// per donor adds its ghosts' columns, in ascending ghost order, and zeroes them.  Donors are
// non-ghost vertices, so no column is both read as a ghost and written as a donor.
__global__ void __launch_bounds__(128) k_adj_ghost_T(int nd, int V, const int32_t* __restrict__ donor,
                                                     const int32_t* __restrict__ ptr,
                                                     const int32_t* __restrict__ ghost,
                                                     const int32_t* __restrict__ flags,
                                                     double* lam) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  const int dn = donor[i];
  double acc[12];
  for (int r = 0; r < 12; ++r) acc[r] = lam[(size_t)r * V + dn];
  for (int t = ptr[i]; t < ptr[i + 1]; ++t) {
    const int g = ghost[t], f = flags[t];
    for (int r = 0; r < 12; ++r) {
      const size_t k = (size_t)r * V + g;
      const bool zeroed = (r >= 4 && r < 8 && (f & 1)) || (r >= 8 && (f & 2));
      if (!zeroed) acc[r] += lam[k];
      lam[k] = 0.0;
    }
  }
  for (int r = 0; r < 12; ++r) lam[(size_t)r * V + dn] = acc[r];
}

}  // namespace hfd

// ------------------------------------------------------------------ host side
using hfd::set_error;

#define ACK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      set_error("hfd_adjoint: %s: %s", #call, cudaGetErrorString(e_));                     \
      return HFD_ERR_CUDA;                                                                 \
    }                                                                                      \
  } while (0)

namespace {

template <typename T>
hfd_status upload_vec(hfd_mesh* m, T** dst, const std::vector<T>& v) {
  void* p = nullptr;
  size_t bytes = std::max<size_t>(v.size() * sizeof(T), 16);
  ACK(mesh_malloc(m, &p, bytes));
  if (!v.empty()) ACK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *dst = static_cast<T*>(p);
  return HFD_OK;
}

template <typename T>
std::vector<T> download(const T* d, size_t n) {
  std::vector<T> h(n);
  if (n) cudaMemcpy(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost);
  return h;
}

// transposed lists: for every vertex / edge, the (row, position) pairs of the divergence rows
// that read it, and for every vertex the (edge, node) pairs of the stencils it belongs to; in
// ascending order, so the gathers sum in a fixed order
hfd_status build_transposes(hfd_mesh* m) {
  hfd::DevMesh& d = m->dm;
  const int V = d.V, A = d.A, Ef = d.Ef;
  auto vptr = download(d.vptr, A + 1), eptr = download(d.eptr, A + 1);
  auto vidx = download(d.vidx, vptr[A]), eidx = download(d.eidx, eptr[A]);
  auto sten = download(d.sten, (size_t)6 * Ef);
  std::vector<int32_t> tvp(V + 1, 0), tep(Ef + 1, 0), tsp(V + 1, 0);
  for (int32_t u : vidx) tvp[u + 1]++;
  for (int32_t e : eidx) tep[e + 1]++;
  for (int32_t u : sten) tsp[u + 1]++;
  for (int i = 0; i < V; ++i) { tvp[i + 1] += tvp[i]; tsp[i + 1] += tsp[i]; }
  for (int i = 0; i < Ef; ++i) tep[i + 1] += tep[i];
  std::vector<int32_t> tvr(vptr[A]), tvq(vptr[A]), ter(eptr[A]), teq(eptr[A]), tse(6 * (size_t)Ef);
  std::vector<int32_t> fv(tvp.begin(), tvp.end() - 1), fe(tep.begin(), tep.end() - 1),
      fs(tsp.begin(), tsp.end() - 1);
  for (int r = 0; r < A; ++r) {
    for (int j = vptr[r]; j < vptr[r + 1]; ++j) {
      int u = vidx[j];
      tvr[fv[u]] = r;
      tvq[fv[u]++] = j - vptr[r];
    }
    for (int j = eptr[r]; j < eptr[r + 1]; ++j) {
      int e = eidx[j];
      ter[fe[e]] = r;
      teq[fe[e]++] = j - eptr[r];
    }
  }
  for (int e = 0; e < Ef; ++e)
    for (int k = 0; k < 6; ++k) {
      int u = sten[(size_t)k * Ef + e];
      tse[fs[u]++] = e * 6 + k;
    }
  hfd_status st;
  if ((st = upload_vec(m, &m->adj_tv_ptr, tvp)) != HFD_OK) return st;
  if ((st = upload_vec(m, &m->adj_tv_row, tvr)) != HFD_OK) return st;
  if ((st = upload_vec(m, &m->adj_tv_pos, tvq)) != HFD_OK) return st;
  if ((st = upload_vec(m, &m->adj_te_ptr, tep)) != HFD_OK) return st;
  if ((st = upload_vec(m, &m->adj_te_row, ter)) != HFD_OK) return st;
  if ((st = upload_vec(m, &m->adj_te_pos, teq)) != HFD_OK) return st;
  if ((st = upload_vec(m, &m->adj_ts_ptr, tsp)) != HFD_OK) return st;
  if ((st = upload_vec(m, &m->adj_ts_ent, tse)) != HFD_OK) return st;
  std::vector<double> zeros;
  zeros.resize((size_t)72 * Ef);
  if ((st = upload_vec(m, &m->adj_Ge, zeros)) != HFD_OK) return st;
  zeros.assign((size_t)12 * V, 0.0);
  if ((st = upload_vec(m, &m->adj_B1, zeros)) != HFD_OK) return st;
  std::vector<int32_t> izeros((size_t)Ef + 1, 0);
  if ((st = upload_vec(m, &m->adj_list, izeros)) != HFD_OK) return st;
  izeros.assign(1, 0);
  if ((st = upload_vec(m, &m->adj_count, izeros)) != HFD_OK) return st;
  if ((st = upload_vec(m, &m->adj_B2, zeros)) != HFD_OK) return st;
  if (d.G > 0) {
    // donors of the transmissive ghosts, each with its ghosts in ascending internal order
    auto gid = download(d.gid, d.G), gdn = download(d.gdonor, d.G), gfl = download(d.gflags, d.G);
    std::vector<int> order;
    for (int g = 0; g < d.G; ++g)
      if (gdn[g] >= 0) order.push_back(g);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      return gdn[a] != gdn[b] ? gdn[a] < gdn[b] : gid[a] < gid[b];
    });
    std::vector<int32_t> dlist, dptr(1, 0), glist, flist;
    for (size_t i = 0; i < order.size(); ++i) {
      int g = order[i];
      if (dlist.empty() || dlist.back() != gdn[g]) {
        if (!dlist.empty()) dptr.push_back((int32_t)glist.size());
        dlist.push_back(gdn[g]);
      }
      glist.push_back(gid[g]);
      flist.push_back(gfl[g]);
    }
    if (!dlist.empty()) dptr.push_back((int32_t)glist.size());
    m->adj_ndonor = (int32_t)dlist.size();
    if ((st = upload_vec(m, &m->adj_gt_donor, dlist)) != HFD_OK) return st;
    if ((st = upload_vec(m, &m->adj_gt_ptr, dptr)) != HFD_OK) return st;
    if ((st = upload_vec(m, &m->adj_gt_ghost, glist)) != HFD_OK) return st;
    if ((st = upload_vec(m, &m->adj_gt_flags, flist)) != HFD_OK) return st;
    if ((st = upload_vec(m, &m->adj_U0, zeros)) != HFD_OK) return st;
    if ((st = upload_vec(m, &m->adj_L, zeros)) != HFD_OK) return st;
  }
  return HFD_OK;
}

hfd_status ghost_transpose(hfd_mesh* m, double* lam, cudaStream_t s) {
  if (m->adj_ndonor == 0) return HFD_OK;
  hfd::k_adj_ghost_T<<<(m->adj_ndonor + 127) / 128, 128, 0, s>>>(
      m->adj_ndonor, m->dm.V, m->adj_gt_donor, m->adj_gt_ptr, m->adj_gt_ghost, m->adj_gt_flags, lam);
  ACK(cudaGetLastError());
  return HFD_OK;
}

// out = cx X + cy Y + cz Z + cg (dR/dU at Us)^T mu
hfd_status residual_vjp(hfd_mesh* m, const double* Us, const double* mu, double* out, double cx,
                        const double* X, double cy, const double* Y, double cz, const double* Z,
                        double cg, cudaStream_t s) {
  const hfd::DevMesh& d = m->dm;
  ACK(hfd::launch_vertex(d, Us, m->ph, s));          // AoS copy of the stage state
  // edges with both sides on the 5-node branch, then the listed remainder
  ACK(cudaMemsetAsync(m->adj_count, 0, sizeof(int32_t), s));
  hfd::k_adj_edge<<<(d.Ef + 127) / 128, 128, 0, s>>>(
      d.Ef, d.V, d.sten, (const double*)d.nrm, (const double*)d.w5, (const double*)d.w3,
      (const double*)d.Ua, d.eptr, (const double*)d.ce, m->adj_te_ptr, m->adj_te_row,
      m->adj_te_pos, mu, m->adj_Ge, m->ph, m->adj_list, m->adj_count);
  ACK(cudaGetLastError());
  hfd::k_adj_edge_full<<<(d.Ef + 127) / 128, 128, 0, s>>>(
      d.Ef, d.V, d.sten, (const double*)d.nrm, (const double*)d.w5, (const double*)d.w3,
      (const double*)d.Ua, d.eptr, (const double*)d.ce, m->adj_te_ptr, m->adj_te_row,
      m->adj_te_pos, mu, m->adj_Ge, m->ph, m->adj_list, m->adj_count);
  ACK(cudaGetLastError());
  hfd::k_adj_vertex<<<(d.V + 127) / 128, 128, 0, s>>>(
      d.V, Us, d.vptr, (const double*)d.cv, d.viscous ? (const double*)d.cvis : nullptr,
      m->adj_tv_ptr, m->adj_tv_row, m->adj_tv_pos,
      m->adj_ts_ptr, m->adj_ts_ent, mu, m->adj_Ge, out, cx, X, cy, Y, cz, Z, cg, m->ph);
  ACK(cudaGetLastError());
  // X, Y, Z are transposed already (zero transmissive ghost columns), so T(out) = cx X + cy Y +
  // cz Z + cg T((dR/dU)^T mu)
  return ghost_transpose(m, out, s);
}

}  // namespace

extern "C" hfd_status hfd_adjoint(hfd_mesh* m, const double* U_n, const double* lam_np1,
                                  double* lam_n, double dt, void* stream) {
  if (!m || !U_n || !lam_np1 || !lam_n || !(dt > 0.0) || lam_n == lam_np1) {
    set_error("hfd_adjoint: invalid argument (dt must be positive, lam_n distinct from lam_np1)");
    return HFD_ERR_ARG;
  }
  hfd::NvtxRange range("hfd_adjoint");
  const hfd::DevMesh& d = m->dm;
  if (d.precision != 0 || m->ph.force_branch != 0) {
    set_error("hfd_adjoint: built for FP64 meshes whose sensor decides the branch");
    return HFD_ERR_UNSUPPORTED;
  }
  if (!m->adj_Ge) {
    hfd_status st = build_transposes(m);
    if (st != HFD_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)12 * d.V * sizeof(double);
  double* U = const_cast<double*>(U_n);               // read only when there are no ghosts
  const double* lam = lam_np1;
  if (d.G) {
    // the caller's arrays stay untouched: the step input with refreshed ghosts, and T lam
    ACK(cudaMemcpyAsync(m->adj_U0, U_n, bytes, cudaMemcpyDeviceToDevice, s));
    ACK(hfd::launch_ghost(d, m->adj_U0, m->adj_U0, s));
    U = m->adj_U0;
    ACK(cudaMemcpyAsync(m->adj_L, lam_np1, bytes, cudaMemcpyDeviceToDevice, s));
    hfd_status st = ghost_transpose(m, m->adj_L, s);
    if (st != HFD_OK) return st;
    lam = m->adj_L;
  }
  double *u1 = m->U1, *u2 = m->U2, *B1 = m->adj_B1, *B2 = m->adj_B2;
  // forward: the first two stage states, each with its ghosts refreshed as the next stage
  // of the step refreshes them (fixed ghosts from the step input)
  ACK(hfd::launch_vertex(d, U, m->ph, s));
  ACK(hfd::launch_edge(d, m->ph, s));
  ACK(hfd::launch_div(d, U, U, u1, hfd::DIV_STAGE, 0.0, 1.0, dt, m->ph, m->lanes, s));
  if (d.G) ACK(hfd::launch_ghost(d, u1, U, s));
  ACK(hfd::launch_vertex(d, u1, m->ph, s));
  ACK(hfd::launch_edge(d, m->ph, s));
  ACK(hfd::launch_div(d, u1, U, u2, hfd::DIV_STAGE, 0.75, 0.25, dt, m->ph, m->lanes, s));
  if (d.G) ACK(hfd::launch_ghost(d, u2, U, s));
  // reverse: lambda_u2 = 2/3 (lam + dt J(u2)^T lam)
  hfd_status st = residual_vjp(m, u2, lam, B2, 2.0 / 3.0, lam, 0, nullptr, 0, nullptr,
                               2.0 / 3.0 * dt, s);
  if (st != HFD_OK) return st;
  // lambda_u1 = 1/4 (lambda_u2 + dt J(u1)^T lambda_u2)
  st = residual_vjp(m, u1, B2, B1, 0.25, B2, 0, nullptr, 0, nullptr, 0.25 * dt, s);
  if (st != HFD_OK) return st;
  // lambda_n = 1/3 lam + 3/4 lambda_u2 + lambda_u1 + dt J(u)^T lambda_u1
  return residual_vjp(m, U, B1, lam_n, 1.0, B1, 1.0 / 3.0, lam, 0.75, B2, dt, s);
}
