// GPU kernels of one right-hand-side evaluation of the Hermite finite-difference method
// (arXiv 2109.01286) for sm_103a, and the SSP-RK3 stage update fused into the divergence.
//
//   k_vertex : analytic Euler (and viscous) fluxes at every vertex (Sec. 2.3) plus an AoS copy
//              of the state for the edge gathers.
//   k_edge   : Alg. 1 on both sides of every flux edge -- Roe average of the end states,
//              characteristic projection of the 6 stencil nodes, uniform-WENO5 sensor,
//              5-node Hermite value or omega-weighted 3-node values (Eq. (2d_hweno_intp)),
//              back-projection -- then the Riemann (Roe) flux along the edge.
//   k_div    : least-squares divergence rows d_0, d_x, d_y (Eq. (flux_polynomials)) as a CSR
//              gather over stencil vertices and edges by a group of lanes per vertex with a
//              fixed shuffle reduction (deterministic, no atomics), fused with the
//              Runge-Kutta stage combination (Sec. 2.3, end).
//
// No step is a dense contraction, so no tensor-core path exists: the kernels are bound by
// FP64 issue (FP64 path) or by memory traffic (FP32-bulk path).  The bulk precision T is
// double or float; the state, the stage combination and the WENO weight ratios are double.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.hpp"

namespace hfd {

enum : unsigned { ERRBIT_NONFINITE = 1u, ERRBIT_POSITIVITY = 2u };

// ------------------------------------------------------------------ vector loads
__device__ __forceinline__ void ld12(const double* p, double* o) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int i = 0; i < 6; ++i) { double2 a = __ldg(q + i); o[2 * i] = a.x; o[2 * i + 1] = a.y; }
}
__device__ __forceinline__ void ld12(const float* p, float* o) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float4 a = __ldg(q + i);
    o[4 * i] = a.x; o[4 * i + 1] = a.y; o[4 * i + 2] = a.z; o[4 * i + 3] = a.w;
  }
}
__device__ __forceinline__ void ld8(const double* p, double* o) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int i = 0; i < 4; ++i) { double2 a = __ldg(q + i); o[2 * i] = a.x; o[2 * i + 1] = a.y; }
}
__device__ __forceinline__ void ld8(const float* p, float* o) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    float4 a = __ldg(q + i);
    o[4 * i] = a.x; o[4 * i + 1] = a.y; o[4 * i + 2] = a.z; o[4 * i + 3] = a.w;
  }
}
__device__ __forceinline__ void ld4(const double* p, double* o) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4(const float* p, float* o) {
  float4 a = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void st4(double* p, const double* v) {
  double2* q = reinterpret_cast<double2*>(p);
  q[0] = make_double2(v[0], v[1]);
  q[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// ------------------------------------------------------------------ physics (Sec. 2.3)
template <typename T>
__device__ __forceinline__ T pressure(const T* w, T g1) {
  return g1 * (w[3] - T(0.5) * (w[1] * w[1] + w[2] * w[2]) / w[0]);
}

// Roe-averaged u, v, H, c of two states (Alg. 1, first step; also the Riemann flux).
template <typename T>
__device__ __forceinline__ void roe_avg(const T* wl, const T* wr, T g1, T& u, T& v, T& H, T& c) {
  T rl = sqrt(wl[0]), rr = sqrt(wr[0]);
  T irl = T(1) / rl, irr = T(1) / rr, is = T(1) / (rl + rr);
  T pl = pressure(wl, g1), pr = pressure(wr, g1);
  u = (wl[1] * irl + wr[1] * irr) * is;
  v = (wl[2] * irl + wr[2] * irr) * is;
  H = ((wl[3] + pl) * irl + (wr[3] + pr) * irr) * is;
  c = sqrt(g1 * (H - T(0.5) * (u * u + v * v)));
}

// Left eigenvectors (rows of L = R^-1) of the Euler flux Jacobian along n (Alg. 1, step 2).
template <typename T>
__device__ __forceinline__ void left_ev(T u, T v, T c, T nx, T ny, T g1, T (*L)[4]) {
  T qn = u * nx + v * ny, qt = -u * ny + v * nx;
  T ic = T(1) / c;
  T b1 = g1 * ic * ic, b2 = T(0.5) * b1 * (u * u + v * v);
  L[0][0] = T(0.5) * (b2 + qn * ic);
  L[0][1] = T(-0.5) * (b1 * u + nx * ic);
  L[0][2] = T(-0.5) * (b1 * v + ny * ic);
  L[0][3] = T(0.5) * b1;
  L[1][0] = T(1) - b2;
  L[1][1] = b1 * u;
  L[1][2] = b1 * v;
  L[1][3] = -b1;
  L[2][0] = -qt;
  L[2][1] = -ny;
  L[2][2] = nx;
  L[2][3] = T(0);
  L[3][0] = T(0.5) * (b2 - qn * ic);
  L[3][1] = T(-0.5) * (b1 * u - nx * ic);
  L[3][2] = T(-0.5) * (b1 * v - ny * ic);
  L[3][3] = T(0.5) * b1;
}

// w = R C with the right eigenvectors as columns (Alg. 1, last step).
template <typename T>
__device__ __forceinline__ void right_apply(T u, T v, T H, T c, T nx, T ny, const T* C, T* w) {
  T qn = u * nx + v * ny, qt = -u * ny + v * nx;
  w[0] = C[0] + C[1] + C[3];
  w[1] = (u - c * nx) * C[0] + u * C[1] - ny * C[2] + (u + c * nx) * C[3];
  w[2] = (v - c * ny) * C[0] + v * C[1] + nx * C[2] + (v + c * ny) * C[3];
  w[3] = (H - c * qn) * C[0] + T(0.5) * (u * u + v * v) * C[1] + qt * C[2] + (H + c * qn) * C[3];
}

template <typename T>
__device__ __forceinline__ void normal_flux(const T* w, T nx, T ny, T g1, T* f) {
  T ir = T(1) / w[0];
  T un = (w[1] * nx + w[2] * ny) * ir;
  T p = pressure(w, g1);
  f[0] = w[0] * un;
  f[1] = w[1] * un + p * nx;
  f[2] = w[2] * un + p * ny;
  f[3] = (w[3] + p) * un;
}

// Roe's flux with Harten's entropy fix on all waves (Riemann flux, Sec. 2.3 after Alg. 1).
template <typename T>
__device__ __forceinline__ void roe_flux(const T* wl, const T* wr, T nx, T ny, T g1, T harten,
                                         T* hq) {
  T u, v, H, c;
  roe_avg(wl, wr, g1, u, v, H, c);
  T L[4][4];
  left_ev(u, v, c, nx, ny, g1, L);
  T d[4] = {wr[0] - wl[0], wr[1] - wl[1], wr[2] - wl[2], wr[3] - wl[3]};
  T qn = u * nx + v * ny;
  T lam[4] = {qn - c, qn, qn, qn + c};
  T del = harten * c;
  T k[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    T a = L[i][0] * d[0] + L[i][1] * d[1] + L[i][2] * d[2] + L[i][3] * d[3];
    T al = fabs(lam[i]);
    if (al < del) al = (lam[i] * lam[i] + del * del) / (T(2) * del);
    k[i] = al * a;
  }
  T diss[4];
  right_apply(u, v, H, c, nx, ny, k, diss);
  T fl[4], fr[4];
  normal_flux(wl, nx, ny, g1, fl);
  normal_flux(wr, nx, ny, g1, fr);
#pragma unroll
  for (int i = 0; i < 4; ++i) hq[i] = T(0.5) * (fl[i] + fr[i]) - T(0.5) * diss[i];
}

// Jiang-Shu smoothness indicators of the three sub-stencils of u0..u4 (uniform WENO5, R2).
template <typename T>
__device__ __forceinline__ void smoothness(T u0, T u1, T u2, T u3, T u4, T* b) {
  T a = u0 - T(2) * u1 + u2, e = u0 - T(4) * u1 + T(3) * u2;
  b[0] = T(13.0 / 12.0) * a * a + T(0.25) * e * e;
  a = u1 - T(2) * u2 + u3;
  e = u1 - u3;
  b[1] = T(13.0 / 12.0) * a * a + T(0.25) * e * e;
  a = u2 - T(2) * u3 + u4;
  e = T(3) * u2 - T(4) * u3 + u4;
  b[2] = T(13.0 / 12.0) * a * a + T(0.25) * e * e;
}

// ------------------------------------------------------------------ k_vertex
template <typename T, bool VISC>
__global__ void __launch_bounds__(256) k_vertex(int V, const double* __restrict__ U, T* Ua, T* FG,
                                                T* FGv, Phys ph) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  double w[12];
#pragma unroll
  for (int r = 0; r < 12; ++r) w[r] = U[(size_t)r * V + v];
  T* ua = Ua + (size_t)v * 12;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T t[4] = {T(w[4 * i]), T(w[4 * i + 1]), T(w[4 * i + 2]), T(w[4 * i + 3])};
    st4(ua + 4 * i, t);
  }
  T g1 = T(ph.gamma - 1.0);
  T q[4] = {T(w[0]), T(w[1]), T(w[2]), T(w[3])};
  T ir = T(1) / q[0];
  T u = q[1] * ir, vv = q[2] * ir;
  T p = pressure(q, g1);
  T F[4] = {q[1], q[1] * u + p, q[2] * u, (q[3] + p) * u};
  T Gf[4] = {q[2], q[1] * vv, q[2] * vv + p, (q[3] + p) * vv};
  st4(FG + (size_t)v * 8, F);
  st4(FG + (size_t)v * 8 + 4, Gf);
  if (VISC) {   // viscous flux from w, w_x, w_y (Sec. 2.3; chain rule for the primitives)
    double rho = w[0], uu = w[1] / rho, vw = w[2] / rho;
    double gm = ph.gamma - 1.0;
    double ux = (w[5] - uu * w[4]) / rho, vx = (w[6] - vw * w[4]) / rho;
    double uy = (w[9] - uu * w[8]) / rho, vy = (w[10] - vw * w[8]) / rho;
    double q2 = uu * uu + vw * vw;
    double pp = gm * (w[3] - 0.5 * rho * q2);
    double px = gm * (w[7] - 0.5 * w[4] * q2 - rho * (uu * ux + vw * vx));
    double py = gm * (w[11] - 0.5 * w[8] * q2 - rho * (uu * uy + vw * vy));
    double Tx = (px / rho - pp * w[4] / (rho * rho)) / ph.R_gas;
    double Ty = (py / rho - pp * w[8] / (rho * rho)) / ph.R_gas;
    double mu = ph.mu;
    double txx = mu * (4.0 / 3.0 * ux - 2.0 / 3.0 * vy);
    double tyy = mu * (4.0 / 3.0 * vy - 2.0 / 3.0 * ux);
    double txy = mu * (uy + vx);
    T Fv[4] = {T(0), T(txx), T(txy), T(uu * txx + vw * txy + ph.kappa * Tx)};
    T Gv[4] = {T(0), T(txy), T(tyy), T(uu * txy + vw * tyy + ph.kappa * Ty)};
    st4(FGv + (size_t)v * 8, Fv);
    st4(FGv + (size_t)v * 8 + 4, Gv);
  }
}

// ------------------------------------------------------------------ k_edge
// One thread per flux edge.  Node order of the stencil: [i-2, i-1, i, i+1, i+2, i+3]; the left
// state uses nodes 0..4, the right state nodes 1..5 with the WENO sub-stencils mirrored.
template <typename T>
__global__ void __launch_bounds__(128) k_edge(int Ef, const int32_t* __restrict__ sten,
                                              const T* __restrict__ nrm, const T* __restrict__ w5,
                                              const T* __restrict__ w3, const T* __restrict__ Ua,
                                              T* __restrict__ h, Phys ph, unsigned* err) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Ef) return;
  const T g1 = T(ph.gamma - 1.0);
  int s[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) s[k] = __ldg(sten + (size_t)k * Ef + e);
  T nx = __ldg(nrm + e), ny = __ldg(nrm + Ef + e);
  T wi[4], wj[4];
  {
    T a[12];
    ld12(Ua + (size_t)s[2] * 12, a);
    wi[0] = a[0]; wi[1] = a[1]; wi[2] = a[2]; wi[3] = a[3];
    ld12(Ua + (size_t)s[3] * 12, a);
    wj[0] = a[0]; wj[1] = a[1]; wj[2] = a[2]; wj[3] = a[3];
  }
  T u, v, H, c;
  roe_avg(wi, wj, g1, u, v, H, c);
  T L[4][4];
  left_ev(u, v, c, nx, ny, g1, L);
  // characteristic values of the 6 nodes and the 5-node Hermite sums of both sides
  T cv[6][4];
  T C5L[4] = {T(0), T(0), T(0), T(0)}, C5R[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    T a[12];
    ld12(Ua + (size_t)s[k] * 12, a);
    T wlv = T(0), wlx = T(0), wly = T(0), wrv = T(0), wrx = T(0), wry = T(0);
    if (k <= 4) {
      wlv = __ldg(w5 + (size_t)(3 * k) * Ef + e);
      wlx = __ldg(w5 + (size_t)(3 * k + 1) * Ef + e);
      wly = __ldg(w5 + (size_t)(3 * k + 2) * Ef + e);
    }
    if (k >= 1) {
      wrv = __ldg(w5 + (size_t)(15 + 3 * (k - 1)) * Ef + e);
      wrx = __ldg(w5 + (size_t)(16 + 3 * (k - 1)) * Ef + e);
      wry = __ldg(w5 + (size_t)(17 + 3 * (k - 1)) * Ef + e);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      T c0 = L[q][0] * a[0] + L[q][1] * a[1] + L[q][2] * a[2] + L[q][3] * a[3];
      T cx = L[q][0] * a[4] + L[q][1] * a[5] + L[q][2] * a[6] + L[q][3] * a[7];
      T cy = L[q][0] * a[8] + L[q][1] * a[9] + L[q][2] * a[10] + L[q][3] * a[11];
      cv[k][q] = c0;
      if (k <= 4) C5L[q] += wlv * c0 + wlx * cx + wly * cy;
      if (k >= 1) C5R[q] += wrv * c0 + wrx * cx + wry * cy;
    }
  }
  T wside[2][4];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    T C[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      T u0, u1, u2, u3, u4;
      if (side == 0) { u0 = cv[0][q]; u1 = cv[1][q]; u2 = cv[2][q]; u3 = cv[3][q]; u4 = cv[4][q]; }
      else           { u0 = cv[5][q]; u1 = cv[4][q]; u2 = cv[3][q]; u3 = cv[2][q]; u4 = cv[1][q]; }
      T b[3];
      smoothness(u0, u1, u2, u3, u4, b);
      // omega_j = (d_j / s_j^2) / sum, s_j = eps + beta_j; with t_j = d_j prod_{k != j} s_k^2
      // the sensor test 0.01 < omega_1 < 0.79 needs no division (FP64, R20)
      double s0 = ph.eps + (double)b[0], s1 = ph.eps + (double)b[1], s2 = ph.eps + (double)b[2];
      s0 *= s0; s1 *= s1; s2 *= s2;
      double t0 = (1.0 / 16.0) * s1 * s2, t1 = (10.0 / 16.0) * s0 * s2, t2 = (5.0 / 16.0) * s0 * s1;
      double S = t0 + t1 + t2;
      bool smooth = (t0 > ph.sens_lo * S) && (t0 < ph.sens_hi * S);
      if (smooth) {
        C[q] = side == 0 ? C5L[q] : C5R[q];
      } else {
        const T* w = w3 + (size_t)(9 * side) * Ef + e;
        T c1 = __ldg(w) * u0 + __ldg(w + Ef) * u1 + __ldg(w + 2 * (size_t)Ef) * u2;
        T c2 = __ldg(w + 3 * (size_t)Ef) * u1 + __ldg(w + 4 * (size_t)Ef) * u2 +
               __ldg(w + 5 * (size_t)Ef) * u3;
        T c3 = __ldg(w + 6 * (size_t)Ef) * u2 + __ldg(w + 7 * (size_t)Ef) * u3 +
               __ldg(w + 8 * (size_t)Ef) * u4;
        double iS = 1.0 / S;
        C[q] = T((t0 * (double)c1 + t1 * (double)c2 + t2 * (double)c3) * iS);
      }
    }
    right_apply(u, v, H, c, nx, ny, C, wside[side]);
  }
  // positivity (R16): fall back to the end state of that side
  if (!(wside[0][0] > T(0)) || !(pressure(wside[0], g1) > T(0)))
#pragma unroll
    for (int q = 0; q < 4; ++q) wside[0][q] = wi[q];
  if (!(wside[1][0] > T(0)) || !(pressure(wside[1], g1) > T(0)))
#pragma unroll
    for (int q = 0; q < 4; ++q) wside[1][q] = wj[q];
  T hq[4];
  roe_flux(wside[0], wside[1], nx, ny, g1, T(ph.harten), hq);
  st4(h + (size_t)e * 4, hq);
}

// ------------------------------------------------------------------ k_div
// G lanes per active vertex; lanes stride over the CSR entries; fixed xor-butterfly
// reduction.  acc = div(f) - div(f_vis) for the 12 rows; R = -acc.
template <typename T, int G, bool VISC>
__global__ void __launch_bounds__(256) k_div(int A, int V, const int32_t* __restrict__ vptr,
                                             const int32_t* __restrict__ vidx,
                                             const int32_t* __restrict__ eptr,
                                             const int32_t* __restrict__ eidx,
                                             const T* __restrict__ cv, const T* __restrict__ ce,
                                             const T* __restrict__ cvis, const T* __restrict__ FG,
                                             const T* __restrict__ FGv, const T* __restrict__ h,
                                             const double* __restrict__ Us,
                                             const double* __restrict__ Un, double* out, int mode,
                                             double a, double b, double dt_fixed,
                                             const unsigned long long* dtbits, double cfl,
                                             double* dt_last, unsigned* err) {
  int gt = blockIdx.x * blockDim.x + threadIdx.x;
  int r = gt / G, lane = gt % G;
  bool live = r < A;
  T acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = T(0);
  if (live) {
    int n0 = __ldg(vptr + r), N = __ldg(vptr + r + 1) - n0;
    const T* c = cv + 6 * (size_t)n0;
    const T* cz = VISC ? cvis + 6 * (size_t)n0 : nullptr;
    for (int j = lane; j < N; j += G) {
      int uu = __ldg(vidx + n0 + j);
      T f[8];
      ld8(FG + (size_t)uu * 8, f);
      T c0f = __ldg(c + j), c0g = __ldg(c + N + j), cxf = __ldg(c + 2 * N + j);
      T cxg = __ldg(c + 3 * N + j), cyf = __ldg(c + 4 * N + j), cyg = __ldg(c + 5 * N + j);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] += c0f * f[q] + c0g * f[4 + q];
        acc[4 + q] += cxf * f[q] + cxg * f[4 + q];
        acc[8 + q] += cyf * f[q] + cyg * f[4 + q];
      }
      if (VISC) {
        ld8(FGv + (size_t)uu * 8, f);
        c0f = __ldg(cz + j); c0g = __ldg(cz + N + j); cxf = __ldg(cz + 2 * N + j);
        cxg = __ldg(cz + 3 * N + j); cyf = __ldg(cz + 4 * N + j); cyg = __ldg(cz + 5 * N + j);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q] -= c0f * f[q] + c0g * f[4 + q];
          acc[4 + q] -= cxf * f[q] + cxg * f[4 + q];
          acc[8 + q] -= cyf * f[q] + cyg * f[4 + q];
        }
      }
    }
    int m0 = __ldg(eptr + r), M = __ldg(eptr + r + 1) - m0;
    const T* d = ce + 3 * (size_t)m0;
    for (int j = lane; j < M; j += G) {
      int e = __ldg(eidx + m0 + j);
      T hv[4];
      ld4(h + (size_t)e * 4, hv);
      T d0 = __ldg(d + j), dx = __ldg(d + M + j), dy = __ldg(d + 2 * M + j);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] += d0 * hv[q];
        acc[4 + q] += dx * hv[q];
        acc[8 + q] += dy * hv[q];
      }
    }
  }
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off, G);
  if (!live) return;
  double dt = dt_fixed > 0.0 ? dt_fixed : cfl * __longlong_as_double((long long)*dtbits);
  if (mode == DIV_STAGE && gt == 0 && dt_last) *dt_last = dt;
  unsigned bad = 0;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    if (k % G != lane) continue;
    double R = -(double)acc[k];
    size_t i = (size_t)k * V + r;
    double o;
    if (mode == DIV_RESIDUAL) {
      o = R;
    } else {
      o = b * (Us[i] + dt * R);
      if (a != 0.0) o += a * Un[i];   // the first stage does not read the base state
    }
    out[i] = o;
    if (!isfinite(o)) bad |= ERRBIT_NONFINITE;
    if (mode == DIV_STAGE && k == 0 && !(o > 0.0)) bad |= ERRBIT_POSITIVITY;
  }
  if (bad) atomicOr(err, bad);
}

// ------------------------------------------------------------------ small kernels
__global__ void k_ghost(int Gn, int V, const int32_t* gid, const int32_t* gdonor,
                        const int32_t* gflags, double* U) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Gn) return;
  int t = gid[g], d = gdonor[g], f = gflags[g];
#pragma unroll
  for (int r = 0; r < 12; ++r) {
    double val = U[(size_t)r * V + d];
    if ((r >= 4 && r < 8 && (f & 1)) || (r >= 8 && (f & 2))) val = 0.0;
    U[(size_t)r * V + t] = val;
  }
}

// min over active vertices of l_min / (|u| + c) (R12), reduced by warp shuffles and an
// atomicMin on the bit pattern (positive doubles order like their bits): order-independent.
__global__ void k_dtmin(int A, int V, const double* __restrict__ U, const double* __restrict__ lmin,
                        double gamma, unsigned long long* bits) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  double val = INFINITY;
  if (v < A) {
    double rho = U[v], m = U[(size_t)V + v], n = U[2 * (size_t)V + v], E = U[3 * (size_t)V + v];
    double uu = m / rho, vv = n / rho;
    double p = (gamma - 1.0) * (E - 0.5 * rho * (uu * uu + vv * vv));
    double s = sqrt(uu * uu + vv * vv) + sqrt(gamma * p / rho);
    val = lmin[v] / s;
    if (!(val > 0.0)) val = INFINITY;   // non-physical states do not set the step
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) val = fmin(val, __shfl_xor_sync(0xffffffffu, val, off));
  if ((threadIdx.x & 31) == 0 && val < INFINITY)
    atomicMin(bits, (unsigned long long)__double_as_longlong(val));
}

__global__ void k_permute(int V, const int32_t* __restrict__ perm, const double* __restrict__ src,
                          double* __restrict__ dst, int gather) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  int p = perm[i];
#pragma unroll
  for (int r = 0; r < 12; ++r) {
    if (gather) dst[(size_t)r * V + i] = src[(size_t)r * V + p];
    else dst[(size_t)r * V + p] = src[(size_t)r * V + i];
  }
}

// ------------------------------------------------------------------ launchers
static inline int blocks(long long n, int b) { return (int)((n + b - 1) / b); }

cudaError_t launch_ghost(const DevMesh& m, double* U, cudaStream_t s) {
  if (m.G == 0) return cudaSuccess;
  k_ghost<<<blocks(m.G, 256), 256, 0, s>>>(m.G, m.V, m.gid, m.gdonor, m.gflags, U);
  return cudaGetLastError();
}

cudaError_t launch_vertex(const DevMesh& m, const double* U, const Phys& ph, cudaStream_t s) {
  int nb = blocks(m.V, 256);
  if (m.precision == 0) {
    if (m.viscous)
      k_vertex<double, true><<<nb, 256, 0, s>>>(m.V, U, (double*)m.Ua, (double*)m.FG,
                                                (double*)m.FGv, ph);
    else
      k_vertex<double, false><<<nb, 256, 0, s>>>(m.V, U, (double*)m.Ua, (double*)m.FG, nullptr, ph);
  } else {
    if (m.viscous)
      k_vertex<float, true><<<nb, 256, 0, s>>>(m.V, U, (float*)m.Ua, (float*)m.FG, (float*)m.FGv, ph);
    else
      k_vertex<float, false><<<nb, 256, 0, s>>>(m.V, U, (float*)m.Ua, (float*)m.FG, nullptr, ph);
  }
  return cudaGetLastError();
}

cudaError_t launch_edge(const DevMesh& m, const Phys& ph, cudaStream_t s) {
  if (m.Ef == 0) return cudaSuccess;
  int nb = blocks(m.Ef, 128);
  if (m.precision == 0)
    k_edge<double><<<nb, 128, 0, s>>>(m.Ef, m.sten, (const double*)m.nrm, (const double*)m.w5,
                                      (const double*)m.w3, (const double*)m.Ua, (double*)m.h, ph,
                                      m.err);
  else
    k_edge<float><<<nb, 128, 0, s>>>(m.Ef, m.sten, (const float*)m.nrm, (const float*)m.w5,
                                     (const float*)m.w3, (const float*)m.Ua, (float*)m.h, ph, m.err);
  return cudaGetLastError();
}

template <typename T, int G>
static void div_dispatch(const DevMesh& m, const double* Us, const double* Un, double* out,
                         int mode, double a, double b, double dt_fixed, const Phys& ph,
                         cudaStream_t s) {
  long long threads = (long long)m.A * G;
  int nb = blocks(threads, 256);
  if (m.viscous)
    k_div<T, G, true><<<nb, 256, 0, s>>>(m.A, m.V, m.vptr, m.vidx, m.eptr, m.eidx, (const T*)m.cv,
                                         (const T*)m.ce, (const T*)m.cvis, (const T*)m.FG,
                                         (const T*)m.FGv, (const T*)m.h, Us, Un, out, mode, a, b,
                                         dt_fixed, m.dtbits, ph.cfl, m.dt_last, m.err);
  else
    k_div<T, G, false><<<nb, 256, 0, s>>>(m.A, m.V, m.vptr, m.vidx, m.eptr, m.eidx,
                                          (const T*)m.cv, (const T*)m.ce, nullptr, (const T*)m.FG,
                                          nullptr, (const T*)m.h, Us, Un, out, mode, a, b, dt_fixed,
                                          m.dtbits, ph.cfl, m.dt_last, m.err);
}

cudaError_t launch_div(const DevMesh& m, const double* Us, const double* Un, double* out, int mode,
                       double a, double b, double dt_fixed, const Phys& ph, int lanes,
                       cudaStream_t s) {
  if (m.A == 0) return cudaSuccess;
  if (m.precision == 0) {
    switch (lanes) {
      case 4: div_dispatch<double, 4>(m, Us, Un, out, mode, a, b, dt_fixed, ph, s); break;
      case 16: div_dispatch<double, 16>(m, Us, Un, out, mode, a, b, dt_fixed, ph, s); break;
      default: div_dispatch<double, 8>(m, Us, Un, out, mode, a, b, dt_fixed, ph, s); break;
    }
  } else {
    switch (lanes) {
      case 4: div_dispatch<float, 4>(m, Us, Un, out, mode, a, b, dt_fixed, ph, s); break;
      case 16: div_dispatch<float, 16>(m, Us, Un, out, mode, a, b, dt_fixed, ph, s); break;
      default: div_dispatch<float, 8>(m, Us, Un, out, mode, a, b, dt_fixed, ph, s); break;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_dtmin(const DevMesh& m, const double* U, const Phys& ph, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(m.dtbits, 0xff, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (m.A == 0) return cudaSuccess;
  k_dtmin<<<blocks(m.A, 256), 256, 0, s>>>(m.A, m.V, U, m.lmin, ph.gamma, m.dtbits);
  return cudaGetLastError();
}

cudaError_t launch_permute(int V, const int32_t* perm, const double* src, double* dst, bool gather,
                           cudaStream_t s) {
  k_permute<<<blocks(V, 256), 256, 0, s>>>(V, perm, src, dst, gather ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace hfd
