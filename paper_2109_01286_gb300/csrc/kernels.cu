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

#include <algorithm>
#include <cstdint>

#include <type_traits>

#include "kernels.hpp"
#include "fp_convert.cuh"

namespace hfd {

enum : unsigned { ERRBIT_NONFINITE = 1u, ERRBIT_POSITIVITY = 2u, ERRBIT_TIMEOUT = 4u, ERRBIT_INDEX = 8u };

// Bounds-checked build (compiled with -DHFD_CHECK=1, the stand-in for a memory checker): every
// gathered index is tested against its array's extent; one outside [0, n) records ERRBIT_INDEX
// in the mesh's error word and is replaced by 0, so that the access stays in bounds (the result
// is then wrong, and hfd_check reports it).  In the normal build this is the identity.
#ifndef HFD_CHECK
#define HFD_CHECK 0
#endif
__device__ __forceinline__ int chk_idx(int i, int n, unsigned* err) {
#if HFD_CHECK
  if ((unsigned)i >= (unsigned)n) {
    atomicOr(err, ERRBIT_INDEX);
    return 0;
  }
#endif
  return i;
}

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

// Loads of the coefficient, weight and index streams: each element is read once per stage, in
// address order within a vertex's block (divergence) or across a warp's edges (edge weights).
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldg(p); }

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

// Reciprocal square roots: the CUDA math library's rsqrt (FP64: at most 1 ulp) and the FP32
// hardware approximation.
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

// Roe's flux with Harten's entropy fix on all waves (Riemann flux, Sec. 2.3 after Alg. 1).
// The primitive quantities of each side (1/rho, u, v, p, H) are formed once and shared by the
// Roe average and the two normal fluxes.  One reciprocal square root per side gives sqrt(rho)
// and 1/rho, one more gives c and 1/c; the entropy fix multiplies by 1/(2 delta) =
// half_inv_harten / c with half_inv_harten = 1/(2 harten).
template <typename T>
__device__ __forceinline__ void roe_flux(const T* wl, const T* wr, T nx, T ny, T g1, T harten,
                                         T half_inv_harten, T* hq) {
  T sl = rsqrt_t(wl[0]), sr = rsqrt_t(wr[0]);
  T irl = sl * sl, irr = sr * sr;
  T rl = wl[0] * sl, rr = wr[0] * sr;
  T ul = wl[1] * irl, vl = wl[2] * irl, ur = wr[1] * irr, vr = wr[2] * irr;
  T pl = g1 * (wl[3] - T(0.5) * (wl[1] * ul + wl[2] * vl));
  T pr = g1 * (wr[3] - T(0.5) * (wr[1] * ur + wr[2] * vr));
  T Hl = (wl[3] + pl) * irl, Hr = (wr[3] + pr) * irr;
  T fl_ = rl / (rl + rr), fr_ = T(1) - fl_;
  T u = fl_ * ul + fr_ * ur, v = fl_ * vl + fr_ * vr, H = fl_ * Hl + fr_ * Hr;
  T c2 = g1 * (H - T(0.5) * (u * u + v * v));
  T ic = rsqrt_t(c2), c = c2 * ic;
  T qn = u * nx + v * ny;
  // wave strengths L (w_r - w_l) from the primitive jumps: by the Roe property of the averages
  // they equal the left-eigenvector products (Roe's own form of the solver)
  T rho = rl * rr, dp = pr - pl, drho = wr[0] - wl[0];
  T dun = (ur - ul) * nx + (vr - vl) * ny, dut = (vr - vl) * nx - (ur - ul) * ny;
  // the strengths carry the factor 1/2 of the flux formula h = (f_l + f_r)/2 - R |Lambda| a / 2
  T ic2 = ic * ic, hc2 = T(0.5) * ic2, qc2 = T(0.25) * ic2;
  T rcd = rho * c * dun;
  T a[4] = {(dp - rcd) * qc2, T(0.5) * drho - dp * hc2, (T(0.5) * rho) * dut, (dp + rcd) * qc2};
  T lam[4] = {qn - c, qn, qn, qn + c};
  T del = harten * c, i2del = half_inv_harten * ic;
  T k[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    T al = fabs(lam[i]);
    if (al < del) al = (lam[i] * lam[i] + del * del) * i2del;
    k[i] = al * a[i];
  }
  T diss[4];
  right_apply(u, v, H, c, nx, ny, k, diss);
  T unl = ul * nx + vl * ny, unr = ur * nx + vr * ny;
  T fl[4] = {wl[0] * unl, wl[1] * unl + pl * nx, wl[2] * unl + pl * ny, (wl[3] + pl) * unl};
  T fr[4] = {wr[0] * unr, wr[1] * unr + pr * nx, wr[2] * unr + pr * ny, (wr[3] + pr) * unr};
#pragma unroll
  for (int i = 0; i < 4; ++i) hq[i] = T(0.5) * (fl[i] + fr[i]) - diss[i];
}

// Rusanov's (local Lax-Friedrichs) flux along n: the mean of the two normal fluxes minus half
// the larger of |u_n| + c over the two states times the jump (the alternative solver).
template <typename T>
__device__ __forceinline__ void rusanov_flux(const T* wl, const T* wr, T nx, T ny, T g1, T* hq) {
  T irl = T(1) / wl[0], irr = T(1) / wr[0];
  T unl = (wl[1] * nx + wl[2] * ny) * irl, unr = (wr[1] * nx + wr[2] * ny) * irr;
  T pl = g1 * (wl[3] - T(0.5) * (wl[1] * wl[1] + wl[2] * wl[2]) * irl);
  T pr = g1 * (wr[3] - T(0.5) * (wr[1] * wr[1] + wr[2] * wr[2]) * irr);
  T gam = g1 + T(1);
  T sl = fabs(unl) + sqrt(gam * pl * irl), sr = fabs(unr) + sqrt(gam * pr * irr);
  T s = sl >= sr ? sl : sr;
  T fl[4] = {wl[0] * unl, wl[1] * unl + pl * nx, wl[2] * unl + pl * ny, (wl[3] + pl) * unl};
  T fr[4] = {wr[0] * unr, wr[1] * unr + pr * nx, wr[2] * unr + pr * ny, (wr[3] + pr) * unr};
#pragma unroll
  for (int i = 0; i < 4; ++i) hq[i] = T(0.5) * (fl[i] + fr[i]) - T(0.5) * s * (wr[i] - wl[i]);
}

// ---- FP32 bulk in deviations from a reference state.  At low Mach number the pressure and
// energy dwarf the flow's variations (Mach 0.1: p ~ 71 against O(1) changes), and FP32 fluxes
// formed from full states lose those variations to rounding.  The FP32 path therefore carries
// the state copy as deviations d = w - w0 from a reference state w0 (vertex 0's state at the
// stage input, rounded to floats; the deviation is formed in FP64) and every flux as its
// deviation F(w) - F(w0).  Each least-squares divergence row annihilates constant fluxes, so the
// divergence is unchanged, and the deviations are formed by exact algebra on d:
//   u - u0 = (d1 - u0 d0) / rho,  p - p0 = (gamma-1) (d3 - (m0 du + d1 u + n0 dv + d2 v) / 2),
//   (rho u_n) - (rho u_n)0 = rho0 du_n + d0 u_n,  (m u_n + p n_x) - (...)0 = m0 du_n + d1 u_n + dp n_x,
//   ((E + p) u_n) - (...)0 = (E0 + p0) du_n + (d3 + dp) u_n,
// so no full-size quantity is subtracted in FP32.
struct Ref0 {
  float rho, m, n, E, u, v, p;
};
__device__ __forceinline__ Ref0 make_ref(const float* w0, float g1) {
  Ref0 r;
  r.rho = w0[0]; r.m = w0[1]; r.n = w0[2]; r.E = w0[3];
  const float ir = 1.0f / r.rho;
  r.u = r.m * ir; r.v = r.n * ir;
  r.p = g1 * (r.E - 0.5f * (r.m * r.u + r.n * r.v));
  return r;
}
// primitive deviations of the state w0 + d: density, velocity and their deviations, pressure
// deviation
struct Dev {
  float rho, ir, du, dv, u, v, dp;
};
__device__ __forceinline__ Dev make_dev(const Ref0& r, const float* d, float g1) {
  Dev q;
  q.rho = r.rho + d[0];
  q.ir = 1.0f / q.rho;
  q.du = (d[1] - r.u * d[0]) * q.ir;
  q.dv = (d[2] - r.v * d[0]) * q.ir;
  q.u = r.u + q.du;
  q.v = r.v + q.dv;
  q.dp = g1 * (d[3] - 0.5f * (r.m * q.du + d[1] * q.u + r.n * q.dv + d[2] * q.v));
  return q;
}
// F_n(w0 + d) - F_n(w0) along (nx, ny)
__device__ __forceinline__ void normal_flux_dev(const Ref0& r, const Dev& q, const float* d, float nx,
                                                float ny, float* f) {
  const float un = q.u * nx + q.v * ny, dun = q.du * nx + q.dv * ny;
  f[0] = r.rho * dun + d[0] * un;
  f[1] = r.m * dun + d[1] * un + q.dp * nx;
  f[2] = r.n * dun + d[2] * un + q.dp * ny;
  f[3] = (r.E + r.p) * dun + (d[3] + q.dp) * un;
}
// Roe's flux with Harten's fix (as roe_flux) minus F_n(w0), from the two sides' deviations dl,
// dr: the averages use the full states, every jump the deviations.
__device__ __forceinline__ void roe_flux_dev(const Ref0& r, const float* dl, const float* dr,
                                             float nx, float ny, float g1, float harten,
                                             float half_inv_harten, float* hq) {
  const Dev L = make_dev(r, dl, g1), R = make_dev(r, dr, g1);
  const float sl = sqrtf(L.rho), sr = sqrtf(R.rho);
  const float Hl = (r.E + dl[3] + r.p + L.dp) * L.ir, Hr = (r.E + dr[3] + r.p + R.dp) * R.ir;
  const float fl_ = sl / (sl + sr), fr_ = 1.0f - fl_;
  const float u = fl_ * L.u + fr_ * R.u, v = fl_ * L.v + fr_ * R.v, H = fl_ * Hl + fr_ * Hr;
  const float c2 = g1 * (H - 0.5f * (u * u + v * v));
  const float ic = rsqrtf(c2), c = c2 * ic;
  const float qn = u * nx + v * ny;
  const float rho = sl * sr, dp = R.dp - L.dp, drho = dr[0] - dl[0];
  const float dux = R.du - L.du, dvy = R.dv - L.dv;
  const float dun = dux * nx + dvy * ny, dut = dvy * nx - dux * ny;
  const float ic2 = ic * ic, hc2 = 0.5f * ic2, qc2 = 0.25f * ic2;
  const float rcd = rho * c * dun;
  const float a[4] = {(dp - rcd) * qc2, 0.5f * drho - dp * hc2, (0.5f * rho) * dut, (dp + rcd) * qc2};
  const float lam[4] = {qn - c, qn, qn, qn + c};
  const float del = harten * c, i2del = half_inv_harten * ic;
  float k[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float al = fabsf(lam[i]);
    if (al < del) al = (lam[i] * lam[i] + del * del) * i2del;
    k[i] = al * a[i];
  }
  float diss[4];
  right_apply(u, v, H, c, nx, ny, k, diss);
  float fl[4], fr[4];
  normal_flux_dev(r, L, dl, nx, ny, fl);
  normal_flux_dev(r, R, dr, nx, ny, fr);
#pragma unroll
  for (int i = 0; i < 4; ++i) hq[i] = 0.5f * (fl[i] + fr[i]) - diss[i];
}
// Rusanov's flux (as rusanov_flux) minus F_n(w0), from deviations.
__device__ __forceinline__ void rusanov_flux_dev(const Ref0& r, const float* dl, const float* dr,
                                                 float nx, float ny, float g1, float* hq) {
  const Dev L = make_dev(r, dl, g1), R = make_dev(r, dr, g1);
  const float gam = g1 + 1.0f;
  const float sl = fabsf(L.u * nx + L.v * ny) + sqrtf(gam * (r.p + L.dp) * L.ir);
  const float sr = fabsf(R.u * nx + R.v * ny) + sqrtf(gam * (r.p + R.dp) * R.ir);
  const float s = sl >= sr ? sl : sr;
  float fl[4], fr[4];
  normal_flux_dev(r, L, dl, nx, ny, fl);
  normal_flux_dev(r, R, dr, nx, ny, fr);
#pragma unroll
  for (int i = 0; i < 4; ++i) hq[i] = 0.5f * (fl[i] + fr[i]) - 0.5f * s * (dr[i] - dl[i]);
}

// ---- double-float arithmetic for the FP64 divergence in folded form.  GB300 issues FP32 at
// 64x its FP64 rate, and converts between FP64 and FP32 at the FP64 rate, so the splits below
// use integer operations only.
struct F2x {
  float hi, lo;
};
// x as hi + lo: hi = x truncated to 24 significant bits, lo = the remaining 29 bits rounded to
// 24, so |x - hi - lo| <= 2^-48 |x| for |x| >= 2^-78 (below that lo underflows and only hi is
// kept).  Zero and values below the float range give 0; infinities and NaN give
// themselves in hi.
__device__ __forceinline__ F2x split_df(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7ffull);
  F2x r;
  r.lo = 0.f;
  if (E == 0x7ff) {
    r.hi = __uint_as_float(sign | 0x7f800000u | ((b & 0xfffffffffffffull) ? 0x400000u : 0u));
    return r;
  }
  const int e = E - 1023;
  if (E == 0 || e < -126) {
    r.hi = __uint_as_float(sign);
    return r;
  }
  if (e > 127) {
    r.hi = __uint_as_float(sign | 0x7f800000u);
    return r;
  }
  r.hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffull));
  const unsigned ml = (unsigned)(b & 0x1fffffffull);          // the low 29 mantissa bits
  if (ml == 0u) return r;
  const int top = 31 - __clz((int)ml);                          // 0 .. 28
  int el = e - 52 + top;
  unsigned mant;
  if (top >= 24) {                                              // round to nearest
    mant = (ml + (1u << (top - 24))) >> (top - 23);
    if (mant >> 24) { mant >>= 1; ++el; }                       // the rounding carried
  } else {
    mant = ml << (23 - top);
  }
  if (el < -126) return r;
  r.lo = __uint_as_float(sign | ((unsigned)(el + 127) << 23) | (mant & 0x7fffffu));
  return r;
}
// A float as the exact double, by integer operations only (as the FP32-to-FP64 conversion
// gives it, subnormal floats included; NaN stays NaN).
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned E = (u >> 23) & 0xffu, mant = u & 0x7fffffu;
  if (E == 0u) {
    if (mant == 0u) return __longlong_as_double((long long)sign);
    // mant * 2^-149 with its leading bit at position t: exponent t - 149, shifted into place
    const int t = 31 - __clz((int)mant);
    const unsigned long long m52 = ((unsigned long long)mant << (52 - t)) & 0xfffffffffffffull;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(t + 874) << 52) | m52));
  }
  const unsigned long long eb = E == 0xffu ? 0x7ffull : (unsigned long long)(E - 127u + 1023u);
  return __longlong_as_double((long long)(sign | (eb << 52) | ((unsigned long long)mant << 29)));
}
// (sh, sl) += (ah, al) * (bh, bl): the product's rounding error by FMA and all four partial
// products, the sum by Knuth's two-sum; the low parts are accumulated without renormalising.  Explicit roundings keep the
// compiler from contracting the two-sum.
__device__ __forceinline__ void df_fma(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  e = __fmaf_rn(al, bl, e);
  const float s = __fadd_rn(sh, p);
  const float v = __fsub_rn(s, sh);
  const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(p, v));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// rho > 0 and p > 0 (R16), without a division: p = (gamma-1)(E - |m|^2/(2 rho)) has the sign
// of E rho - |m|^2/2 when rho > 0.
template <typename T>
__device__ __forceinline__ bool admissible(const T* w) {
  return w[0] > T(0) && w[3] * w[0] - T(0.5) * (w[1] * w[1] + w[2] * w[2]) > T(0);
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
__device__ __forceinline__ void vertex_body(int v, int V, const double* __restrict__ U, T* Ua,
                                            T* FG, T* FGv, const Phys& ph, float* wref,
                                            const float* s0f, const double* s0d) {
  if (v >= V) return;
  double w[12];
#pragma unroll
  for (int r = 0; r < 12; ++r) w[r] = U[(size_t)r * V + v];
  T* ua = Ua + (size_t)v * 12;
  T g1 = phys_g1<T>(ph);
  if constexpr (std::is_same<T, float>::value) {
    // deviations from the reference state (vertex 0 at the stage input, rounded to floats;
    // s0f / s0d hold it as floats and as their exact doubles, formed once per block)
    float w0[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) w0[r] = s0f[r];
    if (v == 0 && wref) st4(wref, w0);
    float d[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) d[r] = d2f_rn(w[r] - s0d[r]);
    st4(ua, d);
#pragma unroll
    for (int i = 1; i < 3; ++i) {
      float t[4] = {d2f_rn(w[4 * i]), d2f_rn(w[4 * i + 1]), d2f_rn(w[4 * i + 2]), d2f_rn(w[4 * i + 3])};
      st4(ua + 4 * i, t);
    }
    const Ref0 r0 = make_ref(w0, g1);
    const Dev q = make_dev(r0, d, g1);
    float F[4], Gf[4];
    normal_flux_dev(r0, q, d, 1.0f, 0.0f, F);
    normal_flux_dev(r0, q, d, 0.0f, 1.0f, Gf);
    st4(FG + (size_t)v * 8, F);
    st4(FG + (size_t)v * 8 + 4, Gf);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T t[4] = {T(w[4 * i]), T(w[4 * i + 1]), T(w[4 * i + 2]), T(w[4 * i + 3])};
      st4(ua + 4 * i, t);
    }
    T q[4] = {T(w[0]), T(w[1]), T(w[2]), T(w[3])};
    T ir = T(1) / q[0];
    T u = q[1] * ir, vv = q[2] * ir;
    T p = pressure(q, g1);
    T F[4] = {q[1], q[1] * u + p, q[2] * u, (q[3] + p) * u};
    T Gf[4] = {q[2], q[1] * vv, q[2] * vv + p, (q[3] + p) * vv};
    st4(FG + (size_t)v * 8, F);
    st4(FG + (size_t)v * 8 + 4, Gf);
  }
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

// The FP32 path's reference state for this block: vertex 0's values at the stage input rounded
// to floats, and those floats as exact doubles (threads 0-3 of the block convert them once).
__device__ __forceinline__ void block_reference(const double* __restrict__ U, int V, float* s0f,
                                                double* s0d) {
  if (threadIdx.x < 4 && V > 0) {
    const float f = (float)U[(size_t)threadIdx.x * V];
    s0f[threadIdx.x] = f;
    s0d[threadIdx.x] = (double)f;
  }
  __syncthreads();
}

template <typename T, bool VISC>
__global__ void __launch_bounds__(256) k_vertex(int V, const double* __restrict__ U, T* Ua, T* FG,
                                                T* FGv, Phys ph, float* wref) {
  __shared__ float s0f[4];
  __shared__ double s0d[4];
  if constexpr (std::is_same<T, float>::value) block_reference(U, V, s0f, s0d);
  vertex_body<T, VISC>(blockIdx.x * blockDim.x + threadIdx.x, V, U, Ua, FG, FGv, ph, wref, s0f, s0d);
}

// ------------------------------------------------------------------ k_edge
// One thread per flux edge.  Node order of the stencil: [i-2, i-1, i, i+1, i+2, i+3]; the left
// state uses nodes 0..4, the right state nodes 1..5 with the WENO sub-stencils mirrored.
//
// Arithmetic layout (same values as Alg. 1, fewer operations in the bulk type T):
//  * The 5-node value of every characteristic component is L times the same 5-node combination
//    of the conservative data (L is shared by all nodes), and R L = I.  So a side whose four
//    components all take the 5-node branch is the 5-node combination in conservative
//    variables, W5, with no projection and no back-projection.
//  * The discontinuity sensor needs only differences of characteristic values (the
//    smoothness indicators are shift-invariant).  They are formed from w_k - w_i, rounded to
//    FP32 and projected with an FP32 L; the test 0.01 < omega_1 < 0.79 is evaluated in that
//    precision with a relative guard band.  Decisions inside the band are re-taken with
//    characteristic values and weights in T / FP64, so every decision equals the one made in
//    the path's own precision.
//  * Only sides with a 3-node (or re-taken) component project W5, recompute the characteristic
//    values of that component, form the omega-weighted candidates and back-project.
constexpr float kGuard = 1e-3f;

__device__ __forceinline__ float to_f32(double x) { return d2f_rn(x); }
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float sensor_diff(double a, double b) { return d2f_rn(a - b); }
__device__ __forceinline__ float sensor_diff(float a, float b) { return a - b; }

template <typename T>
__device__ __forceinline__ void sensor64(T u0, T u1, T u2, T u3, T u4, const Phys& ph,
                                         double* t, double& S) {
  T b[3];
  smoothness(u0, u1, u2, u3, u4, b);
  double s0 = ph.eps + (double)b[0], s1 = ph.eps + (double)b[1], s2 = ph.eps + (double)b[2];
  s0 *= s0; s1 *= s1; s2 *= s2;
  t[0] = (1.0 / 16.0) * s1 * s2;
  t[1] = (10.0 / 16.0) * s0 * s2;
  t[2] = (5.0 / 16.0) * s0 * s1;
  S = t[0] + t[1] + t[2];
}

template <typename T>
__device__ __forceinline__ void edge_body(int e, int Ef, int V, const int32_t* __restrict__ sten,
                                          const T* __restrict__ nrm, const T* __restrict__ w5,
                                          const T* __restrict__ w3, const T* __restrict__ Ua,
                                          T* __restrict__ h, const Phys& ph, unsigned* err,
                                          uint8_t* __restrict__ dbg, const float* __restrict__ wref,
                                          const double* __restrict__ FGd = nullptr) {
  if (e >= Ef) return;
  const T g1 = phys_g1<T>(ph);
  int s[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) s[k] = chk_idx(ld_stream(sten + (size_t)k * Ef + e), V, err);
  T nx = ld_stream(nrm + e), ny = ld_stream(nrm + Ef + e);
  T wi[4], wj[4];
  {
    T a[12];
    ld12(Ua + (size_t)s[2] * 12, a);
    wi[0] = a[0]; wi[1] = a[1]; wi[2] = a[2]; wi[3] = a[3];
    ld12(Ua + (size_t)s[3] * 12, a);
    wj[0] = a[0]; wj[1] = a[1]; wj[2] = a[2]; wj[3] = a[3];
  }
  // FP32 data are deviations from the reference state w0: the averages and the admissibility
  // test take the full states w0 + d (FP64 data are the states)
  float w0[4] = {0.f, 0.f, 0.f, 0.f};
  T fwi[4], fwj[4];
  if constexpr (std::is_same<T, float>::value) {
    const float4 r = __ldg(reinterpret_cast<const float4*>(wref));
    w0[0] = r.x; w0[1] = r.y; w0[2] = r.z; w0[3] = r.w;
#pragma unroll
    for (int q = 0; q < 4; ++q) { fwi[q] = w0[q] + wi[q]; fwj[q] = w0[q] + wj[q]; }
  } else {          // FP64 data are the states themselves (no additions on the FP64 pipe)
#pragma unroll
    for (int q = 0; q < 4; ++q) { fwi[q] = wi[q]; fwj[q] = wj[q]; }
  }
  // FP32 left eigenvectors at the Roe state of the edge ends (sensor only)
  float Lf[4][4];
  {
    float fi[4], fj[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { fi[q] = to_f32(fwi[q]); fj[q] = to_f32(fwj[q]); }
    float u, v, H, c;
    roe_avg(fi, fj, ph.g1f, u, v, H, c);
    left_ev(u, v, c, to_f32(nx), to_f32(ny), ph.g1f, Lf);
  }
  T W5L[4] = {T(0), T(0), T(0), T(0)}, W5R[4] = {T(0), T(0), T(0), T(0)};
  float cf[6][4];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    T a[12];
    ld12(Ua + (size_t)s[k] * 12, a);
    if (k <= 4) {
      T wv = ld_stream(w5 + (size_t)(3 * k) * Ef + e), wx = ld_stream(w5 + (size_t)(3 * k + 1) * Ef + e);
      T wy = ld_stream(w5 + (size_t)(3 * k + 2) * Ef + e);
#pragma unroll
      for (int r = 0; r < 4; ++r) W5L[r] = fma(wv, a[r], fma(wx, a[4 + r], fma(wy, a[8 + r], W5L[r])));
    }
    if (k >= 1) {
      T wv = ld_stream(w5 + (size_t)(15 + 3 * (k - 1)) * Ef + e);
      T wx = ld_stream(w5 + (size_t)(16 + 3 * (k - 1)) * Ef + e);
      T wy = ld_stream(w5 + (size_t)(17 + 3 * (k - 1)) * Ef + e);
#pragma unroll
      for (int r = 0; r < 4; ++r) W5R[r] = fma(wv, a[r], fma(wx, a[4 + r], fma(wy, a[8 + r], W5R[r])));
    }
    // end-state differences rounded once to FP32 (for FP32 data the float subtraction is that
    // correctly rounded difference already; for FP64 data it is formed in FP64 first)
    float d[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) d[r] = sensor_diff(a[r], wi[r]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      cf[k][q] = Lf[q][0] * d[0] + Lf[q][1] * d[1] + Lf[q][2] * d[2] + Lf[q][3] * d[3];
  }
  // sensor in FP32: bit (side*4+q) of `rough` = 3-node branch, of `amb` = inside the guard band
  unsigned rough = 0, amb = 0;
#pragma unroll
  for (int side = 0; side < 2; ++side)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float u0, u1, u2, u3, u4;
      if (side == 0) { u0 = cf[0][q]; u1 = cf[1][q]; u2 = cf[2][q]; u3 = cf[3][q]; u4 = cf[4][q]; }
      else           { u0 = cf[5][q]; u1 = cf[4][q]; u2 = cf[3][q]; u3 = cf[2][q]; u4 = cf[1][q]; }
      float b[3];
      smoothness(u0, u1, u2, u3, u4, b);
      float eps = ph.epsf;
      float s0 = eps + b[0], s1 = eps + b[1], s2 = eps + b[2];
      s0 *= s0; s1 *= s1; s2 *= s2;
      float t0 = 0.0625f * s1 * s2, t1 = 0.625f * s0 * s2, t2 = 0.3125f * s0 * s1;
      float S = t0 + t1 + t2;
      float mlo = t0 - ph.sens_lof * S, mhi = ph.sens_hif * S - t0;
      unsigned bit = 1u << (side * 4 + q);
      if (!(mlo > 0.f && mhi > 0.f)) rough |= bit;
      if (!(fabsf(mlo) > kGuard * S && fabsf(mhi) > kGuard * S)) amb |= bit;
    }
  if (ph.force_branch == 1) rough = amb = 0u;                 // every side 5-node
  else if (ph.force_branch == 2) { rough = 0xffu; amb = 0u; } // every side 3-node WENO
  T wside[2][4];
#pragma unroll
  for (int r = 0; r < 4; ++r) { wside[0][r] = W5L[r]; wside[1][r] = W5R[r]; }
  unsigned taken = ph.force_branch == 2 ? 0xffu : 0u;   // 3-node branch taken (testing aid)
  if (rough | amb) {
    T u, v, H, c;
    roe_avg(fwi, fwj, g1, u, v, H, c);
    T L[4][4];
    left_ev(u, v, c, nx, ny, g1, L);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      unsigned mine = ((rough | amb) >> (side * 4)) & 15u;
      if (!mine) continue;
      const T* W5 = side == 0 ? W5L : W5R;
      T C[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        C[q] = L[q][0] * W5[0] + L[q][1] * W5[1] + L[q][2] * W5[2] + L[q][3] * W5[3];
        if (!((mine >> q) & 1u)) continue;
        T cq[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          int k = side == 0 ? j : 5 - j;
          T a[4];
          ld4(Ua + (size_t)s[k] * 12, a);
          cq[j] = L[q][0] * a[0] + L[q][1] * a[1] + L[q][2] * a[2] + L[q][3] * a[3];
        }
        double t[3], S;
        sensor64(cq[0], cq[1], cq[2], cq[3], cq[4], ph, t, S);
        bool smooth = (t[0] > ph.sens_lo * S) && (t[0] < ph.sens_hi * S);
        if (smooth && ph.force_branch != 2) continue;
        taken |= 1u << (side * 4 + q);
        const T* w = w3 + (size_t)(9 * side) * Ef + e;
        T c1 = ld_stream(w) * cq[0] + ld_stream(w + Ef) * cq[1] + ld_stream(w + 2 * (size_t)Ef) * cq[2];
        T c2 = ld_stream(w + 3 * (size_t)Ef) * cq[1] + ld_stream(w + 4 * (size_t)Ef) * cq[2] +
               ld_stream(w + 5 * (size_t)Ef) * cq[3];
        T c3 = ld_stream(w + 6 * (size_t)Ef) * cq[2] + ld_stream(w + 7 * (size_t)Ef) * cq[3] +
               ld_stream(w + 8 * (size_t)Ef) * cq[4];
        double iS = 1.0 / S;
        C[q] = T((t[0] * (double)c1 + t[1] * (double)c2 + t[2] * (double)c3) * iS);
      }
      right_apply(u, v, H, c, nx, ny, C, wside[side]);
    }
  }
  if (dbg) dbg[e] = (uint8_t)taken;
  // positivity (R16): fall back to the end state of that side
  {
    T fl[4], fr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if constexpr (std::is_same<T, float>::value) {
        fl[q] = w0[q] + wside[0][q];
        fr[q] = w0[q] + wside[1][q];
      } else {
        fl[q] = wside[0][q];
        fr[q] = wside[1][q];
      }
    }
    if (!admissible(fl))
#pragma unroll
      for (int q = 0; q < 4; ++q) wside[0][q] = wi[q];
    if (!admissible(fr))
#pragma unroll
      for (int q = 0; q < 4; ++q) wside[1][q] = wj[q];
  }
  T hq[4];
  if constexpr (std::is_same<T, float>::value) {
    // the flux's deviation from F_n(w0)
    const Ref0 r0 = make_ref(w0, g1);
    if (ph.flux == 1)
      rusanov_flux_dev(r0, wside[0], wside[1], nx, ny, g1, hq);
    else
      roe_flux_dev(r0, wside[0], wside[1], nx, ny, g1, phys_harten<T>(ph), phys_half_inv_harten<T>(ph), hq);
  } else {
    if (ph.flux == 1)
      rusanov_flux(wside[0], wside[1], nx, ny, g1, hq);
    else
      roe_flux(wside[0], wside[1], nx, ny, g1, phys_harten<T>(ph), phys_half_inv_harten<T>(ph), hq);
    if (FGd) {
      // folded divergence: the flux minus the average of the end vertices' projected fluxes
      // (O(h^2) on smooth data), as float pairs
      double fa[8], fb[8];
      ld8(FGd + (size_t)s[2] * 8, fa);
      ld8(FGd + (size_t)s[3] * 8, fb);
      F2x t[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        t[q] = split_df(hq[q] - 0.5 * ((fa[q] + fb[q]) * nx + (fa[4 + q] + fb[4 + q]) * ny));
      float4* o = reinterpret_cast<float4*>(h + (size_t)e * 4);
      o[0] = make_float4(t[0].hi, t[0].lo, t[1].hi, t[1].lo);
      o[1] = make_float4(t[2].hi, t[2].lo, t[3].hi, t[3].lo);
      return;
    }
  }
  st4(h + (size_t)e * 4, hq);
}

// Resident blocks of 128 threads the compiler must allow: 3 for FP64 data (<= 170 registers; an
// explicit bound of 1 lets it take ~214 and lose a block), 5 for FP32 data (96 registers, an
// 8-byte spill; 4 percent faster than 4 blocks on the four-quadrant 1024x1024 step).
template <typename T>
struct EdgeOcc { static constexpr int kMinBlocks = 3; };
template <>
struct EdgeOcc<float> { static constexpr int kMinBlocks = 5; };

template <typename T>
__global__ void __launch_bounds__(128, EdgeOcc<T>::kMinBlocks) k_edge(int Ef, int V, const int32_t* __restrict__ sten,
                                              const T* __restrict__ nrm, const T* __restrict__ w5,
                                              const T* __restrict__ w3, const T* __restrict__ Ua,
                                              T* __restrict__ h, Phys ph, unsigned* err,
                                              uint8_t* __restrict__ dbg, const float* __restrict__ wref,
                                              const double* __restrict__ FGd) {
  edge_body<T>(blockIdx.x * blockDim.x + threadIdx.x, Ef, V, sten, nrm, w5, w3, Ua, h, ph, err, dbg,
               wref, FGd);
}

// ------------------------------------------------------------------ k_div
// G lanes per active vertex (G in {1, 2, 4}); lanes stride over the CSR entries; the 12 partial
// sums are combined by a fixed reduce-scatter over the group (each level halves the values a
// lane holds), so the result is deterministic and every add is useful.  acc = div(f) -
// div(f_vis) for the 12 rows; R = -acc.
template <int G, typename T>
__device__ __forceinline__ void reduce_scatter12(T* acc, int lane) {
  // after the loop lane `lane` holds rows base .. base + 12/G - 1 in acc[0 .. 12/G - 1]
  if (G >= 2) {
    const int o = G / 2;
    bool hi = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      T keep = hi ? acc[6 + i] : acc[i];
      T send = hi ? acc[i] : acc[6 + i];
      acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o, G);
    }
  }
  if (G >= 4) {
    const int o = G / 4;
    bool hi = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T keep = hi ? acc[3 + i] : acc[i];
      T send = hi ? acc[i] : acc[3 + i];
      acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o, G);
    }
  }
  if (G >= 8) {
    // three values left: the lane with bit 0 clear keeps rows 0-1, its partner keeps row 2
    bool hi = (lane & 1) != 0;
    T r0 = __shfl_xor_sync(0xffffffffu, acc[0], 1, G);
    T r1 = __shfl_xor_sync(0xffffffffu, acc[1], 1, G);
    T r2 = __shfl_xor_sync(0xffffffffu, acc[2], 1, G);
    if (hi) {
      acc[0] = acc[2] + r2;
    } else {
      acc[0] += r0;
      acc[1] += r1;
    }
  }
}

// Per-stage arguments of the divergence: out = R (residual) or a*Un + b*(Us + dt*R) (stage).
struct StageArgs {
  const double* Us;
  const double* Un;
  double* out;
  int mode;
  double a, b, dt_fixed;
  const double* dt_member;   // per-mesh step of a batch (dt_fixed <= 0), or nullptr
};

// FP32-bulk gather of one vertex's divergence rows over the chunked layout: lane `lane` of
// the group takes chunks lane, lane + G, ...; per chunk one int4 of indices, 6 (3 for edges)
// float4 coefficient rows and 4 flux gathers, all independent loads.  Padding entries carry
// zero coefficients.
__device__ __forceinline__ float f4c(const float4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
__device__ __forceinline__ int i4c(const int4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

template <int G, bool VISC>
__device__ __forceinline__ void div_gather_chunked(
    int r, int lane, int V, int Ef, unsigned* err, const int32_t* __restrict__ vptr,
    const int32_t* __restrict__ vidx,
    const int32_t* __restrict__ eptr, const int32_t* __restrict__ eidx,
    const float* __restrict__ cv, const float* __restrict__ ce, const float* __restrict__ cvis,
    const float* __restrict__ FG, const float* __restrict__ FGv, const float* __restrict__ h,
    float* acc) {
  static_assert(kDivChunk == 4, "float4 chunks");
  const int c0 = __ldg(vptr + r), nc = __ldg(vptr + r + 1) - c0;
  const int4* vi = reinterpret_cast<const int4*>(vidx) + c0;
  const float4* cc = reinterpret_cast<const float4*>(cv) + 6 * (size_t)c0;
  const float4* cz = VISC ? reinterpret_cast<const float4*>(cvis) + 6 * (size_t)c0 : nullptr;
  for (int ch = lane; ch < nc; ch += G) {
    const int4 u = __ldg(vi + ch);
    float4 k[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) k[i] = __ldg(cc + 6 * ch + i);
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      float f[8];
      ld8(FG + (size_t)chk_idx(i4c(u, q4), V, err) * 8, f);
      const float c0f = f4c(k[0], q4), c0g = f4c(k[1], q4), cxf = f4c(k[2], q4);
      const float cxg = f4c(k[3], q4), cyf = f4c(k[4], q4), cyg = f4c(k[5], q4);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] = fmaf(c0g, f[4 + q], fmaf(c0f, f[q], acc[q]));
        acc[4 + q] = fmaf(cxg, f[4 + q], fmaf(cxf, f[q], acc[4 + q]));
        acc[8 + q] = fmaf(cyg, f[4 + q], fmaf(cyf, f[q], acc[8 + q]));
      }
    }
    if (VISC) {
#pragma unroll
      for (int i = 0; i < 6; ++i) k[i] = __ldg(cz + 6 * ch + i);
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        float f[8];
        ld8(FGv + (size_t)chk_idx(i4c(u, q4), V, err) * 8, f);
        const float c0f = f4c(k[0], q4), c0g = f4c(k[1], q4), cxf = f4c(k[2], q4);
        const float cxg = f4c(k[3], q4), cyf = f4c(k[4], q4), cyg = f4c(k[5], q4);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q] = fmaf(-c0g, f[4 + q], fmaf(-c0f, f[q], acc[q]));
          acc[4 + q] = fmaf(-cxg, f[4 + q], fmaf(-cxf, f[q], acc[4 + q]));
          acc[8 + q] = fmaf(-cyg, f[4 + q], fmaf(-cyf, f[q], acc[8 + q]));
        }
      }
    }
  }
  const int m0 = __ldg(eptr + r), mc = __ldg(eptr + r + 1) - m0;
  const int4* ei = reinterpret_cast<const int4*>(eidx) + m0;
  const float4* dd = reinterpret_cast<const float4*>(ce) + 3 * (size_t)m0;
  for (int ch = lane; ch < mc; ch += G) {
    const int4 e = __ldg(ei + ch);
    const float4 d0 = __ldg(dd + 3 * ch), dx = __ldg(dd + 3 * ch + 1), dy = __ldg(dd + 3 * ch + 2);
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      float hv[4];
      ld4(h + (size_t)chk_idx(i4c(e, q4), Ef, err) * 4, hv);
      const float a0 = f4c(d0, q4), ax = f4c(dx, q4), ay = f4c(dy, q4);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] = fmaf(a0, hv[q], acc[q]);
        acc[4 + q] = fmaf(ax, hv[q], acc[4 + q]);
        acc[8 + q] = fmaf(ay, hv[q], acc[8 + q]);
      }
    }
  }
}

// Finite (not inf or NaN) by the exponent field, on the integer pipe (GB300's FP64 pipe is
// the limit of the FP64 divergence).
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned)(__double_as_longlong(x) >> 52) & 0x7ffu) != 0x7ffu;
}

// Combines the lanes' partial sums of vertex r (every lane of the warp must call this: the
// reduce-scatter shuffles over the whole warp) and writes R = -acc, or the Runge-Kutta stage
// combination a*Un + b*(Us + dt*R), for the rows this lane holds; flags non-finite values and
// non-positive densities in the error word.
template <typename T, int G>
__device__ __forceinline__ void div_finish(int r, int lane, bool live, T* acc, int V,
                                           const StageArgs& sa, const int32_t* __restrict__ vmem,
                                           const unsigned long long* dtbits, double cfl,
                                           double* dt_last, unsigned* err) {
  reduce_scatter12<G>(acc, lane);
  if (!live) return;
  const double* __restrict__ Us = sa.Us;
  const double* __restrict__ Un = sa.Un;
  double* out = sa.out;
  const int mode = sa.mode;
  const double a = sa.a, b = sa.b, dt_fixed = sa.dt_fixed;
  // time step of this vertex's mesh (a batch holds several meshes, each with its own CFL step)
  const int mem = vmem ? __ldg(vmem + r) : 0;
  double dt = dt_fixed > 0.0 ? dt_fixed
               : sa.dt_member ? __ldg(sa.dt_member + mem)
                              : cfl * __longlong_as_double((long long)dtbits[mem]);
  if (mode == DIV_STAGE && lane == 0 && dt_last && (r == 0 || (vmem && __ldg(vmem + r - 1) != mem)))
    dt_last[mem] = dt;
  // rows held by this lane after the reduce-scatter: base .. base + per - 1
  int per = G == 1 ? 12 : G == 2 ? 6 : 3;
  int base = (G >= 2 && (lane & (G / 2)) ? 6 : 0) + (G >= 4 && (lane & (G / 4)) ? 3 : 0);
  if (G >= 8) {
    if (lane & 1) { base += 2; per = 1; } else { per = 2; }
  }
  unsigned bad = 0;
#pragma unroll
  for (int i = 0; i < 12 / (G >= 8 ? 4 : G); ++i) {
    if (i >= per) break;
    int k = base + i;
    double R = -(double)acc[i];
    size_t idx = (size_t)k * V + r;
    double o;
    if (mode == DIV_RESIDUAL) {
      o = R;
    } else {
      // explicit roundings, so that every kernel holding this code (four-launch, staged,
      // persistent) gives the same bits: one FMA, one multiply, one FMA
      o = __dmul_rn(b, __fma_rn(dt, R, Us[idx]));
      if (a != 0.0) o = __fma_rn(a, Un[idx], o);   // the first stage does not read the base state
    }
    out[idx] = o;
    if (!finite_bits(o)) bad |= ERRBIT_NONFINITE;
    if (mode == DIV_STAGE && k == 0 && !(o > 0.0)) bad |= ERRBIT_POSITIVITY;
  }
  if (bad) atomicOr(err, bad);
}

template <typename T, int G, bool VISC>
__device__ __forceinline__ void div_body(int gt, int A, int V, int Ef, const int32_t* __restrict__ vptr,
                                         const int32_t* __restrict__ vidx,
                                         const int32_t* __restrict__ eptr,
                                         const int32_t* __restrict__ eidx,
                                         const T* __restrict__ cv, const T* __restrict__ ce,
                                         const T* __restrict__ cvis, const T* __restrict__ FG,
                                         const T* __restrict__ FGv, const T* __restrict__ h,
                                         const StageArgs& sa, const int32_t* __restrict__ vmem,
                                         const unsigned long long* dtbits, double cfl,
                                         double* dt_last, unsigned* err) {
  int r = gt / G, lane = gt % G;
  bool live = r < A;
  T acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = T(0);
  if constexpr (std::is_same<T, float>::value) {
    if (live) div_gather_chunked<G, VISC>(r, lane, V, Ef, err, vptr, vidx, eptr, eidx, cv, ce, cvis, FG, FGv, h, acc);
  } else if (live) {
    int n0 = __ldg(vptr + r), N = __ldg(vptr + r + 1) - n0;
    const T* c = cv + 6 * (size_t)n0;
    const T* cz = VISC ? cvis + 6 * (size_t)n0 : nullptr;
    // vertex entries, two per lane per iteration so that both entries' loads are in flight
    // before their multiply-adds (the same per-lane summation order as one at a time)
    auto vtx = [&](int j, const T* f, const T* fv) {
      T c0f = ld_stream(c + j), c0g = ld_stream(c + N + j), cxf = ld_stream(c + 2 * N + j);
      T cxg = ld_stream(c + 3 * N + j), cyf = ld_stream(c + 4 * N + j), cyg = ld_stream(c + 5 * N + j);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] = fma(c0g, f[4 + q], fma(c0f, f[q], acc[q]));
        acc[4 + q] = fma(cxg, f[4 + q], fma(cxf, f[q], acc[4 + q]));
        acc[8 + q] = fma(cyg, f[4 + q], fma(cyf, f[q], acc[8 + q]));
      }
      if (VISC) {
        c0f = ld_stream(cz + j); c0g = ld_stream(cz + N + j); cxf = ld_stream(cz + 2 * N + j);
        cxg = ld_stream(cz + 3 * N + j); cyf = ld_stream(cz + 4 * N + j); cyg = ld_stream(cz + 5 * N + j);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q] = fma(-c0g, fv[4 + q], fma(-c0f, fv[q], acc[q]));
          acc[4 + q] = fma(-cxg, fv[4 + q], fma(-cxf, fv[q], acc[4 + q]));
          acc[8 + q] = fma(-cyg, fv[4 + q], fma(-cyf, fv[q], acc[8 + q]));
        }
      }
    };
    int j = lane;
    for (; j + G < N; j += 2 * G) {
      int u0 = chk_idx(ld_stream(vidx + n0 + j), V, err), u1 = chk_idx(ld_stream(vidx + n0 + j + G), V, err);
      T f0[8], f1[8], g0[8], g1[8];
      ld8(FG + (size_t)u0 * 8, f0);
      ld8(FG + (size_t)u1 * 8, f1);
      if (VISC) {
        ld8(FGv + (size_t)u0 * 8, g0);
        ld8(FGv + (size_t)u1 * 8, g1);
      }
      vtx(j, f0, g0);
      vtx(j + G, f1, g1);
    }
    if (j < N) {
      int u0 = chk_idx(ld_stream(vidx + n0 + j), V, err);
      T f0[8], g0[8];
      ld8(FG + (size_t)u0 * 8, f0);
      if (VISC) ld8(FGv + (size_t)u0 * 8, g0);
      vtx(j, f0, g0);
    }
    int m0 = __ldg(eptr + r), M = __ldg(eptr + r + 1) - m0;
    const T* d = ce + 3 * (size_t)m0;
    auto edg = [&](int jj, const T* hv) {
      T d0 = ld_stream(d + jj), dx = ld_stream(d + M + jj), dy = ld_stream(d + 2 * M + jj);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] = fma(d0, hv[q], acc[q]);
        acc[4 + q] = fma(dx, hv[q], acc[4 + q]);
        acc[8 + q] = fma(dy, hv[q], acc[8 + q]);
      }
    };
    j = lane;
    for (; j + G < M; j += 2 * G) {
      int e0 = chk_idx(ld_stream(eidx + m0 + j), Ef, err), e1 = chk_idx(ld_stream(eidx + m0 + j + G), Ef, err);
      T h0[4], h1[4];
      ld4(h + (size_t)e0 * 4, h0);
      ld4(h + (size_t)e1 * 4, h1);
      edg(j, h0);
      edg(j + G, h1);
    }
    if (j < M) {
      int e0 = chk_idx(ld_stream(eidx + m0 + j), Ef, err);
      T h0[4];
      ld4(h + (size_t)e0 * 4, h0);
      edg(j, h0);
    }
  }
  div_finish<T, G>(r, lane, live, acc, V, sa, vmem, dtbits, cfl, dt_last, err);
}

// FP32 divergence with its stencil gathers staged in shared memory (inviscid meshes): block b
// holds the rows of tile b (kGsRows consecutive rows, kGsLanes lanes each, the row and lane
// mapping of k_div<float, 4>).  The host lists, per tile, the distinct vertices and flux edges
// its chunks read (gtv, gte) and rewrites each chunk's indices as 16-bit positions in those
// lists (lvidx, leidx).  The block first copies the listed vertex fluxes (8 floats) and edge
// fluxes (4 floats) into shared memory, each once, then every lane runs the chunk loop of
// div_gather_chunked with the same loads of coefficients and the same multiply-adds in the
// same order, reading the fluxes from shared memory: the result equals k_div<float, 4> bit for
// bit.
__global__ void __launch_bounds__(256, 4) k_div_gs(
    int A, int V, int Ef, const int32_t* __restrict__ vptr, const ushort4* __restrict__ lvidx,
    const int32_t* __restrict__ eptr, const ushort4* __restrict__ leidx,
    const float* __restrict__ cv, const float* __restrict__ ce, const float* __restrict__ FG,
    const float* __restrict__ h, const int32_t* __restrict__ gtv_ptr,
    const int32_t* __restrict__ gtv, const int32_t* __restrict__ gte_ptr,
    const int32_t* __restrict__ gte, StageArgs sa, const int32_t* __restrict__ vmem,
    const unsigned long long* dtbits, double cfl, double* dt_last, unsigned* err) {
  extern __shared__ float4 gs_smem[];
  const int tile = blockIdx.x;
  const int v0 = __ldg(gtv_ptr + tile), nv = __ldg(gtv_ptr + tile + 1) - v0;
  const int e0 = __ldg(gte_ptr + tile), ne = __ldg(gte_ptr + tile + 1) - e0;
  float4* sFG = gs_smem;            // 2 float4 per listed vertex
  float4* sH = gs_smem + 2 * nv;    // 1 float4 per listed edge
  for (int i = threadIdx.x; i < 2 * nv; i += blockDim.x) {
    const int u = chk_idx(__ldg(gtv + v0 + (i >> 1)), V, err);
    sFG[i] = __ldg(reinterpret_cast<const float4*>(FG + (size_t)u * 8) + (i & 1));
  }
  for (int i = threadIdx.x; i < ne; i += blockDim.x) {
    const int e = chk_idx(__ldg(gte + e0 + i), Ef, err);
    sH[i] = __ldg(reinterpret_cast<const float4*>(h + (size_t)e * 4));
  }
  __syncthreads();
  constexpr int G = kGsLanes;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = gt / G, lane = gt % G;
  const bool live = r < A;
  float acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = 0.f;
  if (live) {
    const int c0 = __ldg(vptr + r), nc = __ldg(vptr + r + 1) - c0;
    const float4* cc = reinterpret_cast<const float4*>(cv) + 6 * (size_t)c0;
    for (int ch = lane; ch < nc; ch += G) {
      const ushort4 u = __ldg(lvidx + c0 + ch);
      float4 k[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) k[i] = __ldg(cc + 6 * ch + i);
      const unsigned short ui[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const float4 a = sFG[2 * ui[q4]], bq = sFG[2 * ui[q4] + 1];
        const float f[8] = {a.x, a.y, a.z, a.w, bq.x, bq.y, bq.z, bq.w};
        const float c0f = f4c(k[0], q4), c0g = f4c(k[1], q4), cxf = f4c(k[2], q4);
        const float cxg = f4c(k[3], q4), cyf = f4c(k[4], q4), cyg = f4c(k[5], q4);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q] = fmaf(c0g, f[4 + q], fmaf(c0f, f[q], acc[q]));
          acc[4 + q] = fmaf(cxg, f[4 + q], fmaf(cxf, f[q], acc[4 + q]));
          acc[8 + q] = fmaf(cyg, f[4 + q], fmaf(cyf, f[q], acc[8 + q]));
        }
      }
    }
    const int m0 = __ldg(eptr + r), mc = __ldg(eptr + r + 1) - m0;
    const float4* dd = reinterpret_cast<const float4*>(ce) + 3 * (size_t)m0;
    for (int ch = lane; ch < mc; ch += G) {
      const ushort4 e = __ldg(leidx + m0 + ch);
      const float4 d0 = __ldg(dd + 3 * ch), dx = __ldg(dd + 3 * ch + 1), dy = __ldg(dd + 3 * ch + 2);
      const unsigned short ei[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const float4 t = sH[ei[q4]];
        const float hv[4] = {t.x, t.y, t.z, t.w};
        const float a0 = f4c(d0, q4), ax = f4c(dx, q4), ay = f4c(dy, q4);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q] = fmaf(a0, hv[q], acc[q]);
          acc[4 + q] = fmaf(ax, hv[q], acc[4 + q]);
          acc[8 + q] = fmaf(ay, hv[q], acc[8 + q]);
        }
      }
    }
  }
  div_finish<float, G>(r, lane, live, acc, V, sa, vmem, dtbits, cfl, dt_last, err);
}

// FP32 data: memory-latency bound, so at least 4 resident blocks of 256 threads per SM; FP64
// data: FP64-pipe bound, 2 blocks (without a bound the compiler takes ~168 registers and the
// kernel loses half its warps).
template <typename T>
struct DivOcc { static constexpr int kMinBlocks = 2; };
template <>
struct DivOcc<float> { static constexpr int kMinBlocks = 4; };

template <typename T, int G, bool VISC>
__global__ void __launch_bounds__(256, DivOcc<T>::kMinBlocks) k_div(int A, int V, int Ef, const int32_t* __restrict__ vptr,
                                             const int32_t* __restrict__ vidx,
                                             const int32_t* __restrict__ eptr,
                                             const int32_t* __restrict__ eidx,
                                             const T* __restrict__ cv, const T* __restrict__ ce,
                                             const T* __restrict__ cvis, const T* __restrict__ FG,
                                             const T* __restrict__ FGv, const T* __restrict__ h,
                                             StageArgs sa, const int32_t* __restrict__ vmem,
                                             const unsigned long long* dtbits, double cfl,
                                             double* dt_last, unsigned* err) {
  div_body<T, G, VISC>(blockIdx.x * blockDim.x + threadIdx.x, A, V, Ef, vptr, vidx, eptr, eidx, cv,
                       ce, cvis, FG, FGv, h, sa, vmem, dtbits, cfl, dt_last, err);
}

// ------------------------------------------------------------------ k_div, folded double-float (FP64)
constexpr int kDfLanes = 4;
// The FP64 divergence with its products on the FP32 pipe.  Every least-squares row annihilates
// constant fluxes, and every edge row sees the same edge data.  At upload, each edge row's
// endpoint average, (1/2) d_m (F_a + F_b) . n_m, is folded into the two vertices' coefficients
// (cvdf), and k_edge stores the remainder dh_m = h_m - (F_a + F_b) . n_m / 2, which is O(h^2)
// on smooth data.  The rows are then
//   sum_j a'_j (F_j - F_c) + F_c sum_j a'_j + sum_m d_m dh_m,
// with the centre vertex's flux F_c subtracted exactly in FP64 (one DADD per value) and the
// row sums sum_j a'_j precomputed in FP64 (sig).  No term cancels against another any more, so
// double-float products (48-bit significands, FP32 pipe) keep the FP64 result's accuracy.  The
// viscous rows, when present, stay in FP64.  kDfLanes lanes per vertex, combined in FP64 by the
// fixed reduce-scatter of the other divergence kernels (one lane in the persistent form).
template <int G, bool VISC>
__device__ __forceinline__ void div_body_df(int gt, int A, int V, int Ef,
                                            const int32_t* __restrict__ vptr,
                                            const int32_t* __restrict__ vidx,
                                            const int32_t* __restrict__ eptr,
                                            const int32_t* __restrict__ eidx,
                                            const float2* __restrict__ cvdf,
                                            const float2* __restrict__ cedf,
                                            const double* __restrict__ sig,
                                            const double* __restrict__ cvis,
                                            const double* __restrict__ FG,
                                            const double* __restrict__ FGv,
                                            const float* __restrict__ hdf, const StageArgs& sa,
                                            const int32_t* __restrict__ vmem,
                                            const unsigned long long* dtbits, double cfl,
                                            double* dt_last, unsigned* err) {
  const int r = gt / G, lane = gt % G;
  const bool live = r < A;
  double acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = 0.0;
  if (live) {
    float sh[12], sl[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) { sh[k] = 0.f; sl[k] = 0.f; }
    double fc[8];
    ld8(FG + (size_t)r * 8, fc);
    const int n0 = __ldg(vptr + r), N = __ldg(vptr + r + 1) - n0;
    const float2* c = cvdf + 6 * (size_t)n0;
    auto vtx = [&](int j, const double* f) {
      F2x d[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) d[q] = split_df(f[q] - fc[q]);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 cf = __ldg(c + (size_t)(2 * k) * N + j), cg = __ldg(c + (size_t)(2 * k + 1) * N + j);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          df_fma(sh[4 * k + q], sl[4 * k + q], cf.x, cf.y, d[q].hi, d[q].lo);
          df_fma(sh[4 * k + q], sl[4 * k + q], cg.x, cg.y, d[4 + q].hi, d[4 + q].lo);
        }
      }
    };
    // lanes stride over the entries, two per lane per iteration so that both entries' gathers
    // are in flight before their arithmetic (the per-lane order is that of one at a time)
    int j = lane;
    for (; j + G < N; j += 2 * G) {
      const int u0 = chk_idx(ld_stream(vidx + n0 + j), V, err), u1 = chk_idx(ld_stream(vidx + n0 + j + G), V, err);
      double f0[8], f1[8];
      ld8(FG + (size_t)u0 * 8, f0);
      ld8(FG + (size_t)u1 * 8, f1);
      vtx(j, f0);
      vtx(j + G, f1);
    }
    if (j < N) {
      double f0[8];
      ld8(FG + (size_t)chk_idx(ld_stream(vidx + n0 + j), V, err) * 8, f0);
      vtx(j, f0);
    }
    const int m0 = __ldg(eptr + r), M = __ldg(eptr + r + 1) - m0;
    const float2* dd = cedf + 3 * (size_t)m0;
    auto edg = [&](int jj, const float4& h01, const float4& h23) {
      const float hh[4] = {h01.x, h01.z, h23.x, h23.z}, hl[4] = {h01.y, h01.w, h23.y, h23.w};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 dk = __ldg(dd + (size_t)k * M + jj);
#pragma unroll
        for (int q = 0; q < 4; ++q) df_fma(sh[4 * k + q], sl[4 * k + q], dk.x, dk.y, hh[q], hl[q]);
      }
    };
    j = lane;
    for (; j + G < M; j += 2 * G) {
      const int e0 = chk_idx(ld_stream(eidx + m0 + j), Ef, err), e1 = chk_idx(ld_stream(eidx + m0 + j + G), Ef, err);
      const float4* p0 = reinterpret_cast<const float4*>(hdf + (size_t)e0 * 8);
      const float4* p1 = reinterpret_cast<const float4*>(hdf + (size_t)e1 * 8);
      const float4 a0 = __ldg(p0), a1 = __ldg(p0 + 1), b0 = __ldg(p1), b1 = __ldg(p1 + 1);
      edg(j, a0, a1);
      edg(j + G, b0, b1);
    }
    if (j < M) {
      const float4* p0 = reinterpret_cast<const float4*>(hdf + (size_t)chk_idx(ld_stream(eidx + m0 + j), Ef, err) * 8);
      edg(j, __ldg(p0), __ldg(p0 + 1));
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = f2d_exact(sh[k]) + f2d_exact(sl[k]);
    if (lane == 0) {          // the centre-vertex term, once per vertex
      const double* sg = sig + 6 * (size_t)r;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double sF = __ldg(sg + 2 * k), sG = __ldg(sg + 2 * k + 1);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[4 * k + q] = __fma_rn(fc[4 + q], sG, __fma_rn(fc[q], sF, acc[4 * k + q]));
      }
    }
    if (VISC) {
      const double* cz = cvis + 6 * (size_t)n0;
      for (int jv = lane; jv < N; jv += G) {
        const int u = chk_idx(ld_stream(vidx + n0 + jv), V, err);
        double fv[8];
        ld8(FGv + (size_t)u * 8, fv);
        const double c0f = ld_stream(cz + jv), c0g = ld_stream(cz + N + jv), cxf = ld_stream(cz + 2 * N + jv);
        const double cxg = ld_stream(cz + 3 * N + jv), cyf = ld_stream(cz + 4 * N + jv), cyg = ld_stream(cz + 5 * N + jv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q] = fma(-c0g, fv[4 + q], fma(-c0f, fv[q], acc[q]));
          acc[4 + q] = fma(-cxg, fv[4 + q], fma(-cxf, fv[q], acc[4 + q]));
          acc[8 + q] = fma(-cyg, fv[4 + q], fma(-cyf, fv[q], acc[8 + q]));
        }
      }
    }
  }
  div_finish<double, G>(r, lane, live, acc, V, sa, vmem, dtbits, cfl, dt_last, err);
}

template <int G, bool VISC>
__global__ void __launch_bounds__(256, 2) k_div_df(int A, int V, int Ef, const int32_t* __restrict__ vptr,
                                                   const int32_t* __restrict__ vidx,
                                                   const int32_t* __restrict__ eptr,
                                                   const int32_t* __restrict__ eidx,
                                                   const float2* __restrict__ cvdf,
                                                   const float2* __restrict__ cedf,
                                                   const double* __restrict__ sig,
                                                   const double* __restrict__ cvis,
                                                   const double* __restrict__ FG,
                                                   const double* __restrict__ FGv,
                                                   const float* __restrict__ hdf, StageArgs sa,
                                                   const int32_t* __restrict__ vmem,
                                                   const unsigned long long* dtbits, double cfl,
                                                   double* dt_last, unsigned* err) {
  div_body_df<G, VISC>(blockIdx.x * blockDim.x + threadIdx.x, A, V, Ef, vptr, vidx, eptr, eidx, cvdf,
                    cedf, sig, cvis, FG, FGv, hdf, sa, vmem, dtbits, cfl, dt_last, err);
}

// ------------------------------------------------------------------ k_div_staged (FP32 bulk)
// The FP32 divergence with its streamed operands staged in shared memory by the Tensor Memory
// Accelerator's 1D bulk copies.  About four fifths of the FP32 divergence's bytes are the
// per-vertex index and coefficient chunks, contiguous over consecutive vertices.  The kernel
// is persistent and warp-specialised: each block walks tiles of consecutive active vertices
// (host-built, so that a tile's chunks fit one stage buffer).  One producer thread keeps up to
// kStages tiles in flight -- it waits until the consumers have released a stage buffer (its
// "empty" mbarrier), then copies the tile's row pointers, index chunks and coefficient chunks
// into it with bulk copies completing on the stage's "full" mbarrier.  Eight consumer warps
// compute one tile per stage (8 lanes per vertex) and release the buffer warp by warp, so no
// block-wide barrier couples them and a warp that finishes early starts on the next staged
// tile.  The flux gathers stay direct loads (they hit L2), and each lane loads the state
// values of its stage update before its gathers, so that both latencies overlap.  Per vertex
// the arithmetic, its order and the reduction are those of div_gather_chunked / div_finish
// with 8 lanes per vertex: results equal the unstaged kernel's at that lane count bit for bit.
constexpr int kStageG = 8;                                  // lanes per vertex
constexpr int kStageCW = 8;                                 // consumer warps
constexpr int kStageThreads = 32 * (kStageCW + 1);          // + one producer warp
constexpr unsigned kMbarPolls = 1u << 22;                   // bound of an mbarrier wait
static_assert(kStageCW * 32 / kStageG == kStageTileVerts, "one group of lanes per tile vertex");

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// 1D bulk copy global -> shared, completing `bytes` transactions on `bar` (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Bounded wait for the phase of `bar` with parity `parity`; false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = smem_addr(bar);
  for (unsigned i = 0; i < kMbarPolls; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Byte layout of one staged tile: two row-pointer slots (vptr and eptr from the 16-byte aligned
// vertex pb = r0 & ~3 on), index chunks, vertex coefficient chunks (6 float4 rows), viscous
// chunks, edge index chunks, edge coefficient chunks (3 float4 rows).
struct TileLayout {
  unsigned vi, cv, cz, ei, ce, total;
};
__device__ __forceinline__ TileLayout tile_layout(int nvc, int nec, bool visc) {
  TileLayout L;
  L.vi = 2u * kStagePtrSlot;
  L.cv = L.vi + 16u * nvc;
  L.cz = L.cv + 96u * nvc;
  L.ei = L.cz + (visc ? 96u * nvc : 0u);
  L.ce = L.ei + 16u * nec;
  L.total = L.ce + 48u * nec;
  return L;
}

// meta: per tile {r0, r1, c0, nvc} {m0, nec, pb, 0} (first and end vertex, first vertex chunk
// and count, first edge chunk and count, first vertex of the row-pointer copies)
template <bool VISC>
__global__ void __launch_bounds__(kStageThreads) k_div_staged(
    int A, int V, int Ef, int ntiles, const int4* __restrict__ meta,
    const int32_t* __restrict__ vptr, const int32_t* __restrict__ vidx,
    const int32_t* __restrict__ eptr, const int32_t* __restrict__ eidx,
    const float* __restrict__ cv, const float* __restrict__ ce, const float* __restrict__ cvis,
    const float* __restrict__ FG, const float* __restrict__ FGv, const float* __restrict__ h,
    StageArgs sa, const int32_t* __restrict__ vmem, const unsigned long long* dtbits, double cfl,
    double* dt_last, unsigned* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full[kStages], empty[kStages];
  __shared__ int4 smeta[kStages][2];
  const int warp = threadIdx.x / 32;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kStageCW);
    }
    mbar_init_fence();
  }
  __syncthreads();
  if (warp == kStageCW) {
    // ---- producer: one thread
    if (threadIdx.x % 32 != 0) return;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int st = k % kStages, n = k / kStages;
      if (n > 0 && !mbar_wait(&empty[st], (n - 1) & 1)) {
        atomicOr(err, ERRBIT_TIMEOUT);
        return;
      }
      const int4 a = __ldg(meta + 2 * t), b = __ldg(meta + 2 * t + 1);
      smeta[st][0] = a;
      smeta[st][1] = b;
      const int nseg = (a.y + 1 - b.z + 3) & ~3;           // row pointers pb .. r1, whole int4s
      const TileLayout L = tile_layout(a.w, b.y, VISC);
      unsigned char* buf = smem + st * kStageTileBytes;
      unsigned long long* bar = &full[st];
      mbar_expect_tx(bar, 8u * nseg + (L.total - 2u * kStagePtrSlot));
      bulk_g2s(buf, vptr + b.z, 4u * nseg, bar);
      bulk_g2s(buf + kStagePtrSlot, eptr + b.z, 4u * nseg, bar);
      bulk_g2s(buf + L.vi, vidx + 4 * (size_t)a.z, 16u * a.w, bar);
      bulk_g2s(buf + L.cv, cv + 24 * (size_t)a.z, 96u * a.w, bar);
      if (VISC) bulk_g2s(buf + L.cz, cvis + 24 * (size_t)a.z, 96u * a.w, bar);
      if (b.y > 0) {
        bulk_g2s(buf + L.ei, eidx + 4 * (size_t)b.x, 16u * b.y, bar);
        bulk_g2s(buf + L.ce, ce + 12 * (size_t)b.x, 48u * b.y, bar);
      }
    }
    return;
  }
  // ---- consumers: 8 lanes per vertex, one tile per stage
  const int ct = threadIdx.x;
  const int lane = ct % kStageG;
  const int vloc = ct / kStageG;
  // rows this lane holds after the 8-lane reduce-scatter (as in div_finish)
  const int per = (lane & 1) ? 1 : 2;
  const int base = ((lane & 4) ? 6 : 0) + ((lane & 2) ? 3 : 0) + ((lane & 1) ? 2 : 0);
  const bool stage_mode = sa.mode == DIV_STAGE;
  int k = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const int st = k % kStages, n = k / kStages;
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[st], n & 1));
    if (!ok) {                     // a copy that never completed: report it and leave
      if ((ct & 31) == 0) atomicOr(err, ERRBIT_TIMEOUT);
      return;
    }
    const int4 ma = smeta[st][0], mb = smeta[st][1];
    const int r0 = ma.x, r1 = ma.y, c0 = ma.z, m0 = mb.x, pb = mb.z;
    const int r = r0 + vloc;
    const bool live = r < r1;
    double us[2] = {0.0, 0.0}, un[2] = {0.0, 0.0};
    if (live && stage_mode) {      // state values of the stage update, loaded early
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        if (i >= per) break;
        const size_t idx = (size_t)(base + i) * V + r;
        us[i] = sa.Us[idx];
        if (sa.a != 0.0) un[i] = sa.Un[idx];
      }
    }
    const unsigned char* buf = smem + st * kStageTileBytes;
    const TileLayout L = tile_layout(ma.w, mb.y, VISC);
    const int* s_vp = reinterpret_cast<const int*>(buf);
    const int* s_ep = reinterpret_cast<const int*>(buf + kStagePtrSlot);
    const int4* s_vi = reinterpret_cast<const int4*>(buf + L.vi);
    const float4* s_cv = reinterpret_cast<const float4*>(buf + L.cv);
    const float4* s_cz = reinterpret_cast<const float4*>(buf + L.cz);
    const int4* s_ei = reinterpret_cast<const int4*>(buf + L.ei);
    const float4* s_ce = reinterpret_cast<const float4*>(buf + L.ce);
    float acc[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[q] = 0.f;
    if (live) {
      const int lc0 = s_vp[r - pb] - c0, nc = s_vp[r + 1 - pb] - c0 - lc0;
      for (int ch = lane; ch < nc; ch += kStageG) {
        const int lc = lc0 + ch;
        const int4 u = s_vi[lc];
        float4 kk[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) kk[i] = s_cv[6 * lc + i];
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          float f[8];
          ld8(FG + (size_t)chk_idx(i4c(u, q4), V, err) * 8, f);
          const float c0f = f4c(kk[0], q4), c0g = f4c(kk[1], q4), cxf = f4c(kk[2], q4);
          const float cxg = f4c(kk[3], q4), cyf = f4c(kk[4], q4), cyg = f4c(kk[5], q4);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            acc[q] = fmaf(c0g, f[4 + q], fmaf(c0f, f[q], acc[q]));
            acc[4 + q] = fmaf(cxg, f[4 + q], fmaf(cxf, f[q], acc[4 + q]));
            acc[8 + q] = fmaf(cyg, f[4 + q], fmaf(cyf, f[q], acc[8 + q]));
          }
        }
        if (VISC) {
#pragma unroll
          for (int i = 0; i < 6; ++i) kk[i] = s_cz[6 * lc + i];
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            float f[8];
            ld8(FGv + (size_t)chk_idx(i4c(u, q4), V, err) * 8, f);
            const float c0f = f4c(kk[0], q4), c0g = f4c(kk[1], q4), cxf = f4c(kk[2], q4);
            const float cxg = f4c(kk[3], q4), cyf = f4c(kk[4], q4), cyg = f4c(kk[5], q4);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc[q] = fmaf(-c0g, f[4 + q], fmaf(-c0f, f[q], acc[q]));
              acc[4 + q] = fmaf(-cxg, f[4 + q], fmaf(-cxf, f[q], acc[4 + q]));
              acc[8 + q] = fmaf(-cyg, f[4 + q], fmaf(-cyf, f[q], acc[8 + q]));
            }
          }
        }
      }
      const int le0 = s_ep[r - pb] - m0, mc = s_ep[r + 1 - pb] - m0 - le0;
      for (int ch = lane; ch < mc; ch += kStageG) {
        const int le = le0 + ch;
        const int4 e = s_ei[le];
        const float4 d0 = s_ce[3 * le], dx = s_ce[3 * le + 1], dy = s_ce[3 * le + 2];
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          float hv[4];
          ld4(h + (size_t)chk_idx(i4c(e, q4), Ef, err) * 4, hv);
          const float a0 = f4c(d0, q4), ax = f4c(dx, q4), ay = f4c(dy, q4);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            acc[q] = fmaf(a0, hv[q], acc[q]);
            acc[4 + q] = fmaf(ax, hv[q], acc[4 + q]);
            acc[8 + q] = fmaf(ay, hv[q], acc[8 + q]);
          }
        }
      }
    }
    // this warp is done with the stage buffer
    __syncwarp();
    if ((ct & 31) == 0) mbar_arrive(&empty[st]);
    // combine the 8 lanes and write (the arithmetic of div_finish, on the preloaded state)
    reduce_scatter12<kStageG>(acc, lane);
    if (!live) continue;
    const int mem = vmem ? __ldg(vmem + r) : 0;
    const double dt = sa.dt_fixed > 0.0 ? sa.dt_fixed
                      : sa.dt_member ? __ldg(sa.dt_member + mem)
                                     : cfl * __longlong_as_double((long long)dtbits[mem]);
    if (stage_mode && lane == 0 && dt_last && (r == 0 || (vmem && __ldg(vmem + r - 1) != mem)))
      dt_last[mem] = dt;
    unsigned bad = 0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (i >= per) break;
      const int row = base + i;
      const double R = -(double)acc[i];
      const size_t idx = (size_t)row * V + r;
      double o;
      if (!stage_mode) {
        o = R;
      } else {
        o = __dmul_rn(sa.b, __fma_rn(dt, R, us[i]));
        if (sa.a != 0.0) o = __fma_rn(sa.a, un[i], o);
      }
      sa.out[idx] = o;
      if (!finite_bits(o)) bad |= ERRBIT_NONFINITE;
      if (stage_mode && row == 0 && !(o > 0.0)) bad |= ERRBIT_POSITIVITY;
    }
    if (bad) atomicOr(err, bad);
  }
}

// ------------------------------------------------------------------ small kernels
// Ghost refresh of state U (R14): a transmissive ghost copies its donor in U and zeroes the
// derivative normal to its boundary; a fixed ghost (donor -1, wall bands holding given values)
// takes its values from the step's base state `base` (nothing to do when U is the base).
__device__ __forceinline__ void ghost_body(int g, int Gn, int V, const int32_t* gid,
                                           const int32_t* gdonor, const int32_t* gflags, double* U,
                                           const double* base, unsigned* err) {
  if (g >= Gn) return;
  int t = chk_idx(gid[g], V, err), d = gdonor[g], f = gflags[g];
  if (d >= 0) d = chk_idx(d, V, err);
  if (d < 0) {
    if (base != U)
#pragma unroll
      for (int r = 0; r < 12; ++r) U[(size_t)r * V + t] = base[(size_t)r * V + t];
    return;
  }
#pragma unroll
  for (int r = 0; r < 12; ++r) {
    double val = U[(size_t)r * V + d];
    if ((r >= 4 && r < 8 && (f & 1)) || (r >= 8 && (f & 2))) val = 0.0;
    U[(size_t)r * V + t] = val;
  }
}

__global__ void k_ghost(int Gn, int V, const int32_t* gid, const int32_t* gdonor,
                        const int32_t* gflags, double* U, const double* base, unsigned* err) {
  ghost_body(blockIdx.x * blockDim.x + threadIdx.x, Gn, V, gid, gdonor, gflags, U, base, err);
}

// min over the active vertices of each mesh of l_min / (|u| + c) (R12), in two passes without
// contention on one address.  Pass 1: each block of 256 vertices reduces through warp shuffles
// and shared memory; a block inside one mesh writes its minimum to partial[block], a block that
// straddles meshes (batches only) updates the meshes' minima directly with atomicMin.  Pass 2:
// one block reduces the partial minima; if they all belong to one mesh (always, for a single
// mesh) with one atomicMin, else each thread scans a contiguous run of blocks and issues one
// atomicMin per mesh it meets.  Positive doubles order like their bit patterns, so the result
// does not depend on the order of the atomics.
__global__ void __launch_bounds__(256) k_dtmin(int A, int V, const double* __restrict__ U,
                                               const double* __restrict__ lmin,
                                               const int32_t* __restrict__ vmem, double gamma,
                                               unsigned long long* bits, double* partial) {
  __shared__ double wmin[8];
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  double val = INFINITY;
  if (v < A) {
    // lmin / (|u| + c) = lmin rho / (|m| + sqrt(gamma (gamma-1) (E rho - |m|^2 / 2))): one
    // division instead of three (rho c = sqrt(gamma p rho), p rho = (gamma-1)(E rho - |m|^2/2))
    double rho = U[v], m = U[(size_t)V + v], n = U[2 * (size_t)V + v], E = U[3 * (size_t)V + v];
    double q = m * m + n * n;
    double sr = sqrt(q) + sqrt(gamma * (gamma - 1.0) * (E * rho - 0.5 * q));
    val = lmin[v] * rho / sr;
    if (!(val > 0.0)) val = INFINITY;   // non-physical states do not set the step
  }
  int first = blockIdx.x * blockDim.x, last = min(A - 1, first + (int)blockDim.x - 1);
  bool uniform = !vmem || vmem[first] == vmem[last];
  if (!uniform) {
    if (threadIdx.x == 0) partial[blockIdx.x] = INFINITY;
    int mem = v < A ? vmem[v] : -1;
    if (mem >= 0 && val < INFINITY) atomicMin(bits + mem, (unsigned long long)__double_as_longlong(val));
    return;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) val = fmin(val, __shfl_xor_sync(0xffffffffu, val, off));
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = val;
  __syncthreads();
  if (threadIdx.x < 32) {
    val = threadIdx.x < (blockDim.x >> 5) ? wmin[threadIdx.x] : INFINITY;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) val = fmin(val, __shfl_xor_sync(0xffffffffu, val, off));
    if (threadIdx.x == 0) partial[blockIdx.x] = val;
  }
}

__global__ void __launch_bounds__(1024) k_dtmin_final(int nblk, int A, const int32_t* __restrict__ vmem,
                                                      const double* __restrict__ partial,
                                                      unsigned long long* bits) {
  __shared__ double wmin[32];
  const int bs = 256;                                       // vertices per pass-1 block
  bool one_mesh = !vmem || vmem[0] == vmem[A - 1];
  if (one_mesh) {
    double val = INFINITY;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) val = fmin(val, partial[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) val = fmin(val, __shfl_xor_sync(0xffffffffu, val, off));
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = val;
    __syncthreads();
    if (threadIdx.x < 32) {
      val = threadIdx.x < (blockDim.x >> 5) ? wmin[threadIdx.x] : INFINITY;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) val = fmin(val, __shfl_xor_sync(0xffffffffu, val, off));
      if (threadIdx.x == 0 && val < INFINITY)
        atomicMin(bits + (vmem ? vmem[0] : 0), (unsigned long long)__double_as_longlong(val));
    }
    return;
  }
  int per = (nblk + blockDim.x - 1) / blockDim.x;
  int b0 = threadIdx.x * per, b1 = min(nblk, b0 + per);
  int cur = -1;
  double val = INFINITY;
  for (int b = b0; b < b1; ++b) {
    int mem = vmem[b * bs];
    if (mem != cur) {
      if (cur >= 0 && val < INFINITY) atomicMin(bits + cur, (unsigned long long)__double_as_longlong(val));
      cur = mem;
      val = INFINITY;
    }
    val = fmin(val, partial[b]);
  }
  if (cur >= 0 && val < INFINITY) atomicMin(bits + cur, (unsigned long long)__double_as_longlong(val));
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

// ------------------------------------------------------------------ persistent stage kernel
// One cooperative launch per Runge-Kutta stage: ghost refresh, vertex fluxes, edge fluxes and
// divergence + stage update run as phases of one grid, separated by grid-wide barriers.  The
// launch is cooperative, so all blocks are resident.  Every barrier wait is bounded: a block that
// waits longer than kBarrierSpins polls records HFD_ERR_TIMEOUT in the error word and leaves the
// kernel, and the blocks waiting for it at later barriers time out in turn, so the kernel always
// ends.  Each phase runs the same per-entity code as the separate kernels (results agree with the
// four-launch path to rounding: multiply-adds may be contracted differently when fused).  The poll bound is a launch argument (default 2^24 polls of
// >= 64 ns, i.e. about a second or more).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* err,
                                             unsigned max_spins) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = bar + 1;
    unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned spins = 0;
      while (*gen == g) {
        if (++spins > max_spins) {
          atomicOr(err, ERRBIT_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T, int G, bool VISC>
__global__ void __launch_bounds__(128) k_stage(KernelArgs ka, StageArgs sa, Phys ph, int do_ghost) {
  const unsigned nb = gridDim.x;
  const int stride = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double* U = const_cast<double*>(sa.Us);
  if (do_ghost) {
    for (int g = tid; g < ka.G; g += stride)
      ghost_body(g, ka.G, ka.V, ka.gid, ka.gdonor, ka.gflags, U, sa.Un, ka.err);
    if (!grid_barrier(ka.bar, nb, ka.err, ka.spins)) return;
  }
  __shared__ float s0f[4];
  __shared__ double s0d[4];
  if constexpr (std::is_same<T, float>::value) block_reference(sa.Us, ka.V, s0f, s0d);
  for (int v = tid; v < ka.V; v += stride)
    vertex_body<T, VISC>(v, ka.V, sa.Us, (T*)ka.Ua, (T*)ka.FG, (T*)ka.FGv, ph, ka.wref, s0f, s0d);
  if (!grid_barrier(ka.bar, nb, ka.err, ka.spins)) return;
  const double* FGd = nullptr;
  if constexpr (std::is_same<T, double>::value) FGd = ka.div_df ? (const double*)ka.FG : nullptr;
  for (int e = tid; e < ka.Ef; e += stride)
    edge_body<T>(e, ka.Ef, ka.V, ka.sten, (const T*)ka.nrm, (const T*)ka.w5, (const T*)ka.w3,
                 (const T*)ka.Ua, (T*)ka.h, ph, ka.err, nullptr, ka.wref, FGd);
  if (!grid_barrier(ka.bar, nb, ka.err, ka.spins)) return;
  if constexpr (std::is_same<T, double>::value) {
    if (ka.div_df) {        // folded double-float divergence, one lane per vertex
      for (int r = tid; r < ka.A; r += stride)
        div_body_df<1, VISC>(r, ka.A, ka.V, ka.Ef, ka.vptr, ka.vidx, ka.eptr, ka.eidx,
                          (const float2*)ka.cvdf, (const float2*)ka.cedf, ka.sig,
                          (const double*)ka.cvis, (const double*)ka.FG, (const double*)ka.FGv,
                          (const float*)ka.h, sa, ka.vmem, ka.dtbits, ph.cfl, ka.dt_last, ka.err);
      return;
    }
  }
  // every lane of a warp runs the same number of iterations (shuffles inside div_body)
  const long long total = (long long)ka.A * G;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride)
    div_body<T, G, VISC>((int)(base + threadIdx.x), ka.A, ka.V, ka.Ef, ka.vptr, ka.vidx, ka.eptr, ka.eidx,
                         (const T*)ka.cv, (const T*)ka.ce, (const T*)ka.cvis, (const T*)ka.FG,
                         (const T*)ka.FGv, (const T*)ka.h, sa, ka.vmem, ka.dtbits, ph.cfl,
                         ka.dt_last, ka.err);
}

// ------------------------------------------------------------------ launchers
static inline int blocks(long long n, int b) { return (int)((n + b - 1) / b); }

KernelArgs kernel_args(const DevMesh& m) {
  KernelArgs a;
  a.V = m.V; a.A = m.A; a.Ef = m.Ef; a.G = m.G;
  a.sten = m.sten; a.vptr = m.vptr; a.vidx = m.vidx; a.eptr = m.eptr; a.eidx = m.eidx;
  a.gid = m.gid; a.gdonor = m.gdonor; a.gflags = m.gflags; a.vmem = m.vmem;
  a.nrm = m.nrm; a.w5 = m.w5; a.w3 = m.w3; a.cv = m.cv; a.ce = m.ce; a.cvis = m.cvis;
  a.Ua = m.Ua; a.FG = m.FG; a.FGv = m.FGv; a.h = m.h;
  a.dtbits = m.dtbits; a.dt_last = m.dt_last; a.err = m.err; a.bar = m.bar; a.wref = m.wref;
  a.div_df = m.div_df; a.cvdf = m.cvdf; a.cedf = m.cedf; a.sig = m.sig;
  a.spins = m.barrier_spins;
  return a;
}

cudaError_t launch_ghost(const DevMesh& m, double* U, const double* base, cudaStream_t s) {
  if (m.G == 0) return cudaSuccess;
  k_ghost<<<blocks(m.G, 256), 256, 0, s>>>(m.G, m.V, m.gid, m.gdonor, m.gflags, U, base, m.err);
  return cudaGetLastError();
}

cudaError_t launch_vertex(const DevMesh& m, const double* U, const Phys& ph, cudaStream_t s) {
  int nb = blocks(m.V, 256);
  if (m.precision == 0) {
    if (m.viscous)
      k_vertex<double, true><<<nb, 256, 0, s>>>(m.V, U, (double*)m.Ua, (double*)m.FG,
                                                (double*)m.FGv, ph, nullptr);
    else
      k_vertex<double, false><<<nb, 256, 0, s>>>(m.V, U, (double*)m.Ua, (double*)m.FG, nullptr, ph,
                                                 nullptr);
  } else {
    if (m.viscous)
      k_vertex<float, true><<<nb, 256, 0, s>>>(m.V, U, (float*)m.Ua, (float*)m.FG, (float*)m.FGv, ph,
                                               m.wref);
    else
      k_vertex<float, false><<<nb, 256, 0, s>>>(m.V, U, (float*)m.Ua, (float*)m.FG, nullptr, ph,
                                                m.wref);
  }
  return cudaGetLastError();
}

cudaError_t launch_edge(const DevMesh& m, const Phys& ph, cudaStream_t s) {
  if (m.Ef == 0) return cudaSuccess;
  int nb = blocks(m.Ef, 128);
  if (m.precision == 0)
    k_edge<double><<<nb, 128, 0, s>>>(m.Ef, m.V, m.sten, (const double*)m.nrm, (const double*)m.w5,
                                      (const double*)m.w3, (const double*)m.Ua, (double*)m.h, ph,
                                      m.err, m.dbg_branch, nullptr,
                                      m.div_df ? (const double*)m.FG : nullptr);
  else
    k_edge<float><<<nb, 128, 0, s>>>(m.Ef, m.V, m.sten, (const float*)m.nrm, (const float*)m.w5,
                                     (const float*)m.w3, (const float*)m.Ua, (float*)m.h, ph, m.err,
                                     m.dbg_branch, m.wref, nullptr);
  return cudaGetLastError();
}

template <typename T, int G>
static void div_dispatch(const DevMesh& m, const StageArgs& sa, const Phys& ph, cudaStream_t s) {
  long long threads = (long long)m.A * G;
  int nb = blocks(threads, 256);
  if (m.viscous)
    k_div<T, G, true><<<nb, 256, 0, s>>>(m.A, m.V, m.Ef, m.vptr, m.vidx, m.eptr, m.eidx, (const T*)m.cv,
                                         (const T*)m.ce, (const T*)m.cvis, (const T*)m.FG,
                                         (const T*)m.FGv, (const T*)m.h, sa, m.vmem, m.dtbits,
                                         ph.cfl, m.dt_last, m.err);
  else
    k_div<T, G, false><<<nb, 256, 0, s>>>(m.A, m.V, m.Ef, m.vptr, m.vidx, m.eptr, m.eidx,
                                          (const T*)m.cv, (const T*)m.ce, nullptr, (const T*)m.FG,
                                          nullptr, (const T*)m.h, sa, m.vmem, m.dtbits, ph.cfl,
                                          m.dt_last, m.err);
}

// Staged FP32 divergence: a persistent grid of every co-resident block (kStages stage buffers
// of dynamic shared memory each), at most one block per tile.
template <bool VISC>
static cudaError_t div_staged_launch(const DevMesh& m, const StageArgs& sa, const Phys& ph,
                                     cudaStream_t s) {
  static int per_sm[2] = {0, 0}, nsm = 0;            // per process; one GPU model per process
  const int smem = kStages * kStageTileBytes;
  if (!per_sm[VISC]) {
    cudaError_t e = cudaFuncSetAttribute(k_div_staged<VISC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int b = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_div_staged<VISC>, kStageThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm[VISC] = b > 0 ? b : 1;
  }
  const int grid = (int)std::min<long long>((long long)per_sm[VISC] * nsm, m.ntiles);
  k_div_staged<VISC><<<grid, kStageThreads, smem, s>>>(
      m.A, m.V, m.Ef, m.ntiles, reinterpret_cast<const int4*>(m.tiles), m.vptr, m.vidx, m.eptr,
      m.eidx, (const float*)m.cv, (const float*)m.ce, (const float*)m.cvis, (const float*)m.FG,
      (const float*)m.FGv, (const float*)m.h, sa, m.vmem, m.dtbits, ph.cfl, m.dt_last, m.err);
  return cudaGetLastError();
}

cudaError_t prepare_div_gs(int smem_bytes) {
  if (smem_bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k_div_gs, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
}

cudaError_t launch_div(const DevMesh& m, const double* Us, const double* Un, double* out, int mode,
                       double a, double b, double dt_fixed, const Phys& ph, int lanes,
                       cudaStream_t s, const double* dt_member) {
  if (m.A == 0) return cudaSuccess;
  StageArgs sa{Us, Un, out, mode, a, b, dt_fixed, dt_member};
  if (m.precision == 0 && m.div_df) {
    constexpr int G = kDfLanes;
    const int nb = blocks((long long)m.A * G, 256);
    if (m.viscous)
      k_div_df<G, true><<<nb, 256, 0, s>>>(m.A, m.V, m.Ef, m.vptr, m.vidx, m.eptr, m.eidx,
                                        (const float2*)m.cvdf, (const float2*)m.cedf, m.sig,
                                        (const double*)m.cvis, (const double*)m.FG,
                                        (const double*)m.FGv, (const float*)m.h, sa, m.vmem,
                                        m.dtbits, ph.cfl, m.dt_last, m.err);
    else
      k_div_df<G, false><<<nb, 256, 0, s>>>(m.A, m.V, m.Ef, m.vptr, m.vidx, m.eptr, m.eidx,
                                         (const float2*)m.cvdf, (const float2*)m.cedf, m.sig,
                                         nullptr, (const double*)m.FG, nullptr,
                                         (const float*)m.h, sa, m.vmem, m.dtbits, ph.cfl,
                                         m.dt_last, m.err);
  } else if (m.precision == 0) {
    switch (lanes) {
      case 1: div_dispatch<double, 1>(m, sa, ph, s); break;
      case 2: div_dispatch<double, 2>(m, sa, ph, s); break;
      case 8: div_dispatch<double, 8>(m, sa, ph, s); break;
      default: div_dispatch<double, 4>(m, sa, ph, s); break;
    }
  } else if (m.div_staged == 2 && m.gs_ntiles > 0) {
    k_div_gs<<<m.gs_ntiles, kGsRows * kGsLanes, m.gs_smem, s>>>(
        m.A, m.V, m.Ef, m.vptr, reinterpret_cast<const ushort4*>(m.lvidx), m.eptr,
        reinterpret_cast<const ushort4*>(m.leidx), (const float*)m.cv, (const float*)m.ce,
        (const float*)m.FG, (const float*)m.h, m.gtv_ptr, m.gtv, m.gte_ptr, m.gte, sa, m.vmem,
        m.dtbits, ph.cfl, m.dt_last, m.err);
  } else if (m.div_staged == 1 && m.ntiles > 0) {
    return m.viscous ? div_staged_launch<true>(m, sa, ph, s) : div_staged_launch<false>(m, sa, ph, s);
  } else {
    switch (lanes) {
      case 1: div_dispatch<float, 1>(m, sa, ph, s); break;
      case 2: div_dispatch<float, 2>(m, sa, ph, s); break;
      case 8: div_dispatch<float, 8>(m, sa, ph, s); break;
      default: div_dispatch<float, 4>(m, sa, ph, s); break;
    }
  }
  return cudaGetLastError();
}

template <typename T, int G, bool VISC>
static const void* stage_fn() {
  return reinterpret_cast<const void*>(&k_stage<T, G, VISC>);
}

static const void* pick_stage_fn(const DevMesh& m, int lanes) {
  if (m.precision == 0) {
    if (m.viscous) return lanes == 1 ? stage_fn<double, 1, true>() : lanes == 2 ? stage_fn<double, 2, true>() : stage_fn<double, 4, true>();
    return lanes == 1 ? stage_fn<double, 1, false>() : lanes == 2 ? stage_fn<double, 2, false>() : stage_fn<double, 4, false>();
  }
  if (m.viscous) return lanes == 1 ? stage_fn<float, 1, true>() : lanes == 2 ? stage_fn<float, 2, true>() : stage_fn<float, 4, true>();
  return lanes == 1 ? stage_fn<float, 1, false>() : lanes == 2 ? stage_fn<float, 2, false>() : stage_fn<float, 4, false>();
}

cudaError_t persistent_max_blocks(const DevMesh& m, int lanes, int* per_sm, int* nsm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, pick_stage_fn(m, lanes), 128, 0);
  return e;
}

cudaError_t launch_stage_persistent(const DevMesh& m, const double* Us, const double* Un,
                                    double* out, int mode, double a, double b, double dt_fixed,
                                    const Phys& ph, int lanes, int grid, bool do_ghost,
                                    cudaStream_t s, const double* dt_member) {
  KernelArgs ka = kernel_args(m);
  StageArgs sa{Us, Un, out, mode, a, b, dt_fixed, dt_member};
  Phys p = ph;
  int dg = do_ghost && m.G > 0 ? 1 : 0;
  void* args[] = {&ka, &sa, &p, &dg};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(128);
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, pick_stage_fn(m, lanes), args);
}

cudaError_t launch_dtmin(const DevMesh& m, const double* U, const Phys& ph, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(m.dtbits, 0xff, sizeof(unsigned long long) * m.nmember, s);
  if (e != cudaSuccess) return e;
  if (m.A == 0) return cudaSuccess;
  int nb = blocks(m.A, 256);
  k_dtmin<<<nb, 256, 0, s>>>(m.A, m.V, U, m.lmin, m.vmem, ph.gamma, m.dtbits, m.dtpartial);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_dtmin_final<<<1, 1024, 0, s>>>(nb, m.A, m.vmem, m.dtpartial, m.dtbits);
  return cudaGetLastError();
}

// One thread per (row, vertex) of the batch array; the member is found by binary search of
// the offsets.
__global__ void k_batch_copy(int V, int n, const int64_t* __restrict__ off,
                             double* const* __restrict__ ptrs, double* __restrict__ U,
                             int to_batch) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 12LL * V) return;
  const int r = (int)(i / V), v = (int)(i - (long long)r * V);
  int lo = 0, hi = n;                       // off[lo] <= v < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= v) lo = mid; else hi = mid;
  }
  const long long nvk = __ldg(off + lo + 1) - __ldg(off + lo);
  double* p = ptrs[lo] + (size_t)r * nvk + (v - __ldg(off + lo));
  if (to_batch) U[i] = *p; else *p = U[i];
}

cudaError_t launch_batch_copy(int V, int n, const int64_t* off, double* const* ptrs, double* U,
                              bool to_batch, cudaStream_t s) {
  if (V == 0) return cudaSuccess;
  k_batch_copy<<<blocks(12LL * V, 256), 256, 0, s>>>(V, n, off, ptrs, U, to_batch ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_permute(int V, const int32_t* perm, const double* src, double* dst, bool gather,
                           cudaStream_t s) {
  k_permute<<<blocks(V, 256), 256, 0, s>>>(V, perm, src, dst, gather ? 1 : 0);
  return cudaGetLastError();
}

// The integer-only conversions against the hardware conversions, element by element: x as a
// double rounded to float both ways, and the low 32 bits of x as a float widened both ways.
__global__ void k_conversions(int64_t n, const double* __restrict__ x, float* __restrict__ f_int,
                              float* __restrict__ f_hw, double* __restrict__ d_int,
                              double* __restrict__ d_hw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  f_int[i] = d2f_rn(v);
  f_hw[i] = __double2float_rn(v);
  const float f = __uint_as_float((unsigned)(unsigned long long)__double_as_longlong(v));
  d_int[i] = f2d_exact(f);
  d_hw[i] = (double)f;
}

cudaError_t launch_conversions(int64_t n, const double* x, float* f_int, float* f_hw, double* d_int,
                               double* d_hw, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_conversions<<<(unsigned)blocks, 256, 0, s>>>(n, x, f_int, f_hw, d_int, d_hw);
  return cudaGetLastError();
}

}  // namespace hfd
