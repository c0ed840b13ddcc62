// CUDA kernels (sm_103a) of the three-dimensional extension of the Hermite FD residual and
// SSP-RK3 step; FP64 state, fluxes and sums.  Per Runge-Kutta stage:
//   k3_vertex  one thread per vertex: the vertex-major copy of the 20 unknowns and the analytic
//              flux vectors F, G, K (Sec. 2.3, vertex fluxes, in 3D);
//   k3_edge    one thread per edge: Alg. 1 in 3D (Roe average of the edge ends, five-wave
//              characteristic projection along the edge, uniform WENO5 weights as the sensor --
//              taken in FP32 and again in FP64 inside a band around each threshold -- 5-node
//              Hermite value or weighted 3-node value per component and side,
//              back-projection, positivity fallback) and Roe's flux with Harten's fix;
//   k3_div     1, 2 or 4 lanes per vertex: the CSR gather of the least-squares divergence rows
//              d_0, d_x, d_y, d_z over the vertex fluxes and edge fluxes (Eq.
//              (flux_polynomials) in 3D), fused with the SSP-RK3 stage update.
// The characteristic projection uses the closed forms of the left and right eigenvectors of
// the flux Jacobian along n with the frame (n, t1, t2): waves q_n - c, entropy, shear along
// t1, shear along t2, q_n + c.
#include <cuda_runtime.h>

#include "fp_convert.cuh"
#include "kernels3d.hpp"

namespace hfd {
namespace {

constexpr unsigned kErrNonfinite = 1u, kErrPositivity = 2u, kErrIndex = 4u;

__device__ __forceinline__ bool finite3(double x) { return isfinite(x); }

// The eigen-structure of one Roe state along the frame (n, t1, t2), and the two states'
// reciprocal densities and pressures (shared with the normal fluxes).
struct Eig {
  double u[3], H, c, qn, q1, q2, K, b1, b2, ic;
  double n[3], t1[3], t2[3];
  double irl, irr, pl, pr;
};

// One reciprocal square root per state gives sqrt(rho) and 1/rho, one more gives c and 1/c
// (the CUDA math library's rsqrt); one division forms the Roe weights.
__device__ __forceinline__ void roe_state(const double* wl, const double* wr, double g1, Eig& s) {
  const double sl = rsqrt(wl[0]), sr = rsqrt(wr[0]);
  s.irl = sl * sl;
  s.irr = sr * sr;
  s.pl = g1 * (wl[4] - 0.5 * (wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3]) * s.irl);
  s.pr = g1 * (wr[4] - 0.5 * (wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3]) * s.irr);
  const double is = 1.0 / (wl[0] * sl + wr[0] * sr);
#pragma unroll
  for (int k = 0; k < 3; ++k) s.u[k] = (wl[k + 1] * sl + wr[k + 1] * sr) * is;
  s.H = ((wl[4] + s.pl) * sl + (wr[4] + s.pr) * sr) * is;
  s.K = s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2];
  const double c2 = g1 * (s.H - 0.5 * s.K);
  s.ic = rsqrt(c2);
  s.c = c2 * s.ic;
  s.qn = s.u[0] * s.n[0] + s.u[1] * s.n[1] + s.u[2] * s.n[2];
  s.q1 = s.u[0] * s.t1[0] + s.u[1] * s.t1[1] + s.u[2] * s.t1[2];
  s.q2 = s.u[0] * s.t2[0] + s.u[1] * s.t2[1] + s.u[2] * s.t2[2];
  s.b1 = g1 * s.ic * s.ic;
  s.b2 = 0.5 * s.b1 * s.K;
}

// c = L a for the five conserved components a.
__device__ __forceinline__ void to_char(const Eig& s, const double* a, double* c) {
  const double um = s.u[0] * a[1] + s.u[1] * a[2] + s.u[2] * a[3];
  const double nm = (s.n[0] * a[1] + s.n[1] * a[2] + s.n[2] * a[3]) * s.ic;
  const double t1m = s.t1[0] * a[1] + s.t1[1] * a[2] + s.t1[2] * a[3];
  const double t2m = s.t2[0] * a[1] + s.t2[1] * a[2] + s.t2[2] * a[3];
  const double qc = s.qn * s.ic;
  c[0] = 0.5 * ((s.b2 + qc) * a[0] - s.b1 * um - nm + s.b1 * a[4]);
  c[1] = (1.0 - s.b2) * a[0] + s.b1 * um - s.b1 * a[4];
  c[2] = t1m - s.q1 * a[0];
  c[3] = t2m - s.q2 * a[0];
  c[4] = 0.5 * ((s.b2 - qc) * a[0] - s.b1 * um + nm + s.b1 * a[4]);
}

// w = R c.
__device__ __forceinline__ void from_char(const Eig& s, const double* c, double* w) {
  w[0] = c[0] + c[1] + c[4];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    w[k + 1] = (c[0] + c[1] + c[4]) * s.u[k] + (c[4] - c[0]) * s.c * s.n[k] + c[2] * s.t1[k] +
               c[3] * s.t2[k];
  w[4] = (c[0] + c[4]) * s.H + (c[4] - c[0]) * s.c * s.qn + c[1] * (0.5 * s.K) + c[2] * s.q1 +
         c[3] * s.q2;
}

// The FP32 copy of an eigen-structure for the sensor, rounded by integer operations.
struct EigF {
  float u[3], n[3], t1[3], t2[3], ic, qn, q1, q2, b1, b2;
};

__device__ __forceinline__ void to_f32(const Eig& s, EigF& f) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    f.u[k] = d2f_rn(s.u[k]);
    f.n[k] = d2f_rn(s.n[k]);
    f.t1[k] = d2f_rn(s.t1[k]);
    f.t2[k] = d2f_rn(s.t2[k]);
  }
  f.ic = d2f_rn(s.ic);
  f.qn = d2f_rn(s.qn);
  f.q1 = d2f_rn(s.q1);
  f.q2 = d2f_rn(s.q2);
  f.b1 = d2f_rn(s.b1);
  f.b2 = d2f_rn(s.b2);
}

// c = L a in FP32 (the formulas of to_char).
__device__ __forceinline__ void to_char_f(const EigF& s, const float* a, float* c) {
  const float um = s.u[0] * a[1] + s.u[1] * a[2] + s.u[2] * a[3];
  const float nm = (s.n[0] * a[1] + s.n[1] * a[2] + s.n[2] * a[3]) * s.ic;
  const float t1m = s.t1[0] * a[1] + s.t1[1] * a[2] + s.t1[2] * a[3];
  const float t2m = s.t2[0] * a[1] + s.t2[1] * a[2] + s.t2[2] * a[3];
  const float qc = s.qn * s.ic;
  c[0] = 0.5f * ((s.b2 + qc) * a[0] - s.b1 * um - nm + s.b1 * a[4]);
  c[1] = (1.0f - s.b2) * a[0] + s.b1 * um - s.b1 * a[4];
  c[2] = t1m - s.q1 * a[0];
  c[3] = t2m - s.q2 * a[0];
  c[4] = 0.5f * ((s.b2 - qc) * a[0] - s.b1 * um + nm + s.b1 * a[4]);
}

// rho > 0 and p > 0 (R16): p has the sign of E rho - |m|^2 / 2 when rho > 0.
__device__ __forceinline__ bool admissible3(const double* w) {
  return w[0] > 0.0 && w[4] * w[0] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) > 0.0;
}

// Uniform WENO5 on the five values u0..u4 (Jiang-Shu indicators, linear weights 1/16, 10/16,
// 5/16) with every weight multiplied by (eps+b1)^2 (eps+b2)^2 (eps+b3)^2, so that the sensor
// needs no division: t[i] is weight i times that product and S their sum; omega_i = t[i] / S.
__device__ __forceinline__ void weno3(double u0, double u1, double u2, double u3, double u4,
                                      double eps, double* t, double& S) {
  const double e1 = u0 - 2.0 * u1 + u2, f1 = u0 - 4.0 * u1 + 3.0 * u2;
  const double e2 = u1 - 2.0 * u2 + u3, f2 = u1 - u3;
  const double e3 = u2 - 2.0 * u3 + u4, f3 = 3.0 * u2 - 4.0 * u3 + u4;
  const double b1 = 13.0 / 12.0 * (e1 * e1) + 0.25 * (f1 * f1);
  const double b2 = 13.0 / 12.0 * (e2 * e2) + 0.25 * (f2 * f2);
  const double b3 = 13.0 / 12.0 * (e3 * e3) + 0.25 * (f3 * f3);
  double s1 = eps + b1, s2 = eps + b2, s3 = eps + b3;
  s1 *= s1;
  s2 *= s2;
  s3 *= s3;
  t[0] = (1.0 / 16.0) * (s2 * s3);
  t[1] = (10.0 / 16.0) * (s1 * s3);
  t[2] = (5.0 / 16.0) * (s1 * s2);
  S = t[0] + t[1] + t[2];
}

// weno3 in FP32, for the sensor's first pass.
__device__ __forceinline__ void weno3f(float u0, float u1, float u2, float u3, float u4, float eps,
                                       float& t0, float& S) {
  const float e1 = u0 - 2.0f * u1 + u2, f1 = u0 - 4.0f * u1 + 3.0f * u2;
  const float e2 = u1 - 2.0f * u2 + u3, f2 = u1 - u3;
  const float e3 = u2 - 2.0f * u3 + u4, f3 = 3.0f * u2 - 4.0f * u3 + u4;
  float s1 = eps + (13.0f / 12.0f * (e1 * e1) + 0.25f * (f1 * f1));
  float s2 = eps + (13.0f / 12.0f * (e2 * e2) + 0.25f * (f2 * f2));
  float s3 = eps + (13.0f / 12.0f * (e3 * e3) + 0.25f * (f3 * f3));
  s1 *= s1;
  s2 *= s2;
  s3 *= s3;
  t0 = 0.0625f * (s2 * s3);
  S = t0 + 0.625f * (s1 * s3) + 0.3125f * (s1 * s2);
}

// Relative width of the band around each sensor threshold inside which the FP32 decision is
// taken again in FP64.
constexpr float kGuard3 = 1e-3f;

// F_n(w) from the state, its reciprocal density and its pressure.
__device__ __forceinline__ void normal_flux3(const double* w, double ir, double p, const double* n,
                                             double* f) {
  const double un = (w[1] * n[0] + w[2] * n[1] + w[3] * n[2]) * ir;
  f[0] = w[0] * un;
#pragma unroll
  for (int k = 0; k < 3; ++k) f[k + 1] = w[k + 1] * un + p * n[k];
  f[4] = (w[4] + p) * un;
}

// ------------------------------------------------------------------ k3_vertex
// Ua: 20 values per vertex (160 B); FGK: F, G, K per vertex at a stride of 16 (128 B).
__global__ void __launch_bounds__(256) k3_vertex(int V, const double* __restrict__ U,
                                                 double* __restrict__ Ua, double* __restrict__ FGK,
                                                 double g1) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  double w[20];
#pragma unroll
  for (int r = 0; r < 20; ++r) w[r] = U[(size_t)r * V + v];
  double2* ua = reinterpret_cast<double2*>(Ua + (size_t)20 * v);
#pragma unroll
  for (int i = 0; i < 10; ++i) ua[i] = make_double2(w[2 * i], w[2 * i + 1]);
  const double ir = 1.0 / w[0];
  const double u = w[1] * ir, vv = w[2] * ir, ww = w[3] * ir;
  const double p = g1 * (w[4] - 0.5 * (w[1] * u + w[2] * vv + w[3] * ww));
  const double f[16] = {w[1], w[1] * u + p, w[2] * u, w[3] * u, (w[4] + p) * u,
                        w[2], w[1] * vv, w[2] * vv + p, w[3] * vv, (w[4] + p) * vv,
                        w[3], w[1] * ww, w[2] * ww, w[3] * ww + p, (w[4] + p) * ww, 0.0};
  double2* o = reinterpret_cast<double2*>(FGK + (size_t)16 * v);
#pragma unroll
  for (int i = 0; i < 8; ++i) o[i] = make_double2(f[2 * i], f[2 * i + 1]);
}

// ------------------------------------------------------------------ k3_edge
// One thread per edge.  Stencil ids (6 x E), frame (9 x E), w5 (40 x E) and w3 (18 x E) are
// structure-of-arrays streams; node data are gathered from Ua.  h: 8 doubles per edge (5 used).
__global__ void __launch_bounds__(128) k3_edge(int E, int V, const int32_t* __restrict__ sten,
                                               const double* __restrict__ frame,
                                               const double* __restrict__ w5,
                                               const double* __restrict__ w3,
                                               const double* __restrict__ Ua,
                                               double* __restrict__ h, Phys3 ph,
                                               unsigned* __restrict__ err) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int s[6];
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    s[k] = __ldg(sten + (size_t)k * E + e);
    bad |= (unsigned)s[k] >= (unsigned)V;
  }
  if (bad) {
    atomicOr(err, kErrIndex);
    return;
  }
  const double g1 = ph.g1;
  Eig st;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    st.n[k] = __ldg(frame + (size_t)k * E + e);
    st.t1[k] = __ldg(frame + (size_t)(3 + k) * E + e);
    st.t2[k] = __ldg(frame + (size_t)(6 + k) * E + e);
  }
  double wi[5], wj[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    wi[q] = __ldg(Ua + (size_t)20 * s[2] + q);
    wj[q] = __ldg(Ua + (size_t)20 * s[3] + q);
  }
  roe_state(wi, wj, g1, st);
  // FP32 sensor: characteristic values of the six nodes' differences from the tail state (the
  // WENO indicators see differences only), each difference formed in FP64 and rounded once;
  // and the 5-node sums of both sides in conservative variables, in FP64
  EigF sf;
  to_f32(st, sf);
  float cf[6][5];
  double W[2][5];
#pragma unroll
  for (int q = 0; q < 5; ++q) W[0][q] = W[1][q] = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double a[20];
    const double2* src = reinterpret_cast<const double2*>(Ua + (size_t)20 * s[k]);
#pragma unroll
    for (int i = 0; i < 10; ++i) {
      const double2 t = __ldg(src + i);
      a[2 * i] = t.x;
      a[2 * i + 1] = t.y;
    }
    float d[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) d[q] = d2f_rn(a[q] - wi[q]);
    to_char_f(sf, d, cf[k]);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int j = k - side;                 // node index within this side's five
      if (j < 0 || j > 4) continue;
#pragma unroll
      for (int dd = 0; dd < 4; ++dd) {
        const double wt = __ldg(w5 + (size_t)(20 * side + 4 * j + dd) * E + e);
#pragma unroll
        for (int q = 0; q < 5; ++q) W[side][q] = fma(wt, a[5 * dd + q], W[side][q]);
      }
    }
  }
  // per side and characteristic component: FP32 decision, taken again in FP64 (on the node
  // values' characteristic values, as the 3-node candidates need) inside the guard band or on a
  // non-finite FP32 sum; weighted 3-node values where the decision is rough
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    unsigned flag = 0;                        // rough in FP32, or undecided
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if (ph.force_branch == 1) break;
      if (ph.force_branch == 2) {
        flag |= 1u << q;
        continue;
      }
      float t0, S;
      if (side == 0) weno3f(cf[0][q], cf[1][q], cf[2][q], cf[3][q], cf[4][q], ph.epsf, t0, S);
      else           weno3f(cf[5][q], cf[4][q], cf[3][q], cf[2][q], cf[1][q], ph.epsf, t0, S);
      const float mlo = t0 - ph.sens_lof * S, mhi = ph.sens_hif * S - t0;
      const bool smooth = mlo > 0.f && mhi > 0.f;
      const bool clear = isfinite(S) && fabsf(mlo) > kGuard3 * S && fabsf(mhi) > kGuard3 * S;
      if (!smooth || !clear) flag |= 1u << q;
    }
    if (!flag) continue;
    double C[5];
    to_char(st, W[side], C);
    bool any = false;
    const double* w = w3 + (size_t)(9 * side) * E + e;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if (!((flag >> q) & 1u)) continue;
      double cq[5];
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        const int k = side == 0 ? j : 5 - j;
        double a[5], c[5];
#pragma unroll
        for (int r = 0; r < 5; ++r) a[r] = __ldg(Ua + (size_t)20 * s[k] + r);
        to_char(st, a, c);
        cq[j] = c[q];
      }
      double o[3], S;
      weno3(cq[0], cq[1], cq[2], cq[3], cq[4], ph.eps, o, S);
      const bool smooth = o[0] > ph.sens_lo * S && o[0] < ph.sens_hi * S;
      if (ph.force_branch != 2 && smooth) continue;
      const double iS = 1.0 / S;
      double wt[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) wt[i] = __ldg(w + (size_t)i * E);
      const double c1 = wt[0] * cq[0] + wt[1] * cq[1] + wt[2] * cq[2];
      const double c2 = wt[3] * cq[1] + wt[4] * cq[2] + wt[5] * cq[3];
      const double c3 = wt[6] * cq[2] + wt[7] * cq[3] + wt[8] * cq[4];
      C[q] = (o[0] * iS) * c1 + (o[1] * iS) * c2 + (o[2] * iS) * c3;
      any = true;
    }
    if (any) from_char(st, C, W[side]);
  }
  // positivity (R16): fall back to the end state of that side
  if (!admissible3(W[0]))
#pragma unroll
    for (int q = 0; q < 5; ++q) W[0][q] = wi[q];
  if (!admissible3(W[1]))
#pragma unroll
    for (int q = 0; q < 5; ++q) W[1][q] = wj[q];
  // Roe's flux along n with Harten's fix on all five waves
  Eig r;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.n[k] = st.n[k];
    r.t1[k] = st.t1[k];
    r.t2[k] = st.t2[k];
  }
  roe_state(W[0], W[1], g1, r);
  double dw[5], al[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) dw[q] = W[1][q] - W[0][q];
  to_char(r, dw, al);
  const double lam[5] = {r.qn - r.c, r.qn, r.qn, r.qn, r.qn + r.c};
  const double del = ph.harten * r.c, i2del = ph.half_inv_harten * r.ic;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    double a = fabs(lam[i]);
    if (a < del) a = (lam[i] * lam[i] + del * del) * i2del;
    al[i] *= a;
  }
  double diss[5], fl[5], fr[5];
  from_char(r, al, diss);
  normal_flux3(W[0], r.irl, r.pl, r.n, fl);
  normal_flux3(W[1], r.irr, r.pr, r.n, fr);
  double* o = h + (size_t)8 * e;
  double hq[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) hq[q] = 0.5 * (fl[q] + fr[q]) - 0.5 * diss[q];
  reinterpret_cast<double2*>(o)[0] = make_double2(hq[0], hq[1]);
  reinterpret_cast<double2*>(o)[1] = make_double2(hq[2], hq[3]);
  o[4] = hq[4];
}

// ------------------------------------------------------------------ k3_div
// G lanes per vertex (G = 1, 2 or 4, consecutive threads): the lanes take the vertex's entries
// in turn (lane l the entries l, l + G, ...; adjacent lanes read adjacent coefficient blocks),
// each accumulates acc[5 r + q] over its entries of the row r (d_0, d_x, d_y, d_z): 12
// coefficients per vertex entry against F, G, K of the entry's vertex and 4 per edge entry
// against h of the entry's edge.  The lanes' sums are combined by a fixed butterfly, so the
// result is deterministic.  R = -acc; mode 0 writes R; mode 1 writes the stage update
// b (Us + dt R) + a Un (a = 0: Un is not read) with explicit roundings; lane l writes the
// rows l, l + G, ...
template <int G>
__global__ void __launch_bounds__(128) k3_div(int V, int E, const int32_t* __restrict__ vptr,
                                              const int32_t* __restrict__ vidx,
                                              const double* __restrict__ cv,
                                              const int32_t* __restrict__ eptr,
                                              const int32_t* __restrict__ eidx,
                                              const double* __restrict__ ce,
                                              const double* __restrict__ FGK,
                                              const double* __restrict__ h, int mode,
                                              const double* __restrict__ Us, const double* Un,
                                              double* out, double a, double b, double dt,
                                              unsigned* __restrict__ err) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = gt / G, lane = gt % G;
  // whole groups stay in the warp for the shuffles (V * G threads rounded up to the block)
  const bool live = v < V;
  double acc[20];
#pragma unroll
  for (int i = 0; i < 20; ++i) acc[i] = 0.0;
  unsigned bad = 0;
  if (live) {
    const int j0 = __ldg(vptr + v), j1 = __ldg(vptr + v + 1);
    for (int j = j0 + lane; j < j1; j += G) {
      const int u = __ldg(vidx + j);
      if ((unsigned)u >= (unsigned)V) {
        bad |= kErrIndex;
        continue;
      }
      double c[12], f[16];
      const double2* cs = reinterpret_cast<const double2*>(cv + (size_t)12 * j);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const double2 t = __ldg(cs + i);
        c[2 * i] = t.x;
        c[2 * i + 1] = t.y;
      }
      const double2* fs = reinterpret_cast<const double2*>(FGK + (size_t)16 * u);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const double2 t = __ldg(fs + i);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 5; ++q)
          acc[5 * r + q] = fma(c[3 * r], f[q], fma(c[3 * r + 1], f[5 + q], fma(c[3 * r + 2], f[10 + q], acc[5 * r + q])));
    }
    const int k0 = __ldg(eptr + v), k1 = __ldg(eptr + v + 1);
    for (int j = k0 + lane; j < k1; j += G) {
      const int ed = __ldg(eidx + j);
      if ((unsigned)ed >= (unsigned)E) {
        bad |= kErrIndex;
        continue;
      }
      const double2 c01 = __ldg(reinterpret_cast<const double2*>(ce + (size_t)4 * j));
      const double2 c23 = __ldg(reinterpret_cast<const double2*>(ce + (size_t)4 * j) + 1);
      const double* hp = h + (size_t)8 * ed;
      const double2 h01 = __ldg(reinterpret_cast<const double2*>(hp));
      const double2 h23 = __ldg(reinterpret_cast<const double2*>(hp) + 1);
      const double hq[5] = {h01.x, h01.y, h23.x, h23.y, __ldg(hp + 4)};
      const double cr[4] = {c01.x, c01.y, c23.x, c23.y};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[5 * r + q] = fma(cr[r], hq[q], acc[5 * r + q]);
    }
  }
  // butterfly over the group: every lane ends with the group's sums, in the same order
#pragma unroll
  for (int off = 1; off < G; off <<= 1)
#pragma unroll
    for (int i = 0; i < 20; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off, G);
  if (!live) return;
#pragma unroll
  for (int i = 0; i < 20; ++i) {
    if (i % G != lane) continue;
    const double R = -acc[i];
    const size_t idx = (size_t)i * V + v;
    double o;
    if (mode == 0) {
      o = R;
    } else {
      o = __dmul_rn(b, __fma_rn(dt, R, Us[idx]));
      if (a != 0.0) o = __fma_rn(a, Un[idx], o);
    }
    out[idx] = o;
    if (!finite3(o)) bad |= kErrNonfinite;
    if (mode == 1 && i == 0 && !(o > 0.0)) bad |= kErrPositivity;
  }
  if (bad) atomicOr(err, bad);
}

}  // namespace

cudaError_t launch3_vertex(const DevMesh3& m, const double* U, const Phys3& ph, cudaStream_t s) {
  if (m.V == 0) return cudaSuccess;
  k3_vertex<<<(m.V + 255) / 256, 256, 0, s>>>(m.V, U, m.Ua, m.FGK, ph.g1);
  return cudaGetLastError();
}

cudaError_t launch3_edge(const DevMesh3& m, const Phys3& ph, cudaStream_t s) {
  if (m.E == 0) return cudaSuccess;
  k3_edge<<<(m.E + 127) / 128, 128, 0, s>>>(m.E, m.V, m.sten, m.frame, m.w5, m.w3, m.Ua, m.h, ph,
                                            m.err);
  return cudaGetLastError();
}

cudaError_t launch3_div(const DevMesh3& m, const double* Us, const double* Un, double* out,
                        int mode, double a, double b, double dt, cudaStream_t s) {
  if (m.V == 0) return cudaSuccess;
  const int64_t threads = (int64_t)m.V * m.lanes;
  const unsigned blocks = (unsigned)((threads + 127) / 128);
  if (m.lanes == 4)
    k3_div<4><<<blocks, 128, 0, s>>>(m.V, m.E, m.vptr, m.vidx, m.cv, m.eptr, m.eidx, m.ce, m.FGK,
                                     m.h, mode, Us, Un, out, a, b, dt, m.err);
  else if (m.lanes == 2)
    k3_div<2><<<blocks, 128, 0, s>>>(m.V, m.E, m.vptr, m.vidx, m.cv, m.eptr, m.eidx, m.ce, m.FGK,
                                     m.h, mode, Us, Un, out, a, b, dt, m.err);
  else
    k3_div<1><<<blocks, 128, 0, s>>>(m.V, m.E, m.vptr, m.vidx, m.cv, m.eptr, m.eidx, m.ce, m.FGK,
                                     m.h, mode, Us, Un, out, a, b, dt, m.err);
  return cudaGetLastError();
}

}  // namespace hfd
