// Host preprocessing of the three-dimensional extension: everything geometry-only, in FP64,
// computed once per mesh (the 2D method of arXiv 2109.01286 carried over to tetrahedra; the
// paper names three dimensions as future work, Sec. 4).
//   * edge list and curvilinear 6-node stencils (Sec. 2.1, with 3D cosines);
//   * per edge the frame (n, t1, t2): n the unit edge direction, t1 = e_k x n normalised with
//     e_k the axis of smallest |n_k| (lowest k on ties), t2 = n x t1;
//   * 5-node Hermite weights: first row of the pseudo-inverse of the 20 x 20 system with the
//     data w, w_x, w_y, w_z and the complete degree-3 Taylor basis (Sec. 2.2), by the one-sided
//     Jacobi SVD with the same trial dropping of singular values as in 2D;
//   * 3-node weights (Eq. (3nodes_intp) with the degree-2 basis in 3D), minimum norm, in
//     double-double;
//   * two-level least-squares divergence rows d_0, d_x, d_y, d_z of the three flux vectors
//     with degree-4 polynomials (Eq. (flux_polynomials)), by Householder QR.
// Built with -ffp-contract=off, like the 2D preprocessing.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <set>
#include <thread>

#include "linalg.hpp"
#include "mesh3.hpp"
#include "prep.hpp"

namespace hfd {

void Prep3::disp(int a, int b, double* d) const {
  const double* c[3] = {x.data(), y.data(), z.data()};
  for (int k = 0; k < 3; ++k) {
    double t = c[k][b] - c[k][a];
    d[k] = t - L[k] * std::rint(t / L[k]);
  }
}

static inline double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static int nterms3(int deg) { return (deg + 1) * (deg + 2) * (deg + 3) / 6; }

// Complete 3D Taylor basis x^a y^b z^c / (a! b! c!) by degree, then decreasing a, then
// decreasing b; derivatives optional.
static void taylor3(double x, double y, double z, int deg, double* p, double* px, double* py,
                    double* pz) {
  double xp[8], yp[8], zp[8], fact[8];
  xp[0] = yp[0] = zp[0] = fact[0] = 1.0;
  for (int i = 1; i <= deg; ++i) {
    xp[i] = xp[i - 1] * x;
    yp[i] = yp[i - 1] * y;
    zp[i] = zp[i - 1] * z;
    fact[i] = fact[i - 1] * i;
  }
  int i = 0;
  for (int d = 0; d <= deg; ++d)
    for (int a = d; a >= 0; --a)
      for (int b = d - a; b >= 0; --b, ++i) {
        const int c = d - a - b;
        const double f = 1.0 / (fact[a] * fact[b] * fact[c]);
        p[i] = f * xp[a] * yp[b] * zp[c];
        if (px) px[i] = a > 0 ? a * f * xp[a - 1] * yp[b] * zp[c] : 0.0;
        if (py) py[i] = b > 0 ? b * f * xp[a] * yp[b - 1] * zp[c] : 0.0;
        if (pz) pz[i] = c > 0 ? c * f * xp[a] * yp[b] * zp[c - 1] : 0.0;
      }
}

// 5-node Hermite weights for nodes rel[5] (relative to the edge midpoint), edge length ell,
// near node index 2: scaled coordinates (x / ell), data (c, ell c_x, ell c_y, ell c_z); keep
// singular values > sv_rtol sigma_max, then drop the smallest while any scaled weight has
// magnitude >= 1; unscale the derivative weights and make the value weights sum to one.
// Returns the rank kept (0: none left).
static int five_node3(const double (*rel)[3], double ell, double sv_rtol, double* w) {
  double P[20 * 20], V[20 * 20], s[20];
  double p[20], px[20], py[20], pz[20];
  for (int j = 0; j < 5; ++j) {
    taylor3(rel[j][0] / ell, rel[j][1] / ell, rel[j][2] / ell, 3, p, px, py, pz);
    for (int k = 0; k < 20; ++k) {            // rows 4j .. 4j+3, column-major
      P[(4 * j) + 20 * k] = p[k];
      P[(4 * j + 1) + 20 * k] = px[k];
      P[(4 * j + 2) + 20 * k] = py[k];
      P[(4 * j + 3) + 20 * k] = pz[k];
    }
  }
  jacobi_svd(20, 20, P, V, s);
  int r = 0;
  for (int i = 0; i < 20; ++i)
    if (s[i] > sv_rtol * s[0]) ++r;
  for (;;) {
    double mx = 0;
    for (int i = 0; i < 20; ++i) w[i] = 0.0;
    for (int k = 0; k < r; ++k) {
      const double f = V[0 + 20 * k] / (s[k] * s[k]);   // V[0,k] U[:,k] / s_k with U s = A V
      for (int i = 0; i < 20; ++i) w[i] += f * P[i + 20 * k];
    }
    for (int i = 0; i < 20; ++i) mx = std::max(mx, std::fabs(w[i]));
    if (mx < 1.0) break;
    if (--r == 0) return 0;
  }
  for (int j = 0; j < 5; ++j)
    for (int d = 1; d < 4; ++d) w[4 * j + d] *= ell;
  double sum = 0;
  for (int j = 0; j < 5; ++j) sum += w[4 * j];
  w[8] += 1.0 - sum;
  return r;
}

// 3-node weights with the degree-2 3D basis [1, x, y, z, x^2/2, xy, xz, y^2/2, yz, z^2/2] in
// unscaled midpoint-relative coordinates: w = (A A^T)^-1 1 by Cramer's rule in double-double
// (A A^T is nearly singular for short edges), value weights summing to one at `near`.
static void three_node3(const double (*rel)[3], int near, double* w) {
  dd A[3][10];
  for (int k = 0; k < 3; ++k) {
    const double x = rel[k][0], y = rel[k][1], z = rel[k][2];
    const dd xx = two_prod(x, x), yy = two_prod(y, y), zz = two_prod(z, z);
    A[k][0] = dd_from(1.0);
    A[k][1] = dd_from(x);
    A[k][2] = dd_from(y);
    A[k][3] = dd_from(z);
    A[k][4] = {xx.hi * 0.5, xx.lo * 0.5};
    A[k][5] = two_prod(x, y);
    A[k][6] = two_prod(x, z);
    A[k][7] = {yy.hi * 0.5, yy.lo * 0.5};
    A[k][8] = two_prod(y, z);
    A[k][9] = {zz.hi * 0.5, zz.lo * 0.5};
  }
  dd G[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      dd s = dd_from(0.0);
      for (int k = 0; k < 10; ++k) s = dd_add(s, dd_mul(A[i][k], A[j][k]));
      G[i][j] = s;
    }
  auto det3 = [](dd M[3][3]) {
    dd a = dd_add(dd_mul(M[1][1], M[2][2]), dd_neg(dd_mul(M[1][2], M[2][1])));
    dd b = dd_add(dd_mul(M[1][0], M[2][2]), dd_neg(dd_mul(M[1][2], M[2][0])));
    dd c = dd_add(dd_mul(M[1][0], M[2][1]), dd_neg(dd_mul(M[1][1], M[2][0])));
    return dd_add(dd_add(dd_mul(M[0][0], a), dd_neg(dd_mul(M[0][1], b))), dd_mul(M[0][2], c));
  };
  const dd den = det3(G);
  dd num[3];
  for (int c = 0; c < 3; ++c) {
    dd M[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[i][j] = (j == c) ? dd_from(1.0) : G[i][j];
    num[c] = det3(M);
  }
  const dd sum = dd_add(dd_add(num[0], num[1]), num[2]);
  num[near] = dd_add(num[near], dd_add(den, dd_neg(sum)));
  for (int c = 0; c < 3; ++c) {
    const dd q = dd_div(num[c], den);
    w[c] = q.hi + q.lo;
  }
}

// One stencil extension (Sec. 2.1): the unused neighbour of cur with the largest cosine to the
// travel direction t; ties within 1e-12 keep the lower id (ascending scan).
static int extend3(const Prep3& P, int cur, const double* t, const int* used, int nused, double* d) {
  const double tn = std::sqrt(dot3(t, t));
  int best = -1;
  double bc = -INFINITY;
  for (int k = P.nbr_ptr[cur]; k < P.nbr_ptr[cur + 1]; ++k) {
    const int c = P.nbr_idx[k];
    bool u = false;
    for (int i = 0; i < nused; ++i) u |= (used[i] == c);
    if (u) continue;
    double e[3];
    P.disp(cur, c, e);
    const double cs = dot3(t, e) / (tn * std::sqrt(dot3(e, e)));
    if (cs > bc + 1e-12) {
      best = c;
      bc = cs;
      d[0] = e[0];
      d[1] = e[1];
      d[2] = e[2];
    }
  }
  return best;
}

// Frame of the edge direction n: t1 = e_k x n / |e_k x n|, e_k the axis of smallest |n_k|
// (lowest k on ties), t2 = n x t1.
static void frame3(const double* n, double* t1, double* t2) {
  int k = 0;
  for (int i = 1; i < 3; ++i)
    if (std::fabs(n[i]) < std::fabs(n[k])) k = i;
  double e[3] = {0, 0, 0};
  e[k] = 1.0;
  double c[3] = {e[1] * n[2] - e[2] * n[1], e[2] * n[0] - e[0] * n[2], e[0] * n[1] - e[1] * n[0]};
  const double cn = std::sqrt(dot3(c, c));
  for (int i = 0; i < 3; ++i) t1[i] = c[i] / cn;
  t2[0] = n[1] * t1[2] - n[2] * t1[1];
  t2[1] = n[2] * t1[0] - n[0] * t1[2];
  t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

static const int kLeft5[5] = {0, 1, 2, 3, 4}, kRight5[5] = {1, 2, 3, 4, 5};
static const int kLeft3[3][3] = {{0, 1, 2}, {1, 2, 3}, {2, 3, 4}};
static const int kRight3[3][3] = {{5, 4, 3}, {4, 3, 2}, {3, 2, 1}};

// Stencil, frame and weights of edge e; false (with the message) when a stencil cannot be
// extended or a Hermite system keeps no singular value.
static bool edge3(Prep3& P, const hfd3_options& o, int e, char* msg) {
  const int a = P.edges[2 * e], b = P.edges[2 * e + 1];
  double dab[3], d1[3], d2[3], d3[3], d4[3], back[3];
  P.disp(a, b, dab);
  for (int k = 0; k < 3; ++k) back[k] = -dab[k];
  int used[6] = {a, b, -1, -1, -1, -1};
  const int b1 = extend3(P, a, back, used, 2, d1);
  used[2] = b1;
  const int b2 = b1 < 0 ? -1 : extend3(P, b1, d1, used, 3, d2);
  used[3] = b2;
  const int f1 = b2 < 0 ? -1 : extend3(P, b, dab, used, 4, d3);
  used[4] = f1;
  const int f2 = f1 < 0 ? -1 : extend3(P, f1, d3, used, 5, d4);
  if (f2 < 0) {
    snprintf(msg, 256, "hfd3_mesh_create: the stencil of edge (%d, %d) cannot be extended", a, b);
    return false;
  }
  const int ids[6] = {b2, b1, a, b, f1, f2};
  double pos[6][3];
  for (int k = 0; k < 3; ++k) {
    pos[2][k] = 0.0;
    pos[1][k] = d1[k];
    pos[0][k] = pos[1][k] + d2[k];
    pos[3][k] = dab[k];
    pos[4][k] = pos[3][k] + d3[k];
    pos[5][k] = pos[4][k] + d4[k];
  }
  const double ell = std::sqrt(dot3(dab, dab));
  double rel[6][3];
  for (int j = 0; j < 6; ++j)
    for (int k = 0; k < 3; ++k) rel[j][k] = pos[j][k] - 0.5 * pos[3][k];
  for (int j = 0; j < 6; ++j) P.sten[(size_t)6 * e + j] = ids[j];
  double* fr = &P.frame[(size_t)9 * e];
  for (int k = 0; k < 3; ++k) fr[k] = dab[k] / ell;
  frame3(fr, fr + 3, fr + 6);
  for (int side = 0; side < 2; ++side) {
    const int* five = side == 0 ? kLeft5 : kRight5;
    double r5[5][3];
    for (int j = 0; j < 5; ++j)
      for (int k = 0; k < 3; ++k) r5[j][k] = rel[five[j]][k];
    const int r = five_node3(r5, ell, o.sv_rtol, &P.w5[(size_t)40 * e + 20 * side]);
    if (r == 0) {
      snprintf(msg, 256, "hfd3_mesh_create: no singular value left for edge (%d, %d)", a, b);
      return false;
    }
    P.rank[2 * e + side] = r;
    for (int c = 0; c < 3; ++c) {
      const int* tri = side == 0 ? kLeft3[c] : kRight3[c];
      const int nearnode = side == 0 ? 2 : 3;
      double r3[3][3];
      int near = 0;
      for (int j = 0; j < 3; ++j) {
        for (int k = 0; k < 3; ++k) r3[j][k] = rel[tri[j]][k];
        if (tri[j] == nearnode) near = j;
      }
      three_node3(r3, near, &P.w3[(size_t)18 * e + 9 * side + 3 * c]);
    }
  }
  return true;
}

// sum a[i] b[i] over i < n with four partial sums (the compiler keeps reductions in order, so
// the split is what lets it use vector registers)
static inline double dot4(const double* a, const double* b, int n) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  int i = 0;
  for (; i + 3 < n; i += 4) {
    s0 += a[i] * b[i];
    s1 += a[i + 1] * b[i + 1];
    s2 += a[i + 2] * b[i + 2];
    s3 += a[i + 3] * b[i + 3];
  }
  for (; i < n; ++i) s0 += a[i] * b[i];
  return (s0 + s1) + (s2 + s3);
}

// Rows e_t^T A^+ for the target columns t of a full-column-rank A (m x n, column-major) by
// Householder QR without pivoting: A = Q R, so the row is Q z with R^T z = e_t.  The 3D
// divergence fit has full column rank on the meshes it accepts, so pivoting buys nothing
// there and its repeated column norms cost a third of the factorisation.  Returns
// min |R_kk| / max |R_kk| as the conditioning estimate (0 for a zero column).
static double ls_rows3(int m, int n, std::vector<double>& A, const int* targets, int ntarg,
                       double* rows /* ntarg x m */) {
  std::vector<double> beta(n, 0.0), v0s(n, 0.0);
  auto col = [&](int j) { return &A[(size_t)j * m]; };
  double rmin = INFINITY, rmax = 0.0;
  for (int k = 0; k < n; ++k) {
    double* c = col(k);
    const double nx = std::sqrt(dot4(c + k, c + k, m - k));
    if (nx == 0.0) return 0.0;
    const double alpha = c[k] >= 0 ? -nx : nx;
    const double v0 = c[k] - alpha;
    const double vtv = v0 * v0 + dot4(c + k + 1, c + k + 1, m - k - 1);
    const double b = 2.0 / vtv;
    for (int j = k + 1; j < n; ++j) {
      double* cj = col(j);
      const double dot = b * (v0 * cj[k] + dot4(c + k + 1, cj + k + 1, m - k - 1));
      cj[k] -= dot * v0;
      for (int i = k + 1; i < m; ++i) cj[i] -= dot * c[i];
    }
    c[k] = alpha;
    beta[k] = b;
    v0s[k] = v0;
    rmin = std::min(rmin, std::fabs(alpha));
    rmax = std::max(rmax, std::fabs(alpha));
  }
  std::vector<double> z(n), y(m);
  for (int t = 0; t < ntarg; ++t) {
    for (int k = 0; k < n; ++k) {             // R^T z = e_t (forward substitution)
      double acc = (k == targets[t]) ? 1.0 : 0.0;
      acc -= dot4(&A[(size_t)k * m], z.data(), k);
      z[k] = acc / A[(size_t)k * m + k];
    }
    for (int i = 0; i < m; ++i) y[i] = i < n ? z[i] : 0.0;
    for (int k = n - 1; k >= 0; --k) {        // y = H_0 ... H_{n-1} [z; 0]
      const double* c = col(k);
      const double dot = beta[k] * (v0s[k] * y[k] + dot4(c + k + 1, y.data() + k + 1, m - k - 1));
      y[k] -= dot * v0s[k];
      for (int i = k + 1; i < m; ++i) y[i] -= dot * c[i];
    }
    std::memcpy(rows + (size_t)t * m, y.data(), sizeof(double) * m);
  }
  return rmax > 0 ? rmin / rmax : 0.0;
}

// Two-level stencil of vertex v (every vertex within graph distance 2, ascending id, and every
// edge with both ends in that set, ascending index) and its divergence rows: the least-squares
// fit of the degree-4 Taylor coefficients (a, b, c) of the flux vectors f, g, k about v in
// coordinates scaled by the mean incident edge length l_v, to the vertex data (f, g, k) and the
// edge data (f, g, k) . n at the edge midpoints; d_0 = a_x + b_y + c_z, d_x = a_xx + b_xy + c_xz,
// d_y = a_xy + b_yy + c_yz, d_z = a_xz + b_yz + c_zz (rows of the pseudo-inverse), unscaled.
// Fills verts, edges and the 12-per-vertex / 4-per-edge coefficients; returns the QR
// conditioning estimate min |R_kk| / max |R_kk|.
static double div3(const Prep3& P, int v, std::vector<int>& verts, std::vector<int>& eds,
                   std::vector<double>& cvv, std::vector<double>& cee) {
  std::set<int> s;
  s.insert(v);
  for (int k = P.nbr_ptr[v]; k < P.nbr_ptr[v + 1]; ++k) {
    const int u = P.nbr_idx[k];
    s.insert(u);
    for (int j = P.nbr_ptr[u]; j < P.nbr_ptr[u + 1]; ++j) s.insert(P.nbr_idx[j]);
  }
  verts.assign(s.begin(), s.end());
  eds.clear();
  for (int u : verts)
    for (int j = P.nbr_ptr[u]; j < P.nbr_ptr[u + 1]; ++j) {
      const int w = P.nbr_idx[j];
      if (w > u && s.count(w)) {
        // edge index by binary search in the sorted edge list
        int lo = 0, hi = P.E - 1;
        while (lo < hi) {
          const int mid = (lo + hi) / 2;
          const int ta = P.edges[2 * mid], tb = P.edges[2 * mid + 1];
          if (ta < u || (ta == u && tb < w)) lo = mid + 1; else hi = mid;
        }
        eds.push_back(lo);
      }
    }
  std::sort(eds.begin(), eds.end());
  double ell = 0;
  const int deg_v = P.nbr_ptr[v + 1] - P.nbr_ptr[v];
  for (int k = P.nbr_ptr[v]; k < P.nbr_ptr[v + 1]; ++k) {
    double d[3];
    P.disp(v, P.nbr_idx[k], d);
    ell += std::sqrt(dot3(d, d));
  }
  ell /= deg_v;
  const int K = nterms3(4), N = (int)verts.size(), M = (int)eds.size();
  const int m = 3 * N + M, n = 3 * K;
  std::vector<double> A((size_t)m * n, 0.0);        // column-major
  double p[35];
  for (int j = 0; j < N; ++j) {
    double d[3];
    P.disp(v, verts[j], d);
    taylor3(d[0] / ell, d[1] / ell, d[2] / ell, 4, p, nullptr, nullptr, nullptr);
    for (int f = 0; f < 3; ++f)
      for (int k = 0; k < K; ++k) A[(size_t)(3 * j + f) + (size_t)m * (f * K + k)] = p[k];
  }
  for (int j = 0; j < M; ++j) {
    const int a = P.edges[2 * eds[j]], b = P.edges[2 * eds[j] + 1];
    double da[3], dab[3];
    P.disp(v, a, da);
    P.disp(a, b, dab);
    const double l = std::sqrt(dot3(dab, dab));
    double xm[3], nm[3];
    for (int k = 0; k < 3; ++k) {
      xm[k] = (da[k] + 0.5 * dab[k]) / ell;
      nm[k] = dab[k] / l;
    }
    taylor3(xm[0], xm[1], xm[2], 4, p, nullptr, nullptr, nullptr);
    for (int f = 0; f < 3; ++f)
      for (int k = 0; k < K; ++k) A[(size_t)(3 * N + j) + (size_t)m * (f * K + k)] = p[k] * nm[f];
  }
  // the twelve single rows of A^+ that the four divergence rows sum
  static const int tg[12] = {1, 4, 5, 6, 2, 5, 7, 8, 3, 6, 8, 9};   // per flux f: d0, dx, dy, dz
  int targ[12];
  for (int f = 0; f < 3; ++f)
    for (int r = 0; r < 4; ++r) targ[4 * f + r] = f * K + tg[4 * f + r];
  std::vector<double> rows((size_t)12 * m);
  const double cond = ls_rows3(m, n, A, targ, 12, rows.data());
  const double sc[4] = {1.0 / ell, 1.0 / (ell * ell), 1.0 / (ell * ell), 1.0 / (ell * ell)};
  cvv.assign((size_t)12 * N, 0.0);
  cee.assign((size_t)4 * M, 0.0);
  for (int r = 0; r < 4; ++r) {
    // row r over the data: vertex j, flux f at column 3j + f; edge j at column 3N + j
    for (int j = 0; j < N; ++j)
      for (int f = 0; f < 3; ++f) {
        double t = 0;
        for (int g = 0; g < 3; ++g) t += rows[(size_t)(4 * g + r) * m + 3 * j + f];
        cvv[(size_t)12 * j + 3 * r + f] = t * sc[r];
      }
    for (int j = 0; j < M; ++j) {
      double t = 0;
      for (int g = 0; g < 3; ++g) t += rows[(size_t)(4 * g + r) * m + 3 * N + j];
      cee[(size_t)4 * j + r] = t * sc[r];
    }
  }
  return cond;
}

hfd_status build_prep3(const hfd3_mesh_desc* d, const hfd3_options* o, Prep3* P) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!d || !o || d->nv <= 0 || d->ntet <= 0 || !d->x || !d->y || !d->z || !d->tet ||
      !(d->Lx > 0) || !(d->Ly > 0) || !(d->Lz > 0)) {
    set_error("hfd3_mesh_create: invalid mesh description");
    return HFD_ERR_ARG;
  }
  P->V = d->nv;
  P->L[0] = d->Lx;
  P->L[1] = d->Ly;
  P->L[2] = d->Lz;
  P->x.assign(d->x, d->x + d->nv);
  P->y.assign(d->y, d->y + d->nv);
  P->z.assign(d->z, d->z + d->nv);
  // unique edges of the tetrahedra, tail < head, sorted
  std::vector<std::pair<int, int>> ev;
  ev.reserve((size_t)6 * d->ntet);
  for (int t = 0; t < d->ntet; ++t) {
    const int32_t* q = d->tet + 4 * (size_t)t;
    for (int i = 0; i < 4; ++i) {
      if (q[i] < 0 || q[i] >= d->nv) {
        set_error("hfd3_mesh_create: tetrahedron %d has a vertex id out of range", t);
        return HFD_ERR_ARG;
      }
      for (int j = i + 1; j < 4; ++j) {
        if (q[i] == q[j]) {
          set_error("hfd3_mesh_create: tetrahedron %d repeats a vertex", t);
          return HFD_ERR_ARG;
        }
        ev.emplace_back(std::min(q[i], q[j]), std::max(q[i], q[j]));
      }
    }
  }
  std::sort(ev.begin(), ev.end());
  ev.erase(std::unique(ev.begin(), ev.end()), ev.end());
  const int E = (int)ev.size();
  P->E = E;
  P->edges.resize((size_t)2 * E);
  std::vector<int> deg(d->nv, 0);
  for (int e = 0; e < E; ++e) {
    P->edges[2 * e] = ev[e].first;
    P->edges[2 * e + 1] = ev[e].second;
    ++deg[ev[e].first];
    ++deg[ev[e].second];
  }
  P->nbr_ptr.assign(d->nv + 1, 0);
  for (int v = 0; v < d->nv; ++v) P->nbr_ptr[v + 1] = P->nbr_ptr[v] + deg[v];
  P->nbr_idx.resize(P->nbr_ptr[d->nv]);
  std::vector<int> fill(P->nbr_ptr.begin(), P->nbr_ptr.end() - 1);
  for (int e = 0; e < E; ++e) {
    P->nbr_idx[fill[ev[e].first]++] = ev[e].second;
    P->nbr_idx[fill[ev[e].second]++] = ev[e].first;
  }
  for (int v = 0; v < d->nv; ++v) {
    if (deg[v] == 0) {
      set_error("hfd3_mesh_create: vertex %d belongs to no tetrahedron", v);
      return HFD_ERR_ARG;
    }
    std::sort(P->nbr_idx.begin() + P->nbr_ptr[v], P->nbr_idx.begin() + P->nbr_ptr[v + 1]);
  }
  const int nthreads = o->threads > 0 ? o->threads
                                      : std::max(1, (int)std::thread::hardware_concurrency());
  // edges: stencils, frames, weights
  P->sten.assign((size_t)6 * E, 0);
  P->frame.assign((size_t)9 * E, 0.0);
  P->w5.assign((size_t)40 * E, 0.0);
  P->w3.assign((size_t)18 * E, 0.0);
  P->rank.assign((size_t)2 * E, 0);
  ErrorSlot err;
  parallel_for(E, nthreads, [&](int64_t e, int) {
    char msg[256];
    if (!edge3(*P, *o, (int)e, msg)) err.set(HFD_ERR_SINGULAR, msg);
  });
  if (err.st != HFD_OK) {
    set_error("%s", err.msg);
    return err.st;
  }
  // vertices: two-level stencils and divergence rows, gathered per vertex then concatenated
  std::vector<std::vector<int>> vv(d->nv), ee(d->nv);
  std::vector<std::vector<double>> cvv(d->nv), cee(d->nv);
  parallel_for(d->nv, nthreads, [&](int64_t v, int) {
    const double cond = div3(*P, (int)v, vv[v], ee[v], cvv[v], cee[v]);
    if (!(cond >= o->div_cond_min)) {
      char msg[256];
      snprintf(msg, sizeof msg, "hfd3_mesh_create: the divergence stencil of vertex %d is "
               "ill-conditioned (%.3g)", (int)v, cond);
      err.set(HFD_ERR_SINGULAR, msg);
    }
  });
  if (err.st != HFD_OK) {
    set_error("%s", err.msg);
    return err.st;
  }
  P->vptr.assign(d->nv + 1, 0);
  P->eptr.assign(d->nv + 1, 0);
  for (int v = 0; v < d->nv; ++v) {
    P->vptr[v + 1] = P->vptr[v] + (int)vv[v].size();
    P->eptr[v + 1] = P->eptr[v] + (int)ee[v].size();
  }
  P->vidx.resize(P->vptr[d->nv]);
  P->eidx.resize(P->eptr[d->nv]);
  P->cv.resize((size_t)12 * P->vptr[d->nv]);
  P->ce.resize((size_t)4 * P->eptr[d->nv]);
  for (int v = 0; v < d->nv; ++v) {
    std::copy(vv[v].begin(), vv[v].end(), P->vidx.begin() + P->vptr[v]);
    std::copy(ee[v].begin(), ee[v].end(), P->eidx.begin() + P->eptr[v]);
    std::copy(cvv[v].begin(), cvv[v].end(), P->cv.begin() + (size_t)12 * P->vptr[v]);
    std::copy(cee[v].begin(), cee[v].end(), P->ce.begin() + (size_t)4 * P->eptr[v]);
  }
  P->deficient = 0;
  for (int32_t r : P->rank) P->deficient += r < 20;
  P->micros = std::chrono::duration_cast<std::chrono::microseconds>(
                  std::chrono::steady_clock::now() - t0).count();
  return HFD_OK;
}

}  // namespace hfd
