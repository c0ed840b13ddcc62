// Host preprocessing of the Hermite finite-difference method: everything geometry-only, in FP64,
// computed once per mesh.  Paper: arXiv 2109.01286.
//   * edge list and curvilinear 6-node stencils (Sec. 2.1, Fig. 1);
//   * 5-node Hermite least-squares weights: first row of the pseudo-inverse of the 15x15 system
//     of Eq. (hintp_5) (Sec. 2.2), by a one-sided Jacobi SVD with trial dropping of singular
//     values;
//   * 3-node Lagrangian weights of Eq. (3nodes_intp) (Sec. 2.3), min-norm, in double-double;
//   * two-level least-squares divergence rows d_0, d_x, d_y of Eq. (flux_polynomials) and the
//     viscous vertex-only rows (Sec. 2.3), by Householder QR with column pivoting.
// Host code is compiled with -ffp-contract=off so that the geometric quantities that decide
// discrete choices (stencil cosines) are evaluated exactly as written.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>

#include "linalg.hpp"
#include "prep.hpp"

namespace hfd {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

// ------------------------------------------------------------------ small utilities

double Prep::dispx(int a, int b) const {
  double d = x[b] - x[a];
  if (periodic_x) d = d - Lx * std::rint(d / Lx);
  return d;
}
double Prep::dispy(int a, int b) const {
  double d = y[b] - y[a];
  if (periodic_y) d = d - Ly * std::rint(d / Ly);
  return d;
}

// Complete Taylor basis x^a y^b/(a! b!) ordered by degree, then by decreasing a (Sec. 2.2).
static int nterms(int deg) { return (deg + 1) * (deg + 2) / 2; }

static void taylor(double x, double y, int deg, double* p, double* px, double* py) {
  double xp[8], yp[8], fact[8];
  xp[0] = yp[0] = fact[0] = 1.0;
  for (int k = 1; k <= deg; ++k) {
    xp[k] = xp[k - 1] * x;
    yp[k] = yp[k - 1] * y;
    fact[k] = fact[k - 1] * k;
  }
  int i = 0;
  for (int d = 0; d <= deg; ++d)
    for (int b = 0; b <= d; ++b, ++i) {
      int a = d - b;
      p[i] = xp[a] * yp[b] / (fact[a] * fact[b]);
      if (px) px[i] = a > 0 ? xp[a - 1] * yp[b] / (fact[a - 1] * fact[b]) : 0.0;
      if (py) py[i] = b > 0 ? xp[a] * yp[b - 1] / (fact[a] * fact[b - 1]) : 0.0;
    }
}

// 3-node weights of Eq. (3nodes_intp) in unscaled midpoint-relative coordinates: A = [p_3(x_k)]
// (3 x 6) has full row rank for distinct nodes, A^+ = A^T (A A^T)^-1, and its first row is
// w = (A A^T)^-1 1 because A's first column is all ones.  A A^T is nearly singular for short
// edges, so G and Cramer's rule are evaluated in double-double; the value weights are then
// made to sum to one at node `near` (constant consistency) before the final rounding.
static void three_node(const double (*rel)[2], int near, double* w) {
  dd A[3][6];
  for (int k = 0; k < 3; ++k) {
    double x = rel[k][0], y = rel[k][1];
    dd xx = two_prod(x, x), xy = two_prod(x, y), yy = two_prod(y, y);
    A[k][0] = dd_from(1.0);
    A[k][1] = dd_from(x);
    A[k][2] = dd_from(y);
    A[k][3] = {xx.hi * 0.5, xx.lo * 0.5};
    A[k][4] = xy;
    A[k][5] = {yy.hi * 0.5, yy.lo * 0.5};
  }
  dd G[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      dd s = dd_from(0.0);
      for (int k = 0; k < 6; ++k) s = dd_add(s, dd_mul(A[i][k], A[j][k]));
      G[i][j] = s;
    }
  auto det3 = [](dd M[3][3]) {
    dd a = dd_add(dd_mul(M[1][1], M[2][2]), dd_neg(dd_mul(M[1][2], M[2][1])));
    dd b = dd_add(dd_mul(M[1][0], M[2][2]), dd_neg(dd_mul(M[1][2], M[2][0])));
    dd c = dd_add(dd_mul(M[1][0], M[2][1]), dd_neg(dd_mul(M[1][1], M[2][0])));
    return dd_add(dd_add(dd_mul(M[0][0], a), dd_neg(dd_mul(M[0][1], b))), dd_mul(M[0][2], c));
  };
  dd den = det3(G);
  dd num[3];
  for (int c = 0; c < 3; ++c) {
    dd M[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[i][j] = (j == c) ? dd_from(1.0) : G[i][j];
    num[c] = det3(M);
  }
  dd sum = dd_add(dd_add(num[0], num[1]), num[2]);
  num[near] = dd_add(num[near], dd_add(den, dd_neg(sum)));
  for (int c = 0; c < 3; ++c) {
    dd q = dd_div(num[c], den);
    w[c] = q.hi + q.lo;
  }
}

// 5-node Hermite weights (Sec. 2.2) for nodes rel[5] (relative to the edge midpoint), edge
// length ell, near node index 2.  Scaled coordinates (x/ell): data (c, ell c_x, ell c_y).
// Keep singular values > sv_rtol*sigma_max, then drop the smallest while any stored scaled
// weight has magnitude >= 1.  Unscale derivative weights, fix value weights to sum to one.
static int five_node(const double (*rel)[2], double ell, double sv_rtol, double* w) {
  double P[15 * 15], V[15 * 15], s[15];
  double p[15], px[15], py[15];
  for (int j = 0; j < 5; ++j) {
    taylor(rel[j][0] / ell, rel[j][1] / ell, 4, p, px, py);
    for (int k = 0; k < 15; ++k) {            // row 3j (+1, +2), column-major storage
      P[(3 * j) + 15 * k] = p[k];
      P[(3 * j + 1) + 15 * k] = px[k];
      P[(3 * j + 2) + 15 * k] = py[k];
    }
  }
  jacobi_svd(15, 15, P, V, s);
  int r = 0;
  for (int i = 0; i < 15; ++i)
    if (s[i] > sv_rtol * s[0]) ++r;
  for (;;) {
    double mx = 0;
    for (int i = 0; i < 15; ++i) w[i] = 0.0;
    for (int k = 0; k < r; ++k) {
      double f = V[0 + 15 * k] / (s[k] * s[k]);   // V[0,k] U[:,k] / s_k, with U s = A V
      for (int i = 0; i < 15; ++i) w[i] += f * P[i + 15 * k];
    }
    for (int i = 0; i < 15; ++i) mx = std::max(mx, std::fabs(w[i]));
    if (mx < 1.0) break;
    if (--r == 0) return 0;
  }
  double sum = 0;
  for (int j = 0; j < 5; ++j) {
    w[3 * j + 1] *= ell;
    w[3 * j + 2] *= ell;
  }
  for (int j = 0; j < 5; ++j) sum += w[3 * j];
  w[6] += 1.0 - sum;
  return r;
}

// ------------------------------------------------------------------ build

// One stencil extension (Sec. 2.1): neighbour of cur, not yet used, with the largest cosine
// to the travel direction t; ties within 1e-12 keep the lower id (ascending scan).
static int extend(const Prep& P, int cur, double tx, double ty, const int* used, int nused,
                  double* dx, double* dy) {
  double tn = std::sqrt(tx * tx + ty * ty);
  int best = -1;
  double bc = -INFINITY, bx = 0, by = 0;
  for (int k = P.nbr_ptr[cur]; k < P.nbr_ptr[cur + 1]; ++k) {
    int c = P.nbr_idx[k];
    bool u = false;
    for (int i = 0; i < nused; ++i) u |= (used[i] == c);
    if (u) continue;
    double ex = P.dispx(cur, c), ey = P.dispy(cur, c);
    double cs = (tx * ex + ty * ey) / (tn * std::sqrt(ex * ex + ey * ey));
    if (cs > bc + 1e-12) { best = c; bc = cs; bx = ex; by = ey; }
  }
  *dx = bx;
  *dy = by;
  return best;
}

hfd_status build_prep(const hfd_mesh_desc* d, const hfd_options* o, Prep* P) {
  auto t0 = std::chrono::steady_clock::now();
  if (!d || !o || !d->x || !d->y || !d->tri || d->nv <= 0 || d->ntri <= 0) {
    set_error("hfd_prep_create: null pointer or empty mesh");
    return HFD_ERR_ARG;
  }
  if (o->div_degree < 2 || o->div_degree > 6 || o->visc_degree < 2 || o->visc_degree > 6 ||
      o->precision < 0 || o->precision > 1 || !(o->visc_coef_max > 0.0) ||
      (o->dev_alloc == nullptr) != (o->dev_free == nullptr) || o->flux < 0 || o->flux > 1 ||
      o->conservative < 0 || o->conservative > 1 || o->force_branch < 0 || o->force_branch > 2) {
    set_error("hfd_prep_create: option out of range");
    return HFD_ERR_ARG;
  }
  P->opts = *o;
  const int nv = d->nv;
  P->nv = nv;
  P->x.assign(d->x, d->x + nv);
  P->y.assign(d->y, d->y + nv);
  P->tri.assign(d->tri, d->tri + 3 * (size_t)d->ntri);
  P->Lx = d->Lx;
  P->Ly = d->Ly;
  P->periodic_x = d->periodic_x;
  P->periodic_y = d->periodic_y;
  if ((P->periodic_x && !(d->Lx > 0)) || (P->periodic_y && !(d->Ly > 0))) {
    set_error("hfd_prep_create: periodic axis needs a positive period");
    return HFD_ERR_ARG;
  }
  P->is_ghost.assign(nv, 0);
  if (d->nghost > 0) {
    if (!d->ghost_ids || !d->ghost_donor || !d->ghost_flags) {
      set_error("hfd_prep_create: ghost arrays missing");
      return HFD_ERR_ARG;
    }
    P->ghost_ids.assign(d->ghost_ids, d->ghost_ids + d->nghost);
    P->ghost_donor.assign(d->ghost_donor, d->ghost_donor + d->nghost);
    P->ghost_flags.assign(d->ghost_flags, d->ghost_flags + d->nghost);
    for (int g = 0; g < d->nghost; ++g) {
      int id = d->ghost_ids[g];
      if (id < 0 || id >= nv || P->is_ghost[id]) {
        set_error("hfd_prep_create: ghost id %d invalid or repeated", id);
        return HFD_ERR_MESH;
      }
      P->is_ghost[id] = 1;
    }
    for (int g = 0; g < d->nghost; ++g) {
      int dn = d->ghost_donor[g];
      if (dn == -1) continue;              // fixed ghost: the caller's values are kept
      if (dn < 0 || dn >= nv || P->is_ghost[dn]) {
        set_error("hfd_prep_create: ghost donor %d invalid (must be a non-ghost vertex or -1)", dn);
        return HFD_ERR_MESH;
      }
    }
  }
  // ---- edges
  std::vector<uint64_t> keys;
  keys.reserve(3 * (size_t)d->ntri);
  for (int t = 0; t < d->ntri; ++t) {
    const int* v = &P->tri[3 * (size_t)t];
    for (int k = 0; k < 3; ++k) {
      int a = v[k], b = v[(k + 1) % 3];
      if (a < 0 || a >= nv || b < 0 || b >= nv || a == b) {
        set_error("hfd_prep_create: triangle %d has an invalid vertex", t);
        return HFD_ERR_MESH;
      }
      if (a > b) std::swap(a, b);
      keys.push_back(((uint64_t)a << 32) | (uint32_t)b);
    }
  }
  std::sort(keys.begin(), keys.end());
  {
    // manifold check: an edge may appear in at most two triangles
    size_t run = 1;
    for (size_t i = 1; i <= keys.size(); ++i) {
      if (i < keys.size() && keys[i] == keys[i - 1]) { ++run; continue; }
      if (run > 2) {
        set_error("hfd_prep_create: edge (%u,%u) shared by %zu triangles",
                  (unsigned)(keys[i - 1] >> 32), (unsigned)(keys[i - 1] & 0xffffffffu), run);
        return HFD_ERR_MESH;
      }
      run = 1;
    }
  }
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  const int64_t E = (int64_t)keys.size();
  P->edges.resize(2 * E);
  std::vector<int32_t> deg(nv, 0);
  for (int64_t e = 0; e < E; ++e) {
    int a = (int)(keys[e] >> 32), b = (int)(keys[e] & 0xffffffffu);
    P->edges[2 * e] = a;
    P->edges[2 * e + 1] = b;
    deg[a]++;
    deg[b]++;
  }
  P->nbr_ptr.assign(nv + 1, 0);
  for (int v = 0; v < nv; ++v) P->nbr_ptr[v + 1] = P->nbr_ptr[v] + deg[v];
  P->nbr_idx.resize(2 * E);
  P->nbr_edge.resize(2 * E);
  {
    std::vector<int32_t> fill(P->nbr_ptr.begin(), P->nbr_ptr.end() - 1);
    for (int64_t e = 0; e < E; ++e) {       // edges sorted by (a, b): lists come out sorted
      int a = P->edges[2 * e], b = P->edges[2 * e + 1];
      P->nbr_idx[fill[a]] = b;
      P->nbr_edge[fill[a]++] = (int32_t)e;
    }
    for (int64_t e = 0; e < E; ++e) {
      int a = P->edges[2 * e], b = P->edges[2 * e + 1];
      P->nbr_idx[fill[b]] = a;
      P->nbr_edge[fill[b]++] = (int32_t)e;
    }
    for (int v = 0; v < nv; ++v) {          // sort each list by neighbour id
      int s = P->nbr_ptr[v], t = P->nbr_ptr[v + 1];
      std::vector<std::pair<int, int>> tmp;
      for (int k = s; k < t; ++k) tmp.push_back({P->nbr_idx[k], P->nbr_edge[k]});
      std::sort(tmp.begin(), tmp.end());
      for (int k = s; k < t; ++k) {
        P->nbr_idx[k] = tmp[k - s].first;
        P->nbr_edge[k] = tmp[k - s].second;
      }
    }
  }
  P->lmin.assign(nv, 0.0);
  for (int v = 0; v < nv; ++v) {
    double m = INFINITY;
    for (int k = P->nbr_ptr[v]; k < P->nbr_ptr[v + 1]; ++k) {
      double ex = P->dispx(v, P->nbr_idx[k]), ey = P->dispy(v, P->nbr_idx[k]);
      m = std::min(m, std::sqrt(ex * ex + ey * ey));
    }
    P->lmin[v] = m;
  }
  if (o->conservative) {
    // median-dual geometry: per triangle, the segment from each edge's midpoint to the
    // centroid, turned by 90 degrees and oriented tail -> head, adds to that edge's dual face;
    // a third of the triangle's area goes to each corner's cell (triangle order, as a reference
    // evaluation would sum them)
    P->dual_S.assign(2 * E, 0.0);
    P->dual_A.assign(nv, 0.0);
    for (int t = 0; t < d->ntri; ++t) {
      const int* tv = &P->tri[3 * (size_t)t];
      double x[3][2] = {{0.0, 0.0},
                        {P->dispx(tv[0], tv[1]), P->dispy(tv[0], tv[1])},
                        {P->dispx(tv[0], tv[2]), P->dispy(tv[0], tv[2])}};
      double gx = (x[0][0] + x[1][0] + x[2][0]) / 3.0, gy = (x[0][1] + x[1][1] + x[2][1]) / 3.0;
      static const int pr[3][2] = {{0, 1}, {1, 2}, {2, 0}};
      for (int k = 0; k < 3; ++k) {
        int i = pr[k][0], j = pr[k][1];
        int ia = tv[i] < tv[j] ? i : j, ib = ia == i ? j : i;
        double sx = gx - 0.5 * (x[i][0] + x[j][0]), sy = gy - 0.5 * (x[i][1] + x[j][1]);
        double nx = sy, ny = -sx;
        if (nx * (x[ib][0] - x[ia][0]) + ny * (x[ib][1] - x[ia][1]) < 0) { nx = -nx; ny = -ny; }
        uint64_t key = ((uint64_t)tv[ia] << 32) | (uint32_t)tv[ib];
        int64_t e = std::lower_bound(keys.begin(), keys.end(), key) - keys.begin();
        P->dual_S[2 * e] += nx;
        P->dual_S[2 * e + 1] += ny;
      }
      double area = 0.5 * (x[1][0] * x[2][1] - x[1][1] * x[2][0]);
      for (int k = 0; k < 3; ++k) P->dual_A[tv[k]] += area / 3.0;
    }
  }
  int nthreads = o->nthreads > 0 ? o->nthreads : (int)std::max(1u, std::thread::hardware_concurrency());

  // ---- two-level stencils of active vertices (Fig. 6: distance <= 2, edges inside the set)
  for (int v = 0; v < nv; ++v)
    if (!P->is_ghost[v]) P->active.push_back(v);
  const int64_t A = (int64_t)P->active.size();
  std::vector<std::vector<int32_t>> sv(A), se(A);
  {
    std::vector<std::vector<int32_t>> mark(nthreads, std::vector<int32_t>(nv, -1));
    parallel_for(A, nthreads, [&](int64_t r, int t) {
      int v = P->active[r];
      auto& mk = mark[t];
      std::vector<int32_t>& verts = sv[r];
      verts.push_back(v);
      mk[v] = (int)r;
      for (int k = P->nbr_ptr[v]; k < P->nbr_ptr[v + 1]; ++k) {
        int u = P->nbr_idx[k];
        if (mk[u] != r) { mk[u] = (int)r; verts.push_back(u); }
      }
      size_t n1 = verts.size();
      for (size_t i = 1; i < n1; ++i) {
        int u = verts[i];
        for (int k = P->nbr_ptr[u]; k < P->nbr_ptr[u + 1]; ++k) {
          int w = P->nbr_idx[k];
          if (mk[w] != r) { mk[w] = (int)r; verts.push_back(w); }
        }
      }
      std::sort(verts.begin(), verts.end());
      for (int u : verts)
        for (int k = P->nbr_ptr[u]; k < P->nbr_ptr[u + 1]; ++k) {
          int w = P->nbr_idx[k];
          if (w > u && mk[w] == r) se[r].push_back(P->nbr_edge[k]);
        }
      std::sort(se[r].begin(), se[r].end());
      for (int u : verts) mk[u] = -1;
    });
  }
  P->div_vptr.assign(A + 1, 0);
  P->div_eptr.assign(A + 1, 0);
  P->div_cptr.assign(A + 1, 0);
  for (int64_t r = 0; r < A; ++r) {
    P->div_vptr[r + 1] = P->div_vptr[r] + (int)sv[r].size();
    P->div_eptr[r + 1] = P->div_eptr[r] + (int)se[r].size();
    P->div_cptr[r + 1] = P->div_cptr[r] + 3 * (int64_t)(2 * sv[r].size() + se[r].size());
  }
  P->div_vidx.resize(P->div_vptr[A]);
  P->div_eidx.resize(P->div_eptr[A]);
  P->div_coef.assign(P->div_cptr[A], 0.0);
  P->div_degree.assign(A, 0);
  if (o->viscous) {
    P->visc_cptr.assign(A + 1, 0);
    for (int64_t r = 0; r < A; ++r) P->visc_cptr[r + 1] = P->visc_cptr[r] + 6 * (int64_t)sv[r].size();
    P->visc_coef.assign(P->visc_cptr[A], 0.0);
    P->visc_degree.assign(A, 0);
  }
  ErrorSlot err;
  std::atomic<int64_t> fallbacks(0), visc_fallbacks(0);
  parallel_for(A, nthreads, [&](int64_t r, int) {
    int v = P->active[r];
    const auto& verts = sv[r];
    const auto& eds = se[r];
    std::copy(verts.begin(), verts.end(), P->div_vidx.begin() + P->div_vptr[r]);
    std::copy(eds.begin(), eds.end(), P->div_eidx.begin() + P->div_eptr[r]);
    int N = (int)verts.size(), M = (int)eds.size();
    double ell = 0;
    int nn = 0;
    for (int k = P->nbr_ptr[v]; k < P->nbr_ptr[v + 1]; ++k, ++nn) {
      double ex = P->dispx(v, P->nbr_idx[k]), ey = P->dispy(v, P->nbr_idx[k]);
      ell += std::sqrt(ex * ex + ey * ey);
    }
    ell /= nn;
    std::vector<double> xv(2 * N), xm(2 * M), nm(2 * M);
    for (int j = 0; j < N; ++j) {
      xv[2 * j] = P->dispx(v, verts[j]) / ell;
      xv[2 * j + 1] = P->dispy(v, verts[j]) / ell;
    }
    for (int j = 0; j < M; ++j) {
      int a = P->edges[2 * eds[j]], b = P->edges[2 * eds[j] + 1];
      double ex = P->dispx(a, b), ey = P->dispy(a, b);
      xm[2 * j] = (P->dispx(v, a) + 0.5 * ex) / ell;
      xm[2 * j + 1] = (P->dispy(v, a) + 0.5 * ey) / ell;
      if (o->conservative) {                 // h is the flux along the dual-face normal
        ex = P->dual_S[2 * (size_t)eds[j]];
        ey = P->dual_S[2 * (size_t)eds[j] + 1];
      }
      double len = std::sqrt(ex * ex + ey * ey);
      nm[2 * j] = ex / len;
      nm[2 * j + 1] = ey / len;
    }
    int degv = o->div_degree;
    int rows = 2 * N + M;
    std::vector<double> out(3 * (size_t)rows);
    double p[32];
    for (;;) {
      int K = nterms(degv), n = 2 * K;
      if (rows < n) { --degv; if (degv < 1) break; continue; }
      std::vector<double> Am((size_t)rows * n, 0.0);
      for (int j = 0; j < N; ++j) {
        taylor(xv[2 * j], xv[2 * j + 1], degv, p, nullptr, nullptr);
        for (int k = 0; k < K; ++k) {
          Am[(2 * j) + (size_t)k * rows] = p[k];
          Am[(2 * j + 1) + (size_t)(K + k) * rows] = p[k];
        }
      }
      for (int j = 0; j < M; ++j) {
        taylor(xm[2 * j], xm[2 * j + 1], degv, p, nullptr, nullptr);
        for (int k = 0; k < K; ++k) {
          Am[(2 * N + j) + (size_t)k * rows] = p[k] * nm[2 * j];
          Am[(2 * N + j) + (size_t)(K + k) * rows] = p[k] * nm[2 * j + 1];
        }
      }
      const int targ[3][2] = {{1, K + 2}, {3, K + 4}, {4, K + 5}};
      double cond = ls_rows(rows, n, Am, targ, 3, out.data());
      if (cond >= o->div_cond_min || degv <= 2) break;
      --degv;
      fallbacks++;
    }
    P->div_degree[r] = degv;
    double* c = &P->div_coef[P->div_cptr[r]];
    for (int i = 0; i < rows; ++i) {
      c[i] = out[i] / ell;
      c[rows + i] = out[rows + i] / (ell * ell);
      c[2 * rows + i] = out[2 * rows + i] / (ell * ell);
    }
    if (o->conservative) {
      // the value rows as the median-dual cell's boundary integral: the flux through face e,
      // |S_e| h_e, leaves the tail's cell and enters the head's
      for (int i = 0; i < rows; ++i) c[i] = 0.0;
      for (int j = 0; j < M; ++j) {
        int a = P->edges[2 * eds[j]], b = P->edges[2 * eds[j] + 1];
        if (a != v && b != v) continue;
        double sx = P->dual_S[2 * (size_t)eds[j]], sy = P->dual_S[2 * (size_t)eds[j] + 1];
        double mag = std::sqrt(sx * sx + sy * sy);
        c[2 * N + j] = (a == v ? 1.0 : -1.0) * mag / P->dual_A[v];
      }
    }
    if (o->viscous) {                       // vertex-only LS, f and g decoupled (Sec. 2.3)
      // Degree visc_degree, dropping by one while a weight of the rows used (first and second
      // derivatives, l_v-scaled) exceeds visc_coef_max: nearly unisolvent vertex sets give
      // exploding weights and a locally unstable viscous operator (down to degree 2).
      std::vector<double> q(5 * (size_t)N);
      int degz = o->visc_degree;
      for (;;) {
        int K = nterms(degz);
        std::vector<double> B((size_t)N * K);
        for (int j = 0; j < N; ++j) {
          taylor(xv[2 * j], xv[2 * j + 1], degz, p, nullptr, nullptr);
          for (int k = 0; k < K; ++k) B[j + (size_t)k * N] = p[k];
        }
        if (N >= K) {
          const int targ[5][2] = {{1, -1}, {2, -1}, {3, -1}, {4, -1}, {5, -1}};
          ls_rows(N, K, B, targ, 5, q.data());
        } else {          // fewer stencil vertices than basis terms: minimum-norm solution
          const int t1[5] = {1, 2, 3, 4, 5};
          pinv_rows_svd(N, K, B, t1, 5, q.data());
        }
        double big = 0;
        for (double x : q) big = std::max(big, std::fabs(x));
        if (big <= o->visc_coef_max || degz <= 2) break;
        --degz;
        visc_fallbacks++;
      }
      P->visc_degree[r] = degz;
      double* e = &P->visc_coef[P->visc_cptr[r]];
      double l2 = ell * ell;
      for (int j = 0; j < N; ++j) {           // rows over interleaved (f_j, g_j)
        e[2 * j] = q[0 * N + j] / ell;
        e[2 * j + 1] = q[1 * N + j] / ell;
        e[2 * N + 2 * j] = q[2 * N + j] / l2;
        e[2 * N + 2 * j + 1] = q[3 * N + j] / l2;
        e[4 * N + 2 * j] = q[3 * N + j] / l2;
        e[4 * N + 2 * j + 1] = q[4 * N + j] / l2;
      }
    }
  });
  if (err.st != HFD_OK) {
    set_error("%s", err.msg);
    return err.st;
  }
  P->degree_fallbacks = fallbacks.load();
  P->visc_fallbacks = visc_fallbacks.load();

  // ---- flux edges and their stencils / weights
  {
    std::vector<uint8_t> need(E, 0);
    for (int32_t e : P->div_eidx) need[e] = 1;
    for (int64_t e = 0; e < E; ++e)
      if (need[e]) P->flux_edges.push_back((int32_t)e);
  }
  const int64_t Ef = (int64_t)P->flux_edges.size();
  P->stencil.assign(6 * Ef, 0);
  P->normal.assign(2 * Ef, 0.0);
  P->w5.assign(30 * Ef, 0.0);
  P->w3.assign(18 * Ef, 0.0);
  P->rank.assign(2 * Ef, 0);
  static const int L3[3][3] = {{0, 1, 2}, {1, 2, 3}, {2, 3, 4}};
  static const int R3[3][3] = {{5, 4, 3}, {4, 3, 2}, {3, 2, 1}};
  parallel_for(Ef, nthreads, [&](int64_t f, int) {
    int e = P->flux_edges[f];
    int a = P->edges[2 * e], b = P->edges[2 * e + 1];
    int used[6] = {a, b, 0, 0, 0, 0};
    double dabx = P->dispx(a, b), daby = P->dispy(a, b);
    double d1x, d1y, d2x, d2y, d3x, d3y, d4x, d4y;
    int b1 = extend(*P, a, -dabx, -daby, used, 2, &d1x, &d1y);
    if (b1 < 0) goto fail;
    used[2] = b1;
    {
      int b2 = extend(*P, b1, d1x, d1y, used, 3, &d2x, &d2y);
      if (b2 < 0) goto fail;
      used[3] = b2;
      int f1 = extend(*P, b, dabx, daby, used, 4, &d3x, &d3y);
      if (f1 < 0) goto fail;
      used[4] = f1;
      int f2 = extend(*P, f1, d3x, d3y, used, 5, &d4x, &d4y);
      if (f2 < 0) goto fail;
      int ids[6] = {b2, b1, a, b, f1, f2};
      double pos[6][2];
      pos[2][0] = 0.0; pos[2][1] = 0.0;
      pos[1][0] = d1x; pos[1][1] = d1y;
      pos[0][0] = pos[1][0] + d2x; pos[0][1] = pos[1][1] + d2y;
      pos[3][0] = dabx; pos[3][1] = daby;
      pos[4][0] = pos[3][0] + d3x; pos[4][1] = pos[3][1] + d3y;
      pos[5][0] = pos[4][0] + d4x; pos[5][1] = pos[4][1] + d4y;
      double hx = 0.5 * pos[3][0], hy = 0.5 * pos[3][1];
      double rel[6][2];
      for (int k = 0; k < 6; ++k) { rel[k][0] = pos[k][0] - hx; rel[k][1] = pos[k][1] - hy; }
      double ell = std::sqrt(dabx * dabx + daby * daby);
      for (int k = 0; k < 6; ++k) P->stencil[6 * f + k] = ids[k];
      P->normal[2 * f] = dabx / ell;
      P->normal[2 * f + 1] = daby / ell;
      if (o->conservative) {             // projection and Riemann flux along the dual normal
        double sx = P->dual_S[2 * (size_t)e], sy = P->dual_S[2 * (size_t)e + 1];
        double sl = std::sqrt(sx * sx + sy * sy);
        P->normal[2 * f] = sx / sl;
        P->normal[2 * f + 1] = sy / sl;
      }
      int rl = five_node(&rel[0], ell, o->sv_rtol, &P->w5[30 * f]);
      int rr = five_node(&rel[1], ell, o->sv_rtol, &P->w5[30 * f + 15]);
      if (rl == 0 || rr == 0) {
        err.set(HFD_ERR_SINGULAR, "5-node system kept no singular value");
        return;
      }
      P->rank[2 * f] = rl;
      P->rank[2 * f + 1] = rr;
      for (int j = 0; j < 3; ++j) {
        double r3[3][2];
        int nearL = -1, nearR = -1;
        for (int k = 0; k < 3; ++k) {
          r3[k][0] = rel[L3[j][k]][0]; r3[k][1] = rel[L3[j][k]][1];
          if (L3[j][k] == 2) nearL = k;
        }
        three_node(r3, nearL, &P->w3[18 * f + 3 * j]);
        for (int k = 0; k < 3; ++k) {
          r3[k][0] = rel[R3[j][k]][0]; r3[k][1] = rel[R3[j][k]][1];
          if (R3[j][k] == 3) nearR = k;
        }
        three_node(r3, nearR, &P->w3[18 * f + 9 + 3 * j]);
      }
      return;
    }
  fail:
    char m[160];
    snprintf(m, sizeof m, "stencil of edge (%d,%d) cannot be extended (Sec. 2.1)", a, b);
    err.set(HFD_ERR_STENCIL, m);
  });
  if (err.st != HFD_OK) {
    set_error("%s", err.msg);
    return err.st;
  }
  P->prep_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return HFD_OK;
}

}  // namespace hfd

// ------------------------------------------------------------------ C ABI (host part)
using hfd::Prep;

extern "C" {

void hfd_default_options(hfd_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->precision = 0;
  o->div_degree = 5;
  o->visc_degree = 4;
  o->viscous = 0;
  o->renumber = 1;
  o->nthreads = 0;
  o->gamma = 1.4;
  o->mu = 0.0;
  o->prandtl = 0.72;
  o->R_gas = 1.0;
  o->weno_eps = 1e-2;
  o->sens_lo = 0.01;
  o->sens_hi = 0.79;
  o->sv_rtol = 1e-13;
  o->div_cond_min = 1e-12;
  o->visc_coef_max = 8.0;
  o->harten = 0.1;
  o->cfl = 0.3;
}

const char* hfd_last_error(void) { return hfd::last_error(); }

hfd_status hfd_prep_create(const hfd_mesh_desc* desc, const hfd_options* opts, hfd_prep** out) {
  if (!out) { hfd::set_error("hfd_prep_create: out is null"); return HFD_ERR_ARG; }
  *out = nullptr;
  hfd_options def;
  if (!opts) { hfd_default_options(&def); opts = &def; }
  hfd_prep* p = new (std::nothrow) hfd_prep();
  if (!p) { hfd::set_error("hfd_prep_create: out of host memory"); return HFD_ERR_ARG; }
  hfd_status st;
  try {
    st = hfd::build_prep(desc, opts, p);
  } catch (const std::exception& e) {
    hfd::set_error("hfd_prep_create: %s", e.what());
    st = HFD_ERR_ARG;
  }
  if (st != HFD_OK) { delete p; return st; }
  *out = p;
  return HFD_OK;
}

void hfd_prep_destroy(hfd_prep* p) { delete p; }

namespace {
struct Arr { void* ptr; int64_t n; size_t elt; bool writable; };
Arr lookup(const Prep* P, const char* name) {
  auto I = [](const std::vector<int32_t>& v) {
    return Arr{(void*)v.data(), (int64_t)v.size(), 4, false};
  };
  auto D = [](const std::vector<double>& v, bool w) {
    return Arr{(void*)v.data(), (int64_t)v.size(), 8, w};
  };
  std::string s(name ? name : "");
  if (s == "edges") return I(P->edges);
  if (s == "flux_edges") return I(P->flux_edges);
  if (s == "stencil") return I(P->stencil);
  if (s == "normal") return D(P->normal, false);
  if (s == "w5") return D(P->w5, true);
  if (s == "w3") return D(P->w3, true);
  if (s == "rank") return I(P->rank);
  if (s == "active") return I(P->active);
  if (s == "div_vptr") return I(P->div_vptr);
  if (s == "div_vidx") return I(P->div_vidx);
  if (s == "div_eptr") return I(P->div_eptr);
  if (s == "div_eidx") return I(P->div_eidx);
  if (s == "div_coef") return D(P->div_coef, true);
  if (s == "div_degree") return I(P->div_degree);
  if (s == "visc_coef") return D(P->visc_coef, true);
  if (s == "visc_degree") return I(P->visc_degree);
  if (s == "lmin") return D(P->lmin, false);
  if (s == "dual_S") return D(P->dual_S, false);
  if (s == "dual_A") return D(P->dual_A, false);
  return Arr{nullptr, -1, 0, false};
}
}  // namespace

hfd_status hfd_prep_concat(const hfd_prep* const* preps, int32_t n, hfd_prep** out) {
  if (!preps || n <= 0 || !out) { hfd::set_error("hfd_prep_concat: invalid argument"); return HFD_ERR_ARG; }
  *out = nullptr;
  const hfd_options& o0 = preps[0]->opts;
  for (int k = 0; k < n; ++k) {
    if (!preps[k]) { hfd::set_error("hfd_prep_concat: null prep %d", k); return HFD_ERR_ARG; }
    const hfd_options& o = preps[k]->opts;
    if (o.viscous != o0.viscous || o.gamma != o0.gamma || o.mu != o0.mu || o.prandtl != o0.prandtl ||
        o.R_gas != o0.R_gas || o.weno_eps != o0.weno_eps || o.sens_lo != o0.sens_lo ||
        o.sens_hi != o0.sens_hi || o.harten != o0.harten || o.cfl != o0.cfl ||
        o.precision != o0.precision || o.visc_coef_max != o0.visc_coef_max || o.flux != o0.flux ||
        o.conservative != o0.conservative || o.force_branch != o0.force_branch) {
      hfd::set_error("hfd_prep_concat: member %d has different physical/numerical options", k);
      return HFD_ERR_ARG;
    }
  }
  hfd_prep* B = new (std::nothrow) hfd_prep();
  if (!B) { hfd::set_error("hfd_prep_concat: out of host memory"); return HFD_ERR_ARG; }
  B->opts = o0;
  B->nmember = n;
  int64_t voff = 0, eoff = 0;
  for (int k = 0; k < n; ++k) {
    const Prep& P = *preps[k];
    const int32_t vo = (int32_t)voff, eo = (int32_t)eoff;
    auto addv = [&](std::vector<int32_t>& dst, const std::vector<int32_t>& src, int32_t off) {
      for (int32_t v : src) dst.push_back(v + off);
    };
    B->x.insert(B->x.end(), P.x.begin(), P.x.end());
    B->y.insert(B->y.end(), P.y.begin(), P.y.end());
    addv(B->tri, P.tri, vo);
    addv(B->ghost_ids, P.ghost_ids, vo);
    for (int32_t dn : P.ghost_donor) B->ghost_donor.push_back(dn < 0 ? dn : dn + vo);
    B->ghost_flags.insert(B->ghost_flags.end(), P.ghost_flags.begin(), P.ghost_flags.end());
    B->is_ghost.insert(B->is_ghost.end(), P.is_ghost.begin(), P.is_ghost.end());
    addv(B->edges, P.edges, vo);
    addv(B->active, P.active, vo);
    const int64_t A0 = (int64_t)B->div_vptr.size() ? B->div_vptr.back() : 0;
    const int64_t E0 = (int64_t)B->div_eptr.size() ? B->div_eptr.back() : 0;
    const int64_t C0 = (int64_t)B->div_cptr.size() ? B->div_cptr.back() : 0;
    const int64_t Z0 = (int64_t)B->visc_cptr.size() ? B->visc_cptr.back() : 0;
    if (B->div_vptr.empty()) { B->div_vptr.push_back(0); B->div_eptr.push_back(0); B->div_cptr.push_back(0); }
    if (P.opts.viscous && B->visc_cptr.empty()) B->visc_cptr.push_back(0);
    for (size_t r = 1; r < P.div_vptr.size(); ++r) {
      B->div_vptr.push_back((int32_t)(A0 + P.div_vptr[r]));
      B->div_eptr.push_back((int32_t)(E0 + P.div_eptr[r]));
      B->div_cptr.push_back(C0 + P.div_cptr[r]);
      if (P.opts.viscous) B->visc_cptr.push_back(Z0 + P.visc_cptr[r]);
    }
    addv(B->div_vidx, P.div_vidx, vo);
    addv(B->div_eidx, P.div_eidx, eo);
    B->div_degree.insert(B->div_degree.end(), P.div_degree.begin(), P.div_degree.end());
    B->visc_degree.insert(B->visc_degree.end(), P.visc_degree.begin(), P.visc_degree.end());
    B->div_coef.insert(B->div_coef.end(), P.div_coef.begin(), P.div_coef.end());
    B->visc_coef.insert(B->visc_coef.end(), P.visc_coef.begin(), P.visc_coef.end());
    addv(B->flux_edges, P.flux_edges, eo);
    addv(B->stencil, P.stencil, vo);
    B->normal.insert(B->normal.end(), P.normal.begin(), P.normal.end());
    B->w5.insert(B->w5.end(), P.w5.begin(), P.w5.end());
    B->w3.insert(B->w3.end(), P.w3.begin(), P.w3.end());
    B->rank.insert(B->rank.end(), P.rank.begin(), P.rank.end());
    B->lmin.insert(B->lmin.end(), P.lmin.begin(), P.lmin.end());
    B->member.insert(B->member.end(), (size_t)P.nv, k);
    // the member's own space-filling-curve box, as a single mesh would use it
    double x0 = 0, x1 = P.Lx, y0 = 0, y1 = P.Ly;
    if (!P.periodic_x || !(x1 > 0)) {
      x0 = *std::min_element(P.x.begin(), P.x.end());
      x1 = *std::max_element(P.x.begin(), P.x.end());
    }
    if (!P.periodic_y || !(y1 > 0)) {
      y0 = *std::min_element(P.y.begin(), P.y.end());
      y1 = *std::max_element(P.y.begin(), P.y.end());
    }
    B->member_box.insert(B->member_box.end(), {x0, x1, y0, y1});
    B->degree_fallbacks += P.degree_fallbacks;
    B->visc_fallbacks += P.visc_fallbacks;
    B->prep_seconds += P.prep_seconds;
    voff += P.nv;
    eoff += P.nedges();
  }
  B->nv = (int32_t)voff;
  *out = B;
  return HFD_OK;
}

int64_t hfd_prep_size(const hfd_prep* p, const char* name) {
  if (!p) return -1;
  return lookup(p, name).n;
}

hfd_status hfd_prep_get(const hfd_prep* p, const char* name, void* dst, int64_t count) {
  if (!p || !dst) { hfd::set_error("hfd_prep_get: null argument"); return HFD_ERR_ARG; }
  Arr a = lookup(p, name);
  if (a.n < 0 || count != a.n) {
    hfd::set_error("hfd_prep_get: unknown array '%s' or wrong count", name ? name : "");
    return HFD_ERR_ARG;
  }
  std::memcpy(dst, a.ptr, a.elt * (size_t)a.n);
  return HFD_OK;
}

hfd_status hfd_prep_set(hfd_prep* p, const char* name, const void* src, int64_t count) {
  if (!p || !src) { hfd::set_error("hfd_prep_set: null argument"); return HFD_ERR_ARG; }
  Arr a = lookup(p, name);
  if (a.n < 0 || count != a.n || !a.writable) {
    hfd::set_error("hfd_prep_set: '%s' unknown, read-only or wrong count", name ? name : "");
    return HFD_ERR_ARG;
  }
  std::memcpy(a.ptr, src, a.elt * (size_t)a.n);
  return HFD_OK;
}

}  // extern "C"
