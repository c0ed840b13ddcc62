// C ABI of the device mesh: renumbering, upload of the coefficient streams, residual, SSP-RK3
// steps (direct launches or a replayed CUDA graph), end-to-end host form, error word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <type_traits>
#include <vector>

#include "kernels.hpp"
#include "mesh.hpp"
#include "prep.hpp"

using hfd::DevMesh;
using hfd::Phys;
using hfd::set_error;

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error("%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return HFD_ERR_CUDA;                                                         \
    }                                                                              \
  } while (0)

namespace {

// Hilbert index of (x, y) in [0, 2^16)^2 (the classic rotate-and-flip construction).
uint64_t hilbert(uint32_t x, uint32_t y) {
  uint64_t d = 0;
  for (uint32_t s = 1u << 15; s > 0; s >>= 1) {
    uint32_t rx = (x & s) ? 1 : 0, ry = (y & s) ? 1 : 0;
    d += (uint64_t)s * s * ((3 * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) { x = s - 1 - x; y = s - 1 - y; }
      std::swap(x, y);
    }
  }
  return d;
}

// Re-lays a divergence CSR (per vertex: `rows` SoA rows of n entries each, coef at
// rows * ptr[r]) into chunks of hfd::kDivChunk entries: ptr becomes chunk offsets, idx is
// padded to whole chunks with the vertex's first index, and each chunk holds its rows
// contiguously ([row][kDivChunk]) with zero coefficients in the padding.  `coef2` (the viscous
// rows, same shape as coef) follows the same layout.
template <typename T>
void chunk_rows(int A, std::vector<int32_t>& ptr, std::vector<int32_t>& idx, int rows,
                std::vector<T>& coef, std::vector<T>* coef2) {
  const int C = hfd::kDivChunk;
  std::vector<int32_t> cptr(A + 1, 0);
  for (int r = 0; r < A; ++r) cptr[r + 1] = cptr[r] + (ptr[r + 1] - ptr[r] + C - 1) / C;
  std::vector<int32_t> cidx((size_t)C * cptr[A]);
  std::vector<T> cc((size_t)rows * C * cptr[A], T(0)), cc2;
  if (coef2) cc2.assign(cc.size(), T(0));
  for (int r = 0; r < A; ++r) {
    int n = ptr[r + 1] - ptr[r];
    int nc = cptr[r + 1] - cptr[r];
    for (int k = 0; k < nc * C; ++k) {
      int j = k < n ? k : 0;
      cidx[(size_t)C * cptr[r] + k] = n > 0 ? idx[ptr[r] + j] : 0;
      if (k >= n) continue;
      size_t dst = (size_t)rows * C * cptr[r] + (size_t)(k / C) * rows * C + k % C;
      for (int row = 0; row < rows; ++row) {
        size_t src = (size_t)rows * ptr[r] + (size_t)row * n + k;
        cc[dst + (size_t)row * C] = coef[src];
        if (coef2) cc2[dst + (size_t)row * C] = (*coef2)[src];
      }
    }
  }
  ptr.swap(cptr);
  idx.swap(cidx);
  coef.swap(cc);
  if (coef2) coef2->swap(cc2);
}

template <typename T>
hfd_status dev_upload(hfd_mesh* m, void** dst, const std::vector<T>& src) {
  size_t bytes = std::max<size_t>(src.size() * sizeof(T), 16);
  void* p = nullptr;
  CK(mesh_malloc(m, &p, bytes));
  if (!src.empty()) CK(cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  *dst = p;
  return HFD_OK;
}

hfd_status dev_alloc(hfd_mesh* m, void** dst, size_t bytes) {
  void* p = nullptr;
  bytes = std::max<size_t>(bytes, 16);
  CK(mesh_malloc(m, &p, bytes));
  CK(cudaMemset(p, 0, bytes));
  *dst = p;
  return HFD_OK;
}

#define TRY(x)                       \
  do {                               \
    hfd_status s_ = (x);             \
    if (s_ != HFD_OK) return s_;     \
  } while (0)

// Upload the coefficient streams in bulk precision T.
template <typename T>
hfd_status upload_streams(hfd_mesh* m, const hfd::Prep& P, const std::vector<int32_t>& inv,
                          const std::vector<int32_t>& fint /* prep flux index -> internal */,
                          const std::vector<int32_t>& fperm /* internal -> prep flux index */,
                          const std::vector<int32_t>& emap /* edge -> internal flux id */) {
  DevMesh& d = m->dm;
  const int Ef = d.Ef, A = d.A;
  std::vector<int32_t> sten((size_t)6 * Ef);
  std::vector<T> nrm((size_t)2 * Ef), w5((size_t)30 * Ef), w3((size_t)18 * Ef);
  for (int fi = 0; fi < Ef; ++fi) {
    int f = fperm[fi];
    for (int k = 0; k < 6; ++k) sten[(size_t)k * Ef + fi] = inv[P.stencil[6 * (size_t)f + k]];
    nrm[fi] = (T)P.normal[2 * (size_t)f];
    nrm[(size_t)Ef + fi] = (T)P.normal[2 * (size_t)f + 1];
    for (int k = 0; k < 30; ++k) w5[(size_t)k * Ef + fi] = (T)P.w5[30 * (size_t)f + k];
    for (int k = 0; k < 18; ++k) w3[(size_t)k * Ef + fi] = (T)P.w3[18 * (size_t)f + k];
  }
  (void)fint;
  TRY(dev_upload(m, (void**)&d.sten, sten));
  TRY(dev_upload(m, &d.nrm, nrm));
  TRY(dev_upload(m, &d.w5, w5));
  TRY(dev_upload(m, &d.w3, w3));
  // divergence CSR in internal vertex order
  std::vector<int32_t> arow(P.nv, -1);
  for (size_t r = 0; r < P.active.size(); ++r) arow[P.active[r]] = (int32_t)r;
  std::vector<int32_t> vptr(A + 1, 0), eptr(A + 1, 0);
  for (int ri = 0; ri < A; ++ri) {
    int r = arow[m->perm[ri]];
    vptr[ri + 1] = vptr[ri] + (P.div_vptr[r + 1] - P.div_vptr[r]);
    eptr[ri + 1] = eptr[ri] + (P.div_eptr[r + 1] - P.div_eptr[r]);
  }
  std::vector<int32_t> vidx(vptr[A]), eidx(eptr[A]);
  std::vector<T> cv((size_t)6 * vptr[A]), ce((size_t)3 * eptr[A]), cvis;
  if (P.opts.viscous) cvis.resize((size_t)6 * vptr[A]);
  for (int ri = 0; ri < A; ++ri) {
    int r = arow[m->perm[ri]];
    int N = P.div_vptr[r + 1] - P.div_vptr[r], M = P.div_eptr[r + 1] - P.div_eptr[r];
    int L = 2 * N + M;
    const double* c = &P.div_coef[P.div_cptr[r]];
    T* cvb = &cv[(size_t)6 * vptr[ri]];
    T* ceb = &ce[(size_t)3 * eptr[ri]];
    for (int j = 0; j < N; ++j) {
      vidx[vptr[ri] + j] = inv[P.div_vidx[P.div_vptr[r] + j]];
      for (int row = 0; row < 3; ++row) {
        cvb[(2 * row) * N + j] = (T)c[row * L + 2 * j];
        cvb[(2 * row + 1) * N + j] = (T)c[row * L + 2 * j + 1];
      }
    }
    for (int j = 0; j < M; ++j) {
      eidx[eptr[ri] + j] = emap[P.div_eidx[P.div_eptr[r] + j]];
      for (int row = 0; row < 3; ++row) ceb[row * M + j] = (T)c[row * L + 2 * N + j];
    }
    if (P.opts.viscous) {
      const double* z = &P.visc_coef[P.visc_cptr[r]];
      T* cz = &cvis[(size_t)6 * vptr[ri]];
      for (int j = 0; j < N; ++j)
        for (int row = 0; row < 3; ++row) {
          cz[(2 * row) * N + j] = (T)z[row * 2 * N + 2 * j];
          cz[(2 * row + 1) * N + j] = (T)z[row * 2 * N + 2 * j + 1];
        }
    }
  }
  m->stats.div_nnz = vptr[A] * 2 + eptr[A];
  if (std::is_same<T, double>::value && A > 0) {
    // folded double-float divergence: each edge row's endpoint average (1/2) d (F_a + F_b) . n
    // moves into the two endpoint vertices' coefficients (both are in the row's two-level set),
    // every coefficient is split into a (hi, lo) float pair, and each row's vertex coefficients
    // are summed (the exact centre-vertex term)
    std::vector<float> cvdf(2 * cv.size()), cedf(2 * ce.size());
    std::vector<double> sig((size_t)6 * A), fold;
    auto put = [](float* dst, double x) {
      const float hi = (float)x;
      dst[0] = hi;
      dst[1] = (float)(x - (double)hi);
    };
    for (int ri = 0; ri < A; ++ri) {
      const int N = vptr[ri + 1] - vptr[ri], M = eptr[ri + 1] - eptr[ri];
      const T* cvb = &cv[(size_t)6 * vptr[ri]];
      const T* ceb = &ce[(size_t)3 * eptr[ri]];
      fold.assign(cvb, cvb + (size_t)6 * N);
      for (int j = 0; j < M; ++j) {
        const int e = eidx[eptr[ri] + j];
        const double nx = (double)nrm[e], ny = (double)nrm[(size_t)Ef + e];
        for (int end = 2; end <= 3; ++end) {
          const int v = sten[(size_t)end * Ef + e];
          int pos = -1;
          for (int k = 0; k < N; ++k)
            if (vidx[vptr[ri] + k] == v) { pos = k; break; }
          if (pos < 0) {
            set_error("divergence row %d: an end vertex of its edge %d is not in its vertex set", ri, e);
            return HFD_ERR_MESH;
          }
          for (int row = 0; row < 3; ++row) {
            const double d = (double)ceb[(size_t)row * M + j];
            fold[(size_t)(2 * row) * N + pos] += 0.5 * d * nx;
            fold[(size_t)(2 * row + 1) * N + pos] += 0.5 * d * ny;
          }
        }
      }
      for (int k = 0; k < 6; ++k) {
        double acc = 0.0;
        for (int j = 0; j < N; ++j) acc += fold[(size_t)k * N + j];
        sig[(size_t)6 * ri + k] = acc;
      }
      for (size_t k = 0; k < (size_t)6 * N; ++k) put(&cvdf[2 * ((size_t)6 * vptr[ri] + k)], fold[k]);
      for (size_t k = 0; k < (size_t)3 * M; ++k) put(&cedf[2 * ((size_t)3 * eptr[ri] + k)], (double)ceb[k]);
    }
    TRY(dev_upload(m, &d.cvdf, cvdf));
    TRY(dev_upload(m, &d.cedf, cedf));
    TRY(dev_upload(m, (void**)&d.sig, sig));
    d.div_df = 0;                     // an option (hfd_mesh_set_fp64_div): see hfd.h
  }
  if (std::is_same<T, float>::value) {
    // FP32 bulk: entries in chunks of 4 (hfd::kDivChunk), each chunk's rows contiguous
    chunk_rows(A, vptr, vidx, 6, cv, P.opts.viscous ? &cvis : nullptr);
    chunk_rows(A, eptr, eidx, 3, ce, static_cast<std::vector<T>*>(nullptr));
    // tiles of the staged divergence: runs of at most kStageTileVerts consecutive vertices
    // whose row pointers, index chunks and coefficient chunks fit one stage buffer; per tile
    // {r0, r1, c0, nvc, m0, nec, pb, 0} with pb = r0 rounded down to a multiple of 4 (the
    // 16-byte aligned start of the row-pointer copies)
    std::vector<int32_t> tiles;
    const size_t per_vc = 16 + 96 + (P.opts.viscous ? 96 : 0), per_ec = 16 + 48;
    for (int r0 = 0; r0 < A;) {
      int r1 = r0;
      while (r1 < A && r1 - r0 < hfd::kStageTileVerts &&
             2 * (size_t)hfd::kStagePtrSlot + per_vc * (size_t)(vptr[r1 + 1] - vptr[r0]) +
                     per_ec * (size_t)(eptr[r1 + 1] - eptr[r0]) <=
                 (size_t)hfd::kStageTileBytes)
        ++r1;
      if (r1 == r0) {
        set_error("vertex %d has more divergence entries than one stage buffer holds", r0);
        return HFD_ERR_MESH;
      }
      const int32_t rec[8] = {r0, r1, vptr[r0], vptr[r1] - vptr[r0], eptr[r0], eptr[r1] - eptr[r0],
                              r0 & ~3, 0};
      tiles.insert(tiles.end(), rec, rec + 8);
      r0 = r1;
    }
    d.ntiles = (int)tiles.size() / 8;
    d.div_staged = 0;                 // the unstaged kernel measured faster (see hfd.h)
    TRY(dev_upload(m, (void**)&d.tiles, tiles));
    // the gather-staged divergence (inviscid): per tile of kGsRows rows the sorted distinct
    // vertex and edge ids its chunks read, and every chunk entry as its position in them
    d.gs_ntiles = 0;
    if (!P.opts.viscous && A > 0) {
      const int R = hfd::kGsRows, C = hfd::kDivChunk;
      const int nt = (A + R - 1) / R;
      std::vector<int32_t> tvp(nt + 1, 0), tep(nt + 1, 0), tvl, tel;
      std::vector<uint16_t> lv(vidx.size()), le(eidx.size());
      size_t smem_max = 0;
      bool fits = true;
      auto localise = [](const std::vector<int32_t>& idx, size_t k0, size_t k1,
                         std::vector<int32_t>& list, std::vector<uint16_t>& loc) {
        std::vector<int32_t> u(idx.begin() + k0, idx.begin() + k1);
        std::sort(u.begin(), u.end());
        u.erase(std::unique(u.begin(), u.end()), u.end());
        if (u.size() > 65535) return (size_t)0;
        for (size_t k = k0; k < k1; ++k)
          loc[k] = (uint16_t)(std::lower_bound(u.begin(), u.end(), idx[k]) - u.begin());
        list.insert(list.end(), u.begin(), u.end());
        return u.size();
      };
      for (int t = 0; t < nt && fits; ++t) {
        const int r0 = t * R, r1 = std::min(A, r0 + R);
        const size_t nu = localise(vidx, (size_t)C * vptr[r0], (size_t)C * vptr[r1], tvl, lv);
        const size_t ne = localise(eidx, (size_t)C * eptr[r0], (size_t)C * eptr[r1], tel, le);
        const size_t bytes = 32 * nu + 16 * ne;
        fits = (nu > 0 || vptr[r1] == vptr[r0]) && (ne > 0 || eptr[r1] == eptr[r0]) &&
               bytes <= (size_t)hfd::kGsSmemMax;
        smem_max = std::max(smem_max, bytes);
        tvp[t + 1] = (int32_t)tvl.size();
        tep[t + 1] = (int32_t)tel.size();
      }
      if (fits) {
        TRY(dev_upload(m, (void**)&d.gtv_ptr, tvp));
        TRY(dev_upload(m, (void**)&d.gte_ptr, tep));
        TRY(dev_upload(m, (void**)&d.gtv, tvl));
        TRY(dev_upload(m, (void**)&d.gte, tel));
        TRY(dev_upload(m, (void**)&d.lvidx, lv));
        TRY(dev_upload(m, (void**)&d.leidx, le));
        d.gs_ntiles = nt;
        d.gs_smem = (int)std::max<size_t>(smem_max, 16);
        CK(hfd::prepare_div_gs(d.gs_smem));
      }
    }
    // the row-pointer copies read whole int4s up to 3 entries past vptr[A] / eptr[A]
    vptr.resize((size_t)A + 5, vptr[A]);
    eptr.resize((size_t)A + 5, eptr[A]);
    // every range the staged kernel reads, checked here once: copy extents inside the arrays,
    // the row-pointer slots and the tile inside one stage buffer
    for (int t = 0; t < d.ntiles; ++t) {
      const int32_t* rc = &tiles[(size_t)8 * t];
      const int r0 = rc[0], r1 = rc[1], pb = rc[6];
      const int nseg = (r1 + 1 - pb + 3) & ~3;
      const size_t bytes = 2 * (size_t)hfd::kStagePtrSlot + per_vc * rc[3] + per_ec * rc[5];
      const bool ok = r0 < r1 && r1 - r0 <= hfd::kStageTileVerts && pb % 4 == 0 && pb <= r0 &&
                      4 * nseg <= hfd::kStagePtrSlot && (size_t)(pb + nseg) <= vptr.size() &&
                      (size_t)rc[2] + rc[3] <= (size_t)vptr[A] && (size_t)rc[4] + rc[5] <= (size_t)eptr[A] &&
                      bytes <= (size_t)hfd::kStageTileBytes && (t == 0 || tiles[(size_t)8 * t - 7] == r0);
      if (!ok) {
        set_error("staged divergence tile %d fails its bounds (vertices %d..%d)", t, r0, r1);
        return HFD_ERR_MESH;
      }
    }
  }
  TRY(dev_upload(m, (void**)&d.vptr, vptr));
  TRY(dev_upload(m, (void**)&d.eptr, eptr));
  TRY(dev_upload(m, (void**)&d.vidx, vidx));
  TRY(dev_upload(m, (void**)&d.eidx, eidx));
  TRY(dev_upload(m, &d.cv, cv));
  TRY(dev_upload(m, &d.ce, ce));
  if (P.opts.viscous) TRY(dev_upload(m, &d.cvis, cvis));
  const size_t V = d.V;
  TRY(dev_alloc(m, &d.Ua, V * 12 * sizeof(T)));
  TRY(dev_alloc(m, &d.FG, V * 8 * sizeof(T)));
  if (P.opts.viscous) TRY(dev_alloc(m, &d.FGv, V * 8 * sizeof(T)));
  TRY(dev_alloc(m, &d.h, (size_t)Ef * 4 * sizeof(T)));
  if (std::is_same<T, float>::value) TRY(dev_alloc(m, (void**)&d.wref, 4 * sizeof(float)));
  return HFD_OK;
}

hfd_status upload(const hfd::Prep& P, int precision, hfd_mesh* m) {
  CK(cudaGetDevice(&m->device));
  m->opts = P.opts;
  if (precision >= 0) m->opts.precision = precision;
  DevMesh& d = m->dm;
  const int V = P.nv;
  const int A = (int)P.active.size();
  d.V = V;
  d.A = A;
  d.G = (int)P.ghost_ids.size();
  d.Ef = (int)P.flux_edges.size();
  d.precision = m->opts.precision;
  d.viscous = P.opts.viscous;
  // ---- vertex order: non-ghosts first, then by member mesh (batches), each part along a
  // Hilbert curve of the member's own bounding box
  m->perm.resize(V);
  {
    std::vector<double> box;
    if (P.nmember > 1) {
      box = P.member_box;
    } else {
      double x0 = 0, x1 = P.Lx, y0 = 0, y1 = P.Ly;
      if (!P.periodic_x || !(x1 > 0)) {
        x0 = *std::min_element(P.x.begin(), P.x.end());
        x1 = *std::max_element(P.x.begin(), P.x.end());
      }
      if (!P.periodic_y || !(y1 > 0)) {
        y0 = *std::min_element(P.y.begin(), P.y.end());
        y1 = *std::max_element(P.y.begin(), P.y.end());
      }
      box = {x0, x1, y0, y1};
    }
    std::vector<uint64_t> key(V);
    for (int v = 0; v < V; ++v) {
      int mb = P.nmember > 1 ? P.member[v] : 0;
      double x0 = box[4 * mb], x1 = box[4 * mb + 1], y0 = box[4 * mb + 2], y1 = box[4 * mb + 3];
      double sx = x1 > x0 ? 65535.0 / (x1 - x0) : 0, sy = y1 > y0 ? 65535.0 / (y1 - y0) : 0;
      double xn = (P.x[v] - x0) * sx, yn = (P.y[v] - y0) * sy;
      uint32_t xi = (uint32_t)std::min(65535.0, std::max(0.0, xn));
      uint32_t yi = (uint32_t)std::min(65535.0, std::max(0.0, yn));
      key[v] = P.opts.renumber ? hilbert(xi, yi) : 0;
    }
    std::iota(m->perm.begin(), m->perm.end(), 0);
    auto mem = [&](int v) { return P.nmember > 1 ? P.member[v] : 0; };
    std::stable_sort(m->perm.begin(), m->perm.end(), [&](int a, int b) {
      if (P.is_ghost[a] != P.is_ghost[b]) return P.is_ghost[a] < P.is_ghost[b];
      if (mem(a) != mem(b)) return mem(a) < mem(b);
      if (key[a] != key[b]) return key[a] < key[b];
      return a < b;
    });
  }
  std::vector<int32_t> inv(V);
  for (int i = 0; i < V; ++i) inv[m->perm[i]] = i;
  // ---- flux edge order: by internal (min, max) end ids
  const int Ef = d.Ef;
  std::vector<int32_t> fperm(Ef);
  std::iota(fperm.begin(), fperm.end(), 0);
  auto ekey = [&](int f) {
    int e = P.flux_edges[f];
    int a = inv[P.edges[2 * (size_t)e]], b = inv[P.edges[2 * (size_t)e + 1]];
    return std::make_pair(std::min(a, b), std::max(a, b));
  };
  std::sort(fperm.begin(), fperm.end(), [&](int a, int b) { return ekey(a) < ekey(b); });
  std::vector<int32_t> fint(Ef), emap(P.nedges(), -1);
  for (int i = 0; i < Ef; ++i) {
    fint[fperm[i]] = i;
    emap[P.flux_edges[fperm[i]]] = i;
  }
  m->fperm = fperm;
  hfd_status st = d.precision == 0 ? upload_streams<double>(m, P, inv, fint, fperm, emap)
                                   : upload_streams<float>(m, P, inv, fint, fperm, emap);
  if (st != HFD_OK) return st;
  // ---- ghosts, time-step data, perm, stage buffers, scalars
  std::vector<int32_t> gid(d.G), gdn(d.G), gfl(d.G);
  for (int g = 0; g < d.G; ++g) {
    gid[g] = inv[P.ghost_ids[g]];
    gdn[g] = P.ghost_donor[g] < 0 ? -1 : inv[P.ghost_donor[g]];   // -1: fixed ghost
    gfl[g] = P.ghost_flags[g];
  }
  TRY(dev_upload(m, (void**)&d.gid, gid));
  TRY(dev_upload(m, (void**)&d.gdonor, gdn));
  TRY(dev_upload(m, (void**)&d.gflags, gfl));
  std::vector<double> lmin(A);
  for (int i = 0; i < A; ++i) lmin[i] = P.lmin[m->perm[i]];
  TRY(dev_upload(m, (void**)&d.lmin, lmin));
  TRY(dev_upload(m, (void**)&m->dperm, m->perm));
  d.nmember = P.nmember;
  TRY(dev_alloc(m, (void**)&d.dtbits, sizeof(unsigned long long) * d.nmember));
  TRY(dev_alloc(m, (void**)&d.dt_last, sizeof(double) * d.nmember));
  TRY(dev_alloc(m, (void**)&d.dtpartial, sizeof(double) * ((size_t)A / 256 + 1)));
  TRY(dev_alloc(m, (void**)&d.err, sizeof(unsigned)));
  TRY(dev_alloc(m, (void**)&d.bar, 2 * sizeof(unsigned)));
  if (d.nmember > 1) {
    std::vector<int32_t> vm(A);
    for (int i = 0; i < A; ++i) vm[i] = P.member[m->perm[i]];
    TRY(dev_upload(m, (void**)&d.vmem, vm));
  }
  TRY(dev_alloc(m, (void**)&m->U1, (size_t)12 * V * sizeof(double)));
  TRY(dev_alloc(m, (void**)&m->U2, (size_t)12 * V * sizeof(double)));
  CK(cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking));
  // lanes per vertex in the divergence: FP64 is bound by the FP64 pipe and runs best without a
  // cross-lane reduction (1); the FP32 path is bound by memory and prefers coalesced groups (4)
  m->lanes = m->opts.precision == 0 ? 1 : 4;
  if (const char* env = getenv("HFD_DIV_LANES")) {   // tuning override: 1, 2, 4 or 8
    int l = atoi(env);
    if (l == 1 || l == 2 || l == 4 || l == 8) m->lanes = l;
  }
  const hfd_options& o = P.opts;
  m->ph.gamma = o.gamma;
  m->ph.eps = o.weno_eps;
  m->ph.sens_lo = o.sens_lo;
  m->ph.sens_hi = o.sens_hi;
  m->ph.harten = o.harten;
  m->ph.cfl = o.cfl;
  m->ph.mu = o.mu;
  m->ph.R_gas = o.R_gas;
  m->ph.kappa = o.mu * (o.gamma * o.R_gas / (o.gamma - 1.0)) / o.prandtl;
  m->ph.flux = o.flux;
  m->ph.force_branch = o.force_branch;
  m->ph.finish();
  // ---- stats
  hfd_mesh_stats& s = m->stats;
  s.nv = V;
  s.nactive = A;
  s.nedges = P.nedges();
  s.nflux_edges = Ef;
  s.div_nv_total = P.div_vptr.empty() ? 0 : P.div_vptr.back();
  s.div_ne_total = P.div_eptr.empty() ? 0 : P.div_eptr.back();
  for (int r = 0; r < A; ++r) {
    s.div_nv_max = std::max(s.div_nv_max, P.div_vptr[r + 1] - P.div_vptr[r]);
    s.div_ne_max = std::max(s.div_ne_max, P.div_eptr[r + 1] - P.div_eptr[r]);
  }
  for (int32_t r : P.rank) s.rank_hist[std::min(15, std::max(0, r))]++;
  s.div_degree_fallbacks = P.degree_fallbacks;
  s.visc_degree_fallbacks = P.visc_fallbacks;
  s.nmember = P.nmember;
  s.prep_seconds = P.prep_seconds;
  return HFD_OK;
}

hfd_status residual_impl(hfd_mesh* m, double* U, double* R, cudaStream_t s) {
  CK(hfd::launch_ghost(m->dm, U, U, s));
  CK(hfd::launch_vertex(m->dm, U, m->ph, s));
  CK(hfd::launch_edge(m->dm, m->ph, s));
  CK(hfd::launch_div(m->dm, U, U, R, hfd::DIV_RESIDUAL, 0.0, 1.0, 1.0, m->ph, m->lanes, s));
  const DevMesh& d = m->dm;
  if (d.V > d.A)
    CK(cudaMemset2DAsync(R + d.A, (size_t)d.V * sizeof(double), 0,
                         (size_t)(d.V - d.A) * sizeof(double), 12, s));
  return HFD_OK;
}

// Optional per-kernel timing of the launches of a step (hfd_steps_profiled).
struct Timer {
  cudaStream_t s;
  double ms[6] = {0, 0, 0, 0, 0, 0};
  int64_t launches = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
};

// One SSP-RK3 step: three stages of (ghost refresh, vertex fluxes, edge fluxes, divergence +
// stage combination), plus the device time step and a final ghost refresh.
// One SSP-RK3 step of U.  dt > 0: that step; else dt_member (device array, one step per batch
// member) when given; else each member's CFL step.
hfd_status step_impl(hfd_mesh* m, double* U, double dt, cudaStream_t s, Timer* tm = nullptr,
                     const double* dt_member = nullptr) {
  const DevMesh& d = m->dm;
  auto timed = [&](int kind, auto&& launch) -> cudaError_t {
    cudaEvent_t a = nullptr, b = nullptr;
    if (tm) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, s);
    }
    cudaError_t e = launch();
    if (tm) {
      cudaEventRecord(b, s);
      tm->ev.push_back({kind, {a, b}});
      tm->launches += kind == 4 ? 2 : 1;   // the CFL minimum is two kernels (two-pass reduction)
    }
    return e;
  };
  if (!(dt > 0.0) && !dt_member) CK(timed(4, [&] { return hfd::launch_dtmin(d, U, m->ph, s); }));
  static const double A_[3] = {0.0, 0.75, 1.0 / 3.0}, B_[3] = {1.0, 0.25, 2.0 / 3.0};
  double* in[3] = {U, m->U1, m->U2};
  double* out[3] = {m->U1, m->U2, U};
  static const char* const kStage[3] = {"hfd stage 1", "hfd stage 2", "hfd stage 3"};
  for (int k = 0; k < 3; ++k) {
    hfd::NvtxRange range(kStage[k]);
    if (m->persistent) {
      int grid = m->grid;
      if (grid <= 0) {
        int per_sm = 0, nsm = 0;
        CK(hfd::persistent_max_blocks(d, m->lanes, &per_sm, &nsm));
        grid = std::max(1, per_sm) * nsm;
      }
      CK(cudaMemsetAsync(d.bar, 0, 2 * sizeof(unsigned), s));
      CK(timed(5, [&] {
        return hfd::launch_stage_persistent(d, in[k], U, out[k], hfd::DIV_STAGE, A_[k], B_[k], dt,
                                            m->ph, m->lanes, grid, true, s, dt_member);
      }));
      continue;
    }
    if (d.G) CK(timed(0, [&] { return hfd::launch_ghost(d, in[k], U, s); }));
    CK(timed(1, [&] { return hfd::launch_vertex(d, in[k], m->ph, s); }));
    CK(timed(2, [&] { return hfd::launch_edge(d, m->ph, s); }));
    CK(timed(3, [&] {
      return hfd::launch_div(d, in[k], U, out[k], hfd::DIV_STAGE, A_[k], B_[k], dt, m->ph,
                             m->lanes, s, dt_member);
    }));
  }
  if (d.G) CK(timed(0, [&] { return hfd::launch_ghost(d, U, U, s); }));
  return HFD_OK;
}

void drop_graphs(hfd_mesh* m) {
  for (auto& kv : m->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  m->graphs.clear();
}

}  // namespace

extern "C" {

hfd_status hfd_mesh_upload(const hfd_prep* prep, int32_t precision, hfd_mesh** out) {
  if (!prep || !out || precision < -1 || precision > 1) {
    set_error("hfd_mesh_upload: invalid argument");
    return HFD_ERR_ARG;
  }
  *out = nullptr;
  hfd::NvtxRange range("hfd_mesh_upload");
  hfd_mesh* m = new (std::nothrow) hfd_mesh();
  if (!m) { set_error("hfd_mesh_upload: out of host memory"); return HFD_ERR_ARG; }
  hfd_status st;
  try {
    st = upload(*prep, precision, m);
  } catch (const std::exception& e) {
    set_error("hfd_mesh_upload: %s", e.what());
    st = HFD_ERR_ARG;
  }
  if (st != HFD_OK) { hfd_mesh_destroy(m); return st; }
  *out = m;
  return HFD_OK;
}

hfd_status hfd_mesh_create(const hfd_mesh_desc* desc, const hfd_options* opts, hfd_mesh** out) {
  hfd_prep* p = nullptr;
  hfd_status st = hfd_prep_create(desc, opts, &p);
  if (st != HFD_OK) return st;
  st = hfd_mesh_upload(p, -1, out);
  hfd_prep_destroy(p);
  return st;
}

void hfd_mesh_destroy(hfd_mesh* m) {
  if (!m) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(m->device);
  drop_graphs(m);
  if (m->cap) cudaStreamDestroy(m->cap);
  mesh_free_all(m);
  cudaSetDevice(prev);
  delete m;
}

hfd_status hfd_mesh_info(const hfd_mesh* m, hfd_mesh_stats* out) {
  if (!m || !out) { set_error("hfd_mesh_info: null argument"); return HFD_ERR_ARG; }
  *out = m->stats;
  return HFD_OK;
}

hfd_status hfd_mesh_perm(const hfd_mesh* m, int32_t* perm) {
  if (!m || !perm) { set_error("hfd_mesh_perm: null argument"); return HFD_ERR_ARG; }
  std::memcpy(perm, m->perm.data(), m->perm.size() * sizeof(int32_t));
  return HFD_OK;
}

hfd_status hfd_state_import(hfd_mesh* m, const double* Uin, double* Uint, void* stream) {
  if (!m || !Uin || !Uint) { set_error("hfd_state_import: null argument"); return HFD_ERR_ARG; }
  CK(hfd::launch_permute(m->dm.V, m->dperm, Uin, Uint, true, (cudaStream_t)stream));
  return HFD_OK;
}

hfd_status hfd_state_export(hfd_mesh* m, const double* Uint, double* Uin, void* stream) {
  if (!m || !Uin || !Uint) { set_error("hfd_state_export: null argument"); return HFD_ERR_ARG; }
  CK(hfd::launch_permute(m->dm.V, m->dperm, Uint, Uin, false, (cudaStream_t)stream));
  return HFD_OK;
}

hfd_status hfd_residual(hfd_mesh* m, double* U, double* R, void* stream) {
  if (!m || !U || !R || U == R) { set_error("hfd_residual: invalid argument"); return HFD_ERR_ARG; }
  hfd::NvtxRange range("hfd_residual");
  return residual_impl(m, U, R, (cudaStream_t)stream);
}

hfd_status hfd_step(hfd_mesh* m, double* U, double dt, void* stream) {
  if (!m || !U) { set_error("hfd_step: invalid argument"); return HFD_ERR_ARG; }
  hfd::NvtxRange range("hfd_step");
  return step_impl(m, U, dt, (cudaStream_t)stream);
}

hfd_status hfd_steps(hfd_mesh* m, double* U, double dt, int32_t nsteps, void* stream) {
  if (!m || !U || nsteps < 0) { set_error("hfd_steps: invalid argument"); return HFD_ERR_ARG; }
  if (nsteps == 0) return HFD_OK;
  hfd::NvtxRange range("hfd_steps");
  auto key = std::make_pair((const double*)U, dt > 0.0 ? dt : 0.0);
  GraphEntry& g = m->graphs[key];
  if (!g.exec) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal));
    hfd_status st = step_impl(m, U, dt, m->cap);
    cudaError_t ce = cudaStreamEndCapture(m->cap, &graph);
    if (st != HFD_OK) {
      if (graph) cudaGraphDestroy(graph);
      m->graphs.erase(key);
      return st;
    }
    if (ce != cudaSuccess) {
      m->graphs.erase(key);
      set_error("hfd_steps: capture failed: %s", cudaGetErrorString(ce));
      return HFD_ERR_CUDA;
    }
    ce = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      m->graphs.erase(key);
      set_error("hfd_steps: instantiate failed: %s", cudaGetErrorString(ce));
      return HFD_ERR_CUDA;
    }
  }
  for (int i = 0; i < nsteps; ++i) CK(cudaGraphLaunch(g.exec, (cudaStream_t)stream));
  return HFD_OK;
}

hfd_status hfd_steps_profiled(hfd_mesh* m, double* U, double dt, int32_t nsteps, void* stream,
                              double* kernel_ms, int64_t* launches) {
  if (!m || !U || nsteps < 0 || !kernel_ms) {
    set_error("hfd_steps_profiled: invalid argument");
    return HFD_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Timer tm;
  tm.s = s;
  hfd_status st = HFD_OK;
  for (int i = 0; i < nsteps && st == HFD_OK; ++i) st = step_impl(m, U, dt, s, &tm);
  cudaError_t e = cudaStreamSynchronize(s);
  for (auto& x : tm.ev) {
    float ms = 0;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, x.second.first, x.second.second);
    kernel_ms[x.first] += ms;
    cudaEventDestroy(x.second.first);
    cudaEventDestroy(x.second.second);
  }
  if (launches) *launches = tm.launches;
  if (st != HFD_OK) return st;
  CK(e);
  return HFD_OK;
}

hfd_status hfd_steps_host(hfd_mesh* m, const double* U_in, double* U_out, double dt,
                          int32_t nsteps, void* stream) {
  if (!m || !U_in || !U_out || nsteps < 0) {
    set_error("hfd_steps_host: invalid argument");
    return HFD_ERR_ARG;
  }
  hfd::NvtxRange range("hfd_steps_host");
  size_t bytes = (size_t)12 * m->dm.V * sizeof(double);
  if (!m->Uin) {
    TRY(dev_alloc(m, (void**)&m->Uin, bytes));
    TRY(dev_alloc(m, (void**)&m->Uint, bytes));
  }
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(m->Uin, U_in, bytes, cudaMemcpyHostToDevice, s));
  CK(hfd::launch_permute(m->dm.V, m->dperm, m->Uin, m->Uint, true, s));
  TRY(hfd_steps(m, m->Uint, dt, nsteps, stream));
  CK(hfd::launch_permute(m->dm.V, m->dperm, m->Uint, m->Uin, false, s));
  CK(cudaMemcpyAsync(U_out, m->Uin, bytes, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return HFD_OK;
}

hfd_status hfd_mesh_set_launch(hfd_mesh* m, int32_t persistent, int32_t grid) {
  if (!m || persistent < 0 || persistent > 1 || grid < 0) {
    set_error("hfd_mesh_set_launch: invalid argument");
    return HFD_ERR_ARG;
  }
  if (persistent) {
    int per_sm = 0, nsm = 0;
    CK(hfd::persistent_max_blocks(m->dm, m->lanes, &per_sm, &nsm));
    if (per_sm < 1 || grid > per_sm * nsm) {
      set_error("hfd_mesh_set_launch: %d blocks exceed the %d co-resident blocks", grid, per_sm * nsm);
      return HFD_ERR_ARG;
    }
  }
  m->persistent = persistent;
  m->grid = grid;
  drop_graphs(m);
  return HFD_OK;
}

hfd_status hfd_mesh_set_lanes(hfd_mesh* m, int32_t lanes) {
  if (!m || !(lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8)) {
    set_error("hfd_mesh_set_lanes: lanes must be 1, 2, 4 or 8");
    return HFD_ERR_ARG;
  }
  if (m->persistent && m->grid > 0) {
    int per_sm = 0, nsm = 0;
    CK(hfd::persistent_max_blocks(m->dm, lanes, &per_sm, &nsm));
    if (m->grid > per_sm * nsm) {
      set_error("hfd_mesh_set_lanes: the persistent grid of %d blocks exceeds the %d co-resident "
                "blocks at %d lanes", m->grid, per_sm * nsm, lanes);
      return HFD_ERR_ARG;
    }
  }
  m->lanes = lanes;
  drop_graphs(m);
  return HFD_OK;
}

hfd_status hfd_mesh_set_div_staged(hfd_mesh* m, int32_t staged) {
  if (!m || staged < 0 || staged > 2) {
    set_error("hfd_mesh_set_div_staged: staged must be 0, 1 or 2");
    return HFD_ERR_ARG;
  }
  if (staged == 1 && m->dm.ntiles == 0 && m->dm.A > 0) {
    set_error("hfd_mesh_set_div_staged: the staged divergence exists for FP32-bulk meshes only");
    return HFD_ERR_UNSUPPORTED;
  }
  if (staged == 2 && m->dm.gs_ntiles == 0 && m->dm.A > 0) {
    set_error("hfd_mesh_set_div_staged: the gather-staged divergence exists for inviscid "
              "FP32-bulk meshes only");
    return HFD_ERR_UNSUPPORTED;
  }
  m->dm.div_staged = staged;
  drop_graphs(m);
  return HFD_OK;
}

hfd_status hfd_edge_branches(hfd_mesh* m, double* U, uint8_t* branches, void* stream) {
  if (!m || !U || !branches) {
    set_error("hfd_edge_branches: invalid argument");
    return HFD_ERR_ARG;
  }
  hfd::NvtxRange range("hfd_edge_branches");
  DevMesh d = m->dm;
  const int Ef = d.Ef;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<uint8_t> host((size_t)Ef);
  if (Ef > 0) {
    CK(mesh_malloc(m, (void**)&d.dbg_branch, (size_t)Ef));
    cudaError_t e = hfd::launch_ghost(d, U, U, s);
    if (e == cudaSuccess) e = hfd::launch_vertex(d, U, m->ph, s);
    if (e == cudaSuccess) e = hfd::launch_edge(d, m->ph, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host.data(), d.dbg_branch, (size_t)Ef, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    // the block is one of the mesh's (released with it); drop it from the list now
    if (m->opts.dev_alloc) m->opts.dev_free(d.dbg_branch, m->opts.alloc_ctx); else cudaFree(d.dbg_branch);
    m->allocs.pop_back();
    if (e != cudaSuccess) {
      set_error("hfd_edge_branches: %s", cudaGetErrorString(e));
      return HFD_ERR_CUDA;
    }
  }
  for (int fi = 0; fi < Ef; ++fi) branches[m->fperm[fi]] = host[fi];
  return HFD_OK;
}

hfd_status hfd_check_conversions(int64_t n, const double* x, float* f_int, float* f_hw,
                                 double* d_int, double* d_hw, void* stream) {
  if (n < 0 || (n > 0 && (!x || !f_int || !f_hw || !d_int || !d_hw))) {
    set_error("hfd_check_conversions: invalid argument");
    return HFD_ERR_ARG;
  }
  cudaError_t e = hfd::launch_conversions(n, x, f_int, f_hw, d_int, d_hw, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_error("hfd_check_conversions: %s", cudaGetErrorString(e));
    return HFD_ERR_CUDA;
  }
  return HFD_OK;
}

hfd_status hfd_mesh_set_fp64_div(hfd_mesh* m, int32_t folded) {
  if (!m || (folded != 0 && folded != 1)) {
    set_error("hfd_mesh_set_fp64_div: folded must be 0 or 1");
    return HFD_ERR_ARG;
  }
  if (folded && !m->dm.cvdf && m->dm.A > 0) {
    set_error("hfd_mesh_set_fp64_div: the folded double-float divergence exists for FP64 meshes only");
    return HFD_ERR_UNSUPPORTED;
  }
  m->dm.div_df = folded;
  drop_graphs(m);
  return HFD_OK;
}

hfd_status hfd_mesh_set_barrier_limit(hfd_mesh* m, uint32_t polls) {
  if (!m) { set_error("hfd_mesh_set_barrier_limit: null mesh"); return HFD_ERR_ARG; }
  m->dm.barrier_spins = polls;
  drop_graphs(m);
  return HFD_OK;
}

hfd_status hfd_mesh_autotune(hfd_mesh* m, const double* U, void* stream, int32_t* choice) {
  if (!m || !U) { set_error("hfd_mesh_autotune: invalid argument"); return HFD_ERR_ARG; }
  hfd::NvtxRange range("hfd_mesh_autotune");
  cudaStream_t s = (cudaStream_t)stream;
  const DevMesh& d = m->dm;
  size_t bytes = (size_t)12 * d.V * sizeof(double);
  CK(cudaMemcpyAsync(m->U1, U, bytes, cudaMemcpyDeviceToDevice, s));
  // candidates: lanes per vertex in the divergence x (four-launch form, persistent form at
  // every co-resident block count for those lanes)
  struct Cand { int persistent, grid, lanes, staged; };
  std::vector<Cand> cands;
  if (d.ntiles > 0) cands.push_back({0, 0, 8, 1});    // FP32 bulk: the staged divergence
  if (d.gs_ntiles > 0) cands.push_back({0, 0, 4, 2}); // FP32 bulk, inviscid: staged gathers
  for (int lanes : {1, 2, 4, 8}) {
    int per_sm = 0, nsm = 0;
    CK(hfd::persistent_max_blocks(d, lanes, &per_sm, &nsm));
    cands.push_back({0, 0, lanes, 0});
    if (lanes == 8) continue;                  // the persistent kernel runs 8 lanes as 4
    for (int b = 1; b <= per_sm; ++b) cands.push_back({1, b * nsm, lanes, 0});
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  Cand pick = cands[0];
  DevMesh dd = d;                              // the trial's divergence kernel choice
  const double dt = 1e-12;   // any fixed step: the work does not depend on it
  for (const Cand& c : cands) {
    float tot = 0;
    for (int rep = 0; rep < 4; ++rep) {
      CK(cudaEventRecord(e0, s));
      if (c.persistent) {
        CK(cudaMemsetAsync(d.bar, 0, 2 * sizeof(unsigned), s));
        CK(hfd::launch_stage_persistent(d, m->U1, m->U1, m->U2, hfd::DIV_STAGE, 0.0, 1.0, dt,
                                        m->ph, c.lanes, c.grid, true, s));
      } else {
        dd.div_staged = c.staged;
        if (d.G) CK(hfd::launch_ghost(d, m->U1, m->U1, s));
        CK(hfd::launch_vertex(d, m->U1, m->ph, s));
        CK(hfd::launch_edge(d, m->ph, s));
        CK(hfd::launch_div(dd, m->U1, m->U1, m->U2, hfd::DIV_STAGE, 0.0, 1.0, dt, m->ph, c.lanes, s));
      }
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) tot += ms;                  // the first repetition warms up
    }
    if (tot < best) { best = tot; pick = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  unsigned w = 0;                              // the trial stages must not leave an error
  CK(cudaMemcpy(&w, d.err, sizeof w, cudaMemcpyDeviceToHost));
  if (w & 4u) { set_error("hfd_mesh_autotune: a persistent trial timed out at a barrier"); return HFD_ERR_TIMEOUT; }
  CK(cudaMemsetAsync(d.err, 0, sizeof(unsigned), s));
  m->persistent = pick.persistent;
  m->grid = pick.grid;
  m->lanes = pick.lanes;
  m->dm.div_staged = pick.staged;
  drop_graphs(m);
  if (choice) {
    choice[0] = pick.persistent; choice[1] = pick.grid; choice[2] = pick.lanes; choice[3] = pick.staged;
  }
  return HFD_OK;
}

hfd_status hfd_last_dt(hfd_mesh* m, double* dt, void* stream) {
  if (!m || !dt) { set_error("hfd_last_dt: null argument"); return HFD_ERR_ARG; }
  CK(cudaMemcpyAsync(dt, m->dm.dt_last, sizeof(double) * m->dm.nmember, cudaMemcpyDeviceToHost,
                     (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return HFD_OK;
}

hfd_status hfd_check(hfd_mesh* m, void* stream) {
  if (!m) { set_error("hfd_check: null argument"); return HFD_ERR_ARG; }
  unsigned w = 0;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(&w, m->dm.err, sizeof w, cudaMemcpyDeviceToHost, s));
  CK(cudaMemsetAsync(m->dm.err, 0, sizeof(unsigned), s));
  CK(cudaStreamSynchronize(s));
  if (w & 8u) {
    set_error("device error word: a gathered index out of range (bounds-checked build)");
    return HFD_ERR_MESH;
  }
  if (w & 1u) { set_error("device error word: non-finite value"); return HFD_ERR_NONFINITE; }
  if (w & 4u) { set_error("device error word: a grid barrier wait timed out"); return HFD_ERR_TIMEOUT; }
  if (w & 2u) { set_error("device error word: rho <= 0 after a stage"); return HFD_ERR_POSITIVITY; }
  return HFD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batches with one array per member
struct hfd_batch {
  hfd_mesh* mesh = nullptr;
  int n = 0;
  std::vector<int64_t> off;          // members' first vertex in the batch's input order
  int64_t* d_off = nullptr;
  double** d_ptrs = nullptr;         // the members' arrays of the current call
  double* d_dt = nullptr;            // the members' steps of the current call
  double* Ubat = nullptr;            // 12 x V, input order
  double* Uint = nullptr;            // 12 x V, internal order
};

extern "C" hfd_status hfd_batch_create(const hfd_prep* const* preps, int32_t n, int32_t precision,
                                       hfd_batch** out) {
  if (!preps || n <= 0 || !out) { set_error("hfd_batch_create: invalid argument"); return HFD_ERR_ARG; }
  *out = nullptr;
  hfd_prep* cat = nullptr;
  hfd_status st = hfd_prep_concat(preps, n, &cat);
  if (st != HFD_OK) return st;
  hfd_batch* b = new (std::nothrow) hfd_batch();
  if (!b) { hfd_prep_destroy(cat); set_error("hfd_batch_create: out of host memory"); return HFD_ERR_ARG; }
  st = hfd_mesh_upload(cat, precision, &b->mesh);
  hfd_prep_destroy(cat);
  if (st != HFD_OK) { delete b; return st; }
  b->n = n;
  b->off.assign(n + 1, 0);
  for (int k = 0; k < n; ++k) b->off[k + 1] = b->off[k] + preps[k]->nv;
  hfd_mesh* m = b->mesh;
  const size_t bytes = (size_t)12 * m->dm.V * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = mesh_malloc(m, (void**)&b->d_off, sizeof(int64_t) * (n + 1));
  if (e == cudaSuccess) e = mesh_malloc(m, (void**)&b->d_ptrs, sizeof(double*) * n);
  if (e == cudaSuccess) e = mesh_malloc(m, (void**)&b->d_dt, sizeof(double) * n);
  if (e == cudaSuccess) e = mesh_malloc(m, (void**)&b->Ubat, bytes);
  if (e == cudaSuccess) e = mesh_malloc(m, (void**)&b->Uint, bytes);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_off, b->off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error("hfd_batch_create: %s", cudaGetErrorString(e));
    hfd_batch_destroy(b);
    return HFD_ERR_CUDA;
  }
  *out = b;
  return HFD_OK;
}

extern "C" void hfd_batch_destroy(hfd_batch* b) {
  if (!b) return;
  hfd_mesh_destroy(b->mesh);        // also releases the batch's blocks (mesh allocations)
  delete b;
}

extern "C" hfd_status hfd_batch_mesh(hfd_batch* b, hfd_mesh** mesh) {
  if (!b || !mesh) { set_error("hfd_batch_mesh: invalid argument"); return HFD_ERR_ARG; }
  *mesh = b->mesh;
  return HFD_OK;
}

extern "C" hfd_status hfd_batch_step(hfd_batch* b, double* const* U, const double* dt,
                                     void* stream) {
  if (!b || !U) { set_error("hfd_batch_step: invalid argument"); return HFD_ERR_ARG; }
  hfd::NvtxRange range("hfd_batch_step");
  for (int k = 0; k < b->n; ++k) {
    if (!U[k]) { set_error("hfd_batch_step: member %d has no state", k); return HFD_ERR_ARG; }
    if (dt && !(dt[k] > 0.0)) {
      set_error("hfd_batch_step: member %d: dt must be positive (or pass no dt array)", k);
      return HFD_ERR_ARG;
    }
  }
  hfd_mesh* m = b->mesh;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(b->d_ptrs, U, sizeof(double*) * b->n, cudaMemcpyHostToDevice, s));
  if (dt) CK(cudaMemcpyAsync(b->d_dt, dt, sizeof(double) * b->n, cudaMemcpyHostToDevice, s));
  const int V = m->dm.V;
  CK(hfd::launch_batch_copy(V, b->n, b->d_off, b->d_ptrs, b->Ubat, true, s));
  CK(hfd::launch_permute(V, m->dperm, b->Ubat, b->Uint, true, s));
  TRY(step_impl(m, b->Uint, 0.0, s, nullptr, dt ? b->d_dt : nullptr));
  CK(hfd::launch_permute(V, m->dperm, b->Uint, b->Ubat, false, s));
  CK(hfd::launch_batch_copy(V, b->n, b->d_off, b->d_ptrs, b->Ubat, false, s));
  // the host arrays U and dt may be reused by the caller as soon as this returns
  CK(cudaStreamSynchronize(s));
  return HFD_OK;
}

