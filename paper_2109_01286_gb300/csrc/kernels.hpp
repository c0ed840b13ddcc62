// Device mesh layout and kernel launchers (kernels.cu), used by the C ABI (api.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hfd {

// Physical and numerical constants passed by value to the kernels.
struct Phys {
  double gamma, eps, sens_lo, sens_hi, harten, cfl;
  double mu, kappa, R_gas;      // viscous model (Sec. 2.3; constant mu, kappa = mu c_p / Pr)
  int flux;                     // 0 Roe (Harten's fix), 1 Rusanov
  int force_branch;             // 0 sensor, 1 every side 5-node, 2 every side 3-node WENO
  double g1;                    // gamma - 1
  // the same constants rounded once to FP32 on the host (no FP64 conversions in FP32 kernels)
  float g1f, epsf, sens_lof, sens_hif, hartenf;
  double half_inv_harten;       // 1 / (2 harten): the entropy fix's 1/(2 delta) is this over c
  float half_inv_hartenf;
  void finish() {
    g1 = gamma - 1.0;
    half_inv_harten = 0.5 / harten;   // +inf for harten = 0, where the fix never applies
    half_inv_hartenf = (float)half_inv_harten;
    g1f = (float)g1;
    epsf = (float)eps;
    sens_lof = (float)sens_lo;
    sens_hif = (float)sens_hi;
    hartenf = (float)harten;
  }
};

template <typename T> __host__ __device__ inline T phys_g1(const Phys& p);
template <> __host__ __device__ inline double phys_g1<double>(const Phys& p) { return p.g1; }
template <> __host__ __device__ inline float phys_g1<float>(const Phys& p) { return p.g1f; }
template <typename T> __host__ __device__ inline T phys_harten(const Phys& p);
template <> __host__ __device__ inline double phys_harten<double>(const Phys& p) { return p.harten; }
template <> __host__ __device__ inline float phys_harten<float>(const Phys& p) { return p.hartenf; }
template <typename T> __host__ __device__ inline T phys_half_inv_harten(const Phys& p);
template <> __host__ __device__ inline double phys_half_inv_harten<double>(const Phys& p) { return p.half_inv_harten; }
template <> __host__ __device__ inline float phys_half_inv_harten<float>(const Phys& p) { return p.half_inv_hartenf; }

// Divergence entries per chunk of the FP32-bulk layout (vector loads of 4 coefficients).
constexpr int kDivChunk = 4;
// Staged FP32 divergence: vertices per tile, stage buffers per block, bytes of one stage buffer
// (two row-pointer slots of kStagePtrSlot bytes, then per chunk: vertex indices 16 B, vertex
// coefficients 96 B (+96 B viscous), edge indices 16 B, edge coefficients 48 B).
constexpr int kGsLanes = 4, kGsRows = 64;     // gather-staged divergence: lanes, rows per block
constexpr int kGsSmemMax = 160 * 1024;         // a tile needing more is not built (mode 2 refused)
constexpr int kStageTileVerts = 32;
constexpr int kStages = 3;
constexpr int kStageTileBytes = 36 * 1024;
constexpr int kStagePtrSlot = 160;     // 36 row pointers of a tile (pb .. r1, whole int4s) + slack

// Device arrays of one mesh in internal numbering.  Coefficient and flux arrays hold elements
// of the path's bulk precision T (double or float), addressed through void pointers here.
struct DevMesh {
  int V = 0;        // vertices; internal ids [0, A) are non-ghost, [A, V) ghosts
  int A = 0;
  int Ef = 0;       // flux edges
  int G = 0;        // ghost vertices
  int precision = 0;
  int viscous = 0;
  // edge streams: stencil [6][Ef] (internal vertex ids), normal [2][Ef], 5-node weights
  // [30][Ef] (side L 15, side R 15; node*3 + {value, x, y}), 3-node weights [18][Ef]
  int32_t* sten = nullptr;
  void* nrm = nullptr;
  void* w5 = nullptr;
  void* w3 = nullptr;
  // divergence CSR over active vertices; per-vertex SoA coefficient blocks:
  // cv at 6*vptr[r]: d0F, d0G, dxF, dxG, dyF, dyG (each N long); ce at 3*eptr[r]: d0, dx, dy.
  // FP32 bulk instead: vptr/eptr count chunks of kDivChunk entries, the index lists are padded
  // to whole chunks, and each chunk holds its 6 (cv, cvis) or 3 (ce) rows of kDivChunk
  // coefficients contiguously (zero in the padding)
  int32_t *vptr = nullptr, *vidx = nullptr, *eptr = nullptr, *eidx = nullptr;
  void* cv = nullptr;
  void* ce = nullptr;
  void* cvis = nullptr;  // viscous rows, same layout as cv
  // FP32 bulk: tiles of consecutive active vertices for the staged divergence (8 int32 per
  // tile: {r0, r1, c0, nvc, m0, nec, pb, 0}; a tile's chunks fit one stage buffer), and whether
  // launch_div uses that kernel (1) or the unstaged one with the mesh's lane count (0)
  int32_t* tiles = nullptr;
  int ntiles = 0;
  int div_staged = 0;          // 0 unstaged, 1 coefficient streams staged by TMA, 2 gathers staged
  // FP32 bulk, inviscid: the gather-staged divergence (k_div_gs).  Per tile of kGsRows rows the
  // distinct vertices (gtv) and flux edges (gte) its chunks read, and each chunk's indices as
  // 16-bit positions in those lists (lvidx, leidx: 4 per chunk); gs_smem is the largest
  // tile's shared-memory bytes (32 per vertex, 16 per edge); gs_ntiles 0 = not built.
  uint16_t *lvidx = nullptr, *leidx = nullptr;
  int32_t *gtv_ptr = nullptr, *gtv = nullptr, *gte_ptr = nullptr, *gte = nullptr;
  int gs_ntiles = 0, gs_smem = 0;
  // ghosts
  int32_t *gid = nullptr, *gdonor = nullptr, *gflags = nullptr;
  // time step
  double* lmin = nullptr;                 // [A] shortest incident edge
  unsigned long long* dtbits = nullptr;   // [nmember] min over vertices of lmin/(|u|+c), as bits
  double* dtpartial = nullptr;            // [ceil(A/256)] per-block minima of the dt reduction
  double* dt_last = nullptr;              // [nmember] dt used by the last stage
  unsigned* err = nullptr;                // device error word
  unsigned* bar = nullptr;                // grid barrier state of the persistent kernel [2]
  unsigned barrier_spins = 1u << 24;      // poll bound of a grid barrier wait
  int nmember = 1;                        // meshes in a batch (1 for a single mesh)
  int32_t* vmem = nullptr;                // [A] mesh of each active vertex (batches only)
  // scratch: AoS copies of the state [V][12], vertex fluxes [V][8] (+ viscous), edge fluxes [Ef][4]
  void* Ua = nullptr;
  void* FG = nullptr;
  // FP32 bulk: the reference state of the stage's deviations (4 floats, written by k_vertex)
  float* wref = nullptr;
  // FP64 meshes, folded double-float divergence (div_df = 1): the vertex rows with each edge
  // row's endpoint average folded in, as (hi, lo) float pairs in the cv layout (cvdf), the edge
  // rows as float pairs in the ce layout (cedf), and per active vertex the 6 row sums of the
  // folded vertex rows (sig, FP64: d0F d0G dxF dxG dyF dyG); k_edge then writes each edge's
  // flux minus the average of its end vertices' projected fluxes, as float pairs, into h
  int div_df = 0;
  void* cvdf = nullptr;
  void* cedf = nullptr;
  double* sig = nullptr;
  // testing aid: when set, k_edge writes per flux edge the Alg. 1 branch it took (bit side*4+q
  // set: the WENO-weighted 3-node value of characteristic component q on side L (0) or R (1))
  uint8_t* dbg_branch = nullptr;
  void* FGv = nullptr;
  void* h = nullptr;
};

enum DivMode { DIV_RESIDUAL = 0, DIV_STAGE = 1 };

// Everything the persistent stage kernel reads, passed by value.
struct KernelArgs {
  int V, A, Ef, G;
  const int32_t *sten, *vptr, *vidx, *eptr, *eidx, *gid, *gdonor, *gflags, *vmem;
  const void *nrm, *w5, *w3, *cv, *ce, *cvis;
  void *Ua, *FG, *FGv, *h;
  unsigned long long* dtbits;
  double* dt_last;
  unsigned* err;
  unsigned* bar;
  unsigned spins;
  float* wref;
  int div_df;
  const void *cvdf, *cedf;
  const double* sig;
};

// Ghost refresh of U; fixed ghosts (donor -1) take their values from `base` (the step's input
// state; pass U itself outside a step).
cudaError_t launch_ghost(const DevMesh& m, double* U, const double* base, cudaStream_t s);
// Raises k_div_gs's dynamic shared-memory limit to smem_bytes when above the default 48 KB
// (called once per mesh at upload, outside any stream capture).
cudaError_t prepare_div_gs(int smem_bytes);
cudaError_t launch_conversions(int64_t n, const double* x, float* f_int, float* f_hw,
                               double* d_int, double* d_hw, cudaStream_t s);
cudaError_t launch_vertex(const DevMesh& m, const double* U, const Phys& ph, cudaStream_t s);
cudaError_t launch_edge(const DevMesh& m, const Phys& ph, cudaStream_t s);
// out = R (residual mode) or out = a*Un + b*(Us + dt*R) (stage mode); dt_fixed <= 0 selects
// dt_member[mesh] when dt_member is given (device array, one step per batch member), else
// dt = cfl * (device minimum of the vertex's mesh).
cudaError_t launch_div(const DevMesh& m, const double* Us, const double* Un, double* out,
                       int mode, double a, double b, double dt_fixed, const Phys& ph,
                       int lanes, cudaStream_t s, const double* dt_member = nullptr);
cudaError_t launch_dtmin(const DevMesh& m, const double* U, const Phys& ph, cudaStream_t s);
// One cooperative launch running ghost refresh (optional), vertex fluxes, edge fluxes and the
// divergence + stage update of one RK stage, phases separated by bounded grid barriers.
cudaError_t launch_stage_persistent(const DevMesh& m, const double* Us, const double* Un,
                                    double* out, int mode, double a, double b, double dt_fixed,
                                    const Phys& ph, int lanes, int grid, bool do_ghost,
                                    cudaStream_t s, const double* dt_member = nullptr);
// Copies between one array per batch member (ptrs[k]: 12 x nv_k, input order; off: n + 1
// device offsets of the members in the batch's input order) and the batch's 12 x V array:
// to_batch = true gathers the members into U, false scatters U back to them.
cudaError_t launch_batch_copy(int V, int n, const int64_t* off, double* const* ptrs, double* U,
                              bool to_batch, cudaStream_t s);
cudaError_t persistent_max_blocks(const DevMesh& m, int lanes, int* per_sm, int* nsm);
cudaError_t launch_permute(int V, const int32_t* perm, const double* src, double* dst,
                           bool gather, cudaStream_t s);

}  // namespace hfd
