// Internal data layout of libpsdf_b300 (host + device).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <utility>
#include <string>
#include <vector>

#include "../../include/psdf.h"

namespace psdf {

constexpr int kMaxM = PSDF_MAX_FOOTPRINT;       // robot vertices
constexpr int kMaxObsEdges = PSDF_MAX_OBSTACLE_EDGES;
constexpr int kDefaultTileEdges = 256;
constexpr int kMaxTileEdges = 256;
constexpr int kPairShiftEdge = 8;
constexpr int kPairShiftKind = 4;
constexpr unsigned kMaxEdgeIndex = (1u << 24) - 1;  // fits the pair-id edge field

// Kinds of the active pair (see include/psdf.h).
enum Kind : int {
  kVertEdge = 0,
  kObsVRobotEdge = 1,
  kObsBRobotEdge = 2,
  kRAxisOMax = 3,
  kRAxisRMax = 4,
  kRAxisOMaxB = 5,
  kRAxisRMaxB = 6,
  kOAxisOMax = 7,
  kOAxisRMax = 8,
};

// Robot footprint constants, passed BY VALUE as a kernel parameter so that
// every lane reads them through the constant bank (Sec. IV-A.1: the local
// footprint is pose-invariant).
struct FootprintK {
  float vx[kMaxM], vy[kMaxM];    // vertices v_l (CCW, local)
  float ex[kMaxM], ey[kMaxM];    // robot edges e_l = v_{l+1} - v_l
  float inv_e2[kMaxM];           // 1 / (|e_l|^2 + eps_seg)
  float nx[kMaxM], ny[kMaxM];    // outward unit normals n_l
  float alo[kMaxM], ahi[kMaxM];  // robot interval on n_l: [alpha_P, beta_P]
  float radius;                  // max_l |v_l| (bounding radius about the pose)
  float inner;                   // radius of a disc about the pose inside the footprint,
                                 // or -1 when the pose lies outside it
  int m;
};

// Per-call scalar parameters.
struct ParamsK {
  float eps_sat;
  float eta;  // <= 0: hard minimum
};

// Tile header.  A tile is a contiguous blob in device memory:
//   int4   obs[n_obs]        {vtx_begin (within tile), n_edges, rank, sorted obstacle}
//   float4 vtx[2 * n_vtx]    per obstacle vertex k (= start of edge k):
//                            a = {Ax, Ay, 1/(|u|^2+eps_seg), 1/(|u|+eps_axis)}
//                            b = {alpha', beta', Bx, By}
// alpha', beta': the obstacle's interval on its own edge normal
// rot90(u)/(|u|+eps_axis), measured from the edge's start A (pose-invariant).
// blob_bytes covers these two parts; right after them follow
//   float4 circ[n_obs]       {cx, cy, r, rin}: a circle containing the obstacle
//                            and the radius of a disc about its centre inside it
// which only the cull reads (blob_off of the next tile skips them).
struct TileHdr {
  int blob_off;    // byte offset of the blob (16-byte aligned)
  int blob_bytes;  // multiple of 16
  int n_obs;
  int n_vtx;
  float aabb[4];   // xmin, ymin, xmax, ymax of the tile's endpoints
};

// Obstacle record of a caller row (one per row, so that the per-pose
// epilogue and the backward reach it from a row index in one load): vertex
// records live at vtx[2 * (vtx_global + k)]; n = 0 marks a row outside every
// obstacle.
struct ObsRec {
  int vtx_global;  // first vertex record (sorted order)
  int n;           // edges (1 = segment)
  int orig_first;  // caller's row index of its first edge (the tie-break rank)
  int tile;
};

// Obstacle record of the exact tile cull, one per obstacle in sorted (tile)
// order: a circle containing the obstacle, the radius of a disc about its
// centre inside it, and where the obstacle's vertex records are.
struct CullObs {
  float4 circ;  // {cx, cy, r, rin}
  int4 rec;     // {first vertex record (vtx, sorted order), edges, rank, tile}
};

// What the cull reads of a tile beside its AABB: {first sorted obstacle,
// obstacles, edges, tile index}.
using TileInfo = int4;

// Uniform grid over a scene's bounding box for the cull's tile lookups.
// Cell (i, j) covers [x0 + i cs, x0 + (i + 1) cs) x [y0 + j cs, y0 + (j + 1) cs)
// and lists, in increasing tile order, every tile whose AABB comes within
// `reach` of the cell in the L-infinity sense (so every tile within Euclidean
// distance reach as well).  A pose whose computed cell is (i, j) finds in
// that one list every tile within reach_q of itself: reach_q is reach less
// a margin for the rounding of the pose's cell index.  nx = 0: no grid, every
// lookup scans all tiles.
struct CullGrid {
  float x0 = 0.f, y0 = 0.f, inv_cs = 0.f, reach_q = -1.f;
  int nx = 0, ny = 0;
  const int *off = nullptr;    // [nx * ny + 1] list offsets (device)
  const int *tl = nullptr;     // tile lists (device)
  const float4 *ab = nullptr;  // [entries] AABB of tile tl[i], beside it (device)
  const int4 *info = nullptr;  // [entries] TileInfo of tile tl[i] (device)
  // The same lists padded to a fixed capacity per cell (cell c's entries at
  // c * cap .. c * cap + cap - 1; padding: an empty AABB and tile -2), so
  // that a pose reaches its entries from its cell index in one load; cap = 0
  // when some list is too long (the lists above serve then).
  int cap = 0;
  const float4 *fab = nullptr;
  const int4 *finfo = nullptr;
};

// Candidate grid of the cull: a uniform grid of nx x ny square cells of
// side 1 / inv_cs from (x0, y0).  Cell c lists the kCand obstacles whose
// circles come nearest it -- near distance nd(o) = dist(c_o, cell) - r_o,
// the cell widened by a margin for the rounding of a pose's cell index --
// their circles circ[c * kCand + i] and records rec[c * kCand + i] (the
// CullObs circle {cx, cy, r, rin} and record {first vertex record, edges,
// rank, tile}; padding: r = inf, rin = -inf and no edges), and rc[c], a
// radius that no unlisted obstacle's near distance falls below (+inf when
// every obstacle is listed).  Any circle bounds phi
// from above at any pose; and for a pose in the cell whose upper bound UB
// satisfies rc - r_foot > UB, every unlisted obstacle is separated from the
// footprint by more than UB, so the listed ones are all it needs.  nx = 0:
// no grid.
constexpr int kCand = 32;
struct CandGrid {
  float x0 = 0.f, y0 = 0.f, inv_cs = 0.f;
  int nx = 0, ny = 0;
  const float4 *circ = nullptr;
  const int4 *rec = nullptr;
  const float *rc = nullptr;
};

}  // namespace psdf

struct psdf_scene {
  int64_t rows_total = 0;  // caller's row count (E for CSR, Mbar * mbar padded)
  int32_t M = 0, n_tiles = 0, tile_edges = 0, max_obs_edges = 0;
  int64_t n_edges = 0;
  float bbox[4] = {0, 0, 0, 0};
  float eps_seg = 0.f, eps_axis = 0.f;
  int device = 0;
  // device arrays
  psdf::TileHdr *d_tiles = nullptr;
  unsigned char *d_blob = nullptr;
  psdf::ObsRec *d_row_obs = nullptr;  // [rows_total] obstacle record of each caller row
  float4 *d_vtx = nullptr;            // [2 * n_edges] sorted vertex records
  int *d_far = nullptr;               // [n_edges] far vertex index within its obstacle
  psdf::CullGrid grid;                // the cull's cell -> tile lists
  float grid_cell = 0.f;              // cell side (m)
  int64_t grid_entries = 0;
  int *d_cell_off = nullptr, *d_cell_tiles = nullptr;
  float4 *d_cell_aabbs = nullptr;
  int4 *d_cell_info = nullptr;
  float4 *d_cell_fab = nullptr;  // fixed-capacity lists (grid.cap > 0)
  int4 *d_cell_finfo = nullptr;
  psdf::CandGrid cand;                  // the cull's per-cell candidate obstacles
  float4 *d_cand_circ = nullptr;
  int4 *d_cand_rec = nullptr;
  float *d_cand_rc = nullptr;
  psdf::CullObs *d_cull_obs = nullptr;  // [M] cull records in sorted order
  float4 *d_tile_ab = nullptr;          // [n_tiles] AABBs
  int4 *d_tile_info = nullptr;          // [n_tiles] TileInfo
  size_t device_bytes = 0;
  // host copies used for launch configuration
  int max_blob_bytes = 0;      // largest tile blob (obstacle + vertex records)
  int max_blob_ext_bytes = 0;  // the same with the tile's obstacle circles
};

namespace psdf {
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

// one obstacle of the caller's layout
struct ObsIn {
  int64_t first_row;  // caller's row of the first edge
  int n;              // edges
};

// Host image of a prepared scene (scene.cu), before upload: a scene of its
// own (psdf_scene) or one instance of a batched plan.
struct HostScene {
  int64_t rows_total = 0, n_edges = 0;
  int M = 0, T = 0, tile_edges = 0, max_n = 0, max_blob = 0, max_blob_ext = 0;
  float bb[4] = {0, 0, 0, 0};
  double eps_seg = 0, eps_axis = 0;
  std::vector<TileHdr> tiles;
  std::vector<unsigned char> blob;
  std::vector<float4> vtx;
  std::vector<int> far;
  std::vector<ObsRec> row_obs;
  std::vector<CullObs> cull_obs;  // [M] sorted order
  std::vector<float4> tile_ab;    // [T]
  std::vector<int4> tile_info;    // [T]
};
int build_host_scene(const float *rows, int64_t rows_total, const std::vector<ObsIn> &obs,
                     int tile_edges, const psdf_params *prm, HostScene *hs);

template <class T>
int dev_upload(T **dst, const std::vector<T> &src, cudaStream_t st, size_t *bytes)
{
  size_t nb = std::max<size_t>(src.size(), 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void **)dst, nb);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  *bytes += nb;
  if (!src.empty()) {
    e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(host -> device)");
  }
  return PSDF_OK;
}

// Optional SQP-RTI stage parameters written by an epilogue (Alg. 1, PSDF-MPC
// pipeline): stage[4 p] = phi - d_min (h), stage[4 p + 1 .. 3] = -d phi / d x
// (J_g).
struct StageOut {
  float *stage = nullptr;
  float d_min = 0.f;
  float4 *saved = nullptr;  // saved backward records (psdf_saved_grad), hard minimum
};

// Launch with programmatic stream serialization (see pdl_wait in
// psdf_device.cuh): the kernel may begin while the previous kernel on the
// stream finishes; it must call pdl_wait() before touching that kernel's
// outputs.
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args &&...args)
{
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// shared host helpers (eval.cu)
int device_sms();
// polls a bounded device-side wait makes before it gives up (kernel argument
// of every kernel with such a wait; psdf_debug_set_wait_limit)
unsigned wait_limit();
int make_footprint(const float *fp, int m, float eps_seg, FootprintK *F);
int check_eval_args(const psdf_scene *scene, const float *poses, int64_t P,
                    const psdf_params *params, void *workspace, size_t ws_bytes);
// per-pose epilogue (value, active pair, optional gradient) from 64-bit keys
int launch_epilogue(const FootprintK &F, const psdf_scene *sc, const float *poses, long long P,
                    const ParamsK &pk, const unsigned long long *keys, const int *err,
                    float *phi, float *dphi, unsigned *active, cudaStream_t st,
                    float4 *saved = nullptr);
// value (+ gradient if dphi) evaluation with a given workspace (eval.cu)
int eval_common(const float *footprint, int32_t m, const psdf_scene *scene, const float *poses,
                int64_t P, const psdf_params *params, float *phi, float *dphi, unsigned *active,
                void *ws, size_t ws_bytes, void *stream, const StageOut &so = StageOut());
}  // namespace psdf
