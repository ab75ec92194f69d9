// Exact tile cull with a proposal (psdf_eval_culled and its helpers).
//
// One launch, each pose handled by 16 lanes of its own (cull_kernel):
//   ranking      the tiles of the pose's cell in a uniform grid (every tile
//                within one cell size; all tiles for a pose outside the
//                grid), ordered by their conservative bound; the pose
//                proposes its K nearest tiles, or the K best of its 8 nearest
//                re-ranked by the tile-proposal network on tensor cores
//   upper bound  UB >= phi from the circles of the proposed tiles' obstacles
//   evaluation   every tile whose bound does not exceed UB (the cell's list
//                holds them all while UB's reach is within the cell's; else
//                every tile is tested), the proposed ones always; obstacles
//                whose circle bound exceeds UB are skipped, the others
//                evaluated exactly
//   epilogue     as for the full scan, on the winning obstacle
// The scene's arrays are brought into L2 by bulk prefetches (TMA) at the
// start of the launch.  Every tile holding a value at or below phi has a
// bound <= phi <= UB, so it is evaluated; every obstacle skipped has a value
// above UB, which is never below phi.  The minimum over 64-bit keys does not
// depend on evaluation order, so the result equals the full scan's bit for
// bit.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "profile.h"
#include "psdf_device.cuh"
#include "psdf_internal.h"

struct psdf_mlp {
  uint32_t *d_frag = nullptr;  // [8][32][2] layer-1 B fragments, then [4][32][2] layer 2
  float b2 = 0.f;
  int device = 0;
};

namespace psdf {

constexpr int kMaxK = PSDF_CULL_MAX_K;
constexpr int kPre = 8;  // bound-ranked candidates the network re-ranks per pose
constexpr int kFrag1Words = 8 * 32 * 2;
constexpr int kFrag2Words = 4 * 32 * 2;
constexpr int kMaxScanTiles = 1024 * 64;

// ---------------------------------------------------------------------------
// conservative lower bound and network inputs
// ---------------------------------------------------------------------------
// Lower bound (metres) on the separation of the posed footprint from any
// point of the tile's AABB: distance from p to the AABB minus the footprint
// radius, minus a margin of 1e-4 m + 1e-5 of the distance.  The margin is far
// above the float32 rounding of this bound and of the evaluated values
// (about 1e-6 of the distance), so a positive bound is below every obstacle
// value the kernels compute for the tile.
__device__ __forceinline__ float tile_lb(const float *ab, float px, float py, float rfoot)
{
  const float dx = fmaxf(fmaxf(ab[0] - px, px - ab[2]), 0.f);
  const float dy = fmaxf(fmaxf(ab[1] - py, py - ab[3]), 0.f);
  const float d = sqrtf(dx * dx + dy * dy);
  return (d - rfoot) - (1e-4f + 1e-5f * d);
}

// Bounds from an obstacle's circle {cx, cy, r}: its signed distance to the
// posed footprint lies in [|p - C| - r - r_foot, |p - C| + r + r_foot]
// (every footprint point is within r_foot of p, every obstacle point within r
// of C), each widened by the bound's margin.
__device__ __forceinline__ float circle_ub(float4 cc, float px, float py, float rfoot,
                                           float rin)
{
  const float dx = cc.x - px, dy = cc.y - py;
  const float d = sqrtf(dx * dx + dy * dy);
  // a disc of radius cc.w about the circle's centre lies in the obstacle;
  // with a disc of radius rin about the pose inside the footprint the two
  // come within d - rin - cc.w of each other, else within d + r + r_foot
  const float b = rin >= 0.f ? fmaxf(d - rin - cc.w, 0.f) : (d + cc.z + rfoot);
  return b + (1e-4f + 1e-5f * d);
}

__device__ __forceinline__ float circle_lb_value(float4 cc, float px, float py, float rfoot)
{
  const float dx = cc.x - px, dy = cc.y - py;
  const float d = sqrtf(dx * dx + dy * dy);
  const float lb = (d - cc.z - rfoot) - (1e-4f + 1e-5f * d);
  return lb > 0.f ? lb * lb * (1.f - 1e-6f) : -kInf;
}

// An upper bound (metres) in the min-key value domain (d^2 when positive).
__device__ __forceinline__ float ub_value(float ub)
{
  return ub > 0.f ? ub * ub * (1.f + 1e-6f) : ub;
}

__device__ __forceinline__ float clampf(float x, float lo, float hi)
{
  return fminf(fmaxf(x, lo), hi);
}

__device__ __forceinline__ float approx_sqrt(float x)
{
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Network inputs 2q, 2q+1: AABB corner q (0..3) in the pose frame.
__device__ __forceinline__ void feat_corner(const float *ab, int q, float px, float py, float c,
                                            float s, float &f0, float &f1)
{
  const float cx = (q == 1 || q == 2) ? ab[2] : ab[0];
  const float cy = (q >= 2) ? ab[3] : ab[1];
  const float dx = cx - px, dy = cy - py;
  f0 = 0.1f * clampf(c * dx + s * dy, -20.f, 20.f);
  f1 = 0.1f * clampf(-s * dx + c * dy, -20.f, 20.f);
}

// Network inputs 8 + 2q, 9 + 2q, without divergence across the quad:
// q = 0: distances to corners 0, 1; q = 1: to corners 2, 3; q = 2: distance
// to the AABB, footprint radius; q = 3: edge fraction, 1.
__device__ __forceinline__ void feat_rest(const float *ab, int q, float px, float py,
                                          float rfoot, float edge_frac, float &f0, float &f1)
{
  // point a: corner 0 (q = 0), corner 2 (q = 1), the AABB point nearest p (q = 2)
  const float ax = (q == 0) ? ab[0] : (q == 1) ? ab[2] : clampf(px, ab[0], ab[2]);
  const float ay = (q == 0) ? ab[1] : (q == 1) ? ab[3] : clampf(py, ab[1], ab[3]);
  // point b: corner 1 (q = 0), corner 3 (q = 1)
  const float bx = (q == 0) ? ab[2] : ab[0];
  const float by = (q == 0) ? ab[1] : ab[3];
  const float da = approx_sqrt((ax - px) * (ax - px) + (ay - py) * (ay - py));
  const float db = approx_sqrt((bx - px) * (bx - px) + (by - py) * (by - py));
  f0 = (q == 3) ? edge_frac : 0.1f * fminf(da, 30.f);
  f1 = (q == 3) ? 1.f : (q == 2) ? rfoot : 0.1f * fminf(db, 30.f);
}

// ---------------------------------------------------------------------------
// tensor-core network: 16 -> 64 (ReLU) -> 1, FP16 operands, FP32 accumulate
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi)
{
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ uint32_t pack_relu_f16x2(float lo, float hi)
{
  uint32_t r;
  asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1)
{
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct MlpFrags {
  uint32_t b1[8][2];
  uint32_t b2[4][2];
};

__device__ __forceinline__ void load_frags(const uint32_t *frag, int lane, MlpFrags &w)
{
  const uint2 *f2 = reinterpret_cast<const uint2 *>(frag);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint2 v = __ldg(f2 + j * 32 + lane);
    w.b1[j][0] = v.x;
    w.b1[j][1] = v.y;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint2 v = __ldg(f2 + kFrag1Words / 2 + j * 32 + lane);
    w.b2[j][0] = v.x;
    w.b2[j][1] = v.y;
  }
}

// Scores of 16 rows whose rows g and g + 8 each have their own pose and tile
// (the network re-ranking candidate tiles); same arithmetic as mlp_rows.
__device__ __forceinline__ void mlp_rows_pair(const MlpFrags &w, int q, const float *aba,
                                              float efa, float pxa, float pya, float ca,
                                              float sa, const float *abb, float efb, float pxb,
                                              float pyb, float cb, float sb, float rfoot,
                                              float &sc_a, float &sc_b)
{
  float fa0, fa1, fb0, fb1, ga0, ga1, gb0, gb1;
  feat_corner(aba, q, pxa, pya, ca, sa, fa0, fa1);
  feat_corner(abb, q, pxb, pyb, cb, sb, fb0, fb1);
  feat_rest(aba, q, pxa, pya, rfoot, efa, ga0, ga1);
  feat_rest(abb, q, pxb, pyb, rfoot, efb, gb0, gb1);
  const uint32_t a0 = pack_f16x2(fa0, fa1), a1 = pack_f16x2(fb0, fb1);
  const uint32_t a2 = pack_f16x2(ga0, ga1), a3 = pack_f16x2(gb0, gb1);
  float h[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    h[j][0] = h[j][1] = h[j][2] = h[j][3] = 0.f;
    mma16816(h[j], a0, a1, a2, a3, w.b1[j][0], w.b1[j][1]);
  }
  float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int s2 = 0; s2 < 4; ++s2) {
    const uint32_t c0 = pack_relu_f16x2(h[2 * s2][0], h[2 * s2][1]);
    const uint32_t c1 = pack_relu_f16x2(h[2 * s2][2], h[2 * s2][3]);
    const uint32_t c2 = pack_relu_f16x2(h[2 * s2 + 1][0], h[2 * s2 + 1][1]);
    const uint32_t c3 = pack_relu_f16x2(h[2 * s2 + 1][2], h[2 * s2 + 1][3]);
    mma16816(o, c0, c1, c2, c3, w.b2[s2][0], w.b2[s2][1]);
  }
  sc_a = o[0];
  sc_b = o[2];
}

// Scores of 16 rows (rows g and g + 8 belong to this lane's quad g = lane/4)
// for one tile.  Returns the two scores in lanes with (lane & 3) == 0.
__device__ __forceinline__ void mlp_rows(const MlpFrags &w, const float *ab, int q,
                                         float pxa, float pya, float ca, float sa, float pxb,
                                         float pyb, float cb, float sb, float rfoot,
                                         float efrac, float &sc_a, float &sc_b)
{
  float fa0, fa1, fb0, fb1, ga0, ga1, gb0, gb1;
  feat_corner(ab, q, pxa, pya, ca, sa, fa0, fa1);
  feat_corner(ab, q, pxb, pyb, cb, sb, fb0, fb1);
  feat_rest(ab, q, pxa, pya, rfoot, efrac, ga0, ga1);
  feat_rest(ab, q, pxb, pyb, rfoot, efrac, gb0, gb1);
  const uint32_t a0 = pack_f16x2(fa0, fa1), a1 = pack_f16x2(fb0, fb1);
  const uint32_t a2 = pack_f16x2(ga0, ga1), a3 = pack_f16x2(gb0, gb1);
  float h[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    h[j][0] = h[j][1] = h[j][2] = h[j][3] = 0.f;
    mma16816(h[j], a0, a1, a2, a3, w.b1[j][0], w.b1[j][1]);
  }
  float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int s2 = 0; s2 < 4; ++s2) {
    const uint32_t c0 = pack_relu_f16x2(h[2 * s2][0], h[2 * s2][1]);
    const uint32_t c1 = pack_relu_f16x2(h[2 * s2][2], h[2 * s2][3]);
    const uint32_t c2 = pack_relu_f16x2(h[2 * s2 + 1][0], h[2 * s2 + 1][1]);
    const uint32_t c3 = pack_relu_f16x2(h[2 * s2 + 1][2], h[2 * s2 + 1][3]);
    mma16816(o, c0, c1, c2, c3, w.b2[s2][0], w.b2[s2][1]);
  }
  sc_a = o[0];
  sc_b = o[2];
}

// Squared distance from p to a tile's AABB: the bound's ranking key (the
// bound is increasing in the distance, so no square root is needed to rank).
__device__ __forceinline__ float aabb_d2(float4 a4, float px, float py)
{
  const float dx = fmaxf(fmaxf(a4.x - px, px - a4.z), 0.f);
  const float dy = fmaxf(fmaxf(a4.y - py, py - a4.w), 0.f);
  return dx * dx + dy * dy;
}

// A distance D' such that every tile whose bound does not exceed ub lies
// within D' of p: lb <= ub  <=>  d (1 - 1e-5) <= ub + r_foot + 1e-4, widened
// by far more than the rounding of either side.  Negative: no tile.
__device__ __forceinline__ float cand_radius(float ub, float rfoot)
{
  const float D = (ub + rfoot + 1e-4f) / (1.f - 1e-5f);
  return D * (1.f + 1e-5f) + 1e-6f;
}

// ---------------------------------------------------------------------------
// proposals
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void topk_insert(float (&sc)[K], int (&id)[K], float v, int t)
{
  if (!(v < sc[K - 1])) return;
  sc[K - 1] = v;
  id[K - 1] = t;
#pragma unroll
  for (int i = K - 1; i > 0; --i) {
    if (sc[i] < sc[i - 1]) {
      const float ts = sc[i];
      sc[i] = sc[i - 1];
      sc[i - 1] = ts;
      const int ti = id[i];
      id[i] = id[i - 1];
      id[i - 1] = ti;
    }
  }
}

__device__ __forceinline__ float4 tile_aabb(const TileHdr *__restrict__ tiles, int t)
{
  return __ldg(reinterpret_cast<const float4 *>(tiles + t) + 1);
}

// The pose's cell in the cull grid, or -1 (no grid, or the pose outside it:
// every lookup then scans all tiles).
__device__ __forceinline__ int grid_cell(const CullGrid &g, float px, float py)
{
  if (g.nx == 0) return -1;
  const float fx = __fmul_rn(__fsub_rn(px, g.x0), g.inv_cs);
  const float fy = __fmul_rn(__fsub_rn(py, g.y0), g.inv_cs);
  if (!(fx >= 0.f && fx < (float)g.nx && fy >= 0.f && fy < (float)g.ny)) return -1;
  return (int)fy * g.nx + (int)fx;
}

// The pose's cell in the candidate grid, clamped to the grid (a pose
// outside it takes the nearest cell's circles for its bound: any circle is a
// valid one), and whether the pose lies in it (only then may the cell's list
// stand for the whole scene).
__device__ __forceinline__ long long cand_cell(const CandGrid &g, float px, float py, bool &in)
{
  const float fx = __fmul_rn(__fsub_rn(px, g.x0), g.inv_cs);
  const float fy = __fmul_rn(__fsub_rn(py, g.y0), g.inv_cs);
  in = fx >= 0.f && fx < (float)g.nx && fy >= 0.f && fy < (float)g.ny;
  const float cx = fminf(fmaxf(fx, 0.f), (float)(g.nx - 1));
  const float cy = fminf(fmaxf(fy, 0.f), (float)(g.ny - 1));
  return (long long)(int)cy * g.nx + (int)cx;
}

// ---------------------------------------------------------------------------
// the fused cull: each pose's proposals, exact evaluation and epilogue by
// its own 16 lanes, in one launch
// ---------------------------------------------------------------------------
// CTA shape: 2 poses a warp.  The proposals' tile path shares its tile and
// circle tests over 16 poses (256 threads); the candidate grid, whose poses
// rarely take tiles, waits at its barriers for fewer warps with 8 (128).
template <int THREADS>
struct CullShape {
  static constexpr int kThreads = THREADS;
  static constexpr int kWarps = THREADS / 32;
  static constexpr int kPoses = 2 * kWarps;                 // poses per CTA
  static constexpr int kGroups = THREADS / 4;               // items evaluated per pass
  static constexpr int kSegCap = kPoses * 16;               // segments of one round
  static constexpr int kSegsPerPass = THREADS / 8;          // segments whose circles a pass tests
  static constexpr int kQCap = 2 * THREADS * 8;             // queued items: two steps
  static constexpr int kMinBlocks = 512 / THREADS;          // 128 registers a thread
};
constexpr int kRL = 4;             // best tiles a lane keeps from its ranking pass
constexpr int kFilt = 8;           // circle bounds a thread tests per block
constexpr int kItemLanes = 4;      // lanes per evaluated (pose, obstacle) item
constexpr int kStatWords = 8;      // counters per CTA in the workspace
constexpr int kOutSaved = 4;       // out_s: phi, active pair, -, -, the saved record
constexpr int kOutWords = kOutSaved + 16;
constexpr int kStatBase = 32;      // first counter word (the header is 256 bytes)
constexpr long long kPrefetchChunk = 16384;  // bytes per bulk L2 prefetch
constexpr int kMaxPrefetch = 8;
constexpr unsigned kFull = 0xffffffffu;
// where the upper bound comes from
constexpr int kPropBound = 1;    // the circles of the k tiles of smallest bound
constexpr int kPropNet = 2;      // the circles of the network's k best tiles
constexpr int kPropCircles = 3;  // the pose's cell of the candidate grid
template <int PROP>
using ShapeOf = CullShape<PROP == kPropCircles ? 128 : 256>;
constexpr int kMinPoses = ShapeOf<kPropCircles>::kPoses;  // the smallest CTA's (workspace sizing)

// Per-CTA counters (workspace words kStatBase + kStatWords * CTA + i).
enum CullStat { kStProp, kStFb, kStFbPoses, kStBound, kStCirc, kStObs, kStEdges, kStCount };

// Scene arrays brought into L2 with bulk prefetches at the start of the
// launch (every chunk by thread 0 of one CTA, round-robin): a step then pays
// the scene's bytes once at the HBM bandwidth instead of a chain of
// dependent HBM round trips per pose.  ptr 16-byte aligned, bytes a multiple
// of 16.
struct Prefetch {
  const unsigned char *ptr[kMaxPrefetch];
  long long bytes[kMaxPrefetch];
  long long first[kMaxPrefetch + 1];  // first chunk of each range; first[n] = all chunks
  int n;
};

struct CullArgs {
  const float *poses;
  long long P;
  CullGrid grid;
  CandGrid cand;            // candidate obstacles per cell (kPropCircles)
  const float4 *tile_ab;    // all tiles: poses outside the grid, bounds beyond its reach
  const int4 *tile_info;
  int T;
  int K;                    // proposals per pose
  const CullObs *obs;
  const float4 *vtx;
  const int *far;
  const ObsRec *row_obs;    // obstacle record of each caller row (the key's rank)
  float ub_pad;             // soft minimum: most a penetrating obstacle's value exceeds 0
  float eps_axis;
  const uint32_t *frag;     // network fragments (NET)
  float b2;
  float *phi, *dphi;
  unsigned *active;
  float4 *saved;            // saved backward records (hard minimum), or NULL
  unsigned long long *ws;   // {CTAs, error word, ...} then kStatWords per CTA
  Prefetch pf;
};

__device__ __forceinline__ void bulk_prefetch_l2(const void *p, unsigned bytes)
{
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void prefetch_scene(const Prefetch &pf)
{
  for (long long c = blockIdx.x; c < pf.first[pf.n]; c += gridDim.x) {
    int i = 0;
    while (i + 1 < pf.n && c >= pf.first[i + 1]) ++i;
    const long long off = (c - pf.first[i]) * kPrefetchChunk;
    const long long rest = pf.bytes[i] - off;
    const unsigned sz = (unsigned)((rest < kPrefetchChunk ? rest : kPrefetchChunk) & ~15LL);
    if (sz > 0) bulk_prefetch_l2(pf.ptr[i] + off, sz);
  }
}

// The tiles a pose looks at: entries [lo, hi) of its cell's list, or every
// tile.
struct Entries {
  const float4 *ab;
  const int4 *info;
  int lo, hi;
};

__device__ __forceinline__ Entries entries_of(const CullArgs &a, int cell, bool use_cell)
{
  if (use_cell && a.grid.cap > 0)  // fixed-capacity lists: no offsets to load
    return Entries{a.grid.fab, a.grid.finfo, cell * a.grid.cap, (cell + 1) * a.grid.cap};
  if (use_cell)
    return Entries{a.grid.ab, a.grid.info, __ldg(a.grid.off + cell), __ldg(a.grid.off + cell + 1)};
  return Entries{a.tile_ab, a.tile_info, 0, a.T};
}

// The tile bound in the min-key value domain (as circle_lb_value): every
// obstacle of the tile has a value above it, or -inf (no claim).
__device__ __forceinline__ float tile_lb_value(float4 ab, float px, float py, float rfoot)
{
  const float b[4] = {ab.x, ab.y, ab.z, ab.w};
  const float lb = tile_lb(b, px, py, rfoot);
  return lb > 0.f ? lb * lb * (1.f - 1e-6f) : -kInf;
}

// Obstacle (sorted index) of the flattened position f over a half's tiles:
// tile j holds positions st[j] .. st[j + 1] - 1, its obstacles from s0[j].
__device__ __forceinline__ int flat_obstacle(const int *s0, const int *st, int nseg, int f)
{
  int j = 0;
  while (j + 1 < nseg && f >= st[j + 1]) ++j;
  return s0[j] + (f - st[j]);
}

// One CTA = 16 poses (8 under the candidate grid); one warp = 2 poses, 16
// lanes each (lanes 0-15 pose a, 16-31 pose b) for the per-pose stages:
//  1. ranking (PROP = bound or network): the tiles of the pose's cell in the
//     cull grid (every tile within one cell size of it), else all tiles;
//     lane hl takes entries hl, hl + 16, ... and keeps its 4 smallest AABB
//     distances; rounds of a 16-lane minimum give the pose's smallest ones
//     in order.  The pose proposes its K nearest tiles, or (network) the K
//     best network scores among its 8 nearest (2 poses x 8 candidates = 16
//     rows of one tensor-core pass).
//  2. an upper bound UB >= phi from the circles of the proposed tiles'
//     obstacles, or (PROP = circles, no stage 1) from the 32 candidates of
//     the pose's cell in the scene's candidate grid, two a lane, loaded
//     right after the pose; a pose whose UB lies within its cell's
//     completeness radius queues its candidates that pass their circle
//     test and takes no tiles.
// then, by the whole CTA, in rounds over chunks of 16 list entries per pose
// (the cell's list when every tile whose bound does not exceed UB lies
// within the grid's reach, else all tiles):
//  3. each pose's tiles of the chunk whose bound does not exceed its UB (the
//     proposed ones always) join the round's list of segments (pose, first
//     obstacle, obstacles);
//  4. 8 threads per segment test its obstacles' circle bounds against the
//     pose's UB; the survivors go to one CTA-wide queue, evaluated exactly
//     by 4 lanes each, and merged into the pose's 64-bit key in shared
//     memory (atomicMin); the item holding a pose's minimum after a pass
//     leaves its detail.  Sharing the work over the CTA's threads keeps a
//     pose with several nearby tiles from stretching its own warp.
//  5. epilogue: the hard minimum's gradients from the winners' details by
//     kind class, one class a warp and one lane a pose, then the saved
//     records by each pose's 16 lanes and phi, the active pairs and the
//     gradients as three contiguous blocks; the soft minimum's by one lane
//     a pose in the first warps.  Each warp then adds its counters to the
//     CTA's workspace words.
// No skipped tile or obstacle can hold a value at or below phi, and the key
// minimum does not depend on the order of evaluation, so the outputs equal
// the full scan's bit for bit.
template <int M, int PROP, bool SOFT>
__global__ void __launch_bounds__(ShapeOf<PROP>::kThreads, ShapeOf<PROP>::kMinBlocks)
    cull_kernel(const FootprintK F, const ParamsK prm, const CullArgs a)
{
  using S = ShapeOf<PROP>;
  constexpr int kCullThreads = S::kThreads, kCullWarps = S::kWarps, kPoses = S::kPoses;
  constexpr int kGroups = S::kGroups, kSegCap = S::kSegCap, kSegsPerPass = S::kSegsPerPass;
  constexpr int kQCap = S::kQCap;
  static_assert(kGroups == kCullThreads / kItemLanes && kQCap == 2 * kCullThreads * kFilt,
                "CTA shape");
  static_assert(kPoses * kCand + kCullThreads * kFilt <= kQCap, "queue too small");
  static_assert(kCullWarps % 4 == 0, "the epilogue gives each warp of a group of four one class");
  constexpr bool NET = PROP == kPropNet;
  constexpr bool CIRC = PROP == kPropCircles;
  __shared__ int ub_s0[kCullWarps][2][kMaxK + 1];  // proposed tiles, flattened
  __shared__ int ub_st[kCullWarps][2][kMaxK + 1];
  __shared__ int cand_s[kCullWarps][2][kPre];
  __shared__ float score_s[kCullWarps][2][kPre];
  __shared__ float4 pose_s[kPoses];
  __shared__ float thr_s[kPoses];
  __shared__ unsigned long long key_s[kPoses];
  // hard minimum: the winning item's detail and obstacle record, then each
  // pose's outputs -- phi, the active pair, and the saved record (its first
  // three words the pose gradient); a pose without obstacles keeps the
  // initial ones
  __shared__ Active det_s[kPoses];
  __shared__ int4 drec_s[kPoses];
  __shared__ float out_s[kPoses][kOutWords];
  __shared__ int seg_first[kSegCap], seg_n[kSegCap];
  __shared__ unsigned char seg_pose[kSegCap];
  __shared__ int q_s[kQCap];
  __shared__ int4 q_rec[CIRC ? kPoses * kCand : 1];  // records of the queued candidates
  __shared__ int nseg_s, nq_s;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int half = lane >> 4, hl = lane & 15;
  const unsigned hmask = half ? 0xffff0000u : 0x0000ffffu;
  const int j = 2 * warp + half;  // the pose within the CTA
  const long long p = (long long)blockIdx.x * kPoses + j;
  const bool valid = p < a.P;
  const bool save = a.saved != nullptr;
  const bool want_grad = save || a.dphi != nullptr;
  int *sg0 = ub_s0[warp][half], *sgt = ub_st[warp][half];
  // the CTA's counters, added to by every warp at the end
  if (tid < kStatWords) a.ws[kStatBase + (long long)blockIdx.x * kStatWords + tid] = 0ull;
  if (tid < kPoses) {
    key_s[tid] = ~0ull;
    if constexpr (!SOFT) {  // no obstacle: phi = +inf, no pair, no gradient rows
      out_s[tid][0] = kInf;
      out_s[tid][1] = __uint_as_float(PSDF_PAIR_NONE);
      Grad none;
      none.gp[0] = none.gp[1] = none.gp[2] = 0.f;
      none.nrow = -1;
      saved_words(none, &out_s[tid][kOutSaved]);
    }
  }
  if (tid == 0) {
    nseg_s = 0;
    nq_s = 0;
    prefetch_scene(a.pf);
  }
  // a following kernel (the backward) may launch now; it waits for this grid
  pdl_trigger();
  float px = 0.f, py = 0.f, th = 0.f;
  if (valid) {
    px = a.poses[3 * p];
    py = a.poses[3 * p + 1];
    th = a.poses[3 * p + 2];
  }
  // (candidate grid) the pose's cell's kCand candidates, two a lane, and
  // its completeness radius: the loads that follow the pose's, issued
  // before the barrier below so that no warp waits for another first
  float4 cc[2] = {make_float4(0.f, 0.f, kInf, -kInf), make_float4(0.f, 0.f, kInf, -kInf)};
  int4 cr[2] = {make_int4(0, 0, 0, -1), make_int4(0, 0, 0, -1)};
  float crc = -kInf;
  bool cin = false;
  if constexpr (CIRC) {
    if (valid && a.cand.nx > 0) {
      const long long cc0 = cand_cell(a.cand, px, py, cin) * kCand;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        cc[q] = __ldg(a.cand.circ + cc0 + hl + 16 * q);
        cr[q] = __ldg(a.cand.rec + cc0 + hl + 16 * q);
      }
      crc = __ldg(a.cand.rc + cc0 / kCand);
    }
  }
  float s, c;
  sincosf(th, &s, &c);
  // the CTA's counters, keys and lists initialised (early: every warp is
  // here at about the same time; nothing below waits for another warp
  // before the tile tests are in)
  __syncthreads();
  MlpFrags w;
  if constexpr (NET) load_frags(a.frag, lane, w);
  const int K = a.K;
  unsigned n_bound = 0, n_circ = 0, n_obs = 0, n_edge = 0;

  // ---- 1. ranking and proposals -------------------------------------------
  const int cell = valid ? grid_cell(a.grid, px, py) : -1;
  Entries E = entries_of(a, cell, cell >= 0);
  if (!valid) E.hi = E.lo;
  // the lane's first two entries (hl, hl + 16) stay in registers for the
  // tile tests below (cell lists rarely hold more than 32)
  // (not under the candidate grid, whose poses rarely need tiles: those
  // that do load their entries in the tile tests)
  float4 kab[2];
  int4 kinf[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int i = E.lo + hl + 16 * q;
    kab[q] = make_float4(kInf, kInf, -kInf, -kInf);
    kinf[q] = make_int4(0, 0, 0, -1);
    if (!CIRC && i < E.hi) {
      kab[q] = __ldg(E.ab + i);
      kinf[q] = __ldg(E.info + i);
    }
  }
  if constexpr (!CIRC) {  // a fixed-capacity list's real entries end at its first padding slot
    const int nreal = __popc(__ballot_sync(kFull, kinf[0].w >= 0) & hmask) +
                      __popc(__ballot_sync(kFull, kinf[1].w >= 0) & hmask);
    if (cell >= 0 && a.grid.cap > 0 && nreal < 32) E.hi = E.lo + nreal;
  }
  int best[kMaxK];
#pragma unroll
  for (int i = 0; i < kMaxK; ++i) best[i] = -1;
  if constexpr (!CIRC) {
    float sc[kRL];
    int id[kRL];
#pragma unroll
    for (int i = 0; i < kRL; ++i) {
      sc[i] = kInf;
      id[i] = -1;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (E.lo + hl + 16 * q < E.hi && kinf[q].w != -2) {
        topk_insert<kRL>(sc, id, aabb_d2(kab[q], px, py), hl + 16 * q);
        ++n_bound;
      }
    for (int i = E.lo + hl + 32; i < E.hi; i += 16) {
      const float4 ab = __ldg(E.ab + i);
      if (!(ab.x <= ab.z)) continue;  // a padding slot (empty AABB)
      topk_insert<kRL>(sc, id, aabb_d2(ab, px, py), i - E.lo);
      ++n_bound;
    }
    // rounds of a 16-lane minimum over the lanes' heads, as 32-bit keys (the
    // top 16 bits of the squared distance -- not negative, so its bits order
    // like the value, to 1/128 -- over the entry's 16 bits; an entry sits in
    // one lane only, so the lane whose head won pops it)
    const int R = NET ? kPre : K;
    int cand[kPre];
    {
      int head = 0;
#pragma unroll
      for (int r = 0; r < kPre; ++r) {
        cand[r] = -1;
        if (r < R) {  // uniform over the warp
          unsigned mine = ~0u;
#pragma unroll
          for (int i = 0; i < kRL; ++i)
            if (i == head && id[i] >= 0)
              mine = (__float_as_uint(sc[i]) & 0xffff0000u) | (unsigned)id[i];
          const unsigned k0 = __reduce_min_sync(kFull, half == 0 ? mine : ~0u);
          const unsigned k1 = __reduce_min_sync(kFull, half == 1 ? mine : ~0u);
          const unsigned key = half ? k1 : k0;
          cand[r] = key != ~0u ? (int)(key & 0xffffu) : -1;
          if (key != ~0u && key == mine) ++head;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kMaxK; ++i) best[i] = i < K ? cand[i] : -1;
    if constexpr (NET) {
      if (hl == 0)
#pragma unroll
        for (int r = 0; r < kPre; ++r) cand_s[warp][half][r] = cand[r];
      __syncwarp();
      // lane 4 g + q: candidate g of both poses, quarter q of its inputs
      const int g = lane >> 2, q = lane & 3;
      // each pose's entries (its cell's list, or all tiles): pointers of lanes 0 and 16
      const float4 *abA = (const float4 *)__shfl_sync(kFull, (unsigned long long)E.ab, 0);
      const float4 *abB = (const float4 *)__shfl_sync(kFull, (unsigned long long)E.ab, 16);
      const int4 *infA = (const int4 *)__shfl_sync(kFull, (unsigned long long)E.info, 0);
      const int4 *infB = (const int4 *)__shfl_sync(kFull, (unsigned long long)E.info, 16);
      const int loA = __shfl_sync(kFull, E.lo, 0), loB = __shfl_sync(kFull, E.lo, 16);
      const int ta = cand_s[warp][0][g], tb = cand_s[warp][1][g];
      float aba[4] = {0.f, 0.f, 0.f, 0.f}, abb[4] = {0.f, 0.f, 0.f, 0.f};
      float efa = 0.f, efb = 0.f;
      if (ta >= 0) {
        const float4 v = __ldg(abA + loA + ta);
        const int4 inf = __ldg(infA + loA + ta);
        aba[0] = v.x; aba[1] = v.y; aba[2] = v.z; aba[3] = v.w;
        efa = (float)inf.z * (1.f / 256.f);
      }
      if (tb >= 0) {
        const float4 v = __ldg(abB + loB + tb);
        const int4 inf = __ldg(infB + loB + tb);
        abb[0] = v.x; abb[1] = v.y; abb[2] = v.z; abb[3] = v.w;
        efb = (float)inf.z * (1.f / 256.f);
      }
      const float pxa = __shfl_sync(kFull, px, 0), pya = __shfl_sync(kFull, py, 0);
      const float ca = __shfl_sync(kFull, c, 0), sa = __shfl_sync(kFull, s, 0);
      const float pxb = __shfl_sync(kFull, px, 16), pyb = __shfl_sync(kFull, py, 16);
      const float cb = __shfl_sync(kFull, c, 16), sb = __shfl_sync(kFull, s, 16);
      float s_a, s_b;
      mlp_rows_pair(w, q, aba, efa, pxa, pya, ca, sa, abb, efb, pxb, pyb, cb, sb, F.radius, s_a,
                    s_b);
      if (q == 0) {
        score_s[warp][0][g] = ta >= 0 ? s_a + a.b2 : kInf;
        score_s[warp][1][g] = tb >= 0 ? s_b + a.b2 : kInf;
      }
      __syncwarp();
      float bsc[kMaxK];
#pragma unroll
      for (int i = 0; i < kMaxK; ++i) {
        bsc[i] = kInf;
        best[i] = -1;
      }
#pragma unroll
      for (int i = 0; i < kPre; ++i)
        if (cand[i] >= 0) topk_insert<kMaxK>(bsc, best, score_s[warp][half][i], cand[i]);
#pragma unroll
      for (int i = 0; i < kMaxK; ++i)
        if (i >= K) best[i] = -1;
    }
  }  // !CIRC

  // ---- 2. the upper bound: circles of the proposed tiles' obstacles, or of
  // the pose's upper-bound cell ---------------------------------------------
  int ptile[kMaxK];
  int nseg = 0, N = 0;
  float ubp = kInf;
#pragma unroll
  for (int i = 0; i < kMaxK; ++i) ptile[i] = -1;
  if constexpr (CIRC) {
    if (valid) {
      ubp = fminf(circle_ub(cc[0], px, py, F.radius, F.inner),
                  circle_ub(cc[1], px, py, F.radius, F.inner));
      n_circ += (cr[0].y > 0) + (cr[1].y > 0);
    }
  } else {
#pragma unroll
    for (int i = 0; i < kMaxK; ++i) {
      // entry best[i] of the half: lane best % 16, register slot best / 16
      // (a load for entries beyond the kept ones)
      const int b = best[i];
      const int slot = b >= 0 ? b >> 4 : 0;
      int4 kept = slot == 0 ? kinf[0] : kinf[1];
      int4 inf;
      inf.x = __shfl_sync(kFull, kept.x, (half << 4) + (b & 15));
      inf.y = __shfl_sync(kFull, kept.y, (half << 4) + (b & 15));
      inf.w = __shfl_sync(kFull, kept.w, (half << 4) + (b & 15));
      if (b >= 32) inf = __ldg(E.info + E.lo + b);
      ptile[i] = -1;
      if (b >= 0) {
        ptile[i] = inf.w;
        if (hl == 0) {
          sg0[nseg] = inf.x;
          sgt[nseg] = N;
        }
        N += inf.y;
        ++nseg;
      }
    }
    if (hl == 0) sgt[nseg] = N;
    __syncwarp();
    for (int f0 = hl; f0 < N; f0 += 16 * kFilt) {
      float4 cc[kFilt];
#pragma unroll
      for (int q = 0; q < kFilt; ++q) {
        const int f = f0 + 16 * q;
        if (f < N) cc[q] = __ldg(&a.obs[flat_obstacle(sg0, sgt, nseg, f)].circ);
      }
#pragma unroll
      for (int q = 0; q < kFilt; ++q)
        if (f0 + 16 * q < N) {
          ubp = fminf(ubp, circle_ub(cc[q], px, py, F.radius, F.inner));
          ++n_circ;
        }
    }
  }
  const int n_prop = nseg;
  {  // 16-lane minimum (ubp >= 0, so its bits order like the value)
    const unsigned u = __float_as_uint(ubp);
    const unsigned u0 = __reduce_min_sync(kFull, half == 0 ? u : ~0u);
    const unsigned u1 = __reduce_min_sync(kFull, half == 1 ? u : ~0u);
    ubp = __uint_as_float(half ? u1 : u0);
  }
  ubp += a.ub_pad;
  const float thr = ub_value(ubp);
  bool direct = false;
  if constexpr (CIRC) {
    // A pose in its candidate cell whose bound lies within the cell's
    // completeness radius needs only the cell's candidates: every unlisted
    // obstacle is farther than r_foot + UB from it, so it is separated from
    // the footprint by more than UB (with a margin for this test's
    // rounding).  Their circle bounds are tested here, the survivors queued
    // for the first evaluation pass, and the pose takes no tiles.
    direct = cin && crc > (ubp + F.radius) * (1.f + 1e-6f) + 1e-6f;
    bool keep[2];
#pragma unroll
    for (int q = 0; q < 2; ++q)
      keep[q] = direct && cr[q].y > 0 && !(circle_lb_value(cc[q], px, py, F.radius) > thr);
    // a survivor's vertex records on their way first (the evaluation reads
    // them after the next barrier), then its queue slot: the warp's
    // first-candidate survivors in lane order, then its second-candidate
    // ones (the order of a pose's items does not change its outputs)
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (keep[q]) prefetch_lines_l2(a.vtx + 2 * (long long)cr[q].x, 32 * cr[q].y);
    const unsigned b0 = __ballot_sync(kFull, keep[0]), b1 = __ballot_sync(kFull, keep[1]);
    const int tot = __popc(b0) + __popc(b1);
    int base = 0;
    if (lane == 0 && tot > 0) base = atomicAdd(&nq_s, tot);
    base = __shfl_sync(kFull, base, 0);
    const unsigned lt = (1u << lane) - 1u;
    // a queued candidate carries its record in shared memory (the first
    // items of the round's queue: slot d of q_rec, item ~(16 d + pose))
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (keep[q]) {
        const int d = base + (q ? __popc(b0) + __popc(b1 & lt) : __popc(b0 & lt));
        q_rec[d] = cr[q];
        q_s[d] = ~((d << 4) | j);
      }
  }
  // every tile whose bound does not exceed UB lies within cand_radius(UB) of
  // p: the cell's list holds them all while that is within the grid's reach
  // (a pose that takes only its candidates needs no list)
  const bool in_cell = cell >= 0 && !direct && cand_radius(ubp, F.radius) <= a.grid.reach_q;
  Entries E2 = entries_of(a, cell, in_cell);
  if (!valid || direct) E2.hi = E2.lo;
  const bool same = !CIRC && E2.ab == E.ab && E2.lo == E.lo;  // the first entries, in registers
  if (same) E2.hi = E.hi;
  const int nch = (E2.hi - E2.lo + 15) / 16;
  if (hl == 0) {
    pose_s[j] = make_float4(px, py, c, s);
    thr_s[j] = thr;
  }

  // ---- 3-4. rounds of tile tests, circle tests and exact evaluations -------
  // A round collects, for every pose, the passing tiles of its next chunks
  // of 16 entries while they fit its share of the round's segments (16; a
  // chunk never holds more, so every round makes progress), then tests the
  // circles of all collected segments and evaluates the survivors.
  int n_fb = 0;
  int ch = 0;  // this pose's next chunk
  for (;;) {
    {
      int used = 0;  // segments this pose added in this round (uniform over the half)
      for (; ch < nch; ++ch) {
        const int i = E2.lo + ch * 16 + hl;
        bool passing = false, proposed = false;
        int4 inf = make_int4(0, 0, 0, 0);
        float4 ab = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < E2.hi) {
          if (same && ch < 2) {  // the ranking pass's entries, in registers
            ab = ch == 0 ? kab[0] : kab[1];
            inf = ch == 0 ? kinf[0] : kinf[1];
          } else {
            ab = __ldg(E2.ab + i);
            inf = __ldg(E2.info + i);
          }
#pragma unroll
          for (int q = 0; q < kMaxK; ++q) proposed |= ptile[q] == inf.w;
          passing = proposed || !(tile_lb_value(ab, px, py, F.radius) > thr);
          if (inf.w == -2) passing = false;  // a padding slot
        }
        const unsigned m = __ballot_sync(hmask, passing) & hmask;
        if (used + __popc(m) > 16) break;  // the rest next round
        if (i < E2.hi && inf.w != -2) ++n_bound;
        n_fb += __popc(__ballot_sync(hmask, passing && !proposed) & hmask);
        int base = 0;
        if (hl == 0 && m) base = atomicAdd(&nseg_s, __popc(m));
        base = __shfl_sync(hmask, base, half << 4);
        if (passing) {
          const int pos = base + __popc(m & ((1u << lane) - 1u));
          seg_first[pos] = inf.x;
          seg_n[pos] = inf.y;
          seg_pose[pos] = (unsigned char)j;
          // the tile's obstacle records on their way into this SM's L1
          // while the round's tile tests finish

        }
        used += __popc(m);
      }
    }
    const bool more = ch < nch;  // this pose has chunks left for later rounds
    const bool any_more = __syncthreads_or(more);  // a later round follows
    const int nsg = nseg_s;
    // circle tests: 8 threads per segment, kSegsPerPass segments a pass;
    // thread t takes segment t / 8 (+ kSegsPerPass per pass) and, in step b
    // of the pass, its obstacles 64 b + t % 8 + 8 q (q < kFilt), the loads
    // of a step independent; survivors are queued, and the queue is
    // evaluated when the next step could overflow it and at the end
    const int lt = tid & 7;
    int sp = 0, b = 0;  // first segment of the pass, step within the pass
    for (;;) {
      // (a round without segments evaluates the queued candidates only)
      bool done = true;
      if (nsg > 0) {
        const int seg = sp + (tid >> 3);
        const int sn = seg < nsg ? seg_n[seg] : 0;
        const bool has = b * 8 * kFilt < sn;
        bool keep[kFilt];
        int item[kFilt];
#pragma unroll
        for (int q = 0; q < kFilt; ++q) {
          keep[q] = false;
          item[q] = 0;
        }
        if (has) {
          const int sf = seg_first[seg];
          const int jj = seg_pose[seg];
          const float4 q4 = pose_s[jj];
          const float tq = thr_s[jj];
          float4 cq[kFilt];
#pragma unroll
          for (int q = 0; q < kFilt; ++q) {
            const int o = b * 8 * kFilt + lt + 8 * q;
            if (o < sn) cq[q] = __ldg(&a.obs[sf + o].circ);
          }
#pragma unroll
          for (int q = 0; q < kFilt; ++q) {
            const int o = b * 8 * kFilt + lt + 8 * q;
            keep[q] = o < sn && !(circle_lb_value(cq[q], q4.x, q4.y, F.radius) > tq);
            item[q] = ((sf + o) << 4) | jj;
          }
          // a survivor's vertex records on their way into L1 while the
          // queue fills

        }
        {  // the warp's survivors appended with one shared-memory atomic
          int mine = 0;
#pragma unroll
          for (int q = 0; q < kFilt; ++q) mine += keep[q] ? 1 : 0;
          int x = mine;  // inclusive prefix over the warp's lanes
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
          }
          int base = 0;
          if (lane == 31 && x > 0) base = atomicAdd(&nq_s, x);
          base = __shfl_sync(kFull, base, 31) + x - mine;
#pragma unroll
          for (int q = 0; q < kFilt; ++q)
            if (keep[q]) q_s[base++] = item[q];
        }
        // the next step: the next block of this pass's segments, or the next pass
        const bool more_blocks = __syncthreads_or(has && (b + 1) * 8 * kFilt < sn);
        done = false;
        if (more_blocks) {
          ++b;
        } else {
          b = 0;
          sp += kSegsPerPass;
          done = sp >= nsg;
        }
      }
      const int nq = nq_s;
      if (done || nq > kQCap - kCullThreads * kFilt) {
        // the queued items, kItemLanes lanes each (the obstacle's edges
        // shared out, obstacle_value_coop), kGroups items a pass
        const int g = lane % kItemLanes;
        for (int b0 = 0; b0 < nq; b0 += kGroups) {
          const int slot = b0 + tid / kItemLanes;
          const bool live = slot < nq;
          // a warp's slots are consecutive: one without a live item skips
          // the evaluation (it still meets the pass's barrier)
          const bool wlive = b0 + warp * (32 / kItemLanes) < nq;
          const int it = live ? q_s[slot] : 0;
          // a candidate's record is in shared memory, a tile obstacle's in
          // the cull records
          const int iv = it < 0 ? ~it : it;
          const int ij = iv & 15;
          const float4 pq = pose_s[ij];
          int4 rec = make_int4(0, 0, 0, 0);
          if (live) rec = it < 0 ? q_rec[iv >> 4] : __ldg(&a.obs[iv >> 4].rec);
          if constexpr (SOFT) {
            if (wlive) {
              const float v = obstacle_value_coop<M, kItemLanes, true>(
                  F, pq.x, pq.y, pq.z, pq.w, a.vtx + 2 * (long long)rec.x, rec.y, prm.eps_sat,
                  prm.eta, g);
              if (live && g == 0) atomicMin(&key_s[ij], pack_key(v, rec.z));
            }
          } else {
            // the key and the exact detail in one evaluation: the item that
            // holds its pose's minimum after the pass leaves its detail for
            // the epilogue
            float kv = 0.f;
            Active ad;
            if (wlive)
              ad = obstacle_scan_detail_coop<M, kItemLanes>(
                  F, pq.x, pq.y, pq.z, pq.w, a.vtx + 2 * (long long)rec.x, rec.y, rec.z,
                  prm.eps_sat, g, kv);
            const unsigned long long key = pack_key(kv, rec.z);
            if (live && g == 0) {
              atomicMin(&key_s[ij], key);
              prefetch_lines(a.far + rec.x, 4 * rec.y);  // the gradient's far indices
            }
            __syncthreads();  // the pass's minima are in
            if (live && g == 0 && key_s[ij] == key) {
              // this item holds its pose's minimum so far: its detail for
              // the epilogue (a later pass that finds a smaller key
              // overwrites it)
              det_s[ij] = ad;
              drec_s[ij] = rec;
            }
          }
          if (live && g == 0) {
            ++n_obs;
            n_edge += (unsigned)rec.y;
          }
        }
        __syncthreads();  // the queue consumed, every winner's detail in
        if (!done || any_more) {  // the queue fills again
          if (tid == 0) nq_s = 0;
          __syncthreads();
        }
      }
      if (done) break;
    }
    if (!any_more) break;
    if (tid == 0) nseg_s = 0;
    __syncthreads();
  }

  // (the rounds ended on a barrier: every key and winner's output is final)
  if constexpr (SOFT) {
    // ---- 5. soft-minimum epilogues: 8 poses a warp, one lane each ----------
    const int jj = 8 * warp + (lane >> 2);
    const long long pj = (long long)blockIdx.x * kPoses + jj;
    const bool vj = warp < kPoses / 8 && pj < a.P;
    if (vj && (lane & 3) == 0) {
      const float4 q = pose_s[jj];
      const unsigned long long key = key_s[jj];
      const bool none = key == ~0ull;
      ObsRec o{0, 0, 0, 0};
      if (!none) o = a.row_obs[(int)(unsigned)(key & 0xffffffffu)];
      const PoseOut r = epilogue_obstacle<M, true>(F, prm.eps_sat, a.eps_axis, q.x, q.y, q.z,
                                                   q.w, none, o, a.vtx, a.far, want_grad,
                                                   prm.eta);
      write_pose_out(r, pj, a.phi, a.dphi, a.active, nullptr, 0.f);
    }
  } else {
    // ---- 5. hard minimum: the active pairs' gradients by kind class, one
    // class a warp (warp w of each group of four warps takes class w % 4 for
    // the group's 8 poses, one lane a pose: vertex-edge, vertex-robot edge,
    // robot axis, obstacle axis), so that no warp runs two classes'
    // branches one after the other; then each pose's 16 lanes store its
    // saved record, and the CTA its phi, active pairs and pose gradients as
    // three contiguous blocks (few, full transactions also when they live
    // in host memory) ----------------------------------------------------
    const long long pj = (long long)blockIdx.x * kPoses + j;
    {
      const int i = 8 * (warp >> 2) + lane;  // lanes 0-7: the pose this lane may take
      const long long pi = (long long)blockIdx.x * kPoses + i;
      if (lane < 8 && pi < a.P && key_s[i] != ~0ull) {
        const Active ad = det_s[i];
        const int cls = ad.kind == kVertEdge ? 0
                        : ad.kind <= kObsBRobotEdge ? 1
                        : ad.kind <= kRAxisRMaxB ? 2 : 3;
        if (cls == (warp & 3)) {
          const int4 rec = drec_s[i];
          const float4 pq = pose_s[i];
          float *o = out_s[i];
          o[0] = ad.separated ? sqrtf(ad.val) : ad.val;
          o[1] = __uint_as_float(ad.pid);
          Grad rows;
          rows.nrow = -1;
          if (want_grad && (ad.separated || ad.dlt > 0.f))
            rows = active_grad<M>(F, pq.x, pq.y, pq.z, pq.w, a.vtx + 2 * (long long)rec.x,
                                  a.far + rec.x, rec.y, rec.z, ad.kind, ad.l, ad.k, ad.t,
                                  a.eps_axis);
          saved_words(rows, &o[kOutSaved]);
        }
      }
    }
    __syncthreads();
    if (valid && save) reinterpret_cast<float *>(a.saved)[16 * pj + hl] = out_s[j][kOutSaved + hl];
    const long long p0 = (long long)blockIdx.x * kPoses;
    const int np = (int)(a.P - p0 < kPoses ? a.P - p0 : kPoses);
    if (warp == 0 && lane < np && a.phi) a.phi[p0 + lane] = out_s[lane][0];
    if (warp == 1 && lane < np && a.active) a.active[p0 + lane] = __float_as_uint(out_s[lane][1]);
    if (warp >= 2 && a.dphi) {
      const int i = (warp - 2) * 32 + lane;
      if (i < 3 * np) a.dphi[3 * p0 + i] = out_s[i / 3][kOutSaved + i % 3];
    }
  }
  // ---- counters, after the outputs: each warp adds its sums to the CTA's
  // words ------------------------------------------------------------------
  unsigned cnt[kStCount];
  cnt[kStProp] = (valid && hl == 0) ? (unsigned)n_prop : 0u;
  cnt[kStFb] = (valid && hl == 0) ? (unsigned)n_fb : 0u;
  cnt[kStFbPoses] = (valid && hl == 0 && n_fb > 0) ? 1u : 0u;
  cnt[kStBound] = n_bound;
  cnt[kStCirc] = n_circ;
  cnt[kStObs] = n_obs;
  cnt[kStEdges] = n_edge;
  {  // the warp's sums, then lane k adds sum k (one atomic instruction)
    unsigned mine = 0u;
#pragma unroll
    for (int k = 0; k < kStCount; ++k) {
      const unsigned t = __reduce_add_sync(kFull, cnt[k]);
      mine = lane == k ? t : mine;
    }
    if (lane < kStCount && mine)
      atomicAdd(&a.ws[kStatBase + (long long)blockIdx.x * kStatWords + lane],
                (unsigned long long)mine);
  }
  if (blockIdx.x == 0 && tid == 0) {
    a.ws[0] = gridDim.x;
    a.ws[1] = 0ull;  // the cull has no device-side wait
  }
}

// ---------------------------------------------------------------------------
// helper outputs: per-tile values, bounds, features, network scores
// ---------------------------------------------------------------------------
template <int M>
__global__ void tile_values_kernel(FootprintK F, ParamsK prm, const float *__restrict__ poses,
                                   long long P, const TileHdr *__restrict__ tiles, int n_tiles,
                                   const unsigned char *__restrict__ blob, float *__restrict__ out)
{
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (p >= P) return;
  const float px = poses[3 * p], py = poses[3 * p + 1];
  float s, c;
  sincosf(poses[3 * p + 2], &s, &c);
  const TileHdr h = tiles[t];
  const unsigned char *tb = blob + h.blob_off;
  const int4 *ob = reinterpret_cast<const int4 *>(tb);
  const float4 *vt = reinterpret_cast<const float4 *>(tb + 16 * h.n_obs);
  float best = kInf;
  for (int o = 0; o < h.n_obs; ++o) {
    const int4 rec = ob[o];
    best = fminf(best, obstacle_value<M>(F, px, py, c, s, vt + 2 * rec.x, rec.y, prm.eps_sat));
  }
  out[p * n_tiles + t] = best > 0.f ? sqrtf(best) : best;
}

__global__ void tile_lb_kernel(const float *__restrict__ poses, long long P,
                               const TileHdr *__restrict__ tiles, int n_tiles, float rfoot,
                               float *__restrict__ out)
{
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * n_tiles) return;
  const long long p = i / n_tiles;
  const int t = (int)(i % n_tiles);
  out[i] = tile_lb(tiles[t].aabb, poses[3 * p], poses[3 * p + 1], rfoot);
}

__global__ void tile_features_kernel(const float *__restrict__ poses, long long P,
                                     const TileHdr *__restrict__ tiles, int n_tiles,
                                     float rfoot, float *__restrict__ out)
{
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * n_tiles) return;
  const long long p = i / n_tiles;
  const int t = (int)(i % n_tiles);
  const float px = poses[3 * p], py = poses[3 * p + 1];
  float s, c;
  sincosf(poses[3 * p + 2], &s, &c);
  const TileHdr h = tiles[t];
  float *o = out + i * 16;
  for (int q = 0; q < 4; ++q) {
    feat_corner(h.aabb, q, px, py, c, s, o[2 * q], o[2 * q + 1]);
    feat_rest(h.aabb, q, px, py, rfoot, (float)h.n_vtx * (1.f / 256.f), o[8 + 2 * q],
              o[9 + 2 * q]);
  }
}

// one warp = 16 poses (two per quad) x every tile
__global__ void mlp_scores_kernel(const float *__restrict__ poses, long long P,
                                  const TileHdr *__restrict__ tiles, int n_tiles, float rfoot,
                                  const uint32_t *__restrict__ frag, float b2,
                                  float *__restrict__ out)
{
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int g = lane >> 2, q = lane & 3;
  const long long pa = gw * 16 + g, pb = gw * 16 + g + 8;
  if (gw * 16 >= P) return;
  float pxa = 0.f, pya = 0.f, ca = 1.f, sa = 0.f, pxb = 0.f, pyb = 0.f, cb = 1.f, sb = 0.f;
  if (pa < P) {
    pxa = poses[3 * pa];
    pya = poses[3 * pa + 1];
    sincosf(poses[3 * pa + 2], &sa, &ca);
  }
  if (pb < P) {
    pxb = poses[3 * pb];
    pyb = poses[3 * pb + 1];
    sincosf(poses[3 * pb + 2], &sb, &cb);
  }
  MlpFrags w;
  load_frags(frag, lane, w);
  for (int t = 0; t < n_tiles; ++t) {
    const TileHdr h = tiles[t];
    float s_a, s_b;
    mlp_rows(w, h.aabb, q, pxa, pya, ca, sa, pxb, pyb, cb, sb, rfoot,
             (float)h.n_vtx * (1.f / 256.f), s_a, s_b);
    if (q == 0) {
      if (pa < P) out[pa * n_tiles + t] = s_a + b2;
      if (pb < P) out[pb * n_tiles + t] = s_b + b2;
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Cull workspace: a 256-byte header {CTAs of the last launch, error word},
// then kStatWords counters per CTA (written, never accumulated: nothing to
// clear before a launch).
static size_t cull_workspace_bytes(long long P)
{
  const long long ctas = (std::max<long long>(P, 0) + kMinPoses - 1) / kMinPoses;
  return 8 * (size_t)kStatBase + 8 * (size_t)kStatWords * (size_t)std::max<long long>(ctas, 1);
}

template <int M>
struct CullCall {
  static int run(const FootprintK &F, const ParamsK &pk, const CullArgs &a, int prop, dim3 grid,
                 cudaStream_t st)
  {
    const bool soft = pk.eta > 0.f;
    auto kern = prop == kPropNet
                    ? (soft ? cull_kernel<M, kPropNet, true> : cull_kernel<M, kPropNet, false>)
                : prop == kPropCircles
                    ? (soft ? cull_kernel<M, kPropCircles, true>
                            : cull_kernel<M, kPropCircles, false>)
                    : (soft ? cull_kernel<M, kPropBound, true> : cull_kernel<M, kPropBound, false>);
    const int threads = prop == kPropCircles ? ShapeOf<kPropCircles>::kThreads
                                             : ShapeOf<kPropBound>::kThreads;
    kern<<<grid, threads, 0, st>>>(F, pk, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch (cull)");
  }
};

template <int M>
struct TileValuesCall {
  static int run(const FootprintK &F, const ParamsK &pk, const float *poses, long long P,
                 const psdf_scene *sc, float *out, cudaStream_t st)
  {
    dim3 grid((unsigned)((P + 127) / 128), (unsigned)sc->n_tiles);
    tile_values_kernel<M><<<grid, 128, 0, st>>>(F, pk, poses, P, sc->d_tiles, sc->n_tiles,
                                                sc->d_blob, out);
    return PSDF_OK;
  }
};

template <template <int> class Fn, class... Args>
static int dispatch_m_cull(int m, Args &&...args)
{
  switch (m) {
    case 3: return Fn<3>::run(args...);
    case 4: return Fn<4>::run(args...);
    case 5: return Fn<5>::run(args...);
    case 6: return Fn<6>::run(args...);
    case 7: return Fn<7>::run(args...);
    case 8: return Fn<8>::run(args...);
    case 9: return Fn<9>::run(args...);
    case 10: return Fn<10>::run(args...);
    case 11: return Fn<11>::run(args...);
    case 12: return Fn<12>::run(args...);
    case 13: return Fn<13>::run(args...);
    case 14: return Fn<14>::run(args...);
    case 15: return Fn<15>::run(args...);
    case 16: return Fn<16>::run(args...);
    default: return fail(PSDF_ERR_FOOTPRINT, "unsupported footprint size");
  }
}

static int check_out(const void *p, int64_t P, const char *name)
{
  if (P > 0 && !p) return fail(PSDF_ERR_ARG, std::string(name) + " is NULL");
  return PSDF_OK;
}

}  // namespace psdf

using namespace psdf;

extern "C" int psdf_mlp_create(const float *W1, const float *w2, float b2, psdf_mlp **out)
{
  if (!W1 || !w2 || !out) return fail(PSDF_ERR_ARG, "NULL argument");
  *out = nullptr;
  for (int i = 0; i < PSDF_MLP_HIDDEN * PSDF_MLP_IN; ++i)
    if (!std::isfinite(W1[i])) return fail(PSDF_ERR_ARG, "non-finite weight");
  for (int i = 0; i < PSDF_MLP_HIDDEN; ++i)
    if (!std::isfinite(w2[i])) return fail(PSDF_ERR_ARG, "non-finite weight");
  if (!std::isfinite(b2)) return fail(PSDF_ERR_ARG, "non-finite weight");
  auto h = [](float x) { return (uint32_t)__half_as_ushort(__float2half_rn(x)); };
  auto pk = [&](float lo, float hi) { return h(lo) | (h(hi) << 16); };
  std::vector<uint32_t> frag(kFrag1Words + kFrag2Words, 0u);
  for (int j = 0; j < 8; ++j)
    for (int lane = 0; lane < 32; ++lane) {
      const int g = lane >> 2, t = lane & 3, n = 8 * j + g;
      frag[(j * 32 + lane) * 2] = pk(W1[n * 16 + 2 * t], W1[n * 16 + 2 * t + 1]);
      frag[(j * 32 + lane) * 2 + 1] = pk(W1[n * 16 + 2 * t + 8], W1[n * 16 + 2 * t + 9]);
    }
  for (int s2 = 0; s2 < 4; ++s2)
    for (int lane = 0; lane < 32; ++lane) {
      const int g = lane >> 2, t = lane & 3;
      if (g != 0) continue;  // only output column 0 is used
      const int k = 16 * s2 + 2 * t;
      frag[kFrag1Words + (s2 * 32 + lane) * 2] = pk(w2[k], w2[k + 1]);
      frag[kFrag1Words + (s2 * 32 + lane) * 2 + 1] = pk(w2[k + 8], w2[k + 9]);
    }
  psdf_mlp *m = new psdf_mlp();
  m->b2 = b2;
  cudaGetDevice(&m->device);
  cudaError_t e = cudaMalloc(&m->d_frag, frag.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(m->d_frag, frag.data(), frag.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(m->d_frag);
    delete m;
    return cuda_fail(e, "psdf_mlp_create");
  }
  *out = m;
  return PSDF_OK;
}

extern "C" int psdf_mlp_destroy(psdf_mlp *mlp)
{
  if (mlp) {
    cudaFree(mlp->d_frag);
    delete mlp;
  }
  return PSDF_OK;
}

extern "C" size_t psdf_cull_workspace_bytes(int64_t P, const psdf_scene *scene)
{
  (void)scene;
  return cull_workspace_bytes(P);
}

extern "C" int psdf_tile_features(const float *footprint, int32_t m, const psdf_scene *scene,
                                  const float *poses, int64_t P, float *features, void *stream)
{
  psdf_params prm{scene ? scene->eps_seg : 0.f, scene ? scene->eps_axis : 0.f, 0.f, 0.f};
  int rc = check_eval_args(scene, poses, P, &prm, (void *)256, (size_t)-1);
  if (!rc) rc = check_out(features, P, "features");
  FootprintK F;
  if (!rc) rc = make_footprint(footprint, m, scene->eps_seg, &F);
  if (rc) return rc;
  const long long n = P * (long long)scene->n_tiles;
  if (n == 0) return PSDF_OK;
  tile_features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      poses, P, scene->d_tiles, scene->n_tiles, F.radius, features);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch");
}

extern "C" int psdf_tile_lower_bounds(const float *footprint, int32_t m, const psdf_scene *scene,
                                      const float *poses, int64_t P, float *lb, void *stream)
{
  psdf_params prm{scene ? scene->eps_seg : 0.f, scene ? scene->eps_axis : 0.f, 0.f, 0.f};
  int rc = check_eval_args(scene, poses, P, &prm, (void *)256, (size_t)-1);
  if (!rc) rc = check_out(lb, P, "lb");
  FootprintK F;
  if (!rc) rc = make_footprint(footprint, m, scene->eps_seg, &F);
  if (rc) return rc;
  const long long n = P * (long long)scene->n_tiles;
  if (n == 0) return PSDF_OK;
  tile_lb_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      poses, P, scene->d_tiles, scene->n_tiles, F.radius, lb);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch");
}

extern "C" int psdf_mlp_scores(const psdf_mlp *mlp, const float *footprint, int32_t m,
                               const psdf_scene *scene, const float *poses, int64_t P,
                               float *scores, void *stream)
{
  if (!mlp) return fail(PSDF_ERR_ARG, "mlp is NULL");
  psdf_params prm{scene ? scene->eps_seg : 0.f, scene ? scene->eps_axis : 0.f, 0.f, 0.f};
  int rc = check_eval_args(scene, poses, P, &prm, (void *)256, (size_t)-1);
  if (!rc) rc = check_out(scores, P, "scores");
  FootprintK F;
  if (!rc) rc = make_footprint(footprint, m, scene->eps_seg, &F);
  if (rc) return rc;
  if (P == 0 || scene->n_tiles == 0) return PSDF_OK;
  const long long warps = (P + 15) / 16;
  mlp_scores_kernel<<<(unsigned)((warps + 3) / 4), 128, 0, (cudaStream_t)stream>>>(
      poses, P, scene->d_tiles, scene->n_tiles, F.radius, mlp->d_frag, mlp->b2, scores);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch");
}

extern "C" int psdf_tile_values(const float *footprint, int32_t m, const psdf_scene *scene,
                                const float *poses, int64_t P, const psdf_params *params,
                                float *values, void *stream)
{
  int rc = check_eval_args(scene, poses, P, params, (void *)256, (size_t)-1);
  if (!rc) rc = check_out(values, P, "values");
  FootprintK F;
  if (!rc) rc = make_footprint(footprint, m, scene->eps_seg, &F);
  if (rc) return rc;
  if (P == 0 || scene->n_tiles == 0) return PSDF_OK;
  if (scene->n_tiles > 65535) return fail(PSDF_ERR_CAPACITY, "more than 65535 tiles");
  if (params->eta > 0.f)
    return fail(PSDF_ERR_ARG, "tile values use the hard minimum only (eta must be 0)");
  ParamsK pk{params->eps_sat, params->eta};
  rc = dispatch_m_cull<TileValuesCall>(m, F, pk, poses, (long long)P, scene, values,
                                       (cudaStream_t)stream);
  if (rc) return rc;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch");
}

static int eval_culled(const float *footprint, int32_t m, const psdf_scene *scene,
                       const psdf_mlp *mlp, const psdf_cull_opts *opts, const float *poses,
                       int64_t P, const psdf_params *params, float *phi, float *dphi,
                       uint32_t *active, float4 *saved, void *workspace, size_t workspace_bytes,
                       void *stream)
{
  int rc = check_eval_args(scene, poses, P, params, workspace ? workspace : (void *)256,
                           (size_t)-1);
  if (rc) return rc;
  if (!opts) return fail(PSDF_ERR_ARG, "opts is NULL");
  if (opts->k < 1 || opts->k > kMaxK) return fail(PSDF_ERR_ARG, "k must be in [1, 4]");
  if (opts->mode != PSDF_PROPOSE_BOUND && opts->mode != PSDF_PROPOSE_MLP &&
      opts->mode != PSDF_PROPOSE_CIRCLES)
    return fail(PSDF_ERR_ARG, "unknown proposal mode");
  if (opts->mode == PSDF_PROPOSE_MLP && !mlp) return fail(PSDF_ERR_ARG, "mlp is NULL");
  if ((rc = check_out(phi, P, "phi"))) return rc;
  FootprintK F;
  rc = make_footprint(footprint, m, scene->eps_seg, &F);
  if (rc) return rc;
  if (!workspace) return fail(PSDF_ERR_ARG, "workspace is NULL");
  if (((uintptr_t)workspace & 255u) != 0) return fail(PSDF_ERR_ARG, "workspace must be 256-byte aligned");
  if (workspace_bytes < cull_workspace_bytes(P))
    return fail(PSDF_ERR_CAPACITY, "workspace smaller than psdf_cull_workspace_bytes");
  if (P > (1LL << 31) - 1) return fail(PSDF_ERR_CAPACITY, "P too large for the cull");
  if (scene->n_tiles > kMaxScanTiles) return fail(PSDF_ERR_CAPACITY, "too many tiles for the cull");
  if (scene->M >= (1 << 26)) return fail(PSDF_ERR_CAPACITY, "too many obstacles for the cull");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long *ws = reinterpret_cast<unsigned long long *>(workspace);
  if (P == 0) {  // no launch: the counters read as zero
    cudaError_t e = cudaMemsetAsync(ws, 0, kStatBase * 8, st);
    return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "cudaMemsetAsync(cull counters)");
  }
  const bool net = opts->mode == PSDF_PROPOSE_MLP;
  const int prop = net ? kPropNet : opts->mode == PSDF_PROPOSE_CIRCLES ? kPropCircles : kPropBound;
  CullArgs a;
  std::memset(&a, 0, sizeof(a));
  a.poses = poses;
  a.P = P;
  a.grid = scene->grid;
  a.cand = scene->cand;
  a.tile_ab = scene->d_tile_ab;
  a.tile_info = scene->d_tile_info;
  a.T = scene->n_tiles;
  a.K = opts->k;
  a.obs = scene->d_cull_obs;
  a.vtx = scene->d_vtx;
  a.far = scene->d_far;
  a.row_obs = scene->d_row_obs;
  // soft minimum: an obstacle's value lies below its hard distance when it
  // is separated and at most log(K) / eta (K axes) when it penetrates, so
  // the upper bound taken from distances is raised by that much
  a.ub_pad = 0.f;
  if (params->eta > 0.f)
    a.ub_pad = (float)(std::log((double)(m + scene->max_obs_edges)) / params->eta * (1.0 + 1e-5) +
                       1e-6);
  a.eps_axis = scene->eps_axis;
  a.frag = net ? mlp->d_frag : nullptr;
  a.b2 = net ? mlp->b2 : 0.f;
  a.phi = phi;
  a.dphi = dphi;
  a.active = active;
  a.saved = saved;
  a.ws = ws;
  const int cta_poses = prop == kPropCircles ? ShapeOf<kPropCircles>::kPoses
                                             : ShapeOf<kPropBound>::kPoses;
  const long long grid = (P + cta_poses - 1) / cta_poses;
  // the scene into L2 when the launch reads a good part of it and it fits
  // well within L2 (a few poses on a huge scene read only what they need).
  // Not for the candidate grid: a pose there reads its cell's candidates and
  // its survivors' vertex records, a small part of the scene, and measured
  // faster without the prefetch traffic in front of those reads.
  if (prop != kPropCircles) {
    const size_t scene_bytes = 32 * (size_t)scene->M + 36 * (size_t)scene->n_edges +
                               16 * (size_t)scene->rows_total +
                               32 * (size_t)scene->grid_entries + 32 * (size_t)scene->n_tiles;
    if (P >= 64 && scene_bytes <= (32u << 20)) {
      auto add = [&](const void *ptr, size_t bytes) {
        bytes &= ~(size_t)15;
        if (!ptr || bytes == 0 || a.pf.n >= kMaxPrefetch) return;
        a.pf.ptr[a.pf.n] = reinterpret_cast<const unsigned char *>(ptr);
        a.pf.bytes[a.pf.n] = (long long)bytes;
        a.pf.first[a.pf.n + 1] =
            a.pf.first[a.pf.n] + ((long long)bytes + kPrefetchChunk - 1) / kPrefetchChunk;
        ++a.pf.n;
      };
      if (scene->grid.nx > 0 && scene->grid.cap > 0) {
        const size_t slots = (size_t)scene->grid.nx * scene->grid.ny * scene->grid.cap;
        add(scene->d_cell_fab, 16 * slots);
        add(scene->d_cell_finfo, 16 * slots);
      } else if (scene->grid.nx > 0) {
        add(scene->d_cell_off, 4 * ((size_t)scene->grid.nx * scene->grid.ny + 1));
        add(scene->d_cell_aabbs, 16 * (size_t)scene->grid_entries);
        add(scene->d_cell_info, 16 * (size_t)scene->grid_entries);
      } else {
        add(scene->d_tile_ab, 16 * (size_t)scene->n_tiles);
        add(scene->d_tile_info, 16 * (size_t)scene->n_tiles);
      }
      add(scene->d_cull_obs, sizeof(CullObs) * (size_t)scene->M);
      add(scene->d_vtx, 32 * (size_t)scene->n_edges);
      add(scene->d_far, 4 * (size_t)scene->n_edges);
      // the caller rows' records: only the soft minimum's epilogue reads them
      if (params->eta > 0.f) add(scene->d_row_obs, sizeof(ObsRec) * (size_t)scene->rows_total);
    }
  }
  ParamsK pk{params->eps_sat, params->eta};
  ProfileScope prof("cull", st);
  return dispatch_m_cull<CullCall>(m, F, pk, a, prop, dim3((unsigned)grid), st);
}

extern "C" int psdf_eval_culled(const float *footprint, int32_t m, const psdf_scene *scene,
                                const psdf_mlp *mlp, const psdf_cull_opts *opts,
                                const float *poses, int64_t P, const psdf_params *params,
                                float *phi, float *dphi, uint32_t *active, void *workspace,
                                size_t workspace_bytes, void *stream)
{
  return eval_culled(footprint, m, scene, mlp, opts, poses, P, params, phi, dphi, active, nullptr,
                     workspace, workspace_bytes, stream);
}

extern "C" int psdf_eval_culled_save(const float *footprint, int32_t m,
                                     const psdf_scene *scene, const psdf_mlp *mlp,
                                     const psdf_cull_opts *opts, const float *poses, int64_t P,
                                     const psdf_params *params, float *phi, float *dphi,
                                     uint32_t *active, float *saved, void *workspace,
                                     size_t workspace_bytes, void *stream)
{
  if (P > 0 && !saved) return fail(PSDF_ERR_ARG, "saved is NULL");
  if (params && params->eta > 0.f)
    return fail(PSDF_ERR_ARG, "saved backward records need the hard minimum (eta <= 0)");
  if (((uintptr_t)saved & 15u) != 0) return fail(PSDF_ERR_ARG, "saved must be 16-byte aligned");
  return eval_culled(footprint, m, scene, mlp, opts, poses, P, params, phi, dphi, active,
                     reinterpret_cast<float4 *>(saved), workspace, workspace_bytes, stream);
}

extern "C" int psdf_cull_stats_read(const void *workspace, void *stream, psdf_cull_stats *stats)
{
  if (!workspace || !stats) return fail(PSDF_ERR_ARG, "NULL argument");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  unsigned long long hdr[2];
  e = cudaMemcpy(hdr, workspace, sizeof(hdr), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(cull counters)");
  std::vector<unsigned long long> w((size_t)hdr[0] * kStatWords);
  if (!w.empty()) {
    e = cudaMemcpy(w.data(), reinterpret_cast<const unsigned long long *>(workspace) + kStatBase,
                   w.size() * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(cull counters)");
  }
  unsigned long long sum[kStatWords] = {};
  for (size_t b = 0; b < (size_t)hdr[0]; ++b)
    for (int k = 0; k < kStatWords; ++k) sum[k] += w[b * kStatWords + k];
  stats->evaluated_obstacles = (int64_t)sum[kStObs];
  stats->evaluated_edges = (int64_t)sum[kStEdges];
  stats->proposed_items = (int64_t)sum[kStProp];
  stats->fallback_items = (int64_t)sum[kStFb];
  stats->fallback_poses = (int64_t)sum[kStFbPoses];
  stats->bound_evaluations = (int64_t)sum[kStBound];
  stats->circle_evaluations = (int64_t)sum[kStCirc];
  if (hdr[1]) return fail(PSDF_ERR_TIMEOUT, "a bounded device-side wait ran out");
  return PSDF_OK;
}
