// Exact tile cull with a proposal (psdf_eval_culled and its helpers).
//
// Work is organised as (pose, tile) pairs, bucketed by tile:
//   0. clear_words     per-tile counters and the pipeline counters cleared
//   1. propose         16 lanes per pose rank the tiles of the pose's cell in a
//                      uniform grid (every tile within one cell size; all
//                      tiles for a pose outside the grid) by the conservative
//                      bound; the pose keeps its K best, or its 8 best
//                      re-ranked by the tile-proposal network on tensor cores
//                      (K best kept).  From the circles of the proposed tiles'
//                      obstacles the lanes take an upper bound UB on phi and
//                      list the pose for the proposed tiles and for every other
//                      tile whose lower bound does not exceed UB (the cell's
//                      list holds them all when UB's reach is within the
//                      cell's; else every tile is tested)
//   2. eval_lists      two CTAs per tile, launched as the proposals start:
//                      the tile's blob staged in shared memory, then the
//                      tile's lanes = (pose, obstacle range) pairs in units of
//                      128 so that warps stay full; an obstacle whose circle
//                      bound exceeds the pose's upper bound is skipped, the
//                      others are evaluated exactly; one atomicMin per
//                      evaluated obstacle into the pose's 64-bit key
//   3. epilogue        as for the full scan
// Every tile holding a value at or below phi has a lower bound <= phi <= UB,
// so it is listed; every obstacle skipped has a value above the threshold,
// which is never below phi.  The minimum over 64-bit keys does not depend on
// evaluation order, so the result equals the full scan's bit for bit.
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
constexpr int kPoseThreads = 128;  // 4 warps x 2 poses per propose / fallback CTA
constexpr int kKeep = 2;  // cell entries a propose lane keeps from its ranking pass
constexpr int kListThreads = 128;  // threads of an eval_lists CTA
constexpr int kMaxScanTiles = 1024 * 64;

// counters at the start of the workspace
// Pipeline counters, each spread over kCtrSlots words (CTA b adds to slot
// b % kCtrSlots, so that a few thousand CTAs do not queue on one address);
// psdf_cull_stats_read sums the slots.
constexpr int kCtrSlots = 16;
struct CullCounters {
  int err;
  int pad;
  unsigned long long n_prop[kCtrSlots];       // proposed (pose, tile) pairs
  unsigned long long n_fb[kCtrSlots];         // (pose, tile) pairs added by the bound check
  unsigned long long fallback_poses[kCtrSlots];  // poses with at least one such pair
  unsigned long long n_obs_eval[kCtrSlots];   // obstacles evaluated exactly
  unsigned long long n_edge_eval[kCtrSlots];  // edges of those obstacles
  unsigned long long n_bound[kCtrSlots];      // tile bounds the proposals computed
  unsigned long long n_circ[kCtrSlots];       // obstacle circles of the proposals' upper bounds
};

struct CullLayout {
  size_t hist, clear_bytes, keys, pose4, ub, prop, list, total;
};

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Per-tile pose lists have a fixed capacity of P entries (list[t * P + i]).
// The counters and the per-tile histogram are contiguous (cleared by one kernel).
static CullLayout cull_layout(long long P, int n_tiles)
{
  CullLayout L;
  const size_t Pz = (size_t)std::max<long long>(P, 1);
  const size_t Tz = (size_t)std::max(n_tiles, 1);
  size_t o = align256(sizeof(CullCounters));
  L.hist = o; o = align256(o + 4 * Tz);
  L.clear_bytes = o;
  L.keys = o; o = align256(o + 8 * Pz);
  L.pose4 = o; o = align256(o + 16 * Pz);
  L.ub = o; o = align256(o + 4 * Pz);
  L.prop = o; o = align256(o + 4 * Pz * kMaxK);
  L.list = o; o = align256(o + 4 * Pz * Tz);
  L.total = o;
  return L;
}

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

// ---------------------------------------------------------------------------
// per-tile work units
// ---------------------------------------------------------------------------
// Lanes of a tile's work: its cnt poses are split over S obstacle ranges
// each, so that cnt * S lanes fill about two 128-thread units (one per CTA of
// the tile) when few poses need the tile (short per-lane chains, many warps
// in flight).
constexpr int kTargetLanes = 2 * kListThreads;
__device__ __forceinline__ int tile_split(int cnt, int n_obs)
{
  return max(1, min(kTargetLanes / max(cnt, 1), n_obs));
}

__device__ __forceinline__ int tile_units(int cnt, int n_obs)
{
  return cnt == 0 ? 0 : (int)(((long long)cnt * tile_split(cnt, n_obs) + kListThreads - 1) / kListThreads);
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

// Zeroes the counters and per-tile counts of a cull workspace; the proposal
// kernel, launched after it with programmatic stream serialization, ranks
// its tiles meanwhile and waits for it before its first append.
__global__ void clear_words(unsigned *__restrict__ w, int n)
{
  pdl_trigger();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    w[i] = 0u;
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

// One warp = 2 poses, 16 lanes each (lanes 0-15 pose a, 16-31 pose b).  The
// tiles a pose looks at are its grid cell's list (every tile within one
// cell size of the pose), else all tiles; lane hl takes entries hl, hl + 16,
// ... and keeps its RL best bounds.  R rounds of a 16-lane argmin over the
// lanes' heads give the pose's R smallest (bound, tile) pairs in order,
// written to cand[r] (uniform over the pose's 16 lanes).  With NET the 16
// rows (2 poses x kPre candidates) are scored by the network and the pose
// keeps its K best scores; else its K best bounds.  Lane 0 of each pose
// appends the pose to its proposed tiles.  The pose's 16 lanes then take an
// upper bound on phi from the circles of the proposed tiles' obstacles, and
// append the pose to every other tile whose bound does not exceed it: from
// the cell's list when the bound's reach is within the grid's, else from
// all tiles.
template <int K, bool NET>
__global__ void __launch_bounds__(kPoseThreads)
    propose(const float *__restrict__ poses, long long P, const TileHdr *__restrict__ tiles,
            int T, const CullGrid grid, float rfoot, float rin, float ub_pad,
            const unsigned char *__restrict__ blob,
            const uint32_t *__restrict__ frag, float b2, unsigned long long *__restrict__ keys,
            float4 *__restrict__ pose4, float *__restrict__ ub_out, int *__restrict__ prop,
            int *hist, int *__restrict__ list,
            CullCounters *ctr)
{
  constexpr int R = NET ? kPre : K;  // candidates merged per pose
  constexpr int RL = NET ? 4 : K;    // best tiles each lane keeps
  __shared__ int ct_s[kPoseThreads / 32][2][kPre];
  __shared__ float sc_s[kPoseThreads / 32][2][kPre];
  __shared__ int s_prop, s_fb, s_fbp;
  __shared__ unsigned s_bound, s_circ;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long pw = ((long long)blockIdx.x * (kPoseThreads / 32) + warp) * 2;
  const int half = lane >> 4, hl = lane & 15;
  const long long p = pw + half;
  const bool valid = p < P;
  // the evaluation kernel may launch at once: its CTAs stage their tiles
  // while the proposals run, and wait for this grid before reading its lists
  pdl_trigger();
  if (threadIdx.x == 0) s_prop = s_fb = s_fbp = s_bound = s_circ = 0;
  unsigned n_bound = 0, n_circ = 0;  // this lane's tile bounds and circles
  float px = 0.f, py = 0.f, s = 0.f, c = 1.f;
  int e0 = 0, e1 = 0;  // the cell's list, or all tiles (cell < 0)
  int cell = -1;
  MlpFrags w;  // the network's weights (pose-invariant: read first)
  if constexpr (NET) load_frags(frag, lane, w);
  if (valid) {
    px = poses[3 * p];
    py = poses[3 * p + 1];
    sincosf(poses[3 * p + 2], &s, &c);
    cell = grid_cell(grid, px, py);
    if (cell >= 0) {
      e0 = __ldg(grid.off + cell);
      e1 = __ldg(grid.off + cell + 1);
    }
    if (hl == 0) {
      keys[p] = ~0ull;
      pose4[p] = make_float4(px, py, c, s);
    }
  }
  float sc[RL];
  int id[RL];
#pragma unroll
  for (int i = 0; i < RL; ++i) {
    sc[i] = kInf;
    id[i] = -1;
  }
  // entries i of the cell's list (tile grid.tl[i], its AABB grid.ab[i]) or
  // tiles i; a lane's first kKeep cell entries stay in registers for the
  // candidate pass below
  const int lo = (cell >= 0 ? e0 : 0) + hl, hi = valid ? (cell >= 0 ? e1 : T) : 0;
  int kt[kKeep];
  float kd2[kKeep];
  int i = lo;
#pragma unroll
  for (int q = 0; q < kKeep; ++q, i += 16) {
    kt[q] = -1;
    kd2[q] = kInf;
    if (i < hi) {
      const int t = cell >= 0 ? __ldg(grid.tl + i) : i;
      const float d2 = aabb_d2(cell >= 0 ? __ldg(grid.ab + i) : tile_aabb(tiles, t), px, py);
      topk_insert<RL>(sc, id, d2, t);
      kt[q] = t;
      kd2[q] = d2;
      ++n_bound;
    }
  }
  for (; i < hi; i += 16) {
    const int t = cell >= 0 ? __ldg(grid.tl + i) : i;
    topk_insert<RL>(sc, id, aabb_d2(cell >= 0 ? __ldg(grid.ab + i) : tile_aabb(tiles, t), px, py), t);
    ++n_bound;
  }
  __syncthreads();  // s_prop, s_fb, s_fbp initialised
  int best[K];
#pragma unroll
  for (int i = 0; i < K; ++i) best[i] = -1;
  float ubp = kInf;  // upper bound (metres) on the pose's phi
  if (pw < P) {  // uniform over the warp
    // R rounds of a 16-lane minimum over the lanes' heads, as 32-bit keys
    // (the top 16 bits of the squared distance -- not negative, so its bits
    // order like the value, to 1/128 -- over the tile's 16 bits; a tile sits
    // in one lane only, so the lane whose head won pops it).  A lane keeps
    // only its RL best, so with the network the 8 candidates are the 8
    // smallest bounds it looked at unless one lane held more than RL of them.
    int cand[R];
    int head = 0;
    // tile headers of the candidates {blob_off, blob_bytes, n_obs, n_vtx}:
    // with the network lane 4 g holds candidate g's of pose a (hda) and of
    // pose b (hdb); without it lane r of a pose's half holds candidate r's
    int4 hda = make_int4(0, 0, 0, 0), hdb = hda;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      unsigned mine = ~0u;
#pragma unroll
      for (int i = 0; i < RL; ++i)
        if (i == head && id[i] >= 0) mine = (__float_as_uint(sc[i]) & 0xffff0000u) | (unsigned)id[i];
      const unsigned k0 = __reduce_min_sync(0xffffffffu, half == 0 ? mine : ~0u);
      const unsigned k1 = __reduce_min_sync(0xffffffffu, half == 1 ? mine : ~0u);
      const unsigned key = half ? k1 : k0;
      const bool any = key != ~0u;
      cand[r] = any ? (int)(key & 0xffffu) : -1;
      if (any && key == mine) ++head;
    }
    if constexpr (NET) {
      if (hl == 0)
#pragma unroll
        for (int r = 0; r < kPre; ++r) ct_s[warp][half][r] = cand[r];
      __syncwarp();
      const int g = lane >> 2, q = lane & 3;
      const int ta = ct_s[warp][0][g], tb = ct_s[warp][1][g];
      float aba[4] = {0.f, 0.f, 0.f, 0.f}, abb[4] = {0.f, 0.f, 0.f, 0.f};
      float efa = 0.f, efb = 0.f;
      // the candidates' AABBs and edge fractions
      if (ta >= 0) {
        hda = __ldg(reinterpret_cast<const int4 *>(tiles + ta));
        const float4 a4 = tile_aabb(tiles, ta);
        aba[0] = a4.x; aba[1] = a4.y; aba[2] = a4.z; aba[3] = a4.w;
        efa = (float)hda.w * (1.f / 256.f);
      }
      if (tb >= 0) {
        hdb = __ldg(reinterpret_cast<const int4 *>(tiles + tb));
        const float4 a4 = tile_aabb(tiles, tb);
        abb[0] = a4.x; abb[1] = a4.y; abb[2] = a4.z; abb[3] = a4.w;
        efb = (float)hdb.w * (1.f / 256.f);
      }
      // pose a's and pose b's (x, y, cos, sin) from lanes 0 and 16
      const float pxa = __shfl_sync(0xffffffffu, px, 0), pya = __shfl_sync(0xffffffffu, py, 0);
      const float ca = __shfl_sync(0xffffffffu, c, 0), sa = __shfl_sync(0xffffffffu, s, 0);
      const float pxb = __shfl_sync(0xffffffffu, px, 16), pyb = __shfl_sync(0xffffffffu, py, 16);
      const float cb = __shfl_sync(0xffffffffu, c, 16), sb = __shfl_sync(0xffffffffu, s, 16);
      float s_a, s_b;
      mlp_rows_pair(w, q, aba, efa, pxa, pya, ca, sa, abb, efb, pxb, pyb, cb, sb, rfoot, s_a, s_b);
      if (q == 0) {
        sc_s[warp][0][g] = ta >= 0 ? s_a + b2 : kInf;
        sc_s[warp][1][g] = tb >= 0 ? s_b + b2 : kInf;
      }
      __syncwarp();
      float bs[K];
#pragma unroll
      for (int i = 0; i < K; ++i) {
        bs[i] = kInf;
        best[i] = -1;
      }
#pragma unroll
      for (int i = 0; i < kPre; ++i)
        if (cand[i] >= 0) topk_insert<K>(bs, best, sc_s[warp][half][i], cand[i]);
    } else {
#pragma unroll
      for (int i = 0; i < K; ++i) {
        best[i] = cand[i];
        if (hl == i && cand[i] >= 0) hda = __ldg(reinterpret_cast<const int4 *>(tiles + cand[i]));
      }
    }
    // the per-tile counts and the counters are cleared by the kernel before
    // this one: wait for it before the first append
    pdl_wait();
    if (valid && hl == 0) {
      int n = 0;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        prop[p * kMaxK + i] = best[i];
        if (best[i] >= 0) {
          list[(long long)best[i] * P + atomicAdd(&hist[best[i]], 1)] = (int)p;
          ++n;
        }
      }
#pragma unroll
      for (int i = K; i < kMaxK; ++i) prop[p * kMaxK + i] = -1;
      atomicAdd(&s_prop, n);
    }
    // upper bound on phi from the proposed tiles' obstacle circles (16
    // lanes, four circles a lane per round, their loads issued together)
#pragma unroll
    for (int i = 0; i < K; ++i) {
      // the proposed tile's header from the lane that read it
      int src = (half << 4) + i;
      if constexpr (NET) {
        int r = 0;
#pragma unroll
        for (int q = 0; q < kPre; ++q)
          if (cand[q] == best[i]) r = q;
        src = 4 * r;
      }
      int4 h;
      h.x = __shfl_sync(0xffffffffu, hda.x, src);
      h.y = __shfl_sync(0xffffffffu, hda.y, src);
      h.z = __shfl_sync(0xffffffffu, hda.z, src);
      if constexpr (NET) {
        const int bx = __shfl_sync(0xffffffffu, hdb.x, src);
        const int by = __shfl_sync(0xffffffffu, hdb.y, src);
        const int bz = __shfl_sync(0xffffffffu, hdb.z, src);
        if (half) h = make_int4(bx, by, bz, 0);
      }
      if (best[i] < 0) continue;  // uniform over the pose's lanes
      const float4 *circ = reinterpret_cast<const float4 *>(blob + h.x + h.y);
      for (int o = hl; o < h.z; o += 64) {
        float4 cc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (o + 16 * q < h.z) cc[q] = __ldg(circ + o + 16 * q);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (o + 16 * q < h.z) {
            ubp = fminf(ubp, circle_ub(cc[q], px, py, rfoot, rin));
            ++n_circ;
          }
      }
    }
    {  // 16-lane minimum (ubp >= 0, so its bits order like the value)
      const unsigned u = __float_as_uint(ubp);
      const unsigned u0 = __reduce_min_sync(0xffffffffu, half == 0 ? u : ~0u);
      const unsigned u1 = __reduce_min_sync(0xffffffffu, half == 1 ? u : ~0u);
      ubp = __uint_as_float(half ? u1 : u0);
    }
    ubp += ub_pad;  // soft minimum: a penetrating obstacle's value reaches up to log(K) / eta
    if (valid && hl == 0) ub_out[p] = ubp;
  }
  // every unproposed tile whose bound does not exceed the upper bound is
  // listed too: no other tile can hold a value at or below phi.  A lane's
  // first few tiles are appended after its loop (their atomics in flight
  // together), further ones at once.
  constexpr int kDefer = 4;
  int ncand = 0, defer[kDefer];
  const float Dc = cand_radius(ubp, rfoot);
  const float Dc2 = Dc >= 0.f ? Dc * Dc : -1.f;
  const bool in_cell = cell >= 0 && Dc <= grid.reach_q;
  const int clo = (in_cell ? e0 : 0) + hl, chi = valid ? (in_cell ? e1 : T) : 0;
  auto consider = [&](int t, float d2) {
    bool proposed = false;
#pragma unroll
    for (int q = 0; q < K; ++q) proposed |= (best[q] == t);
    if (!proposed && d2 <= Dc2) {
      if (ncand < kDefer) {
#pragma unroll
        for (int q = 0; q < kDefer; ++q)
          if (q == ncand) defer[q] = t;
      } else {
        list[(long long)t * P + atomicAdd(&hist[t], 1)] = (int)p;
      }
      ++ncand;
    }
  };
  i = clo;
  if (in_cell) {  // the same entries as the ranking pass: its first ones kept
#pragma unroll
    for (int q = 0; q < kKeep; ++q, i += 16)
      if (i < chi) consider(kt[q], kd2[q]);
  }
  for (; i < chi; i += 16) {
    const int t = in_cell ? __ldg(grid.tl + i) : i;
    consider(t, aabb_d2(in_cell ? __ldg(grid.ab + i) : tile_aabb(tiles, t), px, py));
    ++n_bound;
  }
#pragma unroll
  for (int q = 0; q < kDefer; ++q)
    if (q < ncand) list[(long long)defer[q] * P + atomicAdd(&hist[defer[q]], 1)] = (int)p;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) ncand += __shfl_xor_sync(0xffffffffu, ncand, o);
  if (valid && hl == 0 && ncand > 0) {
    atomicAdd(&s_fb, ncand);
    atomicAdd(&s_fbp, 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_bound += __shfl_xor_sync(0xffffffffu, n_bound, o);
    n_circ += __shfl_xor_sync(0xffffffffu, n_circ, o);
  }
  if (lane == 0) {
    atomicAdd(&s_bound, n_bound);
    atomicAdd(&s_circ, n_circ);
  }
  pdl_wait();  // (warps of poses beyond P reach the counters without appending)
  __syncthreads();
  if (threadIdx.x == 0) {
    const int slot = blockIdx.x % kCtrSlots;
    atomicAdd(&ctr->n_prop[slot], (unsigned long long)s_prop);
    atomicAdd(&ctr->n_fb[slot], (unsigned long long)s_fb);
    atomicAdd(&ctr->fallback_poses[slot], (unsigned long long)s_fbp);
    atomicAdd(&ctr->n_bound[slot], (unsigned long long)s_bound);
    atomicAdd(&ctr->n_circ[slot], (unsigned long long)s_circ);
  }
}

// ---------------------------------------------------------------------------
// exact evaluation of the per-tile lists
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// kTileCTAs CTAs per tile: CTA j of tile t takes the tile's work units j,
// j + kTileCTAs, ... (unit i covers lanes [128 i, 128 i + 128) of the tile's
// cnt * S lanes); lane l takes pose list[t * P + l / S] and obstacle range
// l % S of the tile.  The tile's blob and its obstacle circles are staged in
// shared memory (16-byte cp.async per thread) before the CTA waits for the
// proposals (they are pose-invariant).  Each lane tests its obstacles'
// circle bounds against the pose's upper bound; the survivors of the warp's
// 32 lanes are compacted (ballot) into a per-warp queue and evaluated a few
// at a time, kItemLanes lanes per (pose, obstacle) item, so that lanes whose
// obstacles were skipped do not idle through their neighbours' evaluations.  Every
// evaluated obstacle merges its key into the pose's by atomicMin.
constexpr int kTileCTAs = 2;
constexpr int kFilt = 4;    // circle bounds a lane tests between two queue appends
constexpr int kQueue = 31 + 32 * kFilt;  // per-warp queue of (lane, obstacle) items

// The first n_items queued (lane, obstacle) items of the warp, kItemLanes
// lanes per item (the obstacle's edges shared out, see obstacle_value_coop),
// 32 / kItemLanes items a round; every lane takes part in every round.
constexpr int kItemLanes = 4;
template <int M, bool SOFT>
__device__ __forceinline__ void eval_items(const FootprintK &F, const ParamsK &prm,
                                           const int *qw, int n_items, int lane, float px,
                                           float py, float c, float s, long long p,
                                           const int4 *ob, const float4 *vt,
                                           unsigned long long *__restrict__ keys,
                                           unsigned long long &n_obs,
                                           unsigned long long &n_edge)
{
  constexpr int B = 32 / kItemLanes;
  const int g = lane % kItemLanes;
  for (int r0 = 0; r0 < n_items; r0 += B) {
    const int slot = r0 + lane / kItemLanes;
    const bool live = slot < n_items;
    const int item = live ? qw[slot] : 0;
    const int src = item >> 16, o = item & 0xffff;
    // the item's pose from the lane that found it
    const float ipx = __shfl_sync(0xffffffffu, px, src), ipy = __shfl_sync(0xffffffffu, py, src);
    const float ic = __shfl_sync(0xffffffffu, c, src), is = __shfl_sync(0xffffffffu, s, src);
    const long long ip = __shfl_sync(0xffffffffu, p, src);
    const int4 rec = live ? ob[o] : make_int4(0, 0, 0, 0);
    const float v = obstacle_value_coop<M, kItemLanes, SOFT>(F, ipx, ipy, ic, is, vt + 2 * rec.x,
                                                             rec.y, prm.eps_sat, prm.eta, g);
    if (live && g == 0) {
      atomicMin(&keys[ip], pack_key(v, rec.z));
      ++n_obs;
      n_edge += rec.y;
    }
  }
}

template <int M, bool SOFT>
__global__ void __launch_bounds__(kListThreads)
    eval_lists(FootprintK F, ParamsK prm, const float4 *__restrict__ pose4, long long P,
               const TileHdr *__restrict__ tiles, int T, const unsigned char *__restrict__ blob,
               const int *__restrict__ hist, const int *__restrict__ list,
               const float *__restrict__ ub, unsigned long long *__restrict__ keys,
               CullCounters *ctr)
{
  extern __shared__ __align__(16) unsigned char tsm[];
  __shared__ int queue[kListThreads / 32][kQueue];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int *qw = queue[warp];
  const int t = (int)(blockIdx.x / kTileCTAs), j0 = (int)(blockIdx.x % kTileCTAs);
  const TileHdr h = tiles[t];
  {
    const unsigned char *src = blob + h.blob_off;
    const int bytes = h.blob_bytes + 16 * h.n_obs;  // records + circles
    for (int o = 16 * threadIdx.x; o < bytes; o += 16 * kListThreads)
      cp_async16(tsm + o, src + o);
  }
  pdl_wait();  // the proposal kernel's lists
  const int cnt = __ldcg(hist + t);
  const int S = tile_split(cnt, h.n_obs);
  // lane counts fit 32 bits: cnt * S <= max(cnt, 2 * kListThreads) and cnt <= P < 2^31
  const unsigned L = (unsigned)cnt * (unsigned)S;
  const int units = tile_units(cnt, h.n_obs);
  // a unit lane's pose, its frame and upper bound; the first unit's are read
  // while the tile is still being staged, each next one at the end of a unit
  long long pn = -1;
  float4 qn = make_float4(0.f, 0.f, 1.f, 0.f);
  float ubn = -kInf;
  auto fetch = [&](int j) {
    const unsigned l = (unsigned)j * kListThreads + threadIdx.x;
    pn = -1;
    if (j < units && l < L) pn = __ldcg(list + (long long)t * P + l / (unsigned)S);
    if (pn >= 0) {
      qn = __ldcg(pose4 + pn);
      ubn = __ldcg(ub + pn);
    }
  };
  fetch(j0);
  cp_async_wait_all();
  __syncthreads();
  const int4 *ob = reinterpret_cast<const int4 *>(tsm);
  const float4 *vt = reinterpret_cast<const float4 *>(tsm + 16 * h.n_obs);
  const float4 *circ = reinterpret_cast<const float4 *>(tsm + h.blob_bytes);
  unsigned long long n_obs = 0, n_edge = 0;
  for (int j = j0; j < units; j += kTileCTAs) {
    const unsigned l = (unsigned)j * kListThreads + threadIdx.x;
    const long long p = pn;
    float px = 0.f, py = 0.f, c = 1.f, s = 0.f, thr = -kInf;
    int o0 = 0, o1 = 0;
    if (p >= 0) {
      px = qn.x;
      py = qn.y;
      c = qn.z;
      s = qn.w;
      thr = ub_value(ubn);
      const int part = (int)(l % (unsigned)S);
      o0 = h.n_obs * part / S;  // n_obs <= 256 and part < S <= 256
      o1 = h.n_obs * (part + 1) / S;
    }
    int span = o1 - o0;
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) span = max(span, __shfl_xor_sync(0xffffffffu, span, k));
    // kFilt circle bounds at a time (independent), then their survivors
    // appended in obstacle order; whole batches of 32 evaluated at once
    int nq = 0;
    for (int k0 = 0; k0 < span; k0 += kFilt) {
      bool keep[kFilt];
#pragma unroll
      for (int q = 0; q < kFilt; ++q) {
        const int o = o0 + k0 + q;
        keep[q] = false;
        if (o < o1) keep[q] = !(circle_lb_value(circ[o], px, py, F.radius) > thr);
      }
#pragma unroll
      for (int q = 0; q < kFilt; ++q) {
        const unsigned mask = __ballot_sync(0xffffffffu, keep[q]);
        if (keep[q]) qw[nq + __popc(mask & ((1u << lane) - 1u))] = (lane << 16) | (o0 + k0 + q);
        nq += __popc(mask);
      }
      if (nq >= 32) {  // uniform: whole batches, the rest (< 32) moved to the front
        __syncwarp();
        int head = 0;
        for (; nq - head >= 32; head += 32)
          eval_items<M, SOFT>(F, prm, qw + head, 32, lane, px, py, c, s, p, ob, vt, keys, n_obs,
                              n_edge);
        const int rest = nq - head;
        const int v = lane < rest ? qw[head + lane] : 0;
        __syncwarp();
        if (lane < rest) qw[lane] = v;
        __syncwarp();
        nq = rest;
      }
    }
    if (nq > 0) {
      __syncwarp();
      eval_items<M, SOFT>(F, prm, qw, nq, lane, px, py, c, s, p, ob, vt, keys, n_obs, n_edge);
    }
    __syncwarp();  // the queue is refilled by the next unit
    fetch(j + kTileCTAs);
  }
  pdl_trigger();  // the epilogue may launch; it waits for this grid
  // evaluated obstacles and edges (the roofline's work count)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_obs += __shfl_xor_sync(0xffffffffu, n_obs, o);
    n_edge += __shfl_xor_sync(0xffffffffu, n_edge, o);
  }
  __shared__ unsigned long long s_cnt[2];
  if (threadIdx.x == 0) s_cnt[0] = s_cnt[1] = 0ull;
  __syncthreads();
  if (lane == 0 && n_obs) {
    atomicAdd(&s_cnt[0], n_obs);
    atomicAdd(&s_cnt[1], n_edge);
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_cnt[0]) {
    const int slot = blockIdx.x % kCtrSlots;
    atomicAdd(&ctr->n_obs_eval[slot], s_cnt[0]);
    atomicAdd(&ctr->n_edge_eval[slot], s_cnt[1]);
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
template <int M>
struct ListEvalCall {
  static int run(const FootprintK &F, const ParamsK &pk, const float4 *pose4, long long P,
                 const psdf_scene *sc, const int *hist,
                 const int *list, const float *ub, unsigned long long *keys,
                 CullCounters *ctr, cudaStream_t st)
  {
    const size_t smem = (size_t)(sc->max_blob_ext_bytes + 15) / 16 * 16;
    const bool soft = pk.eta > 0.f;
    auto kern = soft ? eval_lists<M, true> : eval_lists<M, false>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(eval_lists)");
    }
    const unsigned grid = (unsigned)sc->n_tiles * kTileCTAs;
    // follows the proposal kernel: may start while it finishes
    cudaError_t e = launch_pdl(kern, dim3(grid), dim3(kListThreads), smem, st, F, pk,
                               pose4, P, (const TileHdr *)sc->d_tiles, sc->n_tiles,
                               (const unsigned char *)sc->d_blob, hist, list, ub, keys, ctr);
    return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch (eval_lists)");
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
  return cull_layout(P, scene ? scene->n_tiles : 1).total;
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
  if (opts->mode != PSDF_PROPOSE_BOUND && opts->mode != PSDF_PROPOSE_MLP)
    return fail(PSDF_ERR_ARG, "unknown proposal mode");
  if (opts->mode == PSDF_PROPOSE_MLP && !mlp) return fail(PSDF_ERR_ARG, "mlp is NULL");
  if ((rc = check_out(phi, P, "phi"))) return rc;
  FootprintK F;
  rc = make_footprint(footprint, m, scene->eps_seg, &F);
  if (rc) return rc;
  if (P == 0) return PSDF_OK;
  if (P > (1LL << 31) - 1) return fail(PSDF_ERR_CAPACITY, "P too large for the cull");
  if (scene->n_tiles > kMaxScanTiles) return fail(PSDF_ERR_CAPACITY, "too many tiles for the cull");
  const int T = scene->n_tiles;
  if ((long long)P * std::max(T, 1) > (1LL << 31) - 1)
    return fail(PSDF_ERR_CAPACITY, "poses x tiles too large for the cull's pair lists");
  const CullLayout L = cull_layout(P, T);
  if (!workspace) return fail(PSDF_ERR_ARG, "workspace is NULL");
  if (((uintptr_t)workspace & 255u) != 0) return fail(PSDF_ERR_ARG, "workspace must be 256-byte aligned");
  if (workspace_bytes < L.total)
    return fail(PSDF_ERR_CAPACITY, "workspace smaller than psdf_cull_workspace_bytes");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char *ws = reinterpret_cast<unsigned char *>(workspace);
  CullCounters *ctr = reinterpret_cast<CullCounters *>(ws);
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + L.keys);
  float4 *pose4 = reinterpret_cast<float4 *>(ws + L.pose4);
  float *ub = reinterpret_cast<float *>(ws + L.ub);
  int *prop = reinterpret_cast<int *>(ws + L.prop);
  int *hist = reinterpret_cast<int *>(ws + L.hist);
  int *list = reinterpret_cast<int *>(ws + L.list);
  ParamsK pk{params->eps_sat, params->eta};
  cudaError_t e;
  {
    const int words = (int)(L.clear_bytes / 4);
    clear_words<<<std::min((words + 255) / 256, 64), 256, 0, st>>>(
        reinterpret_cast<unsigned *>(ws), words);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch (clear)");
  }
  if (T == 0) {
    e = cudaMemsetAsync(keys, 0xff, 8 * (size_t)P, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(keys)");
  } else {
    const int K = opts->k;
    const bool net = opts->mode == PSDF_PROPOSE_MLP;
    // soft minimum: an obstacle's value lies below its hard distance when it
    // is separated and at most log(K) / eta (K axes) when it penetrates, so
    // the upper bound taken from distances is raised by that much
    float ub_pad = 0.f;
    if (params->eta > 0.f)
      ub_pad = (float)(std::log((double)(m + scene->max_obs_edges)) / params->eta * (1.0 + 1e-5) +
                       1e-6);
    const unsigned pb = (unsigned)((P + 7) / 8);  // 4 warps x 2 poses per CTA
    const uint32_t *frag = net ? mlp->d_frag : nullptr;
    const float b2 = net ? mlp->b2 : 0.f;
    {
      ProfileScope prof("propose", st);
#define PSDF_PROPOSE(KK)                                                                      \
  e = launch_pdl(net ? propose<KK, true> : propose<KK, false>, dim3(pb), dim3(kPoseThreads), 0, \
                 st, poses, (long long)P, (const TileHdr *)scene->d_tiles, T, scene->grid,      \
                 F.radius, F.inner, ub_pad, (const unsigned char *)scene->d_blob, frag, b2,     \
                 keys, pose4,                                                                   \
                 ub,                                                                            \
                 prop, hist, list, ctr);
      switch (K) {
        case 1: PSDF_PROPOSE(1) break;
        case 2: PSDF_PROPOSE(2) break;
        case 3: PSDF_PROPOSE(3) break;
        default: PSDF_PROPOSE(4) break;
      }
#undef PSDF_PROPOSE
      if (e != cudaSuccess) return cuda_fail(e, "kernel launch (propose)");
    }
    {
      ProfileScope prof("cull_eval", st);
      rc = dispatch_m_cull<ListEvalCall>(m, F, pk, (const float4 *)pose4, (long long)P, scene,
                                         (const int *)hist, (const int *)list,
                                         (const float *)ub, keys, ctr, st);
      if (rc) return rc;
    }
  }
  rc = launch_epilogue(F, scene, poses, P, pk, keys, &ctr->err, phi, dphi, active, st, saved);
  if (rc) return rc;
  e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch");
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
  CullCounters c;
  e = cudaMemcpy(&c, workspace, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(cull counters)");
  auto sum = [](const unsigned long long (&v)[kCtrSlots]) {
    unsigned long long t = 0;
    for (int i = 0; i < kCtrSlots; ++i) t += v[i];
    return (int64_t)t;
  };
  stats->evaluated_obstacles = sum(c.n_obs_eval);
  stats->evaluated_edges = sum(c.n_edge_eval);
  stats->proposed_items = sum(c.n_prop);
  stats->fallback_items = sum(c.n_fb);
  stats->fallback_poses = sum(c.fallback_poses);
  stats->bound_evaluations = sum(c.n_bound);
  stats->circle_evaluations = sum(c.n_circ);
  if (c.err) return fail(PSDF_ERR_TIMEOUT, "a bounded device-side wait ran out");
  return PSDF_OK;
}
