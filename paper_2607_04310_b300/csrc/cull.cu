// Exact tile cull with a proposal (psdf_eval_culled and its helpers).
//
// Pipeline (one stream, no host synchronization):
//   1. cull_init        keys = +inf, counters and cell histogram cleared
//   2. cull_cells / cull_scan / cull_scatter
//                       spatial counting sort of the poses on a 64 x 64 grid
//                       in Morton order; blocks of 32 consecutive sorted poses
//   3. propose_*        every pose ranks all tiles (tile-proposal network on
//                       tensor cores, or the conservative bound) and keeps its
//                       k best; each block's union -> (block, tile) work items
//   4. eval_items       one warp per item: the block's 32 poses x the tile's
//                       obstacles, exactly as the full scan evaluates them
//   5. cull_fallback    per pose and tile not yet evaluated: lower bound on
//                       the tile's values vs the pose's current minimum; any
//                       pose of the block that cannot rule the tile out adds a
//                       work item
//   6. eval_items       the fallback items
//   7. epilogue         as for the full scan
// Skipped tiles hold only values strictly above each pose's minimum, and the
// minimum over 64-bit keys does not depend on evaluation order, so the result
// is the full scan's bit for bit.
#include <cuda_fp16.h>

#include <algorithm>
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

constexpr int kBlockPoses = 32;
constexpr int kCellBits = 6;
constexpr int kCells = 1 << (2 * kCellBits);
constexpr int kEvalParts = 4;  // obstacle ranges per (block, tile) item
constexpr int kMaxK = PSDF_CULL_MAX_K;
constexpr int kFallbackWarps = 8;
constexpr int kTileChunk = 512;  // tiles staged in shared memory at a time
constexpr int kFrag1Words = 8 * 32 * 2;
constexpr int kFrag2Words = 4 * 32 * 2;

// counters at the start of the workspace (after the error word)
struct CullCounters {
  int err;
  int n_items1;
  int n_items2;
  int fallback_poses;
};

struct CullLayout {
  size_t keys, perm, cell, hist, bits, items1, items2, cand_s, cand_i, total;
  long long nb;
  int words, splits;
};

// Tile splits of the proposal scoring: enough (group, split) warps to fill
// the GPU, at most 1024 tiles per split staged in shared memory.
static int score_splits(long long P, int n_tiles)
{
  const long long groups = std::max<long long>(1, (P + 15) / 16);
  long long sp = (2048 + groups - 1) / groups;
  sp = std::max<long long>(sp, (n_tiles + 1023) / 1024);
  return (int)std::max<long long>(1, std::min<long long>(sp, 64));
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

static CullLayout cull_layout(long long P, int n_tiles)
{
  CullLayout L;
  L.nb = (std::max<long long>(P, 1) + kBlockPoses - 1) / kBlockPoses;
  L.words = std::max(1, (n_tiles + 31) / 32);
  size_t o = 256;
  L.keys = o; o = align256(o + 8 * (size_t)std::max<long long>(P, 1));
  L.perm = o; o = align256(o + 4 * (size_t)std::max<long long>(P, 1));
  L.cell = o; o = align256(o + 4 * (size_t)std::max<long long>(P, 1));
  L.hist = o; o = align256(o + 4 * (size_t)kCells);
  L.bits = o; o = align256(o + 4 * (size_t)L.nb * L.words);
  L.items1 = o; o = align256(o + 8 * (size_t)L.nb * kBlockPoses * kMaxK);
  L.items2 = o; o = align256(o + 8 * (size_t)L.nb * std::max(n_tiles, 1));
  L.splits = score_splits(P, n_tiles);
  const size_t nc = (size_t)std::max<long long>(P, 1) * L.splits * kMaxK;
  L.cand_s = o; o = align256(o + 4 * nc);
  L.cand_i = o; o = align256(o + 4 * nc);
  L.total = o;
  return L;
}

// ---------------------------------------------------------------------------
// conservative lower bound and network inputs
// ---------------------------------------------------------------------------
// Lower bound (metres) on the separation of the posed footprint from any
// point of the tile's AABB, with a margin that covers the float32 error of
// the evaluated values; every operation rounds toward -inf.
__device__ __forceinline__ float tile_lb(const float *ab, float px, float py, float rfoot)
{
  const float dx = fmaxf(fmaxf(__fsub_rd(ab[0], px), __fsub_rd(px, ab[2])), 0.f);
  const float dy = fmaxf(fmaxf(__fsub_rd(ab[1], py), __fsub_rd(py, ab[3])), 0.f);
  const float d = __fsqrt_rd(__fadd_rd(__fmul_rd(dx, dx), __fmul_rd(dy, dy)));
  const float margin = __fmaf_ru(d, 1e-5f, 1e-4f);
  return __fsub_rd(__fsub_rd(d, rfoot), margin);
}

// The same bound in the min-key value domain (squared separation, or -inf
// when the tile may touch the footprint).
__device__ __forceinline__ float tile_lb_value(const float *ab, float px, float py, float rfoot)
{
  const float lb = tile_lb(ab, px, py, rfoot);
  return lb > 0.f ? __fmul_rd(lb, lb) : -kInf;
}

__device__ __forceinline__ float clampf(float x, float lo, float hi)
{
  return fminf(fmaxf(x, lo), hi);
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

__device__ __forceinline__ float corner_dist(const float *ab, int q, float px, float py)
{
  const float cx = (q == 1 || q == 2) ? ab[2] : ab[0];
  const float cy = (q >= 2) ? ab[3] : ab[1];
  return 0.1f * fminf(sqrtf((cx - px) * (cx - px) + (cy - py) * (cy - py)), 30.f);
}

// Network inputs 8 + 2q, 9 + 2q.
__device__ __forceinline__ void feat_rest(const float *ab, int q, float px, float py,
                                          float rfoot, float edge_frac, float &f0, float &f1)
{
  if (q < 2) {
    f0 = corner_dist(ab, 2 * q, px, py);
    f1 = corner_dist(ab, 2 * q + 1, px, py);
  } else if (q == 2) {
    const float dx = fmaxf(fmaxf(ab[0] - px, px - ab[2]), 0.f);
    const float dy = fmaxf(fmaxf(ab[1] - py, py - ab[3]), 0.f);
    f0 = 0.1f * fminf(sqrtf(dx * dx + dy * dy), 30.f);
    f1 = rfoot;
  } else {
    f0 = edge_frac;
    f1 = 1.f;
  }
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
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    w.b1[j][0] = frag[(j * 32 + lane) * 2];
    w.b1[j][1] = frag[(j * 32 + lane) * 2 + 1];
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    w.b2[j][0] = frag[kFrag1Words + (j * 32 + lane) * 2];
    w.b2[j][1] = frag[kFrag1Words + (j * 32 + lane) * 2 + 1];
  }
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
// pose sort
// ---------------------------------------------------------------------------
__device__ __forceinline__ int spread6(int x)
{
  x &= 63;
  x = (x | (x << 4)) & 0x30F;
  x = (x | (x << 2)) & 0x333;
  x = (x | (x << 1)) & 0x555;
  return x;
}

__global__ void cull_init(unsigned long long *keys, long long P, int *hist,
                          CullCounters *ctr)
{
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) keys[i] = ~0ull;
  if (i < kCells) hist[i] = 0;
  if (i == 0) {
    ctr->err = 0;
    ctr->n_items1 = 0;
    ctr->n_items2 = 0;
    ctr->fallback_poses = 0;
  }
}

__global__ void cull_cells(const float *__restrict__ poses, long long P, float x0, float y0,
                           float inv_cell, int *__restrict__ cell, int *__restrict__ hist)
{
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float fx = (poses[3 * p] - x0) * inv_cell, fy = (poses[3 * p + 1] - y0) * inv_cell;
  fx = (fx == fx) ? clampf(fx, 0.f, 63.f) : 0.f;  // NaN poses go to cell 0
  fy = (fy == fy) ? clampf(fy, 0.f, 63.f) : 0.f;
  const int code = spread6((int)fx) | (spread6((int)fy) << 1);
  cell[p] = code;
  atomicAdd(&hist[code], 1);
}

// exclusive scan of the 4096-bin histogram, one CTA of 1024 threads
__global__ void __launch_bounds__(1024) cull_scan(int *hist)
{
  __shared__ int warp_sum[32];
  const int tid = threadIdx.x;
  int v[4], s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[i] = hist[4 * tid + i];
    s += v[i];
  }
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, incl, o);
    if ((tid & 31) >= o) incl += n;
  }
  if ((tid & 31) == 31) warp_sum[tid >> 5] = incl;
  __syncthreads();
  if (tid < 32) {
    int w = warp_sum[tid], wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, wi, o);
      if (tid >= o) wi += n;
    }
    warp_sum[tid] = wi - w;
  }
  __syncthreads();
  int base = warp_sum[tid >> 5] + incl - s;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    hist[4 * tid + i] = base;
    base += v[i];
  }
}

__global__ void cull_scatter(const int *__restrict__ cell, long long P, int *__restrict__ offs,
                             int *__restrict__ perm)
{
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int pos = atomicAdd(&offs[cell[p]], 1);
  perm[pos] = (int)p;
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

// Candidates of a pose for one tile split: its K best (score, tile), kept in
// global memory at cand[(sorted pose * splits + split) * K + i].
template <int K>
__device__ __forceinline__ void store_cand(float *cand_s, int *cand_i, long long ps, int split,
                                           int splits, const float (&sc)[K], const int (&id)[K])
{
#pragma unroll
  for (int i = 0; i < K; ++i) {
    cand_s[(ps * splits + split) * K + i] = sc[i];
    cand_i[(ps * splits + split) * K + i] = id[i];
  }
}

// Stage the AABBs (and edge fractions) of tiles [t0, t1) in shared memory.
__device__ __forceinline__ void stage_tiles(const TileHdr *__restrict__ tiles, int t0, int t1,
                                            float4 *ab_s, float *ef_s)
{
  for (int i = threadIdx.x; i < t1 - t0; i += blockDim.x) {
    const TileHdr h = tiles[t0 + i];
    ab_s[i] = make_float4(h.aabb[0], h.aabb[1], h.aabb[2], h.aabb[3]);
    if (ef_s) ef_s[i] = (float)h.n_vtx * (1.f / 256.f);
  }
}

constexpr int kScoreWarps = 4;
constexpr int kMaxSplitTiles = 1024;  // tiles per split staged in shared memory

// Bound proposal scores: warp = 32 sorted poses, blockIdx.y = tile split.
template <int K>
__global__ void __launch_bounds__(kScoreWarps * 32)
    score_bound(const float *__restrict__ poses, const int *__restrict__ perm, long long P,
                const TileHdr *__restrict__ tiles, int n_tiles, int splits, float rfoot,
                float *__restrict__ cand_s, int *__restrict__ cand_i)
{
  __shared__ float4 ab_s[kMaxSplitTiles];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int split = blockIdx.y;
  const int t0 = (int)((long long)n_tiles * split / splits);
  const int t1 = (int)((long long)n_tiles * (split + 1) / splits);
  stage_tiles(tiles, t0, t1, ab_s, nullptr);
  __syncthreads();
  const long long ps = ((long long)blockIdx.x * kScoreWarps + warp) * 32 + lane;
  if (ps >= P) return;
  const long long p = perm[ps];
  const float px = poses[3 * p], py = poses[3 * p + 1];
  float sc[K];
  int id[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    sc[i] = kInf;
    id[i] = -1;
  }
  for (int i = 0; i < t1 - t0; ++i) {
    const float4 a4 = ab_s[i];
    const float ab[4] = {a4.x, a4.y, a4.z, a4.w};
    topk_insert<K>(sc, id, tile_lb(ab, px, py, rfoot), t0 + i);
  }
  store_cand<K>(cand_s, cand_i, ps, split, splits, sc, id);
}

// Network proposal scores: warp = 16 sorted poses (the 16 rows of every
// tensor-core tile), blockIdx.y = tile split; two tiles in flight per step.
template <int K>
__global__ void __launch_bounds__(kScoreWarps * 32)
    score_mlp(const float *__restrict__ poses, const int *__restrict__ perm, long long P,
              const TileHdr *__restrict__ tiles, int n_tiles, int splits, float rfoot,
              const uint32_t *__restrict__ frag, float b2, float *__restrict__ cand_s,
              int *__restrict__ cand_i)
{
  __shared__ float4 ab_s[kMaxSplitTiles];
  __shared__ float ef_s[kMaxSplitTiles];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int split = blockIdx.y;
  const int t0 = (int)((long long)n_tiles * split / splits);
  const int t1 = (int)((long long)n_tiles * (split + 1) / splits);
  stage_tiles(tiles, t0, t1, ab_s, ef_s);
  __syncthreads();
  const long long group = (long long)blockIdx.x * kScoreWarps + warp;
  if (group * 16 >= P) return;  // uniform over the warp
  const int g = lane >> 2, q = lane & 3;
  const long long psa = group * 16 + g, psb = group * 16 + g + 8;
  float pxa = 0.f, pya = 0.f, ca = 1.f, sa = 0.f, pxb = 0.f, pyb = 0.f, cb = 1.f, sb = 0.f;
  if (psa < P) {
    const long long p = perm[psa];
    pxa = poses[3 * p];
    pya = poses[3 * p + 1];
    sincosf(poses[3 * p + 2], &sa, &ca);
  }
  if (psb < P) {
    const long long p = perm[psb];
    pxb = poses[3 * p];
    pyb = poses[3 * p + 1];
    sincosf(poses[3 * p + 2], &sb, &cb);
  }
  MlpFrags w;
  load_frags(frag, lane, w);
  float sca[K], scb[K];
  int ida[K], idb[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    sca[i] = scb[i] = kInf;
    ida[i] = idb[i] = -1;
  }
  const int n = t1 - t0;
  for (int i = 0; i < n; i += 2) {
    const int j = min(i + 1, n - 1);
    const float4 a4 = ab_s[i], b4 = ab_s[j];
    const float ab0[4] = {a4.x, a4.y, a4.z, a4.w};
    const float ab1[4] = {b4.x, b4.y, b4.z, b4.w};
    float s0a, s0b, s1a, s1b;
    mlp_rows(w, ab0, q, pxa, pya, ca, sa, pxb, pyb, cb, sb, rfoot, ef_s[i], s0a, s0b);
    mlp_rows(w, ab1, q, pxa, pya, ca, sa, pxb, pyb, cb, sb, rfoot, ef_s[j], s1a, s1b);
    if (q == 0) {
      topk_insert<K>(sca, ida, s0a + b2, t0 + i);
      topk_insert<K>(scb, idb, s0b + b2, t0 + i);
      if (j != i) {
        topk_insert<K>(sca, ida, s1a + b2, t0 + j);
        topk_insert<K>(scb, idb, s1b + b2, t0 + j);
      }
    }
  }
  if (q == 0) {
    if (psa < P) store_cand<K>(cand_s, cand_i, psa, split, splits, sca, ida);
    if (psb < P) store_cand<K>(cand_s, cand_i, psb, split, splits, scb, idb);
  }
}

// One warp per block of 32 sorted poses: merge each pose's candidates over
// the splits into its K best, mark the block's union, emit (block, tile) items.
template <int K>
__global__ void __launch_bounds__(128)
    propose_union(long long P, long long nb, int splits, int words,
                  const float *__restrict__ cand_s, const int *__restrict__ cand_i,
                  unsigned *__restrict__ prop_bits, int2 *__restrict__ items, CullCounters *ctr)
{
  extern __shared__ unsigned ubits[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long b = (long long)blockIdx.x * 4 + warp;
  unsigned *bits_s = ubits + warp * words;
  if (b >= nb) return;  // uniform over the warp
  for (int wd = lane; wd < words; wd += 32) bits_s[wd] = 0u;
  __syncwarp();
  const long long ps = b * kBlockPoses + lane;
  if (ps < P) {
    float sc[K];
    int id[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      sc[i] = kInf;
      id[i] = -1;
    }
    for (int sp = 0; sp < splits; ++sp)
      for (int i = 0; i < K; ++i) {
        const long long c = (ps * splits + sp) * K + i;
        const int t = cand_i[c];
        if (t >= 0) topk_insert<K>(sc, id, cand_s[c], t);
      }
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (id[i] >= 0) atomicOr(&bits_s[id[i] >> 5], 1u << (id[i] & 31));
  }
  __syncwarp();
  for (int wd = lane; wd < words; wd += 32) {
    unsigned m = bits_s[wd];
    prop_bits[b * words + wd] = m;
    if (m) {
      int base = atomicAdd(&ctr->n_items1, __popc(m));
      while (m) {
        const int bit = __ffs(m) - 1;
        m &= m - 1;
        items[base++] = make_int2((int)b, wd * 32 + bit);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// exact evaluation of (block, tile) items, fallback check
// ---------------------------------------------------------------------------
constexpr int kEvalWarps = 4;

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

// One warp per work unit = (block, tile, part): part `pt` of `parts` covers
// the tile's obstacles [pt * n_obs / parts, (pt + 1) * n_obs / parts).  The
// warp copies those obstacle records and their vertex records into its own
// slice of shared memory (16-byte cp.async per lane), then every lane
// evaluates them for its pose, reading the records as a broadcast.
template <int M>
__global__ void __launch_bounds__(kEvalWarps * 32)
    eval_items(FootprintK F, ParamsK prm, const float *__restrict__ poses,
               const int *__restrict__ perm, long long P, const TileHdr *__restrict__ tiles,
               const unsigned char *__restrict__ blob, const int2 *__restrict__ items,
               const int *__restrict__ n_items, int parts, int blob_cap,
               unsigned long long *__restrict__ keys)
{
  extern __shared__ __align__(16) unsigned char esm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *mine = esm + (size_t)warp * blob_cap;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long n = (long long)(*n_items) * parts;
  for (long long u = gw; u < n; u += nw) {
    const int2 it = items[u / parts];
    const int pt = (int)(u % parts);
    const TileHdr h = tiles[it.y];
    const int o0 = (int)((long long)h.n_obs * pt / parts);
    const int o1 = (int)((long long)h.n_obs * (pt + 1) / parts);
    if (o0 >= o1) continue;  // uniform over the warp
    const unsigned char *src = blob + h.blob_off;
    const int4 *gob = reinterpret_cast<const int4 *>(src);
    const int4 first = gob[o0], last = gob[o1 - 1];
    const int v0 = first.x, v1 = last.x + last.y;  // vertex range of the part
    const int obytes = 16 * (o1 - o0);
    const int vbytes = 32 * (v1 - v0);
    const unsigned char *vsrc = src + 16 * h.n_obs + 32 * v0;
    __syncwarp();  // the previous unit's reads of `mine` are done
    for (int off = 16 * lane; off < obytes; off += 16 * 32)
      cp_async16(mine + off, src + 16 * o0 + off);
    for (int off = 16 * lane; off < vbytes; off += 16 * 32)
      cp_async16(mine + obytes + off, vsrc + off);
    const long long ps = (long long)it.x * kBlockPoses + lane;
    const bool valid = ps < P;
    float px = 0.f, py = 0.f, c = 1.f, s = 0.f;
    long long p = 0;
    if (valid) {
      p = perm[ps];
      px = poses[3 * p];
      py = poses[3 * p + 1];
      sincosf(poses[3 * p + 2], &s, &c);
    }
    cp_async_wait_all();
    __syncwarp();
    const int4 *ob = reinterpret_cast<const int4 *>(mine);
    const float4 *vt = reinterpret_cast<const float4 *>(mine + obytes);
    unsigned long long best = ~0ull;
    for (int o = 0; o < o1 - o0; ++o) {
      const int4 rec = ob[o];
      const float v =
          obstacle_value<M>(F, px, py, c, s, vt + 2 * (rec.x - v0), rec.y, prm.eps_sat);
      const unsigned long long key = pack_key(v, rec.z);
      best = key < best ? key : best;
    }
    if (valid && best != ~0ull) atomicMin(&keys[p], best);
  }
}

// One CTA per pose block; each warp takes every 8th tile of a staged chunk,
// its lanes are the block's 32 poses.
__global__ void __launch_bounds__(kFallbackWarps * 32)
    cull_fallback(const float *__restrict__ poses, const int *__restrict__ perm, long long P,
                  long long nb, const TileHdr *__restrict__ tiles, int n_tiles, float rfoot,
                  int words, const unsigned *__restrict__ prop_bits,
                  const unsigned long long *__restrict__ keys, int2 *__restrict__ items,
                  CullCounters *ctr)
{
  __shared__ float4 ab_s[kTileChunk];
  __shared__ unsigned bits_s[kTileChunk / 32];
  __shared__ unsigned any_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
    const long long ps = b * kBlockPoses + lane;
    const bool valid = ps < P;
    float px = 0.f, py = 0.f, best = -kInf;
    if (valid) {
      const long long p = perm[ps];
      px = poses[3 * p];
      py = poses[3 * p + 1];
      const unsigned long long key = keys[p];
      best = (key == ~0ull) ? kInf : from_ordered_bits((uint32_t)(key >> 32));
    }
    if (threadIdx.x == 0) any_s = 0u;
    bool any = false;
    for (int c0 = 0; c0 < n_tiles; c0 += kTileChunk) {
      const int cn = min(kTileChunk, n_tiles - c0);
      __syncthreads();
      for (int i = threadIdx.x; i < cn; i += blockDim.x) {
        const TileHdr h = tiles[c0 + i];
        ab_s[i] = make_float4(h.aabb[0], h.aabb[1], h.aabb[2], h.aabb[3]);
      }
      for (int i = threadIdx.x; i < (cn + 31) / 32; i += blockDim.x)
        bits_s[i] = prop_bits[b * words + (c0 >> 5) + i];
      __syncthreads();
      for (int i = warp; i < cn; i += kFallbackWarps) {
        const float4 a4 = ab_s[i];
        const float ab[4] = {a4.x, a4.y, a4.z, a4.w};
        const bool proposed = (bits_s[i >> 5] >> (i & 31)) & 1u;
        const bool need = valid && !proposed && !(tile_lb_value(ab, px, py, rfoot) > best);
        const unsigned m = __ballot_sync(0xffffffffu, need);
        if (m && lane == 0) {
          const int idx = atomicAdd(&ctr->n_items2, 1);
          items[idx] = make_int2((int)b, c0 + i);
        }
        any |= need;
      }
    }
    const unsigned fm = __ballot_sync(0xffffffffu, any);
    if (lane == 0 && fm) atomicOr(&any_s, fm);
    __syncthreads();
    if (threadIdx.x == 0 && any_s) atomicAdd(&ctr->fallback_poses, __popc(any_s));
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
struct CullEvalCall {
  static int run(const FootprintK &F, const ParamsK &pk, const float *poses, const int *perm,
                 long long P, const psdf_scene *sc, const int2 *items, const int *n_items,
                 unsigned long long *keys, int grid, cudaStream_t st)
  {
    const int blob_cap = (sc->max_blob_bytes + 15) / 16 * 16;
    const size_t smem = (size_t)kEvalWarps * blob_cap;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(eval_items<M>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(eval_items)");
    }
    eval_items<M><<<grid, kEvalWarps * 32, smem, st>>>(F, pk, poses, perm, P, sc->d_tiles,
                                                       sc->d_blob, items, n_items, kEvalParts,
                                                       blob_cap, keys);
    return PSDF_OK;
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
  ParamsK pk{params->eps_sat, params->eta};
  rc = dispatch_m_cull<TileValuesCall>(m, F, pk, poses, (long long)P, scene, values,
                                       (cudaStream_t)stream);
  if (rc) return rc;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch");
}

extern "C" int psdf_eval_culled(const float *footprint, int32_t m, const psdf_scene *scene,
                                const psdf_mlp *mlp, const psdf_cull_opts *opts,
                                const float *poses, int64_t P, const psdf_params *params,
                                float *phi, float *dphi, uint32_t *active, void *workspace,
                                size_t workspace_bytes, void *stream)
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
  const CullLayout L = cull_layout(P, scene->n_tiles);
  if (!workspace) return fail(PSDF_ERR_ARG, "workspace is NULL");
  if (((uintptr_t)workspace & 255u) != 0) return fail(PSDF_ERR_ARG, "workspace must be 256-byte aligned");
  if (workspace_bytes < L.total)
    return fail(PSDF_ERR_CAPACITY, "workspace smaller than psdf_cull_workspace_bytes");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char *ws = reinterpret_cast<unsigned char *>(workspace);
  CullCounters *ctr = reinterpret_cast<CullCounters *>(ws);
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + L.keys);
  int *perm = reinterpret_cast<int *>(ws + L.perm);
  int *cell = reinterpret_cast<int *>(ws + L.cell);
  int *hist = reinterpret_cast<int *>(ws + L.hist);
  unsigned *bits = reinterpret_cast<unsigned *>(ws + L.bits);
  int2 *items1 = reinterpret_cast<int2 *>(ws + L.items1);
  int2 *items2 = reinterpret_cast<int2 *>(ws + L.items2);
  ParamsK pk{params->eps_sat, params->eta};
  const int init_n = (int)std::max<long long>(P, kCells);
  cull_init<<<(init_n + 255) / 256, 256, 0, st>>>(keys, P, hist, ctr);
  if (scene->n_tiles > 0) {
    // spatial sort of the poses over the scene's bounding box (poses outside
    // it clamp to the border cells)
    const float span = std::max(std::max(scene->bbox[2] - scene->bbox[0],
                                         scene->bbox[3] - scene->bbox[1]), 1e-3f);
    const int pb = (int)((P + 255) / 256);
    cull_cells<<<pb, 256, 0, st>>>(poses, P, scene->bbox[0], scene->bbox[1], 64.f / span, cell,
                                   hist);
    cull_scan<<<1, 1024, 0, st>>>(hist);
    cull_scatter<<<pb, 256, 0, st>>>(cell, P, hist, perm);
    // proposals: per-pose K best tiles per split, then each block's union
    const int K = opts->k;
    if (L.splits > 64 || (scene->n_tiles + L.splits - 1) / L.splits > kMaxSplitTiles)
      return fail(PSDF_ERR_CAPACITY, "scene has too many tiles for the cull");
    float *cand_s = reinterpret_cast<float *>(ws + L.cand_s);
    int *cand_i = reinterpret_cast<int *>(ws + L.cand_i);
    {
      ProfileScope prof("propose", st);
      const bool net = opts->mode == PSDF_PROPOSE_MLP;
      const long long warps = net ? (P + 15) / 16 : (P + 31) / 32;
      dim3 sg((unsigned)((warps + kScoreWarps - 1) / kScoreWarps), (unsigned)L.splits);
      const unsigned ub = (unsigned)((L.nb + 3) / 4);
      const size_t usmem = 4 * sizeof(unsigned) * (size_t)L.words;
      if (usmem > 48 * 1024) return fail(PSDF_ERR_CAPACITY, "scene has too many tiles for the cull");
#define PSDF_PROPOSE(KK)                                                                      \
  if (net)                                                                                    \
    score_mlp<KK><<<sg, kScoreWarps * 32, 0, st>>>(poses, perm, P, scene->d_tiles,            \
                                                   scene->n_tiles, L.splits, F.radius,        \
                                                   mlp->d_frag, mlp->b2, cand_s, cand_i);     \
  else                                                                                        \
    score_bound<KK><<<sg, kScoreWarps * 32, 0, st>>>(poses, perm, P, scene->d_tiles,          \
                                                     scene->n_tiles, L.splits, F.radius,      \
                                                     cand_s, cand_i);                         \
  propose_union<KK><<<ub, 128, usmem, st>>>(P, L.nb, L.splits, L.words, cand_s, cand_i, bits, \
                                            items1, ctr);
      switch (K) {
        case 1: PSDF_PROPOSE(1) break;
        case 2: PSDF_PROPOSE(2) break;
        case 3: PSDF_PROPOSE(3) break;
        default: PSDF_PROPOSE(4) break;
      }
#undef PSDF_PROPOSE
    }
    const int eval_grid = device_sms() * 8;
    {
      ProfileScope prof("cull_eval", st);
      rc = dispatch_m_cull<CullEvalCall>(m, F, pk, poses, (const int *)perm, (long long)P, scene,
                                         (const int2 *)items1, (const int *)&ctr->n_items1,
                                         keys, eval_grid, st);
      if (rc) return rc;
    }
    {
      ProfileScope prof("fallback", st);
      const long long fb_ctas = std::min<long long>(L.nb, (long long)device_sms() * 8);
      cull_fallback<<<(unsigned)fb_ctas, kFallbackWarps * 32, 0, st>>>(
          poses, perm, P, L.nb, scene->d_tiles, scene->n_tiles, F.radius, L.words, bits, keys,
          items2, ctr);
    }
    {
      ProfileScope prof("cull_eval", st);
      rc = dispatch_m_cull<CullEvalCall>(m, F, pk, poses, (const int *)perm, (long long)P, scene,
                                         (const int2 *)items2, (const int *)&ctr->n_items2,
                                         keys, eval_grid, st);
      if (rc) return rc;
    }
  }
  rc = launch_epilogue(F, scene, poses, P, pk, keys, &ctr->err, phi, dphi, active, st);
  if (rc) return rc;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch");
}

extern "C" int psdf_cull_stats_read(const void *workspace, void *stream, psdf_cull_stats *stats)
{
  if (!workspace || !stats) return fail(PSDF_ERR_ARG, "NULL argument");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  CullCounters c;
  e = cudaMemcpy(&c, workspace, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(cull counters)");
  stats->pose_blocks = 0;
  stats->tiles = 0;
  stats->proposed_items = c.n_items1;
  stats->fallback_items = c.n_items2;
  stats->fallback_poses = c.fallback_poses;
  if (c.err) return fail(PSDF_ERR_TIMEOUT, "a bounded device-side wait ran out");
  return PSDF_OK;
}
