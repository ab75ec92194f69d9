// Batched plan (psdf_plan_*): many instances -- each a footprint, an obstacle
// edge set of its own and a run of poses (an MPC horizon, an SQP iterate, a
// rollout; Sec. IV-B stacks the horizon, Sec. V gives each stage its edge set)
// -- evaluated in ONE persistent launch.
//
// Device image: every instance's scene is prepared exactly as a psdf_scene
// (same tiles, blobs, per-row obstacle records) and the images are
// concatenated, so each instance's results equal psdf_eval_grad's bit for bit.
//
// Work: an item is (pose block, run of the instance's tiles).  A pose block
// holds up to `threads` poses of one instance; the (pose, obstacle) pairs of
// each tile are dealt round-robin over the lanes, so a short horizon still
// fills the CTA evenly.  Items are sorted by decreasing work and
// taken from an atomic queue by persistent CTAs; tiles stream through shared
// memory by TMA bulk copies (double-buffered, bounded waits).  Pair keys are
// merged per pose in shared memory and into the pose's global 64-bit key with
// one atomicMin per pose per item; an epilogue kernel then writes value,
// active pair and closed-form gradient.  No CTA ever waits for another.
//
// Autotuner: a grid of (threads, tiles per item) is timed on the caller's
// poses; the fastest is kept and cached per plan shape for the process.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "profile.h"
#include "psdf_device.cuh"
#include "psdf_internal.h"
#include "tma.cuh"

namespace psdf {

constexpr int kPlanMaxThreads = 256;
constexpr int kPlanMaxTilesPerItem = 64;
// A footprint laid out as the shared-memory records of FootprintS.
struct FootprintRec {
  float4 rec[2 * kMaxM];        // {vx, vy, ex, ey}, {inv_e2, nx, ny, 0} per robot vertex
  float4 pair[4 * (kMaxM / 2)];  // vertex pairs for the paired edge step (FootprintS)
  float2 ivl[kMaxM];            // {alo, ahi}
  int m;
  int pad[3];
};
constexpr int kFpBytes = (int)((sizeof(FootprintRec) + 15) / 16 * 16);
constexpr int kPlanSmemHead = 128;  // two mbarriers, padded

struct PlanItem {
  int block;  // pose block
  int tile0;  // first (global) tile
  int ntile;  // tiles; 0 for an instance without obstacles
  int pad;
};

struct PlanBlock {
  long long pose0;  // first (global) pose
  int inst;
  int npose;
  int n_items;
  int pad[3];
};

struct PlanInst {
  long long row0;  // first (global) edge row of the instance
  long long rows;  // edge rows of the instance
};

// counters: [0] work queue, [1] a timed-out wait
constexpr int kCtrWords = 2;

// Sizes of the plan's device arrays, for the index checks of a debug build.
struct PlanBounds {
  long long n_poses, n_rows, n_vtx, blob_bytes;
  int n_items, n_blocks, n_inst, n_tiles;
};

// Debug builds (PSDF_DEBUG_CHECKS) check every index a batched kernel takes
// from its data before using it: the first violation (site << 48 | index)
// is recorded and the access skipped.  Release builds compile the checks out.
#ifdef PSDF_DEBUG_CHECKS
static __device__ unsigned long long g_plan_debug;
__device__ __forceinline__ bool dbg_ok(bool cond, int site, long long idx)
{
  if (cond) return true;
  atomicCAS(&g_plan_debug, 0ull,
            ((unsigned long long)(site & 0xffff) << 48) | ((unsigned long long)idx & 0xffffffffffffull));
  return false;
}
#define PSDF_DBG(cond, site, idx) dbg_ok((cond), (site), (long long)(idx))
#else
#define PSDF_DBG(cond, site, idx) true
#endif

// ---------------------------------------------------------------------------
// device
// ---------------------------------------------------------------------------
// One item: for each of the item's tiles the npose x n_obs (pose, obstacle)
// pairs are dealt round-robin over all lanes, so that every lane has the
// same share whatever the horizon; a pair's key goes into the pose's key in
// shared memory, and the block's keys into global memory once per item.
// False when a bounded wait ran out (uniform over the CTA).
template <int M, bool SOFT>
__device__ bool scan_item(const FootprintS &F, ParamsK prm, const float *__restrict__ poses,
                          long long pose0, int npose, const TileHdr *__restrict__ tiles,
                          const unsigned char *__restrict__ blob, int tile0, int ntile,
                          unsigned char *buf0, int blob_cap, uint64_t *bars, unsigned &phase,
                          float4 *spose, unsigned long long *skey, unsigned long long *keys,
                          const PlanBounds &bnd, unsigned wait_polls)
{
  if (ntile == 0) return true;
#ifdef PSDF_DEBUG_CHECKS
  for (int k = 0; k < ntile; ++k) {
    const TileHdr h = tiles[tile0 + k];
    const bool good = h.blob_off >= 0 && h.blob_off % 16 == 0 && h.blob_bytes >= 16 &&
                      h.blob_bytes % 16 == 0 && h.blob_bytes <= blob_cap &&
                      (long long)h.blob_off + h.blob_bytes <= bnd.blob_bytes &&
                      h.blob_bytes == 16 * h.n_obs + 32 * h.n_vtx;
    if (!PSDF_DBG(good, 6, tile0 + k)) return true;
  }
#endif
  // pair i = pose i % npose, obstacle i / npose: a stride of blockDim.x
  // pairs moves the pose by dj and the obstacle by do_ (plus a carry)
  const int dj = (int)blockDim.x % npose, do_ = (int)blockDim.x / npose;
  // the block's poses (x, y, cos, sin) and their keys for this item
  for (int j = threadIdx.x; j < npose; j += blockDim.x) {
    const long long p = pose0 + j;
    float sn, cs;
    sincosf(poses[3 * p + 2], &sn, &cs);
    spose[j] = make_float4(poses[3 * p], poses[3 * p + 1], cs, sn);
    skey[j] = ~0ull;
  }
  if (threadIdx.x == 0) {
    const TileHdr h = tiles[tile0];
    fence_proxy_async();  // the previous item's generic reads of buffer 0
    mbar_arrive_expect_tx(&bars[0], (unsigned)h.blob_bytes);
    bulk_g2s(buf0, blob + h.blob_off, (unsigned)h.blob_bytes, &bars[0]);
  }
  unsigned pending = 1u;
  bool ok = true;
  for (int k = 0; k < ntile; ++k) {
    const int b = k & 1;
    if (k + 1 < ntile) {
      if (threadIdx.x == 0) {
        const TileHdr hn = tiles[tile0 + k + 1];
        fence_proxy_async();
        mbar_arrive_expect_tx(&bars[b ^ 1], (unsigned)hn.blob_bytes);
        bulk_g2s(buf0 + (b ^ 1) * blob_cap, blob + hn.blob_off, (unsigned)hn.blob_bytes,
                 &bars[b ^ 1]);
      }
      pending |= 1u << (b ^ 1);
    }
    bool got = mbar_wait_bounded(&bars[b], (phase >> b) & 1u, wait_polls);
    got = __syncthreads_and(got);
    if (!got) {
      ok = false;
      break;
    }
    pending &= ~(1u << b);
    phase ^= 1u << b;
    const TileHdr h = tiles[tile0 + k];
    const unsigned char *tb = buf0 + b * blob_cap;
    const int4 *ob = reinterpret_cast<const int4 *>(tb);
    const float4 *vt = reinterpret_cast<const float4 *>(tb + 16 * h.n_obs);
    // (pose, obstacle) pairs of the tile dealt round-robin over all lanes:
    // pair i = pose i % npose, obstacle i / npose
    // (the lane's pose advances by dj and its obstacle by do_ per pair; a
    // lane keeps its best key while its pose stays the same)
    const int n_obs = h.n_obs;
    int j = (int)threadIdx.x % npose, o = (int)threadIdx.x / npose;
    int cur = -1;
    unsigned long long best = ~0ull;
    for (; o < n_obs; o += do_) {
      const int4 rec = ob[o];
      if (PSDF_DBG(rec.x >= 0 && rec.y >= 1 && rec.y <= kMaxObsEdges &&
                       rec.x + (rec.y == 1 ? 1 : rec.y) <= h.n_vtx,
                   7, tile0 + k)) {
        const float4 q = spose[j];
        const float v = obstacle_value<M, FootprintS, SOFT>(F, q.x, q.y, q.z, q.w, vt + 2 * rec.x,
                                                            rec.y, prm.eps_sat, prm.eta);
        const unsigned long long key = pack_key(v, rec.z);
        if (j != cur) {
          if (cur >= 0) atomicMin(&skey[cur], best);
          cur = j;
          best = key;
        } else {
          best = key < best ? key : best;
        }
      }
      j += dj;
      if (j >= npose) {
        j -= npose;
        ++o;
      }
    }
    if (cur >= 0) atomicMin(&skey[cur], best);
    __syncthreads();
  }
  if (!ok) {
    // give copies still in flight a bounded chance to land before the CTA
    // leaves (its shared memory is then released)
    for (int q = 0; q < 2; ++q)
      if ((pending >> q) & 1u) (void)mbar_wait_bounded(&bars[q], (phase >> q) & 1u);
    return false;
  }
  for (int j = threadIdx.x; j < npose; j += blockDim.x)
    if (skey[j] != ~0ull) atomicMin(&keys[pose0 + j], skey[j]);
  return true;
}

#define PSDF_FOR_EACH_M(X) \
  X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

template <bool SOFT>
__global__ void __launch_bounds__(kPlanMaxThreads, 2)
    batched_kernel(const PlanItem *__restrict__ items, int n_items,
                   const PlanBlock *__restrict__ blocks, const FootprintRec *__restrict__ fps,
                   ParamsK prm, const float *__restrict__ poses,
                   const TileHdr *__restrict__ tiles,
                   const unsigned char *__restrict__ blob, int blob_cap,
                   unsigned long long *keys, unsigned *ctr, PlanBounds bnd,
                   unsigned wait_polls)
{
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  FootprintRec *Fs = reinterpret_cast<FootprintRec *>(smem + kPlanSmemHead);
  const FootprintS Fv{Fs->rec, Fs->ivl, Fs->pair};
  unsigned char *buf0 = smem + kPlanSmemHead + kFpBytes;
  __shared__ int s_item;
  __shared__ float4 spose[kPlanMaxThreads];
  __shared__ unsigned long long skey[kPlanMaxThreads];
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  unsigned phase = 0u;
  int cur_inst = -1;
  for (;;) {
    __syncthreads();  // s_item and Fs are free again
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&ctr[0], 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const PlanItem I = items[it];
    if (!PSDF_DBG(I.block >= 0 && I.block < bnd.n_blocks, 1, it)) continue;
    const PlanBlock B = blocks[I.block];
    if (!PSDF_DBG(B.inst >= 0 && B.inst < bnd.n_inst, 2, I.block)) continue;
    if (!PSDF_DBG(B.npose >= 1 && B.npose <= (int)blockDim.x && B.pose0 >= 0 &&
                      B.pose0 + B.npose <= bnd.n_poses,
                  3, I.block))
      continue;
    if (!PSDF_DBG(I.ntile >= 0 && I.tile0 >= 0 && I.tile0 + I.ntile <= bnd.n_tiles, 4, it))
      continue;
    if (B.inst != cur_inst) {
      const int *src = reinterpret_cast<const int *>(fps + B.inst);
      int *dst = reinterpret_cast<int *>(Fs);
      for (int w = threadIdx.x; w < (int)(sizeof(FootprintRec) / 4); w += blockDim.x)
        dst[w] = src[w];
      cur_inst = B.inst;
      __syncthreads();
    }
    bool ok = true;
    switch (Fs->m) {
#define PSDF_SCAN_CASE(MM)                                                                    \
  case MM:                                                                                    \
    ok = scan_item<MM, SOFT>(Fv, prm, poses, B.pose0, B.npose, tiles, blob, I.tile0, I.ntile, \
                       buf0, blob_cap, bars, phase, spose, skey, keys, bnd, wait_polls);      \
    break;
      PSDF_FOR_EACH_M(PSDF_SCAN_CASE)
#undef PSDF_SCAN_CASE
      default:
        (void)PSDF_DBG(false, 5, B.inst);
        break;
    }
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(&ctr[1], 1u);
      break;  // uniform: this CTA stops taking items
    }
  }
}

// Per-pose epilogue of the plan: one thread per pose, its instance's
// footprint read from global memory (an instance's poses are contiguous, so a
// warp rarely mixes footprint sizes).
template <bool SOFT>
__global__ void batched_epilogue_kernel(const int *__restrict__ pose_inst, long long P,
                                        const FootprintK *__restrict__ fps,
                                        const PlanInst *__restrict__ inst, ParamsK prm,
                                        float eps_axis, const float *__restrict__ poses,
                                        const ObsRec *__restrict__ row_obs,
                                        const float4 *__restrict__ vtx,
                                        const int *__restrict__ far,
                                        const unsigned long long *__restrict__ keys,
                                        const unsigned *__restrict__ ctr,
                                        float *__restrict__ phi, float *__restrict__ dphi,
                                        unsigned *__restrict__ active,
                                        float *__restrict__ stage, float d_min, PlanBounds bnd)
{
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int i = pose_inst[p];
  PoseOut r = pose_out_failed();
  if (!PSDF_DBG(i >= 0 && i < bnd.n_inst, 10, p)) {
    write_pose_out(r, p, phi, dphi, active, stage, d_min);
    return;
  }
  const FootprintK &F = fps[i];
  bool checked = true;
#ifdef PSDF_DEBUG_CHECKS
  {
    const unsigned long long key = keys[p];
    if (key != ~0ull) {
      const long long rank = (long long)(key & 0xffffffffu);
      const PlanInst in = inst[i];
      checked = PSDF_DBG(rank < in.rows && in.row0 + rank < bnd.n_rows, 11, p);
      if (checked) {
        const ObsRec o = row_obs[in.row0 + rank];
        checked = PSDF_DBG(o.n >= 1 && o.n <= kMaxObsEdges && o.vtx_global >= 0 &&
                               (long long)o.vtx_global + o.n <= bnd.n_vtx,
                           12, p);
      }
    }
    checked = checked && PSDF_DBG(F.m >= 3 && F.m <= kMaxM, 13, p);
  }
#endif
  if (checked && ctr[1] == 0u) {
    const ObsRec *ro = row_obs + inst[i].row0;
    switch (F.m) {
#define PSDF_EPI_CASE(MM)                                                                  \
  case MM:                                                                                 \
    r = epilogue_pose<MM, SOFT>(F, prm.eps_sat, eps_axis, poses[3 * p], poses[3 * p + 1],  \
                                poses[3 * p + 2], keys[p], ro, vtx, far,                   \
                                dphi != nullptr || stage != nullptr, prm.eta);             \
    break;
      PSDF_FOR_EACH_M(PSDF_EPI_CASE)
#undef PSDF_EPI_CASE
      default: break;
    }
  }
  write_pose_out(r, p, phi, dphi, active, stage, d_min);
}

// Backward: one thread per pose, the instance's footprint read from global
// memory (poses of one instance are contiguous, so warps rarely mix sizes).
template <bool SOFT>
__global__ void batched_backward_kernel(const int *__restrict__ pose_inst, long long P,
                                        const FootprintK *__restrict__ fps,
                                        const PlanInst *__restrict__ inst, ParamsK prm,
                                        float eps_axis,
                                        const float *__restrict__ poses,
                                        const ObsRec *__restrict__ row_obs,
                                        const float4 *__restrict__ vtx,
                                        const int *__restrict__ far,
                                        const unsigned *__restrict__ active,
                                        const float *__restrict__ grad_phi,
                                        float *__restrict__ grad_pose,
                                        float *__restrict__ grad_edges)
{
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int i = pose_inst[p];
  const FootprintK &F = fps[i];
  const PlanInst in = inst[i];
  const float gphi = grad_phi[p];
  if (SOFT) {
    // a penetration pair names a non-separated obstacle: the softmax-weighted
    // sum over the obstacle's axes
    float gp[3];
    bool soft = false;
    const auto edge = [&](float w, const Grad &g) {
      if (!grad_edges) return;
      const float sc = gphi * w;
      for (int r = 0; r < kGradRows; ++r) {
        if (r >= g.nrow) break;
        const long long row = in.row0 + g.row[r];
        atomicAdd(&grad_edges[4 * row + g.col[r]], sc * g.gx[r]);
        atomicAdd(&grad_edges[4 * row + g.col[r] + 1], sc * g.gy[r]);
      }
    };
    switch (F.m) {
#define PSDF_SOFT_BWD_CASE(MM)                                                                \
  case MM:                                                                                    \
    soft = soft_backward_pose<MM>(F, prm.eps_sat, prm.eta, eps_axis, poses[3 * p],            \
                                  poses[3 * p + 1], poses[3 * p + 2], active[p],              \
                                  row_obs + in.row0, in.rows, vtx, far, gp, edge);            \
    break;
      PSDF_FOR_EACH_M(PSDF_SOFT_BWD_CASE)
#undef PSDF_SOFT_BWD_CASE
      default: break;
    }
    if (soft) {
      if (grad_pose) {
        grad_pose[3 * p] = gphi * gp[0];
        grad_pose[3 * p + 1] = gphi * gp[1];
        grad_pose[3 * p + 2] = gphi * gp[2];
      }
      return;
    }
  }
  Grad g;
  bool has = false;
  switch (F.m) {
#define PSDF_BWD_CASE(MM)                                                                  \
  case MM:                                                                                 \
    has = backward_pose<MM>(F, eps_axis, poses[3 * p], poses[3 * p + 1], poses[3 * p + 2], \
                            active[p], row_obs + in.row0, in.rows, vtx, far, g);           \
    break;
    PSDF_FOR_EACH_M(PSDF_BWD_CASE)
#undef PSDF_BWD_CASE
    default: break;
  }
  if (grad_pose) {
    grad_pose[3 * p] = has ? gphi * g.gp[0] : 0.f;
    grad_pose[3 * p + 1] = has ? gphi * g.gp[1] : 0.f;
    grad_pose[3 * p + 2] = has ? gphi * g.gp[2] : 0.f;
  }
  if (has && grad_edges) {
    for (int r = 0; r < kGradRows; ++r) {
      if (r >= g.nrow) break;
      const long long row = in.row0 + g.row[r];
      atomicAdd(&grad_edges[4 * row + g.col[r]], gphi * g.gx[r]);
      atomicAdd(&grad_edges[4 * row + g.col[r] + 1], gphi * g.gy[r]);
    }
  }
}

}  // namespace psdf

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
struct psdf_plan {
  int device = 0;
  int n_inst = 0;
  long long n_poses = 0, n_rows = 0;
  int n_tiles = 0, blob_cap = 16;
  long long n_vtx = 0, blob_total = 0;
  float eps_sat = 0.f, eps_axis = 0.f, eta = 0.f;
  std::vector<long long> inst_pose0, inst_npose;
  std::vector<int> inst_tile0, inst_ntile, inst_m;
  std::vector<int> tile_vtx;  // edges of each tile (work estimate)
  psdf::TileHdr *d_tiles = nullptr;
  unsigned char *d_blob = nullptr;
  float4 *d_vtx = nullptr;
  int *d_far = nullptr;
  psdf::ObsRec *d_row_obs = nullptr;
  psdf::FootprintK *d_fp = nullptr;
  psdf::FootprintRec *d_fprec = nullptr;
  psdf::PlanInst *d_inst = nullptr;
  int *d_pose_inst = nullptr;
  psdf::PlanItem *d_items = nullptr;
  psdf::PlanBlock *d_blocks = nullptr;
  unsigned *d_ctr = nullptr;
  unsigned long long *d_keys = nullptr;
  size_t item_cap = 0, block_cap = 0;
  psdf_plan_config cfg{128, 4};
  int n_items = 0, n_blocks = 0, grid = 0;
  size_t smem = 0;
  size_t device_bytes = 0;
  uint64_t shape_key = 0;
};

namespace psdf {
namespace {

void free_plan(psdf_plan *p)
{
  if (!p) return;
  cudaFree(p->d_tiles);
  cudaFree(p->d_blob);
  cudaFree(p->d_vtx);
  cudaFree(p->d_far);
  cudaFree(p->d_row_obs);
  cudaFree(p->d_fp);
  cudaFree(p->d_fprec);
  cudaFree(p->d_inst);
  cudaFree(p->d_pose_inst);
  cudaFree(p->d_items);
  cudaFree(p->d_blocks);
  cudaFree(p->d_ctr);
  cudaFree(p->d_keys);
  delete p;
}

template <class T>
int dev_alloc(T **dst, size_t n, size_t *bytes)
{
  const size_t nb = std::max<size_t>(n, 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void **)dst, nb);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(plan)");
  *bytes += nb;
  return PSDF_OK;
}

bool valid_config(const psdf_plan_config &c)
{
  return (c.threads == 128 || c.threads == 256) && c.tiles_per_item >= 1 &&
         c.tiles_per_item <= kPlanMaxTilesPerItem;
}

// Work items and pose blocks of a configuration, items by decreasing work.
void build_items(const psdf_plan *pl, const psdf_plan_config &cfg, std::vector<PlanItem> *items,
                 std::vector<PlanBlock> *blocks)
{
  items->clear();
  blocks->clear();
  std::vector<long long> work;
  for (int i = 0; i < pl->n_inst; ++i) {
    const long long np = pl->inst_npose[i];
    const int nt = pl->inst_ntile[i];
    for (long long pb = 0; pb < np; pb += cfg.threads) {
      PlanBlock b{};
      b.pose0 = pl->inst_pose0[i] + pb;
      b.inst = i;
      b.npose = (int)std::min<long long>(cfg.threads, np - pb);
      const int bi = (int)blocks->size();
      if (nt == 0) {
        items->push_back(PlanItem{bi, pl->inst_tile0[i], 0, 0});
        work.push_back(b.npose);
        b.n_items = 1;
      } else {
        for (int t = 0; t < nt; t += cfg.tiles_per_item) {
          const int n = std::min(cfg.tiles_per_item, nt - t);
          long long w = 0;
          for (int q = 0; q < n; ++q) w += pl->tile_vtx[pl->inst_tile0[i] + t + q];
          items->push_back(PlanItem{bi, pl->inst_tile0[i] + t, n, 0});
          work.push_back((long long)b.npose * pl->inst_m[i] * w + b.npose);
          ++b.n_items;
        }
      }
      blocks->push_back(b);
    }
  }
  std::vector<int> order(items->size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
  std::vector<PlanItem> sorted(items->size());
  for (size_t k = 0; k < order.size(); ++k) sorted[k] = (*items)[order[k]];
  items->swap(sorted);
}

int apply_config(psdf_plan *pl, const psdf_plan_config &cfg, cudaStream_t st)
{
  if (!valid_config(cfg))
    return fail(PSDF_ERR_ARG, "plan config: threads must be 128 or 256, tiles_per_item 1..64");
  std::vector<PlanItem> items;
  std::vector<PlanBlock> blocks;
  build_items(pl, cfg, &items, &blocks);
  if (items.size() > pl->item_cap || blocks.size() > pl->block_cap)
    return fail(PSDF_ERR_CAPACITY, "plan work queue capacity exceeded");
  cudaError_t e = cudaSuccess;
  if (!items.empty())
    e = cudaMemcpyAsync(pl->d_items, items.data(), items.size() * sizeof(PlanItem),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !blocks.empty())
    e = cudaMemcpyAsync(pl->d_blocks, blocks.data(), blocks.size() * sizeof(PlanBlock),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "plan work queue upload");
  const size_t smem = kPlanSmemHead + kFpBytes + 2 * (size_t)pl->blob_cap;
  if (smem > 48 * 1024) {
    for (auto k : {batched_kernel<false>, batched_kernel<true>}) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(batched_kernel)");
    }
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, pl->eta > 0.f ? batched_kernel<true> : batched_kernel<false>, cfg.threads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  per_sm = std::max(per_sm, 1);
  pl->cfg = cfg;
  pl->n_items = (int)items.size();
  pl->n_blocks = (int)blocks.size();
  pl->smem = smem;
  pl->grid = (int)std::max<long long>(
      1, std::min<long long>((long long)per_sm * device_sms(), (long long)items.size()));
  return PSDF_OK;
}

PlanBounds plan_bounds(const psdf_plan *pl)
{
  PlanBounds b;
  b.n_poses = pl->n_poses;
  b.n_rows = pl->n_rows;
  b.n_vtx = pl->n_vtx;
  b.blob_bytes = pl->blob_total;
  b.n_items = pl->n_items;
  b.n_blocks = pl->n_blocks;
  b.n_inst = pl->n_inst;
  b.n_tiles = pl->n_tiles;
  return b;
}

int launch_batched(const psdf_plan *pl, const float *poses, float *phi, float *dphi,
                   unsigned *active, cudaStream_t st, const StageOut &so = StageOut())
{
  if (pl->n_items == 0) return PSDF_OK;
  cudaError_t e = cudaMemsetAsync(pl->d_ctr, 0, kCtrWords * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_keys, 0xff, 8 * (size_t)pl->n_poses, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(plan workspace)");
  {
    ProfileScope prof("batched", st);
    const ParamsK pk{pl->eps_sat, pl->eta};
    (pl->eta > 0.f ? batched_kernel<true> : batched_kernel<false>)<<<pl->grid, pl->cfg.threads,
                                                                      pl->smem, st>>>(
        pl->d_items, pl->n_items, pl->d_blocks, pl->d_fprec, pk, poses, pl->d_tiles,
        pl->d_blob, pl->blob_cap, pl->d_keys, pl->d_ctr, plan_bounds(pl), wait_limit());
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch (batched)");
  }
  {
    ProfileScope prof("batched_epilogue", st);
    const long long P = pl->n_poses;
    const ParamsK pk{pl->eps_sat, pl->eta};
    (pl->eta > 0.f ? batched_epilogue_kernel<true>
                   : batched_epilogue_kernel<false>)<<<(unsigned)((P + 127) / 128), 128, 0, st>>>(
        pl->d_pose_inst, P, pl->d_fp, pl->d_inst, pk, pl->eps_axis, poses,
        pl->d_row_obs, pl->d_vtx, pl->d_far, pl->d_keys, pl->d_ctr, phi, dphi, active,
        so.stage, so.d_min, plan_bounds(pl));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch (batched epilogue)");
  }
  return PSDF_OK;
}

uint64_t fnv(uint64_t h, uint64_t v)
{
  for (int b = 0; b < 8; ++b) {
    h ^= (v >> (8 * b)) & 0xffu;
    h *= 1099511628211ull;
  }
  return h;
}

std::mutex g_tune_mu;
std::map<uint64_t, psdf_plan_config> g_tune_cache;

}  // namespace
}  // namespace psdf

using namespace psdf;

extern "C" int psdf_plan_create(int32_t n_inst, const float *footprints,
                                const int32_t *fp_offsets, const float *edges,
                                const int32_t *obs_offsets, const int32_t *inst_obs,
                                const int64_t *pose_offsets, int32_t tile_edges,
                                const psdf_params *params, void *stream, psdf_plan **out)
{
  if (!out) return fail(PSDF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_inst < 0) return fail(PSDF_ERR_ARG, "n_inst < 0");
  if (!params) return fail(PSDF_ERR_ARG, "params is NULL");
  if (!(params->eta >= 0.f) || !std::isfinite(params->eta))
    return fail(PSDF_ERR_ARG, "eta must be finite and >= 0");
  if (!(params->eps_sat >= 0.f)) return fail(PSDF_ERR_ARG, "eps_sat must be >= 0");
  if (n_inst > 0 && (!footprints || !fp_offsets || !obs_offsets || !inst_obs || !pose_offsets))
    return fail(PSDF_ERR_ARG, "NULL array");
  if (n_inst == 0 && (!inst_obs || !pose_offsets || !fp_offsets))
    return fail(PSDF_ERR_ARG, "NULL array");
  if (fp_offsets[0] != 0 || inst_obs[0] != 0 || pose_offsets[0] != 0)
    return fail(PSDF_ERR_LAYOUT, "fp_offsets, inst_obs and pose_offsets must start at 0");
  if (n_inst > 0 && obs_offsets[0] != 0) return fail(PSDF_ERR_LAYOUT, "obs_offsets[0] must be 0");
  for (int i = 0; i < n_inst; ++i) {
    if (fp_offsets[i + 1] < fp_offsets[i] || inst_obs[i + 1] < inst_obs[i] ||
        pose_offsets[i + 1] < pose_offsets[i])
      return fail(PSDF_ERR_LAYOUT, "offsets must be non-decreasing (instance " +
                                       std::to_string(i) + ")");
  }
  const int n_obs = n_inst > 0 ? inst_obs[n_inst] : 0;
  for (int q = 0; q < n_obs; ++q)
    if (obs_offsets[q + 1] < obs_offsets[q])
      return fail(PSDF_ERR_LAYOUT, "obs_offsets must be non-decreasing");
  const long long R = n_obs > 0 ? obs_offsets[n_obs] : 0;
  if (R > 0 && !edges) return fail(PSDF_ERR_ARG, "edges is NULL");
  if (n_inst > 0 && pose_offsets[n_inst] > (1LL << 40))
    return fail(PSDF_ERR_CAPACITY, "too many poses");

  cudaStream_t st = (cudaStream_t)stream;
  psdf_plan *pl = new psdf_plan();
  cudaGetDevice(&pl->device);
  pl->n_inst = n_inst;
  pl->eps_sat = params->eps_sat;
  pl->eta = params->eta;
  pl->eps_axis = params->eps_axis;
  pl->n_poses = n_inst > 0 ? pose_offsets[n_inst] : 0;
  pl->n_rows = R;
  std::vector<TileHdr> tiles;
  std::vector<unsigned char> blob;
  std::vector<float4> vtx;
  std::vector<int> far;
  std::vector<ObsRec> row_obs((size_t)R, ObsRec{0, 0, 0, -1});
  std::vector<FootprintK> fps(n_inst);
  std::vector<PlanInst> pinst(n_inst);
  std::vector<int> pose_inst((size_t)pl->n_poses);
  int max_blob = 0;
  int rc = PSDF_OK;
  for (int i = 0; i < n_inst && !rc; ++i) {
    const int m = fp_offsets[i + 1] - fp_offsets[i];
    rc = make_footprint(footprints + 2 * (size_t)fp_offsets[i], m, params->eps_seg, &fps[i]);
    if (rc) {
      set_error("instance " + std::to_string(i) + ": " + psdf_last_error());
      break;
    }
    const int q0 = inst_obs[i], q1 = inst_obs[i + 1];
    const long long row0 = obs_offsets[q0], row1 = obs_offsets[q1];
    std::vector<ObsIn> obs;
    obs.reserve(q1 - q0);
    for (int q = q0; q < q1; ++q)
      obs.push_back(ObsIn{obs_offsets[q] - row0, obs_offsets[q + 1] - obs_offsets[q]});
    HostScene hs;
    rc = build_host_scene(edges ? edges + 4 * row0 : nullptr, row1 - row0, obs, tile_edges, params,
                          &hs);
    if (rc) {
      set_error("instance " + std::to_string(i) + ": " + psdf_last_error());
      break;
    }
    const int tile0 = (int)tiles.size();
    const long long vbase = (long long)vtx.size() / 2;
    const int bbase = (int)blob.size();
    if ((long long)blob.size() + hs.blob.size() > (1LL << 31) - 1 ||
        vbase + (long long)hs.vtx.size() / 2 > (1LL << 31) - 1) {
      rc = fail(PSDF_ERR_CAPACITY, "plan too large (blob or vertex records above 2^31)");
      break;
    }
    for (TileHdr h : hs.tiles) {
      h.blob_off += bbase;
      tiles.push_back(h);
      pl->tile_vtx.push_back(h.n_vtx);
    }
    blob.insert(blob.end(), hs.blob.begin(), hs.blob.end());
    vtx.insert(vtx.end(), hs.vtx.begin(), hs.vtx.end());
    far.insert(far.end(), hs.far.begin(), hs.far.end());
    for (long long r = 0; r < row1 - row0; ++r) {
      ObsRec o = hs.row_obs[r];
      if (o.n > 0) {
        o.vtx_global += (int)vbase;
        o.tile += tile0;
      }
      row_obs[row0 + r] = o;
    }
    max_blob = std::max(max_blob, hs.max_blob);
    pinst[i] = PlanInst{row0, row1 - row0};
    pl->inst_pose0.push_back(pose_offsets[i]);
    pl->inst_npose.push_back(pose_offsets[i + 1] - pose_offsets[i]);
    pl->inst_tile0.push_back(tile0);
    pl->inst_ntile.push_back(hs.T);
    pl->inst_m.push_back(m);
    for (long long p = pose_offsets[i]; p < pose_offsets[i + 1]; ++p) pose_inst[p] = i;
  }
  if (rc) {
    free_plan(pl);
    return rc;
  }
  pl->n_tiles = (int)tiles.size();
  pl->n_vtx = (long long)vtx.size() / 2;
  pl->blob_total = (long long)blob.size();
  pl->blob_cap = std::max(16, (max_blob + 15) / 16 * 16);
  // capacity: the configuration with the most items and blocks
  size_t icap = 0, bcap = 0;
  for (int i = 0; i < n_inst; ++i) {
    const long long nb = (pl->inst_npose[i] + 127) / 128;
    bcap += nb;
    icap += nb * std::max(1, pl->inst_ntile[i]);
  }
  pl->item_cap = icap;
  pl->block_cap = bcap;
  size_t *db = &pl->device_bytes;
  if (!rc) rc = dev_upload(&pl->d_tiles, tiles, st, db);
  if (!rc) rc = dev_upload(&pl->d_blob, blob, st, db);
  if (!rc) rc = dev_upload(&pl->d_vtx, vtx, st, db);
  if (!rc) rc = dev_upload(&pl->d_far, far, st, db);
  if (!rc) rc = dev_upload(&pl->d_row_obs, row_obs, st, db);
  std::vector<FootprintRec> fprec(n_inst);
  for (int i = 0; i < n_inst; ++i) {
    FootprintRec &r = fprec[i];
    std::memset(&r, 0, sizeof(r));
    const FootprintK &F = fps[i];
    for (int l = 0; l < F.m; ++l) {
      r.rec[2 * l] = make_float4(F.vx[l], F.vy[l], F.ex[l], F.ey[l]);
      r.rec[2 * l + 1] = make_float4(F.inv_e2[l], F.nx[l], F.ny[l], 0.f);
      r.ivl[l] = make_float2(F.alo[l], F.ahi[l]);
    }
    for (int q = 0; q < F.m / 2; ++q) {
      const int a = 2 * q, b = 2 * q + 1;
      r.pair[4 * q] = make_float4(F.vx[a], F.vx[b], F.vy[a], F.vy[b]);
      r.pair[4 * q + 1] = make_float4(F.ex[a], F.ex[b], F.ey[a], F.ey[b]);
      r.pair[4 * q + 2] = make_float4(-F.inv_e2[a], -F.inv_e2[b], F.nx[a], F.nx[b]);
      r.pair[4 * q + 3] = make_float4(F.ny[a], F.ny[b], 0.f, 0.f);
    }
    r.m = F.m;
  }
  if (!rc) rc = dev_upload(&pl->d_fp, fps, st, db);
  if (!rc) rc = dev_upload(&pl->d_fprec, fprec, st, db);
  if (!rc) rc = dev_upload(&pl->d_inst, pinst, st, db);
  if (!rc) rc = dev_upload(&pl->d_pose_inst, pose_inst, st, db);
  if (!rc) rc = dev_alloc(&pl->d_items, icap, db);
  if (!rc) rc = dev_alloc(&pl->d_blocks, bcap, db);
  if (!rc) rc = dev_alloc(&pl->d_ctr, kCtrWords, db);
  if (!rc) rc = dev_alloc(&pl->d_keys, (size_t)pl->n_poses, db);
  if (!rc) {
    cudaError_t e = cudaMemsetAsync(pl->d_ctr, 0, kCtrWords * sizeof(unsigned), st);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync(plan counters)");
  }
  if (!rc) {
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, (uint64_t)device_sms());
    h = fnv(h, (uint64_t)n_inst);
    h = fnv(h, (uint64_t)(pl->eta > 0.f));  // the soft minimum's kernel times differently
    for (int i = 0; i < n_inst; ++i) {
      h = fnv(h, (uint64_t)pl->inst_npose[i]);
      h = fnv(h, (uint64_t)pl->inst_ntile[i]);
      h = fnv(h, (uint64_t)pl->inst_m[i]);
    }
    pl->shape_key = h;
    // default: 128 threads, about 1 K edges per item
    rc = apply_config(pl, psdf_plan_config{128, 4}, st);
  }
  if (rc) {
    free_plan(pl);
    return rc;
  }
  *out = pl;
  return PSDF_OK;
}

extern "C" int psdf_plan_debug_read(uint64_t *violation, int32_t *enabled)
{
  if (!violation || !enabled) return fail(PSDF_ERR_ARG, "NULL argument");
  *violation = 0;
#ifdef PSDF_DEBUG_CHECKS
  *enabled = 1;
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_plan_debug, sizeof(v));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyFromSymbol(debug word)");
  *violation = v;
#else
  *enabled = 0;
#endif
  return PSDF_OK;
}

extern "C" int psdf_plan_destroy(psdf_plan *plan)
{
  free_plan(plan);
  return PSDF_OK;
}

extern "C" int psdf_plan_get_info(const psdf_plan *plan, psdf_plan_info *info)
{
  if (!plan || !info) return fail(PSDF_ERR_ARG, "NULL argument");
  info->n_inst = plan->n_inst;
  info->n_tiles = plan->n_tiles;
  info->n_poses = plan->n_poses;
  info->n_rows = plan->n_rows;
  info->n_items = plan->n_items;
  info->n_blocks = plan->n_blocks;
  info->grid = plan->grid;
  info->reserved = 0;
  info->config = plan->cfg;
  info->device_bytes = plan->device_bytes;
  return PSDF_OK;
}

extern "C" int psdf_plan_set_config(psdf_plan *plan, const psdf_plan_config *config,
                                    void *stream)
{
  if (!plan || !config) return fail(PSDF_ERR_ARG, "NULL argument");
  return apply_config(plan, *config, (cudaStream_t)stream);
}

extern "C" int psdf_eval_batched(psdf_plan *plan, const float *poses, float *phi, float *dphi,
                                 uint32_t *active, void *stream)
{
  if (!plan) return fail(PSDF_ERR_ARG, "plan is NULL");
  if (plan->n_poses > 0 && (!poses || !phi)) return fail(PSDF_ERR_ARG, "poses or phi is NULL");
  return launch_batched(plan, poses, phi, dphi, active, (cudaStream_t)stream);
}

extern "C" int psdf_stage_params_batched(psdf_plan *plan, const float *poses, float d_min,
                                         float *stage, uint32_t *active, void *stream)
{
  if (!plan) return fail(PSDF_ERR_ARG, "plan is NULL");
  if (plan->n_poses > 0 && (!poses || !stage)) return fail(PSDF_ERR_ARG, "poses or stage is NULL");
  if (!std::isfinite(d_min)) return fail(PSDF_ERR_ARG, "d_min must be finite");
  StageOut so;
  so.stage = stage;
  so.d_min = d_min;
  return launch_batched(plan, poses, nullptr, nullptr, active, (cudaStream_t)stream, so);
}

extern "C" int psdf_plan_status(const psdf_plan *plan, void *stream)
{
  if (!plan) return fail(PSDF_ERR_ARG, "plan is NULL");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  unsigned c[kCtrWords] = {0u, 0u};
  e = cudaMemcpy(c, plan->d_ctr, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(plan counters)");
  if (c[1]) return fail(PSDF_ERR_TIMEOUT, "a bounded device-side wait ran out");
  return PSDF_OK;
}

extern "C" int psdf_plan_autotune(psdf_plan *plan, const float *poses, int32_t reps,
                                  void *stream, psdf_plan_config *chosen, int32_t *from_cache)
{
  if (!plan) return fail(PSDF_ERR_ARG, "plan is NULL");
  if (plan->n_poses > 0 && !poses) return fail(PSDF_ERR_ARG, "poses is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (from_cache) *from_cache = 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(plan->shape_key);
    if (it != g_tune_cache.end()) {
      int rc = apply_config(plan, it->second, st);
      if (rc) return rc;
      if (chosen) *chosen = plan->cfg;
      if (from_cache) *from_cache = 1;
      return PSDF_OK;
    }
  }
  reps = std::max(1, std::min(reps, 100));
  float *d_phi = nullptr, *d_dphi = nullptr;
  unsigned *d_act = nullptr;
  size_t scratch = 0;
  int rc = dev_alloc(&d_phi, (size_t)plan->n_poses, &scratch);
  if (!rc) rc = dev_alloc(&d_dphi, 3 * (size_t)plan->n_poses, &scratch);
  if (!rc) rc = dev_alloc(&d_act, (size_t)plan->n_poses, &scratch);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = fail(PSDF_ERR_CUDA, "cudaEventCreate");
  psdf_plan_config best{0, 0};
  float best_ms = 0.f;
  const int thr[2] = {128, 256};
  const int tpi[6] = {1, 2, 4, 8, 16, 32};
  for (int a = 0; a < 2 && !rc; ++a)
    for (int b = 0; b < 6 && !rc; ++b) {
      const psdf_plan_config c{thr[a], tpi[b]};
      rc = apply_config(plan, c, st);
      if (!rc) rc = launch_batched(plan, poses, d_phi, d_dphi, d_act, st);  // warm-up
      if (!rc && cudaEventRecord(e0, st) != cudaSuccess) rc = fail(PSDF_ERR_CUDA, "event");
      for (int r = 0; r < reps && !rc; ++r)
        rc = launch_batched(plan, poses, d_phi, d_dphi, d_act, st);
      if (!rc && cudaEventRecord(e1, st) != cudaSuccess) rc = fail(PSDF_ERR_CUDA, "event");
      if (!rc) {
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = cuda_fail(e, "autotune timing");
        else if (best.threads == 0 || ms < best_ms) {
          best = c;
          best_ms = ms;
        }
      }
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_phi);
  cudaFree(d_dphi);
  cudaFree(d_act);
  if (rc) return rc;
  rc = apply_config(plan, best, st);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[plan->shape_key] = best;
  }
  if (chosen) *chosen = best;
  return PSDF_OK;
}

extern "C" int psdf_backward_batched(const psdf_plan *plan, const float *poses,
                                     const uint32_t *active, const float *grad_phi,
                                     float *grad_pose, float *grad_edges, void *stream)
{
  if (!plan) return fail(PSDF_ERR_ARG, "plan is NULL");
  if (plan->n_poses == 0) return PSDF_OK;
  if (!poses || !active || !grad_phi) return fail(PSDF_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  ProfileScope prof("batched_backward", st);
  const long long P = plan->n_poses;
  const ParamsK pk{plan->eps_sat, plan->eta};
  (plan->eta > 0.f ? batched_backward_kernel<true>
                   : batched_backward_kernel<false>)<<<(unsigned)((P + 127) / 128), 128, 0, st>>>(
      plan->d_pose_inst, P, plan->d_fp, plan->d_inst, pk, plan->eps_axis, poses, plan->d_row_obs,
      plan->d_vtx, plan->d_far, active, grad_phi, grad_pose, grad_edges);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch (batched backward)");
}
