// PSDF_Forward / PSDF_Backward (Alg. 1) on sm_103a.
//
// Full-scan forward: grid = (pose blocks of 128) x (chunks of edge tiles).
// One thread owns one pose; the CTA streams its chunk of obstacle-contiguous
// edge tiles through shared memory with bulk asynchronous copies (TMA,
// cp.async.bulk + mbarrier, double-buffered).  Every lane reads the same
// edge record at the same time (shared-memory broadcast) and keeps all
// per-obstacle reductions (min distance, SAT intervals, min overlap) in
// registers, so no shuffles are needed inside the hot loop.  The per-pose
// result is a 64-bit min-key (ordered value, obstacle rank) merged across
// CTAs with one atomicMin per pose per CTA.  A per-pose epilogue re-derives
// the active pair of the winning obstacle and its closed-form gradient.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "profile.h"
#include "psdf_device.cuh"
#include "psdf_internal.h"
#include "tma.cuh"

namespace psdf {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int fail(int code, const std::string &msg)
{
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return PSDF_ERR_CUDA;
}

constexpr int kScanThreads = 128;

static std::atomic<unsigned> g_wait_limit{kWaitLimit};
unsigned wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__global__ void init_keys_kernel(unsigned long long *keys, long long P, int *err)
{
  pdl_trigger();  // the scan may launch now; it waits for this grid before its atomics
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) keys[i] = ~0ull;
  if (i == 0) *err = 0;
}

// Full scan: each CTA = a block of npb poses x tiles [t0, t1).  With npb =
// kScanThreads every lane owns one pose; a smaller batch (npb < kScanThreads)
// splits each tile's obstacles over S = kScanThreads / npb lanes per pose
// (lane l: pose l % npb, obstacle range l / npb), so that a short horizon
// still fills the CTA and each lane's chain stays short.
template <int M, bool SOFT = false>
__global__ void __launch_bounds__(kScanThreads) scan_kernel(
    FootprintK F, ParamsK prm, const float *__restrict__ poses, long long P, int npb,
    const TileHdr *__restrict__ tiles, const unsigned char *__restrict__ blob, int n_tiles,
    int tiles_per_chunk, int blob_cap, unsigned long long *__restrict__ keys,
    int *__restrict__ err, unsigned wait_polls)
{
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  unsigned char *const buf0 = smem + 128;  // buffer b lives at buf0 + b * blob_cap

  const int t0 = blockIdx.y * tiles_per_chunk;
  const int t1 = min(n_tiles, t0 + tiles_per_chunk);
  if (t0 >= t1) return;  // uniform over the CTA

  const int S = kScanThreads / npb;
  const int part = threadIdx.x / npb;
  const long long p = (long long)blockIdx.x * npb + threadIdx.x % npb;
  const bool live = p < P && part < S;
  float px = 0.f, py = 0.f, c = 1.f, s = 0.f;
  if (live) {
    px = poses[3 * p];
    py = poses[3 * p + 1];
    sincosf(poses[3 * p + 2], &s, &c);
  }
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const TileHdr h = tiles[t0];
    mbar_arrive_expect_tx(&bars[0], (unsigned)h.blob_bytes);
    bulk_g2s(buf0, blob + h.blob_off, (unsigned)h.blob_bytes, &bars[0]);
  }
  unsigned pending = 1u;  // bit b: a copy into buffer b is in flight
  unsigned phase = 0u;    // bit b: parity of buffer b's next completion
  unsigned long long best = ~0ull;
  bool ok = true;
  for (int t = t0; t < t1; ++t) {
    const int b = (t - t0) & 1;
    if (t + 1 < t1) {
      if (threadIdx.x == 0) {
        const TileHdr hn = tiles[t + 1];
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
    const TileHdr h = tiles[t];
    const unsigned char *tb = buf0 + b * blob_cap;
    const int4 *ob = reinterpret_cast<const int4 *>(tb);
    const float4 *vt = reinterpret_cast<const float4 *>(tb + 16 * h.n_obs);
    // lanes beyond the S ranges (part >= S) take an empty range
    const int o0 = part >= S ? 0 : (S == 1 ? 0 : h.n_obs * part / S);
    const int o1 = part >= S ? 0 : (S == 1 ? h.n_obs : h.n_obs * (part + 1) / S);
    for (int o = o0; o < o1; ++o) {
      const int4 rec = ob[o];
      const float v = obstacle_value<M, FootprintK, SOFT>(F, px, py, c, s, vt + 2 * rec.x, rec.y,
                                                          prm.eps_sat, prm.eta);
      const unsigned long long key = pack_key(v, rec.z);
      best = key < best ? key : best;
    }
    __syncthreads();
  }
  // the keys and the error word are initialised by the kernel before this
  // one (launched programmatically behind it): wait for it before merging
  pdl_wait();
  pdl_trigger();  // the epilogue may launch; it waits for this grid
  if (!ok) {
    // record the failure, then give copies still in flight a bounded chance
    // to land before the CTA's shared memory is released
    if (threadIdx.x == 0) atomicOr(err, 1);
    for (int q = 0; q < 2; ++q)
      if ((pending >> q) & 1u) (void)mbar_wait_bounded(&bars[q], (phase >> q) & 1u);
    return;
  }
  if (live && best != ~0ull) atomicMin(&keys[p], best);
}

constexpr int kEpiLanes = 4;  // lanes sharing one pose's epilogue (hard minimum)
// Lanes per pose in the backward (one of them works): a whole warp per pose
// while the launch stays within about two waves of the GPU's threads (the
// kernel is a chain of dependent loads and a per-kind branch, so fewer poses
// per warp shorten it), fewer lanes for larger batches.
inline int backward_spread_shift(long long P)
{
  const long long budget = 2LL * device_sms() * 2048;
  int shift = 5;
  while (shift > 0 && (P << shift) > budget) --shift;
  return shift;
}

// Per-pose epilogue: value, active pair, optional pose gradient; SAVE (hard
// minimum) also writes the saved backward records.
template <int M, bool SOFT = false, bool SAVE = false>
__global__ void epilogue_kernel(FootprintK F, ParamsK prm, float eps_axis,
                                const float *__restrict__ poses, long long P,
                                const ObsRec *__restrict__ row_obs,
                                const float4 *__restrict__ vtx, const int *__restrict__ far,
                                const unsigned long long *__restrict__ keys,
                                const int *__restrict__ err, float *__restrict__ phi,
                                float *__restrict__ dphi, unsigned *__restrict__ active,
                                float *__restrict__ stage, float d_min,
                                float4 *__restrict__ saved)
{
  // the pose (an input of the call, not an output of the kernel before) is
  // read before the wait
  float px = 0.f, py = 0.f, th = 0.f;
  if (!SOFT) {
    const long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kEpiLanes;
    if (p < P) {
      px = poses[3 * p];
      py = poses[3 * p + 1];
      th = poses[3 * p + 2];
    }
  }
  pdl_wait();
  pdl_trigger();  // a following backward may launch now; it waits for this grid
  const bool want_grad = SAVE || dphi != nullptr || stage != nullptr;
  if constexpr (SOFT) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    PoseOut r;
    if (*err) {
      r = pose_out_failed();
    } else {
      r = epilogue_pose<M, true>(F, prm.eps_sat, eps_axis, poses[3 * p], poses[3 * p + 1],
                                 poses[3 * p + 2], keys[p], row_obs, vtx, far, want_grad,
                                 prm.eta);
    }
    write_pose_out(r, p, phi, dphi, active, stage, d_min);
  } else {
    // kEpiLanes lanes per pose, every lane of the block through the shared
    // detail (no early exit before it)
    const long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kEpiLanes;
    const int g = (int)(threadIdx.x % kEpiLanes);
    const bool valid = p < P;
    PoseOut r;
    Grad rows;
    rows.nrow = -1;
    if (*err) {
      r = pose_out_failed();
    } else {
      r = epilogue_pose_coop<M, kEpiLanes>(F, prm.eps_sat, eps_axis, px, py, th,
                                           valid ? keys[p] : ~0ull, row_obs, vtx, far,
                                           want_grad, g, SAVE ? &rows : nullptr);
    }
    if (valid && g == 0) {
      write_pose_out(r, p, phi, dphi, active, stage, d_min);
      if constexpr (SAVE) write_saved(saved, p, rows);
    }
  }
}

// Launch shape of the epilogue: hard minimum kEpiLanes lanes per pose in
// blocks of 128, soft minimum one thread per pose in blocks of 64.
inline dim3 epilogue_blocks(long long P, bool soft)
{
  return soft ? dim3((unsigned)((P + 63) / 64)) : dim3((unsigned)((P * kEpiLanes + 127) / 128));
}
inline dim3 epilogue_threads(bool soft) { return soft ? dim3(64) : dim3(128); }

template <int M, bool SOFT = false>
__global__ void backward_kernel(FootprintK F, ParamsK prm, float eps_axis,
                                const float *__restrict__ poses, long long P,
                                const ObsRec *__restrict__ row_obs,
                                const float4 *__restrict__ vtx, const int *__restrict__ far,
                                long long rows_total,
                                const unsigned *__restrict__ active,
                                const float *__restrict__ grad_phi, float *__restrict__ grad_pose,
                                float *__restrict__ grad_edges, int spread)
{
  // one pose per 2^spread lanes: fewer poses (and active-pair kinds, whose
  // gradient branches a warp runs one after another) per warp
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid & ((1LL << spread) - 1)) return;
  const long long p = gid >> spread;
  if (p >= P) return;
  // the pose is read before the wait: it is an input of the call, never an
  // output of the epilogue that usually precedes this kernel (the active
  // pair and the incoming gradient may be, so they are read after it)
  const float px = poses[3 * p], py = poses[3 * p + 1], th = poses[3 * p + 2];
  pdl_wait();
  const float gphi = grad_phi[p];
  const unsigned pid = active[p];
  if (SOFT) {
    // a penetration pair names a non-separated obstacle: its gradient is the
    // softmax-weighted sum over the obstacle's axes
    float gp[3];
    if (soft_backward_pose<M>(F, prm.eps_sat, prm.eta, eps_axis, px, py, th, pid, row_obs,
                              rows_total, vtx, far, gp, [&](float w, const Grad &g) {
                                if (!grad_edges) return;
                                const float sc = gphi * w;
                                for (int i = 0; i < kGradRows; ++i) {
                                  if (i >= g.nrow) break;
                                  atomicAdd(&grad_edges[4 * (long long)g.row[i] + g.col[i]],
                                            sc * g.gx[i]);
                                  atomicAdd(&grad_edges[4 * (long long)g.row[i] + g.col[i] + 1],
                                            sc * g.gy[i]);
                                }
                              })) {
      if (grad_pose) {
        grad_pose[3 * p] = gphi * gp[0];
        grad_pose[3 * p + 1] = gphi * gp[1];
        grad_pose[3 * p + 2] = gphi * gp[2];
      }
      return;
    }
  }
  Grad g;
  const bool has = backward_pose<M>(F, eps_axis, px, py, th, pid, row_obs, rows_total, vtx, far,
                                    g);
  if (grad_pose) {
    grad_pose[3 * p] = has ? gphi * g.gp[0] : 0.f;
    grad_pose[3 * p + 1] = has ? gphi * g.gp[1] : 0.f;
    grad_pose[3 * p + 2] = has ? gphi * g.gp[2] : 0.f;
  }
  if (has && grad_edges) {
    for (int i = 0; i < kGradRows; ++i) {
      if (i >= g.nrow) break;
      atomicAdd(&grad_edges[4 * (long long)g.row[i] + g.col[i]], gphi * g.gx[i]);
      atomicAdd(&grad_edges[4 * (long long)g.row[i] + g.col[i] + 1], gphi * g.gy[i]);
    }
  }
}

// Backward from the forward's saved records (psdf_backward_saved): the pose
// gradient and the edge-endpoint rows scaled by the incoming gradient, the
// same products the recomputing backward forms.  One thread per pose; a row
// whose two columns do not both lie in [0, 4 rows_total) is skipped.
__global__ void backward_saved_kernel(const float4 *__restrict__ saved, long long P,
                                      long long rows_total, const float *__restrict__ grad_phi,
                                      float *__restrict__ grad_pose,
                                      float *__restrict__ grad_edges)
{
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // a cache hint while the forward finishes (a prefetch reads nothing the
  // kernel uses before the wait): the incoming gradient's lines.  (The edge
  // gradients the atomics below update are not prefetched: a bulk prefetch
  // of the whole buffer competes with a short forward's first reads, which
  // measured slower on the culled step than the atomics' own misses.)
  if (p < P && (threadIdx.x & 31) == 0)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(grad_phi + p));
  pdl_wait();  // the records may come from the epilogue just before
  if (p >= P) return;
  const float gphi = grad_phi[p];
  float w[16];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 v = saved[4 * p + q];
    w[4 * q] = v.x;
    w[4 * q + 1] = v.y;
    w[4 * q + 2] = v.z;
    w[4 * q + 3] = v.w;
  }
  const int nrow = __float_as_int(w[3]);
  const bool has = nrow >= 0;
  if (grad_pose) {
    grad_pose[3 * p] = has ? gphi * w[0] : 0.f;
    grad_pose[3 * p + 1] = has ? gphi * w[1] : 0.f;
    grad_pose[3 * p + 2] = has ? gphi * w[2] : 0.f;
  }
  if (!grad_edges) return;
#pragma unroll
  for (int i = 0; i < kGradRows; ++i) {
    const int idx = __float_as_int(w[4 + 3 * i]);
    if (i < nrow && idx >= 0 && idx + 1 < 4 * rows_total) {
      atomicAdd(&grad_edges[idx], gphi * w[5 + 3 * i]);
      atomicAdd(&grad_edges[idx + 1], gphi * w[6 + 3 * i]);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

struct DeviceInfo {
  int sms = 0;
};

DeviceInfo device_info_impl()
{
  static std::mutex mu;
  static std::vector<DeviceInfo> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if ((int)cache.size() <= dev) cache.resize(dev + 1);
  if (cache[dev].sms == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev].sms = v > 0 ? v : 1;
  }
  return cache[dev];
}

}  // namespace

int device_sms() { return device_info_impl().sms; }

// Footprint validation (Assumption 1) and constants.
int make_footprint(const float *fp, int m, float eps_seg, FootprintK *F)
{
  if (!fp) return fail(PSDF_ERR_ARG, "footprint is NULL");
  if (m < 3 || m > kMaxM)
    return fail(PSDF_ERR_FOOTPRINT, "footprint must have 3..16 vertices, got " + std::to_string(m));
  std::memset(F, 0, sizeof(*F));
  F->m = m;
  double turn = 0.0, rad = 0.0;
  for (int l = 0; l < m; ++l) {
    if (!std::isfinite(fp[2 * l]) || !std::isfinite(fp[2 * l + 1]))
      return fail(PSDF_ERR_FOOTPRINT, "footprint has a non-finite vertex");
    const int ln = (l + 1) % m, l2 = (l + 2) % m;
    const float ex = fp[2 * ln] - fp[2 * l], ey = fp[2 * ln + 1] - fp[2 * l + 1];
    const float fx = fp[2 * l2] - fp[2 * ln], fy = fp[2 * l2 + 1] - fp[2 * ln + 1];
    const double len = std::sqrt((double)ex * ex + (double)ey * ey);
    if (len < 1e-6) return fail(PSDF_ERR_FOOTPRINT, "footprint edge shorter than 1e-6 m");
    const double cr = (double)ex * fy - (double)ey * fx, dt = (double)ex * fx + (double)ey * fy;
    if (!(cr > 0.0))
      return fail(PSDF_ERR_FOOTPRINT, "footprint is not strictly convex counter-clockwise");
    turn += std::atan2(cr, dt);
    F->vx[l] = fp[2 * l];
    F->vy[l] = fp[2 * l + 1];
    F->ex[l] = ex;
    F->ey[l] = ey;
    F->inv_e2[l] = (float)(1.0 / ((double)ex * ex + (double)ey * ey + eps_seg));
    F->nx[l] = (float)(ey / len);
    F->ny[l] = (float)(-ex / len);
    rad = std::max(rad, std::sqrt((double)fp[2 * l] * fp[2 * l] + (double)fp[2 * l + 1] * fp[2 * l + 1]));
  }
  if (std::fabs(turn - 2.0 * M_PI) > 1e-6)
    return fail(PSDF_ERR_FOOTPRINT, "footprint does not turn exactly once");
  for (int l = 0; l < m; ++l) {
    double lo = INFINITY, hi = -INFINITY;
    for (int q = 0; q < m; ++q) {
      const double pr = (double)F->vx[q] * F->nx[l] + (double)F->vy[q] * F->ny[l];
      lo = std::min(lo, pr);
      hi = std::max(hi, pr);
    }
    F->alo[l] = (float)lo;
    F->ahi[l] = (float)hi;
  }
  F->radius = (float)(rad * (1.0 + 1e-6));
  // the largest disc about the pose inside the footprint: the smallest
  // distance from the pose to an edge line (all positive iff the pose lies
  // inside), rounded down
  double inner = INFINITY;
  for (int l = 0; l < m; ++l)
    inner = std::min(inner, (double)F->vx[l] * F->nx[l] + (double)F->vy[l] * F->ny[l]);
  F->inner = inner > 1e-6 ? (float)(inner * (1.0 - 1e-5) - 1e-7) : -1.f;
  return PSDF_OK;
}

int check_eval_args(const psdf_scene *scene, const float *poses, int64_t P,
                    const psdf_params *params, void *workspace, size_t ws_bytes)
{
  if (!scene) return fail(PSDF_ERR_ARG, "scene is NULL");
  if (P < 0) return fail(PSDF_ERR_ARG, "P < 0");
  if (P > ((int64_t)1 << 40)) return fail(PSDF_ERR_CAPACITY, "P too large");
  if (P > 0 && !poses) return fail(PSDF_ERR_ARG, "poses is NULL");
  if (!params) return fail(PSDF_ERR_ARG, "params is NULL");
  if (params->eps_seg != scene->eps_seg || params->eps_axis != scene->eps_axis)
    return fail(PSDF_ERR_ARG,
                "params eps_seg/eps_axis differ from the values the scene was prepared with");
  if (!(params->eps_sat >= 0.f)) return fail(PSDF_ERR_ARG, "eps_sat must be >= 0");
  if (!(params->eta >= 0.f) || !std::isfinite(params->eta))
    return fail(PSDF_ERR_ARG, "eta must be finite and >= 0 (0 = hard minimum)");
  if (P > 0) {
    if (!workspace) return fail(PSDF_ERR_ARG, "workspace is NULL");
    if (((uintptr_t)workspace & 255u) != 0) return fail(PSDF_ERR_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < psdf_workspace_bytes(P))
      return fail(PSDF_ERR_CAPACITY, "workspace smaller than psdf_workspace_bytes(P)");
  }
  // device memory, managed memory, or pinned host memory mapped into the
  // device's address space at the same address (read across the host link)
  cudaPointerAttributes attr;
  if (P > 0 && cudaPointerGetAttributes(&attr, poses) == cudaSuccess &&
      attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged &&
      !(attr.type == cudaMemoryTypeHost && attr.devicePointer == (const void *)poses))
    return fail(PSDF_ERR_ARG, "poses must be device memory or device-mapped pinned host memory");
  cudaGetLastError();
  return PSDF_OK;
}

// ---------------------------------------------------------------------------
// scene parts: keys with a row offset, their minimum, the owner's epilogue
// ---------------------------------------------------------------------------
// Adds row_offset to the rank of every key that names an obstacle, so that
// keys of scene parts whose rows are consecutive ranges of one numbering
// compare as keys of the whole scene.  Waits for the scan (programmatic).
__global__ void offset_keys_kernel(unsigned long long *keys, long long P, unsigned row_offset)
{
  pdl_wait();
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P && keys[p] != ~0ull) keys[p] += row_offset;
}

// b[p] = min(a[p], b[p]).
__global__ void merge_keys_kernel(const unsigned long long *__restrict__ a,
                                  unsigned long long *__restrict__ b, long long P)
{
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P) b[p] = a[p] < b[p] ? a[p] : b[p];
}

// Epilogue of the poses whose (merged) key names an obstacle of this scene
// part, rows [row_offset, row_offset + rows), or names none when own_empty;
// the other poses' outputs are left as they are.  The active pair's edge is
// reported in the whole scene's numbering.  Hard minimum: kEpiLanes lanes a
// pose (every lane through the shared detail); soft minimum: one thread.
template <int M, bool SOFT>
__global__ void finish_keys_kernel(FootprintK F, ParamsK prm, float eps_axis,
                                   const float *__restrict__ poses, long long P,
                                   const ObsRec *__restrict__ row_obs,
                                   const float4 *__restrict__ vtx, const int *__restrict__ far,
                                   const unsigned long long *__restrict__ keys,
                                   long long row_offset, long long rows, int own_empty,
                                   float *__restrict__ phi, float *__restrict__ dphi,
                                   unsigned *__restrict__ active)
{
  const int lanes = SOFT ? 1 : kEpiLanes;
  const long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / lanes;
  const int g = (int)(threadIdx.x % lanes);
  bool own = false;
  unsigned long long key = ~0ull;
  if (p < P) {
    key = keys[p];
    if (key == ~0ull) {
      own = own_empty != 0;
    } else {
      const long long rank = (long long)(key & 0xffffffffull);
      own = rank >= row_offset && rank < row_offset + rows;
      key = own ? key - (unsigned long long)row_offset : ~0ull;
    }
  }
  float px = 0.f, py = 0.f, th = 0.f;
  if (p < P) {
    px = poses[3 * p];
    py = poses[3 * p + 1];
    th = poses[3 * p + 2];
  }
  const bool want_grad = dphi != nullptr;
  PoseOut r;
  if constexpr (SOFT) {
    if (!own) return;
    r = epilogue_pose<M, true>(F, prm.eps_sat, eps_axis, px, py, th, key, row_obs, vtx, far,
                               want_grad, prm.eta);
  } else {
    r = epilogue_pose_coop<M, kEpiLanes>(F, prm.eps_sat, eps_axis, px, py, th,
                                         own ? key : ~0ull, row_obs, vtx, far, want_grad, g);
    if (!own || g != 0) return;
  }
  if (r.pid != PSDF_PAIR_NONE) r.pid += (unsigned)row_offset << kPairShiftEdge;
  write_pose_out(r, p, phi, dphi, active, nullptr, 0.f);
}

// Keys of every pose over the scene's tiles: key initialisation + the full
// scan (its atomicMin merges into keys[]); err receives a timed-out wait.
template <int M>
static int launch_scan(const FootprintK &F, const psdf_scene *sc, const float *poses, long long P,
                       const ParamsK &pk, unsigned long long *keys, int *err, cudaStream_t st)
{
  const int init_blocks = (int)((P + 255) / 256);
  init_keys_kernel<<<init_blocks, 256, 0, st>>>(keys, P, err);
  if (sc->n_tiles > 0) {
    const DeviceInfo di = device_info_impl();
    // a small launch (fewer pose blocks x tiles than SMs) splits each tile's
    // obstacles over more lanes per pose: halve the poses per CTA (down to 8)
    // until the grid covers the GPU
    int npb = P < kScanThreads ? (int)P : kScanThreads;
    while (npb > 8 && ((P + npb - 1) / npb) * sc->n_tiles < di.sms) npb = (npb + 1) / 2;
    const long long pose_blocks = (P + npb - 1) / npb;
    if (pose_blocks > 2147483647LL) return fail(PSDF_ERR_CAPACITY, "too many poses for one launch");
    // aim for about 32 CTAs per SM in total (several waves of resident CTAs)
    const long long target = (long long)di.sms * 32;
    long long tpc = (pose_blocks * sc->n_tiles + target - 1) / target;
    tpc = std::max<long long>(1, std::min<long long>(tpc, sc->n_tiles));
    const long long chunks = (sc->n_tiles + tpc - 1) / tpc;
    if (chunks > 65535) return fail(PSDF_ERR_CAPACITY, "too many tile chunks");
    const int blob_cap = (sc->max_blob_bytes + 127) / 128 * 128;
    const size_t smem = 128 + 2 * (size_t)blob_cap;
    dim3 grid((unsigned)pose_blocks, (unsigned)chunks);
    ProfileScope prof("scan", st);
    // behind the key initialisation: the scan runs while it finishes
    cudaError_t le = launch_pdl(pk.eta > 0.f ? scan_kernel<M, true> : scan_kernel<M, false>,
                                grid, dim3(kScanThreads), smem, st, F, pk, poses, P, npb,
                                (const TileHdr *)sc->d_tiles, (const unsigned char *)sc->d_blob,
                                sc->n_tiles, (int)tpc, blob_cap, keys, err, wait_limit());
    if (le != cudaSuccess) return cuda_fail(le, "kernel launch (scan)");
  }
  return PSDF_OK;
}

template <int M>
static int launch_eval(const FootprintK &F, const psdf_scene *sc, const float *poses, long long P,
                       const psdf_params *prm, float *phi, float *dphi, unsigned *active,
                       void *ws, const StageOut &so, cudaStream_t st)
{
  int *err = reinterpret_cast<int *>(ws);
  unsigned long long *keys =
      reinterpret_cast<unsigned long long *>(reinterpret_cast<unsigned char *>(ws) + 256);
  ParamsK pk{prm->eps_sat, prm->eta};
  int rc = launch_scan<M>(F, sc, poses, P, pk, keys, err, st);
  if (rc) return rc;
  {
    ProfileScope prof("epilogue", st);
    const bool soft = pk.eta > 0.f;
    // behind the scan: its CTAs are resident when the scan completes
    cudaError_t le = launch_pdl(soft       ? epilogue_kernel<M, true>
                                : so.saved ? epilogue_kernel<M, false, true>
                                           : epilogue_kernel<M, false>,
                                epilogue_blocks(P, soft), epilogue_threads(soft), 0, st, F, pk,
                                sc->eps_axis, poses, P, (const ObsRec *)sc->d_row_obs,
                                (const float4 *)sc->d_vtx, (const int *)sc->d_far,
                                (const unsigned long long *)keys, (const int *)err, phi, dphi,
                                active, so.stage, so.d_min, so.saved);
    if (le != cudaSuccess) return cuda_fail(le, "kernel launch (epilogue)");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return PSDF_OK;
}

template <int M>
static int launch_backward(const FootprintK &F, const psdf_scene *sc, const float *poses,
                           long long P, const ParamsK &pk, const unsigned *active,
                           const float *grad_phi, float *grad_pose, float *grad_edges,
                           cudaStream_t st)
{
  const int spread = backward_spread_shift(P);
  const unsigned blocks = (unsigned)(((P << spread) + 127) / 128);
  ProfileScope prof("backward", st);
  // usually follows an epilogue on the stream: may start while it finishes
  cudaError_t le;
  if (pk.eta > 0.f)
    le = launch_pdl(backward_kernel<M, true>, dim3(blocks), dim3(128), 0, st, F, pk, sc->eps_axis,
                    poses, P, (const ObsRec *)sc->d_row_obs, (const float4 *)sc->d_vtx,
                    (const int *)sc->d_far, (long long)sc->rows_total, active, grad_phi,
                    grad_pose, grad_edges, spread);
  else
    le = launch_pdl(backward_kernel<M, false>, dim3(blocks), dim3(128), 0, st, F, pk,
                    sc->eps_axis, poses, P, (const ObsRec *)sc->d_row_obs,
                    (const float4 *)sc->d_vtx, (const int *)sc->d_far,
                    (long long)sc->rows_total, active, grad_phi, grad_pose, grad_edges, spread);
  if (le != cudaSuccess) return cuda_fail(le, "kernel launch");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return PSDF_OK;
}

// Runtime footprint size -> compile-time M (fully unrolled robot loops).
template <template <int> class Fn, class... Args>
static int dispatch_m(int m, Args &&...args)
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

template <int M>
struct EvalCall {
  static int run(const FootprintK &F, const psdf_scene *sc, const float *poses, long long P,
                 const psdf_params *prm, float *phi, float *dphi, unsigned *active, void *ws,
                 const StageOut &so, cudaStream_t st)
  {
    return launch_eval<M>(F, sc, poses, P, prm, phi, dphi, active, ws, so, st);
  }
};

template <int M>
struct EpilogueCall {
  static int run(const FootprintK &F, const psdf_scene *sc, const float *poses, long long P,
                 const ParamsK &pk, const unsigned long long *keys, const int *err, float *phi,
                 float *dphi, unsigned *active, float4 *saved, cudaStream_t st)
  {
    ProfileScope prof("epilogue", st);
    // after the cull's evaluation kernel: may start while it finishes
    const bool soft = pk.eta > 0.f;
    cudaError_t e = launch_pdl(soft    ? epilogue_kernel<M, true>
                               : saved ? epilogue_kernel<M, false, true>
                                       : epilogue_kernel<M, false>,
                               epilogue_blocks(P, soft), epilogue_threads(soft), 0, st, F, pk,
                               sc->eps_axis, poses, P, (const ObsRec *)sc->d_row_obs,
                               (const float4 *)sc->d_vtx, (const int *)sc->d_far, keys, err,
                               phi, dphi, active, (float *)nullptr, 0.f, saved);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return PSDF_OK;
  }
};

template <int M>
struct BackwardCall {
  static int run(const FootprintK &F, const psdf_scene *sc, const float *poses, long long P,
                 const ParamsK &pk, const unsigned *active, const float *grad_phi,
                 float *grad_pose, float *grad_edges, cudaStream_t st)
  {
    return launch_backward<M>(F, sc, poses, P, pk, active, grad_phi, grad_pose, grad_edges, st);
  }
};

template <int M>
struct KeysCall {
  static int run(const FootprintK &F, const psdf_scene *sc, const float *poses, long long P,
                 const ParamsK &pk, unsigned long long *keys, int *err, unsigned row_offset,
                 cudaStream_t st)
  {
    int rc = launch_scan<M>(F, sc, poses, P, pk, keys, err, st);
    if (rc) return rc;
    if (row_offset == 0) return PSDF_OK;
    cudaError_t e = launch_pdl(offset_keys_kernel, dim3((unsigned)((P + 255) / 256)), dim3(256), 0,
                               st, keys, P, row_offset);
    return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch (offset keys)");
  }
};

template <int M>
struct FinishCall {
  static int run(const FootprintK &F, const psdf_scene *sc, const float *poses, long long P,
                 const ParamsK &pk, const unsigned long long *keys, long long row_offset,
                 int own_empty, float *phi, float *dphi, unsigned *active, cudaStream_t st)
  {
    const bool soft = pk.eta > 0.f;
    const long long threads = soft ? P : P * kEpiLanes;
    (soft ? finish_keys_kernel<M, true> : finish_keys_kernel<M, false>)
        <<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(
            F, pk, sc->eps_axis, poses, P, (const ObsRec *)sc->d_row_obs,
            (const float4 *)sc->d_vtx, (const int *)sc->d_far, keys, row_offset,
            (long long)sc->rows_total, own_empty, phi, dphi, active);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch (finish keys)");
  }
};

int launch_epilogue(const FootprintK &F, const psdf_scene *sc, const float *poses, long long P,
                    const ParamsK &pk, const unsigned long long *keys, const int *err,
                    float *phi, float *dphi, unsigned *active, cudaStream_t st, float4 *saved)
{
  return dispatch_m<EpilogueCall>(F.m, F, sc, poses, P, pk, keys, err, phi, dphi, active, saved,
                                  st);
}

int eval_common(const float *footprint, int32_t m, const psdf_scene *scene, const float *poses,
                int64_t P, const psdf_params *params, float *phi, float *dphi, unsigned *active,
                void *ws, size_t ws_bytes, void *stream, const StageOut &so)
{
  int rc = check_eval_args(scene, poses, P, params, ws, ws_bytes);
  if (rc) return rc;
  if (P > 0 && !phi && !so.stage) return fail(PSDF_ERR_ARG, "phi is NULL");
  FootprintK F;
  rc = make_footprint(footprint, m, scene->eps_seg, &F);
  if (rc) return rc;
  if (P == 0) return PSDF_OK;
  return dispatch_m<EvalCall>(m, F, scene, poses, (long long)P, params, phi, dphi, active, ws,
                              so, (cudaStream_t)stream);
}

}  // namespace psdf

using namespace psdf;

extern "C" int psdf_eval(const float *footprint, int32_t m, const psdf_scene *scene,
                         const float *poses, int64_t P, const psdf_params *params, float *phi,
                         uint32_t *active, void *workspace, size_t workspace_bytes, void *stream)
{
  return eval_common(footprint, m, scene, poses, P, params, phi, nullptr, active, workspace,
                     workspace_bytes, stream);
}

extern "C" int psdf_eval_grad(const float *footprint, int32_t m, const psdf_scene *scene,
                              const float *poses, int64_t P, const psdf_params *params,
                              float *phi, float *dphi, uint32_t *active, void *workspace,
                              size_t workspace_bytes, void *stream)
{
  if (P > 0 && !dphi) return fail(PSDF_ERR_ARG, "dphi is NULL");
  return eval_common(footprint, m, scene, poses, P, params, phi, dphi, active, workspace,
                     workspace_bytes, stream);
}

extern "C" int psdf_eval_grad_save(const float *footprint, int32_t m, const psdf_scene *scene,
                                   const float *poses, int64_t P, const psdf_params *params,
                                   float *phi, float *dphi, uint32_t *active, float *saved,
                                   void *workspace, size_t workspace_bytes, void *stream)
{
  if (P > 0 && (!dphi || !saved)) return fail(PSDF_ERR_ARG, "dphi or saved is NULL");
  if (params && params->eta > 0.f)
    return fail(PSDF_ERR_ARG, "saved backward records need the hard minimum (eta <= 0)");
  if (((uintptr_t)saved & 15u) != 0) return fail(PSDF_ERR_ARG, "saved must be 16-byte aligned");
  StageOut so;
  so.saved = reinterpret_cast<float4 *>(saved);
  return eval_common(footprint, m, scene, poses, P, params, phi, dphi, active, workspace,
                     workspace_bytes, stream, so);
}

extern "C" int psdf_backward_saved(const psdf_scene *scene, const float *saved, int64_t P,
                                   const float *grad_phi, float *grad_pose, float *grad_edges,
                                   void *stream)
{
  if (!scene) return fail(PSDF_ERR_ARG, "scene is NULL");
  if (P < 0) return fail(PSDF_ERR_ARG, "P < 0");
  if (P == 0) return PSDF_OK;
  if (!saved || !grad_phi) return fail(PSDF_ERR_ARG, "saved or grad_phi is NULL");
  if (((uintptr_t)saved & 15u) != 0) return fail(PSDF_ERR_ARG, "saved must be 16-byte aligned");
  // one warp per CTA: the few thousand poses of a step spread over every SM
  const unsigned blocks = (unsigned)((P + 31) / 32);
  ProfileScope prof("backward", (cudaStream_t)stream);
  // usually follows an epilogue on the stream: may start while it finishes
  cudaError_t e = launch_pdl(backward_saved_kernel, dim3(blocks), dim3(32), 0,
                             (cudaStream_t)stream, reinterpret_cast<const float4 *>(saved),
                             (long long)P, (long long)scene->rows_total, grad_phi, grad_pose,
                             grad_edges);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch (backward_saved)");
}

extern "C" int psdf_eval_keys(const float *footprint, int32_t m, const psdf_scene *scene,
                              const float *poses, int64_t P, const psdf_params *params,
                              int64_t row_offset, uint64_t *keys, void *workspace,
                              size_t workspace_bytes, void *stream)
{
  // the workspace holds only the error word here (the keys are the caller's)
  int rc = check_eval_args(scene, poses, P, params, workspace, (size_t)-1);
  if (rc) return rc;
  if (P > 0 && workspace_bytes < 256) return fail(PSDF_ERR_CAPACITY, "workspace below 256 bytes");
  if (P > 0 && !keys) return fail(PSDF_ERR_ARG, "keys is NULL");
  if (row_offset < 0 || row_offset + scene->rows_total > (int64_t)kMaxEdgeIndex + 1)
    return fail(PSDF_ERR_ARG, "row_offset outside the pair id's edge range");
  FootprintK F;
  rc = make_footprint(footprint, m, scene->eps_seg, &F);
  if (rc) return rc;
  if (P == 0) return PSDF_OK;
  const ParamsK pk{params->eps_sat, params->eta};
  return dispatch_m<KeysCall>(m, F, scene, poses, (long long)P, pk,
                              reinterpret_cast<unsigned long long *>(keys),
                              reinterpret_cast<int *>(workspace), (unsigned)row_offset,
                              (cudaStream_t)stream);
}

extern "C" int psdf_merge_keys(const uint64_t *a, uint64_t *b, int64_t P, void *stream)
{
  if (P < 0) return fail(PSDF_ERR_ARG, "P < 0");
  if (P == 0) return PSDF_OK;
  if (!a || !b) return fail(PSDF_ERR_ARG, "NULL argument");
  merge_keys_kernel<<<(unsigned)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const unsigned long long *>(a), reinterpret_cast<unsigned long long *>(b),
      (long long)P);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch (merge keys)");
}

extern "C" int psdf_finish_keys(const float *footprint, int32_t m, const psdf_scene *scene,
                                const float *poses, int64_t P, const psdf_params *params,
                                int64_t row_offset, int32_t own_empty, const uint64_t *keys,
                                float *phi, float *dphi, uint32_t *active, void *stream)
{
  int rc = check_eval_args(scene, poses, P, params, (void *)256, (size_t)-1);
  if (rc) return rc;
  if (P > 0 && (!keys || !phi)) return fail(PSDF_ERR_ARG, "keys or phi is NULL");
  if (row_offset < 0 || row_offset + scene->rows_total > (int64_t)kMaxEdgeIndex + 1)
    return fail(PSDF_ERR_ARG, "row_offset outside the pair id's edge range");
  FootprintK F;
  rc = make_footprint(footprint, m, scene->eps_seg, &F);
  if (rc) return rc;
  if (P == 0) return PSDF_OK;
  const ParamsK pk{params->eps_sat, params->eta};
  return dispatch_m<FinishCall>(m, F, scene, poses, (long long)P, pk,
                                reinterpret_cast<const unsigned long long *>(keys),
                                (long long)row_offset, (int)own_empty, phi, dphi, active,
                                (cudaStream_t)stream);
}

extern "C" int psdf_stage_params(const float *footprint, int32_t m, const psdf_scene *scene,
                                 const float *poses, int64_t P, const psdf_params *params,
                                 float d_min, float *stage, uint32_t *active, void *workspace,
                                 size_t workspace_bytes, void *stream)
{
  if (P > 0 && !stage) return fail(PSDF_ERR_ARG, "stage is NULL");
  if (!std::isfinite(d_min)) return fail(PSDF_ERR_ARG, "d_min must be finite");
  StageOut so;
  so.stage = stage;
  so.d_min = d_min;
  return eval_common(footprint, m, scene, poses, P, params, nullptr, nullptr, active, workspace,
                     workspace_bytes, stream, so);
}

extern "C" int psdf_backward(const float *footprint, int32_t m, const psdf_scene *scene,
                             const float *poses, int64_t P, const psdf_params *params,
                             const uint32_t *active, const float *grad_phi, float *grad_pose,
                             float *grad_edges, void *stream)
{
  int rc = check_eval_args(scene, poses, P, params, (void *)256, (size_t)-1);
  if (rc) return rc;
  if (P > 0 && (!active || !grad_phi)) return fail(PSDF_ERR_ARG, "active or grad_phi is NULL");
  FootprintK F;
  rc = make_footprint(footprint, m, scene->eps_seg, &F);
  if (rc) return rc;
  if (P == 0) return PSDF_OK;
  const ParamsK pk{params->eps_sat, params->eta};
  return dispatch_m<BackwardCall>(m, F, scene, poses, (long long)P, pk, active, grad_phi,
                                  grad_pose, grad_edges, (cudaStream_t)stream);
}

extern "C" const char *psdf_last_error(void) { return g_err.c_str(); }

extern "C" int psdf_version(void) { return 100; }

extern "C" int psdf_debug_set_wait_limit(uint32_t polls, uint32_t *previous)
{
  const unsigned old = g_wait_limit.exchange(polls);
  if (previous) *previous = old;
  return PSDF_OK;
}

extern "C" size_t psdf_workspace_bytes(int64_t P)
{
  if (P < 1) P = 1;
  return 256 + (size_t)((8 * P + 255) / 256 * 256);
}

extern "C" int psdf_workspace_status(const void *workspace, void *stream)
{
  if (!workspace) return fail(PSDF_ERR_ARG, "workspace is NULL");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int v = 0;
  e = cudaMemcpy(&v, workspace, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(workspace status)");
  if (v) return fail(PSDF_ERR_TIMEOUT, "a bounded device-side wait ran out (edge tile copy)");
  return PSDF_OK;
}
