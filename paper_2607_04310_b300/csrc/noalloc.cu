// psdf_eval_grad_noalloc: the value + gradient evaluation for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc once they are running: a control loop
// with a hard period (cudaMalloc may synchronize the device and take an
// unbounded time), a plug-in hosted by a framework that owns the whole
// device memory pool, or code that runs inside a region where the allocator
// is locked.  For them this entry point takes its scratch (one 64-bit key per
// pose plus an error word) from a fixed array compiled into the library
// instead of a caller workspace.  Everything else -- inputs, outputs, the
// kernels and their results -- is exactly psdf_eval_grad.
#include <mutex>

#include "psdf_internal.h"

namespace psdf {

constexpr long long kNoAllocMaxPoses = PSDF_NOALLOC_MAX_POSES;
constexpr size_t kNoAllocBytes = 256 + 8 * (size_t)kNoAllocMaxPoses;

// The scratch array.  Every GPU that loads the library holds it until the
// process exits.  In host code its name is only a host-side stand-in; the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};  // context the address belongs to

// Identity of the context current on this thread (0 = none yet), from the
// driver's cuCtxGetCurrent / cuCtxGetId, reached through the runtime's
// entry-point query so that the library does not link the driver library.
// Neither call allocates.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

unsigned long long current_context_id()
{
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx) return 0;
  if (get_id(ctx, &id) != 0) return 0;
  return id;
}

// The array's device address on the current device: looked up once per
// device (with that device current) and again whenever the device's context
// is no longer the one the address was taken in (after cudaDeviceReset the
// runtime makes a new primary context, and the old address is gone).
int scratch_address(void **out)
{
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return fail(PSDF_ERR_CAPACITY, "device index beyond the no-allocation table");
  std::lock_guard<std::mutex> lk(g_mu);
  const unsigned long long id = current_context_id();
  if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    g_addr[dev] = p;
    // the lookup made the device's primary context current if none was
    g_ctx_id[dev] = id != 0 ? id : current_context_id();
  }
  *out = g_addr[dev];
  return PSDF_OK;
}

}  // namespace
}  // namespace psdf

using namespace psdf;

extern "C" int psdf_eval_grad_noalloc(const float *footprint, int32_t m, const psdf_scene *scene,
                                      const float *poses, int64_t P, const psdf_params *params,
                                      float *phi, float *dphi, uint32_t *active, void *stream)
{
  if (P > kNoAllocMaxPoses)
    return fail(PSDF_ERR_CAPACITY, "psdf_eval_grad_noalloc takes at most " +
                                       std::to_string(kNoAllocMaxPoses) + " poses per call");
  if (P > 0 && !dphi) return fail(PSDF_ERR_ARG, "dphi is NULL");
  void *ws = nullptr;
  int rc = scratch_address(&ws);
  if (rc) return rc;
  // the init kernel of the evaluation clears the keys and the error word,
  // so the previous call's contents never leak into this one
  return eval_common(footprint, m, scene, poses, P, params, phi, dphi, active, ws,
                     kNoAllocBytes, stream);
}
