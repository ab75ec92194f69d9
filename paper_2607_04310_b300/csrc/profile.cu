// Event-based kernel tracing (psdf_profile_*).  Off by default.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "profile.h"
#include "psdf_internal.h"

namespace psdf {

namespace {
struct Rec {
  std::string name;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
}  // namespace

bool profiling_on() { return g_on; }

ProfileScope::ProfileScope(const char *name, cudaStream_t st) : name_(name), st_(st)
{
  if (!g_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaEventRecord(a_, st);
  active_ = true;
}

ProfileScope::~ProfileScope()
{
  if (!active_) return;
  cudaEventRecord(b_, st_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back(Rec{name_, a_, b_});
}

}  // namespace psdf

using namespace psdf;

extern "C" int psdf_profile_enable(int on)
{
  g_on = on != 0;
  return PSDF_OK;
}

extern "C" int psdf_profile_reset(void)
{
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &r : g_recs) {
    cudaEventSynchronize(r.b);
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
  return PSDF_OK;
}

extern "C" int psdf_profile_read(const char *kernel, int64_t *launches, double *total_ms)
{
  if (!kernel || !launches || !total_ms) return fail(PSDF_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(g_mu);
  int64_t n = 0;
  double ms = 0.0;
  const bool all = std::strcmp(kernel, "all") == 0;
  for (auto &r : g_recs) {
    if (!all && r.name != kernel) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize(profile)");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime(profile)");
    ms += t;
    ++n;
  }
  *launches = n;
  *total_ms = ms;
  return PSDF_OK;
}
