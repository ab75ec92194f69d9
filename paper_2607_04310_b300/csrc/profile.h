// RAII event bracket around one kernel launch (active only when tracing is on).
#pragma once
#include <cuda_runtime.h>

#include <string>

namespace psdf {

bool profiling_on();

class ProfileScope {
 public:
  ProfileScope(const char *name, cudaStream_t st);
  ~ProfileScope();
  ProfileScope(const ProfileScope &) = delete;
  ProfileScope &operator=(const ProfileScope &) = delete;

 private:
  std::string name_;
  cudaStream_t st_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  bool active_ = false;
};

}  // namespace psdf
