// smem_optin.h -- bookkeeping of the dynamic shared memory opt-in of kernels.
//
// cudaFuncAttributeMaxDynamicSharedMemorySize is a setting of a kernel on one
// device: a kernel launched with more than 48 KB of dynamic shared memory on a
// device where it was not raised fails to launch.  SmemOptIn remembers, per
// (kernel, device), the largest size already set, so the attribute is set once
// per device and size, from any thread.  The call that sets it is passed in,
// which keeps this header free of CUDA (it is also compiled by a host-only test).
#pragma once

#include <stddef.h>

#include <map>
#include <mutex>
#include <utility>

namespace dfacto {

class SmemOptIn {
 public:
  // Make sure `kernel` may use `bytes` of dynamic shared memory on `device`.
  // set() raises the limit to `bytes` on that device and returns 0 on success;
  // it runs only when no earlier call for this (kernel, device) covered
  // `bytes`.  Returns set()'s error, or 0.
  template <class Set>
  int ensure(const void* kernel, int device, size_t bytes, Set&& set) {
    std::lock_guard<std::mutex> lock(mu_);
    size_t& have = done_[std::make_pair(kernel, device)];
    if (bytes <= have) return 0;
    const int e = set();
    if (e == 0) have = bytes;
    return e;
  }

 private:
  std::mutex mu_;
  std::map<std::pair<const void*, int>, size_t> done_;
};

}  // namespace dfacto
