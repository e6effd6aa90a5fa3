// Per-device cache of the device address of a file-scope __device__ array (host logic only,
// no CUDA types, so it also builds in a plain C++ test).
//
// The address of a __device__ array belongs to the CUDA context that loaded the module: after a
// device reset, or any teardown and re-creation of the primary context, the module is loaded
// again and the array may sit at another address.  An entry therefore records the identifier
// of the context it was looked up in (unique for the life of the process, never reused), and a
// lookup under any other context misses, so the caller looks the address up again.
#pragma once

#include <mutex>

namespace qf {

class ScratchAddressCache {
 public:
  static constexpr int kMaxDevices = 64;

  // Cached address for (device, context id), or nullptr when absent, stale or out of range.
  void* find(int dev, unsigned long long ctx_id) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(mu_);
    const Entry& e = entry_[dev];
    return (e.ptr && e.ctx_id == ctx_id) ? e.ptr : nullptr;
  }

  // Records the address looked up under (device, context id); replaces an older context's entry.
  bool put(int dev, unsigned long long ctx_id, void* ptr) {
    if (dev < 0 || dev >= kMaxDevices || !ptr) return false;
    std::lock_guard<std::mutex> lock(mu_);
    entry_[dev] = Entry{ctx_id, ptr};
    return true;
  }

 private:
  struct Entry {
    unsigned long long ctx_id = 0;
    void* ptr = nullptr;
  };
  std::mutex mu_;
  Entry entry_[kMaxDevices];
};

}  // namespace qf
