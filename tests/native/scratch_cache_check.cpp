// Host-only check of the per-context scratch address cache used by the allocation-free
// dressing entry point: an address is returned only for the (device, context) it was recorded
// under, a new context (as after a device reset) misses and replaces the old entry, devices are
// independent, and out-of-range devices are refused.  Exit status 0 on success.
#include <cstdio>

#include "../../paper_2606_04186_gb300/csrc/scratch_cache.h"

#define CHECK(c)                                         \
  do {                                                   \
    if (!(c)) {                                          \
      std::fprintf(stderr, "failed: %s (line %d)\n", #c, __LINE__); \
      return 1;                                          \
    }                                                    \
  } while (0)

int main() {
  qf::ScratchAddressCache c;
  int a = 0, b = 0, d = 0;
  CHECK(c.find(0, 7) == nullptr);
  CHECK(c.put(0, 7, &a));
  CHECK(c.find(0, 7) == &a);
  CHECK(c.find(0, 8) == nullptr);  // another context on the same device: look up again
  CHECK(c.find(1, 7) == nullptr);  // another device
  CHECK(c.put(0, 8, &b));          // the re-created context's address replaces the old one
  CHECK(c.find(0, 8) == &b);
  CHECK(c.find(0, 7) == nullptr);  // the destroyed context's address is never handed out again
  CHECK(c.put(1, 9, &d));
  CHECK(c.find(1, 9) == &d && c.find(0, 8) == &b);
  CHECK(!c.put(-1, 1, &a) && !c.put(qf::ScratchAddressCache::kMaxDevices, 1, &a));
  CHECK(c.find(-1, 1) == nullptr && c.find(qf::ScratchAddressCache::kMaxDevices, 1) == nullptr);
  CHECK(!c.put(2, 1, nullptr) && c.find(2, 1) == nullptr);
  std::puts("ok");
  return 0;
}
