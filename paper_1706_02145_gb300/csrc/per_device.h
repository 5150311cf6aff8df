// One-time, per-device set-up values (plain C++, no CUDA types).
//
// CUDA applies a kernel's attributes (the opt-in above 48 KB of dynamic
// shared memory) per device, and occupancy and SM counts are per-device
// facts.  A process that drives several GPUs must therefore do such set-up
// once on EACH device, with that device current, and keep one cached value
// per device ordinal.  PerDevice holds those values: slot d is filled by the
// first get() that runs while device d is current.
//
// The device query and the set-up step are passed in as callables, so this
// logic is unit-tested on the CPU with a fake device query.
#pragma once

#include <atomic>

namespace celes {

constexpr int kMaxDevices = 64;

// Cached positive int per device.  init() returns the value (> 0) or a value
// <= 0 on failure; failures are not cached, so a later call retries.  Two
// threads that race on the first use of one device may both run init(); the
// set-up steps used here (attribute set, occupancy query) are idempotent.
struct PerDevice {
  std::atomic<int> v[kMaxDevices];

  PerDevice() {
    for (auto& a : v) a.store(0, std::memory_order_relaxed);
  }

  // dev_of(int*) -> bool (true on success) gives the current device ordinal
  template <typename DevOf, typename Init>
  int get(DevOf&& dev_of, Init&& init) {
    int dev = -1;
    if (!dev_of(&dev) || dev < 0 || dev >= kMaxDevices) {
      const int r = init();  // no slot for this device: set up, uncached
      return r > 0 ? r : 0;
    }
    int r = v[dev].load(std::memory_order_acquire);
    if (r > 0) return r;
    r = init();
    if (r <= 0) return 0;
    v[dev].store(r, std::memory_order_release);
    return r;
  }
};

}  // namespace celes
