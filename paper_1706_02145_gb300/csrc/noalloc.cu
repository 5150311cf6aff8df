// Coupling matvec for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a host
// application's own device-memory pool (where every byte is owned by that
// pool and direct allocations are forbidden), and code on a latency-critical
// path that cannot tolerate the device-wide synchronisation that cudaMalloc
// and cudaFree imply.  celes_coupling_matvec_noalloc serves them: it needs no
// context and allocates nothing.  The caller passes the inputs and the output
// in its own device memory; the only scratch (the per-chunk partial sums of the
// coupling kernel) lives in the fixed array below, which is part of the
// library image: every GPU that loads the library holds these 32 MiB until the
// process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/celes.h"
#include "kernels.h"

namespace celes {
#define CELES_DECLARE_RTR(LL)                                                                               \
  cudaError_t launch_coupling_rtr_##LL(int precision, int64_t N, const void* pos, const void* x,           \
                                       void* partial, double k, int chunks, cudaStream_t st, int maxcl,    \
                                       int atomic);                                                        \
  int coupling_rtr_rpb_##LL(int precision);                                                                \
  int coupling_rtr_slices_##LL(int precision, int chunks, int maxcl, int atomic);                          \
  int coupling_rtr_slots_##LL(int precision);
CELES_DECLARE_RTR(1)
CELES_DECLARE_RTR(2)
CELES_DECLARE_RTR(3)
CELES_DECLARE_RTR(4)
CELES_DECLARE_RTR(5)
#undef CELES_DECLARE_RTR
}  // namespace celes

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;

// The scratch of every call of celes_coupling_matvec_noalloc.  In host code
// this name is only a stand-in for the device array; the device address is
// obtained once per device with cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_noalloc_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch_dev[celes::kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call on each device).
cudaError_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= celes::kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

cudaError_t launch_rtr(int L, int precision, int64_t N, const void* pos, const void* x, void* partial, double k,
                       int chunks, cudaStream_t st) {
  using namespace celes;
  switch (L) {
    case 1: return launch_coupling_rtr_1(precision, N, pos, x, partial, k, chunks, st, 1, 0);
    case 2: return launch_coupling_rtr_2(precision, N, pos, x, partial, k, chunks, st, 1, 0);
    case 3: return launch_coupling_rtr_3(precision, N, pos, x, partial, k, chunks, st, 1, 0);
    case 4: return launch_coupling_rtr_4(precision, N, pos, x, partial, k, chunks, st, 1, 0);
    case 5: return launch_coupling_rtr_5(precision, N, pos, x, partial, k, chunks, st, 1, 0);
    default: return cudaErrorInvalidValue;
  }
}

int rtr_slots(int L, int precision) {
  using namespace celes;
  switch (L) {
    case 1: return coupling_rtr_slots_1(precision);
    case 2: return coupling_rtr_slots_2(precision);
    case 3: return coupling_rtr_slots_3(precision);
    case 4: return coupling_rtr_slots_4(precision);
    case 5: return coupling_rtr_slots_5(precision);
    default: return 0;
  }
}

int rtr_slices(int L, int precision, int chunks) {
  using namespace celes;
  switch (L) {
    case 1: return coupling_rtr_slices_1(precision, chunks, 1, 0);
    case 2: return coupling_rtr_slices_2(precision, chunks, 1, 0);
    case 3: return coupling_rtr_slices_3(precision, chunks, 1, 0);
    case 4: return coupling_rtr_slices_4(precision, chunks, 1, 0);
    case 5: return coupling_rtr_slices_5(precision, chunks, 1, 0);
    default: return chunks;
  }
}

int rtr_rpb(int L, int precision) {
  using namespace celes;
  switch (L) {
    case 1: return coupling_rtr_rpb_1(precision);
    case 2: return coupling_rtr_rpb_2(precision);
    case 3: return coupling_rtr_rpb_3(precision);
    case 4: return coupling_rtr_rpb_4(precision);
    case 5: return coupling_rtr_rpb_5(precision);
    default: return 1;
  }
}

}  // namespace

extern "C" int celes_coupling_matvec_noalloc(int64_t N, int lmax, double k, const double* positions4, const void* x,
                                             void* y, int precision, void* stream) {
  if (N < 1 || N > (int64_t(1) << 30) || lmax < 1 || lmax > 5 || !(k > 0.0) || !positions4 || !x || !y ||
      (precision != CELES_FP64 && precision != CELES_FP32))
    return CELES_EINVAL;
  if (reinterpret_cast<uintptr_t>(positions4) % 32 != 0) return CELES_EINVAL;
  const int nmax = 2 * lmax * (lmax + 2);
  const size_t elem = precision == CELES_FP64 ? 16 : 8;
  const size_t vec_bytes = static_cast<size_t>(N) * nmax * elem;
  // one partial sum per source chunk must fit in the static scratch
  const size_t max_chunks = kStaticScratchBytes / vec_bytes;
  if (max_chunks < 1) return CELES_ETOOBIG;
  const char* xb = static_cast<const char*>(x);
  const char* yb = static_cast<const char*>(y);
  if (xb < yb + vec_bytes && yb < xb + vec_bytes) return CELES_EINVAL;  // x and y overlap
  const int rpb = rtr_rpb(lmax, precision);
  const int64_t rb = (N + rpb - 1) / rpb;
  const int slots = rtr_slots(lmax, precision);
  int64_t chunks = (8LL * (slots > 0 ? slots : 304) + rb - 1) / rb;  // about eight waves
  chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, N / 64));
  chunks = std::min<int64_t>(chunks, 256);
  chunks = std::min<int64_t>(chunks, static_cast<int64_t>(max_chunks));
  chunks = std::max<int64_t>(chunks, 1);
  void* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return CELES_ECUDA;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double k_bg = k;
  if (launch_rtr(lmax, precision, N, positions4, x, scratch, k_bg, static_cast<int>(chunks), st) != cudaSuccess)
    return CELES_ECUDA;
  const int slices = rtr_slices(lmax, precision, static_cast<int>(chunks));
  const cudaError_t e = precision == CELES_FP64
                            ? celes::launch_coupling_epilogue<double>(N, lmax, slices, scratch, x, nullptr, y, 0, st)
                            : celes::launch_coupling_epilogue<float>(N, lmax, slices, scratch, x, nullptr, y, 0, st);
  return e == cudaSuccess ? CELES_OK : CELES_ECUDA;
}
