// C ABI and host runtime of the solver: context and device memory, incident
// fields, coupling / master matvecs, block preconditioner, GMRES in FP64 and
// FP32 with FP64 iterative refinement (Sec. 3.2), far field (App. D).
//
// All arithmetic on problem data runs in the CUDA kernels of this library;
// the host side holds only bookkeeping, the Givens rotations of the small
// GMRES Hessenberg matrix and the cuboid partition of the preconditioner.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/celes.h"
#include "coupling_kernel.cuh"
#include "kernels.h"

namespace celes {
// per-degree coupling launchers (coupling_L*.cu)
#define CELES_DECLARE(LL)                                                                                   \
  cudaError_t launch_coupling_partial_##LL(int precision, int64_t N, const void* pos, const void* x,       \
                                            void* partial, double k, int chunks, cudaStream_t st);         \
  int coupling_rpb_##LL(int precision);                                                                    \
  cudaError_t launch_coupling_rtr_##LL(int precision, int64_t N, const void* pos, const void* x,           \
                                       void* partial, double k, int chunks, cudaStream_t st, int maxcl,    \
                                       int atomic);                                                        \
  int coupling_rtr_rpb_##LL(int precision);                                                                \
  int coupling_rtr_slices_##LL(int precision, int chunks, int maxcl, int atomic);                          \
  int coupling_rtr_slots_##LL(int precision);                                                              \
  long long coupling_rtr_flops_##LL();                                                                     \
  int coupling_terms_export_##LL(int* idx, double* val, int cap);
#define CELES_DECLARE_ALT(LL)                                                                              \
  cudaError_t launch_coupling_rtr_alt_##LL(int64_t N, const void* pos, const void* x, void* partial,       \
                                           double k, int chunks, cudaStream_t st, int maxcl, int atomic);  \
  int coupling_rtr_alt_rpb_##LL();                                                                         \
  int coupling_rtr_alt_slices_##LL(int chunks, int maxcl, int atomic);                                     \
  int coupling_rtr_alt_slots_##LL();
CELES_DECLARE_ALT(1)
CELES_DECLARE_ALT(2)
CELES_DECLARE_ALT(3)
CELES_DECLARE_ALT(4)
CELES_DECLARE_ALT(5)
#undef CELES_DECLARE_ALT
CELES_DECLARE(1)
CELES_DECLARE(2)
CELES_DECLARE(3)
CELES_DECLARE(4)
CELES_DECLARE(5)
#undef CELES_DECLARE

cudaError_t launch_coupling_partial(int L, int precision, int64_t N, const void* pos, const void* x, void* partial,
                                    double k, int chunks, cudaStream_t st) {
  switch (L) {
    case 1: return launch_coupling_partial_1(precision, N, pos, x, partial, k, chunks, st);
    case 2: return launch_coupling_partial_2(precision, N, pos, x, partial, k, chunks, st);
    case 3: return launch_coupling_partial_3(precision, N, pos, x, partial, k, chunks, st);
    case 4: return launch_coupling_partial_4(precision, N, pos, x, partial, k, chunks, st);
    case 5: return launch_coupling_partial_5(precision, N, pos, x, partial, k, chunks, st);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t launch_coupling_rtr(int L, int precision, int64_t N, const void* pos, const void* x, void* partial,
                                double k, int chunks, cudaStream_t st, int maxcl = 1, int atomic = 0) {
  switch (L) {
    case 1: return launch_coupling_rtr_1(precision, N, pos, x, partial, k, chunks, st, maxcl, atomic);
    case 2: return launch_coupling_rtr_2(precision, N, pos, x, partial, k, chunks, st, maxcl, atomic);
    case 3: return launch_coupling_rtr_3(precision, N, pos, x, partial, k, chunks, st, maxcl, atomic);
    case 4: return launch_coupling_rtr_4(precision, N, pos, x, partial, k, chunks, st, maxcl, atomic);
    case 5: return launch_coupling_rtr_5(precision, N, pos, x, partial, k, chunks, st, maxcl, atomic);
    default: return cudaErrorInvalidValue;
  }
}
int coupling_rtr_receivers_per_block(int L, int precision);
int coupling_rtr_slots(int L, int precision);

// launch shape `variant`: bit 0 the compile-time shape (0: Config, 1:
// ConfigAlt, FP32 only), bit 1 the cluster reduction of the partial sums
// (clusters of up to 8 chunks), bit 2 the in-L2 vector reduction of all
// chunks into one slice (FP32 only)
cudaError_t launch_coupling_rtr_v(int L, int precision, int variant, int64_t N, const void* pos, const void* x,
                                  void* partial, double k, int chunks, cudaStream_t st) {
  const int maxcl = (variant & 2) ? 8 : 1;
  const int atomic = (variant & 4) && precision == CELES_FP32 ? 1 : 0;
  if ((variant & 1) == 0 || precision == CELES_FP64)
    return launch_coupling_rtr(L, precision, N, pos, x, partial, k, chunks, st, maxcl, atomic);
  switch (L) {
    case 1: return launch_coupling_rtr_alt_1(N, pos, x, partial, k, chunks, st, maxcl, atomic);
    case 2: return launch_coupling_rtr_alt_2(N, pos, x, partial, k, chunks, st, maxcl, atomic);
    case 3: return launch_coupling_rtr_alt_3(N, pos, x, partial, k, chunks, st, maxcl, atomic);
    case 4: return launch_coupling_rtr_alt_4(N, pos, x, partial, k, chunks, st, maxcl, atomic);
    case 5: return launch_coupling_rtr_alt_5(N, pos, x, partial, k, chunks, st, maxcl, atomic);
    default: return cudaErrorInvalidValue;
  }
}
int coupling_rtr_rpb_v(int L, int precision, int variant) {
  if ((variant & 1) == 0 || precision == CELES_FP64) return coupling_rtr_receivers_per_block(L, precision);
  switch (L) {
    case 1: return coupling_rtr_alt_rpb_1();
    case 2: return coupling_rtr_alt_rpb_2();
    case 3: return coupling_rtr_alt_rpb_3();
    case 4: return coupling_rtr_alt_rpb_4();
    case 5: return coupling_rtr_alt_rpb_5();
    default: return 0;
  }
}
// partial-sum slices a launch with `chunks` source chunks writes (the
// cluster reduction of the shared-memory accumulator shapes divides it)
int coupling_rtr_slices_v(int L, int precision, int variant, int chunks) {
  const int maxcl = (variant & 2) ? 8 : 1;
  const int atomic = (variant & 4) && precision == CELES_FP32 ? 1 : 0;
  if ((variant & 1) == 0 || precision == CELES_FP64) {
    switch (L) {
      case 1: return coupling_rtr_slices_1(precision, chunks, maxcl, atomic);
      case 2: return coupling_rtr_slices_2(precision, chunks, maxcl, atomic);
      case 3: return coupling_rtr_slices_3(precision, chunks, maxcl, atomic);
      case 4: return coupling_rtr_slices_4(precision, chunks, maxcl, atomic);
      case 5: return coupling_rtr_slices_5(precision, chunks, maxcl, atomic);
      default: return chunks;
    }
  }
  switch (L) {
    case 1: return coupling_rtr_alt_slices_1(chunks, maxcl, atomic);
    case 2: return coupling_rtr_alt_slices_2(chunks, maxcl, atomic);
    case 3: return coupling_rtr_alt_slices_3(chunks, maxcl, atomic);
    case 4: return coupling_rtr_alt_slices_4(chunks, maxcl, atomic);
    case 5: return coupling_rtr_alt_slices_5(chunks, maxcl, atomic);
    default: return chunks;
  }
}
int coupling_rtr_slots_v(int L, int precision, int variant) {
  if ((variant & 1) == 0 || precision == CELES_FP64) return coupling_rtr_slots(L, precision);
  switch (L) {
    case 1: return coupling_rtr_alt_slots_1();
    case 2: return coupling_rtr_alt_slots_2();
    case 3: return coupling_rtr_alt_slots_3();
    case 4: return coupling_rtr_alt_slots_4();
    case 5: return coupling_rtr_alt_slots_5();
    default: return 0;
  }
}
int coupling_rtr_receivers_per_block(int L, int precision) {
  switch (L) {
    case 1: return coupling_rtr_rpb_1(precision);
    case 2: return coupling_rtr_rpb_2(precision);
    case 3: return coupling_rtr_rpb_3(precision);
    case 4: return coupling_rtr_rpb_4(precision);
    case 5: return coupling_rtr_rpb_5(precision);
    default: return 0;
  }
}
int coupling_rtr_slots(int L, int precision) {
  switch (L) {
    case 1: return coupling_rtr_slots_1(precision);
    case 2: return coupling_rtr_slots_2(precision);
    case 3: return coupling_rtr_slots_3(precision);
    case 4: return coupling_rtr_slots_4(precision);
    case 5: return coupling_rtr_slots_5(precision);
    default: return 0;
  }
}
long long coupling_rtr_flops(int L) {
  switch (L) {
    case 1: return coupling_rtr_flops_1();
    case 2: return coupling_rtr_flops_2();
    case 3: return coupling_rtr_flops_3();
    case 4: return coupling_rtr_flops_4();
    case 5: return coupling_rtr_flops_5();
    default: return -1;
  }
}
int coupling_receivers_per_block(int L, int precision) {
  switch (L) {
    case 1: return coupling_rpb_1(precision);
    case 2: return coupling_rpb_2(precision);
    case 3: return coupling_rpb_3(precision);
    case 4: return coupling_rpb_4(precision);
    case 5: return coupling_rpb_5(precision);
    default: return 0;
  }
}
int coupling_terms_export(int L, int* idx, double* val, int cap) {
  switch (L) {
    case 1: return coupling_terms_export_1(idx, val, cap);
    case 2: return coupling_terms_export_2(idx, val, cap);
    case 3: return coupling_terms_export_3(idx, val, cap);
    case 4: return coupling_terms_export_4(idx, val, cap);
    case 5: return coupling_terms_export_5(idx, val, cap);
    default: return -1;
  }
}
}  // namespace celes

using namespace celes;

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t ensure(size_t b) {
    if (b <= bytes && p) return cudaSuccess;
    release();
    if (b == 0) return cudaSuccess;
    const cudaError_t e = cudaMalloc(&p, b);
    if (e == cudaSuccess) bytes = b;
    else p = nullptr;
    return e;
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct celes_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t N = 0;
  int L = 0, NH = 0, nmax = 0;
  double n0 = 1.0, k0 = 0.0, k = 0.0;
  int chunks_opt = 0;
  int kernel = CELES_KERNEL_AUTO;
  int autotune = 1;
  // launch shape of the coupling kernel per precision (FP64, FP32): -1 until
  // the first product picks it (autotuner) or the default is taken
  int tune_variant[2] = {-1, -1};
  int tune_chunks[2] = {0, 0};
  double tune_ms[2] = {0.0, 0.0};
  DevBuf pos, radii, nrel, tq, tq32, tdiag;
  int nrhs = 0;
  std::vector<celes_incident> incidents;  // descriptors of the current RHS
  DevBuf ain, rhs, b, x0;
  bool has_b = false, has_x0 = false, x0_learned = false;
  DevBuf partial;
  // preconditioner
  bool has_precond = false;
  int64_t nblocks = 0;
  int64_t mat_entries = 0;  // complex entries of all blocks' factors
  int max_block_dim = 0;
  DevBuf block_off, mat_off, perm, mats, mats32, piv, pivperm, info, pwork;
  DevBuf tile_off, tinv, tinv32;  // explicit inverses of the diagonal 32 x 32 tiles of L and U
  int precond_csize = 1;          // CTAs per block in the cluster-form apply
  bool precond_inverse = false;  // mats / mats32 hold the inverses of L and U (two-product apply)
  // small device scratch
  DevBuf dots, dot_partial, flag;
  std::string err;
  // kernel timing (celes_profile)
  bool profiling = false;
  struct Rec {
    cudaEvent_t a, b;
    int which;
  };
  std::vector<Rec> recs;
  double prof_ms[3] = {0, 0, 0};
  int64_t prof_n[3] = {0, 0, 0};
};

static std::atomic<int64_t> g_launches{0};

namespace {

int fail(celes_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

int cuda_fail(celes_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(c, CELES_ENOMEM, "%s: device allocation failed", what);
  }
  return fail(c, CELES_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ck_status(celes_ctx* c, cudaError_t e, const char* what) { return e == cudaSuccess ? CELES_OK : cuda_fail(c, e, what); }

// CK(expression returning cudaError_t, "what"): return a celes_status on error
#define CK(...)                                   \
  do {                                            \
    const int rc_ = ck_status(c, __VA_ARGS__);    \
    if (rc_ != CELES_OK) return rc_;              \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

cudaStream_t pick_stream(celes_ctx* c, void* s) { return s ? static_cast<cudaStream_t>(s) : c->stream; }

bool use_rtr(const celes_ctx* c, int precision) {
  (void)precision;
  return c->kernel != CELES_KERNEL_DIRECT;
}

int auto_chunks(const celes_ctx* c, int precision) {
  if (c->chunks_opt > 0) return c->chunks_opt;
  const bool rtr = use_rtr(c, precision);
  const int rpb = rtr ? coupling_rtr_receivers_per_block(c->L, precision)
                      : coupling_receivers_per_block(c->L, precision);
  const int64_t rb = (c->N + rpb - 1) / rpb;
  // about eight waves of resident CTAs: the last, partly filled wave then
  // idles the GPU for a small fraction of the launch (measured: 12.7 ms at
  // eight waves vs 13.7 ms at four, lmax 4, N = 10 000)
  const int slots = rtr ? coupling_rtr_slots(c->L, precision) : 2 * device_sms();
  const int64_t target = 8LL * (slots > 0 ? slots : 2 * device_sms());
  int64_t ch = (target + rb - 1) / rb;
  const int64_t max_by_src = std::max<int64_t>(1, c->N / 64);
  ch = std::min<int64_t>(ch, max_by_src);
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ch, 256)));
}

// ---- autotuner of the coupling kernel's launch shape ----------------------
// Candidates: the compile-time shape (Config, and for FP32 ConfigAlt) times
// the number of source chunks (about 4, 8 or 16 waves of resident CTAs).
// Each is timed with CUDA events on the context's own positions (the first
// 20 000 spheres of larger problems) and the fastest kept, once per (device,
// lmax, precision, log2 N) for the whole process.
struct TuneKey {
  int dev, L, prec, bucket;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, L, prec, bucket) < std::tie(o.dev, o.L, o.prec, o.bucket);
  }
};
struct TuneVal {
  int variant = 0;
  double waves = 8.0;
  double ms = 0.0;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

int chunks_for(const celes_ctx* c, int64_t N, int precision, int variant, double waves) {
  const int rpb = coupling_rtr_rpb_v(c->L, precision, variant);
  const int64_t rb = (N + rpb - 1) / rpb;
  const int slots = coupling_rtr_slots_v(c->L, precision, variant);
  const double target = waves * (slots > 0 ? slots : 2 * device_sms());
  int64_t ch = static_cast<int64_t>(std::ceil(target / static_cast<double>(rb)));
  ch = std::min<int64_t>(ch, std::max<int64_t>(1, N / 64));
  ch = std::max<int64_t>(1, std::min<int64_t>(ch, 256));
  // a multiple of 8 (of 4 below 8): whole clusters for the partial-sum reduction
  if (ch >= 8) ch = (ch + 7) / 8 * 8;
  else if (ch >= 4) ch = 4;
  return static_cast<int>(std::min<int64_t>(ch, 256));
}

int autotune(celes_ctx* c, int precision, const void* x, cudaStream_t st) {
  const int pi = precision == CELES_FP64 ? 0 : 1;
  const int64_t Nt = std::min<int64_t>(c->N, 20000);
  int bucket = 0;
  while ((int64_t(1) << (bucket + 1)) <= c->N) ++bucket;
  const TuneKey key{c->device, c->L, precision, bucket};
  TuneVal best;
  bool have = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      best = it->second;
      have = true;
    }
  }
  if (!have) {
    const size_t elem = precision == CELES_FP64 ? 16 : 8;
    const size_t per = static_cast<size_t>(c->N) * c->nmax * elem;
    // shapes: FP32 built-in / alternative, each with the partial sums in
    // slices, added in clusters, added in L2, or both
    std::vector<int> vars =
        precision == CELES_FP64 ? std::vector<int>{0, 2} : std::vector<int>{0, 1, 2, 3, 4, 5, 6, 7};
    // waves of CTAs per launch; the L2 reduction (bit 2) makes more chunks
    // cost no DRAM traffic, so it also tries twice the largest count
    const double waves[4] = {4.0, 8.0, 16.0, 32.0};
    auto nwaves = [](int v) { return (v & 4) ? 4 : 3; };
    int maxch = 1;
    for (int v : vars)
      for (int wi = 0; wi < nwaves(v); ++wi) maxch = std::max(maxch, chunks_for(c, Nt, precision, v, waves[wi]));
    CK(c->partial.ensure(per * std::max(maxch, 1)), "coupling scratch");
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a), "event");
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return cuda_fail(c, cudaErrorMemoryAllocation, "event");
    }
    best.ms = 1e300;
    cudaError_t e = cudaSuccess;
    for (int v : vars) {
      if (e != cudaSuccess) break;
      for (int wi = 0; wi < nwaves(v); ++wi) {
        const double w = waves[wi];
        const int ch = chunks_for(c, Nt, precision, v, w);
        // one untimed launch (first use of the shape on this device), then one timed
        e = launch_coupling_rtr_v(c->L, precision, v, Nt, c->pos.p, x, c->partial.p, c->k, ch, st);
        if (e == cudaSuccess) e = cudaEventRecord(a, st);
        if (e == cudaSuccess) e = launch_coupling_rtr_v(c->L, precision, v, Nt, c->pos.p, x, c->partial.p, c->k, ch, st);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) break;
        if (ms < best.ms) {
          best.ms = ms;
          best.variant = v;
          best.waves = w;
        }
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  c->tune_variant[pi] = best.variant;
  c->tune_chunks[pi] = chunks_for(c, c->N, precision, best.variant, best.waves);
  c->tune_ms[pi] = best.ms;
  return CELES_OK;
}

// coupling (mode 0: y = W x) or master (mode 1: y = x - T W x) products
int prof_begin(celes_ctx* c, cudaStream_t st, celes_ctx::Rec& r, int which) {
  r.which = which;
  r.a = r.b = nullptr;
  cudaError_t e = cudaEventCreate(&r.a);
  if (e == cudaSuccess) e = cudaEventCreate(&r.b);
  if (e == cudaSuccess) e = cudaEventRecord(r.a, st);
  if (e != cudaSuccess) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
    r.a = r.b = nullptr;
    return cuda_fail(c, e, "event");
  }
  return CELES_OK;
}

int coupling_apply(celes_ctx* c, const void* x, void* y, int nrhs, int precision, int mode, cudaStream_t st) {
  const int pi = precision == CELES_FP64 ? 0 : 1;
  if (c->tune_chunks[pi] == 0) {
    const bool rtr = use_rtr(c, precision);
    // FP32 only: the FP64 kernel runs twice or so per solve (refinement
    // residuals), too few launches to repay timing its candidates
    if (c->tune_variant[pi] < 0 && c->autotune && c->chunks_opt == 0 && rtr && precision == CELES_FP32) {
      const int s = autotune(c, precision, x, st);
      if (s) return s;
    } else {
      if (c->tune_variant[pi] < 0) c->tune_variant[pi] = 0;
      c->tune_chunks[pi] = c->chunks_opt > 0 ? c->chunks_opt
                           : rtr             ? chunks_for(c, c->N, precision, c->tune_variant[pi], 8.0)
                                             : auto_chunks(c, precision);
    }
  }
  const int variant = c->tune_variant[pi];
  const int chunks = c->tune_chunks[pi];
  const int slices = use_rtr(c, precision) ? coupling_rtr_slices_v(c->L, precision, variant, chunks) : chunks;
  const size_t elem = precision == CELES_FP64 ? 16 : 8;
  const size_t per = static_cast<size_t>(c->N) * c->nmax * elem;
  CK(c->partial.ensure(per * chunks), "coupling scratch");
  for (int r = 0; r < nrhs; ++r) {
    const char* xr = static_cast<const char*>(x) + per * r;
    char* yr = static_cast<char*>(y) + per * r;
    celes_ctx::Rec rec{};
    if (c->profiling) {
      int s = prof_begin(c, st, rec, precision == CELES_FP64 ? 1 : 0);
      if (s) return s;
    }
    if (use_rtr(c, precision))
      CK(launch_coupling_rtr_v(c->L, precision, variant, c->N, c->pos.p, xr, c->partial.p, c->k, chunks, st),
         "coupling kernel");
    else
      CK(launch_coupling_partial(c->L, precision, c->N, c->pos.p, xr, c->partial.p, c->k, chunks, st),
         "coupling kernel");
    if (c->profiling) {
      CK(cudaEventRecord(rec.b, st), "event");
      c->recs.push_back(rec);
      int s = prof_begin(c, st, rec, 2);
      if (s) return s;
    }
    if (precision == CELES_FP64)
      CK(launch_coupling_epilogue<double>(c->N, c->L, slices, c->partial.p, xr, c->tq.p, yr, mode, st), "epilogue");
    else
      CK(launch_coupling_epilogue<float>(c->N, c->L, slices, c->partial.p, xr, c->tq32.p, yr, mode, st), "epilogue");
    if (c->profiling) {
      CK(cudaEventRecord(rec.b, st), "event");
      c->recs.push_back(rec);
    }
  }
  return CELES_OK;
}

void gauss_legendre(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  // Newton's iteration on P_n from the Chebyshev-like first guess
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      const double pn = n == 1 ? z : p1;
      const double pm = n == 1 ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      const double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (b - a) * (z + 1.0) + a;
    w[i] = (b - a) / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// creation / destruction
// ---------------------------------------------------------------------------
extern "C" int celes_create(celes_ctx** out, int64_t N, const double* positions, const double* radii,
                            const double* n_i, double n0, double k0, int lmax, const celes_options* opt) {
  celes::NvtxRange nvtx_range_("celes_create");
  if (!out) return CELES_EINVAL;
  *out = nullptr;
  if (N < 1 || !positions || !radii || !n_i || lmax < 1 || lmax > 5 || !(n0 > 0.0) || !(k0 > 0.0) ||
      N > (int64_t)1 << 30)
    return CELES_EINVAL;
  for (int64_t i = 0; i < N; ++i) {
    if (!(radii[i] > 0.0) || !std::isfinite(positions[3 * i]) || !std::isfinite(positions[3 * i + 1]) ||
        !std::isfinite(positions[3 * i + 2]))
      return CELES_EINVAL;
  }
  std::unique_ptr<celes_ctx> c(new celes_ctx());
  c->device = opt ? opt->device : 0;
  c->chunks_opt = opt ? opt->chunks : 0;
  c->kernel = opt ? opt->kernel : CELES_KERNEL_AUTO;
  c->autotune = opt ? opt->autotune : 1;
  if (opt && opt->variant >= 0) {
    // a forced launch shape (tests and measurements); the chunks as usual
    if (opt->variant > 7) return CELES_EINVAL;
    c->tune_variant[0] = opt->variant & 2;
    c->tune_variant[1] = opt->variant;
  }
  if (c->kernel < CELES_KERNEL_AUTO || c->kernel > CELES_KERNEL_RTR) return CELES_EINVAL;
  const int check_overlap = opt ? opt->check_overlap : 1;
  c->N = N;
  c->L = lmax;
  c->NH = lmax * (lmax + 2);
  c->nmax = 2 * c->NH;
  c->n0 = n0;
  c->k0 = k0;
  c->k = n0 * k0;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return CELES_ECUDA;
  }
  if (c->device < 0 || c->device >= ndev) return CELES_EINVAL;
  DeviceGuard dg(c->device);
  celes_ctx* cp = c.get();
#define CKC(expr, what)                                   \
  do {                                                    \
    const cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) {                              \
      cudaGetLastError();                                 \
      return e_ == cudaErrorMemoryAllocation ? CELES_ENOMEM : CELES_ECUDA; \
    }                                                     \
  } while (0)
  CKC(cudaStreamCreateWithFlags(&cp->stream, cudaStreamNonBlocking), "stream");
  std::vector<Pos4> hp(N);
  for (int64_t i = 0; i < N; ++i) hp[i] = Pos4{positions[3 * i], positions[3 * i + 1], positions[3 * i + 2], 0.0};
  std::vector<double> hn(2 * N);
  for (int64_t i = 0; i < N; ++i) {
    hn[2 * i] = n_i[2 * i] / n0;
    hn[2 * i + 1] = n_i[2 * i + 1] / n0;
  }
  CKC(cp->pos.ensure(sizeof(Pos4) * N), "positions");
  CKC(cp->radii.ensure(sizeof(double) * N), "radii");
  CKC(cp->nrel.ensure(sizeof(double) * 2 * N), "n");
  CKC(cp->tq.ensure(sizeof(double) * 2 * N * 2 * lmax), "tq");
  CKC(cp->tq32.ensure(sizeof(float) * 2 * N * 2 * lmax), "tq32");
  CKC(cp->tdiag.ensure(sizeof(double) * 2 * N * cp->nmax), "tdiag");
  CKC(cp->flag.ensure(sizeof(int) * 4), "flag");
  CKC(cudaMemcpyAsync(cp->pos.p, hp.data(), sizeof(Pos4) * N, cudaMemcpyHostToDevice, cp->stream), "h2d");
  CKC(cudaMemcpyAsync(cp->radii.p, radii, sizeof(double) * N, cudaMemcpyHostToDevice, cp->stream), "h2d");
  CKC(cudaMemcpyAsync(cp->nrel.p, hn.data(), sizeof(double) * 2 * N, cudaMemcpyHostToDevice, cp->stream), "h2d");
  if (check_overlap) {
    CKC(cudaMemsetAsync(cp->flag.p, 0, sizeof(int), cp->stream), "memset");
    CKC(launch_overlap_check(N, cp->pos.p, cp->radii.as<double>(), cp->flag.as<int>(), cp->stream), "overlap");
    int h = 0;
    CKC(cudaMemcpyAsync(&h, cp->flag.p, sizeof(int), cudaMemcpyDeviceToHost, cp->stream), "d2h");
    CKC(cudaStreamSynchronize(cp->stream), "sync");
    if (h) {
      cudaStreamDestroy(cp->stream);
      cp->stream = nullptr;
      return CELES_EOVERLAP;
    }
  }
  CKC(launch_mie(N, lmax, cp->k, cp->radii.as<double>(), cp->nrel.as<double>(), cp->tq.as<double>(), cp->stream),
      "mie");
  CKC(launch_tq_expand(N, lmax, cp->tq.as<double>(), cp->tdiag.as<double>(), cp->tq32.as<float>(), cp->stream),
      "tq expand");
  CKC(cudaMemsetAsync(cp->flag.p, 0, sizeof(int), cp->stream), "memset");
  CKC(launch_nonfinite<double>(4 * N * lmax, cp->tq.p, cp->flag.as<int>(), cp->stream), "scan");
  int bad = 0;
  CKC(cudaMemcpyAsync(&bad, cp->flag.p, sizeof(int), cudaMemcpyDeviceToHost, cp->stream), "d2h");
  CKC(cudaStreamSynchronize(cp->stream), "sync");
#undef CKC
  if (bad) {
    cudaStreamDestroy(cp->stream);
    cp->stream = nullptr;
    return CELES_ENUMERIC;
  }
  *out = c.release();
  return CELES_OK;
}

static void prof_flush(celes_ctx* c);

extern "C" void celes_destroy(celes_ctx* c) {
  if (!c) return;
  {
    DeviceGuard dg(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    prof_flush(c);
    if (c->stream) cudaStreamDestroy(c->stream);
    c->pos.release();
    c->radii.release();
    c->nrel.release();
    c->tq.release();
    c->tq32.release();
    c->tdiag.release();
    c->ain.release();
    c->rhs.release();
    c->b.release();
    c->x0.release();
    c->partial.release();
    c->block_off.release();
    c->mat_off.release();
    c->perm.release();
    c->mats.release();
    c->mats32.release();
    c->pivperm.release();
    c->tile_off.release();
    c->tinv.release();
    c->tinv32.release();
    c->piv.release();
    c->info.release();
    c->pwork.release();
    c->dots.release();
    c->dot_partial.release();
    c->flag.release();
  }
  delete c;
}

static void prof_flush(celes_ctx* c) {
  for (auto& r : c->recs) {
    float ms = 0.0f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.which] += ms;
      c->prof_n[r.which] += 1;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  c->recs.clear();
  cudaGetLastError();
}

extern "C" int celes_profile(celes_ctx* c, int on) {
  if (!c) return CELES_EINVAL;
  DeviceGuard dg(c->device);
  prof_flush(c);
  if (on) {
    for (int q = 0; q < 3; ++q) {
      c->prof_ms[q] = 0.0;
      c->prof_n[q] = 0;
    }
  }
  c->profiling = on != 0;
  return CELES_OK;
}

extern "C" int celes_kernel_time(celes_ctx* c, int which, double* ms, int64_t* launches) {
  if (!c) return CELES_EINVAL;
  if (which < 0 || which > 2 || !ms || !launches) return fail(c, CELES_EINVAL, "kernel_time: bad arguments");
  DeviceGuard dg(c->device);
  prof_flush(c);
  *ms = c->prof_ms[which];
  *launches = c->prof_n[which];
  return CELES_OK;
}

extern "C" int64_t celes_kernel_launches(void) { return g_launches.load() + celes::kernel_launch_count(); }

extern "C" double celes_flops_per_pair(int lmax, int kernel) {
  if (lmax < 1 || lmax > 5) return -1.0;
  if (kernel == CELES_KERNEL_DIRECT) {
    // per-entry evaluation: 4 (A + B terms) + 12 NH^2 + 2 NS (build) + 4 nmax^2 (apply)
    const int NH = lmax * (lmax + 2), NS = (2 * lmax + 1) * (2 * lmax + 2) / 2;
    return 4.0 * coupling_terms_export(lmax, nullptr, nullptr, 0) + 12.0 * NH * NH + 2.0 * NS + 4.0 * (2.0 * NH) * (2.0 * NH);
  }
  return static_cast<double>(coupling_rtr_flops(lmax));
}

extern "C" const char* celes_last_error(const celes_ctx* c) { return c ? c->err.c_str() : "null context"; }
extern "C" const char* celes_version(void) { return "celes-gb300 0.1 (sm_103a)"; }
extern "C" int64_t celes_num_spheres(const celes_ctx* c) { return c ? c->N : 0; }
extern "C" int celes_nmax(const celes_ctx* c) { return c ? c->nmax : 0; }
extern "C" int celes_num_rhs(const celes_ctx* c) { return c ? c->nrhs : 0; }

extern "C" int celes_coupling_terms(int lmax, int* idx, double* val, int cap) {
  if (lmax < 1 || lmax > 5 || cap < 0) return CELES_EINVAL;
  return coupling_terms_export(lmax, idx, val, cap);
}

// ---------------------------------------------------------------------------
// incident field
// ---------------------------------------------------------------------------
extern "C" int celes_set_incident(celes_ctx* c, const celes_incident* inc, int nrhs) {
  celes::NvtxRange nvtx_range_("celes_set_incident");
  if (!c) return CELES_EINVAL;
  if (!inc || nrhs < 1) return fail(c, CELES_EINVAL, "set_incident: need nrhs >= 1 descriptors");
  for (int r = 0; r < nrhs; ++r) {
    const celes_incident& d = inc[r];
    if (d.kind != CELES_PLANE_WAVE && d.kind != CELES_GAUSSIAN_BEAM)
      return fail(c, CELES_EINVAL, "set_incident: unknown kind %d", d.kind);
    if (d.kind == CELES_PLANE_WAVE && d.pol != 1 && d.pol != 2)
      return fail(c, CELES_EINVAL, "set_incident: pol must be 1 or 2");
    if (d.kind == CELES_GAUSSIAN_BEAM && !(d.waist > 0.0))
      return fail(c, CELES_EINVAL, "set_incident: waist must be > 0");
    if (d.kind == CELES_GAUSSIAN_BEAM && (d.n_beta < 0 || d.n_beta > 100000))
      return fail(c, CELES_EINVAL, "set_incident: n_beta out of range");
  }
  DeviceGuard dg(c->device);
  const size_t per = sizeof(double) * 2 * c->N * c->nmax;
  CK(c->ain.ensure(per * nrhs), "a_in");
  CK(c->rhs.ensure(per * nrhs), "rhs");
  CK(c->b.ensure(per * nrhs), "b");
  c->nrhs = nrhs;
  c->incidents.assign(inc, inc + nrhs);
  c->has_b = false;
  c->has_x0 = false;
  DevBuf nodes, weights;
  for (int r = 0; r < nrhs; ++r) {
    const celes_incident& d = inc[r];
    double* a = reinterpret_cast<double*>(c->ain.as<char>() + per * r);
    if (d.kind == CELES_PLANE_WAVE) {
      CK(launch_plane_wave(c->N, c->L, c->k, c->pos.p, d.beta, d.alpha, d.pol, d.E0_re, d.E0_im, a, c->stream),
         "plane wave");
    } else {
      const int nb = d.n_beta > 0 ? d.n_beta : 128;
      // beta range: the Gaussian factor exp(-w^2 k^2 sin^2(beta)/4) is below
      // 1e-17 beyond sin^2(beta) = 39.2 / (w k / 2)^2
      const double aa = std::pow(d.waist * c->k, 2) / 4.0;
      const double s2 = 39.2 / aa;
      const double bmax = s2 >= 1.0 ? M_PI / 2 : std::asin(std::sqrt(s2));
      std::vector<double> hx, hw;
      gauss_legendre(nb, 0.0, bmax, hx, hw);
      CK(nodes.ensure(sizeof(double) * nb), "nodes");
      CK(weights.ensure(sizeof(double) * nb), "weights");
      CK(cudaMemcpyAsync(nodes.p, hx.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, c->stream), "h2d");
      CK(cudaMemcpyAsync(weights.p, hw.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, c->stream), "h2d");
      CK(launch_gaussian_beam(c->N, c->L, c->k, c->pos.p, d.waist, d.focus, d.alpha_G, d.E0_re, d.E0_im, nb,
                              nodes.as<double>(), weights.as<double>(), a, c->stream),
         "gaussian beam");
      CK(cudaStreamSynchronize(c->stream), "sync");  // nodes/weights are freed at scope end
    }
  }
  CK(launch_tdiag_mul(c->N * c->nmax, nrhs, c->tdiag.as<double>(), c->ain.as<double>(), c->rhs.as<double>(),
                      c->stream),
     "T a");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CELES_OK;
}

// ---------------------------------------------------------------------------
// matvecs and preconditioner apply (device pointers, stream ordered)
// ---------------------------------------------------------------------------
extern "C" int celes_coupling_matvec(celes_ctx* c, const void* x, void* y, int nrhs, int precision, void* stream) {
  if (!c) return CELES_EINVAL;
  if (!x || !y || nrhs < 1 || (precision != CELES_FP64 && precision != CELES_FP32))
    return fail(c, CELES_EINVAL, "coupling_matvec: bad arguments");
  if (x == y) return fail(c, CELES_EINVAL, "coupling_matvec: x and y must not overlap");
  DeviceGuard dg(c->device);
  return coupling_apply(c, x, y, nrhs, precision, 0, pick_stream(c, stream));
}

extern "C" int celes_master_matvec(celes_ctx* c, const void* x, void* y, int nrhs, int precision, void* stream) {
  if (!c) return CELES_EINVAL;
  if (!x || !y || nrhs < 1 || (precision != CELES_FP64 && precision != CELES_FP32))
    return fail(c, CELES_EINVAL, "master_matvec: bad arguments");
  if (x == y) return fail(c, CELES_EINVAL, "master_matvec: x and y must not overlap");
  DeviceGuard dg(c->device);
  return coupling_apply(c, x, y, nrhs, precision, 1, pick_stream(c, stream));
}

extern "C" int celes_precond_build(celes_ctx* c, double edge) {
  celes::NvtxRange nvtx_range_("celes_precond_build");
  if (!c) return CELES_EINVAL;
  if (!(edge > 0.0)) return fail(c, CELES_EINVAL, "precond_build: edge must be > 0");
  DeviceGuard dg(c->device);
  // partition on the host (index bookkeeping only): cuboid of each centre,
  // grid anchored at the minimum corner, order (z, y, x), stable inside
  std::vector<Pos4> hp(c->N);
  CK(cudaMemcpy(hp.data(), c->pos.p, sizeof(Pos4) * c->N, cudaMemcpyDeviceToHost), "d2h");
  double lo[3] = {hp[0].x, hp[0].y, hp[0].z};
  for (const Pos4& p : hp) {
    lo[0] = std::min(lo[0], p.x);
    lo[1] = std::min(lo[1], p.y);
    lo[2] = std::min(lo[2], p.z);
  }
  std::vector<std::tuple<int64_t, int64_t, int64_t, int>> key(c->N);
  for (int64_t i = 0; i < c->N; ++i) {
    key[i] = std::make_tuple(static_cast<int64_t>(std::floor((hp[i].z - lo[2]) / edge)),
                             static_cast<int64_t>(std::floor((hp[i].y - lo[1]) / edge)),
                             static_cast<int64_t>(std::floor((hp[i].x - lo[0]) / edge)), static_cast<int>(i));
  }
  std::sort(key.begin(), key.end());
  std::vector<int> perm(c->N);
  std::vector<int64_t> boff{0};
  for (int64_t q = 0; q < c->N; ++q) {
    perm[q] = std::get<3>(key[q]);
    if (q > 0 && (std::get<0>(key[q]) != std::get<0>(key[q - 1]) || std::get<1>(key[q]) != std::get<1>(key[q - 1]) ||
                  std::get<2>(key[q]) != std::get<2>(key[q - 1])))
      boff.push_back(q);
  }
  boff.push_back(c->N);
  const int64_t nb = static_cast<int64_t>(boff.size()) - 1;
  std::vector<int64_t> moff(nb + 1, 0), toff(nb + 1, 0);
  int64_t max_pairs = 0, max_dim = 0, max_tiles = 0;
  for (int64_t q = 0; q < nb; ++q) {
    const int64_t ns = boff[q + 1] - boff[q];
    const int64_t n = ns * c->nmax;
    const int64_t nt = (n + 31) / 32;
    moff[q + 1] = moff[q] + n * n;
    toff[q + 1] = toff[q] + nt * 2048;
    max_pairs = std::max(max_pairs, ns * ns);
    max_dim = std::max(max_dim, n);
    max_tiles = std::max(max_tiles, nt);
  }
  c->has_precond = false;
  CK(c->block_off.ensure(sizeof(int64_t) * (nb + 1)), "block offsets");
  CK(c->mat_off.ensure(sizeof(int64_t) * (nb + 1)), "matrix offsets");
  CK(c->perm.ensure(sizeof(int) * c->N), "perm");
  CK(c->mats.ensure(sizeof(double) * 2 * moff[nb]), "LU factors");
  CK(c->mats32.ensure(sizeof(float) * 2 * moff[nb]), "LU factors (FP32 copy)");
  CK(c->piv.ensure(sizeof(int) * c->N * c->nmax), "pivots");
  CK(c->info.ensure(sizeof(int) * nb), "info");
  CK(cudaMemcpyAsync(c->block_off.p, boff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, c->stream), "h2d");
  CK(cudaMemcpyAsync(c->mat_off.p, moff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, c->stream), "h2d");
  CK(cudaMemcpyAsync(c->perm.p, perm.data(), sizeof(int) * c->N, cudaMemcpyHostToDevice, c->stream), "h2d");
  CK(launch_precond_assemble(c->L, nb, c->block_off.as<int64_t>(), c->mat_off.as<int64_t>(), c->perm.as<int>(),
                             c->pos.p, c->tq.as<double>(), c->k, c->mats.as<double>(), max_pairs, c->stream),
     "precond assembly");
  CK(launch_precond_lu(nb, c->block_off.as<int64_t>(), c->mat_off.as<int64_t>(), c->nmax, c->mats.as<double>(),
                       c->piv.as<int>(), c->info.as<int>(), c->stream),
     "precond LU");
  CK(launch_f64_to_f32(2 * moff[nb], c->mats.as<double>(), c->mats32.as<float>(), c->stream), "FP32 factors");
  CK(c->tile_off.ensure(sizeof(int64_t) * (nb + 1)), "tile offsets");
  CK(c->tinv.ensure(sizeof(double) * 2 * toff[nb]), "tile inverses");
  CK(c->tinv32.ensure(sizeof(float) * 2 * toff[nb]), "tile inverses (FP32 copy)");
  CK(cudaMemcpyAsync(c->tile_off.p, toff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, c->stream),
     "h2d");
  CK(launch_precond_tile_inverse(nb, max_tiles, c->block_off.as<int64_t>(), c->mat_off.as<int64_t>(),
                                 c->tile_off.as<int64_t>(), c->nmax, c->mats.as<double>(), c->tinv.as<double>(),
                                 c->stream),
     "tile inverses");
  CK(launch_f64_to_f32(2 * toff[nb], c->tinv.as<double>(), c->tinv32.as<float>(), c->stream), "FP32 tile inverses");
  c->precond_csize = precond_cluster_size(static_cast<double>(toff[nb] / 2048) / static_cast<double>(nb));
  // the apply's operator: the explicit inverses of L and U (FP64, and their
  // FP32 rounding), in place of the LU factors, when the block vectors fit in
  // shared memory
  c->precond_inverse = false;
  if (precond_inverse_fits(static_cast<int>(max_dim))) {
    DevBuf inv;
    CK(inv.ensure(sizeof(double) * 2 * moff[nb]), "inverse factors");
    CK(launch_precond_tri_inverse(nb, max_tiles, c->block_off.as<int64_t>(), c->mat_off.as<int64_t>(),
                                  c->tile_off.as<int64_t>(), c->nmax, c->mats.as<double>(), c->tinv.as<double>(),
                                  inv.as<double>(), c->stream),
       "inverse factors");
    CK(cudaStreamSynchronize(c->stream), "sync");
    std::swap(c->mats.p, inv.p);
    std::swap(c->mats.bytes, inv.bytes);
    CK(launch_f64_to_f32(2 * moff[nb], c->mats.as<double>(), c->mats32.as<float>(), c->stream), "FP32 inverses");
    c->precond_inverse = true;
  }
  CK(c->pivperm.ensure(sizeof(int) * c->N * c->nmax), "pivot permutation");
  CK(launch_pivot_perm(nb, c->block_off.as<int64_t>(), c->nmax, c->piv.as<int>(), c->pivperm.as<int>(), c->stream),
     "pivot permutation");
  std::vector<int> hinfo(nb);
  CK(cudaMemcpyAsync(hinfo.data(), c->info.p, sizeof(int) * nb, cudaMemcpyDeviceToHost, c->stream), "d2h");
  CK(cudaStreamSynchronize(c->stream), "sync");
  for (int64_t q = 0; q < nb; ++q)
    if (hinfo[q] != 0) return fail(c, CELES_ENUMERIC, "precond_build: block %lld is singular", (long long)q);
  c->nblocks = nb;
  c->mat_entries = moff[nb];
  c->max_block_dim = static_cast<int>(max_dim);
  c->has_precond = true;
  return CELES_OK;
}

extern "C" int celes_coupling_shape(const celes_ctx* c, int precision, int* variant, int* chunks, double* ms) {
  if (!c || (precision != CELES_FP64 && precision != CELES_FP32)) return CELES_EINVAL;
  const int pi = precision == CELES_FP64 ? 0 : 1;
  if (c->tune_chunks[pi] == 0) return CELES_ESTATE;
  if (variant) *variant = c->tune_variant[pi];
  if (chunks) *chunks = c->tune_chunks[pi];
  if (ms) *ms = c->tune_ms[pi];
  return CELES_OK;
}

extern "C" int celes_precond_stats(const celes_ctx* c, int64_t* nblocks, int64_t* max_dim, int64_t* entries) {
  if (!c) return CELES_EINVAL;
  if (!c->has_precond) return CELES_ESTATE;
  if (nblocks) *nblocks = c->nblocks;
  if (max_dim) *max_dim = c->max_block_dim;
  if (entries) *entries = c->mat_entries;
  return CELES_OK;
}

static int precond_apply_internal(celes_ctx* c, const void* x, void* y, int nrhs, int precision, cudaStream_t st) {
  CK(c->pwork.ensure(sizeof(double) * 2 * c->N * c->nmax * nrhs), "precond work");
  if (precision == CELES_FP64)
    CK(launch_precond_apply<double>(c->nblocks, c->block_off.as<int64_t>(), c->mat_off.as<int64_t>(), c->nmax,
                                    c->perm.as<int>(), c->mats.as<double>(), c->mats32.as<float>(), c->pivperm.as<int>(),
                                    c->N, nrhs, x, y, c->pwork.as<double>(), c->max_block_dim, st,
                                    c->tile_off.as<int64_t>(), c->tinv.as<double>(), c->tinv32.as<float>(),
                                    c->precond_csize, c->precond_inverse),
       "precond apply");
  else
    CK(launch_precond_apply<float>(c->nblocks, c->block_off.as<int64_t>(), c->mat_off.as<int64_t>(), c->nmax,
                                   c->perm.as<int>(), c->mats.as<double>(), c->mats32.as<float>(), c->pivperm.as<int>(),
                                   c->N, nrhs, x, y, c->pwork.as<double>(), c->max_block_dim, st,
                                   c->tile_off.as<int64_t>(), c->tinv.as<double>(), c->tinv32.as<float>(),
                                   c->precond_csize, c->precond_inverse),
       "precond apply");
  return CELES_OK;
}

extern "C" int celes_precond_apply(celes_ctx* c, const void* x, void* y, int nrhs, int precision, void* stream) {
  if (!c) return CELES_EINVAL;
  if (!x || !y || nrhs < 1 || (precision != CELES_FP64 && precision != CELES_FP32))
    return fail(c, CELES_EINVAL, "precond_apply: bad arguments");
  if (!c->has_precond) return fail(c, CELES_ESTATE, "precond_apply: no preconditioner built");
  DeviceGuard dg(c->device);
  return precond_apply_internal(c, x, y, nrhs, precision, pick_stream(c, stream));
}

// ---------------------------------------------------------------------------
// GMRES (right preconditioned, restarted, classical Gram-Schmidt applied
// twice, Givens rotations on the host)
// ---------------------------------------------------------------------------
namespace {

template <typename R>
struct Gmres {
  celes_ctx* c;
  int64_t n;        // unknowns of one RHS
  int m;            // restart
  bool precond;
  DevBuf V, w, z;   // basis (m+1 vectors), work vectors
  std::vector<std::complex<double>> H, cs_s, g;
  std::vector<double> cs_c;
  int prec() const { return sizeof(R) == 8 ? CELES_FP64 : CELES_FP32; }
  size_t vbytes() const { return sizeof(R) * 2 * n; }
  char* Vp(int j) { return V.as<char>() + vbytes() * j; }

  int init() {
    CK(V.ensure(vbytes() * (m + 1)), "Krylov basis");
    CK(w.ensure(vbytes()), "work");
    CK(z.ensure(vbytes()), "work");
    CK(c->dots.ensure(sizeof(double) * 2 * (m + 2)), "dots");
    CK(c->dot_partial.ensure(sizeof(double) * 2 * (m + 2) * vec_dot_blocks(n)), "dot partials");
    return CELES_OK;
  }
  // h[0..nv) = V[0..nv)^H v, on the host
  int dots(const void* Vbase, int nv, const void* v, std::vector<std::complex<double>>& h) {
    CK(launch_multi_dotc<R>(n, nv, Vbase, n, v, c->dot_partial.as<double>(), c->dots.as<double>(), c->stream), "dot");

    h.resize(nv);
    CK(cudaMemcpyAsync(h.data(), c->dots.p, sizeof(double) * 2 * nv, cudaMemcpyDeviceToHost, c->stream), "d2h");
    CK(cudaStreamSynchronize(c->stream), "sync");
    return CELES_OK;
  }
  int norm(const void* v, double& out) {
    std::vector<std::complex<double>> h;
    int s = dots(v, 1, v, h);
    if (s) return s;
    out = norm_from_dot(h[0].real());
    return CELES_OK;
  }
  // A v = M P^{-1} v
  int apply_op(const void* v, void* out, int& nmv) {
    const void* src = v;
    if (precond) {
      int s = precond_apply_internal(c, v, z.p, 1, prec(), c->stream);
      if (s) return s;
      src = z.p;
    }
    ++nmv;
    return coupling_apply(c, src, out, 1, prec(), 1, c->stream);
  }
  // Solve A u = r with x = P^{-1} u accumulated into x (x += P^{-1} u).
  // x0 of the Krylov iteration is zero.  r is not modified.  Stops when the
  // residual estimate <= tol * ||r|| or after max_it iterations.
  // hist_scale converts the estimate to the caller's relative residual.
  int solve(const void* r, void* x, double tol, int max_it, int& its, double& rel_est, int& nmv,
            std::vector<double>* hist, double hist_scale) {
    double rnorm = 0.0;
    int s = norm(r, rnorm);
    if (s) return s;
    its = 0;
    rel_est = 1.0;
    if (!std::isfinite(rnorm)) return fail(c, CELES_ENUMERIC, "GMRES: non-finite residual");
    if (!(rnorm > 0.0)) {
      rel_est = 0.0;
      return CELES_OK;
    }
    // start: u = 0, residual r; restarts use the updated residual computed
    // from the Arnoldi relation (no extra matvec), tracked by beta
    CK(launch_axpby<R, R>(n, 1.0 / rnorm, r, 0.0, Vp(0), c->stream), "v0");
    double beta = rnorm;  // current residual norm (estimate)
    bool first = true;
    while (its < max_it) {
      if (!first) {
        // explicit residual of the current correction: r - A u, where the
        // correction so far is already folded into x; recompute from w
        // (w holds r - A u_total, maintained below)
        double nb = 0.0;
        s = norm(w.p, nb);
        if (s) return s;
        if (!std::isfinite(nb)) return fail(c, CELES_ENUMERIC, "GMRES: non-finite residual");
        beta = nb;
        if (beta <= tol * rnorm) break;
        CK(launch_axpby<R, R>(n, 1.0 / beta, w.p, 0.0, Vp(0), c->stream), "v0");
      }
      first = false;
      H.assign((size_t)(m + 1) * m, 0.0);
      cs_c.assign(m, 0.0);
      cs_s.assign(m, 0.0);
      g.assign(m + 1, 0.0);
      g[0] = beta;
      int kk = 0;
      std::vector<std::complex<double>> h1, h2;
      for (kk = 0; kk < m && its < max_it; ++kk) {
        s = apply_op(Vp(kk), w.p, nmv);
        if (s) return s;
        // classical Gram-Schmidt, twice
        s = dots(V.p, kk + 1, w.p, h1);
        if (s) return s;
        CK(cudaMemcpyAsync(c->dots.p, h1.data(), sizeof(double) * 2 * (kk + 1), cudaMemcpyHostToDevice, c->stream),
           "h2d");
        CK(launch_multi_axpy<R>(n, kk + 1, V.p, n, c->dots.as<double>(), 1.0, w.p, c->stream), "axpy");
        s = dots(V.p, kk + 1, w.p, h2);
        if (s) return s;
        CK(cudaMemcpyAsync(c->dots.p, h2.data(), sizeof(double) * 2 * (kk + 1), cudaMemcpyHostToDevice, c->stream),
           "h2d");
        CK(launch_multi_axpy<R>(n, kk + 1, V.p, n, c->dots.as<double>(), 1.0, w.p, c->stream), "axpy");
        for (int j = 0; j <= kk; ++j) H[(size_t)j * m + kk] = h1[j] + h2[j];
        double hn = 0.0;
        s = norm(w.p, hn);
        if (s) return s;
        if (!std::isfinite(hn)) return fail(c, CELES_ENUMERIC, "GMRES: non-finite Krylov vector");
        H[(size_t)(kk + 1) * m + kk] = hn;
        if (hn > 0.0) CK(launch_axpby<R, R>(n, 1.0 / hn, w.p, 0.0, Vp(kk + 1), c->stream), "normalise");
        for (int j = 0; j < kk; ++j) {
          const std::complex<double> a = H[(size_t)j * m + kk], b = H[(size_t)(j + 1) * m + kk];
          H[(size_t)j * m + kk] = cs_c[j] * a + cs_s[j] * b;
          H[(size_t)(j + 1) * m + kk] = -std::conj(cs_s[j]) * a + cs_c[j] * b;
        }
        const std::complex<double> a = H[(size_t)kk * m + kk], b = H[(size_t)(kk + 1) * m + kk];
        if (std::abs(b) == 0.0) {
          cs_c[kk] = 1.0;
          cs_s[kk] = 0.0;
        } else if (std::abs(a) == 0.0) {
          cs_c[kk] = 0.0;
          cs_s[kk] = 1.0;
        } else {
          const double den = std::sqrt(std::norm(a) + std::norm(b));
          cs_c[kk] = std::abs(a) / den;
          cs_s[kk] = (a / std::abs(a)) * std::conj(b) / den;
        }
        H[(size_t)kk * m + kk] = cs_c[kk] * a + cs_s[kk] * b;
        H[(size_t)(kk + 1) * m + kk] = 0.0;
        g[kk + 1] = -std::conj(cs_s[kk]) * g[kk];
        g[kk] = cs_c[kk] * g[kk];
        ++its;
        rel_est = std::abs(g[kk + 1]) / rnorm;
        if (hist) hist->push_back(rel_est * hist_scale);
        if (std::abs(g[kk + 1]) <= tol * rnorm || hn == 0.0) {
          ++kk;
          break;
        }
      }
      // y = H^{-1} g (upper triangular), u = V y, x += P^{-1} u
      std::vector<std::complex<double>> y(kk);
      for (int i = kk - 1; i >= 0; --i) {
        std::complex<double> sacc = g[i];
        for (int j = i + 1; j < kk; ++j) sacc -= H[(size_t)i * m + j] * y[j];
        const std::complex<double> d = H[(size_t)i * m + i];
        if (std::abs(d) == 0.0) return fail(c, CELES_ENUMERIC, "GMRES: singular Hessenberg");
        y[i] = sacc / d;
      }
      CK(cudaMemcpyAsync(c->dots.p, y.data(), sizeof(double) * 2 * kk, cudaMemcpyHostToDevice, c->stream), "h2d");
      CK(launch_multi_combine<R>(n, kk, V.p, n, c->dots.as<double>(), 0.0, z.p, c->stream), "combine");
      if (precond) {
        s = precond_apply_internal(c, z.p, z.p, 1, prec(), c->stream);
        if (s) return s;
      }
      CK(launch_axpby<R, R>(n, 1.0, z.p, 1.0, x, c->stream), "update");
      if (std::abs(g[kk]) <= tol * rnorm || its >= max_it) break;
      // true residual of the correction for the restart: w = r - A x_corr is
      // not available without the accumulated correction, so the caller's x
      // must hold only this solve's correction (it does: solve() is called
      // with x = 0 on entry); w = r - M x
      s = coupling_apply(c, x, w.p, 1, prec(), 1, c->stream);
      ++nmv;
      if (s) return s;
      CK(launch_axpby<R, R>(n, 1.0, r, -1.0, w.p, c->stream), "residual");
    }
    return CELES_OK;
  }
};

// BiCGSTAB (van der Vorst 1992), right preconditioned, for the same inner
// problem as Gmres::solve: A u = r with A = M P^{-1}, u0 = 0, x += P^{-1} u.
// Per iteration two operator applications and three host reductions:
// [rho, ||r||^2], <r^, v>, [<t, t>, <s, t>].
template <typename R>
struct Bicgstab {
  celes_ctx* c;
  int64_t n;
  bool precond;
  DevBuf W, z;  // W: 7 vectors [r^ | r | t | s | p | v | u], z: preconditioned work vector
  enum { RH = 0, RR = 1, TT = 2, SS = 3, PP = 4, VV = 5, UU = 6 };
  int prec() const { return sizeof(R) == 8 ? CELES_FP64 : CELES_FP32; }
  size_t vbytes() const { return sizeof(R) * 2 * n; }
  char* Wp(int j) { return W.as<char>() + vbytes() * j; }

  int init() {
    CK(W.ensure(vbytes() * 7), "BiCGSTAB vectors");
    CK(z.ensure(vbytes()), "work");
    CK(c->dots.ensure(sizeof(double) * 2 * 4), "dots");
    CK(c->dot_partial.ensure(sizeof(double) * 2 * 4 * vec_dot_blocks(n)), "dot partials");
    return CELES_OK;
  }
  int dots(const void* Vbase, int nv, const void* v, std::complex<double>* h) {
    CK(launch_multi_dotc<R>(n, nv, Vbase, n, v, c->dot_partial.as<double>(), c->dots.as<double>(), c->stream), "dot");
    CK(cudaMemcpyAsync(h, c->dots.p, sizeof(double) * 2 * nv, cudaMemcpyDeviceToHost, c->stream), "d2h");
    CK(cudaStreamSynchronize(c->stream), "sync");
    return CELES_OK;
  }
  int apply_op(const void* v, void* out, int& nmv) {
    const void* src = v;
    if (precond) {
      int s = precond_apply_internal(c, v, z.p, 1, prec(), c->stream);
      if (s) return s;
      src = z.p;
    }
    ++nmv;
    return coupling_apply(c, src, out, 1, prec(), 1, c->stream);
  }
  int zaxpby(std::complex<double> a, int x, std::complex<double> b, int y, int zz) {
    CK(launch_caxpbyz<R>(n, a.real(), a.imag(), Wp(x), b.real(), b.imag(), Wp(y), Wp(zz), c->stream), "axpby");
    return CELES_OK;
  }
  int solve(const void* r, void* x, double tol, int max_it, int& its, double& rel_est, int& nmv,
            std::vector<double>* hist, double hist_scale) {
    its = 0;
    rel_est = 1.0;
    CK(cudaMemcpyAsync(Wp(RH), r, vbytes(), cudaMemcpyDeviceToDevice, c->stream), "r^");
    CK(cudaMemcpyAsync(Wp(RR), r, vbytes(), cudaMemcpyDeviceToDevice, c->stream), "r");
    CK(cudaMemsetAsync(Wp(UU), 0, vbytes(), c->stream), "u");
    std::complex<double> h[2];
    int s = dots(Wp(RH), 2, Wp(RR), h);  // [<r^, r>, <r, r>]
    if (s) return s;
    const double r0 = norm_from_dot(h[1].real());
    if (!std::isfinite(r0)) return fail(c, CELES_ENUMERIC, "BiCGSTAB: non-finite residual");
    if (!(r0 > 0.0)) {
      rel_est = 0.0;
      return CELES_OK;
    }
    std::complex<double> rho = h[0], rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    while (its < max_it) {
      if (std::abs(rho) == 0.0) break;  // breakdown: keep the current iterate
      if (its == 0) {
        CK(cudaMemcpyAsync(Wp(PP), Wp(RR), vbytes(), cudaMemcpyDeviceToDevice, c->stream), "p");
      } else {
        const std::complex<double> beta = (rho / rho_prev) * (alpha / omega);
        s = zaxpby(1.0, PP, -omega, VV, PP);  // p = p - omega v
        if (s) return s;
        s = zaxpby(1.0, RR, beta, PP, PP);  // p = r + beta p
        if (s) return s;
      }
      s = apply_op(Wp(PP), Wp(VV), nmv);
      if (s) return s;
      std::complex<double> rv;
      s = dots(Wp(RH), 1, Wp(VV), &rv);
      if (s) return s;
      if (std::abs(rv) == 0.0) break;
      alpha = rho / rv;
      s = zaxpby(1.0, RR, -alpha, VV, SS);  // s = r - alpha v
      if (s) return s;
      s = apply_op(Wp(SS), Wp(TT), nmv);
      if (s) return s;
      s = dots(Wp(TT), 2, Wp(TT), h);  // [<t, t>, <s, t>]
      if (s) return s;
      const double tt = h[0].real();
      omega = tt > 0.0 ? std::conj(h[1]) / tt : 0.0;  // <t, s> / <t, t>
      s = zaxpby(1.0, UU, alpha, PP, UU);  // u += alpha p + omega s
      if (s) return s;
      s = zaxpby(1.0, UU, omega, SS, UU);
      if (s) return s;
      s = zaxpby(1.0, SS, -omega, TT, RR);  // r = s - omega t
      if (s) return s;
      ++its;
      rho_prev = rho;
      s = dots(Wp(RH), 2, Wp(RR), h);
      if (s) return s;
      rho = h[0];
      const double rn = norm_from_dot(h[1].real());
      if (!std::isfinite(rn)) return fail(c, CELES_ENUMERIC, "BiCGSTAB: non-finite residual");
      rel_est = rn / r0;
      if (hist) hist->push_back(rel_est * hist_scale);
      if (rn <= tol * r0 || std::abs(omega) == 0.0) break;
    }
    // x += P^{-1} u
    if (precond) {
      int q = precond_apply_internal(c, Wp(UU), z.p, 1, prec(), c->stream);
      if (q) return q;
      CK(launch_axpby<R, R>(n, 1.0, z.p, 1.0, x, c->stream), "update");
    } else {
      CK(launch_axpby<R, R>(n, 1.0, Wp(UU), 1.0, x, c->stream), "update");
    }
    return CELES_OK;
  }
};

// the inner solver chosen by the options
template <typename R>
struct Inner {
  Gmres<R> g;
  Bicgstab<R> b;
  bool bicg;
  Inner(celes_ctx* c, int64_t n, int m, bool pc, bool use_bicg)
      : g{c, n, m, pc}, b{c, n, pc}, bicg(use_bicg) {}
  int init() { return bicg ? b.init() : g.init(); }
  int norm(const void* v, double& out) { return g.norm(v, out); }
  int solve(const void* r, void* x, double tol, int max_it, int& its, double& rel_est, int& nmv,
            std::vector<double>* hist, double hist_scale) {
    return bicg ? b.solve(r, x, tol, max_it, its, rel_est, nmv, hist, hist_scale)
                : g.solve(r, x, tol, max_it, its, rel_est, nmv, hist, hist_scale);
  }
};

}  // namespace

namespace celes {
void gauss_legendre_nodes(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  gauss_legendre(n, a, b, x, w);
}

int ctx_view(celes_ctx* c, CtxView* v) {
  if (!c || !v) return CELES_EINVAL;
  v->N = c->N;
  v->L = c->L;
  v->nmax = c->nmax;
  v->nrhs = c->nrhs;
  v->k = c->k;
  v->pos = c->pos.p;
  v->radii = c->radii.as<double>();
  v->nrel = c->nrel.as<double>();
  v->rhs = c->rhs.as<double>();
  v->b = c->b.as<double>();
  v->has_b = c->has_b;
  v->tq = c->tq.p;
  v->tq32 = c->tq32.p;
  v->device = c->device;
  v->incidents = c->incidents.data();
  v->stream = c->stream;
  if (c->nrhs < 1) return CELES_ESTATE;
  return CELES_OK;
}

int ctx_mark_solved(celes_ctx* c) {
  if (!c || c->nrhs < 1) return CELES_EINVAL;
  c->has_b = true;
  return CELES_OK;
}

int ctx_set_learned_guess(celes_ctx* c, int rhs, const double* b0_dev) {
  if (!c || !b0_dev || rhs < 0 || rhs >= c->nrhs) return CELES_EINVAL;
  DeviceGuard dg(c->device);
  const size_t per = sizeof(double) * 2 * c->N * c->nmax;
  CK(c->x0.ensure(per * c->nrhs), "x0");
  if (!c->x0_learned) CK(cudaMemcpyAsync(c->x0.p, c->rhs.p, per * c->nrhs, cudaMemcpyDeviceToDevice, c->stream), "x0");
  CK(cudaMemcpyAsync(c->x0.as<char>() + per * rhs, b0_dev, per, cudaMemcpyDeviceToDevice, c->stream), "x0");
  CK(cudaStreamSynchronize(c->stream), "sync");
  c->has_x0 = true;
  c->x0_learned = true;
  return CELES_OK;
}
}  // namespace celes

extern "C" int celes_set_initial_guess(celes_ctx* c, const double* b0) {
  if (!c) return CELES_EINVAL;
  if (!b0) return fail(c, CELES_EINVAL, "set_initial_guess: null pointer");
  if (c->nrhs < 1) return fail(c, CELES_ESTATE, "set_initial_guess: call set_incident first");
  DeviceGuard dg(c->device);
  const size_t bytes = sizeof(double) * 2 * c->N * c->nmax * c->nrhs;
  CK(c->x0.ensure(bytes), "x0");
  CK(cudaMemcpy(c->x0.p, b0, bytes, cudaMemcpyHostToDevice), "h2d");
  c->has_x0 = true;
  c->x0_learned = false;
  return CELES_OK;
}

extern "C" int celes_solve(celes_ctx* c, double tol, const celes_solve_opts* o, celes_solve_info* info) {
  celes::NvtxRange nvtx_range_("celes_solve");
  if (!c) return CELES_EINVAL;
  if (c->nrhs < 1) return fail(c, CELES_ESTATE, "solve: call set_incident first");
  if (!(tol > 0.0)) return fail(c, CELES_EINVAL, "solve: tol must be > 0");
  celes_solve_opts opt{CELES_SOLVE_MIXED, 100, 2000, 20, CELES_X0_TA, 1, 1e-5, CELES_SOLVER_GMRES};
  if (o) opt = *o;
  if (opt.restart <= 0) opt.restart = 100;
  if (opt.max_iter <= 0) opt.max_iter = 2000;
  if (opt.max_outer <= 0) opt.max_outer = 20;
  if (!(opt.inner_tol > 0.0)) opt.inner_tol = 1e-5;
  if (opt.mode != CELES_SOLVE_FP64 && opt.mode != CELES_SOLVE_MIXED)
    return fail(c, CELES_EINVAL, "solve: unknown mode %d", opt.mode);
  if (opt.x0 == CELES_X0_USER && !c->has_x0) return fail(c, CELES_ESTATE, "solve: no user initial guess set");
  if (opt.x0 == CELES_X0_LEARNED && !(c->has_x0 && c->x0_learned))
    return fail(c, CELES_ESTATE, "solve: no learned guess (call celes_gnn_predict)");
  if (opt.x0 < CELES_X0_TA || opt.x0 > CELES_X0_LEARNED) return fail(c, CELES_EINVAL, "solve: unknown x0 kind");
  if (opt.solver != CELES_SOLVER_GMRES && opt.solver != CELES_SOLVER_BICGSTAB)
    return fail(c, CELES_EINVAL, "solve: unknown solver %d", opt.solver);
  const bool bicg = opt.solver == CELES_SOLVER_BICGSTAB;
  DeviceGuard dg(c->device);
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = c->N * c->nmax;
  const size_t per64 = sizeof(double) * 2 * n;
  const bool use_pc = opt.use_precond && c->has_precond;
  std::vector<double> hist;
  int total_its = 0, outer = 0, mv64 = 0, mv32 = 0, guess_used = 0;
  double worst = 0.0;
  int status = CELES_OK;
  DevBuf r64, d64, r32, d32;
  CK(r64.ensure(per64), "residual");
  Inner<double> g64(c, n, opt.restart, use_pc, bicg);
  Inner<float> g32(c, n, opt.restart, use_pc, bicg);
  if (opt.mode == CELES_SOLVE_FP64) {
    int s = g64.init();
    if (s) return s;
    CK(d64.ensure(per64), "correction");
  } else {
    int s = g32.init();
    if (s) return s;
    CK(r32.ensure(per64 / 2), "residual32");
    CK(d32.ensure(per64 / 2), "correction32");
  }
  for (int rr = 0; rr < c->nrhs; ++rr) {
    double* rhs = reinterpret_cast<double*>(c->rhs.as<char>() + per64 * rr);
    double* b = reinterpret_cast<double*>(c->b.as<char>() + per64 * rr);
    // initial guess
    if (opt.x0 == CELES_X0_TA) CK(cudaMemcpyAsync(b, rhs, per64, cudaMemcpyDeviceToDevice, c->stream), "x0");
    else if (opt.x0 == CELES_X0_USER || opt.x0 == CELES_X0_LEARNED)
      CK(cudaMemcpyAsync(b, c->x0.as<char>() + per64 * rr, per64, cudaMemcpyDeviceToDevice, c->stream), "x0");
    else CK(cudaMemsetAsync(b, 0, per64, c->stream), "x0");
    double rhs_norm = 0.0;
    {
      int s = g64.norm(rhs, rhs_norm);
      if (s) return s;
    }
    if (opt.x0 == CELES_X0_LEARNED) {
      // keep the learned first iterate only if its residual is below that of
      // T a_in (residuals in the precision of the solve's first residual)
      const int pr = opt.mode == CELES_SOLVE_FP64 ? CELES_FP64 : CELES_FP32;
      double rn[2] = {0.0, 0.0};
      for (int cand = 0; cand < 2; ++cand) {
        const double* xv = cand == 0 ? rhs : b;
        if (pr == CELES_FP64) {
          int s = coupling_apply(c, xv, r64.p, 1, CELES_FP64, 1, c->stream);
          if (s) return s;
          ++mv64;
          CK(launch_axpby<double, double>(n, 1.0, rhs, -1.0, r64.p, c->stream), "residual");
          s = g64.norm(r64.p, rn[cand]);
          if (s) return s;
        } else {
          CK(launch_axpby<double, float>(n, 1.0, xv, 0.0, d32.p, c->stream), "cast");
          int s = coupling_apply(c, d32.p, r32.p, 1, CELES_FP32, 1, c->stream);
          if (s) return s;
          ++mv32;
          CK(launch_axpby<double, float>(n, 1.0, rhs, -1.0, r32.p, c->stream), "residual32");
          s = g32.norm(r32.p, rn[cand]);
          if (s) return s;
        }
      }
      if (rn[1] < rn[0]) {
        ++guess_used;
      } else {
        CK(cudaMemcpyAsync(b, rhs, per64, cudaMemcpyDeviceToDevice, c->stream), "x0");
      }
    } else if (opt.x0 == CELES_X0_USER) {
      ++guess_used;
    }
    if (!(rhs_norm > 0.0)) {
      CK(cudaMemsetAsync(b, 0, per64, c->stream), "zero");
      continue;
    }
    double rel = 1.0;
    if (opt.mode == CELES_SOLVE_FP64) {
      int its_left = opt.max_iter - total_its;
      while (true) {
        // r = rhs - M b
        int s = coupling_apply(c, b, r64.p, 1, CELES_FP64, 1, c->stream);
        if (s) return s;
        ++mv64;
        CK(launch_axpby<double, double>(n, 1.0, rhs, -1.0, r64.p, c->stream), "residual");
        double rn = 0.0;
        s = g64.norm(r64.p, rn);
        if (s) return s;
        if (!std::isfinite(rn)) return fail(c, CELES_ENUMERIC, "solve: non-finite residual");
        rel = rn / rhs_norm;
        hist.push_back(rel);
        if (rel <= tol || its_left <= 0) break;
        int its = 0;
        double est = 0.0;
        CK(cudaMemsetAsync(d64.p, 0, per64, c->stream), "zero");
        s = g64.solve(r64.p, d64.p, tol / rel, its_left, its, est, mv64, &hist, rel);
        if (s) return s;
        CK(launch_axpby<double, double>(n, 1.0, d64.p, 1.0, b, c->stream), "update");
        total_its += its;
        its_left -= its;
        ++outer;
        if (its == 0) break;
      }
    } else {
      // FP32 inner solves with FP64 residuals (iterative refinement)
      int its_left = opt.max_iter - total_its;
      int k_outer = 0;
      CK(launch_axpby<double, float>(n, 1.0, b, 0.0, d32.p, c->stream), "cast");
      // first residual in FP32: r = rhs - M b
      int s = coupling_apply(c, d32.p, r32.p, 1, CELES_FP32, 1, c->stream);
      if (s) return s;
      ++mv32;
      CK(launch_axpby<double, float>(n, 1.0, rhs, -1.0, r32.p, c->stream), "residual32");
      double rn = 0.0;
      {
        s = g32.norm(r32.p, rn);
        if (s) return s;
      }
      if (!std::isfinite(rn)) return fail(c, CELES_ENUMERIC, "solve: non-finite residual");
      rel = rn / rhs_norm;
      hist.push_back(rel);
      while (true) {
        if (k_outer > 0) {
          s = coupling_apply(c, b, r64.p, 1, CELES_FP64, 1, c->stream);
          if (s) return s;
          ++mv64;
          CK(launch_axpby<double, double>(n, 1.0, rhs, -1.0, r64.p, c->stream), "residual");
          s = g64.norm(r64.p, rn);
          if (s) return s;
          if (!std::isfinite(rn)) return fail(c, CELES_ENUMERIC, "solve: non-finite residual");
          rel = rn / rhs_norm;
          hist.push_back(rel);
          if (rel <= tol || its_left <= 0 || k_outer >= opt.max_outer) break;
          CK(launch_axpby<double, float>(n, 1.0 / rn, r64.p, 0.0, r32.p, c->stream), "cast residual");
        } else {
          CK(launch_axpby<float, float>(n, 1.0 / rn, r32.p, 0.0, r32.p, c->stream), "scale");
        }
        const double inner_tol = std::max(opt.inner_tol, 0.3 * tol / rel);
        CK(cudaMemsetAsync(d32.p, 0, per64 / 2, c->stream), "zero");
        int its = 0;
        double est = 0.0;
        s = g32.solve(r32.p, d32.p, inner_tol, its_left, its, est, mv32, &hist, rel);
        if (s) return s;
        total_its += its;
        its_left -= its;
        // b += rn * d
        CK(launch_axpby<float, double>(n, rn, d32.p, 1.0, b, c->stream), "update");
        ++k_outer;
        if (its == 0) break;
      }
      outer += k_outer;
    }
    worst = std::max(worst, rel);
    if (rel > tol) status = CELES_ENOCONV;
  }
  CK(cudaStreamSynchronize(c->stream), "sync");
  c->has_b = true;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) {
    info->status = status;
    info->iterations = total_its;
    info->outer = outer;
    info->matvecs_fp64 = mv64;
    info->matvecs_fp32 = mv32;
    info->residual = worst;
    info->seconds = secs;
    info->history_len = 0;
    info->guess_used = guess_used;
    if (info->history && info->history_cap > 0) {
      const int nh = std::min<int>(info->history_cap, static_cast<int>(hist.size()));
      std::memcpy(info->history, hist.data(), sizeof(double) * nh);
      info->history_len = nh;
    }
  }
  if (status == CELES_ENOCONV) return fail(c, CELES_ENOCONV, "solve: residual %.3e above tol %.3e", worst, tol);
  return CELES_OK;
}

// ---------------------------------------------------------------------------
// results
// ---------------------------------------------------------------------------
extern "C" int celes_get_coefficients(celes_ctx* c, double* out) {
  if (!c) return CELES_EINVAL;
  if (!out) return fail(c, CELES_EINVAL, "get_coefficients: null pointer");
  if (!c->has_b) return fail(c, CELES_ESTATE, "get_coefficients: no solution yet");
  DeviceGuard dg(c->device);
  CK(cudaMemcpy(out, c->b.p, sizeof(double) * 2 * c->N * c->nmax * c->nrhs, cudaMemcpyDeviceToHost), "d2h");
  return CELES_OK;
}

extern "C" int celes_get_incident_coefficients(celes_ctx* c, double* out) {
  if (!c) return CELES_EINVAL;
  if (!out) return fail(c, CELES_EINVAL, "get_incident_coefficients: null pointer");
  if (c->nrhs < 1) return fail(c, CELES_ESTATE, "get_incident_coefficients: call set_incident first");
  DeviceGuard dg(c->device);
  CK(cudaMemcpy(out, c->ain.p, sizeof(double) * 2 * c->N * c->nmax * c->nrhs, cudaMemcpyDeviceToHost), "d2h");
  return CELES_OK;
}

extern "C" int celes_get_tmatrix(celes_ctx* c, double* out) {
  if (!c) return CELES_EINVAL;
  if (!out) return fail(c, CELES_EINVAL, "get_tmatrix: null pointer");
  DeviceGuard dg(c->device);
  CK(cudaMemcpy(out, c->tdiag.p, sizeof(double) * 2 * c->N * c->nmax, cudaMemcpyDeviceToHost), "d2h");
  return CELES_OK;
}

extern "C" int celes_farfield(celes_ctx* c, const double* dirs, int64_t Nd, double* g, int rhs) {
  celes::NvtxRange nvtx_range_("celes_farfield");
  if (!c) return CELES_EINVAL;
  if (!dirs || !g || Nd < 1) return fail(c, CELES_EINVAL, "farfield: bad arguments");
  if (!c->has_b) return fail(c, CELES_ESTATE, "farfield: no solution yet");
  if (rhs < 0 || rhs >= c->nrhs) return fail(c, CELES_EINVAL, "farfield: rhs out of range");
  DeviceGuard dg(c->device);
  DevBuf dd, dg_;
  CK(dd.ensure(sizeof(double) * 2 * Nd), "dirs");
  CK(dg_.ensure(sizeof(double) * 4 * Nd), "g");
  CK(cudaMemcpyAsync(dd.p, dirs, sizeof(double) * 2 * Nd, cudaMemcpyHostToDevice, c->stream), "h2d");
  const double* b = reinterpret_cast<const double*>(c->b.as<char>() + sizeof(double) * 2 * c->N * c->nmax * rhs);
  CK(launch_farfield(c->N, c->L, c->k, c->pos.p, b, Nd, dd.as<double>(), dg_.as<double>(), c->stream), "farfield");
  CK(cudaMemcpyAsync(g, dg_.p, sizeof(double) * 4 * Nd, cudaMemcpyDeviceToHost, c->stream), "d2h");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CELES_OK;
}
