// Batched solves over many sphere ensembles and right-hand sides.
//
// A "system" is one right-hand side of one ensemble (context).  The batch
// concatenates the unknowns of all its systems into flat vectors and runs one
// lockstep solve of the master equation (I - T W) b = T a_in (Sec. 2.2) for
// all of them:
//  * the coupling products of every system of the same lmax are one persistent
//    launch (rtr_batch_kernel): CTAs draw (system, receiver block, source
//    chunk) tiles from a global counter, so ensembles of very different size
//    share the GPU without a tail per ensemble;
//  * the operator (all lmax groups plus the epilogue y = x - T (W x)) is
//    captured once in a CUDA graph per precision and replayed; the graph reads
//    its input/output pointers and the per-system active flags from a device
//    descriptor array, so it is replayed unchanged for every Krylov vector;
//  * the Krylov vector work (Gram-Schmidt dots and updates, scaling, the final
//    combination) runs in segmented kernels over all systems, with one
//    device-to-host copy per Gram-Schmidt stage for the whole batch;
//  * converged systems are masked out of every later launch.
// The solve is the same restarted right-preconditioner-free GMRES with
// classical Gram-Schmidt applied twice and FP64 residual refinement as the
// per-context solver (Sec. 3.2), run per system; Givens rotations run on the
// host per system.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/celes.h"
#include "coupling_kernel.cuh"
#include "kernels.h"
#include "rtr_kernel.cuh"

namespace celes {
#define CELES_DECLARE_RTR_BATCH(LL)                                                                       \
  cudaError_t launch_rtr_batch_##LL(int precision, const void* sys, int nsys, long long ntiles,          \
                                    unsigned long long* counter, cudaStream_t st);                       \
  int coupling_rtr_rpb_##LL(int precision);
}  // namespace celes
namespace celes {
int coupling_rtr_slots(int L, int precision);
CELES_DECLARE_RTR_BATCH(1)
CELES_DECLARE_RTR_BATCH(2)
CELES_DECLARE_RTR_BATCH(3)
CELES_DECLARE_RTR_BATCH(4)
CELES_DECLARE_RTR_BATCH(5)
#undef CELES_DECLARE_RTR_BATCH
}  // namespace celes

using celes::Pair2;
using celes::rtr::BatchSys;

namespace {

constexpr int kSegBlocks = 16;   // blocks per system in the segmented kernels
constexpr int kSegThreads = 256;
constexpr int kDotJ = 8;         // basis vectors per pass of the segmented dot

struct VecSeg {
  long long off;  // first complex element of the system in the flat vector
  int n;          // complex elements
  int active;
};

// ---- segmented vector kernels (grid: kSegBlocks x systems) ----------------

// partial[s][b][j] = sum over block b's share of system s of conj(V_j) w;
// per-thread and warp sums in the vector's own precision (at most a few dozen
// terms each: the FP64 pipe runs at 1/64 of the FP32 rate on this part), block
// sums in FP64
template <typename R>
__global__ void seg_dotc_kernel(const VecSeg* __restrict__ seg, int nv, const Pair2<R>* __restrict__ V,
                                long long ldv, const Pair2<R>* __restrict__ w, double* __restrict__ partial) {
  const int s = blockIdx.y;
  const VecSeg S = seg[s];
  __shared__ double red[2 * kDotJ][kSegThreads / 32];
  for (int j0 = 0; j0 < nv; j0 += kDotJ) {
    const int nj = nv - j0 < kDotJ ? nv - j0 : kDotJ;
    R sr[kDotJ], si[kDotJ];
#pragma unroll
    for (int q = 0; q < kDotJ; ++q) sr[q] = si[q] = static_cast<R>(0);
    if (S.active) {
      for (int t = blockIdx.x * kSegThreads + threadIdx.x; t < S.n; t += kSegBlocks * kSegThreads) {
        const Pair2<R> b = w[S.off + t];
#pragma unroll
        for (int q = 0; q < kDotJ; ++q) {
          if (q < nj) {
            const Pair2<R> a = V[(j0 + q) * ldv + S.off + t];
            sr[q] = celes::fma_(a.re, b.re, celes::fma_(a.im, b.im, sr[q]));
            si[q] = celes::fma_(a.re, b.im, celes::fma_(-a.im, b.re, si[q]));
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kDotJ; ++q) {
      R a = sr[q], b = si[q];
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
      }
      if ((threadIdx.x & 31) == 0) {
        red[2 * q][threadIdx.x >> 5] = static_cast<double>(a);
        red[2 * q + 1][threadIdx.x >> 5] = static_cast<double>(b);
      }
    }
    __syncthreads();
    if (threadIdx.x < 2 * nj) {
      double acc = 0.0;
      for (int q = 0; q < kSegThreads / 32; ++q) acc += red[threadIdx.x][q];
      const int q = threadIdx.x >> 1;
      partial[(((long long)s * kSegBlocks + blockIdx.x) * nv + j0 + q) * 2 + (threadIdx.x & 1)] = acc;
    }
    __syncthreads();
  }
}

// out[s][j] = sum_b partial[s][b][j]   (fixed order)
__global__ void seg_dot_reduce_kernel(int nsys, int nv, const double* __restrict__ partial, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nsys * nv) return;
  const int s = t / nv, j = t % nv;
  double a = 0.0, b = 0.0;
  for (int q = 0; q < kSegBlocks; ++q) {
    a += partial[(((long long)s * kSegBlocks + q) * nv + j) * 2];
    b += partial[(((long long)s * kSegBlocks + q) * nv + j) * 2 + 1];
  }
  out[2 * t] = a;
  out[2 * t + 1] = b;
}

// w_s <- w_s - sum_j h[s][j] V_j,s      (h: [nsys][nv] complex128)
template <typename R>
__global__ void seg_axpy_kernel(const VecSeg* __restrict__ seg, int nv, const Pair2<R>* __restrict__ V, long long ldv,
                                const double* __restrict__ h, Pair2<R>* __restrict__ w) {
  const int s = blockIdx.y;
  const VecSeg S = seg[s];
  if (!S.active) return;
  const double* hs = h + (long long)s * nv * 2;
  constexpr int U = 8;  // basis vectors whose loads are issued before their FMAs
  for (int t = blockIdx.x * kSegThreads + threadIdx.x; t < S.n; t += kSegBlocks * kSegThreads) {
    R ar = w[S.off + t].re, ai = w[S.off + t].im;
    int j = 0;
    for (; j + U <= nv; j += U) {
      Pair2<R> v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = V[(j + u) * ldv + S.off + t];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const R hr = static_cast<R>(hs[2 * (j + u)]), hi = static_cast<R>(hs[2 * (j + u) + 1]);
        ar = celes::fma_(-hr, v[u].re, celes::fma_(hi, v[u].im, ar));
        ai = celes::fma_(-hr, v[u].im, celes::fma_(-hi, v[u].re, ai));
      }
    }
    for (; j < nv; ++j) {
      const Pair2<R> v = V[j * ldv + S.off + t];
      const R hr = static_cast<R>(hs[2 * j]), hi = static_cast<R>(hs[2 * j + 1]);
      ar = celes::fma_(-hr, v.re, celes::fma_(hi, v.im, ar));
      ai = celes::fma_(-hr, v.im, celes::fma_(-hi, v.re, ai));
    }
    w[S.off + t] = Pair2<R>{ar, ai};
  }
}

// dst_s = scale[s] * src_s
template <typename R>
__global__ void seg_scale_kernel(const VecSeg* __restrict__ seg, const double* __restrict__ scale,
                                 const Pair2<R>* __restrict__ src, Pair2<R>* __restrict__ dst) {
  const int s = blockIdx.y;
  const VecSeg S = seg[s];
  if (!S.active) return;
  const R a = static_cast<R>(scale[s]);
  for (int t = blockIdx.x * kSegThreads + threadIdx.x; t < S.n; t += kSegBlocks * kSegThreads) {
    const Pair2<R> v = src[S.off + t];
    dst[S.off + t] = Pair2<R>{a * v.re, a * v.im};
  }
}

// y_s = sum_{j < nv} c[s][j] V_j,s     (c: [nsys][m] complex128, zero-padded;
// only the first nv <= m columns are read).  A zero coefficient skips its basis
// vector: a system that stopped after k < nv steps never wrote V_k+1.. in its
// segment, and 0 * (stale memory) may be NaN.
template <typename R>
__global__ void seg_combine_kernel(const VecSeg* __restrict__ seg, int m, int nv, const Pair2<R>* __restrict__ V,
                                   long long ldv, const double* __restrict__ c, Pair2<R>* __restrict__ y) {
  const int s = blockIdx.y;
  const VecSeg S = seg[s];
  if (!S.active) return;
  const double* cs = c + (long long)s * m * 2;
  for (int t = blockIdx.x * kSegThreads + threadIdx.x; t < S.n; t += kSegBlocks * kSegThreads) {
    R ar = 0, ai = 0;
    for (int j = 0; j < nv; ++j) {
      const R cr = static_cast<R>(cs[2 * j]), ci = static_cast<R>(cs[2 * j + 1]);
      if (cr == R(0) && ci == R(0)) continue;
      const Pair2<R> v = V[j * ldv + S.off + t];
      ar = celes::fma_(cr, v.re, celes::fma_(-ci, v.im, ar));
      ai = celes::fma_(cr, v.im, celes::fma_(ci, v.re, ai));
    }
    y[S.off + t] = Pair2<R>{ar, ai};
  }
}

// epilogue of the batched operator: y = x - T (W x) from the chunk partials
// (grid: blocks x systems of one lmax group); ATOM: the one slice the
// coupling launch added into, zeroed again after it is read (each element by
// the thread that read it) for the next launch
template <typename R, bool ATOM>
__global__ void batch_epilogue_kernel(const BatchSys* __restrict__ sys) {
  const BatchSys S = sys[blockIdx.y];
  if (!S.active) return;
  const int L = S.L, NH = L * (L + 2);
  const long long total = (long long)S.N * NH;
  Pair2<R>* partial = static_cast<Pair2<R>*>(S.partial);
  const Pair2<R>* x = static_cast<const Pair2<R>*>(S.x);
  const Pair2<R>* tq = static_cast<const Pair2<R>*>(S.tq);
  Pair2<R>* y = static_cast<Pair2<R>*>(S.y);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / NH;
    const int r = static_cast<int>(t - i * NH);
    R pr = 0, pi = 0, mr = 0, mi = 0;
    for (int c = 0; c < (ATOM ? 1 : S.chunks); ++c) {
      Pair2<R>* pc = partial + ((long long)c * S.N + i) * (2 * NH);
      const Pair2<R> a = pc[r];
      const Pair2<R> b = pc[NH + r];
      pr += a.re;
      pi += a.im;
      mr += b.re;
      mi += b.im;
      if (ATOM) {
        pc[r] = Pair2<R>{0, 0};
        pc[NH + r] = Pair2<R>{0, 0};
      }
    }
    const Pair2<R> y1{static_cast<R>(0.5) * (pr + mr), static_cast<R>(0.5) * (pi + mi)};
    const Pair2<R> y2{static_cast<R>(0.5) * (pr - mr), static_cast<R>(0.5) * (pi - mi)};
    int l = 1;
    while ((l + 1) * (l + 1) - 1 <= r) ++l;  // degree l holds rows l^2 - 1 .. (l+1)^2 - 2
    const long long o1 = i * 2 * NH + r, o2 = o1 + NH;
    const Pair2<R> q1 = tq[(i * 2 + 0) * L + (l - 1)];
    const Pair2<R> q2 = tq[(i * 2 + 1) * L + (l - 1)];
    const Pair2<R> x1 = x[o1], x2 = x[o2];
    y[o1] = Pair2<R>{x1.re - (q1.re * y1.re - q1.im * y1.im), x1.im - (q1.re * y1.im + q1.im * y1.re)};
    y[o2] = Pair2<R>{x2.re - (q2.re * y2.re - q2.im * y2.im), x2.im - (q2.re * y2.im + q2.im * y2.re)};
  }
}

// flat y = a x + b y with x, y of possibly different precision
template <typename RX, typename RY>
__global__ void flat_axpby_kernel(long long n, double a, const Pair2<RX>* __restrict__ x, double b,
                                  Pair2<RY>* __restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const Pair2<RX> v = x[t];
    const double yr = b == 0.0 ? 0.0 : b * static_cast<double>(y[t].re);
    const double yi = b == 0.0 ? 0.0 : b * static_cast<double>(y[t].im);
    y[t] = Pair2<RY>{static_cast<RY>(a * static_cast<double>(v.re) + yr),
                     static_cast<RY>(a * static_cast<double>(v.im) + yi)};
  }
}

cudaError_t launch_rtr_batch(int L, int precision, const void* sys, int nsys, long long ntiles,
                             unsigned long long* counter, cudaStream_t st) {
  using namespace celes;
  switch (L) {
    case 1: return launch_rtr_batch_1(precision, sys, nsys, ntiles, counter, st);
    case 2: return launch_rtr_batch_2(precision, sys, nsys, ntiles, counter, st);
    case 3: return launch_rtr_batch_3(precision, sys, nsys, ntiles, counter, st);
    case 4: return launch_rtr_batch_4(precision, sys, nsys, ntiles, counter, st);
    case 5: return launch_rtr_batch_5(precision, sys, nsys, ntiles, counter, st);
    default: return cudaErrorInvalidValue;
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

struct Buf {
  void* p = nullptr;
  size_t n = 0;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() {
    if (p) cudaFree(p);
  }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    if (!bytes) return cudaSuccess;
    const cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct HostBuf {  // pinned host staging
  void* p = nullptr;
  size_t n = 0;
  HostBuf() = default;
  HostBuf(const HostBuf&) = delete;
  HostBuf& operator=(const HostBuf&) = delete;
  ~HostBuf() {
    if (p) cudaFreeHost(p);
  }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n && p) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
    const cudaError_t e = cudaMallocHost(&p, bytes);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct System {
  int e, r;      // ensemble (context index) and right-hand side
  int L, N, nmax;
  long long off;  // flat offset (complex elements)
  long long n;    // unknowns
  int chunks, chunk;                 // FP64 source chunks (one partial slice each)
  int chunks32, chunk32;             // FP32 source chunks (all added into one slice in L2)
  long long part_off32, part_off64;  // partial-sum offsets (bytes)
};

struct Group {
  int L;
  std::vector<int> members;      // system indices
  long long ntiles[2] = {0, 0};  // per precision (0: FP32, 1: FP64)
  std::vector<long long> tile0[2];
};

}  // namespace

struct celes_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<celes_ctx*> ctx;
  std::vector<celes::CtxView> view;
  std::vector<System> sys;
  std::vector<Group> groups;
  long long ntot = 0;
  int maxL = 0;
  // device state
  Buf part32, part64;        // coupling partial sums
  Buf desc[2];               // BatchSys per group, concatenated (FP32 / FP64)
  Buf vseg;                  // VecSeg per system
  Buf counters;              // one tile counter per group and precision
  Buf ta, b, r64, w64;       // flat FP64 vectors
  Buf V, w, z, x, rr;        // Krylov basis and work vectors (inner precision)
  Buf dotp, dots, coef;      // dot partials, dot results, coefficients
  HostBuf hdots;             // pinned dot results
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_kernels[2] = {0, 0};
  cudaStream_t side[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // branches of the lmax groups
  cudaEvent_t fork = nullptr, join[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  const void* graph_in[2] = {nullptr, nullptr};
  void* graph_out[2] = {nullptr, nullptr};
  std::vector<int> active;  // per system
  std::string err;
  ~celes_batch() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto& g : graph)
      if (g) cudaGraphExecDestroy(g);
    for (int q = 0; q < 5; ++q) {
      if (side[q]) cudaStreamDestroy(side[q]);
      if (join[q]) cudaEventDestroy(join[q]);
    }
    if (fork) cudaEventDestroy(fork);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

#define BK(expr, what)                        \
  do {                                        \
    const cudaError_t e_ = (expr);            \
    if (e_ != cudaSuccess) {                  \
      bt->err = std::string(what) + ": " + cudaGetErrorString(e_); \
      return CELES_ECUDA;                     \
    }                                         \
  } while (0)

inline unsigned flat_blocks(long long n) {
  const long long b = (n + 255) / 256;
  const long long cap = 16LL * celes::device_sms();
  return static_cast<unsigned>(b < cap ? (b > 0 ? b : 1) : cap);
}

// descriptors of the operator y = x - T W x for flat vectors in/out (device
// pointers of precision `prec`, 0 = FP64) and the current active flags
int upload_descriptors(celes_batch* bt, int prec, const void* in, void* out) {
  const size_t elem = prec == 0 ? 16 : 8;
  std::vector<BatchSys> d;
  d.reserve(bt->sys.size());
  for (const Group& g : bt->groups) {
    for (size_t q = 0; q < g.members.size(); ++q) {
      const System& S = bt->sys[g.members[q]];
      const celes::CtxView& v = bt->view[S.e];
      BatchSys b{};
      b.pos = static_cast<const celes::Pos4*>(v.pos);
      b.x = static_cast<const char*>(in) + S.off * elem;
      b.y = static_cast<char*>(out) + S.off * elem;
      b.partial = prec == 0 ? bt->part64.as<char>() + S.part_off64 : bt->part32.as<char>() + S.part_off32;
      b.tq = prec == 0 ? v.tq : v.tq32;
      b.k = v.k;
      b.tile0 = g.tile0[prec == 0 ? 1 : 0][q];
      b.N = S.N;
      b.L = S.L;
      b.chunk = prec == 0 ? S.chunk : S.chunk32;
      b.nrb = (S.N + rtr_rpb(S.L, prec == 0 ? CELES_FP64 : CELES_FP32) - 1) /
              rtr_rpb(S.L, prec == 0 ? CELES_FP64 : CELES_FP32);
      b.chunks = prec == 0 ? S.chunks : S.chunks32;
      b.active = bt->active[g.members[q]];
      d.push_back(b);
    }
  }
  // pageable sources: the copy is staged before cudaMemcpyAsync returns, so
  // the host vectors may go out of scope while the stream is still running
  const size_t bytes = d.size() * sizeof(BatchSys);
  BK(cudaMemcpyAsync(bt->desc[prec == 0 ? 1 : 0].p, d.data(), bytes, cudaMemcpyHostToDevice, bt->stream),
     "descriptors");
  std::vector<VecSeg> vs(bt->sys.size());
  for (size_t s = 0; s < bt->sys.size(); ++s)
    vs[s] = VecSeg{bt->sys[s].off, static_cast<int>(bt->sys[s].n), bt->active[s]};
  BK(cudaMemcpyAsync(bt->vseg.p, vs.data(), vs.size() * sizeof(VecSeg), cudaMemcpyHostToDevice, bt->stream),
     "segments");
  return CELES_OK;
}

// record the operator on the stream: the lmax groups' persistent launches on
// parallel branches (so one group's last wave overlaps the others' work),
// joined before the epilogues
int record_operator(celes_batch* bt, int prec) {
  const int p = prec == 0 ? 1 : 0;
  const BatchSys* base = bt->desc[p].as<BatchSys>();
  size_t off = 0;
  BK(cudaEventRecord(bt->fork, bt->stream), "fork");
  for (size_t gi = 0; gi < bt->groups.size(); ++gi) {
    const Group& g = bt->groups[gi];
    const cudaStream_t sg = gi == 0 ? bt->stream : bt->side[gi];
    if (gi > 0) BK(cudaStreamWaitEvent(sg, bt->fork, 0), "fork wait");
    unsigned long long* ctr = bt->counters.as<unsigned long long>() + 2 * gi + p;
    BK(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), sg), "counter");
    BK(launch_rtr_batch(g.L, prec == 0 ? CELES_FP64 : CELES_FP32, base + off, static_cast<int>(g.members.size()),
                        g.ntiles[p], ctr, sg),
       "batched coupling");
    if (gi > 0) {
      BK(cudaEventRecord(bt->join[gi], sg), "join");
      BK(cudaStreamWaitEvent(bt->stream, bt->join[gi], 0), "join wait");
    }
    off += g.members.size();
  }
  off = 0;
  for (const Group& g : bt->groups) {
    dim3 grid(64, static_cast<unsigned>(g.members.size()));
    if (prec == 0)
      batch_epilogue_kernel<double, false><<<grid, 256, 0, bt->stream>>>(base + off);
    else
      batch_epilogue_kernel<float, true><<<grid, 256, 0, bt->stream>>>(base + off);
    celes::note_launch();
    BK(cudaGetLastError(), "batched epilogue");
    off += g.members.size();
  }
  return CELES_OK;
}

// out = (I - T W) in for every active system, through the captured graph
int apply_operator(celes_batch* bt, int prec, const void* in, void* out) {
  const int p = prec == 0 ? 1 : 0;
  int s = upload_descriptors(bt, prec, in, out);
  if (s) return s;
  if (!bt->graph[p]) {
    // function attributes and occupancy are set up outside the capture
    for (const Group& g : bt->groups)
      BK(launch_rtr_batch(g.L, prec == 0 ? CELES_FP64 : CELES_FP32, nullptr, 0, 0, nullptr, bt->stream), "setup");
    cudaGraph_t g = nullptr;
    const int64_t before = celes::kernel_launch_count();
    BK(cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal), "capture");
    s = record_operator(bt, prec);
    bt->graph_kernels[p] = static_cast<int>(celes::kernel_launch_count() - before);
    celes::note_launch(-bt->graph_kernels[p]);  // counted per replay below
    cudaGraph_t got = nullptr;
    const cudaError_t e = cudaStreamEndCapture(bt->stream, &got);
    if (s) {
      if (got) cudaGraphDestroy(got);
      return s;
    }
    BK(e, "end capture");
    g = got;
    const cudaError_t ei = cudaGraphInstantiate(&bt->graph[p], g, 0);
    cudaGraphDestroy(g);
    BK(ei, "graph instantiate");
  }
  BK(cudaGraphLaunch(bt->graph[p], bt->stream), "graph launch");
  celes::note_launch(bt->graph_kernels[p]);
  return CELES_OK;
}

// h[s][0..nv) = V_j,s^H w_s for all systems (host copy in bt->hdots)
template <typename R>
int seg_dots(celes_batch* bt, const void* Vb, long long ldv, int nv, const void* w) {
  const int S = static_cast<int>(bt->sys.size());
  dim3 grid(kSegBlocks, S);
  seg_dotc_kernel<R><<<grid, kSegThreads, 0, bt->stream>>>(bt->vseg.as<VecSeg>(), nv, static_cast<const Pair2<R>*>(Vb),
                                                           ldv, static_cast<const Pair2<R>*>(w),
                                                           bt->dotp.as<double>());
  const int n = S * nv;
  seg_dot_reduce_kernel<<<(n + 127) / 128, 128, 0, bt->stream>>>(S, nv, bt->dotp.as<double>(), bt->dots.as<double>());
  celes::note_launch(2);
  BK(cudaGetLastError(), "dots");
  BK(cudaMemcpyAsync(bt->hdots.p, bt->dots.p, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, bt->stream), "d2h");
  BK(cudaStreamSynchronize(bt->stream), "sync");
  return CELES_OK;
}

int upload_coef(celes_batch* bt, const std::vector<std::complex<double>>& c) {
  BK(cudaMemcpyAsync(bt->coef.p, c.data(), c.size() * 16, cudaMemcpyHostToDevice, bt->stream), "h2d");
  return CELES_OK;
}
// per-system real scale factors, [nsys] doubles
int upload_scale(celes_batch* bt, const std::vector<double>& a) {
  BK(cudaMemcpyAsync(bt->coef.p, a.data(), a.size() * 8, cudaMemcpyHostToDevice, bt->stream), "h2d");
  return CELES_OK;
}

// Lockstep restarted GMRES on all systems with active flag set in `want`:
// solves (I - T W) u_s = r_s (flat r, precision R) from u = 0, accumulating
// into x (flat, zeroed by the caller).  tol[s] is relative to ||r_s||.
template <typename R>
int lockstep_gmres(celes_batch* bt, const void* r, void* x, const std::vector<int>& want,
                   const std::vector<double>& tol, int m, int max_it, std::vector<int>& its,
                   std::vector<double>& rel_est, int& nmv) {
  const int prec = sizeof(R) == 8 ? 0 : 1;
  const int S = static_cast<int>(bt->sys.size());
  const long long n = bt->ntot;
  const size_t vb = sizeof(R) * 2 * n;
  auto Vp = [&](int j) { return bt->V.as<char>() + vb * j; };
  dim3 sgrid(kSegBlocks, S);
  its.assign(S, 0);
  rel_est.assign(S, 0.0);
  // ||r_s||
  bt->active = want;
  int st = upload_descriptors(bt, prec, r, bt->w.p);
  if (st) return st;
  st = seg_dots<R>(bt, r, 0, 1, r);
  if (st) return st;
  std::vector<double> rnorm(S, 0.0), beta(S, 0.0);
  std::vector<int> live(S, 0);
  {
    const std::complex<double>* h = bt->hdots.as<std::complex<double>>();
    std::vector<double> sc(S, 0.0);
    for (int s = 0; s < S; ++s) {
      rnorm[s] = celes::norm_from_dot(h[s].real());
      if (!want[s]) continue;
      if (!std::isfinite(rnorm[s])) {
        bt->err = "batched GMRES: non-finite residual";
        return CELES_ENUMERIC;
      }
      if (rnorm[s] > 0.0) {
        live[s] = 1;
        beta[s] = rnorm[s];
        sc[s] = 1.0 / rnorm[s];
        rel_est[s] = 1.0;
      }
    }
    bt->active = live;
    st = upload_descriptors(bt, prec, r, bt->w.p);
    if (st) return st;
    st = upload_scale(bt, sc);
    if (st) return st;
    seg_scale_kernel<R><<<sgrid, kSegThreads, 0, bt->stream>>>(bt->vseg.as<VecSeg>(), bt->coef.as<double>(),
                                                                static_cast<const Pair2<R>*>(r),
                                                                reinterpret_cast<Pair2<R>*>(Vp(0)));
    celes::note_launch();
    BK(cudaGetLastError(), "v0");
  }
  std::vector<std::vector<std::complex<double>>> H(S), g(S), sn(S);
  std::vector<std::vector<double>> cs(S);
  std::vector<int> kk_s(S, 0);
  bool any = std::any_of(live.begin(), live.end(), [](int v) { return v != 0; });
  while (any) {
    std::vector<int> cycle = live;  // systems iterating in this cycle
    for (int s = 0; s < S; ++s) {
      if (!cycle[s]) continue;
      H[s].assign((size_t)(m + 1) * m, 0.0);
      g[s].assign(m + 1, 0.0);
      g[s][0] = beta[s];
      sn[s].assign(m, 0.0);
      cs[s].assign(m, 0.0);
      kk_s[s] = 0;
    }
    std::vector<int> run = cycle;
    for (int kk = 0; kk < m; ++kk) {
      bool anyrun = false;
      for (int s = 0; s < S; ++s) {
        if (run[s] && its[s] >= max_it) run[s] = 0;
        anyrun = anyrun || run[s];
      }
      if (!anyrun) break;
      bt->active = run;
      st = apply_operator(bt, prec, Vp(kk), bt->w.p);
      if (st) return st;
      ++nmv;
      std::vector<std::complex<double>> h1((size_t)S * (kk + 1)), h2((size_t)S * (kk + 1));
      for (int pass = 0; pass < 2; ++pass) {
        st = seg_dots<R>(bt, bt->V.p, n, kk + 1, bt->w.p);
        if (st) return st;
        std::vector<std::complex<double>>& hh = pass == 0 ? h1 : h2;
        std::copy(bt->hdots.as<std::complex<double>>(), bt->hdots.as<std::complex<double>>() + hh.size(), hh.begin());
        st = upload_coef(bt, hh);
        if (st) return st;
        seg_axpy_kernel<R><<<sgrid, kSegThreads, 0, bt->stream>>>(bt->vseg.as<VecSeg>(), kk + 1,
                                                                   static_cast<const Pair2<R>*>(bt->V.p), n,
                                                                   bt->coef.as<double>(),
                                                                   static_cast<Pair2<R>*>(bt->w.p));
        celes::note_launch();
        BK(cudaGetLastError(), "axpy");
      }
      st = seg_dots<R>(bt, bt->w.p, 0, 1, bt->w.p);
      if (st) return st;
      std::vector<double> hn(S, 0.0), inv(S, 0.0);
      for (int s = 0; s < S; ++s) {
        if (!run[s]) continue;
        hn[s] = celes::norm_from_dot(bt->hdots.as<std::complex<double>>()[s].real());
        if (!std::isfinite(hn[s])) {
          bt->err = "batched GMRES: non-finite Krylov vector";
          return CELES_ENUMERIC;
        }
        inv[s] = hn[s] > 0.0 ? 1.0 / hn[s] : 0.0;
      }
      {
        st = upload_scale(bt, inv);
        if (st) return st;
        seg_scale_kernel<R><<<sgrid, kSegThreads, 0, bt->stream>>>(bt->vseg.as<VecSeg>(), bt->coef.as<double>(),
                                                                    static_cast<const Pair2<R>*>(bt->w.p),
                                                                    reinterpret_cast<Pair2<R>*>(Vp(kk + 1)));
        celes::note_launch();
        BK(cudaGetLastError(), "normalise");
      }
      for (int s = 0; s < S; ++s) {
        if (!run[s]) continue;
        std::vector<std::complex<double>>& Hs = H[s];
        for (int j = 0; j <= kk; ++j) Hs[(size_t)j * m + kk] = h1[(size_t)s * (kk + 1) + j] + h2[(size_t)s * (kk + 1) + j];
        Hs[(size_t)(kk + 1) * m + kk] = hn[s];
        for (int j = 0; j < kk; ++j) {
          const std::complex<double> a = Hs[(size_t)j * m + kk], b = Hs[(size_t)(j + 1) * m + kk];
          Hs[(size_t)j * m + kk] = cs[s][j] * a + sn[s][j] * b;
          Hs[(size_t)(j + 1) * m + kk] = -std::conj(sn[s][j]) * a + cs[s][j] * b;
        }
        const std::complex<double> a = Hs[(size_t)kk * m + kk], b = Hs[(size_t)(kk + 1) * m + kk];
        if (std::abs(b) == 0.0) {
          cs[s][kk] = 1.0;
          sn[s][kk] = 0.0;
        } else if (std::abs(a) == 0.0) {
          cs[s][kk] = 0.0;
          sn[s][kk] = 1.0;
        } else {
          const double den = std::sqrt(std::norm(a) + std::norm(b));
          cs[s][kk] = std::abs(a) / den;
          sn[s][kk] = (a / std::abs(a)) * std::conj(b) / den;
        }
        Hs[(size_t)kk * m + kk] = cs[s][kk] * a + sn[s][kk] * b;
        Hs[(size_t)(kk + 1) * m + kk] = 0.0;
        g[s][kk + 1] = -std::conj(sn[s][kk]) * g[s][kk];
        g[s][kk] = cs[s][kk] * g[s][kk];
        ++its[s];
        kk_s[s] = kk + 1;
        rel_est[s] = std::abs(g[s][kk + 1]) / rnorm[s];
        if (std::abs(g[s][kk + 1]) <= tol[s] * rnorm[s] || hn[s] == 0.0) run[s] = 0;
      }
    }
    // u_s = V y_s for the systems of this cycle; x += u
    std::vector<std::complex<double>> coef((size_t)S * m, 0.0);
    for (int s = 0; s < S; ++s) {
      if (!cycle[s]) continue;
      const int k = kk_s[s];
      for (int i = k - 1; i >= 0; --i) {
        std::complex<double> acc = g[s][i];
        for (int j = i + 1; j < k; ++j) acc -= H[s][(size_t)i * m + j] * coef[(size_t)s * m + j];
        const std::complex<double> d = H[s][(size_t)i * m + i];
        if (std::abs(d) == 0.0) {
          bt->err = "batched GMRES: singular Hessenberg";
          return CELES_ENUMERIC;
        }
        coef[(size_t)s * m + i] = acc / d;
      }
    }
    bt->active = cycle;
    st = upload_descriptors(bt, prec, x, bt->w.p);
    if (st) return st;
    st = upload_coef(bt, coef);
    if (st) return st;
    int kmax = 0;
    for (int s = 0; s < S; ++s)
      if (cycle[s]) kmax = std::max(kmax, kk_s[s]);
    BK(cudaMemsetAsync(bt->z.p, 0, vb, bt->stream), "zero");
    seg_combine_kernel<R><<<sgrid, kSegThreads, 0, bt->stream>>>(bt->vseg.as<VecSeg>(), m, kmax,
                                                                  static_cast<const Pair2<R>*>(bt->V.p), n,
                                                                  bt->coef.as<double>(), static_cast<Pair2<R>*>(bt->z.p));
    flat_axpby_kernel<R, R><<<flat_blocks(n), 256, 0, bt->stream>>>(n, 1.0, static_cast<const Pair2<R>*>(bt->z.p), 1.0,
                                                                    static_cast<Pair2<R>*>(x));
    celes::note_launch(2);
    BK(cudaGetLastError(), "update");
    // systems that need another cycle: explicit residual w = r - (I - T W) x
    std::vector<int> again(S, 0);
    any = false;
    for (int s = 0; s < S; ++s) {
      if (!cycle[s]) continue;
      const bool conv = std::abs(g[s][kk_s[s]]) <= tol[s] * rnorm[s];
      if (!conv && its[s] < max_it) {
        again[s] = 1;
        any = true;
      }
    }
    if (!any) break;
    bt->active = again;
    st = apply_operator(bt, prec, x, bt->w.p);
    if (st) return st;
    ++nmv;
    flat_axpby_kernel<R, R><<<flat_blocks(n), 256, 0, bt->stream>>>(n, 1.0, static_cast<const Pair2<R>*>(r), -1.0,
                                                                    static_cast<Pair2<R>*>(bt->w.p));
    celes::note_launch();
    BK(cudaGetLastError(), "residual");
    st = seg_dots<R>(bt, bt->w.p, 0, 1, bt->w.p);
    if (st) return st;
    std::vector<double> packed((size_t)S, 0.0);
    live.assign(S, 0);
    any = false;
    for (int s = 0; s < S; ++s) {
      if (!again[s]) continue;
      beta[s] = celes::norm_from_dot(bt->hdots.as<std::complex<double>>()[s].real());
      if (!std::isfinite(beta[s])) {
        bt->err = "batched GMRES: non-finite residual";
        return CELES_ENUMERIC;
      }
      rel_est[s] = beta[s] / rnorm[s];
      if (beta[s] <= tol[s] * rnorm[s] || !(beta[s] > 0.0)) continue;
      live[s] = 1;
      any = true;
      packed[s] = 1.0 / beta[s];
    }
    if (!any) break;
    bt->active = live;
    st = upload_descriptors(bt, prec, x, bt->w.p);
    if (st) return st;
    st = upload_scale(bt, packed);
    if (st) return st;
    seg_scale_kernel<R><<<sgrid, kSegThreads, 0, bt->stream>>>(bt->vseg.as<VecSeg>(), bt->coef.as<double>(),
                                                                static_cast<const Pair2<R>*>(bt->w.p),
                                                                reinterpret_cast<Pair2<R>*>(Vp(0)));
    celes::note_launch();
    BK(cudaGetLastError(), "v0");
  }
  return CELES_OK;
}

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  EventPair(const EventPair&) = delete;
  EventPair& operator=(const EventPair&) = delete;
};

int batch_set_error(celes_batch* bt, int code, const char* msg) {
  if (bt) bt->err = msg;
  return code;
}

}  // namespace

extern "C" int celes_batch_create(celes_batch** out, celes_ctx* const* ctxs, int count, int restart) {
  celes::NvtxRange nvtx_range_("celes_batch_create");
  if (!out) return CELES_EINVAL;
  *out = nullptr;
  if (!ctxs || count < 1) return CELES_EINVAL;
  std::unique_ptr<celes_batch> bt(new celes_batch());
  const int m = restart > 0 ? restart : 30;
  for (int e = 0; e < count; ++e) {
    celes::CtxView v{};
    if (!ctxs[e] || celes::ctx_view(ctxs[e], &v) != CELES_OK) return CELES_ESTATE;  // no incident field yet
    if (e == 0) bt->device = v.device;
    if (v.device != bt->device) return CELES_EINVAL;
    bt->ctx.push_back(ctxs[e]);
    bt->view.push_back(v);
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(bt->device) != cudaSuccess) return CELES_ECUDA;
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  celes_batch* b = bt.get();
  // systems, flat offsets, chunking, partial offsets
  long long off = 0, p32 = 0, p64 = 0;
  for (int e = 0; e < count; ++e) {
    const celes::CtxView& v = bt->view[e];
    for (int r = 0; r < v.nrhs; ++r) {
      System S{};
      S.e = e;
      S.r = r;
      S.L = v.L;
      S.N = static_cast<int>(v.N);
      S.nmax = v.nmax;
      S.off = off;
      S.n = v.N * v.nmax;
      S.part_off32 = 0;
      S.part_off64 = 0;
      off += S.n;
      bt->maxL = std::max(bt->maxL, S.L);
      bt->sys.push_back(S);
    }
  }
  // source chunk length per lmax group: about eight waves of tiles over the
  // group's work (FP32 launch shape), between 32 and 512 sources, so that
  // groups of a few large-lmax ensembles do not run in less than one wave
  for (int L = 1; L <= 5; ++L) {
    double work = 0.0;  // ordered pairs x RHS of the group
    for (const System& Sy : bt->sys)
      if (Sy.L == L) work += static_cast<double>(Sy.N) * Sy.N;
    if (work == 0.0) continue;
    const int rpb = rtr_rpb(L, CELES_FP32);
    const double slots = static_cast<double>(celes::coupling_rtr_slots(L, CELES_FP32));
    const double want = work / (8.0 * std::max(1.0, slots) * rpb);
    int chunk = static_cast<int>(std::ceil(want / 32.0)) * 32;
    chunk = std::max(32, std::min(512, chunk));
    // FP32: chunks cost no partial-sum traffic (one slice per system), so
    // each system gets about two waves of tiles of its own, which keeps the
    // GPU busy once only a few systems remain active
    const int nrb_den = rpb > 0 ? rpb : 1;
    for (System& Sy : bt->sys)
      if (Sy.L == L) {
        Sy.chunk = std::min(Sy.N, chunk);
        Sy.chunks = (Sy.N + Sy.chunk - 1) / Sy.chunk;
        const int nrb = (Sy.N + nrb_den - 1) / nrb_den;
        const double ch32 = std::ceil(2.0 * std::max(1.0, slots) / nrb);
        int c32 = static_cast<int>(std::ceil(Sy.N / ch32 / 32.0)) * 32;
        c32 = std::max(64, std::min(chunk, c32));
        Sy.chunk32 = std::min(Sy.N, c32);
        Sy.chunks32 = (Sy.N + Sy.chunk32 - 1) / Sy.chunk32;
      }
  }
  for (System& Sy : bt->sys) {
    Sy.part_off32 = p32;
    Sy.part_off64 = p64;
    p32 += (long long)Sy.n * 8;
    p64 += (long long)Sy.chunks * Sy.n * 16;
  }
  bt->ntot = off;
  for (int L = 1; L <= 5; ++L) {
    Group g;
    g.L = L;
    for (size_t s = 0; s < bt->sys.size(); ++s) {
      if (bt->sys[s].L != L) continue;
      g.members.push_back(static_cast<int>(s));
      for (int p = 0; p < 2; ++p) {
        const int rpb = rtr_rpb(L, p == 0 ? CELES_FP32 : CELES_FP64);
        g.tile0[p].push_back(g.ntiles[p]);
        g.ntiles[p] += (long long)((bt->sys[s].N + rpb - 1) / rpb) * (p == 0 ? bt->sys[s].chunks32 : bt->sys[s].chunks);
      }
    }
    if (!g.members.empty()) bt->groups.push_back(std::move(g));
  }
  const size_t S = bt->sys.size();
  bt->active.assign(S, 1);
  auto ok = [&](cudaError_t e) { return e == cudaSuccess; };
  if (!ok(cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming))) return CELES_ECUDA;
  for (size_t gi = 1; gi < bt->groups.size(); ++gi)
    if (!ok(cudaStreamCreateWithFlags(&bt->side[gi], cudaStreamNonBlocking)) ||
        !ok(cudaEventCreateWithFlags(&bt->join[gi], cudaEventDisableTiming)))
      return CELES_ECUDA;
  if (!ok(cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking)) || !ok(bt->part32.ensure(p32)) ||
      !ok(bt->part64.ensure(p64)) || !ok(bt->desc[0].ensure(S * sizeof(BatchSys))) ||
      !ok(bt->desc[1].ensure(S * sizeof(BatchSys))) || !ok(bt->vseg.ensure(S * sizeof(VecSeg))) ||
      !ok(bt->counters.ensure(2 * bt->groups.size() * sizeof(unsigned long long))) ||
      !ok(bt->ta.ensure(off * 16)) || !ok(bt->b.ensure(off * 16)) || !ok(bt->r64.ensure(off * 16)) ||
      !ok(bt->w64.ensure(off * 16)) || !ok(bt->dotp.ensure(S * kSegBlocks * (m + 2) * 16)) ||
      !ok(bt->dots.ensure(S * (m + 2) * 16)) || !ok(bt->coef.ensure(S * (m + 2) * 16)) ||
      !ok(bt->hdots.ensure(S * (m + 2) * 16))) {
    return CELES_ENOMEM;
  }
  // the FP32 partial slices start at zero; each batched epilogue leaves them so
  if (p32 > 0 && !ok(cudaMemsetAsync(bt->part32.p, 0, static_cast<size_t>(p32), bt->stream))) return CELES_ECUDA;
  // T a of every system into the flat vector
  for (const System& Sy : bt->sys) {
    const celes::CtxView& v = bt->view[Sy.e];
    if (cudaMemcpyAsync(bt->ta.as<char>() + Sy.off * 16, v.rhs + (size_t)Sy.r * Sy.n * 2, Sy.n * 16,
                        cudaMemcpyDeviceToDevice, bt->stream) != cudaSuccess)
      return batch_set_error(b, CELES_ECUDA, "copy T a");
  }
  if (cudaStreamSynchronize(bt->stream) != cudaSuccess) return CELES_ECUDA;
  (void)m;
  *out = bt.release();
  return CELES_OK;
}

extern "C" void celes_batch_destroy(celes_batch* bt) {
  if (!bt) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(bt->device);
  delete bt;  // the destructor releases graphs, streams and events
  cudaSetDevice(prev);
}

extern "C" int celes_batch_num_systems(const celes_batch* bt) {
  return bt ? static_cast<int>(bt->sys.size()) : CELES_EINVAL;
}

extern "C" long long celes_batch_num_unknowns(const celes_batch* bt) { return bt ? bt->ntot : CELES_EINVAL; }

extern "C" int celes_batch_master_matvec(celes_batch* bt, const void* x, void* y, int precision) {
  if (!bt || !x || !y || (precision != CELES_FP64 && precision != CELES_FP32)) return CELES_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(bt->device);
  bt->active.assign(bt->sys.size(), 1);
  int s = apply_operator(bt, precision == CELES_FP64 ? 0 : 1, x, y);
  if (!s && cudaStreamSynchronize(bt->stream) != cudaSuccess) s = CELES_ECUDA;
  cudaSetDevice(prev);
  return s;
}

extern "C" int celes_batch_solve(celes_batch* bt, double tol, const celes_solve_opts* opts, celes_solve_info* infos) {
  celes::NvtxRange nvtx_range_("celes_batch_solve");
  if (!bt || !(tol > 0.0)) return CELES_EINVAL;
  celes_solve_opts o{};
  o.mode = CELES_SOLVE_MIXED;
  o.restart = 30;
  o.max_iter = 2000;
  o.max_outer = 8;
  o.inner_tol = 1e-5;
  if (opts) o = *opts;
  if (o.restart <= 0) o.restart = 30;
  if (o.max_iter <= 0) o.max_iter = 2000;
  if (o.max_outer <= 0) o.max_outer = 8;
  // the batch starts every system from T a and applies no preconditioner
  if (o.x0 != CELES_X0_TA) return batch_set_error(bt, CELES_EINVAL, "batch solve: x0 = T a only");
  if (o.solver != CELES_SOLVER_GMRES) return batch_set_error(bt, CELES_EINVAL, "batch solve: GMRES only");
  const int m = o.restart;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(bt->device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  const int S = static_cast<int>(bt->sys.size());
  const long long n = bt->ntot;
  const bool mixed = o.mode == CELES_SOLVE_MIXED;
  const size_t elem = mixed ? 8 : 16;
  if (bt->V.ensure(elem * n * (m + 1)) != cudaSuccess || bt->w.ensure(elem * n) != cudaSuccess ||
      bt->z.ensure(elem * n) != cudaSuccess || bt->x.ensure(elem * n) != cudaSuccess ||
      bt->rr.ensure(elem * n) != cudaSuccess || bt->dotp.ensure((size_t)S * kSegBlocks * (m + 2) * 16) != cudaSuccess ||
      bt->dots.ensure((size_t)S * (m + 2) * 16) != cudaSuccess || bt->coef.ensure((size_t)S * (m + 2) * 16) != cudaSuccess ||
      bt->hdots.ensure((size_t)S * (m + 2) * 16) != cudaSuccess)
    return batch_set_error(bt, CELES_ENOMEM, "batch solve: device memory");
  EventPair ev;  // solve time; released on every return path
  const cudaEvent_t t0 = ev.a, t1 = ev.b;
  cudaEventRecord(t0, bt->stream);
  // b = T a
  if (cudaMemcpyAsync(bt->b.p, bt->ta.p, n * 16, cudaMemcpyDeviceToDevice, bt->stream) != cudaSuccess)
    return CELES_ECUDA;
  std::vector<int> iters(S, 0), outer(S, 0), done(S, 0);
  std::vector<double> rel(S, 1.0), tanorm(S, 0.0);
  int nmv64 = 0, nmv32 = 0;
  // ||T a_s||
  bt->active.assign(S, 1);
  int st = upload_descriptors(bt, 0, bt->b.p, bt->w64.p);
  if (st) return st;
  st = seg_dots<double>(bt, bt->ta.p, 0, 1, bt->ta.p);
  if (st) return st;
  for (int s = 0; s < S; ++s) {
    tanorm[s] = celes::norm_from_dot(bt->hdots.as<std::complex<double>>()[s].real());
    if (!std::isfinite(tanorm[s])) return batch_set_error(bt, CELES_ENUMERIC, "batch solve: non-finite T a");
  }
  for (int it = 0; it <= o.max_outer; ++it) {
    // r = T a - (I - T W) b in FP64 for the systems not yet done
    std::vector<int> act(S, 0);
    for (int s = 0; s < S; ++s) act[s] = !done[s];
    bt->active = act;
    st = apply_operator(bt, 0, bt->b.p, bt->w64.p);
    if (st) return st;
    ++nmv64;
    flat_axpby_kernel<double, double><<<flat_blocks(n), 256, 0, bt->stream>>>(
        n, 1.0, static_cast<const Pair2<double>*>(bt->ta.p), -1.0, static_cast<Pair2<double>*>(bt->w64.p));
    celes::note_launch();
    st = seg_dots<double>(bt, bt->w64.p, 0, 1, bt->w64.p);
    if (st) return st;
    bool all = true;
    for (int s = 0; s < S; ++s) {
      if (done[s]) continue;
      const double rn = celes::norm_from_dot(bt->hdots.as<std::complex<double>>()[s].real());
      rel[s] = tanorm[s] > 0.0 ? rn / tanorm[s] : 0.0;
      if (!std::isfinite(rel[s])) return batch_set_error(bt, CELES_ENUMERIC, "batch solve: non-finite residual");
      if (rel[s] <= tol || iters[s] >= o.max_iter) done[s] = 1;
      else all = false;
    }
    if (all || it == o.max_outer) break;
    std::vector<int> want(S, 0);
    std::vector<double> itol(S, 0.0);
    for (int s = 0; s < S; ++s) {
      if (done[s]) continue;
      want[s] = 1;
      ++outer[s];
      itol[s] = mixed ? std::max(o.inner_tol, 0.3 * tol / rel[s]) : 0.9 * tol / rel[s];
      itol[s] = std::min(itol[s], 0.5);
    }
    std::vector<int> its;
    std::vector<double> est;
    if (mixed) {
      flat_axpby_kernel<double, float><<<flat_blocks(n), 256, 0, bt->stream>>>(
          n, 1.0, static_cast<const Pair2<double>*>(bt->w64.p), 0.0, static_cast<Pair2<float>*>(bt->rr.p));
      celes::note_launch();
      if (cudaMemsetAsync(bt->x.p, 0, elem * n, bt->stream) != cudaSuccess) return CELES_ECUDA;
      int budget = o.max_iter;
      for (int s = 0; s < S; ++s)
        if (want[s]) budget = std::min(budget, o.max_iter - iters[s]);
      st = lockstep_gmres<float>(bt, bt->rr.p, bt->x.p, want, itol, m, std::max(1, budget), its, est, nmv32);
      if (st) return st;
      flat_axpby_kernel<float, double><<<flat_blocks(n), 256, 0, bt->stream>>>(
          n, 1.0, static_cast<const Pair2<float>*>(bt->x.p), 1.0, static_cast<Pair2<double>*>(bt->b.p));
      celes::note_launch();
    } else {
      if (cudaMemcpyAsync(bt->rr.p, bt->w64.p, elem * n, cudaMemcpyDeviceToDevice, bt->stream) != cudaSuccess ||
          cudaMemsetAsync(bt->x.p, 0, elem * n, bt->stream) != cudaSuccess)
        return CELES_ECUDA;
      int budget = o.max_iter;
      for (int s = 0; s < S; ++s)
        if (want[s]) budget = std::min(budget, o.max_iter - iters[s]);
      st = lockstep_gmres<double>(bt, bt->rr.p, bt->x.p, want, itol, m, std::max(1, budget), its, est, nmv64);
      if (st) return st;
      flat_axpby_kernel<double, double><<<flat_blocks(n), 256, 0, bt->stream>>>(
          n, 1.0, static_cast<const Pair2<double>*>(bt->x.p), 1.0, static_cast<Pair2<double>*>(bt->b.p));
      celes::note_launch();
    }
    for (int s = 0; s < S; ++s) iters[s] += its[s];
  }
  cudaEventRecord(t1, bt->stream);
  // scatter b into the contexts
  for (const System& Sy : bt->sys) {
    const celes::CtxView& v = bt->view[Sy.e];
    if (cudaMemcpyAsync(const_cast<double*>(v.b) + (size_t)Sy.r * Sy.n * 2, bt->b.as<char>() + Sy.off * 16, Sy.n * 16,
                        cudaMemcpyDeviceToDevice, bt->stream) != cudaSuccess)
      return CELES_ECUDA;
  }
  if (cudaStreamSynchronize(bt->stream) != cudaSuccess) return CELES_ECUDA;
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, t0, t1);
  for (celes_ctx* c : bt->ctx) celes::ctx_mark_solved(c);
  bool all_ok = true;
  for (int s = 0; s < S; ++s) all_ok = all_ok && rel[s] <= tol;
  if (infos) {
    for (size_t e = 0; e < bt->ctx.size(); ++e) {
      celes_solve_info inf{};
      inf.history = infos[e].history;  // no residual history in batch mode
      inf.history_cap = infos[e].history_cap;
      inf.status = CELES_OK;
      for (int s = 0; s < S; ++s) {
        if (bt->sys[s].e != static_cast<int>(e)) continue;
        inf.iterations = std::max(inf.iterations, iters[s]);
        inf.outer = std::max(inf.outer, outer[s]);
        inf.residual = std::max(inf.residual, rel[s]);
        if (rel[s] > tol) inf.status = CELES_ENOCONV;
      }
      inf.matvecs_fp64 = nmv64;
      inf.matvecs_fp32 = nmv32;
      inf.seconds = ms * 1e-3;
      infos[e] = inf;
    }
  }
  return all_ok ? CELES_OK : CELES_ENOCONV;
}

extern "C" const char* celes_batch_last_error(const celes_batch* bt) { return bt ? bt->err.c_str() : "null batch"; }
