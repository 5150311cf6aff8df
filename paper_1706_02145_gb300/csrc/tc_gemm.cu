// Tensor-core GEMM for the graph-network layers: C = alpha * A B^T + beta * C
// with A [M][K] and B [N][K] in BF16 (row-major, K contiguous), C [M][N] in FP32.
//
// sm_103a tcgen05 path:
//  * one CTA of 128 threads computes a 128 x BN tile of C;
//  * each K step of 64 stages the A (128 x 64) and B (BN x 64) tiles in shared
//    memory in the canonical no-swizzle K-major layout (8-row x 16-byte core
//    matrices, core matrix (g, c) of a tile at byte (g * 8 + c) * 128);
//  * one elected thread issues tcgen05.mma.kind::f16 (M = 128, N = BN, K = 16
//    per instruction, BF16 inputs, FP32 accumulation in tensor memory) and
//    commits to an mbarrier; the CTA waits on it (bounded) before reusing the
//    tiles;
//  * the epilogue reads the accumulator with tcgen05.ld (warp w owns rows
//    32w..32w+31) and applies alpha/beta.
// Every wait is bounded: a wait that runs out sets *err and the kernel skips
// the remaining work.  Before it frees its tensor memory it waits once more
// (bounded) for the commit of the step it gave up on, so that no MMA it issued
// is still writing the accumulator when the columns are released.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "../../include/celes.h"
#include "kernels.h"

namespace celes {
namespace tc {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kThreads = 128;
constexpr unsigned kSpinLimit = 1u << 26;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor (no swizzle, K-major canonical layout)
//  bits  0-13 start address >> 4
//  bits 16-29 leading-dimension byte offset >> 4 (between core matrices along K)
//  bits 32-45 stride-dimension byte offset >> 4 (between 8-row groups)
//  bits 46-47 descriptor version (1)
//  bits 61-63 layout (0: no swizzle)
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// instruction descriptor of tcgen05.mma.kind::f16: D = F32 (bits 4-5 = 1),
// A = BF16 (bits 7-9 = 1), B = BF16 (bits 10-12 = 1), both K-major
// (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// bounded wait on the given phase parity; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  for (unsigned it = 0; it < kSpinLimit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int BN>
__global__ void __launch_bounds__(kThreads) gemm_bf16_tn_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                               int lda, const __nv_bfloat16* __restrict__ B, int ldb,
                                                               float* __restrict__ C, int ldc, float alpha, float beta,
                                                               int* __restrict__ err) {
  __shared__ __align__(1024) unsigned char sA[kBM * kBK * 2];
  __shared__ __align__(1024) unsigned char sB[BN * kBK * 2];
  __shared__ __align__(8) uint64_t bar;
  __shared__ unsigned tmem_base_s;
  __shared__ int abort_s;
  __shared__ unsigned abort_phase_s;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int m0 = blockIdx.y * kBM;
  const int n0 = blockIdx.x * BN;

  if (tid == 0) {
    mbar_init(&bar, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base_s;

  const int ksteps = (K + kBK - 1) / kBK;
  unsigned phase = 0;
  for (int ks = 0; ks < ksteps; ++ks) {
    const int k0 = ks * kBK;
    // stage A: 128 rows x 8 chunks of 8 bf16 (16 bytes)
    for (int q = tid; q < kBM * (kBK / 8); q += kThreads) {
      const int r = q >> 3, c = q & 7;
      const int gr = m0 + r, gk = k0 + c * 8;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (gr < M && gk < K) v = *reinterpret_cast<const uint4*>(A + (size_t)gr * lda + gk);
      const int off = (((r >> 3) * 8 + c) * 128) + (r & 7) * 16;
      *reinterpret_cast<uint4*>(sA + off) = v;
    }
    for (int q = tid; q < BN * (kBK / 8); q += kThreads) {
      const int r = q >> 3, c = q & 7;
      const int gr = n0 + r, gk = k0 + c * 8;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (gr < N && gk < K) v = *reinterpret_cast<const uint4*>(B + (size_t)gr * ldb + gk);
      const int off = (((r >> 3) * 8 + c) * 128) + (r & 7) * 16;
      *reinterpret_cast<uint4*>(sB + off) = v;
    }
    // make the generic-proxy writes visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const unsigned a0 = smem_u32(sA), b0 = smem_u32(sB);
      constexpr uint32_t idesc = idesc_bf16_f32(kBM, BN);
#pragma unroll
      for (int s = 0; s < kBK / 16; ++s) {
        // K = 16 bf16 = two core matrices along K: advance 2 * 128 bytes
        const uint64_t da = smem_desc(a0 + s * 256, 128, 1024);
        const uint64_t db = smem_desc(b0 + s * 256, 128, 1024);
        const unsigned acc = (ks > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar))
                   : "memory");
    }
    // all threads wait until the MMAs have read the tiles
    if (!mbar_wait(&bar, phase)) {
      if (tid == 0) atomicExch(err, 1);
      abort_s = 1;
      abort_phase_s = phase;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_s) break;
  }

  if (!abort_s) {
    // epilogue: warp w reads tensor-memory lanes 32w..32w+31 (rows), 16 columns at a time
    const int row = m0 + warp * 32 + (tid & 31);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      unsigned v[16];
      const unsigned taddr = tmem + (static_cast<unsigned>(warp * 32) << 16) + c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col < N) {
            float* cp = C + (size_t)row * ldc + col;
            const float r = alpha * __uint_as_float(v[j]);
            *cp = beta == 0.0f ? r : fmaf(beta, *cp, r);
          }
        }
      }
    }
  }
  if (abort_s && tid == 0) {
    // the commit of the abandoned step may still be outstanding: drain it
    // (bounded) before the tensor memory is released
    (void)mbar_wait(&bar, abort_phase_s);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

}  // namespace tc

cudaError_t launch_gemm_bf16_tn(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C, int ldc,
                                float alpha, float beta, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  if (K % 8 || lda % 8 || ldb % 8 || (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
    return cudaErrorInvalidValue;
  const int BN = N <= 64 ? 64 : 128;
  dim3 grid((N + BN - 1) / BN, (M + tc::kBM - 1) / tc::kBM);
  if (BN == 64)
    tc::gemm_bf16_tn_kernel<64><<<grid, tc::kThreads, 0, st>>>(M, N, K, static_cast<const __nv_bfloat16*>(A), lda,
                                                               static_cast<const __nv_bfloat16*>(B), ldb, C, ldc,
                                                               alpha, beta, err);
  else
    tc::gemm_bf16_tn_kernel<128><<<grid, tc::kThreads, 0, st>>>(M, N, K, static_cast<const __nv_bfloat16*>(A), lda,
                                                                static_cast<const __nv_bfloat16*>(B), ldb, C, ldc,
                                                                alpha, beta, err);
  note_launch();
  return cudaGetLastError();
}

}  // namespace celes

namespace {
// One error flag per call: concurrent calls (from several host threads) take
// different slots of this ring, so one call's timeout is not read by another.
constexpr int kErrSlots = 256;
__device__ int g_gemm_err[kErrSlots];
std::atomic<unsigned> g_gemm_err_next{0};
}  // namespace

extern "C" int celes_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C, int ldc,
                               float alpha, float beta, void* stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C || ldc < N) return CELES_EINVAL;
  if (K % 8 || lda % 8 || ldb % 8 || lda < K || ldb < K || (reinterpret_cast<uintptr_t>(A) & 15) ||
      (reinterpret_cast<uintptr_t>(B) & 15))
    return CELES_EINVAL;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* errs = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void**>(&errs), g_gemm_err) != cudaSuccess) return CELES_ECUDA;
  int* err = errs + (g_gemm_err_next.fetch_add(1, std::memory_order_relaxed) % kErrSlots);
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return CELES_ECUDA;
  if (celes::launch_gemm_bf16_tn(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, err, st) != cudaSuccess)
    return CELES_ECUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CELES_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CELES_ECUDA;
  return h ? CELES_ETIMEOUT : CELES_OK;
}
