// Host launchers of the coupling kernel for one degree L (instantiated once
// per translation unit coupling_L<L>.cu so that the large unrolled kernels
// compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "coupling_kernel.cuh"

namespace celes {

template <int L, typename R>
cudaError_t launch_coupling_partial_t(int64_t N, const void* pos, const void* x, void* partial, double k, int chunks,
                                      cudaStream_t st) {
  using C = CouplingConfig<L, R>;
  using LY = CouplingLayout<L, R>;
  const size_t smem = LY::bytes;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(coupling_partial_kernel<L, R>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (N <= 0) return cudaSuccess;
  if (chunks < 1) chunks = 1;
  const int64_t chunk = (N + chunks - 1) / chunks;
  dim3 grid(static_cast<unsigned>((N + LY::RPB - 1) / LY::RPB), static_cast<unsigned>(chunks));
  coupling_partial_kernel<L, R><<<grid, C::BLOCK, smem, st>>>(
      static_cast<int>(N), static_cast<const Pos4*>(pos), static_cast<const Pair2<R>*>(x),
      static_cast<Pair2<R>*>(partial), k, static_cast<int>(chunk));
  return cudaGetLastError();
}

template <int L>
int coupling_terms_export_t(int* idx, double* val, int cap) {
  constexpr int NH = L * (L + 2);
  int t = 0;
  for (int ri = 0; ri < NH; ++ri) {
    const tab::RowTerms<L> T = tab::make_row_terms<L>(ri);
    for (int ro = 0; ro < NH; ++ro) {
      for (int q = T.off[ro]; q < T.off[ro + 1]; ++q) {
        if (idx && val && t < cap) {
          const int s = T.s[q];
          int p = 0;
          while ((p + 1) * (p + 2) / 2 <= s) ++p;
          idx[5 * t + 0] = ri;
          idx[5 * t + 1] = ro;
          idx[5 * t + 2] = p;
          idx[5 * t + 3] = s - p * (p + 1) / 2;
          idx[5 * t + 4] = T.kind[q];
          val[t] = T.c[q];
        }
        ++t;
      }
    }
  }
  return t;
}

// FP64 coupling with runtime term tables (generic.cu)
cudaError_t launch_generic_coupling_fp64(int L, int64_t N, const void* pos, const void* x, void* partial, double k,
                                         int chunks, cudaStream_t st);
constexpr int kGenericRPB = 64;

// FP64_UNROLLED: 1 = compile-time FP64 kernel, 0 = runtime-table FP64 kernel
#define CELES_INSTANTIATE_COUPLING(LL, FP64_UNROLLED)                                                       \
  cudaError_t launch_coupling_partial_##LL(int precision, int64_t N, const void* pos, const void* x,       \
                                            void* partial, double k, int chunks, cudaStream_t st) {        \
    if (precision == 0) {                                                                                  \
      if constexpr (FP64_UNROLLED)                                                                         \
        return launch_coupling_partial_t<LL, double>(N, pos, x, partial, k, chunks, st);                   \
      else                                                                                                 \
        return launch_generic_coupling_fp64(LL, N, pos, x, partial, k, chunks, st);                        \
    }                                                                                                      \
    return launch_coupling_partial_t<LL, float>(N, pos, x, partial, k, chunks, st);                        \
  }                                                                                                        \
  int coupling_rpb_##LL(int precision) {                                                                   \
    if (precision == 0) return (FP64_UNROLLED) ? CouplingLayout<LL, double>::RPB : kGenericRPB;           \
    return CouplingLayout<LL, float>::RPB;                                                                 \
  }                                                                                                        \
  int coupling_terms_export_##LL(int* idx, double* val, int cap) {                                         \
    return coupling_terms_export_t<LL>(idx, val, cap);                                                     \
  }

}  // namespace celes
