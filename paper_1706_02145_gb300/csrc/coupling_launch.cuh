// Host launchers of the coupling kernel for one degree L (instantiated once
// per translation unit coupling_L<L>.cu so that the large unrolled kernels
// compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "coupling_kernel.cuh"
#include "rtr_kernel.cuh"
#include "kernels.h"

namespace celes {

template <int L, typename R>
cudaError_t launch_coupling_partial_t(int64_t N, const void* pos, const void* x, void* partial, double k, int chunks,
                                      cudaStream_t st) {
  using C = CouplingConfig<L, R>;
  using LY = CouplingLayout<L, R>;
  const size_t smem = LY::bytes;
  // the shared-memory opt-in, once on each device
  static PerDevice attr;
  cudaError_t se = cudaSuccess;
  if (attr.get(current_device, [&] {
        se = cudaFuncSetAttribute(coupling_partial_kernel<L, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem));
        return se == cudaSuccess ? 1 : 0;
      }) == 0)
    return se != cudaSuccess ? se : cudaErrorInvalidConfiguration;
  if (N <= 0) return cudaSuccess;
  if (chunks < 1) chunks = 1;
  const int64_t chunk = (N + chunks - 1) / chunks;
  dim3 grid(static_cast<unsigned>((N + LY::RPB - 1) / LY::RPB), static_cast<unsigned>(chunks));
  coupling_partial_kernel<L, R><<<grid, C::BLOCK, smem, st>>>(
      static_cast<int>(N), static_cast<const Pos4*>(pos), static_cast<const Pair2<R>*>(x),
      static_cast<Pair2<R>*>(partial), k, static_cast<int>(chunk));
  note_launch();
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
// Algorithmic flops per ordered sphere pair and RHS of the rotation-
// translation-rotation evaluation, counted from the same compile-time tables
// the kernel uses (FMA = 2 flops, complex multiply = 6, complex MAC = 8):
//   z-rotation of x+- (2 NH complex multiplies), Wigner-d entries (monomials
//   and one FMA per term, evaluated twice), forward and backward block
//   rotations (8 flops per R entry each), axial build (4 flops per term plus 4
//   for the W+- combination per (mu >= 0, l, l') block), axial apply (2 complex
//   MACs per (mu, l, l')), output phase (2 NH complex MACs), h_p recurrence.
// f(integral_constant<l>) for l = 1 .. sizeof...(I)
template <typename F, int... I>
void for_each_degree(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I + 1>{}), ...);
}

template <int L>
long long rtr_flops_per_pair_t() {
  long long f = 0;
  constexpr int NH = L * (L + 2);
  f += 2LL * NH * 6;                                   // e^{i m phi} x+-
  f += 2LL * (4 * L - 2) + 8;                          // h_p recurrence and start
  long long rot = 0, dm = 0;
  auto per_l = [&](auto LL_) {
    constexpr int l = decltype(LL_)::value;
    rot += 8LL * (2 * l + 1) * (2 * l + 1);
    dm += (2 * l + 1) + 2LL * rtr::DTab<l>::value.off[rtr::DTab<l>::value.ncanon];
  };
  for_each_degree(per_l, std::make_integer_sequence<int, L>{});
  f += 2 * rot + 2 * dm;
  // axial entries: with the transpose symmetry only the entries lo <= li are
  // formed; every entry is applied to both rows
  constexpr bool sym = rtr::Config<L, float>::SYM_AXIAL;
  for (int mu = 0; mu <= L; ++mu) {
    for (int lo = (mu > 1 ? mu : 1); lo <= L; ++lo) {
      for (int li = (mu > 1 ? mu : 1); li <= L; ++li) {
        const rtr::AxialRow<L> a = rtr::make_axial<L>(mu, lo, li);
        if (!sym || lo <= li) f += 4LL * (a.na + a.nb) + 4;
        f += (mu > 0 ? 2 : 1) * 16LL;
      }
    }
  }
  f += 2LL * NH * 8;                                   // output phase and accumulate
  return f;
}

// the alternative FP32 shape (ConfigAlt), in a translation unit of its own
#define CELES_INSTANTIATE_RTR_ALT(LL)                                                                      \
  cudaError_t launch_coupling_rtr_alt_##LL(int64_t N, const void* pos, const void* x, void* partial,       \
                                           double k, int chunks, cudaStream_t st, int maxcl, int atomic) { \
    return rtr::launch_partial<LL, float, rtr::ConfigAlt<LL, float>>(N, pos, x, partial, k, chunks, st,    \
                                                                     maxcl, atomic != 0);                  \
  }                                                                                                         \
  int coupling_rtr_alt_rpb_##LL() { return rtr::ConfigAlt<LL, float>::BLOCK; }                             \
  int coupling_rtr_alt_slices_##LL(int chunks, int maxcl, int atomic) {                                    \
    return rtr::partial_slices<LL, float, rtr::ConfigAlt<LL, float>>(chunks, maxcl, atomic != 0);          \
  }                                                                                                         \
  int coupling_rtr_alt_slots_##LL() { return rtr::resident_slots<LL, float, rtr::ConfigAlt<LL, float>>(); }

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
  cudaError_t launch_coupling_rtr_##LL(int precision, int64_t N, const void* pos, const void* x,           \
                                       void* partial, double k, int chunks, cudaStream_t st, int maxcl,    \
                                       int atomic) {                                                       \
    return precision == 0                                                                                  \
               ? rtr::launch_partial<LL, double>(N, pos, x, partial, k, chunks, st, maxcl, false)          \
               : rtr::launch_partial<LL, float>(N, pos, x, partial, k, chunks, st, maxcl, atomic != 0);    \
  }                                                                                                        \
  int coupling_rtr_rpb_##LL(int precision) {                                                               \
    return precision == 0 ? rtr::Config<LL, double>::BLOCK : rtr::Config<LL, float>::BLOCK;               \
  }                                                                                                        \
  int coupling_rtr_slices_##LL(int precision, int chunks, int maxcl, int atomic) {                         \
    return precision == 0 ? rtr::partial_slices<LL, double>(chunks, maxcl, false)                          \
                          : rtr::partial_slices<LL, float>(chunks, maxcl, atomic != 0);                    \
  }                                                                                                        \
  int coupling_rpb_##LL(int precision) {                                                                   \
    if (precision == 0) return (FP64_UNROLLED) ? CouplingLayout<LL, double>::RPB : kGenericRPB;           \
    return CouplingLayout<LL, float>::RPB;                                                                 \
  }                                                                                                        \
  long long coupling_rtr_flops_##LL() { return rtr_flops_per_pair_t<LL>(); }                                 \
  int coupling_rtr_slots_##LL(int precision) {                                                             \
    return precision == 0 ? rtr::resident_slots<LL, double>() : rtr::resident_slots<LL, float>();           \
  }                                                                                                        \
  cudaError_t launch_rtr_batch_##LL(int precision, const void* sys, int nsys, long long ntiles,              \
                                    unsigned long long* counter, cudaStream_t st) {                          \
    return precision == 0 ? rtr::launch_batch<LL, double>(sys, nsys, ntiles, counter, st)                   \
                          : rtr::launch_batch<LL, float>(sys, nsys, ntiles, counter, st);                   \
  }                                                                                                        \
  int coupling_terms_export_##LL(int* idx, double* val, int cap) {                                         \
    return coupling_terms_export_t<LL>(idx, val, cap);                                                     \
  }

}  // namespace celes
