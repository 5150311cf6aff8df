// Host-side declarations of the kernel launchers (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "../../include/celes.h"
#include "per_device.h"

struct celes_ctx;

namespace celes {

// 2-norm from a reduced <v, v>: rounding may make a tiny value negative
// (clamped to 0), but a NaN stays NaN so that the solvers' finiteness checks
// see it (std::max(0.0, NaN) is 0.0)
inline double norm_from_dot(double q) { return std::isnan(q) ? q : std::sqrt(std::max(0.0, q)); }

// named NVTX range over one API call (shows the phases in a profiler's
// timeline; a no-op when no tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// read-only view of a context's device data (for the learned-guess module)
struct CtxView {
  int64_t N;
  int L, nmax, nrhs;
  double k;
  const void* pos;       // [N] Pos4
  const double* radii;   // [N]
  const double* nrel;    // [N] complex
  const double* rhs;     // [nrhs][N][nmax] complex, T a_in
  const double* b;       // [nrhs][N][nmax] complex, current solution
  bool has_b;
  const void* tq;        // [N][2][L] complex128, T
  const void* tq32;      // [N][2][L] complex64, T
  int device;
  const celes_incident* incidents;  // [nrhs] host descriptors
  cudaStream_t stream;
};
int ctx_view(celes_ctx* c, CtxView* v);
// store a learned first iterate for RHS `rhs` (device pointer, complex128 [N][nmax])
int ctx_set_learned_guess(celes_ctx* c, int rhs, const double* b0_dev);
// the solution buffer (b, [nrhs][N][nmax] complex128) now holds a solution
int ctx_mark_solved(celes_ctx* c);

// process-wide count of kernels launched by this library
void note_launch(int n = 1);
int64_t kernel_launch_count();

// coupling: partial products per source chunk (coupling_L*.cu)
cudaError_t launch_coupling_partial(int L, int precision, int64_t N, const void* pos, const void* x, void* partial,
                                    double k, int chunks, cudaStream_t st);
int coupling_receivers_per_block(int L, int precision);
int coupling_term_count(int L);
int coupling_terms_export(int L, int* idx, double* val, int cap);

template <typename R>
cudaError_t launch_coupling_epilogue(int64_t N, int L, int chunks, const void* partial, const void* x, const void* tq,
                                     void* y, int mode, cudaStream_t st);

cudaError_t launch_mie(int64_t N, int L, double k, const double* radii, const double* n_rel, double* tq,
                       cudaStream_t st);
cudaError_t launch_tq_expand(int64_t N, int L, const double* tq, double* tdiag, float* tq32, cudaStream_t st);
cudaError_t launch_plane_wave(int64_t N, int L, double k, const void* pos, double beta, double alpha, int pol,
                              double e0r, double e0i, double* a, cudaStream_t st);
cudaError_t launch_gaussian_beam(int64_t N, int L, double k, const void* pos, double w, const double* focus,
                                 double alphaG, double e0r, double e0i, int nb, const double* nodes,
                                 const double* weights, double* a, cudaStream_t st);

// the current device's ordinal (PerDevice's device query)
inline bool current_device(int* d) { return cudaGetDevice(d) == cudaSuccess; }

int vec_dot_blocks(int64_t n);
// streaming multiprocessors of the current device (queried once per device)
int device_sms();
template <typename R>
cudaError_t launch_multi_dotc(int64_t n, int nv, const void* V, int64_t ldv, const void* w, double* partial,
                              double* out, cudaStream_t st);
template <typename R>
cudaError_t launch_multi_axpy(int64_t n, int nv, const void* V, int64_t ldv, const double* h, double alpha0, void* w,
                              cudaStream_t st);
template <typename R>
cudaError_t launch_multi_combine(int64_t n, int nv, const void* V, int64_t ldv, const double* c, double beta, void* y,
                                 cudaStream_t st);
template <typename RX, typename RY>
cudaError_t launch_axpby(int64_t n, double a, const void* x, double b, void* y, cudaStream_t st);
// z = a x + b y, complex a = ar + i ai, b = br + i bi (z may alias x or y)
template <typename R>
cudaError_t launch_caxpbyz(int64_t n, double ar, double ai, const void* x, double br, double bi, const void* y,
                           void* z, cudaStream_t st);
cudaError_t launch_tdiag_mul(int64_t n_per_rhs, int nrhs, const double* tdiag, const double* x, double* y,
                             cudaStream_t st);
template <typename R>
cudaError_t launch_nonfinite(int64_t n, const void* v, int* flag, cudaStream_t st);

cudaError_t launch_farfield(int64_t N, int L, double k, const void* pos, const double* b, int64_t Nd,
                            const double* dirs, double* g, cudaStream_t st);
cudaError_t launch_overlap_check(int64_t N, const void* pos, const double* radii, int* flag, cudaStream_t st);

// tensor-core GEMM (tc_gemm.cu): C = alpha A B^T + beta C, BF16 in, FP32 out
cudaError_t launch_gemm_bf16_tn(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C, int ldc,
                                float alpha, float beta, int* err, cudaStream_t st);

// block-diagonal preconditioner (precond.cu)
cudaError_t launch_precond_assemble(int L, int64_t nblocks, const int64_t* block_off, const int64_t* mat_off,
                                    const int* perm, const void* pos, const double* tq, double k, double* mats,
                                    int64_t max_pairs, cudaStream_t st);
cudaError_t launch_precond_lu(int64_t nblocks, const int64_t* block_off, const int64_t* mat_off, int nmax,
                              double* mats, int* piv, int* info, cudaStream_t st);
// tile_off/tinv/tinv32: explicit inverses of the 32 x 32 diagonal tiles of
// each block's L and U (launch_precond_tile_inverse; tinv = nullptr selects
// the one-CTA-per-block substitution); csize: CTAs per block (cluster size)
template <typename R>
cudaError_t launch_precond_apply(int64_t nblocks, const int64_t* block_off, const int64_t* mat_off, int nmax,
                                 const int* perm, const double* mats, const float* mats32, const int* piv, int64_t N,
                                 int nrhs, const void* x, void* y, double* work, int max_block_dim, cudaStream_t st,
                                 const int64_t* tile_off = nullptr, const double* tinv = nullptr,
                                 const float* tinv32 = nullptr, int csize = 0, bool inverse = false);
// FP64 explicit inverses of each block's L and U from its FP64 LU factors and
// FP64 tile inverses (same layout as the factors)
cudaError_t launch_precond_tri_inverse(int64_t nblocks, int64_t max_tiles, const int64_t* block_off,
                                       const int64_t* mat_off, const int64_t* tile_off, int nmax, const double* lu,
                                       const double* tinv, double* inv, cudaStream_t st);
bool precond_inverse_fits(int max_block_dim);
cudaError_t launch_precond_tile_inverse(int64_t nblocks, int64_t max_tiles, const int64_t* block_off,
                                        const int64_t* mat_off, const int64_t* tile_off, int nmax, const double* mats,
                                        double* tinv, cudaStream_t st);
int precond_cluster_size(double mean_tiles);
// per block, the gather permutation equivalent to the LU's row interchanges
cudaError_t launch_pivot_perm(int64_t nblocks, const int64_t* block_off, int nmax, const int* piv, int* pivperm,
                              cudaStream_t st);
// elementwise FP64 -> FP32
cudaError_t launch_f64_to_f32(int64_t n, const double* a, float* b, cudaStream_t st);

}  // namespace celes
