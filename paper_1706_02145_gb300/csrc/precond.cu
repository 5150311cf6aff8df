// Block-diagonal preconditioner (Sec. 3.2.1): assembly of the diagonal blocks
// M_j of M = I - T W, batched LU factorisation with partial pivoting
// (P_j M_j = L_j U_j) and the block solve x = M_j^{-1} y, all in FP64.
//
// Storage: block j holds n_j = N_j nmax unknowns (its spheres in partition
// order); its matrix is column-major at mats + mat_off[j] (complex128), LU
// factors overwrite it in place (unit lower L below the diagonal, U on and
// above), piv holds the LAPACK-style row interchanges (row k swapped with
// piv[k] at step k).
#include <cuda_runtime.h>

#include <cstdint>

#include "cmath.cuh"
#include "coupling_kernel.cuh"
#include "kernels.h"

namespace celes {

// ---------------------------------------------------------------------------
// batched LU with partial pivoting: one CTA per block, right-looking
// ---------------------------------------------------------------------------
constexpr int kLuThreads = 512;

__global__ void __launch_bounds__(kLuThreads) precond_lu_kernel(const int64_t* __restrict__ block_off,
                                                                const int64_t* __restrict__ mat_off, int nmax,
                                                                double2* __restrict__ mats, int* __restrict__ piv,
                                                                int* __restrict__ info) {
  const int64_t q = blockIdx.x;
  const int64_t n = (block_off[q + 1] - block_off[q]) * nmax;
  double2* A = mats + mat_off[q];
  int* pv = piv + block_off[q] * nmax;
  __shared__ double sval[kLuThreads / 32];
  __shared__ int sidx[kLuThreads / 32];
  __shared__ int s_p;
  __shared__ double2 s_pivot;
  if (threadIdx.x == 0) info[q] = 0;
  for (int64_t kk = 0; kk < n; ++kk) {
    // pivot search in column kk
    double best = -1.0;
    int bi = static_cast<int>(kk);
    for (int64_t i = kk + threadIdx.x; i < n; i += blockDim.x) {
      const double2 v = A[i + kk * n];
      const double a = fabs(v.x) + fabs(v.y);
      if (a > best) {
        best = a;
        bi = static_cast<int>(i);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if ((threadIdx.x & 31) == 0) {
      sval[threadIdx.x >> 5] = best;
      sidx[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = -1.0;
      int ix = static_cast<int>(kk);
      for (int w = 0; w < kLuThreads / 32; ++w) {
        if (sval[w] > b || (sval[w] == b && sidx[w] < ix)) {
          b = sval[w];
          ix = sidx[w];
        }
      }
      s_p = ix;
      pv[kk] = ix;
      if (b <= 0.0 && info[q] == 0) info[q] = static_cast<int>(kk) + 1;
    }
    __syncthreads();
    const int64_t p = s_p;
    // swap rows kk and p over all columns
    if (p != kk) {
      for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double2 t = A[kk + j * n];
        A[kk + j * n] = A[p + j * n];
        A[p + j * n] = t;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_pivot = A[kk + kk * n];
    __syncthreads();
    const cd piv_v = mkc(s_pivot.x, s_pivot.y);
    const bool ok = abs2(piv_v) > 0.0;
    // scale the column below the pivot
    for (int64_t i = kk + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double2 v = A[i + kk * n];
      const cd l = ok ? mkc(v.x, v.y) / piv_v : mkc(0.0);
      A[i + kk * n] = make_double2(l.re, l.im);
    }
    __syncthreads();
    // rank-1 update of the trailing matrix, threads over rows (coalesced)
    const int64_t m = n - kk - 1;
    for (int64_t t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int64_t jj = t / m, ii = t - jj * m;
      const int64_t i = kk + 1 + ii, j = kk + 1 + jj;
      const double2 l = A[i + kk * n];
      const double2 u = A[kk + j * n];
      double2 a = A[i + j * n];
      a.x -= l.x * u.x - l.y * u.y;
      a.y -= l.x * u.y + l.y * u.x;
      A[i + j * n] = a;
    }
    __syncthreads();
  }
}

cudaError_t launch_precond_lu(int64_t nblocks, const int64_t* block_off, const int64_t* mat_off, int nmax,
                              double* mats, int* piv, int* info, cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  precond_lu_kernel<<<static_cast<unsigned>(nblocks), kLuThreads, 0, st>>>(
      block_off, mat_off, nmax, reinterpret_cast<double2*>(mats), piv, info);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// apply: one CTA per (block, rhs): gather, permute, forward and back
// substitution in FP64, scatter
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) precond_apply_kernel(const int64_t* __restrict__ block_off,
                                                            const int64_t* __restrict__ mat_off, int nmax,
                                                            const int* __restrict__ perm,
                                                            const double2* __restrict__ mats,
                                                            const int* __restrict__ piv, int64_t N,
                                                            const Pair2<R>* __restrict__ x, Pair2<R>* __restrict__ y,
                                                            double2* __restrict__ work) {
  const int64_t q = blockIdx.x;
  const int rhs = blockIdx.y;
  const int64_t s0 = block_off[q];
  const int64_t ns = block_off[q + 1] - s0;
  const int64_t n = ns * nmax;
  const double2* A = mats + mat_off[q];
  const int* pv = piv + s0 * nmax;
  double2* v = work + (int64_t)rhs * N * nmax + s0 * nmax;
  const Pair2<R>* xr = x + (int64_t)rhs * N * nmax;
  Pair2<R>* yr = y + (int64_t)rhs * N * nmax;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    const int64_t a = t / nmax;
    const int r = static_cast<int>(t - a * nmax);
    const Pair2<R> e = xr[(int64_t)perm[s0 + a] * nmax + r];
    v[t] = make_double2(static_cast<double>(e.re), static_cast<double>(e.im));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int64_t kk = 0; kk < n; ++kk) {
      const int64_t p = pv[kk];
      if (p != kk) {
        const double2 t = v[kk];
        v[kk] = v[p];
        v[p] = t;
      }
    }
  }
  __syncthreads();
  // forward substitution with the unit lower factor (column oriented)
  for (int64_t kk = 0; kk < n; ++kk) {
    const double2 yk = v[kk];
    for (int64_t i = kk + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double2 l = A[i + kk * n];
      double2 a = v[i];
      a.x -= l.x * yk.x - l.y * yk.y;
      a.y -= l.x * yk.y + l.y * yk.x;
      v[i] = a;
    }
    __syncthreads();
  }
  // back substitution with the upper factor
  for (int64_t kk = n - 1; kk >= 0; --kk) {
    if (threadIdx.x == 0) {
      const double2 u = A[kk + kk * n];
      const cd z = mkc(v[kk].x, v[kk].y) / mkc(u.x, u.y);
      v[kk] = make_double2(z.re, z.im);
    }
    __syncthreads();
    const double2 xk = v[kk];
    for (int64_t i = threadIdx.x; i < kk; i += blockDim.x) {
      const double2 u = A[i + kk * n];
      double2 a = v[i];
      a.x -= u.x * xk.x - u.y * xk.y;
      a.y -= u.x * xk.y + u.y * xk.x;
      v[i] = a;
    }
    __syncthreads();
  }
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    const int64_t a = t / nmax;
    const int r = static_cast<int>(t - a * nmax);
    yr[(int64_t)perm[s0 + a] * nmax + r] = Pair2<R>{static_cast<R>(v[t].x), static_cast<R>(v[t].y)};
  }
}

template <typename R>
cudaError_t launch_precond_apply(int64_t nblocks, const int64_t* block_off, const int64_t* mat_off, int nmax,
                                 const int* perm, const double* mats, const int* piv, int64_t N, int nrhs,
                                 const void* x, void* y, double* work, int max_block_dim, cudaStream_t st) {
  (void)max_block_dim;
  if (nblocks <= 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(nblocks), static_cast<unsigned>(nrhs));
  precond_apply_kernel<R><<<grid, 256, 0, st>>>(block_off, mat_off, nmax, perm,
                                                reinterpret_cast<const double2*>(mats), piv, N,
                                                static_cast<const Pair2<R>*>(x), static_cast<Pair2<R>*>(y),
                                                reinterpret_cast<double2*>(work));
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_precond_apply<float>(int64_t, const int64_t*, const int64_t*, int, const int*,
                                                 const double*, const int*, int64_t, int, const void*, void*, double*,
                                                 int, cudaStream_t);
template cudaError_t launch_precond_apply<double>(int64_t, const int64_t*, const int64_t*, int, const int*,
                                                  const double*, const int*, int64_t, int, const void*, void*,
                                                  double*, int, cudaStream_t);

}  // namespace celes
