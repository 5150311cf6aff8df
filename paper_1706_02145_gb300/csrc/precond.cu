// Block-diagonal preconditioner (Sec. 3.2.1): assembly of the diagonal blocks
// M_j of M = I - T W, batched LU factorisation with partial pivoting
// (P_j M_j = L_j U_j) and the block solve x = M_j^{-1} y, all in FP64.
//
// Storage: block j holds n_j = N_j nmax unknowns (its spheres in partition
// order); its matrix is column-major at mats + mat_off[j] (complex128), LU
// factors overwrite it in place (unit lower L below the diagonal, U on and
// above), piv holds the LAPACK-style row interchanges (row k swapped with
// piv[k] at step k).
#include <cooperative_groups.h>
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
// substitution, scatter.  The block's vector lives in shared memory when it
// fits (one barrier per substitution step), else in the global work array.
// Factors in the precision F: FP64, or an FP32 copy for FP32 vectors (a
// preconditioner only has to be the same operator wherever it is applied).
// ---------------------------------------------------------------------------
template <typename F>
__device__ __forceinline__ Pair2<F> cmul_sub(Pair2<F> a, Pair2<F> l, Pair2<F> y) {
  return Pair2<F>{a.re - (l.re * y.re - l.im * y.im), a.im - (l.re * y.im + l.im * y.re)};
}

// acc - sum_{j < tb} A[i, kb + j] v[kb + j]; a full 32-column tile is
// unrolled so that a thread's 32 factor loads are all in flight at once
template <typename F>
__device__ __forceinline__ Pair2<F> tile_gemv(const Pair2<F>* __restrict__ A, int64_t n, int64_t i, int64_t kb,
                                              int tb, const Pair2<F>* v, Pair2<F> acc) {
  const Pair2<F>* col = A + i + kb * n;
  if (tb == 32) {
    Pair2<F> a[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) a[j] = col[j * n];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc = cmul_sub(acc, a[j], v[kb + j]);
  } else {
    for (int j = 0; j < tb; ++j) acc = cmul_sub(acc, col[j * n], v[kb + j]);
  }
  return acc;
}

template <typename F>
__device__ __forceinline__ Pair2<F> shfl_pair(Pair2<F> v, int src) {
  return Pair2<F>{__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}

// Blocked substitution: warp 0 resolves each 32-row diagonal tile with
// shuffles (no block barrier inside a tile), then the whole CTA applies the
// tile's columns to the remaining rows (a GEMV over contiguous column
// segments).  Two barriers per 32 unknowns instead of one or two per unknown.
// The row permutation of partial pivoting is folded into the gather (pivperm:
// position i of the permuted vector holds original entry pivperm[i]).
template <typename R, typename F, bool SMEM>
__global__ void __launch_bounds__(256) precond_apply_kernel(const int64_t* __restrict__ block_off,
                                                            const int64_t* __restrict__ mat_off, int nmax,
                                                            const int* __restrict__ perm,
                                                            const Pair2<F>* __restrict__ mats,
                                                            const int* __restrict__ pivperm, int64_t N,
                                                            const Pair2<R>* __restrict__ x, Pair2<R>* __restrict__ y,
                                                            Pair2<F>* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char pa_smem[];
  const int64_t q = blockIdx.x;
  const int rhs = blockIdx.y;
  const int64_t s0 = block_off[q];
  const int64_t ns = block_off[q + 1] - s0;
  const int64_t n = ns * nmax;
  const Pair2<F>* A = mats + mat_off[q];
  const int* pp = pivperm + s0 * nmax;
  Pair2<F>* v = SMEM ? reinterpret_cast<Pair2<F>*>(pa_smem) : work + (int64_t)rhs * N * nmax + s0 * nmax;
  const Pair2<R>* xr = x + (int64_t)rhs * N * nmax;
  Pair2<R>* yr = y + (int64_t)rhs * N * nmax;
  const int lane = threadIdx.x & 31;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    const int64_t src = pp[t];
    const int64_t a = src / nmax;
    const int r = static_cast<int>(src - a * nmax);
    const Pair2<R> e = xr[(int64_t)perm[s0 + a] * nmax + r];
    v[t] = Pair2<F>{static_cast<F>(e.re), static_cast<F>(e.im)};
  }
  __syncthreads();
  // the diagonal tile is staged in shared memory by the whole CTA (one
  // memory latency) before warp 0 walks its 32 dependent steps
  __shared__ Pair2<F> dt[32][33];
  auto stage = [&](int64_t kb, int tb) {
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
      const int j = t >> 5, i = t & 31;  // column j, row i: coalesced along i
      dt[j][i] = (i < tb && j < tb) ? A[(kb + i) + (kb + j) * n] : Pair2<F>{0, 0};
    }
  };
  // forward substitution with the unit lower factor
  for (int64_t kb = 0; kb < n; kb += 32) {
    const int tb = static_cast<int>(n - kb < 32 ? n - kb : 32);
    stage(kb, tb);
    __syncthreads();
    if (threadIdx.x < 32) {
      Pair2<F> yl = lane < tb ? v[kb + lane] : Pair2<F>{0, 0};
      for (int j = 0; j < tb; ++j) {
        const Pair2<F> yj = shfl_pair(yl, j);
        if (lane > j && lane < tb) yl = cmul_sub(yl, dt[j][lane], yj);
      }
      if (lane < tb) v[kb + lane] = yl;
    }
    __syncthreads();
    for (int64_t i = kb + tb + threadIdx.x; i < n; i += blockDim.x) v[i] = tile_gemv(A, n, i, kb, tb, v, v[i]);
    __syncthreads();
  }
  // back substitution with the upper factor (tiles from the bottom)
  const int64_t ntile = (n + 31) / 32;
  for (int64_t tt = ntile - 1; tt >= 0; --tt) {
    const int64_t kb = tt * 32;
    const int tb = static_cast<int>(n - kb < 32 ? n - kb : 32);
    stage(kb, tb);
    __syncthreads();
    if (threadIdx.x < 32) {
      Pair2<F> yl = lane < tb ? v[kb + lane] : Pair2<F>{0, 0};
      for (int j = tb - 1; j >= 0; --j) {
        if (lane == j) {
          const Pair2<F> u = dt[j][j];
          const F den = u.re * u.re + u.im * u.im;
          yl = Pair2<F>{(yl.re * u.re + yl.im * u.im) / den, (yl.im * u.re - yl.re * u.im) / den};
        }
        const Pair2<F> xj = shfl_pair(yl, j);
        if (lane < j) yl = cmul_sub(yl, dt[j][lane], xj);
      }
      if (lane < tb) v[kb + lane] = yl;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < kb; i += blockDim.x) v[i] = tile_gemv(A, n, i, kb, tb, v, v[i]);
    __syncthreads();
  }
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    const int64_t a = t / nmax;
    const int r = static_cast<int>(t - a * nmax);
    yr[(int64_t)perm[s0 + a] * nmax + r] = Pair2<R>{static_cast<R>(v[t].re), static_cast<R>(v[t].im)};
  }
}

// ---------------------------------------------------------------------------
// apply, cluster form: each block's triangular solves are spread over a
// thread-block cluster of C CTAs (distributed shared memory).  CTA s of the
// cluster owns a contiguous run of the block's 32-row tiles.  Per tile step
// the owner multiplies its (updated) tile by the explicit inverse of the
// 32 x 32 diagonal tile of L (forward) or U (backward), both formed at build
// time, and writes the 32 solved values into every CTA's copy of the block
// vector; after one cluster barrier every CTA applies that tile column to its
// own rows.  The serial chain of a block is then one barrier and one short
// GEMV per tile, the factor traffic is spread over C SMs, and blocks much
// fewer than SMs still fill the GPU.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

// explicit inverses of the diagonal tiles of each block's LU (unit lower L,
// upper U), column-major 32 x 32 each, tiles beyond the block padded with the
// identity; one CTA of 64 threads per tile (32 columns of Linv, 32 of Uinv)
__global__ void __launch_bounds__(64) precond_tile_inverse_kernel(const int64_t* __restrict__ block_off,
                                                                  const int64_t* __restrict__ mat_off,
                                                                  const int64_t* __restrict__ tile_off, int nmax,
                                                                  const double2* __restrict__ mats,
                                                                  double2* __restrict__ tinv) {
  const int64_t q = blockIdx.y;
  const int64_t n = (block_off[q + 1] - block_off[q]) * nmax;
  const int64_t ntile = (n + 31) / 32;
  const int64_t k = blockIdx.x;
  if (k >= ntile) return;
  const int64_t kb = k * 32;
  const int tb = static_cast<int>(n - kb < 32 ? n - kb : 32);
  const double2* A = mats + mat_off[q];
  __shared__ double2 t[32][33];  // t[c][r] = A[kb + r, kb + c]
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int c = e >> 5, r = e & 31;
    t[c][r] = (r < tb && c < tb) ? A[(kb + r) + (kb + c) * n] : make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  double2* Li = tinv + tile_off[q] + k * 2048;
  double2* Ui = Li + 1024;
  const int j = threadIdx.x & 31;
  cd x[32];
  if (threadIdx.x < 32) {
    // column j of L^{-1}: L x = e_j, unit diagonal
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      cd acc = mkc(r == j ? 1.0 : 0.0);
#pragma unroll
      for (int c = 0; c < r; ++c) {
        if (r < tb && c < tb) acc = acc - mkc(t[c][r].x, t[c][r].y) * x[c];
      }
      x[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) Li[j * 32 + r] = make_double2(x[r].re, x[r].im);
  } else {
    // column j of U^{-1}: U x = e_j
#pragma unroll
    for (int r = 31; r >= 0; --r) {
      cd acc = mkc(r == j ? 1.0 : 0.0);
#pragma unroll
      for (int c = r + 1; c < 32; ++c) acc = acc - mkc(t[c][r].x, t[c][r].y) * x[c];
      x[r] = acc / mkc(t[r][r].x, t[r][r].y);
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) Ui[j * 32 + r] = make_double2(x[r].re, x[r].im);
  }
}

cudaError_t launch_precond_tile_inverse(int64_t nblocks, int64_t max_tiles, const int64_t* block_off,
                                        const int64_t* mat_off, const int64_t* tile_off, int nmax, const double* mats,
                                        double* tinv, cudaStream_t st) {
  if (nblocks <= 0 || max_tiles <= 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(max_tiles), static_cast<unsigned>(nblocks));
  precond_tile_inverse_kernel<<<grid, 64, 0, st>>>(block_off, mat_off, tile_off, nmax,
                                                   reinterpret_cast<const double2*>(mats),
                                                   reinterpret_cast<double2*>(tinv));
  note_launch();
  return cudaGetLastError();
}

constexpr int kApplyThreads = 256;
constexpr int kApplyClusterMaxSmem = 160 * 1024;  // largest block vector of the cluster form

// FP64 vectors: the CTA of cluster rank s owns tiles [s * per, min(ntile, (s + 1) * per))
template <typename R, typename F>
__global__ void __launch_bounds__(kApplyThreads) precond_apply_cluster_kernel(
    const int64_t* __restrict__ block_off, const int64_t* __restrict__ mat_off, const int64_t* __restrict__ tile_off,
    int nmax, const int* __restrict__ perm, const Pair2<F>* __restrict__ mats, const Pair2<F>* __restrict__ tinv,
    const int* __restrict__ pivperm, int64_t N, const Pair2<R>* __restrict__ x, Pair2<R>* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char pc_smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int s = static_cast<int>(cluster.block_rank());
  const int64_t q = blockIdx.x / C;
  const int rhs = blockIdx.y;
  const int64_t s0 = block_off[q];
  const int64_t n = (block_off[q + 1] - s0) * nmax;
  const int64_t ntile = (n + 31) / 32;
  const int64_t per = (ntile + C - 1) / C;
  const int64_t t_lo = s * per < ntile ? s * per : ntile;
  const int64_t t_hi = (s + 1) * per < ntile ? (s + 1) * per : ntile;
  const int64_t r_lo = t_lo * 32, r_hi = t_hi * 32 < n ? t_hi * 32 : n;
  const Pair2<F>* A = mats + mat_off[q];
  const Pair2<F>* TI = tinv + tile_off[q];
  const int* pp = pivperm + s0 * nmax;
  const Pair2<R>* xr = x + (int64_t)rhs * N * nmax;
  Pair2<R>* yr = y + (int64_t)rhs * N * nmax;
  Pair2<F>* v = reinterpret_cast<Pair2<F>*>(pc_smem);  // [n]: own rows (partial sums) + solved tiles
  __shared__ Pair2<F> dt[32][33];
  __shared__ Pair2<F> w[32];
  // gather own rows (the pivot permutation folded in)
  for (int64_t t = r_lo + threadIdx.x; t < r_hi; t += blockDim.x) {
    const int64_t src = pp[t];
    const int64_t a = src / nmax;
    const int r = static_cast<int>(src - a * nmax);
    const Pair2<R> e = xr[(int64_t)perm[s0 + a] * nmax + r];
    v[t] = Pair2<F>{static_cast<F>(e.re), static_cast<F>(e.im)};
  }
  __syncthreads();
  cluster.sync();  // every CTA of the cluster has started before any writes into another's shared memory
  const int lane = threadIdx.x & 31;
  // one triangular sweep; fwd: tiles 0..ntile-1 with L, else ntile-1..0 with U
  auto sweep = [&](bool fwd) {
    for (int64_t step = 0; step < ntile; ++step) {
      const int64_t k = fwd ? step : ntile - 1 - step;
      const int64_t kb = k * 32;
      const int tb = static_cast<int>(n - kb < 32 ? n - kb : 32);
      const bool owner = k >= t_lo && k < t_hi;
      if (owner) {
        const Pair2<F>* Ti = TI + k * 2048 + (fwd ? 0 : 1024);
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) dt[e >> 5][e & 31] = Ti[e];
        __syncthreads();
        if (threadIdx.x < 32) {
          F re = 0, im = 0;
#pragma unroll 8
          for (int c = 0; c < 32; ++c) {
            if (c < tb) {
              const Pair2<F> a = dt[c][lane], u = v[kb + c];
              re += a.re * u.re - a.im * u.im;
              im += a.re * u.im + a.im * u.re;
            }
          }
          w[lane] = Pair2<F>{re, im};
        }
        __syncthreads();
        // the solved tile into every CTA's copy of the block vector
        for (int e = threadIdx.x; e < C * 32; e += blockDim.x) {
          const int dst = e >> 5, r = e & 31;
          if (r < tb) cluster.map_shared_rank(v, dst)[kb + r] = w[r];
        }
      }
      cluster.sync();
      // apply tile column k to own rows below (fwd) / above (back) the tile
      const int64_t a0 = fwd ? (r_lo > kb + tb ? r_lo : kb + tb) : r_lo;
      const int64_t a1 = fwd ? r_hi : (r_hi < kb ? r_hi : kb);
      for (int64_t i = a0 + threadIdx.x; i < a1; i += blockDim.x) v[i] = tile_gemv(A, n, i, kb, tb, v, v[i]);
      __syncthreads();
    }
  };
  sweep(true);
  sweep(false);
  for (int64_t t = r_lo + threadIdx.x; t < r_hi; t += blockDim.x) {
    const int64_t a = t / nmax;
    const int r = static_cast<int>(t - a * nmax);
    yr[(int64_t)perm[s0 + a] * nmax + r] = Pair2<R>{static_cast<R>(v[t].re), static_cast<R>(v[t].im)};
  }
  // no CTA leaves while others may still write its shared memory
  cluster.sync();
}

// ---------------------------------------------------------------------------
// The block solve as two triangular products with explicit inverses.  At
// build time each block's FP64 factors are turned into L^{-1} (strictly lower
// part; unit diagonal implied) and U^{-1} (upper part with the diagonal), in
// FP64, stored in the same n x n column-major slot (an FP32 copy serves FP32
// vectors).  The
// apply x = U^{-1} (L^{-1} (P y)) is then two matrix-vector products with no
// serial chain: a cluster of C CTAs per block deals the 32-row tiles round
// robin, computes its rows of t = L^{-1} P y, writes them into every CTA's
// copy of t, meets the others at one cluster barrier and computes its rows of
// x = U^{-1} t.  It reads the same bytes as a substitution (one entry per
// factor element) and is bound by memory bandwidth.  A preconditioner only
// has to be a fixed linear operator close to the block inverse; forming the
// inverses in FP64 keeps the FP32 copy within FP32 rounding of the FP64 one.
// ---------------------------------------------------------------------------

// Column tile j of L^{-1} (z = 0) or U^{-1} (z = 1) of block q, by blocked
// substitution: X_jj = (tile inverse), and for the other row tiles i (below j
// for L, above for U) X_ij = -inv(T_ii) sum_k T_ik X_kj over the tiles k
// between them.  One CTA of 256 threads per (column tile, block, factor);
// thread (row r, column group g) owns X[r][4g .. 4g + 3].
template <typename F>
__global__ void __launch_bounds__(256) precond_tri_inverse_kernel(const int64_t* __restrict__ block_off,
                                                                  const int64_t* __restrict__ mat_off,
                                                                  const int64_t* __restrict__ tile_off, int nmax,
                                                                  const Pair2<F>* __restrict__ lu,
                                                                  const Pair2<F>* __restrict__ tinv,
                                                                  Pair2<F>* __restrict__ inv) {
  using V = Pair2<F>;
  const int64_t q = blockIdx.y;
  const int64_t n = (block_off[q + 1] - block_off[q]) * nmax;
  const int64_t T = (n + 31) / 32;
  const int64_t j = blockIdx.x;
  if (j >= T) return;
  const bool upper = blockIdx.z == 1;
  const V* A = lu + mat_off[q];
  V* X = inv + mat_off[q];
  const V* TI = tinv + tile_off[q];
  __shared__ V as[32][33];  // as[m][r]: factor tile, column m, row r
  __shared__ V xs[32][33];  // xs[c][m]: X tile, column c, row m
  const int tid = threadIdx.x;
  const int r = tid & 31, g = tid >> 5;
  auto tb_of = [&](int64_t t) { return static_cast<int>(n - t * 32 < 32 ? n - t * 32 : 32); };
  const int tbj = tb_of(j);
  // stage tile (ti, tk) of a column-major n x n matrix as dst[col][row]
  // (zero outside the block)
  auto load_tile = [&](V (*dst)[33], const V* M, int64_t ti, int64_t tk) {
    const int tbr = tb_of(ti), tbc = tb_of(tk);
    for (int e = tid; e < 1024; e += 256) {
      const int c = e >> 5, rr = e & 31;
      dst[c][rr] = (rr < tbr && c < tbc) ? M[(ti * 32 + rr) + (tk * 32 + c) * n] : V{0, 0};
    }
  };
  // the inverse of diagonal tile t (the whole unit-lower L or upper U
  // inverse, identity-padded), as dst[col][row]
  auto load_tinv = [&](V (*dst)[33], int64_t t) {
    const V* Ti = TI + t * 2048 + (upper ? 1024 : 0);
    for (int e = tid; e < 1024; e += 256) dst[e >> 5][e & 31] = Ti[e];
  };
  // X_jj: write its part (strictly lower for L, upper for U) into the slot
  load_tinv(xs, j);
  __syncthreads();
  for (int e = tid; e < 1024; e += 256) {
    const int c = e >> 5, rr = e & 31;
    if (rr < tbj && c < tbj && (upper ? rr <= c : rr > c)) X[(j * 32 + rr) + (j * 32 + c) * n] = xs[c][rr];
  }
  __syncthreads();
  const int64_t i0 = upper ? j - 1 : j + 1;
  const int64_t di = upper ? -1 : 1;
  for (int64_t i = i0; upper ? i >= 0 : i < T; i += di) {
    V acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = V{0, 0};
    // S = sum over the tiles k strictly between i and j, and k = j
    const int64_t k0 = upper ? i + 1 : j, k1 = upper ? j : i - 1;
    for (int64_t k = k0; k <= k1; ++k) {
      load_tile(as, A, i, k);  // as[m][r] = T_ik[r][m]
      if (k == j) load_tinv(xs, j);
      else load_tile(xs, X, k, j);  // xs[c][m] = X_kj[m][c]
      __syncthreads();
#pragma unroll 8
      for (int m = 0; m < 32; ++m) {
        const V a = as[m][r];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const V b = xs[4 * g + u][m];
          acc[u].re += a.re * b.re - a.im * b.im;
          acc[u].im += a.re * b.im + a.im * b.re;
        }
      }
      __syncthreads();
    }
    // X_ij = -inv(T_ii) S
#pragma unroll
    for (int u = 0; u < 4; ++u) xs[4 * g + u][r] = acc[u];
    load_tinv(as, i);
    __syncthreads();
    V out[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) out[u] = V{0, 0};
#pragma unroll 8
    for (int m = 0; m < 32; ++m) {
      const V a = as[m][r];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const V b = xs[4 * g + u][m];
        out[u].re -= a.re * b.re - a.im * b.im;
        out[u].im -= a.re * b.im + a.im * b.re;
      }
    }
    const int tbi = tb_of(i);
    if (r < tbi) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = 4 * g + u;
        if (c < tbj) X[(i * 32 + r) + (j * 32 + c) * n] = out[u];
      }
    }
    __syncthreads();  // X_ij is read back by the next row tiles
  }
}
constexpr int kInvThreads = 256;

// x = U^{-1} (L^{-1} (P y)) for one (block, RHS) per cluster of C CTAs; the
// 32-row tiles are dealt round robin (warp w of CTA s takes tiles s + C (w +
// 8 m)), one lane per row, so each column of a tile is one coalesced 256-byte
// read.  Every CTA gathers the whole (pivot-permuted) block vector.
template <typename R, typename F>
__global__ void __launch_bounds__(kInvThreads) precond_apply_inv_kernel(const int64_t* __restrict__ block_off,
                                                                        const int64_t* __restrict__ mat_off, int nmax,
                                                                        const int* __restrict__ perm,
                                                                        const Pair2<F>* __restrict__ inv,
                                                                        const int* __restrict__ pivperm, int64_t N,
                                                                        const Pair2<R>* __restrict__ x,
                                                                        Pair2<R>* __restrict__ y) {
  using V = Pair2<F>;
  extern __shared__ __align__(16) unsigned char pi_smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int s = static_cast<int>(cluster.block_rank());
  const int64_t q = blockIdx.x / C;
  const int rhs = blockIdx.y;
  const int64_t s0 = block_off[q];
  const int64_t n = (block_off[q + 1] - s0) * nmax;
  const int64_t T = (n + 31) / 32;
  const V* A = inv + mat_off[q];
  const int* pp = pivperm + s0 * nmax;
  const Pair2<R>* xr = x + (int64_t)rhs * N * nmax;
  Pair2<R>* yr = y + (int64_t)rhs * N * nmax;
  V* xv = reinterpret_cast<V*>(pi_smem);  // [n] P y
  V* tv = xv + n;                         // [n] t = L^{-1} P y
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int NW = kInvThreads / 32;
  for (int64_t t = tid; t < n; t += blockDim.x) {
    const int64_t src = pp[t];
    const int64_t a = src / nmax;
    const int r = static_cast<int>(src - a * nmax);
    const Pair2<R> e = xr[(int64_t)perm[s0 + a] * nmax + r];
    xv[t] = V{static_cast<F>(e.re), static_cast<F>(e.im)};
  }
  // every CTA of the cluster has started (and gathered) before any writes
  // into another's shared memory
  cluster.sync();
  // row i: sum over columns [j0, j1) of A[i, j] v[j]
  auto rowdot = [&](int64_t i, int64_t j0, int64_t j1, const V* v) {
    F ar0 = 0, ai0 = 0, ar1 = 0, ai1 = 0;
    const V* a = A + i;
    int64_t jj = j0;
    for (; jj + 8 <= j1; jj += 8) {
      V m[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) m[u] = a[(jj + u) * n];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        const V v0 = v[jj + u], v1 = v[jj + u + 1];
        ar0 += m[u].re * v0.re - m[u].im * v0.im;
        ai0 += m[u].re * v0.im + m[u].im * v0.re;
        ar1 += m[u + 1].re * v1.re - m[u + 1].im * v1.im;
        ai1 += m[u + 1].re * v1.im + m[u + 1].im * v1.re;
      }
    }
    for (; jj < j1; ++jj) {
      const V m = a[jj * n], v0 = v[jj];
      ar0 += m.re * v0.re - m.im * v0.im;
      ai0 += m.re * v0.im + m.im * v0.re;
    }
    return V{ar0 + ar1, ai0 + ai1};
  };
  // t = L^{-1} P y on own tiles (unit diagonal), into every CTA's copy of t
  for (int64_t tt = s + (int64_t)C * wid; tt < T; tt += (int64_t)C * NW) {
    const int64_t i = tt * 32 + lane;
    if (i < n) {
      const V d = rowdot(i, 0, i, xv);
      const V t = V{xv[i].re + d.re, xv[i].im + d.im};
      for (int dst = 0; dst < C; ++dst) cluster.map_shared_rank(tv, dst)[i] = t;
    }
  }
  cluster.sync();
  // x = U^{-1} t on own tiles
  for (int64_t tt = s + (int64_t)C * wid; tt < T; tt += (int64_t)C * NW) {
    const int64_t i = tt * 32 + lane;
    if (i < n) {
      const V o = rowdot(i, i, n, tv);
      const int64_t a = i / nmax;
      const int r = static_cast<int>(i - a * nmax);
      yr[(int64_t)perm[s0 + a] * nmax + r] = Pair2<R>{static_cast<R>(o.re), static_cast<R>(o.im)};
    }
  }
}

// FP64 explicit inverses of L and U of every block (from the FP64 LU and
// FP64 tile inverses) into inv64
cudaError_t launch_precond_tri_inverse(int64_t nblocks, int64_t max_tiles, const int64_t* block_off,
                                       const int64_t* mat_off, const int64_t* tile_off, int nmax, const double* lu,
                                       const double* tinv, double* inv, cudaStream_t st) {
  if (nblocks <= 0 || max_tiles <= 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(max_tiles), static_cast<unsigned>(nblocks), 2);
  precond_tri_inverse_kernel<double><<<grid, 256, 0, st>>>(block_off, mat_off, tile_off, nmax,
                                                           reinterpret_cast<const Pair2<double>*>(lu),
                                                           reinterpret_cast<const Pair2<double>*>(tinv),
                                                           reinterpret_cast<Pair2<double>*>(inv));
  note_launch();
  return cudaGetLastError();
}

// position -> source index of the row interchanges of each block's LU
// (applied in order kk = 0..n-1, as the factorisation recorded them)
__global__ void pivot_perm_kernel(const int64_t* __restrict__ block_off, int nmax, const int* __restrict__ piv,
                                  int* __restrict__ pivperm) {
  const int64_t q = blockIdx.x;
  const int64_t s0 = block_off[q];
  const int64_t n = (block_off[q + 1] - s0) * nmax;
  const int* pv = piv + s0 * nmax;
  int* pp = pivperm + s0 * nmax;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) pp[t] = static_cast<int>(t);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int64_t kk = 0; kk < n; ++kk) {
      const int64_t p = pv[kk];
      if (p != kk) {
        const int t = pp[kk];
        pp[kk] = pp[p];
        pp[p] = t;
      }
    }
  }
}

cudaError_t launch_pivot_perm(int64_t nblocks, const int64_t* block_off, int nmax, const int* piv, int* pivperm,
                              cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  pivot_perm_kernel<<<static_cast<unsigned>(nblocks), 256, 0, st>>>(block_off, nmax, piv, pivperm);
  note_launch();
  return cudaGetLastError();
}

template <typename R, typename F>
cudaError_t launch_apply_t(int64_t nblocks, const int64_t* block_off, const int64_t* mat_off, int nmax,
                           const int* perm, const void* mats, const int* piv, int64_t N, int nrhs, const void* x,
                           void* y, void* work, int max_block_dim, cudaStream_t st) {
  dim3 grid(static_cast<unsigned>(nblocks), static_cast<unsigned>(nrhs));
  const size_t smem = sizeof(Pair2<F>) * static_cast<size_t>(max_block_dim);
  if (smem <= 200 * 1024) {
    // the shared-memory opt-in, once on each device
    static PerDevice attr;
    cudaError_t se = cudaSuccess;
    if (attr.get(current_device, [&] {
          se = cudaFuncSetAttribute(precond_apply_kernel<R, F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024);
          return se == cudaSuccess ? 1 : 0;
        }) == 0)
      return se != cudaSuccess ? se : cudaErrorInvalidConfiguration;
    precond_apply_kernel<R, F, true><<<grid, 256, smem, st>>>(
        block_off, mat_off, nmax, perm, static_cast<const Pair2<F>*>(mats), piv, N, static_cast<const Pair2<R>*>(x),
        static_cast<Pair2<R>*>(y), static_cast<Pair2<F>*>(work));
  } else {
    precond_apply_kernel<R, F, false><<<grid, 256, 0, st>>>(
        block_off, mat_off, nmax, perm, static_cast<const Pair2<F>*>(mats), piv, N, static_cast<const Pair2<R>*>(x),
        static_cast<Pair2<R>*>(y), static_cast<Pair2<F>*>(work));
  }
  note_launch();
  return cudaGetLastError();
}

template <typename R, typename F>
cudaError_t launch_apply_cluster_t(int64_t nblocks, const int64_t* block_off, const int64_t* mat_off,
                                   const int64_t* tile_off, int nmax, const int* perm, const void* mats,
                                   const void* tinv, const int* pivperm, int64_t N, int nrhs, const void* x, void* y,
                                   int max_block_dim, int csize, cudaStream_t st) {
  const size_t smem = sizeof(Pair2<F>) * static_cast<size_t>(max_block_dim);
  static PerDevice attr;
  cudaError_t se = cudaSuccess;
  if (attr.get(current_device, [&] {
        se = cudaFuncSetAttribute(precond_apply_cluster_kernel<R, F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kApplyClusterMaxSmem);
        return se == cudaSuccess ? 1 : 0;
      }) == 0)
    return se != cudaSuccess ? se : cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(nblocks * csize), static_cast<unsigned>(nrhs));
  cfg.blockDim = dim3(kApplyThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = static_cast<unsigned>(csize);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, precond_apply_cluster_kernel<R, F>, block_off, mat_off, tile_off, nmax,
                                           perm, static_cast<const Pair2<F>*>(mats), static_cast<const Pair2<F>*>(tinv),
                                           pivperm, N, static_cast<const Pair2<R>*>(x), static_cast<Pair2<R>*>(y));
  note_launch();
  return e;
}

// cluster size of the apply for blocks of about `mean_tiles` 32-row tiles
int precond_cluster_size(double mean_tiles) {
  if (mean_tiles >= 12.0) return 4;
  if (mean_tiles >= 4.0) return 2;
  return 1;
}

// the two-product form fits when both FP64 block vectors fit in shared memory
bool precond_inverse_fits(int max_block_dim) {
  return 2 * sizeof(Pair2<double>) * static_cast<size_t>(max_block_dim) <= kApplyClusterMaxSmem;
}

template <typename R>
cudaError_t launch_apply_inv(int64_t nblocks, const int64_t* block_off, const int64_t* mat_off, int nmax,
                             const int* perm, const R* inv, const int* pivperm, int64_t N, int nrhs, const void* x,
                             void* y, int max_block_dim, int csize, cudaStream_t st) {
  static PerDevice attr;
  cudaError_t se = cudaSuccess;
  if (attr.get(current_device, [&] {
        se = cudaFuncSetAttribute(precond_apply_inv_kernel<R, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kApplyClusterMaxSmem);
        return se == cudaSuccess ? 1 : 0;
      }) == 0)
    return se != cudaSuccess ? se : cudaErrorInvalidConfiguration;
  const size_t smem = 2 * sizeof(Pair2<R>) * static_cast<size_t>(max_block_dim);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(nblocks * csize), static_cast<unsigned>(nrhs));
  cfg.blockDim = dim3(kInvThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = static_cast<unsigned>(csize);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, precond_apply_inv_kernel<R, R>, block_off, mat_off, nmax, perm,
                                           reinterpret_cast<const Pair2<R>*>(inv), pivperm, N,
                                           static_cast<const Pair2<R>*>(x), static_cast<Pair2<R>*>(y));
  note_launch();
  return e;
}

// FP64 vectors use the FP64 factors (mats), FP32 vectors the FP32 copy
// (mats32).  With `inverse` set both hold the explicit inverses of L and U
// (the two-product form); otherwise the LU factors, solved by substitution:
// in the cluster form when tile inverses exist and the block vector fits in
// shared memory, else one CTA per block.
template <typename R>
cudaError_t launch_precond_apply(int64_t nblocks, const int64_t* block_off, const int64_t* mat_off, int nmax,
                                 const int* perm, const double* mats, const float* mats32, const int* piv, int64_t N,
                                 int nrhs, const void* x, void* y, double* work, int max_block_dim, cudaStream_t st,
                                 const int64_t* tile_off, const double* tinv, const float* tinv32, int csize,
                                 bool inverse) {
  if (nblocks <= 0) return cudaSuccess;
  constexpr size_t esz = sizeof(R) == 8 ? 16 : 8;
  if (inverse) {
    if constexpr (sizeof(R) == 8)
      return launch_apply_inv<double>(nblocks, block_off, mat_off, nmax, perm, mats, piv, N, nrhs, x, y,
                                      max_block_dim, csize >= 1 ? csize : 1, st);
    else
      return launch_apply_inv<float>(nblocks, block_off, mat_off, nmax, perm, mats32, piv, N, nrhs, x, y,
                                     max_block_dim, csize >= 1 ? csize : 1, st);
  }
  if (tinv && csize >= 1 && esz * static_cast<size_t>(max_block_dim) <= kApplyClusterMaxSmem) {
    if constexpr (sizeof(R) == 8)
      return launch_apply_cluster_t<double, double>(nblocks, block_off, mat_off, tile_off, nmax, perm, mats, tinv,
                                                    piv, N, nrhs, x, y, max_block_dim, csize, st);
    else
      return launch_apply_cluster_t<float, float>(nblocks, block_off, mat_off, tile_off, nmax, perm, mats32, tinv32,
                                                  piv, N, nrhs, x, y, max_block_dim, csize, st);
  }
  if constexpr (sizeof(R) == 8)
    return launch_apply_t<double, double>(nblocks, block_off, mat_off, nmax, perm, mats, piv, N, nrhs, x, y, work,
                                          max_block_dim, st);
  else
    return launch_apply_t<float, float>(nblocks, block_off, mat_off, nmax, perm, mats32, piv, N, nrhs, x, y, work,
                                        max_block_dim, st);
}
template cudaError_t launch_precond_apply<float>(int64_t, const int64_t*, const int64_t*, int, const int*,
                                                 const double*, const float*, const int*, int64_t, int, const void*,
                                                 void*, double*, int, cudaStream_t, const int64_t*, const double*,
                                                 const float*, int, bool);
template cudaError_t launch_precond_apply<double>(int64_t, const int64_t*, const int64_t*, int, const int*,
                                                  const double*, const float*, const int*, int64_t, int, const void*,
                                                  void*, double*, int, cudaStream_t, const int64_t*, const double*,
                                                  const float*, int, bool);

__global__ void f64_to_f32_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    b[t] = static_cast<float>(a[t]);
}
cudaError_t launch_f64_to_f32(int64_t n, const double* a, float* b, cudaStream_t st) {
  const int64_t blocks = (n + 255) / 256;
  const int64_t cap = 16LL * device_sms();
  f64_to_f32_kernel<<<static_cast<unsigned>(blocks < cap ? (blocks > 0 ? blocks : 1) : cap), 256, 0, st>>>(
      n, a, b);
  note_launch();
  return cudaGetLastError();
}

}  // namespace celes
