// Setup, epilogue, vector and far-field kernels of the solver.
//
//  * coupling epilogue: sum of the per-chunk partial products, change from the
//    +- basis back to (tau = 1, tau = 2), optional M x = x - T (W x) (Sec. 2.2)
//  * Mie T-matrix (App. B)
//  * incident-field coefficients: plane wave (App. A.2) and Gaussian beam (App. C)
//  * GMRES vector operations (Sec. 3.2): multi-dot, multi-axpy, norms, casts
//  * far-field amplitude g_j (App. D)
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "cmath.cuh"
#include "coupling_kernel.cuh"
#include "kernels.h"

namespace celes {

static std::atomic<int64_t> g_launch_count{0};
void note_launch(int n) { g_launch_count += n; }
int64_t kernel_launch_count() { return g_launch_count.load(); }

static __device__ __forceinline__ int row_l_rt(int r) {
  int l = static_cast<int>(sqrt(static_cast<double>(r + 1)));
  while ((l + 1) * (l + 1) - 1 <= r) ++l;
  while (l * l - 1 > r) --l;
  return l;
}

// ---------------------------------------------------------------------------
// coupling epilogue
// ---------------------------------------------------------------------------
template <typename R>
__global__ void coupling_epilogue_kernel(int64_t N, int L, int chunks, const Pair2<R>* __restrict__ partial,
                                         const Pair2<R>* __restrict__ x, const Pair2<R>* __restrict__ tq,
                                         Pair2<R>* __restrict__ y, int mode) {
  const int NH = L * (L + 2);
  const int64_t total = N * NH;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / NH;
    const int r = static_cast<int>(t - i * NH);
    R pr = 0, pi = 0, mr = 0, mi = 0;
    for (int c = 0; c < chunks; ++c) {
      const Pair2<R>* pc = partial + ((int64_t)c * N + i) * (2 * NH);
      const Pair2<R> a = pc[r];
      const Pair2<R> b = pc[NH + r];
      pr += a.re;
      pi += a.im;
      mr += b.re;
      mi += b.im;
    }
    // y_1 = (y+ + y-)/2, y_2 = (y+ - y-)/2
    Pair2<R> y1{static_cast<R>(0.5) * (pr + mr), static_cast<R>(0.5) * (pi + mi)};
    Pair2<R> y2{static_cast<R>(0.5) * (pr - mr), static_cast<R>(0.5) * (pi - mi)};
    const int64_t o1 = i * 2 * NH + r, o2 = o1 + NH;
    if (mode == 1) {
      const int l = row_l_rt(r);
      const Pair2<R> q1 = tq[(i * 2 + 0) * L + (l - 1)];
      const Pair2<R> q2 = tq[(i * 2 + 1) * L + (l - 1)];
      const Pair2<R> x1 = x[o1], x2 = x[o2];
      y1 = Pair2<R>{x1.re - (q1.re * y1.re - q1.im * y1.im), x1.im - (q1.re * y1.im + q1.im * y1.re)};
      y2 = Pair2<R>{x2.re - (q2.re * y2.re - q2.im * y2.im), x2.im - (q2.re * y2.im + q2.im * y2.re)};
    }
    y[o1] = y1;
    y[o2] = y2;
  }
}

template <typename R>
cudaError_t launch_coupling_epilogue(int64_t N, int L, int chunks, const void* partial, const void* x, const void* tq,
                                     void* y, int mode, cudaStream_t st) {
  const int64_t total = N * L * (L + 2);
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  const int64_t cap = 32LL * device_sms();
  const int grid = static_cast<int>(blocks < cap ? blocks : cap);
  coupling_epilogue_kernel<R><<<grid > 0 ? grid : 1, threads, 0, st>>>(
      N, L, chunks, static_cast<const Pair2<R>*>(partial), static_cast<const Pair2<R>*>(x),
      static_cast<const Pair2<R>*>(tq), static_cast<Pair2<R>*>(y), mode);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_coupling_epilogue<float>(int64_t, int, int, const void*, const void*, const void*, void*,
                                                     int, cudaStream_t);
template cudaError_t launch_coupling_epilogue<double>(int64_t, int, int, const void*, const void*, const void*, void*,
                                                      int, cudaStream_t);

// ---------------------------------------------------------------------------
// Mie T-matrix (App. B): one thread per sphere, all l
//   Q_1l = [j(x) dj(y) - j(y) dj(x)] / [j(y) dh(x) - h(x) dj(y)]
//   Q_2l = [j(x) dj(y) - m^2 j(y) dj(x)] / [m^2 j(y) dh(x) - h(x) dj(y)]
// x = k R, y = m k R, m = n_i / n0, dz(t) = d/dt [t z_l(t)] = t z_{l-1}(t) - l z_l(t)
// ---------------------------------------------------------------------------
__global__ void mie_kernel(int64_t N, int L, double k, const double* __restrict__ radii,
                           const double* __restrict__ n_rel, double* __restrict__ tq) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double R = radii[i];
  const cd m = mkc(n_rel[2 * i], n_rel[2 * i + 1]);
  const double x = k * R;
  const cd y = m * x;
  cd jx[16], jy[16], hx[16];
  double yx[16];
  sph_jn_c(L, mkc(x), jx);
  sph_jn_c(L, y, jy);
  sph_yn_r(L, x, yx);
  for (int l = 0; l <= L; ++l) hx[l] = jx[l] + cd{0.0, yx[l]};
  const cd m2 = m * m;
  for (int l = 1; l <= L; ++l) {
    const cd djx = x * jx[l - 1] - static_cast<double>(l) * jx[l];
    const cd djy = y * jy[l - 1] - static_cast<double>(l) * jy[l];
    const cd dhx = x * hx[l - 1] - static_cast<double>(l) * hx[l];
    const cd q1 = (jx[l] * djy - jy[l] * djx) / (jy[l] * dhx - hx[l] * djy);
    const cd q2 = (jx[l] * djy - m2 * jy[l] * djx) / (m2 * jy[l] * dhx - hx[l] * djy);
    double* o = tq + ((i * 2 + 0) * L + (l - 1)) * 2;
    o[0] = q1.re;
    o[1] = q1.im;
    o = tq + ((i * 2 + 1) * L + (l - 1)) * 2;
    o[0] = q2.re;
    o[1] = q2.im;
  }
}

cudaError_t launch_mie(int64_t N, int L, double k, const double* radii, const double* n_rel, double* tq,
                       cudaStream_t st) {
  const int threads = 128;
  mie_kernel<<<static_cast<unsigned>((N + threads - 1) / threads), threads, 0, st>>>(N, L, k, radii, n_rel, tq);
  note_launch();
  return cudaGetLastError();
}

// T-matrix as an [N][nmax] diagonal and as FP32 copies
__global__ void tq_expand_kernel(int64_t N, int L, const double* __restrict__ tq, double* __restrict__ tdiag,
                                 float* __restrict__ tq32) {
  const int NH = L * (L + 2);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < N * 2 * L) {
    tq32[2 * t] = static_cast<float>(tq[2 * t]);
    tq32[2 * t + 1] = static_cast<float>(tq[2 * t + 1]);
  }
  if (t >= N * NH) return;
  const int64_t i = t / NH;
  const int r = static_cast<int>(t - i * NH);
  const int l = row_l_rt(r);
  for (int tau = 0; tau < 2; ++tau) {
    const double* q = tq + ((i * 2 + tau) * L + (l - 1)) * 2;
    double* o = tdiag + (i * 2 * NH + tau * NH + r) * 2;
    o[0] = q[0];
    o[1] = q[1];
  }
}

cudaError_t launch_tq_expand(int64_t N, int L, const double* tq, double* tdiag, float* tq32, cudaStream_t st) {
  const int64_t total = N * (L * (L + 2) > 2 * L ? L * (L + 2) : 2 * L);
  const int threads = 256;
  tq_expand_kernel<<<static_cast<unsigned>((total + threads - 1) / threads), threads, 0, st>>>(N, L, tq, tdiag, tq32);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// incident coefficients
// ---------------------------------------------------------------------------
static __device__ __forceinline__ void row_decode(int n, int L, int& tau, int& l, int& m) {
  const int NH = L * (L + 2);
  tau = n < NH ? 1 : 2;
  const int r = n < NH ? n : n - NH;
  l = row_l_rt(r);
  m = r - (l * (l + 1) - 1);
}

// Plane wave (App. A.2): a_n = 4 E0 e^{i k.r_i} e^{-i m alpha} B^dagger_nj(beta)
__global__ void plane_wave_kernel(int64_t N, int L, double k, const Pos4* __restrict__ pos, double beta, double alpha,
                                  int pol, double e0r, double e0i, double* __restrict__ a) {
  const int nmax = 2 * L * (L + 2);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N * nmax) return;
  const int64_t i = t / nmax;
  const int n = static_cast<int>(t - i * nmax);
  int tau, l, m;
  row_decode(n, L, tau, l, m);
  const int am = m < 0 ? -m : m;
  double pi[16], ta[16];
  double sb, cb;
  sincos(beta, &sb, &cb);
  pi_tau_m(L, am, cb, sb, pi, ta);
  const cd bd = b_transform(tau, l, m, pol, pi[l], ta[l], true);
  double sa, ca;
  sincos(alpha, &sa, &ca);
  const Pos4 r = pos[i];
  const double kr = k * (sb * ca * r.x + sb * sa * r.y + cb * r.z);
  const cd v = 4.0 * (mkc(e0r, e0i) * cexp_i(kr - m * alpha)) * bd;
  a[2 * t] = v.re;
  a[2 * t + 1] = v.im;
}

cudaError_t launch_plane_wave(int64_t N, int L, double k, const void* pos, double beta, double alpha, int pol,
                              double e0r, double e0i, double* a, cudaStream_t st) {
  const int64_t total = N * 2 * L * (L + 2);
  const int threads = 128;
  plane_wave_kernel<<<static_cast<unsigned>((total + threads - 1) / threads), threads, 0, st>>>(
      N, L, k, static_cast<const Pos4*>(pos), beta, alpha, pol, e0r, e0i, a);
  note_launch();
  return cudaGetLastError();
}

// Gaussian beam (App. C):
//   a_n = E0 k^2 w^2 / pi  sum_j int_0^{pi/2} dbeta sin cos exp(-w^2 k^2 sin^2/4 + i k z_G cos)
//         B^dagger_nj(beta) I_jn(beta)
//   I_jn = 2 pi e^{-i aG} i^{|m-1|} e^{-i(m-1) phi_G} J_{|m-1|}(k rho_G sin) (d_j1 - i d_j2)/2
//        + 2 pi e^{+i aG} i^{|m+1|} e^{-i(m+1) phi_G} J_{|m+1|}(k rho_G sin) (d_j1 + i d_j2)/2
// (rho_G, phi_G, z_G) cylindrical coordinates of r_i - r_G.  beta integral by
// the Gauss-Legendre nodes/weights given in (nodes, weights).
// One CTA per sphere; its threads take the beta nodes.  Per node a thread
// forms what all rows of the sphere share (the Gaussian weight, e^{i k z_G
// cos}, J_mu(k rho_G sin) for mu = 0..L+1 and pi/tau for every |m|), then adds
// each row's term; the terms of a row are summed over the warp by shuffles and
// over the warps in shared memory.
constexpr int kGbThreads = 128;
constexpr int kGbMaxL = 5;
constexpr int kGbMaxRows = 2 * kGbMaxL * (kGbMaxL + 2);

__global__ void __launch_bounds__(kGbThreads)
    gaussian_beam_kernel(int64_t N, int L, double k, const Pos4* __restrict__ pos, double w, double fx, double fy,
                         double fz, double alphaG, double e0r, double e0i, int nb, const double* __restrict__ nodes,
                         const double* __restrict__ weights, double* __restrict__ a) {
  __shared__ cd sU[2 * kGbMaxL + 1], sV[2 * kGbMaxL + 1];
  __shared__ double red[kGbThreads / 32][kGbMaxRows][2];
  const int nmax = 2 * L * (L + 2);
  const int64_t i = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const Pos4 r = pos[i];
  const double dx = r.x - fx, dy = r.y - fy, dz = r.z - fz;
  const double rho = sqrt(dx * dx + dy * dy);
  const double phiG = atan2(dy, dx);
  if (tid <= 2 * L) {
    const int m = tid - L;
    sU[tid] = cexp_i(-alphaG - (m - 1) * phiG) * ipow(abs(m - 1));
    sV[tid] = cexp_i(alphaG - (m + 1) * phiG) * ipow(abs(m + 1));
  }
  for (int q = tid; q < (kGbThreads / 32) * kGbMaxRows * 2; q += blockDim.x) (&red[0][0][0])[q] = 0.0;
  __syncthreads();
  for (int q0 = 0; q0 < nb; q0 += blockDim.x) {
    const int q = q0 + tid;
    double gw = 0.0, sb = 0.0, cb = 1.0;
    if (q < nb) {
      sincos(nodes[q], &sb, &cb);
      gw = weights[q] * sb * cb * exp(-0.25 * (w * k * sb) * (w * k * sb));
    }
    const bool live = gw != 0.0;
    double J[kGbMaxL + 2];
    double pi_all[kGbMaxL + 1][kGbMaxL + 1], ta_all[kGbMaxL + 1][kGbMaxL + 1];
    cd ez = mkc(0.0);
    if (live) {
      const double xr = k * rho * sb;
      for (int mu = 0; mu <= L + 1; ++mu) J[mu] = jn(mu, xr);
      for (int am = 0; am <= L; ++am) pi_tau_m(L, am, cb, sb, pi_all[am], ta_all[am]);
      ez = gw * cexp_i(k * dz * cb);
    }
    for (int n = 0; n < nmax; ++n) {
      cd c = mkc(0.0);
      if (live) {
        int tau, l, m;
        row_decode(n, L, tau, l, m);
        const int am = m < 0 ? -m : m;
        // I_1 = pi (U + V), I_2 = pi (-i U + i V), U = Um J_|m-1|, V = Vm J_|m+1| (2 pi * 1/2 = pi)
        const cd U = J[abs(m - 1)] * sU[m + L], V = J[abs(m + 1)] * sV[m + L];
        const cd I1 = 3.14159265358979323846 * (U + V);
        const cd I2 = 3.14159265358979323846 * (cd{0, -1} * U + cd{0, 1} * V);
        const cd B1 = b_transform(tau, l, m, 1, pi_all[am][l], ta_all[am][l], true);
        const cd B2 = b_transform(tau, l, m, 2, pi_all[am][l], ta_all[am][l], true);
        c = ez * (B1 * I1 + B2 * I2);
      }
      for (int o = 16; o > 0; o >>= 1) {
        c.re += __shfl_down_sync(0xffffffffu, c.re, o);
        c.im += __shfl_down_sync(0xffffffffu, c.im, o);
      }
      if (lane == 0) {
        red[wid][n][0] += c.re;
        red[wid][n][1] += c.im;
      }
    }
  }
  __syncthreads();
  for (int n = tid; n < nmax; n += blockDim.x) {
    cd acc = mkc(0.0);
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) acc = acc + cd{red[q][n][0], red[q][n][1]};
    const cd v = (k * k * w * w / 3.14159265358979323846) * (mkc(e0r, e0i) * acc);
    a[2 * (i * nmax + n)] = v.re;
    a[2 * (i * nmax + n) + 1] = v.im;
  }
}

cudaError_t launch_gaussian_beam(int64_t N, int L, double k, const void* pos, double w, const double* focus,
                                 double alphaG, double e0r, double e0i, int nb, const double* nodes,
                                 const double* weights, double* a, cudaStream_t st) {
  if (L < 1 || L > kGbMaxL) return cudaErrorInvalidValue;
  if (N <= 0) return cudaSuccess;
  gaussian_beam_kernel<<<static_cast<unsigned>(N), kGbThreads, 0, st>>>(
      N, L, k, static_cast<const Pos4*>(pos), w, focus[0], focus[1], focus[2], alphaG, e0r, e0i, nb, nodes, weights,
      a);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// vector kernels (complex vectors of n elements, element type Pair2<R>)
// ---------------------------------------------------------------------------
constexpr int kVecThreads = 256;

// partial[b][j] = sum over this block's range of conj(V_j) w, sixteen vectors
// per pass (w read once per pass), two elements per loop step so that 34
// loads are in flight per thread; per-thread and warp sums in the vector's own
// precision (a few dozen terms each), block sums in FP64.  Launched with two
// CTAs per SM (vec_dot_blocks): each thread then covers enough elements per
// pass to repay the pass's reduction (measured on GB300 at 480 000 elements
// and 50 vectors: 62 us against 118 us for eight vectors per pass at four
// CTAs per SM).
template <typename R>
__global__ void __launch_bounds__(kVecThreads) multi_dotc_kernel(int64_t n, int nv, const Pair2<R>* __restrict__ V,
                                                                int64_t ldv, const Pair2<R>* __restrict__ w,
                                                                double* __restrict__ partial) {
  constexpr int JT = 16;
  __shared__ double red[2 * JT][kVecThreads / 32];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int j0 = 0; j0 < nv; j0 += JT) {
    const int nj = nv - j0 < JT ? nv - j0 : JT;
    R sr[JT], si[JT];
#pragma unroll
    for (int q = 0; q < JT; ++q) sr[q] = si[q] = static_cast<R>(0);
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; t + stride < n; t += 2 * stride) {
      const Pair2<R> b0 = w[t], b1 = w[t + stride];
#pragma unroll
      for (int q = 0; q < JT; ++q) {
        if (q < nj) {
          const Pair2<R> a0 = V[(j0 + q) * ldv + t];
          const Pair2<R> a1 = V[(j0 + q) * ldv + t + stride];
          sr[q] = fma_(a0.re, b0.re, fma_(a0.im, b0.im, sr[q]));
          si[q] = fma_(a0.re, b0.im, fma_(-a0.im, b0.re, si[q]));
          sr[q] = fma_(a1.re, b1.re, fma_(a1.im, b1.im, sr[q]));
          si[q] = fma_(a1.re, b1.im, fma_(-a1.im, b1.re, si[q]));
        }
      }
    }
    if (t < n) {
      const Pair2<R> b0 = w[t];
#pragma unroll
      for (int q = 0; q < JT; ++q) {
        if (q < nj) {
          const Pair2<R> a0 = V[(j0 + q) * ldv + t];
          sr[q] = fma_(a0.re, b0.re, fma_(a0.im, b0.im, sr[q]));
          si[q] = fma_(a0.re, b0.im, fma_(-a0.im, b0.re, si[q]));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < JT; ++q) {
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
      double s = 0.0;
      for (int q = 0; q < kVecThreads / 32; ++q) s += red[threadIdx.x][q];
      const int q = threadIdx.x >> 1;
      partial[((int64_t)blockIdx.x * nv + j0 + q) * 2 + (threadIdx.x & 1)] = s;
    }
    __syncthreads();
  }
}

__global__ void reduce_partials_kernel(int nblocks, int nv, const double* __restrict__ partial,
                                       double* __restrict__ out) {
  const int j = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
    a += partial[((int64_t)q * nv + j) * 2];
    b += partial[((int64_t)q * nv + j) * 2 + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  __shared__ double red[2][32];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q) {
      sa += red[0][q];
      sb += red[1][q];
    }
    out[2 * j] = sa;
    out[2 * j + 1] = sb;
  }
}

int device_sms() {
  static PerDevice cache;
  const int n = cache.get(current_device, [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return v;
  });
  return n > 0 ? n : 1;
}

int vec_dot_blocks(int64_t n) {
  const int64_t b = (n + kVecThreads - 1) / kVecThreads;
  const int64_t cap = 2LL * device_sms();
  return static_cast<int>(b < cap ? (b > 0 ? b : 1) : cap);
}

template <typename R>
cudaError_t launch_multi_dotc(int64_t n, int nv, const void* V, int64_t ldv, const void* w, double* partial,
                              double* out, cudaStream_t st) {
  const int nb = vec_dot_blocks(n);
  multi_dotc_kernel<R><<<nb, kVecThreads, 0, st>>>(n, nv, static_cast<const Pair2<R>*>(V), ldv,
                                                   static_cast<const Pair2<R>*>(w), partial);
  reduce_partials_kernel<<<nv, 256, 0, st>>>(nb, nv, partial, out);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_multi_dotc<float>(int64_t, int, const void*, int64_t, const void*, double*, double*,
                                              cudaStream_t);
template cudaError_t launch_multi_dotc<double>(int64_t, int, const void*, int64_t, const void*, double*, double*,
                                               cudaStream_t);

// w <- alpha0 * w - sum_j h_j V_j   (h given as FP64 complex on the device;
// arithmetic in the vector's precision).  Two elements
// per thread step and the loads of eight vectors issued before their FMAs
// (16 loads in flight per thread), four CTAs per SM; each element's sum is
// formed in the same order as a plain loop over j (measured on GB300 at
// 480 000 elements and 50 vectors: 70 us against 110 us for one element and
// one vector at a time).
template <typename R>
__global__ void __launch_bounds__(kVecThreads) multi_axpy_kernel(int64_t n, int nv, const Pair2<R>* __restrict__ V,
                                                                int64_t ldv, const double* __restrict__ h,
                                                                double alpha0, Pair2<R>* __restrict__ w) {
  constexpr int U = 8;
  __shared__ R hs[2 * 128];
  for (int q = threadIdx.x; q < 2 * nv && q < 256; q += blockDim.x) hs[q] = static_cast<R>(h[q]);
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += 2 * stride) {
    const bool two = t + stride < n;
    const int64_t t1 = two ? t + stride : t;
    R ar0 = static_cast<R>(alpha0) * w[t].re, ai0 = static_cast<R>(alpha0) * w[t].im;
    R ar1 = static_cast<R>(alpha0) * w[t1].re, ai1 = static_cast<R>(alpha0) * w[t1].im;
    int j = 0;
    for (; j + U <= nv; j += U) {
      Pair2<R> v0[U], v1[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        v0[u] = V[(j + u) * ldv + t];
        v1[u] = V[(j + u) * ldv + t1];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int jj = j + u;
        const R hr = jj < 128 ? hs[2 * jj] : static_cast<R>(h[2 * jj]);
        const R hi = jj < 128 ? hs[2 * jj + 1] : static_cast<R>(h[2 * jj + 1]);
        ar0 = fma_(-hr, v0[u].re, fma_(hi, v0[u].im, ar0));
        ai0 = fma_(-hr, v0[u].im, fma_(-hi, v0[u].re, ai0));
        ar1 = fma_(-hr, v1[u].re, fma_(hi, v1[u].im, ar1));
        ai1 = fma_(-hr, v1[u].im, fma_(-hi, v1[u].re, ai1));
      }
    }
    for (; j < nv; ++j) {
      const Pair2<R> a = V[j * ldv + t], b = V[j * ldv + t1];
      const R hr = j < 128 ? hs[2 * j] : static_cast<R>(h[2 * j]);
      const R hi = j < 128 ? hs[2 * j + 1] : static_cast<R>(h[2 * j + 1]);
      ar0 = fma_(-hr, a.re, fma_(hi, a.im, ar0));
      ai0 = fma_(-hr, a.im, fma_(-hi, a.re, ai0));
      ar1 = fma_(-hr, b.re, fma_(hi, b.im, ar1));
      ai1 = fma_(-hr, b.im, fma_(-hi, b.re, ai1));
    }
    w[t] = Pair2<R>{ar0, ai0};
    if (two) w[t1] = Pair2<R>{ar1, ai1};
  }
}

// y <- beta * y + sum_j c_j V_j    (c given on the device)
template <typename R>
__global__ void multi_combine_kernel(int64_t n, int nv, const Pair2<R>* __restrict__ V, int64_t ldv,
                                     const double* __restrict__ c, double beta, Pair2<R>* __restrict__ y) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    R ar = 0, ai = 0;
    if (beta != 0.0) {
      ar = static_cast<R>(beta) * y[t].re;
      ai = static_cast<R>(beta) * y[t].im;
    }
    for (int j = 0; j < nv; ++j) {
      const Pair2<R> v = V[j * ldv + t];
      const R cr = static_cast<R>(c[2 * j]), ci = static_cast<R>(c[2 * j + 1]);
      ar = fma_(cr, v.re, fma_(-ci, v.im, ar));
      ai = fma_(cr, v.im, fma_(ci, v.re, ai));
    }
    y[t] = Pair2<R>{ar, ai};
  }
}

static int vec_grid(int64_t n) {
  const int64_t b = (n + kVecThreads - 1) / kVecThreads;
  const int64_t cap = 16LL * device_sms();
  return static_cast<int>(b < cap ? (b > 0 ? b : 1) : cap);
}

template <typename R>
cudaError_t launch_multi_axpy(int64_t n, int nv, const void* V, int64_t ldv, const double* h, double alpha0, void* w,
                              cudaStream_t st) {
  const int64_t pairs = (n + 2 * kVecThreads - 1) / (2 * kVecThreads);
  const int64_t cap = 4LL * device_sms();
  const unsigned grid = static_cast<unsigned>(pairs < cap ? (pairs > 0 ? pairs : 1) : cap);
  multi_axpy_kernel<R><<<grid, kVecThreads, 0, st>>>(n, nv, static_cast<const Pair2<R>*>(V), ldv, h, alpha0,
                                                            static_cast<Pair2<R>*>(w));
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_multi_axpy<float>(int64_t, int, const void*, int64_t, const double*, double, void*,
                                              cudaStream_t);
template cudaError_t launch_multi_axpy<double>(int64_t, int, const void*, int64_t, const double*, double, void*,
                                               cudaStream_t);

template <typename R>
cudaError_t launch_multi_combine(int64_t n, int nv, const void* V, int64_t ldv, const double* c, double beta, void* y,
                                 cudaStream_t st) {
  multi_combine_kernel<R><<<vec_grid(n), kVecThreads, 0, st>>>(n, nv, static_cast<const Pair2<R>*>(V), ldv, c, beta,
                                                               static_cast<Pair2<R>*>(y));
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_multi_combine<float>(int64_t, int, const void*, int64_t, const double*, double, void*,
                                                 cudaStream_t);
template cudaError_t launch_multi_combine<double>(int64_t, int, const void*, int64_t, const double*, double, void*,
                                                  cudaStream_t);

// y <- a * x + b * y (real scalars), element types may differ (cast)
template <typename RX, typename RY>
__global__ void axpby_kernel(int64_t n, double a, const Pair2<RX>* x, double b, Pair2<RY>* y) {  // x may alias y
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double r = a * static_cast<double>(x[t].re), i = a * static_cast<double>(x[t].im);
    if (b != 0.0) {
      r += b * static_cast<double>(y[t].re);
      i += b * static_cast<double>(y[t].im);
    }
    y[t] = Pair2<RY>{static_cast<RY>(r), static_cast<RY>(i)};
  }
}

// z = a x + b y with complex a, b (z may alias x or y)
template <typename R>
__global__ void caxpbyz_kernel(int64_t n, R ar, R ai, const Pair2<R>* x, R br, R bi, const Pair2<R>* y,
                               Pair2<R>* z) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const Pair2<R> u = x[t], v = y[t];
    const R re = fma_(ar, u.re, fma_(-ai, u.im, fma_(br, v.re, -bi * v.im)));
    const R im = fma_(ar, u.im, fma_(ai, u.re, fma_(br, v.im, bi * v.re)));
    z[t] = Pair2<R>{re, im};
  }
}
template <typename R>
cudaError_t launch_caxpbyz(int64_t n, double ar, double ai, const void* x, double br, double bi, const void* y,
                           void* z, cudaStream_t st) {
  caxpbyz_kernel<R><<<vec_grid(n), kVecThreads, 0, st>>>(n, static_cast<R>(ar), static_cast<R>(ai),
                                                           static_cast<const Pair2<R>*>(x), static_cast<R>(br),
                                                           static_cast<R>(bi), static_cast<const Pair2<R>*>(y),
                                                           static_cast<Pair2<R>*>(z));
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_caxpbyz<float>(int64_t, double, double, const void*, double, double, const void*, void*,
                                           cudaStream_t);
template cudaError_t launch_caxpbyz<double>(int64_t, double, double, const void*, double, double, const void*, void*,
                                            cudaStream_t);

template <typename RX, typename RY>
cudaError_t launch_axpby(int64_t n, double a, const void* x, double b, void* y, cudaStream_t st) {
  axpby_kernel<RX, RY><<<vec_grid(n), kVecThreads, 0, st>>>(n, a, static_cast<const Pair2<RX>*>(x), b,
                                                            static_cast<Pair2<RY>*>(y));
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_axpby<float, float>(int64_t, double, const void*, double, void*, cudaStream_t);
template cudaError_t launch_axpby<double, double>(int64_t, double, const void*, double, void*, cudaStream_t);
template cudaError_t launch_axpby<float, double>(int64_t, double, const void*, double, void*, cudaStream_t);
template cudaError_t launch_axpby<double, float>(int64_t, double, const void*, double, void*, cudaStream_t);

// y = T x elementwise with the [N][nmax] FP64 diagonal (RHS T a_in)
__global__ void tdiag_mul_kernel(int64_t n_per_rhs, int nrhs, const double* __restrict__ tdiag,
                                 const double* __restrict__ x, double* __restrict__ y) {
  const int64_t total = n_per_rhs * nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t % n_per_rhs;
    const cd v = mkc(tdiag[2 * e], tdiag[2 * e + 1]) * mkc(x[2 * t], x[2 * t + 1]);
    y[2 * t] = v.re;
    y[2 * t + 1] = v.im;
  }
}

cudaError_t launch_tdiag_mul(int64_t n_per_rhs, int nrhs, const double* tdiag, const double* x, double* y,
                             cudaStream_t st) {
  tdiag_mul_kernel<<<vec_grid(n_per_rhs * nrhs), kVecThreads, 0, st>>>(n_per_rhs, nrhs, tdiag, x, y);
  note_launch();
  return cudaGetLastError();
}

// non-finite scan: flag[0] = 1 if any element is NaN or Inf
template <typename R>
__global__ void nonfinite_kernel(int64_t n, const R* __restrict__ v, int* __restrict__ flag) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    if (!isfinite(v[t])) *flag = 1;
  }
}
template <typename R>
cudaError_t launch_nonfinite(int64_t n, const void* v, int* flag, cudaStream_t st) {
  nonfinite_kernel<R><<<vec_grid(n), kVecThreads, 0, st>>>(n, static_cast<const R*>(v), flag);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_nonfinite<float>(int64_t, const void*, int*, cudaStream_t);
template cudaError_t launch_nonfinite<double>(int64_t, const void*, int*, cudaStream_t);

// ---------------------------------------------------------------------------
// far field (App. D): one block per direction
//   g_j = 1/(2 pi) sum_i e^{-i k.r_i} sum_n B_nj(beta) e^{i m alpha} b^i_n
// ---------------------------------------------------------------------------
__global__ void farfield_kernel(int64_t N, int L, double k, const Pos4* __restrict__ pos, const double* __restrict__ b,
                                const double* __restrict__ dirs, double* __restrict__ g) {
  extern __shared__ double fsm[];
  const int nmax = 2 * L * (L + 2);
  double* tb = fsm;  // [nmax][2 j][2 re/im]
  const double beta = dirs[2 * blockIdx.x], alpha = dirs[2 * blockIdx.x + 1];
  double sb, cb, sa, ca;
  sincos(beta, &sb, &cb);
  sincos(alpha, &sa, &ca);
  for (int n = threadIdx.x; n < nmax; n += blockDim.x) {
    int tau, l, m;
    row_decode(n, L, tau, l, m);
    double pi[16], ta[16];
    pi_tau_m(L, m < 0 ? -m : m, cb, sb, pi, ta);
    const cd em = cexp_i(m * alpha);
    for (int j = 1; j <= 2; ++j) {
      const cd v = b_transform(tau, l, m, j, pi[l], ta[l], false) * em;
      tb[(n * 2 + (j - 1)) * 2] = v.re;
      tb[(n * 2 + (j - 1)) * 2 + 1] = v.im;
    }
  }
  __syncthreads();
  const double kx = k * sb * ca, ky = k * sb * sa, kz = k * cb;
  cd g1 = mkc(0.0), g2 = mkc(0.0);
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    const Pos4 r = pos[i];
    cd s1 = mkc(0.0), s2 = mkc(0.0);
    const double* bi = b + i * nmax * 2;
    for (int n = 0; n < nmax; ++n) {
      const cd bn = mkc(bi[2 * n], bi[2 * n + 1]);
      s1 = s1 + mkc(tb[(n * 2) * 2], tb[(n * 2) * 2 + 1]) * bn;
      s2 = s2 + mkc(tb[(n * 2 + 1) * 2], tb[(n * 2 + 1) * 2 + 1]) * bn;
    }
    const cd ph = cexp_i(-(kx * r.x + ky * r.y + kz * r.z));
    g1 = g1 + ph * s1;
    g2 = g2 + ph * s2;
  }
  __shared__ double red[4][32];
  double v[4] = {g1.re, g1.im, g2.re, g2.im};
  for (int q = 0; q < 4; ++q) {
    double x = v[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += red[threadIdx.x][w];
    g[4 * blockIdx.x + threadIdx.x] = s / (2.0 * 3.14159265358979323846);
  }
}

cudaError_t launch_farfield(int64_t N, int L, double k, const void* pos, const double* b, int64_t Nd,
                            const double* dirs, double* g, cudaStream_t st) {
  const int nmax = 2 * L * (L + 2);
  const size_t smem = sizeof(double) * nmax * 4;
  for (int64_t d0 = 0; d0 < Nd; d0 += 65535) {
    const int64_t nd = Nd - d0 < 65535 ? Nd - d0 : 65535;
    farfield_kernel<<<static_cast<unsigned>(nd), 256, smem, st>>>(N, L, k, static_cast<const Pos4*>(pos), b,
                                                                  dirs + 2 * d0, g + 4 * d0);
  }
  note_launch();
  return cudaGetLastError();
}

// overlap check: flag[0] = 1 if some pair overlaps (|r_i - r_j| < R_i + R_j)
__global__ void overlap_kernel(int64_t N, const Pos4* __restrict__ pos, const double* __restrict__ radii,
                               int* __restrict__ flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const Pos4 a = pos[i];
  const double ra = radii[i];
  for (int64_t j = i + 1; j < N; ++j) {
    const Pos4 b = pos[j];
    const double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    const double s = ra + radii[j];
    if (dx * dx + dy * dy + dz * dz < s * s) {
      *flag = 1;
      return;
    }
  }
}

cudaError_t launch_overlap_check(int64_t N, const void* pos, const double* radii, int* flag, cudaStream_t st) {
  const int threads = 128;
  overlap_kernel<<<static_cast<unsigned>((N + threads - 1) / threads), threads, 0, st>>>(
      N, static_cast<const Pos4*>(pos), radii, flag);
  note_launch();
  return cudaGetLastError();
}

}  // namespace celes
