// Reflected and transmitted power of a Gaussian-beam simulation (App. D; the
// reflectivity / transmittivity of Sec. 4), FP64.
//
// A plane-wave expansion E = sum_j int dalpha int dbeta sin(beta) g_j Phi_j
// carries the flux P = C sum_j int dalpha int dbeta sin(beta) |g_j|^2 with
// C = 2 pi^2/(omega k mu0) (App. D).  Transmitted power: the forward
// hemisphere of |g_in + g_sca|^2; reflected: the backward hemisphere of
// |g_sca|^2; both divided by the beam's power P_in (closed 1D integral of
// App. D), so C cancels.  g_sca is the far-field amplitude (farfield_kernel)
// and the beam's amplitude is
//   g_in,j = E0 k^2 w^2/(4 pi) cos(b) exp(-w^2 k^2 sin^2(b)/4) e^{-i k.r_G}
//            (cos(a - a_G), sin(a - a_G))
// on b in [0, pi/2].  Quadrature: Gauss-Legendre in beta on each hemisphere,
// trapezoid in alpha.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/celes.h"
#include "cmath.cuh"
#include "kernels.h"

namespace celes {
void gauss_legendre_nodes(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);

namespace {

constexpr int kPowThreads = 256;

// partial[block] = sum over this block's directions of weight * sum_j |g_j (+ g_in,j)|^2
__global__ void power_sum_kernel(int64_t Nd, int64_t nfwd, const double* __restrict__ dirs,
                                 const double* __restrict__ wts, const double* __restrict__ g, double k, double w,
                                 double fx, double fy, double fz, double aG, double e0r, double e0i,
                                 double* __restrict__ partial) {
  __shared__ double red[kPowThreads];
  double s = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Nd; q += (int64_t)gridDim.x * blockDim.x) {
    cd g1 = cd{g[4 * q], g[4 * q + 1]}, g2 = cd{g[4 * q + 2], g[4 * q + 3]};
    if (q < nfwd) {
      const double b = dirs[2 * q], a = dirs[2 * q + 1];
      double sb, cb, sa, ca;
      sincos(b, &sb, &cb);
      sincos(a, &sa, &ca);
      const double amp = k * k * w * w / (4.0 * 3.14159265358979323846264338328) * cb *
                         exp(-(w * k * sb) * (w * k * sb) / 4.0);
      const cd ph = cd{e0r, e0i} * cexp_i(-k * (sb * ca * fx + sb * sa * fy + cb * fz));
      double sd, cdl;
      sincos(a - aG, &sd, &cdl);
      g1 = g1 + (amp * cdl) * ph;
      g2 = g2 + (amp * sd) * ph;
    }
    s += wts[q] * (abs2(g1) + abs2(g2));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kPowThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

}  // namespace
}  // namespace celes

extern "C" int celes_power(celes_ctx* ctx, int rhs, int n_beta, int n_alpha, double* R, double* T) {
  celes::NvtxRange nvtx_range_("celes_power");
  using namespace celes;
  if (!ctx || !R || !T || n_beta < 2 || n_beta > 8192 || n_alpha < 4 || n_alpha > 65536) return CELES_EINVAL;
  CtxView v{};
  int s = ctx_view(ctx, &v);
  if (s) return s;
  if (rhs < 0 || rhs >= v.nrhs) return CELES_EINVAL;
  if (!v.has_b) return CELES_ESTATE;
  const celes_incident& d = v.incidents[rhs];
  if (d.kind != CELES_GAUSSIAN_BEAM) return CELES_EINVAL;  // a plane wave carries infinite power
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(v.device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  // directions: forward hemisphere first, then backward
  const int64_t nh = (int64_t)n_beta * n_alpha, Nd = 2 * nh;
  std::vector<double> dirs(2 * Nd), wts(Nd);
  for (int h = 0; h < 2; ++h) {
    std::vector<double> x, wb;
    gauss_legendre_nodes(n_beta, h == 0 ? 0.0 : 0.5 * M_PI, h == 0 ? 0.5 * M_PI : M_PI, x, wb);
    for (int ib = 0; ib < n_beta; ++ib)
      for (int ia = 0; ia < n_alpha; ++ia) {
        const int64_t q = h * nh + (int64_t)ib * n_alpha + ia;
        dirs[2 * q] = x[ib];
        dirs[2 * q + 1] = 2.0 * M_PI * ia / n_alpha;
        wts[q] = wb[ib] * std::sin(x[ib]) * (2.0 * M_PI / n_alpha);
      }
  }
  // P_in / C = |E0|^2 (k^2 w^2 / (4 pi))^2 2 pi int_0^{pi/2} sin b cos^2 b exp(-w^2 k^2 sin^2 b / 2) db
  double pin = 0.0;
  {
    std::vector<double> x, wb;
    gauss_legendre_nodes(4000, 0.0, 0.5 * M_PI, x, wb);
    const double kw = v.k * d.waist;
    for (size_t q = 0; q < x.size(); ++q) {
      const double sb = std::sin(x[q]), cb = std::cos(x[q]);
      pin += wb[q] * sb * cb * cb * std::exp(-kw * kw * sb * sb / 2.0);
    }
    const double a = v.k * v.k * d.waist * d.waist / (4.0 * M_PI);
    pin *= (d.E0_re * d.E0_re + d.E0_im * d.E0_im) * a * a * 2.0 * M_PI;
  }
  const cudaStream_t st = v.stream;
  const int nblk = 304;
  double *dd = nullptr, *dw = nullptr, *dg = nullptr, *dp = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    if (dd) cudaFree(dd);
    if (dw) cudaFree(dw);
    if (dg) cudaFree(dg);
    if (dp) cudaFree(dp);
  };
  if (cudaMalloc(&dd, sizeof(double) * 2 * Nd) != cudaSuccess || cudaMalloc(&dw, sizeof(double) * Nd) != cudaSuccess ||
      cudaMalloc(&dg, sizeof(double) * 4 * Nd) != cudaSuccess || cudaMalloc(&dp, sizeof(double) * 2 * nblk) != cudaSuccess) {
    cleanup();
    return CELES_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(dd, dirs.data(), sizeof(double) * 2 * Nd, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dw, wts.data(), sizeof(double) * Nd, cudaMemcpyHostToDevice, st);
  const double* b = v.b + (size_t)rhs * v.N * v.nmax * 2;
  if (e == cudaSuccess) e = launch_farfield(v.N, v.L, v.k, v.pos, b, Nd, dd, dg, st);
  if (e == cudaSuccess) {
    // forward hemisphere with the beam, backward without it
    power_sum_kernel<<<nblk, kPowThreads, 0, st>>>(nh, nh, dd, dw, dg, v.k, d.waist, d.focus[0], d.focus[1],
                                                   d.focus[2], d.alpha_G, d.E0_re, d.E0_im, dp);
    power_sum_kernel<<<nblk, kPowThreads, 0, st>>>(nh, 0, dd + 2 * nh, dw + nh, dg + 4 * nh, v.k, d.waist,
                                                   d.focus[0], d.focus[1], d.focus[2], d.alpha_G, d.E0_re, d.E0_im,
                                                   dp + nblk);
    note_launch(2);
    e = cudaGetLastError();
  }
  std::vector<double> hp(2 * nblk, 0.0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), dp, sizeof(double) * 2 * nblk, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return CELES_ECUDA;
  double pf = 0.0, pb = 0.0;
  for (int q = 0; q < nblk; ++q) {
    pf += hp[q];
    pb += hp[nblk + q];
  }
  *T = pf / pin;
  *R = pb / pin;
  return CELES_OK;
}

namespace celes {
namespace {
// s11[ib] = (1 / (2 n_alpha)) sum_alpha sum_j (|g_a,j|^2 + |g_b,j|^2), one block per beta
__global__ void s11_kernel(int n_alpha, const double* __restrict__ ga, const double* __restrict__ gb,
                           double* __restrict__ s11) {
  __shared__ double red[kPowThreads];
  const int64_t base = (int64_t)blockIdx.x * n_alpha;
  double s = 0.0;
  for (int ia = threadIdx.x; ia < n_alpha; ia += blockDim.x) {
    const double* p = ga + 4 * (base + ia);
    const double* q = gb + 4 * (base + ia);
    s += p[0] * p[0] + p[1] * p[1] + p[2] * p[2] + p[3] * p[3] + q[0] * q[0] + q[1] * q[1] + q[2] * q[2] +
         q[3] * q[3];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kPowThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) s11[blockIdx.x] = red[0] / (2.0 * n_alpha);
}
}  // namespace
}  // namespace celes

extern "C" int celes_s11(celes_ctx* ctx, int rhs_a, int rhs_b, const double* betas, int n_beta, int n_alpha,
                         double* s11) {
  celes::NvtxRange nvtx_range_("celes_s11");
  using namespace celes;
  if (!ctx || !betas || !s11 || n_beta < 1 || n_alpha < 1 || n_alpha > 1 << 20) return CELES_EINVAL;
  CtxView v{};
  int s = ctx_view(ctx, &v);
  if (s) return s;
  if (rhs_a < 0 || rhs_a >= v.nrhs || rhs_b < 0 || rhs_b >= v.nrhs) return CELES_EINVAL;
  if (!v.has_b) return CELES_ESTATE;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(v.device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  const int64_t Nd = (int64_t)n_beta * n_alpha;
  std::vector<double> dirs(2 * Nd);
  for (int ib = 0; ib < n_beta; ++ib)
    for (int ia = 0; ia < n_alpha; ++ia) {
      dirs[2 * ((int64_t)ib * n_alpha + ia)] = betas[ib];
      dirs[2 * ((int64_t)ib * n_alpha + ia) + 1] = 2.0 * M_PI * ia / n_alpha;
    }
  const cudaStream_t st = v.stream;
  double *dd = nullptr, *ga = nullptr, *gb = nullptr, *ds = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    if (dd) cudaFree(dd);
    if (ga) cudaFree(ga);
    if (gb) cudaFree(gb);
    if (ds) cudaFree(ds);
  };
  if (cudaMalloc(&dd, sizeof(double) * 2 * Nd) != cudaSuccess || cudaMalloc(&ga, sizeof(double) * 4 * Nd) != cudaSuccess ||
      cudaMalloc(&gb, sizeof(double) * 4 * Nd) != cudaSuccess || cudaMalloc(&ds, sizeof(double) * n_beta) != cudaSuccess) {
    cleanup();
    return CELES_ENOMEM;
  }
  const size_t per = (size_t)v.N * v.nmax * 2;
  cudaError_t e = cudaMemcpyAsync(dd, dirs.data(), sizeof(double) * 2 * Nd, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_farfield(v.N, v.L, v.k, v.pos, v.b + per * rhs_a, Nd, dd, ga, st);
  if (e == cudaSuccess) e = launch_farfield(v.N, v.L, v.k, v.pos, v.b + per * rhs_b, Nd, dd, gb, st);
  if (e == cudaSuccess) {
    s11_kernel<<<n_beta, kPowThreads, 0, st>>>(n_alpha, ga, gb, ds);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(s11, ds, sizeof(double) * n_beta, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  return e == cudaSuccess ? CELES_OK : CELES_ECUDA;
}
