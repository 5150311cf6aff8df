// Electric field at arbitrary points (Sec. 2.1; the near-field maps of the
// paper's examples), FP64:
//   scattered  E_s(r) = sum_i sum_n b^i_n Psi^(3)_n(r - r_i)
//   incident   plane wave E0 Phi_pol(alpha, beta; r) (App. A.1), or the
//              Gaussian beam's angular spectrum integral (App. C), evaluated
//              with the same beta range and Gauss-Legendre nodes as its
//              expansion coefficients and a trapezoid rule in alpha
//   total      E_s + E_in
// Psi^(3) in the form of App. A.1 with the normalised Legendre functions
// P_l^m, pi_l^m = P_l^m / sin(theta) and tau_l^m = dP_l^m/dtheta (no
// Condon-Shortley phase).  The expansion about sphere i holds outside that
// sphere only, so points inside a sphere get NaN in the scattered and total
// fields (the internal field is not part of this call).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/celes.h"
#include "cmath.cuh"
#include "coupling_kernel.cuh"
#include "kernels.h"

namespace celes {
namespace {

constexpr int kNfThreads = 128;

// normalised P_l^0(cos t), l = 0..lmax
__device__ inline void legendre_p0(int lmax, double ct, double* p) {
  p[0] = 0.70710678118654752440;
  if (lmax >= 1) p[1] = sqrt(3.0) * ct * p[0];
  for (int l = 2; l <= lmax; ++l) {
    const double a = sqrt((4.0 * l * l - 1.0) / (1.0 * l * l));
    const double b = sqrt(((l - 1.0) * (l - 1.0)) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
    p[l] = a * (ct * p[l - 1] - b * p[l - 2]);
  }
}

__global__ void __launch_bounds__(kNfThreads)
    nearfield_scattered_kernel(int64_t Np, const double* __restrict__ pts, int64_t N, int L, double k,
                               const Pos4* __restrict__ pos, const double* __restrict__ radii,
                               const double* __restrict__ b, double* __restrict__ E) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Np) return;
  const int NH = L * (L + 2), nmax = 2 * NH;
  const double px = pts[3 * t], py = pts[3 * t + 1], pz = pts[3 * t + 2];
  cd Ex = mkc(0.0), Ey = mkc(0.0), Ez = mkc(0.0);
  bool inside = false;
  double pi[16], tau[16], p0[16];
  cd h[16];
  for (int64_t i = 0; i < N; ++i) {
    const Pos4 c = pos[i];
    const double dx = px - c.x, dy = py - c.y, dz = pz - c.z;
    const double d2 = dx * dx + dy * dy + dz * dz;
    const double R = radii[i];
    if (d2 < R * R) {
      inside = true;
      break;
    }
    const double d = sqrt(d2);
    const double x = k * d;
    // h_l(x), l = 0..L (upward recurrence, stable for the outgoing function)
    const cd e = cexp_i(x);
    h[0] = cd{0.0, -1.0} * e / x;                        // -i e^{ix}/x
    h[1] = e * cd{-1.0 / x, -1.0 / (x * x)};             // e^{ix} (-1/x - i/x^2)
    for (int l = 1; l < L; ++l) h[l + 1] = (2.0 * l + 1.0) / x * h[l] - h[l - 1];
    const double rho = sqrt(dx * dx + dy * dy);
    const double ct = dz / d, st = rho / d;
    const double cph = rho > 0.0 ? dx / rho : 1.0, sph = rho > 0.0 ? dy / rho : 0.0;
    // unit vectors
    const double er[3] = {st * cph, st * sph, ct};
    const double et[3] = {ct * cph, ct * sph, -st};
    const double ep[3] = {-sph, cph, 0.0};
    legendre_p0(L, ct, p0);
    const double* bi = b + (size_t)i * nmax * 2;
    cd emp = mkc(1.0);  // e^{i |m| phi}
    for (int am = 0; am <= L; ++am) {
      if (am > 0) emp = emp * cd{cph, sph};
      pi_tau_m(L, am, ct, st, pi, tau);
      for (int sgn = 0; sgn < (am == 0 ? 1 : 2); ++sgn) {
        const int m = sgn == 0 ? am : -am;
        const cd eim = sgn == 0 ? emp : conj(emp);
        for (int l = (am > 0 ? am : 1); l <= L; ++l) {
          const double P = am == 0 ? p0[l] : st * pi[l];
          const cd pref = (1.0 / sqrt(2.0 * l * (l + 1.0))) * eim;
          const int r = l * (l + 1) - 1 + m;
          const cd b1 = cd{bi[2 * r], bi[2 * r + 1]};
          const cd b2 = cd{bi[2 * (NH + r)], bi[2 * (NH + r) + 1]};
          const cd hl = h[l];
          const cd dxh = h[l - 1] - (static_cast<double>(l) / x) * hl;  // d/dx (x h_l) / x
          // Psi_1 = pref h_l (i m pi e_t - tau e_p)
          const cd c1 = b1 * pref * hl;
          const cd a_t1 = c1 * cd{0.0, m * pi[l]};
          const cd a_p1 = -tau[l] * c1;
          // Psi_2 = pref (l(l+1) h_l/x P e_r + dxh (tau e_t + i m pi e_p))
          const cd c2 = b2 * pref;
          const cd a_r2 = c2 * ((l * (l + 1.0) * P / x) * hl);
          const cd a_t2 = c2 * (tau[l] * dxh);
          const cd a_p2 = c2 * (dxh * cd{0.0, m * pi[l]});
          const cd Ar = a_r2, At = a_t1 + a_t2, Ap = a_p1 + a_p2;
          Ex = Ex + er[0] * Ar + et[0] * At + ep[0] * Ap;
          Ey = Ey + er[1] * Ar + et[1] * At + ep[1] * Ap;
          Ez = Ez + er[2] * Ar + et[2] * At + ep[2] * Ap;
        }
      }
    }
  }
  double* o = E + 6 * t;
  if (inside) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int q = 0; q < 6; ++q) o[q] = nan;
    return;
  }
  o[0] = Ex.re;
  o[1] = Ex.im;
  o[2] = Ey.re;
  o[3] = Ey.im;
  o[4] = Ez.re;
  o[5] = Ez.im;
}

// E += E0 e^{i k.r} e_pol(alpha, beta)
__global__ void nearfield_plane_kernel(int64_t Np, const double* __restrict__ pts, double k, double beta,
                                       double alpha, int pol, double e0r, double e0i, double* __restrict__ E) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Np) return;
  double sb, cb, sa, ca;
  sincos(beta, &sb, &cb);
  sincos(alpha, &sa, &ca);
  const double kx = k * sb * ca, ky = k * sb * sa, kz = k * cb;
  const cd ph = cexp_i(kx * pts[3 * t] + ky * pts[3 * t + 1] + kz * pts[3 * t + 2]) * cd{e0r, e0i};
  const double e[3] = {pol == 1 ? -sa : cb * ca, pol == 1 ? ca : cb * sa, pol == 1 ? 0.0 : -sb};
  double* o = E + 6 * t;
  for (int q = 0; q < 3; ++q) {
    o[2 * q] += ph.re * e[q];
    o[2 * q + 1] += ph.im * e[q];
  }
}

// E += E0 (k w)^2/(4 pi) int_0^bmax dbeta int_0^2pi dalpha sin(b) cos(b)
//        exp(-(w k sin b)^2/4) e^{i k(b,a).(r - r_G)} (cos(a - aG) e_a + sin(a - aG) e_b)
__global__ void nearfield_gauss_kernel(int64_t Np, const double* __restrict__ pts, double k, double w,
                                       double fx, double fy, double fz, double aG, double e0r, double e0i,
                                       int nb, const double* __restrict__ bnode, const double* __restrict__ bw,
                                       double* __restrict__ E) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Np) return;
  const double rx = pts[3 * t] - fx, ry = pts[3 * t + 1] - fy, rz = pts[3 * t + 2] - fz;
  const double rho = sqrt(rx * rx + ry * ry);
  // trapezoid in alpha is exact to rounding once the number of nodes exceeds
  // the band limit k rho sin(beta) + 1 by a margin
  const int na = 2 * (static_cast<int>(k * rho) + 40);
  const double da = 6.283185307179586476925286766559 / na;
  cd Ex = mkc(0.0), Ey = mkc(0.0), Ez = mkc(0.0);
  for (int ib = 0; ib < nb; ++ib) {
    double sb, cb;
    sincos(bnode[ib], &sb, &cb);
    const double g = sb * cb * exp(-(w * k * sb) * (w * k * sb) / 4.0) * bw[ib] * da;
    if (g == 0.0) continue;
    for (int ia = 0; ia < na; ++ia) {
      double sa, ca;
      sincos(ia * da, &sa, &ca);
      double sd, cdl;
      sincos(ia * da - aG, &sd, &cdl);
      const cd ph = g * cexp_i(k * (sb * ca * rx + sb * sa * ry + cb * rz));
      const double vx = cdl * (-sa) + sd * (cb * ca);
      const double vy = cdl * ca + sd * (cb * sa);
      const double vz = sd * (-sb);
      Ex = Ex + vx * ph;
      Ey = Ey + vy * ph;
      Ez = Ez + vz * ph;
    }
  }
  const cd s = cd{e0r, e0i} * ((k * w) * (k * w) / (4.0 * 3.14159265358979323846264338328));
  Ex = s * Ex;
  Ey = s * Ey;
  Ez = s * Ez;
  double* o = E + 6 * t;
  o[0] += Ex.re;
  o[1] += Ex.im;
  o[2] += Ey.re;
  o[3] += Ey.im;
  o[4] += Ez.re;
  o[5] += Ez.im;
}

inline unsigned nblocks(int64_t n) { return static_cast<unsigned>((n + kNfThreads - 1) / kNfThreads); }

}  // namespace

// Gauss-Legendre nodes and weights on [a, b] (the rule of the Gaussian-beam coefficients)
void gauss_legendre_nodes(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);

}  // namespace celes

extern "C" int celes_nearfield(celes_ctx* ctx, const double* points, int64_t Np, int rhs, int what, double* E) {
  celes::NvtxRange nvtx_range_("celes_nearfield");
  using namespace celes;
  if (!ctx || Np < 0 || (Np > 0 && (!points || !E)) || what < 0 || what > 2) return CELES_EINVAL;
  CtxView v{};
  int s = ctx_view(ctx, &v);
  if (s) return s;
  if (rhs < 0 || rhs >= v.nrhs) return CELES_EINVAL;
  if (what != 1 && !v.has_b) return CELES_ESTATE;
  if (Np == 0) return CELES_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(v.device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  const cudaStream_t st = v.stream;
  double *dp = nullptr, *dE = nullptr, *dn = nullptr, *dw = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    if (dp) cudaFree(dp);
    if (dE) cudaFree(dE);
    if (dn) cudaFree(dn);
    if (dw) cudaFree(dw);
  };
  if (cudaMalloc(&dp, sizeof(double) * 3 * Np) != cudaSuccess || cudaMalloc(&dE, sizeof(double) * 6 * Np) != cudaSuccess) {
    cleanup();
    return CELES_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(dp, points, sizeof(double) * 3 * Np, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dE, 0, sizeof(double) * 6 * Np, st);
  if (e != cudaSuccess) {
    cleanup();
    return CELES_ECUDA;
  }
  if (what != 1) {
    const double* b = v.b + (size_t)rhs * v.N * v.nmax * 2;
    nearfield_scattered_kernel<<<nblocks(Np), kNfThreads, 0, st>>>(Np, dp, v.N, v.L, v.k,
                                                                   static_cast<const Pos4*>(v.pos), v.radii, b, dE);
    note_launch();
  }
  if (what != 0) {
    const celes_incident& d = v.incidents[rhs];
    if (d.kind == CELES_PLANE_WAVE) {
      nearfield_plane_kernel<<<nblocks(Np), kNfThreads, 0, st>>>(Np, dp, v.k, d.beta, d.alpha, d.pol, d.E0_re,
                                                                 d.E0_im, dE);
    } else {
      const int nb = d.n_beta > 0 ? d.n_beta : 128;
      const double aa = std::pow(d.waist * v.k, 2) / 4.0;
      const double s2 = 39.2 / aa;
      const double bmax = s2 >= 1.0 ? M_PI / 2 : std::asin(std::sqrt(s2));
      std::vector<double> hx, hw;
      gauss_legendre_nodes(nb, 0.0, bmax, hx, hw);
      if (cudaMalloc(&dn, sizeof(double) * nb) != cudaSuccess || cudaMalloc(&dw, sizeof(double) * nb) != cudaSuccess) {
        cleanup();
        return CELES_ENOMEM;
      }
      if (cudaMemcpyAsync(dn, hx.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(dw, hw.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cleanup();
        return CELES_ECUDA;
      }
      nearfield_gauss_kernel<<<nblocks(Np), kNfThreads, 0, st>>>(Np, dp, v.k, d.waist, d.focus[0], d.focus[1],
                                                                 d.focus[2], d.alpha_G, d.E0_re, d.E0_im, nb, dn, dw,
                                                                 dE);
    }
    note_launch();
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(E, dE, sizeof(double) * 6 * Np, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  return e == cudaSuccess ? CELES_OK : CELES_ECUDA;
}
