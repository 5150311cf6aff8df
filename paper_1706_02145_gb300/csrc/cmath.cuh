// Small complex-arithmetic helpers and special functions for the FP64 setup
// kernels (Mie coefficients, incident fields, far field).
#pragma once

#include <cuda_runtime.h>

namespace celes {

struct cd {
  double re, im;
};

__host__ __device__ __forceinline__ cd mkc(double r, double i = 0.0) { return cd{r, i}; }
__host__ __device__ __forceinline__ cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cd operator-(cd a) { return cd{-a.re, -a.im}; }
__host__ __device__ __forceinline__ cd operator*(cd a, cd b) {
  return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cd operator*(double s, cd a) { return cd{s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cd operator*(cd a, double s) { return cd{s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cd conj(cd a) { return cd{a.re, -a.im}; }
__host__ __device__ __forceinline__ double abs2(cd a) { return a.re * a.re + a.im * a.im; }
// Smith's algorithm for complex division (avoids overflow of |b|^2)
__host__ __device__ __forceinline__ cd operator/(cd a, cd b) {
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, den = b.re + b.im * r;
    return cd{(a.re + a.im * r) / den, (a.im - a.re * r) / den};
  } else {
    const double r = b.re / b.im, den = b.re * r + b.im;
    return cd{(a.re * r + a.im) / den, (a.im * r - a.re) / den};
  }
}
__host__ __device__ __forceinline__ cd operator/(cd a, double s) { return cd{a.re / s, a.im / s}; }
// i^n for integer n
__host__ __device__ __forceinline__ cd ipow(int n) {
  const int r = ((n % 4) + 4) % 4;
  return r == 0 ? cd{1, 0} : (r == 1 ? cd{0, 1} : (r == 2 ? cd{-1, 0} : cd{0, -1}));
}
__device__ __forceinline__ cd cexp_i(double phase) {
  double s, c;
  sincos(phase, &s, &c);
  return cd{c, s};
}
__device__ __forceinline__ cd csin(cd z) { return cd{sin(z.re) * cosh(z.im), cos(z.re) * sinh(z.im)}; }
__device__ __forceinline__ cd ccos(cd z) { return cd{cos(z.re) * cosh(z.im), -sin(z.re) * sinh(z.im)}; }

// Spherical Bessel functions j_0..j_lmax at complex z by Miller's downward
// recurrence j_{l-1} = (2l+1)/z j_l - j_{l+1}, normalised with the closed
// forms j_0 = sin z / z or j_1 = sin z / z^2 - cos z / z (whichever is larger
// in modulus).  Stable for every l; lmax <= 15.
__device__ inline void sph_jn_c(int lmax, cd z, cd* out) {
  const double az = sqrt(abs2(z));
  int lstart = lmax + 24 + static_cast<int>(az);
  cd jp1 = mkc(0.0), jl = mkc(1e-30);
  for (int l = lstart; l >= 1; --l) {
    const cd jm1 = (static_cast<double>(2 * l + 1) * (jl / z)) - jp1;
    jp1 = jl;
    jl = jm1;
    if (l - 1 <= lmax) out[l - 1] = jl;
    if (l <= lmax) out[l] = jp1;
    if (abs2(jl) > 1e200) {  // rescale to stay in range
      jl = jl * 1e-100;
      jp1 = jp1 * 1e-100;
      for (int q = l - 1; q <= lmax; ++q)
        if (q >= 0) out[q] = out[q] * 1e-100;
    }
  }
  const cd s = csin(z), c = ccos(z);
  const cd j0 = s / z;
  const cd j1 = s / (z * z) - c / z;
  cd scale;
  if (lmax == 0 || abs2(j0) >= abs2(j1)) {
    scale = j0 / out[0];
  } else {
    scale = j1 / out[1];
  }
  for (int l = 0; l <= lmax; ++l) out[l] = out[l] * scale;
}

// Spherical Neumann functions y_0..y_lmax at real x > 0 (upward recurrence,
// stable for y).
__device__ inline void sph_yn_r(int lmax, double x, double* out) {
  double s, c;
  sincos(x, &s, &c);
  out[0] = -c / x;
  if (lmax >= 1) out[1] = -c / (x * x) - s / x;
  for (int l = 1; l < lmax; ++l) out[l + 1] = (2 * l + 1) / x * out[l] - out[l - 1];
}

// Normalised pi_l^m(theta) and tau_l^m(theta) for one m >= 0 and l = m..lmax
// (index l), from the recursions
//   pi_m^m = c_m sin^{m-1}(t),  c_m = prod_{q=1}^{m} sqrt((2q+1)/(2q)) / sqrt(2)
//   pi_{m+1}^m = sqrt(2m+3) cos(t) pi_m^m,
//   pi_l^m = a_lm (cos(t) pi_{l-1}^m - b_lm pi_{l-2}^m)
//   tau_l^m = l cos(t) pi_l^m - sqrt((2l+1)(l^2-m^2)/(2l-1)) pi_{l-1}^m   (m >= 1)
//   tau_l^0 = -sqrt(l(l+1)) sin(t) pi_l^1
// valid at sin(t) = 0.  Entries with l < max(m, 1) are zero.
__device__ inline void pi_tau_m(int lmax, int m, double ct, double st, double* pi, double* tau) {
  for (int l = 0; l <= lmax; ++l) pi[l] = tau[l] = 0.0;
  const int mm = m == 0 ? 1 : m;  // tau_l^0 needs pi_l^1
  double pil[16];
  for (int l = 0; l <= lmax; ++l) pil[l] = 0.0;
  double c = 0.70710678118654752440;
  for (int q = 1; q <= mm; ++q) c *= sqrt((2.0 * q + 1.0) / (2.0 * q));
  double sp = 1.0;
  for (int q = 0; q < mm - 1; ++q) sp *= st;
  if (mm <= lmax) pil[mm] = c * sp;
  if (mm + 1 <= lmax) pil[mm + 1] = sqrt(2.0 * mm + 3.0) * ct * pil[mm];
  for (int l = mm + 2; l <= lmax; ++l) {
    const double a = sqrt((4.0 * l * l - 1.0) / (1.0 * l * l - 1.0 * mm * mm));
    const double b = sqrt(((l - 1.0) * (l - 1.0) - 1.0 * mm * mm) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
    pil[l] = a * (ct * pil[l - 1] - b * pil[l - 2]);
  }
  if (m == 0) {
    for (int l = 1; l <= lmax; ++l) tau[l] = -sqrt(l * (l + 1.0)) * st * pil[l];
  } else {
    for (int l = m; l <= lmax; ++l) {
      pi[l] = pil[l];
      const double prev = l - 1 >= m ? pil[l - 1] : 0.0;
      tau[l] = l * ct * pil[l] - sqrt((2.0 * l + 1.0) * (1.0 * l * l - 1.0 * m * m) / (2.0 * l - 1.0)) * prev;
    }
  }
}

// Transformation coefficient B_nj(beta) (App. A.2) and its dagger (every
// explicit i replaced by -i), from pi_l^|m| and tau_l^|m| at beta.
__device__ __forceinline__ cd b_transform(int tau, int l, int m, int j, double pi_lm, double tau_lm, bool dagger) {
  const double ang = (tau == j) ? tau_lm : m * pi_lm;
  const double nrm = 1.0 / sqrt(2.0 * l * (l + 1.0));
  // -1/i^{l+1} = -(-i)^{l+1};  dagger: -1/(-i)^{l+1} = -i^{l+1}
  const cd pre = dagger ? ipow(l + 1) : ipow(-(l + 1));
  const cd jf = (j == 1) ? (dagger ? cd{0, -1} : cd{0, 1}) : cd{1, 0};
  return (-nrm * ang) * (pre * jf);
}

}  // namespace celes
