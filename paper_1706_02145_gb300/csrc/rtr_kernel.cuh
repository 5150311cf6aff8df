// Coupling matvec y_i = sum_{j != i} W^{ij} x_j by rotation-translation-
// rotation (see rtr_tables.cuh for the factorisation W = D^H W_z D).
//
// Per ordered pair (i, j), one thread (the receiver's):
//   1. geometry: k|d| and its phase (FP32 kernel: float-float arithmetic;
//      FP64 kernel: FP64), h_p(k|d|), cos/sin(theta/2), e^{i m phi}
//   2. x'+-[l, mu] = sum_m R^l_{mu m}(theta) e^{i m phi} x+-[l, m]
//   3. y'+-[l, mu] = sum_{l'} (A_z +- i B_z)[l, l', mu] x'+-[l', mu]
//      (built once for mu >= 0 and reused, B sign flipped, for -mu)
//   4. y+-[l, m] += e^{-i m phi} sum_mu R^l_{mu m}(theta) y'+-[l, mu]
// with x+- = x_1 +- x_2 (the tau structure [[A, B], [B, A]] of W, App. A.2).
// All coefficients (Wigner-d sums, axial a5/b5 terms) are compile-time
// immediates; one code stream serves every warp.  Per pair the thread does
// O(L^3) work instead of the O(L^4) of the direct per-entry evaluation.
#pragma once

#include <cooperative_groups.h>

#include <type_traits>

#include "coupling_kernel.cuh"
#include "rtr_tables.cuh"
#include "kernels.h"

namespace celes {
namespace rtr {

// FP32 rotations (steps 2 and 4) on the packed two-lane FMA of sm_100+
// (__ffma2_rn, per lane the rounding of fmaf: results are bit-identical to the
// scalar form).  It halves the issue slots of the rotations, which dominate
// the instruction stream: N = 10 000 matvec 12.4 -> 10.4 ms at lmax 4, 5.65 ->
// 5.17 ms at lmax 3.  At lmax 5 ptxas then moves the rotated coefficients to
// the stack (8.7 vs 4.1 ms at N = 4000), so lmax 5 keeps the scalar form.
template <int L, typename R>
constexpr bool kPacked = std::is_same<R, float>::value && L <= 4;
// launch-shape option bits of the pair code: 1 = the x+ phase multiply on the
// packed FMA, 2 = packed rotations at every lmax (lmax 5 with x' and y' in
// shared memory has the registers for them)
template <int L, typename R, int OPT>
constexpr bool kPackedRot = std::is_same<R, float>::value && (L <= 4 || (OPT & 2) != 0);

template <typename R>
struct alignas(4 * sizeof(R)) Quad4 {
  R x, y, z, w;
};

template <int L, typename R>
struct Geom {
  R hre[2 * L + 1], him[2 * L + 1];
  R cp[2 * L + 1], sp[2 * L + 1];  // powers of cos(theta/2), sin(theta/2)
  R ere[L + 1], eim[L + 1];
};

// ---- FP32 pair geometry without FP64 arithmetic ----------------------------
// Positions are scaled by k and split into float pairs (hi + lo, 48
// significant bits).  Per pair, k|d| is formed with error-free float
// transformations (two-sum and fma-based two-product, Knuth / Dekker) to about
// 2^-44 relative, then reduced mod pi/2 with an exact fma (the product of an
// integer quadrant count and the float nearest pi/2 has no bits below 2^-23),
// so the phase e^{i k|d|} keeps FP32 accuracy at any cluster size while the
// FP64 pipe (1/64 of the FP32 rate on this part) stays idle.
struct alignas(16) PosFF {
  float xh, yh, zh, ph;
  float xl, yl, zl, pl;
};

static_assert(sizeof(PosFF) == sizeof(Pos4), "the source tile holds either form");

__device__ __forceinline__ PosFF split_pos(const Pos4& p, double k) {
  const double x = k * p.x, y = k * p.y, z = k * p.z;
  PosFF o;
  o.xh = static_cast<float>(x);
  o.yh = static_cast<float>(y);
  o.zh = static_cast<float>(z);
  o.xl = static_cast<float>(x - static_cast<double>(o.xh));
  o.yl = static_cast<float>(y - static_cast<double>(o.yh));
  o.zl = static_cast<float>(z - static_cast<double>(o.zh));
  o.ph = o.pl = 0.0f;
  return o;
}

// s + e == a - b exactly (two-sum of a and -b)
__device__ __forceinline__ void two_diff(float a, float b, float& s, float& e) {
  s = __fsub_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fsub_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fadd_rn(b, bb));
}
// s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// sin and cos of q pi/2 + y, |y| <= pi/4 (+ rounding): Taylor series to y^9 /
// y^10 (truncation below 2e-9), quadrant q mod 4 selects signs and the swap
__device__ __forceinline__ void sincos_quadrant(float y, int iq, float& s, float& c) {
  const float y2 = y * y;
  float ps = fma_(y2, 1.0f / 362880.0f, -1.0f / 5040.0f);
  ps = fma_(y2, ps, 1.0f / 120.0f);
  ps = fma_(y2, ps, -1.0f / 6.0f);
  const float sr = fma_(y * y2, ps, y);
  float pc = fma_(y2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
  pc = fma_(y2, pc, -1.0f / 720.0f);
  pc = fma_(y2, pc, 1.0f / 24.0f);
  pc = fma_(y2, pc, -0.5f);
  const float cr = fma_(y2, pc, 1.0f);
  const float s0 = (iq & 1) ? cr : sr;
  const float c0 = (iq & 1) ? sr : cr;
  s = (iq & 2) ? -s0 : s0;
  c = ((iq + 1) & 2) ? -c0 : c0;
}

template <int L, typename R>
__device__ __forceinline__ void geometry_angles_t(R ct, R st, R cph, R sph, Geom<L, R>& g);
template <int L>
__device__ __forceinline__ void geometry_angles(float ct, float st, float cph, float sph, Geom<L, float>& g) {
  geometry_angles_t<L, float>(ct, st, cph, sph, g);
}

// the few scalars every table of a pair derives from
struct GeomS {
  float ix, sn, cs;        // 1/(k d), sin(k d), cos(k d)
  float ct, st, cph, sph;  // cos/sin theta, cos/sin phi of d
};

// h_p(k d), p = 0..2L (closed forms of h_0, h_1 and upward recurrence)
template <int L>
__device__ __forceinline__ void fill_hankel(const GeomS& q, Geom<L, float>& g) {
  constexpr int PM = 2 * L;
  const float ix = q.ix, sn = q.sn, cs = q.cs;
  g.hre[0] = sn * ix;
  g.him[0] = -cs * ix;
  g.hre[1] = -ix * fma_(-sn, ix, cs);
  g.him[1] = -ix * fma_(cs, ix, sn);
#pragma unroll
  for (int p = 1; p < PM; ++p) {
    const float c = static_cast<float>(2 * p + 1) * ix;
    g.hre[p + 1] = fma_(c, g.hre[p], -g.hre[p - 1]);
    g.him[p + 1] = fma_(c, g.him[p], -g.him[p - 1]);
  }
}

template <int L>
__device__ __forceinline__ GeomS geometry_ff_scalars(const PosFF& a, const PosFF& b);

template <int L>
__device__ __forceinline__ void geometry_ff(const PosFF& a, const PosFF& b, Geom<L, float>& g) {
  const GeomS q = geometry_ff_scalars<L>(a, b);
  fill_hankel<L>(q, g);
  geometry_angles<L>(q.ct, q.st, q.cph, q.sph, g);
}

template <int L>
__device__ __forceinline__ GeomS geometry_ff_scalars(const PosFF& a, const PosFF& b) {
  // k (r_a - r_b) per axis as s + e (unnormalised; |e| << |s| or s == 0)
  float sx, ex, sy, ey, sz, ez;
  two_diff(a.xh, b.xh, sx, ex);
  two_diff(a.yh, b.yh, sy, ey);
  two_diff(a.zh, b.zh, sz, ez);
  ex = __fadd_rn(ex, __fsub_rn(a.xl, b.xl));
  ey = __fadd_rn(ey, __fsub_rn(a.yl, b.yl));
  ez = __fadd_rn(ez, __fsub_rn(a.zl, b.zl));
  // (k d)^2 = sum (s + e)^2 = sum s^2 (exact two-products) + e (2 s + e)
  const float px = __fmul_rn(sx, sx), py = __fmul_rn(sy, sy), pz = __fmul_rn(sz, sz);
  float lo = __fadd_rn(__fadd_rn(__fmaf_rn(sx, sx, -px), __fmaf_rn(sy, sy, -py)), __fmaf_rn(sz, sz, -pz));
  lo = __fmaf_rn(ex, __fmaf_rn(2.0f, sx, ex), lo);
  lo = __fmaf_rn(ey, __fmaf_rn(2.0f, sy, ey), lo);
  lo = __fmaf_rn(ez, __fmaf_rn(2.0f, sz, ez), lo);
  float S, E1, S2, E2;
  two_sum(px, py, S, E1);
  two_sum(S, pz, S2, E2);
  lo = __fadd_rn(lo, __fadd_rn(E1, E2));
  // k d = r + delta: one Newton correction of the FP32 square root
  const float rinv = rsqrtf(S2);
  const float r = __fmul_rn(S2, rinv);
  const float rr = __fmul_rn(r, r);
  const float rre = __fmaf_rn(r, r, -rr);
  const float resid = __fadd_rn(__fsub_rn(__fsub_rn(S2, rr), rre), lo);
  const float delta = __fmul_rn(resid, 0.5f * rinv);
  // phase: k d = n pi/2 + y
  constexpr double HALF_PI = 1.5707963267948966192313216916398;
  constexpr float H1 = static_cast<float>(HALF_PI);
  constexpr float H2 = static_cast<float>(HALF_PI - static_cast<double>(H1));
  const float n = rintf(__fmul_rn(r, static_cast<float>(1.0 / HALF_PI)));
  float y = __fmaf_rn(-n, H1, r);  // exact
  y = __fadd_rn(y, __fmaf_rn(-n, H2, delta));
  float sn, cs;
  sincos_quadrant(y, static_cast<int>(n) & 3, sn, cs);
  const float kd = __fadd_rn(r, delta);
  GeomS q;
  q.ix = 1.0f / kd;
  q.sn = sn;
  q.cs = cs;
  const float dxf = __fadd_rn(sx, ex), dyf = __fadd_rn(sy, ey), dzf = __fadd_rn(sz, ez);
  const float rho = sqrtf(fma_(dxf, dxf, dyf * dyf));
  q.ct = fminf(1.0f, fmaxf(-1.0f, dzf * rinv));
  q.st = fminf(1.0f, rho * rinv);
  const float ir = rho > 0.0f ? 1.0f / rho : 0.0f;
  q.cph = rho > 0.0f ? dxf * ir : 1.0f;
  q.sph = dyf * ir;
  return q;
}

// FP64 pair geometry (the FP64 kernel)
template <int L, typename R>
__device__ __forceinline__ void geometry(double dx, double dy, double dz, double k, Geom<L, R>& g) {
  static_assert(sizeof(R) == 8, "the FP32 kernel uses geometry_ff");
  constexpr int PM = 2 * L;
  const double d2 = fma_(dx, dx, fma_(dy, dy, dz * dz));
  const double d = sqrt(d2);
  const double kd = k * d;
  const double TWO_PI = 6.283185307179586476925286766559;
  const double ph = fma_(-rint(kd * (1.0 / TWO_PI)), TWO_PI, kd);
  double sn, cs;
  sincos(ph, &sn, &cs);
  const double ix = 1.0 / kd;
  g.hre[0] = sn * ix;
  g.him[0] = -cs * ix;
  g.hre[1] = -ix * fma_(-sn, ix, cs);
  g.him[1] = -ix * fma_(cs, ix, sn);
#pragma unroll
  for (int p = 1; p < PM; ++p) {
    const double a = static_cast<double>(2 * p + 1) * ix;
    g.hre[p + 1] = fma_(a, g.hre[p], -g.hre[p - 1]);
    g.him[p + 1] = fma_(a, g.him[p], -g.him[p - 1]);
  }
  const double id = 1.0 / d;
  const double rho = sqrt(fma_(dx, dx, dy * dy));
  const double ct = dz * id;
  const double st = rho * id;
  const double ir = rho > 0.0 ? 1.0 / rho : 0.0;
  const double cph = rho > 0.0 ? dx * ir : 1.0;
  const double sph = dy * ir;
  geometry_angles_t<L, R>(ct, st, cph, sph, g);
}

// half angles, their powers and e^{i m phi}
template <int L, typename R>
__device__ __forceinline__ void geometry_angles_t(R ct, R st, R cph, R sph, Geom<L, R>& g) {
  constexpr int PM = 2 * L;
  // half angles without cancellation: c = sqrt((1+ct)/2), s = st/(2c) for
  // ct >= 0, and the mirror formulas otherwise
  R c, s;
  if (ct >= static_cast<R>(0)) {
    c = sqrt(static_cast<R>(0.5) * (static_cast<R>(1) + ct));
    s = static_cast<R>(0.5) * st / c;
  } else {
    s = sqrt(static_cast<R>(0.5) * (static_cast<R>(1) - ct));
    c = static_cast<R>(0.5) * st / s;
  }
  g.cp[0] = static_cast<R>(1);
  g.sp[0] = static_cast<R>(1);
#pragma unroll
  for (int q = 1; q <= PM; ++q) {
    g.cp[q] = g.cp[q - 1] * c;
    g.sp[q] = g.sp[q - 1] * s;
  }
  g.ere[0] = static_cast<R>(1);
  g.eim[0] = static_cast<R>(0);
#pragma unroll
  for (int m = 1; m <= L; ++m) {
    g.ere[m] = fma_(g.ere[m - 1], cph, -g.eim[m - 1] * sph);
    g.eim[m] = fma_(g.ere[m - 1], sph, g.eim[m - 1] * cph);
  }
}

// ---- Wigner-d canonical entries of degree l --------------------------------
template <int l, int T, typename R>
__device__ __forceinline__ void dterm(const R* q, R& acc) {
  constexpr R C = static_cast<R>(DTerm<l, T>::c);
  acc = fma_(C, q[DTerm<l, T>::j], acc);
}
template <int l, int T0, typename R, int... K>
__device__ __forceinline__ R dsum(const R* q, std::integer_sequence<int, K...>) {
  R acc = static_cast<R>(0);
  (dterm<l, T0 + K>(q, acc), ...);
  return acc;
}
template <int l, typename R, int... C>
__device__ __forceinline__ void dcanon(const R* q, R* dv, std::integer_sequence<int, C...>) {
  ((dv[C] = dsum<l, DCanon<l, C>::t0>(q, std::make_integer_sequence<int, DCanon<l, C>::t1 - DCanon<l, C>::t0>{})),
   ...);
}
template <int L, int l, typename R>
__device__ __forceinline__ void dmatrix(const Geom<L, R>& g, R* dv) {
  R q[2 * l + 1];
#pragma unroll
  for (int j = 0; j <= 2 * l; ++j) q[j] = g.cp[2 * l - j] * g.sp[j];
  dcanon<l, R>(q, dv, std::make_integer_sequence<int, DCount<l>::ncanon>{});
}

// row index of (l, m) inside one polarisation block
template <int l, int m>
struct Row {
  static constexpr int r = l * (l + 1) - 1 + m;
};

// ---- step 2: x'[l, MU] = sum_M R_{MU,M} e^{i M phi} x[l, M] ----------------
// x~ (rotated about z) of degree l held in xt[2][2l+1][2]
template <int L, int l, int MU, int OPT, typename R, typename XV, int... MI>
__device__ __forceinline__ void rot_fwd_row(const R* dv, const R (&xt)[2][2 * l + 1][2], XV& xp,
                                            std::integer_sequence<int, MI...>) {
  constexpr int NH = L * (L + 2);
  R a0 = 0, a1 = 0, b0 = 0, b1 = 0;
  if constexpr (kPackedRot<L, R, OPT>) {
    // (re, im) of one complex value per packed FMA, same rounding as fma_
    float2 a = make_float2(0.0f, 0.0f), b = a;
    (
        [&] {
          constexpr int M = MI - l;
          using RA = RAt<l, MU, M>;
          const float w = RA::sign > 0 ? dv[RA::id] : -dv[RA::id];
          const float2 ww = make_float2(w, w);
          a = __ffma2_rn(ww, make_float2(xt[0][MI][0], xt[0][MI][1]), a);
          b = __ffma2_rn(ww, make_float2(xt[1][MI][0], xt[1][MI][1]), b);
        }(),
        ...);
    a0 = a.x;
    a1 = a.y;
    b0 = b.x;
    b1 = b.y;
  } else {
    (
        [&] {
          constexpr int M = MI - l;
          using RA = RAt<l, MU, M>;
          const R w = RA::sign > 0 ? dv[RA::id] : -dv[RA::id];
          a0 = fma_(w, xt[0][MI][0], a0);
          a1 = fma_(w, xt[0][MI][1], a1);
          b0 = fma_(w, xt[1][MI][0], b0);
          b1 = fma_(w, xt[1][MI][1], b1);
        }(),
        ...);
  }
  constexpr int r = Row<l, MU>::r;
  xp(2 * r) = a0;
  xp(2 * r + 1) = a1;
  xp(2 * (NH + r)) = b0;
  xp(2 * (NH + r) + 1) = b1;
}

// PP (packed phase): the x+ half's e^{i m phi} multiply on the packed
// two-lane FMA, which moves work from the scalar half of the FP32 lanes (that
// carries the axial entries, the axial apply and the phases) to the half that
// carries the packed rotations; an autotuner candidate (ConfigAlt at lmax 4)
template <int L, int l, int OPT, typename R, typename XV, int... MUI>
__device__ __forceinline__ void rot_fwd_block(const Geom<L, R>& g, const Pair2<R>* __restrict__ xs, XV& xp,
                                              std::integer_sequence<int, MUI...>) {
  constexpr int NH = L * (L + 2);
  R dv[DCount<l>::ncanon];
  dmatrix<L, l>(g, dv);
  R xt[2][2 * l + 1][2];
#pragma unroll
  for (int mi = 0; mi <= 2 * l; ++mi) {
    const int m = mi - l;
    const int am = m < 0 ? -m : m;
    const R er = g.ere[am];
    const R ei = m < 0 ? -g.eim[am] : g.eim[am];
    const int r = l * (l + 1) - 1 + m;
    const Pair2<R> xa = xs[r], xb = xs[NH + r];
    if constexpr ((OPT & 1) != 0 && kPackedRot<L, R, OPT>) {
      const float2 t = __fmul2_rn(make_float2(xa.im, xa.im), make_float2(-ei, er));
      const float2 u = __ffma2_rn(make_float2(xa.re, xa.re), make_float2(er, ei), t);
      xt[0][mi][0] = u.x;
      xt[0][mi][1] = u.y;
    } else {
      xt[0][mi][0] = fma_(xa.re, er, -xa.im * ei);
      xt[0][mi][1] = fma_(xa.re, ei, xa.im * er);
    }
    xt[1][mi][0] = fma_(xb.re, er, -xb.im * ei);
    xt[1][mi][1] = fma_(xb.re, ei, xb.im * er);
  }
  (rot_fwd_row<L, l, MUI - l, OPT>(dv, xt, xp, std::make_integer_sequence<int, 2 * l + 1>{}), ...);
}

template <int L, int OPT, typename R, typename XV, int... LI>
__device__ __forceinline__ void rot_fwd(const Geom<L, R>& g, const Pair2<R>* __restrict__ xs, XV& xp,
                                        std::integer_sequence<int, LI...>) {
  (rot_fwd_block<L, LI + 1, OPT>(g, xs, xp, std::make_integer_sequence<int, 2 * (LI + 1) + 1>{}), ...);
}

// ---- step 3: axial translation --------------------------------------------
template <int L, int MU, int LO, int LI, int T, typename R>
__device__ __forceinline__ void ax_a(const Geom<L, R>& g, R& ar, R& ai) {
  using A = AxialA<L, MU, LO, LI, T>;
  constexpr R C = static_cast<R>(A::c);
  ar = fma_(C, g.hre[A::p], ar);
  ai = fma_(C, g.him[A::p], ai);
}
template <int L, int MU, int LO, int LI, int T, typename R>
__device__ __forceinline__ void ax_b(const Geom<L, R>& g, R& br, R& bi) {
  using B = AxialB<L, MU, LO, LI, T>;
  constexpr R C = static_cast<R>(B::c);
  br = fma_(C, g.hre[B::p], br);
  bi = fma_(C, g.him[B::p], bi);
}
template <int L, int MU, int LO, int LI, typename R, int... KA, int... KB>
__device__ __forceinline__ void ax_entry(const Geom<L, R>& g, R& ar, R& ai, R& br, R& bi,
                                         std::integer_sequence<int, KA...>, std::integer_sequence<int, KB...>) {
  (ax_a<L, MU, LO, LI, KA>(g, ar, ai), ...);
  (ax_b<L, MU, LO, LI, KB>(g, br, bi), ...);
}

template <typename R>
__device__ __forceinline__ void cmac(R& yr, R& yi, R wr, R wi, R xr, R xi) {
  yr = fma_(wr, xr, fma_(-wi, xi, yr));
  yi = fma_(wr, xi, fma_(wi, xr, yi));
}

// one (l, l') entry of the axial block for +MU (and the mirrored -MU),
// accumulated into the row sums y[0..3] (+MU: y+ re/im, y- re/im) and
// y[4..7] (-MU)
template <int L, int MU, int LO, int LI, typename R, typename XV>
__device__ __forceinline__ void ax_pair(const Geom<L, R>& g, XV& xp, R (&y)[8]) {
  constexpr int NH = L * (L + 2);
  if constexpr (LI >= MU) {
    R ar = 0, ai = 0, br = 0, bi = 0;
    ax_entry<L, MU, LO, LI>(g, ar, ai, br, bi, std::make_integer_sequence<int, AxialN<L, MU, LO, LI>::na>{},
                            std::make_integer_sequence<int, AxialN<L, MU, LO, LI>::nb>{});
    // W+ = A + i B', W- = A - i B'
    const R wpr = ar - bi, wpi = ai + br, wmr = ar + bi, wmi = ai - br;
    constexpr int ri = Row<LI, MU>::r;
    cmac(y[0], y[1], wpr, wpi, xp(2 * ri), xp(2 * ri + 1));
    cmac(y[2], y[3], wmr, wmi, xp(2 * (NH + ri)), xp(2 * (NH + ri) + 1));
    if constexpr (MU > 0) {
      // -mu: B changes sign, so W+ and W- swap
      constexpr int rim = Row<LI, -MU>::r;
      cmac(y[4], y[5], wmr, wmi, xp(2 * rim), xp(2 * rim + 1));
      cmac(y[6], y[7], wpr, wpi, xp(2 * (NH + rim)), xp(2 * (NH + rim) + 1));
    }
  }
}

template <int L, int MU, int LO, typename R, typename YV>
__device__ __forceinline__ void ax_store(YV& yp, const R (&y)[8]);

// y += S w x for one (row, column) entry, S = +-1 at compile time
template <int S, typename R>
__device__ __forceinline__ void cmac_s(R& yr, R& yi, R wr, R wi, R xr, R xi) {
  if constexpr (S > 0) {
    cmac(yr, yi, wr, wi, xr, xi);
  } else {
    cmac(yr, yi, -wr, -wi, xr, xi);
  }
}

// Transpose symmetry of the axial block: for a translation along +z the entry
// (l', l) of every |mu| equals (-1)^{l + l'} times the entry (l, l') (A and B
// alike; it follows from the inversion parity of the SVWFs, and is checked
// against the dense coupling matrix).  So each entry with LO <= LI is formed
// once and applied to row LO (column LI) and, with that sign, to row LI
// (column LO).  y[l - 1] holds row l: (+mu: y+ re/im, y- re/im; -mu: same).
template <int L, int MU, int LO, int LI, typename R, typename XV>
__device__ __forceinline__ void ax_sym_pair(const Geom<L, R>& g, XV& xp, R (&y)[L][8]) {
  constexpr int NH = L * (L + 2);
  if constexpr (LO >= MU && LI >= MU && LO <= LI) {
    R ar = 0, ai = 0, br = 0, bi = 0;
    ax_entry<L, MU, LO, LI>(g, ar, ai, br, bi, std::make_integer_sequence<int, AxialN<L, MU, LO, LI>::na>{},
                            std::make_integer_sequence<int, AxialN<L, MU, LO, LI>::nb>{});
    const R wpr = ar - bi, wpi = ai + br, wmr = ar + bi, wmi = ai - br;
    {
      R(&yo)[8] = y[LO - 1];
      constexpr int ri = Row<LI, MU>::r;
      cmac(yo[0], yo[1], wpr, wpi, xp(2 * ri), xp(2 * ri + 1));
      cmac(yo[2], yo[3], wmr, wmi, xp(2 * (NH + ri)), xp(2 * (NH + ri) + 1));
      if constexpr (MU > 0) {
        constexpr int rim = Row<LI, -MU>::r;
        cmac(yo[4], yo[5], wmr, wmi, xp(2 * rim), xp(2 * rim + 1));
        cmac(yo[6], yo[7], wpr, wpi, xp(2 * (NH + rim)), xp(2 * (NH + rim) + 1));
      }
    }
    if constexpr (LO != LI) {
      constexpr int S = ((LO + LI) & 1) ? -1 : 1;
      R(&yt)[8] = y[LI - 1];
      constexpr int rj = Row<LO, MU>::r;
      cmac_s<S>(yt[0], yt[1], wpr, wpi, xp(2 * rj), xp(2 * rj + 1));
      cmac_s<S>(yt[2], yt[3], wmr, wmi, xp(2 * (NH + rj)), xp(2 * (NH + rj) + 1));
      if constexpr (MU > 0) {
        constexpr int rjm = Row<LO, -MU>::r;
        cmac_s<S>(yt[4], yt[5], wmr, wmi, xp(2 * rjm), xp(2 * rjm + 1));
        cmac_s<S>(yt[6], yt[7], wpr, wpi, xp(2 * (NH + rjm)), xp(2 * (NH + rjm) + 1));
      }
    }
  }
}
template <int L, int MU, int LO, typename R, typename XV, int... LII>
__device__ __forceinline__ void ax_sym_row(const Geom<L, R>& g, XV& xp, R (&y)[L][8],
                                           std::integer_sequence<int, LII...>) {
  (ax_sym_pair<L, MU, LO, LII + 1>(g, xp, y), ...);
}
template <int L, int MU, typename R, typename XV, typename YV, int... LOI>
__device__ __forceinline__ void ax_mu_sym(const Geom<L, R>& g, XV& xp, YV& yp, std::integer_sequence<int, LOI...>) {
  R y[L][8];
#pragma unroll
  for (int a = 0; a < L; ++a)
#pragma unroll
    for (int q = 0; q < 8; ++q) y[a][q] = static_cast<R>(0);
  (ax_sym_row<L, MU, LOI + 1>(g, xp, y, std::make_integer_sequence<int, L>{}), ...);
  (ax_store<L, MU, LOI + 1>(yp, y[LOI]), ...);
}

template <int L, int MU, int LO, typename R, typename XV, int... LII>
__device__ __forceinline__ void ax_row(const Geom<L, R>& g, XV& xp, R (&y)[8], std::integer_sequence<int, LII...>) {
  if constexpr (LO >= MU) {
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = static_cast<R>(0);
    (ax_pair<L, MU, LO, LII + 1>(g, xp, y), ...);
  }
}
template <int L, int MU, int LO, typename R, typename YV>
__device__ __forceinline__ void ax_store(YV& yp, const R (&y)[8]) {
  constexpr int NH = L * (L + 2);
  if constexpr (LO >= MU) {
    constexpr int ro = Row<LO, MU>::r;
    yp(2 * ro) = y[0];
    yp(2 * ro + 1) = y[1];
    yp(2 * (NH + ro)) = y[2];
    yp(2 * (NH + ro) + 1) = y[3];
    if constexpr (MU > 0) {
      constexpr int rom = Row<LO, -MU>::r;
      yp(2 * rom) = y[4];
      yp(2 * rom + 1) = y[5];
      yp(2 * (NH + rom)) = y[6];
      yp(2 * (NH + rom) + 1) = y[7];
    }
  }
}
template <int L, int MU, int LO, typename R, typename XV, typename YV>
__device__ __forceinline__ void ax_row_store(const Geom<L, R>& g, XV& xp, YV& yp) {
  R y[8];
  ax_row<L, MU, LO>(g, xp, y, std::make_integer_sequence<int, L>{});
  ax_store<L, MU, LO>(yp, y);
}
// in place (y' overwrites x'): all rows of one |mu| are formed before any is
// stored, since the rows of |mu| read every x'[., +-mu]; otherwise each row is
// stored as soon as it is formed
template <int L, int MU, bool INPLACE, typename R, typename XV, typename YV, int... LOI>
__device__ __forceinline__ void ax_mu(const Geom<L, R>& g, XV& xp, YV& yp, std::integer_sequence<int, LOI...>) {
  if constexpr (INPLACE) {
    R y[L][8];
    (ax_row<L, MU, LOI + 1>(g, xp, y[LOI], std::make_integer_sequence<int, L>{}), ...);
    (ax_store<L, MU, LOI + 1>(yp, y[LOI]), ...);
  } else {
    (ax_row_store<L, MU, LOI + 1>(g, xp, yp), ...);
  }
}
template <int L, bool INPLACE, bool SYM, typename R, typename XV, typename YV, int... MUS>
__device__ __forceinline__ void axial(const Geom<L, R>& g, XV& xp, YV& yp, std::integer_sequence<int, MUS...>) {
  if constexpr (SYM) {
    (ax_mu_sym<L, MUS>(g, xp, yp, std::make_integer_sequence<int, L>{}), ...);
  } else {
    (ax_mu<L, MUS, INPLACE>(g, xp, yp, std::make_integer_sequence<int, L>{}), ...);
  }
}

// ---- step 4: y[l, M] += e^{-i M phi} sum_MU R_{MU,M} y'[l, MU] -------------
template <int L, int l, int M, int OPT, typename R, typename YV, typename Acc, int... MUI>
__device__ __forceinline__ void rot_bwd_col(const Geom<L, R>& g, const R* dv, YV& yp, Acc& acc,
                                            std::integer_sequence<int, MUI...>) {
  constexpr int NH = L * (L + 2);
  R a0 = 0, a1 = 0, b0 = 0, b1 = 0;
  if constexpr (kPackedRot<L, R, OPT>) {
    float2 a = make_float2(0.0f, 0.0f), b = a;
    (
        [&] {
          constexpr int MU = MUI - l;
          using RA = RAt<l, MU, M>;
          const float w = RA::sign > 0 ? dv[RA::id] : -dv[RA::id];
          const float2 ww = make_float2(w, w);
          constexpr int r = Row<l, MU>::r;
          a = __ffma2_rn(ww, make_float2(yp(2 * r), yp(2 * r + 1)), a);
          b = __ffma2_rn(ww, make_float2(yp(2 * (NH + r)), yp(2 * (NH + r) + 1)), b);
        }(),
        ...);
    a0 = a.x;
    a1 = a.y;
    b0 = b.x;
    b1 = b.y;
  } else {
    (
        [&] {
          constexpr int MU = MUI - l;
          using RA = RAt<l, MU, M>;
          const R w = RA::sign > 0 ? dv[RA::id] : -dv[RA::id];
          constexpr int r = Row<l, MU>::r;
          a0 = fma_(w, yp(2 * r), a0);
          a1 = fma_(w, yp(2 * r + 1), a1);
          b0 = fma_(w, yp(2 * (NH + r)), b0);
          b1 = fma_(w, yp(2 * (NH + r) + 1), b1);
        }(),
        ...);
  }
  constexpr int AM = M < 0 ? -M : M;
  const R er = g.ere[AM];
  const R ei = M < 0 ? g.eim[AM] : -g.eim[AM];  // e^{-i M phi}
  constexpr int r = Row<l, M>::r;
  // row r of the receiver's sums: (y+ re, y+ im, y- re, y- im)
  R c[4];
  acc.load(r, c);
  c[0] = fma_(a0, er, fma_(-a1, ei, c[0]));
  c[1] = fma_(a0, ei, fma_(a1, er, c[1]));
  c[2] = fma_(b0, er, fma_(-b1, ei, c[2]));
  c[3] = fma_(b0, ei, fma_(b1, er, c[3]));
  acc.store(r, c);
  (void)NH;
}

template <int L, int l, int OPT, typename R, typename YV, typename Acc, int... MI>
__device__ __forceinline__ void rot_bwd_block(const Geom<L, R>& g, YV& yp, Acc& acc,
                                              std::integer_sequence<int, MI...>) {
  R dv[DCount<l>::ncanon];
  dmatrix<L, l>(g, dv);
  (rot_bwd_col<L, l, MI - l, OPT>(g, dv, yp, acc, std::make_integer_sequence<int, 2 * l + 1>{}), ...);
}

template <int L, int OPT, typename R, typename YV, typename Acc, int... LI>
__device__ __forceinline__ void rot_bwd(const Geom<L, R>& g, YV& yp, Acc& acc, std::integer_sequence<int, LI...>) {
  (rot_bwd_block<L, LI + 1, OPT>(g, yp, acc, std::make_integer_sequence<int, 2 * (LI + 1) + 1>{}), ...);
}

// storage views: registers (compile-time index) or a per-thread column of a
// shared-memory array [4 NH][BLOCK]
template <typename R>
struct AccReg {
  R* a;
  __device__ __forceinline__ R& operator()(int q) const { return a[q]; }
};
template <typename R, int BLOCK>
struct AccSmem {
  R* a;
  __device__ __forceinline__ R& operator()(int q) const { return a[q * BLOCK]; }
};

// receiver sums, one 4-vector (y+ re, y+ im, y- re, y- im) per output row:
// registers [NH][4], or shared memory [NH][BLOCK] of 4-vectors (one 16- or
// 32-byte access per row)
template <typename R>
struct RowAccReg {
  R* a;
  __device__ __forceinline__ void load(int r, R (&c)[4]) const {
    c[0] = a[4 * r];
    c[1] = a[4 * r + 1];
    c[2] = a[4 * r + 2];
    c[3] = a[4 * r + 3];
  }
  __device__ __forceinline__ void store(int r, const R (&c)[4]) const {
    a[4 * r] = c[0];
    a[4 * r + 1] = c[1];
    a[4 * r + 2] = c[2];
    a[4 * r + 3] = c[3];
  }
};
template <typename R, int BLOCK>
struct RowAccSmem {
  Quad4<R>* a;  // this thread's element of row 0
  __device__ __forceinline__ void load(int r, R (&c)[4]) const {
    const Quad4<R> v = a[r * BLOCK];
    c[0] = v.x;
    c[1] = v.y;
    c[2] = v.z;
    c[3] = v.w;
  }
  __device__ __forceinline__ void store(int r, const R (&c)[4]) const { a[r * BLOCK] = Quad4<R>{c[0], c[1], c[2], c[3]}; }
};

template <int L, bool INPLACE, bool SYM, typename R, int OPT = 0, typename XV, typename YV, typename Acc>
__device__ __forceinline__ void pair(const Geom<L, R>& g, const Pair2<R>* __restrict__ xs, XV& xp, YV& yp, Acc& acc) {
  rot_fwd<L, OPT>(g, xs, xp, std::make_integer_sequence<int, L>{});
  axial<L, INPLACE, SYM>(g, xp, yp, std::make_integer_sequence<int, L + 1>{});
  rot_bwd<L, OPT>(g, yp, acc, std::make_integer_sequence<int, L>{});
}

// One pair with the tables rebuilt per stage from the pair's scalars: the
// half-angle powers and e^{i m phi} for each rotation, h_p for the axial
// step.  The rebuild before the backward rotation reads the scalars through
// an optimizer barrier, so the compiler cannot keep the forward rotation's
// tables alive across the axial step (fewer live registers per thread).
template <int L, bool INPLACE, bool SYM, int OPT = 0, typename XV, typename YV, typename Acc>
__device__ __forceinline__ void pair_lazy(const GeomS& q, const Pair2<float>* __restrict__ xs, XV& xp, YV& yp,
                                          Acc& acc) {
  {
    Geom<L, float> g;
    geometry_angles<L>(q.ct, q.st, q.cph, q.sph, g);
    rot_fwd<L, OPT>(g, xs, xp, std::make_integer_sequence<int, L>{});
  }
  {
    Geom<L, float> g;
    fill_hankel<L>(q, g);
    axial<L, INPLACE, SYM>(g, xp, yp, std::make_integer_sequence<int, L + 1>{});
  }
  float ct = q.ct, st = q.st, cph = q.cph, sph = q.sph;
  asm volatile("" : "+f"(ct), "+f"(st), "+f"(cph), "+f"(sph));
  {
    Geom<L, float> g;
    geometry_angles<L>(ct, st, cph, sph, g);
    rot_bwd<L, OPT>(g, yp, acc, std::make_integer_sequence<int, L>{});
  }
}

// Launch shape per (lmax, precision), chosen by timing sweeps on GB300 at
// N = 10 000
template <int L, typename R>
struct Config {
  static constexpr bool FP64 = sizeof(R) == 8;
  static constexpr int BLOCK = FP64 ? (L >= 5 ? 32 : 64) : 128;
  static constexpr int TJ = FP64 ? 16 : 32;
  static constexpr bool ACC_SMEM = FP64 ? (L >= 2) : (L >= 3);
  static constexpr bool XY_SMEM = FP64 && L >= 3;
  static constexpr bool XY_INPLACE = XY_SMEM;  // y' overwrites x' (one shared-memory array)
  static constexpr bool SYM_AXIAL = true;       // axial entries formed once per (l, l') pair
  // FP32: per-stage geometry tables (pair_lazy); removes the spills at lmax 5
  // (22.8 vs 26.1 ms); at lmax 4 the full tables are faster (12.3 vs 12.8 ms),
  // at lmax 3 the two are within run-to-run noise
  static constexpr bool LAZY_GEOM = !FP64 && L == 5;
  static constexpr bool SYNC_PAIR = false;  // barrier per source (keeps a CTA's warps in step)
  static constexpr int MINB = (!FP64 && L == 3) ? 3 : 1;  // minimum resident CTAs per SM for the allocator
  static constexpr int OPT = 0;  // pair-code option bits (kPackedRot)
};

// The alternative FP32 launch shape of each lmax, the second candidate of
// the autotuner (celes_ctx tuning): lmax 1-2 64-receiver CTAs, lmax 3 the
// register allocator left free (two CTAs per SM), lmax 4 the x+ phase
// multiply on the packed FMA, lmax 5 64-receiver CTAs with x' and y' in shared
// memory (in place) and the rotations on the packed FMA.  Everything else as
// in Config.
template <int L, typename R>
struct ConfigAlt : Config<L, R> {
  static constexpr int BLOCK = (L <= 2 || L == 5) ? 64 : 128;
  static constexpr int MINB = 1;
  static constexpr int OPT = L == 4 ? 1 : (L == 5 ? 2 : 0);
  static constexpr bool XY_SMEM = Config<L, R>::XY_SMEM || L == 5;
  static constexpr bool XY_INPLACE = XY_SMEM;
};

template <int L, typename R, typename C = Config<L, R>>
struct Layout {
  static constexpr int NH = L * (L + 2);
  static constexpr size_t col = sizeof(R) * 4 * NH * C::BLOCK;  // one [4 NH][BLOCK] array
  static constexpr size_t off_pos = 0;
  static constexpr size_t off_x = off_pos + sizeof(Pos4) * C::TJ;
  static constexpr size_t off_acc = off_x + sizeof(Pair2<R>) * 2 * NH * C::TJ;
  static constexpr size_t off_xy = off_acc + (C::ACC_SMEM ? col : 0);
  static constexpr size_t bytes = off_xy + (C::XY_SMEM ? (C::XY_INPLACE ? 1 : 2) * col : 0);
};

// whether `atomic` asks for the in-L2 vector reduction of the partial sums
// (FP32 only; otherwise the request is ignored)
template <typename R>
constexpr bool partial_atomic(bool atomic) {
  return atomic && sizeof(R) == 4;
}

// One tile: receivers rb*BLOCK .. +BLOCK against sources j0 .. j1 - 1; writes
// this tile's partial sums in the +- basis to out ([N][2][NH] complex, the
// slice of the tile's source chunk).  Called by every thread of the CTA.
// CRED (shared-memory accumulators only): the CTAs of one thread-block
// cluster (one receiver block, consecutive source chunks) add their sums
// through distributed shared memory and write one partial per cluster, so
// the partial-sum traffic shrinks by the cluster size.
// ATOM (FP32): the sums are added into out with vector reductions in L2
// (out zeroed before the launch), so all source chunks share one slice and
// only the final sums reach DRAM; the order of the additions, and so the
// last bits of the result, vary from launch to launch.
template <int L, typename R, typename C, bool CRED = false, bool ATOM = false>
__device__ __forceinline__ void rtr_tile(int N, const Pos4* __restrict__ pos, const Pair2<R>* __restrict__ x,
                                         Pair2<R>* __restrict__ outp, double k, int rb, int j0, int j1,
                                         unsigned char* smem_raw) {
  using LY = Layout<L, R, C>;
  constexpr int NH = L * (L + 2);
  constexpr int BLOCK = C::BLOCK;
  constexpr int TJ = C::TJ;
  Pos4* spos = reinterpret_cast<Pos4*>(smem_raw + LY::off_pos);
  Pair2<R>* sx = reinterpret_cast<Pair2<R>*>(smem_raw + LY::off_x);
  R* sacc = reinterpret_cast<R*>(smem_raw + LY::off_acc);
  R* sxy = reinterpret_cast<R*>(smem_raw + LY::off_xy);

  const int tid = threadIdx.x;
  const int i = rb * BLOCK + tid;
  const bool active = i < N;
  constexpr bool FF = sizeof(R) == 4;  // FP32: float-float positions scaled by k
  Pos4 ri = Pos4{0, 0, 0, 0};
  if (active) ri = pos[i];
  const PosFF rf = split_pos(ri, k);
  PosFF* sposf = reinterpret_cast<PosFF*>(spos);

  R areg[C::ACC_SMEM ? 1 : 4 * NH];
  Quad4<R>* sacc4 = reinterpret_cast<Quad4<R>*>(sacc);
  if constexpr (C::ACC_SMEM) {
    for (int r = 0; r < NH; ++r) sacc4[r * BLOCK + tid] = Quad4<R>{0, 0, 0, 0};
  } else {
#pragma unroll
    for (int q = 0; q < 4 * NH; ++q) areg[q] = static_cast<R>(0);
  }

  for (int jt = j0; jt < j1; jt += TJ) {
    const int nj = min(TJ, j1 - jt);
    __syncthreads();
    for (int q = tid; q < nj * NH; q += BLOCK) {
      const int jj = q / NH;
      const int r = q - jj * NH;
      const Pair2<R> a = x[(size_t)(jt + jj) * (2 * NH) + r];
      const Pair2<R> b = x[(size_t)(jt + jj) * (2 * NH) + NH + r];
      sx[jj * 2 * NH + r] = Pair2<R>{a.re + b.re, a.im + b.im};
      sx[jj * 2 * NH + NH + r] = Pair2<R>{a.re - b.re, a.im - b.im};
    }
    if constexpr (FF) {
      for (int q = tid; q < nj; q += BLOCK) sposf[q] = split_pos(pos[jt + q], k);
    } else {
      for (int q = tid; q < nj; q += BLOCK) spos[q] = pos[jt + q];
    }
    __syncthreads();
    {
      for (int jj = 0; jj < nj; ++jj) {
        // optional barrier per pair: keeps the warps of a CTA on the same
        // stretch of the (long, fully unrolled) pair code
        if constexpr (C::SYNC_PAIR) __syncthreads();
        if (!active || jt + jj == i) continue;  // no self coupling
        constexpr bool LAZY = FF && C::LAZY_GEOM;
        Geom<L, R> g;
        GeomS gs;
        if constexpr (LAZY) {
          gs = geometry_ff_scalars<L>(rf, sposf[jj]);
        } else if constexpr (FF) {
          geometry_ff<L>(rf, sposf[jj], g);
        } else {
          const Pos4 rj = spos[jj];
          geometry<L, R>(ri.x - rj.x, ri.y - rj.y, ri.z - rj.z, k, g);
        }
        const Pair2<R>* xs = sx + jj * 2 * NH;
        auto run = [&](auto& xp, auto& yp) {
          constexpr bool INPL = C::XY_SMEM && C::XY_INPLACE;
          if constexpr (C::ACC_SMEM) {
            RowAccSmem<R, BLOCK> acc{sacc4 + tid};
            if constexpr (LAZY) pair_lazy<L, INPL, C::SYM_AXIAL, C::OPT>(gs, xs, xp, yp, acc);
            else pair<L, INPL, C::SYM_AXIAL, R, C::OPT>(g, xs, xp, yp, acc);
          } else {
            RowAccReg<R> acc{areg};
            if constexpr (LAZY) pair_lazy<L, INPL, C::SYM_AXIAL, C::OPT>(gs, xs, xp, yp, acc);
            else pair<L, INPL, C::SYM_AXIAL, R, C::OPT>(g, xs, xp, yp, acc);
          }
        };
        if constexpr (C::XY_SMEM) {
          AccSmem<R, BLOCK> xp{sxy + tid};
          AccSmem<R, BLOCK> yp{sxy + (C::XY_INPLACE ? 0 : 4 * NH * BLOCK) + tid};
          run(xp, yp);
        } else {
          R xa[4 * NH], ya[4 * NH];
          AccReg<R> xp{xa};
          AccReg<R> yp{ya};
          run(xp, yp);
        }
      }
    }
  }
  if constexpr (CRED) {
    static_assert(C::ACC_SMEM, "the cluster reduction reads shared-memory accumulators");
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int ncl = static_cast<int>(cl.num_blocks());
    const int rk = static_cast<int>(cl.block_rank());
    cl.sync();  // every CTA of the cluster has its sums in shared memory
    if (active) {
      Pair2<R>* out = outp + (size_t)i * (2 * NH);
      // rows dealt round robin over the cluster's CTAs; ranks added in order
      for (int r = rk; r < NH; r += ncl) {
        R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int q = 0; q < ncl; ++q) {
          const Quad4<R> v = cl.map_shared_rank(sacc4, q)[r * BLOCK + tid];
          a0 += v.x;
          a1 += v.y;
          a2 += v.z;
          a3 += v.w;
        }
        if constexpr (ATOM) {
          atomicAdd(reinterpret_cast<float2*>(out + r), make_float2(a0, a1));
          atomicAdd(reinterpret_cast<float2*>(out + NH + r), make_float2(a2, a3));
        } else {
          out[r] = Pair2<R>{a0, a1};
          out[NH + r] = Pair2<R>{a2, a3};
        }
      }
    }
    cl.sync();  // no CTA leaves while others read its shared memory
    return;
  }
  if constexpr (ATOM) {
    static_assert(sizeof(R) == 4, "vector reductions of the partial sums are FP32 only");
    // the 2 NH complex sums of a receiver are NH float4 (element pairs 2p,
    // 2p+1 of the flattened [2][NH] row: the + rows, then the - rows)
    auto elem = [&](int t, int e, float& re, float& im) {
      const int r = e < NH ? e : e - NH;
      if constexpr (C::ACC_SMEM) {
        const Quad4<R> v = sacc4[r * BLOCK + t];
        re = e < NH ? v.x : v.z;
        im = e < NH ? v.y : v.w;
      } else {
        re = areg[4 * r + (e < NH ? 0 : 2)];
        im = areg[4 * r + (e < NH ? 1 : 3)];
      }
    };
    if constexpr (C::ACC_SMEM) {
      // a warp's 32 receivers are contiguous in out: lane-consecutive float4
      // (512 B per warp instruction); each thread's sums are written by its
      // own thread only, so the warp's accumulators are complete here
      __syncwarp();
      const int w0 = tid & ~31;
      const int lane = tid & 31;
      float4* base = reinterpret_cast<float4*>(outp + (size_t)(rb * BLOCK + w0) * (2 * NH));
      for (int q = lane; q < 32 * NH; q += 32) {
        const int t = q / NH;
        const int p = q - t * NH;
        if (rb * BLOCK + w0 + t >= N) break;  // q ascending: later q are further receivers
        float4 v;
        elem(w0 + t, 2 * p, v.x, v.y);
        elem(w0 + t, 2 * p + 1, v.z, v.w);
        atomicAdd(base + q, v);
      }
    } else if (active) {
      float4* base = reinterpret_cast<float4*>(outp + (size_t)i * (2 * NH));
#pragma unroll
      for (int p = 0; p < NH; ++p) {
        float4 v;
        elem(tid, 2 * p, v.x, v.y);
        elem(tid, 2 * p + 1, v.z, v.w);
        atomicAdd(base + p, v);
      }
    }
    return;
  }
  if (active) {
    // partial layout [2][NH] complex: y+ rows, then y- rows
    Pair2<R>* out = outp + (size_t)i * (2 * NH);
    if constexpr (C::ACC_SMEM) {
      for (int r = 0; r < NH; ++r) {
        const Quad4<R> v = sacc4[r * BLOCK + tid];
        out[r] = Pair2<R>{v.x, v.y};
        out[NH + r] = Pair2<R>{v.z, v.w};
      }
    } else {
#pragma unroll
      for (int r = 0; r < NH; ++r) {
        out[r] = Pair2<R>{areg[4 * r], areg[4 * r + 1]};
        out[NH + r] = Pair2<R>{areg[4 * r + 2], areg[4 * r + 3]};
      }
    }
  }
}

// grid (receiver blocks of BLOCK, source chunks); writes partial sums in the
// +- basis, [chunks][N][2][NH] complex (same layout as the direct kernel)
// CRED: launched with clusters of `ncl` CTAs along y; cluster c writes
// partial slice c (the grid's y extent is a multiple of ncl)
// ATOM: every tile adds into slice 0 (zeroed before the launch)
template <int L, typename R, typename C = Config<L, R>, bool CRED = false, bool ATOM = false>
__global__ void __launch_bounds__(C::BLOCK, C::MINB)
    rtr_partial_kernel(int N, const Pos4* __restrict__ pos, const Pair2<R>* __restrict__ x,
                       Pair2<R>* __restrict__ partial, double k, int chunk, int ncl) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  constexpr int NH = L * (L + 2);
  const int j0 = blockIdx.y * chunk;
  const int j1 = min(N, j0 + chunk);
  const int slice = ATOM ? 0 : (CRED ? static_cast<int>(blockIdx.y) / ncl : static_cast<int>(blockIdx.y));
  rtr_tile<L, R, C, CRED, ATOM>(N, pos, x, partial + (size_t)slice * N * (2 * NH), k, blockIdx.x, j0, j1,
                                smem_raw);
}

// ---- batched form: one persistent launch over the tiles of many systems ----
// A system is one right-hand side of one sphere ensemble (all of the same
// lmax in one launch).  Its tiles are (receiver block, source chunk) pairs
// numbered tile0 .. tile0 + nrb * chunks - 1 within the launch; CTAs take
// tiles from a global counter (dynamic scheduling, so uneven ensembles
// balance), and systems whose flag `active` is 0 are skipped.  The FP32
// launch adds all chunks of a system into its one partial slice in L2 (the
// batched epilogue reads the slice and zeroes it again); the FP64 launch
// writes one slice per chunk.
struct BatchSys {
  const Pos4* pos;
  const void* x;      // input vector [N][nmax] complex (FP32 or FP64 as launched)
  void* y;            // output [N][nmax]
  void* partial;      // [chunks][N][2][NH] scratch
  const void* tq;     // T [N][2][L] complex in the launch's precision (master operator)
  double k;
  long long tile0;
  int N, L, chunk, nrb, chunks, active;
};

template <int L, typename R, typename C = Config<L, R>, bool ATOM = partial_atomic<R>(true)>
__global__ void __launch_bounds__(C::BLOCK, C::MINB)
    rtr_batch_kernel(const BatchSys* __restrict__ sys, int nsys, long long ntiles,
                     unsigned long long* __restrict__ counter) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  constexpr int NH = L * (L + 2);
  __shared__ long long tile_s;
  for (;;) {
    if (threadIdx.x == 0) tile_s = static_cast<long long>(atomicAdd(counter, 1ULL));
    __syncthreads();
    const long long t = tile_s;
    __syncthreads();
    if (t >= ntiles) break;
    // system holding tile t (tile0 ascending)
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sys[mid].tile0 <= t) lo = mid;
      else hi = mid - 1;
    }
    const BatchSys& S = sys[lo];
    if (!S.active) continue;
    const int local = static_cast<int>(t - S.tile0);
    const int rb = local % S.nrb, ch = local / S.nrb;
    if (ch >= S.chunks) continue;  // never taken with consistent descriptors
    const int j0 = ch * S.chunk;
    const int j1 = min(S.N, j0 + S.chunk);
    rtr_tile<L, R, C, false, ATOM>(S.N, S.pos, static_cast<const Pair2<R>*>(S.x),
                                   static_cast<Pair2<R>*>(S.partial) + (ATOM ? 0 : (size_t)ch * S.N * (2 * NH)), S.k,
                                   rb, j0, j1, smem_raw);
  }
}

// one-time setup of a kernel's shared-memory limit; returns its resident CTAs
// per SM (0 on error)
template <typename K>
int kernel_setup(K* kern, int block, size_t smem) {
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem) != cudaSuccess) return 0;
  return occ;
}

// resident CTAs per SM of the per-context and the batched kernel on the
// current device; the first call on each device sets the kernel's
// shared-memory limit there (0 on error)
template <int L, typename R, typename C = Config<L, R>>
int partial_occupancy() {
  static PerDevice cache;
  return cache.get(current_device,
                   [] { return kernel_setup(rtr_partial_kernel<L, R, C, false>, C::BLOCK, Layout<L, R, C>::bytes); });
}
template <int L, typename R, typename C = Config<L, R>>
int batch_occupancy() {
  static PerDevice cache;
  return cache.get(current_device,
                   [] { return kernel_setup(rtr_batch_kernel<L, R, C>, C::BLOCK, Layout<L, R, C>::bytes); });
}

// resident CTAs of the per-context kernel on the whole GPU (SMs x CTAs per SM)
template <int L, typename R, typename C = Config<L, R>>
int resident_slots() {
  const int occ = partial_occupancy<L, R, C>();
  return device_sms() * (occ > 0 ? occ : 1);
}

// cluster size of the partial-sum reduction for `chunks` source chunks: the
// largest of 8, 4, 2 that divides it (shared-memory accumulators only), else 1
template <int L, typename R, typename C = Config<L, R>>
int partial_cluster(int chunks, int maxcl) {
  if constexpr (!C::ACC_SMEM) {
    return 1;
  } else {
    for (int c = 8; c > 1; c >>= 1)
      if (c <= maxcl && chunks % c == 0) return c;
    return 1;
  }
}

// resident CTAs per SM of one reduction form of the per-context kernel (the
// first call on each device sets its shared-memory limit there)
template <int L, typename R, typename C, bool CRED, bool ATOM>
int partial_form_occupancy() {
  static PerDevice cache;
  return cache.get(current_device, [] {
    return kernel_setup(rtr_partial_kernel<L, R, C, CRED, ATOM>, C::BLOCK, Layout<L, R, C>::bytes);
  });
}

// partial-sum slices the epilogue must add after a launch with these options
template <int L, typename R, typename C = Config<L, R>>
int partial_slices(int chunks, int maxcl, bool atomic) {
  if (partial_atomic<R>(atomic)) return 1;
  return chunks / partial_cluster<L, R, C>(chunks, maxcl);
}

template <int L, typename R, typename C, bool CRED, bool ATOM>
cudaError_t launch_partial_form(int64_t N, const void* pos, const void* x, void* partial, double k, int chunks,
                                int ncl, cudaStream_t st) {
  using LY = Layout<L, R, C>;
  if (partial_form_occupancy<L, R, C, CRED, ATOM>() < 1) return cudaErrorInvalidConfiguration;
  const int64_t chunk = (N + chunks - 1) / chunks;
  dim3 grid(static_cast<unsigned>((N + C::BLOCK - 1) / C::BLOCK), static_cast<unsigned>(chunks));
  if constexpr (ATOM) {
    const cudaError_t e = cudaMemsetAsync(partial, 0, sizeof(Pair2<R>) * 2 * (L * (L + 2)) * N, st);
    if (e != cudaSuccess) return e;
  }
  if constexpr (CRED) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(C::BLOCK);
    cfg.dynamicSmemBytes = LY::bytes;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = static_cast<unsigned>(ncl);
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, rtr_partial_kernel<L, R, C, true, ATOM>, static_cast<int>(N),
                                             static_cast<const Pos4*>(pos), static_cast<const Pair2<R>*>(x),
                                             static_cast<Pair2<R>*>(partial), k, static_cast<int>(chunk), ncl);
    note_launch();
    return e;
  } else {
    rtr_partial_kernel<L, R, C, false, ATOM><<<grid, C::BLOCK, LY::bytes, st>>>(
        static_cast<int>(N), static_cast<const Pos4*>(pos), static_cast<const Pair2<R>*>(x),
        static_cast<Pair2<R>*>(partial), k, static_cast<int>(chunk), 1);
    note_launch();
    return cudaGetLastError();
  }
}

// `chunks` source chunks, partial-sum clusters of at most `maxcl` CTAs (1:
// no cluster reduction), `atomic`: all chunks added into one slice in L2
// (FP32); writes partial_slices(chunks, maxcl, atomic) partial slices (the
// count the epilogue must add)
template <int L, typename R, typename C = Config<L, R>>
cudaError_t launch_partial(int64_t N, const void* pos, const void* x, void* partial, double k, int chunks,
                           cudaStream_t st, int maxcl = 1, bool atomic = false) {
  const int occ = partial_occupancy<L, R, C>();
  if (occ < 1) return cudaErrorInvalidConfiguration;
  if (N <= 0) return cudaSuccess;
  if (chunks < 1) chunks = 1;
  const int ncl = partial_cluster<L, R, C>(chunks, maxcl);
  constexpr bool AT_OK = partial_atomic<R>(true);
  if (ncl > 1) {
    if constexpr (C::ACC_SMEM) {
      if (AT_OK && atomic) return launch_partial_form<L, R, C, true, AT_OK>(N, pos, x, partial, k, chunks, ncl, st);
      return launch_partial_form<L, R, C, true, false>(N, pos, x, partial, k, chunks, ncl, st);
    }
  }
  if (AT_OK && atomic) return launch_partial_form<L, R, C, false, AT_OK>(N, pos, x, partial, k, chunks, 1, st);
  return launch_partial_form<L, R, C, false, false>(N, pos, x, partial, k, chunks, 1, st);
}

// persistent batched launch: one CTA per resident slot, tiles from `counter`
// (zeroed by the caller before the launch)
template <int L, typename R, typename C = Config<L, R>>
cudaError_t launch_batch(const void* sys, int nsys, long long ntiles, unsigned long long* counter, cudaStream_t st) {
  using LY = Layout<L, R, C>;
  const int occ = batch_occupancy<L, R, C>();
  if (occ < 1) return cudaErrorInvalidConfiguration;
  if (nsys <= 0 || ntiles <= 0) return cudaSuccess;
  const long long slots = static_cast<long long>(device_sms()) * occ;
  const unsigned grid = static_cast<unsigned>(ntiles < slots ? ntiles : slots);
  rtr_batch_kernel<L, R, C><<<grid, C::BLOCK, LY::bytes, st>>>(static_cast<const BatchSys*>(sys), nsys, ntiles,
                                                                counter);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rtr
}  // namespace celes

namespace celes {
namespace rtr {
static_assert(Layout<5, float>::bytes <= 227 * 1024, "shared memory of the lmax 5 FP32 kernel");
static_assert(Layout<5, double>::bytes <= 227 * 1024, "shared memory of the lmax 5 FP64 kernel");
static_assert(Layout<4, float>::bytes <= 227 * 1024, "shared memory of the lmax 4 FP32 kernel");
}  // namespace rtr
}  // namespace celes
