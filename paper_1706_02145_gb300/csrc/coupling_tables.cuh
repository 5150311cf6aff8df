// Compile-time tables of the SVWF translation coefficients (App. A.2).
//
// The coefficients a5(l,m|l',m'|p) and b5(l,m|l',m'|p) do not depend on the
// sphere pair (Sec. 3.2.2: "evaluated only once and stored in a table").  Here
// the "table" is built by the C++ compiler: every nonzero term becomes an
// immediate operand of the generated FMA instructions, so the coupling kernel
// reads no coefficient memory at all.
//
//   a5 = i^{|m-m'|-|m|-|m'|+l'-l+p} (-1)^{m-m'} (l(l+1) + l'(l'+1) - p(p+1)) sqrt(2p+1)
//        sqrt((2l+1)(2l'+1) / (2l(l+1)l'(l'+1))) (l l' p; m -m' m'-m) (l l' p; 0 0 0)
//   b5 = i^{...same...} (-1)^{m-m'} sqrt((l+l'+1+p)(l+l'+1-p)(p+l-l')(p-l+l')(2p+1))
//        sqrt((2l'+1)(2l+1) / (2l(l+1)l'(l'+1))) (l l' p; m -m' m'-m) (l l' p-1; 0 0 0)
//
// For a nonzero a5 the exponent of i is even (a5 is real); for a nonzero b5 it
// is odd (b5 = i * b5' with b5' real).  Only the real factors are stored.
//
// Wigner-3j symbols use Racah's closed formula, evaluated in double precision
// at compile time; factorials up to 23! are exact in double and the alternating
// sums stay short for the degrees used here (l, l' <= 5, p <= 10).
#pragma once

namespace celes {
namespace tab {

constexpr int iabs(int a) { return a < 0 ? -a : a; }
constexpr int imin(int a, int b) { return a < b ? a : b; }
constexpr int imax(int a, int b) { return a > b ? a : b; }

// Square root by Newton's iteration after scaling the argument into [1, 4)
// by powers of 4 (compile-time use only).
constexpr double csqrt(double a) {
  if (a <= 0.0) return 0.0;
  double scale = 1.0;
  while (a >= 18446744073709551616.0) { a /= 18446744073709551616.0; scale *= 4294967296.0; }
  while (a < 1.0 / 18446744073709551616.0) { a *= 18446744073709551616.0; scale /= 4294967296.0; }
  while (a >= 4.0) { a *= 0.25; scale *= 2.0; }
  while (a < 1.0) { a *= 4.0; scale *= 0.5; }
  double x = 0.5 * (a + 1.0);
  for (int it = 0; it < 8; ++it) x = 0.5 * (x + a / x);
  return x * scale;
}

struct FactTable {
  double v[48] = {};
  constexpr FactTable() {
    v[0] = 1.0;
    for (int i = 1; i < 48; ++i) v[i] = v[i - 1] * static_cast<double>(i);
  }
};
inline constexpr FactTable kFact{};
constexpr double fact(int n) { return kFact.v[n]; }

// Racah's formula for the Wigner-3j symbol (j1 j2 j3; m1 m2 m3).
constexpr double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j3 < iabs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (iabs(m1) > j1 || iabs(m2) > j2 || iabs(m3) > j3) return 0.0;
  if (m1 == 0 && m2 == 0 && ((j1 + j2 + j3) & 1)) return 0.0;
  const double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
  const double pre = fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) * fact(j3 + m3) * fact(j3 - m3);
  const int kmin = imax(0, imax(j2 - j3 - m1, j1 - j3 + m2));
  const int kmax = imin(j1 + j2 - j3, imin(j1 - m1, j2 + m2));
  double s = 0.0;
  for (int k = kmin; k <= kmax; ++k) {
    const double den = fact(k) * fact(j3 - j2 + k + m1) * fact(j3 - j1 + k - m2) * fact(j1 + j2 - j3 - k) *
                       fact(j1 - k - m1) * fact(j2 - k + m2);
    s += ((k & 1) ? -1.0 : 1.0) / den;
  }
  const int e = j1 - j2 - m3;
  const double sgn = (((e % 2) + 2) % 2) ? -1.0 : 1.0;
  return sgn * csqrt(tri * pre) * s;
}

// Row index inside one polarisation block: r = l(l+1) - 1 + m.
constexpr int row_l(int r) {
  int l = 1;
  while ((l + 1) * (l + 2) - 1 - (l + 1) <= r) ++l;
  return l;
}
constexpr int row_m(int r) { return r - (row_l(r) * (row_l(r) + 1) - 1); }

// Index of s_{p,mu} = h_p(kd) P_p^mu(cos theta) in the per-pair array.
constexpr int sidx(int p, int mu) { return p * (p + 1) / 2 + mu; }

// Real factor of a5 (A-type term) or of b5/i (B-type term), with
// (l, m) the SOURCE row of the translation operator A_{n n'} and (lp, mp) the
// row it is translated onto.  kind: 0 -> a5, 1 -> b5'.
constexpr double ab5_real(int kind, int l, int m, int lp, int mp, int p) {
  // (l l' p; 0 0 0) vanishes unless l + l' + p is even, (l l' p-1; 0 0 0)
  // unless l + l' + p - 1 is even
  if (kind == 0 && ((l + lp + p) & 1)) return 0.0;
  if (kind == 1 && !((l + lp + p) & 1)) return 0.0;
  const double w_m = wigner3j(l, lp, p, m, -mp, mp - m);
  if (w_m == 0.0) return 0.0;
  const int ipow = iabs(m - mp) - iabs(m) - iabs(mp) + lp - l + p;
  const double sgn_m = ((iabs(m - mp) & 1) ? -1.0 : 1.0);
  const double fac1 = csqrt((2.0 * l + 1.0) * (2.0 * lp + 1.0) / (2.0 * l * (l + 1.0) * lp * (lp + 1.0)));
  if (kind == 0) {
    if (ipow & 1) return 0.0;  // a5 nonzero only for even powers of i
    const double w0 = wigner3j(l, lp, p, 0, 0, 0);
    const double ipw = (((ipow / 2) & 1) ? -1.0 : 1.0);  // i^{ipow}, ipow even
    return ipw * sgn_m * (l * (l + 1.0) + lp * (lp + 1.0) - p * (p + 1.0)) * csqrt(2.0 * p + 1.0) * fac1 * w_m * w0;
  } else {
    if (!(ipow & 1) || p < 1) return 0.0;
    const double prod = (l + lp + 1.0 + p) * (l + lp + 1.0 - p) * (p + l - lp + 0.0) * (p - l + lp + 0.0) * (2.0 * p + 1.0);
    if (prod <= 0.0) return 0.0;
    const double w1 = wigner3j(l, lp, p - 1, 0, 0, 0);
    // i^{ipow} = i * i^{ipow-1}, ipow odd
    const int e = ipow - 1;
    const double ipw = ((((e / 2) % 2) + 2) % 2) ? -1.0 : 1.0;
    return ipw * sgn_m * csqrt(prod) * fac1 * w_m * w1;
  }
}

// All nonzero terms of the coupling block W^{ij} (Sec. 2.2: W_{nn'} = A_{n'n})
// for one SOURCE row ri = (l', m'), grouped by the receiving row ro = (l, m):
//   A-part of W_{ro,ri} = sum_p a5(l',m'|l,m|p) s_{p,|m'-m|}
//   B-part of W_{ro,ri} = i sum_p b5'(l',m'|l,m|p) s_{p,|m'-m|}
// (the phase e^{i(m'-m) phi} is applied outside, as e^{i m' phi} on the source
// and e^{-i m phi} on the result).  One constant evaluation per source row
// keeps each evaluation small.
template <int L>
struct RowTerms {
  static constexpr int NH = L * (L + 2);
  static constexpr int MAXT = NH * (2 * L + 2);
  int count = 0;
  int off[NH + 1] = {};
  int s[MAXT] = {};
  int kind[MAXT] = {};
  double c[MAXT] = {};
};

template <int L>
constexpr RowTerms<L> make_row_terms(int ri) {
  RowTerms<L> T{};
  constexpr int NH = RowTerms<L>::NH;
  int t = 0;
  const int lp = row_l(ri), mp = row_m(ri);
  for (int ro = 0; ro < NH; ++ro) {
    const int l = row_l(ro), m = row_m(ro);
    T.off[ro] = t;
    const int mu = iabs(mp - m);
    for (int p = iabs(l - lp); p <= l + lp; ++p) {
      if (p < mu) continue;
      for (int kind = 0; kind < 2; ++kind) {
        const double c = ab5_real(kind, lp, mp, l, m, p);
        if (c != 0.0) {
          T.s[t] = sidx(p, mu);
          T.kind[t] = kind;
          T.c[t] = c;
          ++t;
        }
      }
    }
  }
  T.off[NH] = t;
  T.count = t;
  return T;
}

template <int L, int RI>
struct RowTable {
  static constexpr RowTerms<L> value = make_row_terms<L>(RI);
};

// Scalar views of one term of entry (RI, RO) (scalars are usable as
// compile-time constants in device code).
template <int L, int RI, int T>
struct TermAt {
  static constexpr int s = RowTable<L, RI>::value.s[T];
  static constexpr int kind = RowTable<L, RI>::value.kind[T];
  static constexpr double c = RowTable<L, RI>::value.c[T];
};

template <int L, int RI, int RO>
struct EntryAt {
  static constexpr int t0 = RowTable<L, RI>::value.off[RO];
  static constexpr int t1 = RowTable<L, RI>::value.off[RO + 1];
};

// Normalised associated Legendre recursion constants (no Condon-Shortley
// phase, int_{-1}^{1} P^2 = 1):
//   P_0^0 = 1/sqrt(2),  P_m^m = sqrt((2m+1)/(2m)) sin(t) P_{m-1}^{m-1},
//   P_{m+1}^m = sqrt(2m+3) cos(t) P_m^m,
//   P_p^m = a_pm (cos(t) P_{p-1}^m - b_pm P_{p-2}^m),
//   a_pm = sqrt((4p^2-1)/(p^2-m^2)),  b_pm = sqrt(((p-1)^2-m^2)/(4(p-1)^2-1)).
constexpr double leg_diag(int m) { return csqrt((2.0 * m + 1.0) / (2.0 * m)); }
constexpr double leg_sub(int m) { return csqrt(2.0 * m + 3.0); }
constexpr double leg_a(int p, int m) { return csqrt((4.0 * p * p - 1.0) / (1.0 * p * p - 1.0 * m * m)); }
constexpr double leg_b(int p, int m) {
  return csqrt(((p - 1.0) * (p - 1.0) - 1.0 * m * m) / (4.0 * (p - 1.0) * (p - 1.0) - 1.0));
}

}  // namespace tab
}  // namespace celes
