// Compile-time tables of the rotation-translation-rotation factorisation of
// the coupling block (the O(lmax^3) scheme of Sec. 5; exact, not an
// approximation):
//
//   W(d) = D^H W_z(k|d|) D,   D = blockdiag_l R^l(theta) diag(e^{i m phi})
//
// where (|d|, theta, phi) are the spherical coordinates of d = r_i - r_j,
// R^l_{mu m}(theta) = s_mu s_m d^l_{m mu}(theta) with Wigner's small-d matrix
// and s_m = (-1)^m for m >= 0, 1 for m < 0 (the sign that converts the
// Condon-Shortley convention to the normalised Legendre functions of App. A.1
// used here), and W_z is the coupling block of a translation along +z: it is
// diagonal in m, with (theta = 0, so only P_p^0(1) = sqrt((2p+1)/2) survives)
//
//   W_z[(tau,l,mu),(tau',l',mu)] = sum_p {a5 | i b5'}(l',mu|l,mu|p) sqrt((2p+1)/2) h_p(k|d|)
//
// (a5 for tau = tau', i b5' otherwise; App. A.2).  Under mu -> -mu the a5
// factor is unchanged and b5' changes sign.
//
// Wigner's small-d matrix from its explicit sum:
//   d^l_{m'm}(b) = sum_k (-1)^{k-m+m'} sqrt((l+m')!(l-m')!(l+m)!(l-m)!)
//                  / [(l+m-k)! k! (l-k-m')! (k-m+m')!]  c^{2l-j} s^j,
//   c = cos(b/2), s = sin(b/2), j = 2k - m + m'.
// With d_{m'm} = (-1)^{m-m'} d_{mm'} = d_{-m,-m'} only one entry of each orbit
// is evaluated.
#pragma once

#include "coupling_tables.cuh"

namespace celes {
namespace rtr {

using tab::csqrt;
using tab::fact;
using tab::iabs;
using tab::imax;
using tab::imin;

constexpr int sgn_pm1(int e) { return (((e % 2) + 2) % 2) ? -1 : 1; }
constexpr int sigma(int m) { return m >= 0 ? sgn_pm1(m) : 1; }

// ---------------------------------------------------------------------------
// Wigner small-d for one degree l
// ---------------------------------------------------------------------------
template <int l>
struct DTable {
  static constexpr int W = 2 * l + 1;
  static constexpr int MAXT = W * W * (l + 1);
  int ncanon = 0;
  int canon_mp[W * W] = {};  // canonical entries (m', m)
  int canon_m[W * W] = {};
  int cid[W * W] = {};       // entry (m' + l, m + l) -> canonical id
  int csgn[W * W] = {};      // and its sign
  int off[W * W + 1] = {};   // terms of canonical id c: [off[c], off[c+1])
  int tj[MAXT] = {};         // monomial index j
  double tc[MAXT] = {};      // coefficient
};

template <int l>
constexpr DTable<l> make_dtable() {
  DTable<l> T{};
  constexpr int W = 2 * l + 1;
  for (int q = 0; q < W * W; ++q) T.cid[q] = -1;
  int t = 0;
  for (int mp = -l; mp <= l; ++mp) {
    for (int m = -l; m <= l; ++m) {
      const int q = (mp + l) * W + (m + l);
      if (T.cid[q] >= 0) continue;
      const int c = T.ncanon++;
      T.canon_mp[c] = mp;
      T.canon_m[c] = m;
      // orbit: (m',m) +1, (m,m') (-1)^{m-m'}, (-m,-m') +1, (-m',-m) (-1)^{m-m'}
      const int s1 = sgn_pm1(m - mp);
      const int om[4][3] = {{mp, m, 1}, {m, mp, s1}, {-m, -mp, 1}, {-mp, -m, s1}};
      for (int o = 0; o < 4; ++o) {
        const int qq = (om[o][0] + l) * W + (om[o][1] + l);
        if (T.cid[qq] < 0) {
          T.cid[qq] = c;
          T.csgn[qq] = om[o][2];
        }
      }
      T.off[c] = t;
      const double num = csqrt(fact(l + mp) * fact(l - mp) * fact(l + m) * fact(l - m));
      for (int k = 0; k <= 2 * l; ++k) {
        const int a1 = l + m - k, a2 = l - k - mp, a3 = k - m + mp;
        if (a1 < 0 || a2 < 0 || a3 < 0) continue;
        T.tj[t] = 2 * k - m + mp;
        T.tc[t] = sgn_pm1(k - m + mp) * num / (fact(a1) * fact(k) * fact(a2) * fact(a3));
        ++t;
      }
    }
  }
  T.off[T.ncanon] = t;
  return T;
}

template <int l>
struct DTab {
  static constexpr DTable<l> value = make_dtable<l>();
};
template <int l, int T>
struct DTerm {
  static constexpr int j = DTab<l>::value.tj[T];
  static constexpr double c = DTab<l>::value.tc[T];
};
template <int l, int C>
struct DCanon {
  static constexpr int t0 = DTab<l>::value.off[C];
  static constexpr int t1 = DTab<l>::value.off[C + 1];
};
template <int l>
struct DCount {
  static constexpr int ncanon = DTab<l>::value.ncanon;
};
// R^l_{mu m} = s_mu s_m d^l_{m mu} = sign * (canonical entry id)
template <int l, int MU, int M>
struct RAt {
  static constexpr int q = (M + l) * (2 * l + 1) + (MU + l);
  static constexpr int id = DTab<l>::value.cid[q];
  static constexpr int sign = DTab<l>::value.csgn[q] * sigma(MU) * sigma(M);
};

// ---------------------------------------------------------------------------
// axial coupling terms, one table per (mu >= 0, l, l')
// ---------------------------------------------------------------------------
template <int L>
struct AxialRow {
  static constexpr int MAXT = 2 * (2 * L + 2);
  int na = 0, nb = 0;
  int ap[MAXT] = {}, bp[MAXT] = {};
  double ac[MAXT] = {}, bc[MAXT] = {};
};

template <int L>
constexpr AxialRow<L> make_axial(int mu, int l, int lp) {
  AxialRow<L> T{};
  for (int p = iabs(l - lp); p <= l + lp; ++p) {
    const double w = csqrt((2.0 * p + 1.0) / 2.0);
    const double a = tab::ab5_real(0, lp, mu, l, mu, p);
    const double b = tab::ab5_real(1, lp, mu, l, mu, p);
    if (a != 0.0) {
      T.ap[T.na] = p;
      T.ac[T.na] = a * w;
      ++T.na;
    }
    if (b != 0.0) {
      T.bp[T.nb] = p;
      T.bc[T.nb] = b * w;
      ++T.nb;
    }
  }
  return T;
}

template <int L, int MU, int LO, int LI>
struct Axial {
  static constexpr AxialRow<L> value = make_axial<L>(MU, LO, LI);
};
template <int L, int MU, int LO, int LI, int T>
struct AxialA {
  static constexpr int p = Axial<L, MU, LO, LI>::value.ap[T];
  static constexpr double c = Axial<L, MU, LO, LI>::value.ac[T];
};
template <int L, int MU, int LO, int LI, int T>
struct AxialB {
  static constexpr int p = Axial<L, MU, LO, LI>::value.bp[T];
  static constexpr double c = Axial<L, MU, LO, LI>::value.bc[T];
};
template <int L, int MU, int LO, int LI>
struct AxialN {
  static constexpr int na = Axial<L, MU, LO, LI>::value.na;
  static constexpr int nb = Axial<L, MU, LO, LI>::value.nb;
};

}  // namespace rtr
}  // namespace celes
