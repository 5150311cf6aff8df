"""Special functions of the FP64 oracle (test infrastructure only).

* Spherical Bessel j_l, Neumann y_l and Hankel h_l = j_l + i y_l of the first
  kind (App. A.1: z^(1) = j_l, z^(3) = h_l^(1)).  ``scipy.special`` supplies
  j_l and y_l as single library steps; everything else is composed here.
* Normalised associated Legendre functions P_l^m (App. A.1, "normalized
  associated Legendre functions").  The paper does not define the
  normalisation.  Reading used throughout: ``P_l^m(x) = sqrt((2l+1)/2 *
  (l-m)!/(l+m)!) (1-x^2)^{m/2} d^m/dx^m P_l(x)`` for m >= 0, no Condon-Shortley
  phase, so that int_{-1}^{1} P_l^m(x)^2 dx = 1.  It is the reading under which
  the paper's a5/b5 coefficients satisfy the SVWF addition theorem (pinned in
  tests/test_oracle_translation.py).
* pi_l^m = P_l^m(cos t)/sin t and tau_l^m = d/dt P_l^m(cos t) (App. A.1),
  evaluated from the derivative polynomials so that they are exact at t = 0.
* Wigner-3j symbols from the Racah formula in exact rational arithmetic.
"""

from fractions import Fraction
from functools import lru_cache
from math import factorial, sqrt

import numpy as np
import numpy.polynomial.legendre as npleg
import scipy.special as sps


# ----------------------------------------------------------------------------
# radial functions
# ----------------------------------------------------------------------------

def sph_j(l, z):
    """Spherical Bessel function j_l(z) (real or complex z)."""
    return sps.spherical_jn(l, z)


def sph_y(l, z):
    """Spherical Neumann function y_l(z)."""
    return sps.spherical_yn(l, z)


def sph_h1(l, x):
    """Spherical Hankel function of the first kind h_l^(1)(x) = j_l + i y_l."""
    return sps.spherical_jn(l, x) + 1j * sps.spherical_yn(l, x)


def dxxj(l, z):
    """d/dz [z j_l(z)] = z j_{l-1}(z) - l j_l(z)  (l >= 1)."""
    return z * sph_j(l - 1, z) - l * sph_j(l, z)


def dxxh(l, x):
    """d/dx [x h_l(x)] = x h_{l-1}(x) - l h_l(x)  (l >= 1)."""
    return x * sph_h1(l - 1, x) - l * sph_h1(l, x)


def sph_h1_closed(l, x):
    """Finite closed form of h_l^(1)(x) (a polynomial in 1/x times e^{ix}).

    h_l(x) = (-i)^{l+1} e^{ix}/x * sum_{k=0}^{l} i^k (l+k)! / (k! (l-k)! (2x)^k).
    Independent of ``sph_h1``; used only as a pin.
    """
    x = np.asarray(x, dtype=float)
    s = np.zeros(x.shape, dtype=complex)
    for k in range(l + 1):
        s = s + (1j ** k) * factorial(l + k) / (factorial(k) * factorial(l - k)) / (2.0 * x) ** k
    return (-1j) ** (l + 1) * np.exp(1j * x) / x * s


# ----------------------------------------------------------------------------
# angular functions
# ----------------------------------------------------------------------------

@lru_cache(maxsize=None)
def _deriv_poly(l, m):
    """m-th derivative of the Legendre polynomial P_l as a Legendre series."""
    if m > l:
        return None
    return npleg.Legendre.basis(l).deriv(m)


def _dm(l, m, ct):
    p = _deriv_poly(l, m)
    if p is None:
        return np.zeros(np.shape(ct))
    return p(ct)


def norm_lm(l, m):
    """sqrt((2l+1)/2 * (l-m)!/(l+m)!)."""
    return sqrt((2 * l + 1) / 2.0 * factorial(l - m) / factorial(l + m))


def legendre_p(l, m, ct, st):
    """Normalised associated Legendre function P_l^m(cos t), m >= 0."""
    m = abs(m)
    if m > l:
        return np.zeros(np.shape(ct))
    return norm_lm(l, m) * st ** m * _dm(l, m, ct)


def legendre_pi(l, m, ct, st):
    """pi_l^m(t) = P_l^m(cos t)/sin t, m >= 0 (0 for m = 0, where it only
    appears multiplied by m)."""
    m = abs(m)
    if m == 0 or m > l:
        return np.zeros(np.shape(ct))
    return norm_lm(l, m) * st ** (m - 1) * _dm(l, m, ct)


def legendre_tau(l, m, ct, st):
    """tau_l^m(t) = d/dt P_l^m(cos t), m >= 0."""
    m = abs(m)
    if m > l:
        return np.zeros(np.shape(ct))
    val = -st ** (m + 1) * _dm(l, m + 1, ct)
    if m > 0:
        val = val + m * st ** (m - 1) * ct * _dm(l, m, ct)
    return norm_lm(l, m) * val


# ----------------------------------------------------------------------------
# Wigner 3j (exact)
# ----------------------------------------------------------------------------

@lru_cache(maxsize=None)
def wigner3j_sq_signed(j1, j2, j3, m1, m2, m3):
    """Return (sign, value^2 as Fraction) of the Wigner-3j symbol.

    Racah formula:
      (j1 j2 j3; m1 m2 m3) = (-1)^{j1-j2-m3} sqrt(Delta * prod (j_i +- m_i)!)
          * sum_k (-1)^k / [k! (j3-j2+k+m1)! (j3-j1+k-m2)! (j1+j2-j3-k)!
                            (j1-k-m1)! (j2-k+m2)!]
      Delta = (j1+j2-j3)! (j1-j2+j3)! (-j1+j2+j3)! / (j1+j2+j3+1)!
    """
    if m1 + m2 + m3 != 0:
        return 0, Fraction(0)
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0, Fraction(0)
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0, Fraction(0)
    delta = Fraction(factorial(j1 + j2 - j3) * factorial(j1 - j2 + j3) * factorial(-j1 + j2 + j3),
                     factorial(j1 + j2 + j3 + 1))
    pre = (factorial(j1 + m1) * factorial(j1 - m1) * factorial(j2 + m2) * factorial(j2 - m2)
           * factorial(j3 + m3) * factorial(j3 - m3))
    kmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    kmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    s = Fraction(0)
    for k in range(kmin, kmax + 1):
        den = (factorial(k) * factorial(j3 - j2 + k + m1) * factorial(j3 - j1 + k - m2)
               * factorial(j1 + j2 - j3 - k) * factorial(j1 - k - m1) * factorial(j2 - k + m2))
        s += Fraction((-1) ** k, den)
    if s == 0:
        return 0, Fraction(0)
    sign = (-1) ** ((j1 - j2 - m3) % 2) * (1 if s > 0 else -1)
    return sign, delta * pre * s * s


def wigner3j(j1, j2, j3, m1, m2, m3):
    """Wigner-3j symbol as a float (exact up to the final square root)."""
    sign, sq = wigner3j_sq_signed(j1, j2, j3, m1, m2, m3)
    if sign == 0:
        return 0.0
    # int / int true division is correctly rounded in Python
    return sign * sqrt(sq.numerator / sq.denominator)


# ----------------------------------------------------------------------------
# cylindrical Bessel (Gaussian beam, App. C)
# ----------------------------------------------------------------------------

def besselj(nu, x):
    """Bessel function of the first kind J_nu(x)."""
    return sps.jv(nu, x)
