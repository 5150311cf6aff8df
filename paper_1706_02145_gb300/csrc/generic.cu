// Runtime-table variants of the coupling-block evaluation (FP64):
//  * the preconditioner block assembly (Sec. 3.2.1, step 2), which writes
//    every entry of W^{ab} explicitly, and
//  * the FP64 coupling matvec for lmax = 5, whose fully unrolled form is too
//    large to compile quickly.
// Both read the (a5, b5) terms of App. A.2 from a device table made from the
// same compile-time term lists that the unrolled kernels use; FP64
// throughput on GB300 is ~1/64 of FP32, so the table loads are not the
// bottleneck of these kernels.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "cmath.cuh"
#include "coupling_kernel.cuh"
#include "kernels.h"

namespace celes {

// term table: per entry e = ri * NH + ro a range [off[e], off[e+1]) of terms,
// term t = (s index | kind << 16, value)
struct TermTableDev {
  const int* off;
  const int* sk;
  const double* c;
};

static __device__ __forceinline__ int row_l_g(int r) {
  int l = static_cast<int>(sqrt(static_cast<double>(r + 1)));
  while ((l + 1) * (l + 1) - 1 <= r) ++l;
  while (l * l - 1 > r) --l;
  return l;
}

constexpr int kGMaxL = 5;
constexpr int kGMaxNS = (2 * kGMaxL + 1) * (2 * kGMaxL + 2) / 2;
constexpr int kGMaxNH = kGMaxL * (kGMaxL + 2);

// s_{p,mu} = h_p(kd) P_p^mu(cos theta) (p <= 2L) and e^{i m phi} (m <= L)
static __device__ void generic_pair_functions(int L, double dx, double dy, double dz, double k, cd* s, cd* e) {
  const int PM = 2 * L;
  const double d = sqrt(dx * dx + dy * dy + dz * dz);
  const double kd = k * d;
  const double TWO_PI = 6.283185307179586476925286766559;
  const double ph = fma(-rint(kd * (1.0 / TWO_PI)), TWO_PI, kd);
  double sn, cs;
  sincos(ph, &sn, &cs);
  const double ix = 1.0 / kd;
  cd h[2 * kGMaxL + 1];
  h[0] = cd{sn * ix, -cs * ix};
  h[1] = cd{-ix * (cs - sn * ix), -ix * (sn + cs * ix)};
  for (int p = 1; p < PM; ++p) h[p + 1] = ((2 * p + 1) * ix) * h[p] - h[p - 1];
  const double ct = dz / d;
  const double rho = sqrt(dx * dx + dy * dy);
  const double st = rho / d;
  const double cph = rho > 0.0 ? dx / rho : 1.0;
  const double sph = rho > 0.0 ? dy / rho : 0.0;
  // normalised Legendre columns
  double diag = 0.70710678118654752440;  // P_0^0
  for (int mu = 0; mu <= PM; ++mu) {
    if (mu > 0) diag *= sqrt((2.0 * mu + 1.0) / (2.0 * mu)) * st;
    double pm2 = 0.0, pm1 = diag;
    s[mu * (mu + 1) / 2 + mu] = pm1 * h[mu];
    for (int p = mu + 1; p <= PM; ++p) {
      double pv;
      if (p == mu + 1) {
        pv = sqrt(2.0 * mu + 3.0) * ct * pm1;
      } else {
        const double a = sqrt((4.0 * p * p - 1.0) / (1.0 * p * p - 1.0 * mu * mu));
        const double b = sqrt(((p - 1.0) * (p - 1.0) - 1.0 * mu * mu) / (4.0 * (p - 1.0) * (p - 1.0) - 1.0));
        pv = a * (ct * pm1 - b * pm2);
      }
      s[p * (p + 1) / 2 + mu] = pv * h[p];
      pm2 = pm1;
      pm1 = pv;
    }
  }
  e[0] = cd{1.0, 0.0};
  for (int m = 1; m <= L; ++m) e[m] = e[m - 1] * cd{cph, sph};
}

static __device__ __forceinline__ cd eim(const cd* e, int m) { return m >= 0 ? e[m] : conj(e[-m]); }

// W_{ro,ri} parts A and B (B including its factor i), without the phase
static __device__ __forceinline__ void generic_entry(const TermTableDev& T, int e, const cd* s, cd& A, cd& B) {
  A = mkc(0.0);
  B = mkc(0.0);
  const int t0 = T.off[e], t1 = T.off[e + 1];
  for (int t = t0; t < t1; ++t) {
    const int sk = T.sk[t];
    const double c = T.c[t];
    const cd v = c * s[sk & 0xffff];
    if (sk >> 16) B = B + v;
    else A = A + v;
  }
  B = cd{-B.im, B.re};
}

// ---------------------------------------------------------------------------
// device tables, built once per (device, L) from the compile-time lists
// ---------------------------------------------------------------------------
struct DevTable {
  int* off = nullptr;
  int* sk = nullptr;
  double* c = nullptr;
};

static std::mutex g_tab_mu;
static DevTable g_tab[64][kGMaxL + 1];

static cudaError_t get_table(int L, TermTableDev& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_tab_mu);
  DevTable& t = g_tab[dev][L];
  if (!t.off) {
    const int NH = L * (L + 2);
    const int cnt = coupling_terms_export(L, nullptr, nullptr, 0);
    std::vector<int> idx(5 * (size_t)cnt);
    std::vector<double> val(cnt);
    coupling_terms_export(L, idx.data(), val.data(), cnt);
    std::vector<int> off(NH * NH + 1, 0), sk(cnt);
    // terms are exported ordered by (ri, ro)
    for (int q = 0; q < cnt; ++q) {
      const int ri = idx[5 * q], ro = idx[5 * q + 1], p = idx[5 * q + 2], mu = idx[5 * q + 3], kind = idx[5 * q + 4];
      off[ri * NH + ro + 1]++;
      sk[q] = (p * (p + 1) / 2 + mu) | (kind << 16);
    }
    for (int q = 0; q < NH * NH; ++q) off[q + 1] += off[q];
    if ((e = cudaMalloc(&t.off, sizeof(int) * off.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t.sk, sizeof(int) * (size_t)cnt)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t.c, sizeof(double) * (size_t)cnt)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(t.off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(t.sk, sk.data(), sizeof(int) * (size_t)cnt, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(t.c, val.data(), sizeof(double) * (size_t)cnt, cudaMemcpyHostToDevice)) != cudaSuccess)
      return e;
  }
  out = TermTableDev{t.off, t.sk, t.c};
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// preconditioner block assembly: one thread per ordered pair (a, b) of a block
//   M_{ab} = delta_ab I - T_a W^{ab},  W_{(tau,ro),(tau',ri)} = e^{i(m'-m)phi} {A, B}
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) generic_assemble_kernel(int L, TermTableDev T,
                                                               const int64_t* __restrict__ block_off,
                                                               const int64_t* __restrict__ mat_off,
                                                               const int* __restrict__ perm,
                                                               const Pos4* __restrict__ pos,
                                                               const double* __restrict__ tq, double k,
                                                               double2* __restrict__ mats) {
  const int NH = L * (L + 2);
  const int NM = 2 * NH;
  const int64_t q = blockIdx.y;
  const int64_t s0 = block_off[q];
  const int64_t nq = block_off[q + 1] - s0;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nq * nq) return;
  const int64_t a = p / nq, b = p - a * nq;
  const int64_t ld = nq * NM;
  double2* M = mats + mat_off[q];
  if (a == b) {
    for (int r = 0; r < NM; ++r)
      for (int cc = 0; cc < NM; ++cc) M[(a * NM + r) + (b * NM + cc) * ld] = make_double2(r == cc ? 1.0 : 0.0, 0.0);
    return;
  }
  const int ia = perm[s0 + a], ib = perm[s0 + b];
  const Pos4 ra = pos[ia], rb = pos[ib];
  cd s[kGMaxNS], e[kGMaxL + 1];
  generic_pair_functions(L, ra.x - rb.x, ra.y - rb.y, ra.z - rb.z, k, s, e);
  const double* qa = tq + (int64_t)ia * 2 * L * 2;
  for (int ri = 0; ri < NH; ++ri) {
    const int lp = row_l_g(ri);
    const int mp = ri - (lp * (lp + 1) - 1);
    const cd e1 = eim(e, mp);
    for (int ro = 0; ro < NH; ++ro) {
      const int l = row_l_g(ro);
      const int m = ro - (l * (l + 1) - 1);
      cd A, B;
      generic_entry(T, ri * NH + ro, s, A, B);
      const cd ph = e1 * eim(e, -m);
      A = ph * A;
      B = ph * B;
      const cd q1 = mkc(qa[2 * (l - 1)], qa[2 * (l - 1) + 1]);
      const cd q2 = mkc(qa[2 * (L + l - 1)], qa[2 * (L + l - 1) + 1]);
      const cd m11 = -(q1 * A), m12 = -(q1 * B), m21 = -(q2 * B), m22 = -(q2 * A);
      const int64_t r1 = a * NM + ro, r2 = r1 + NH;
      const int64_t k1 = b * NM + ri, k2 = k1 + NH;
      M[r1 + k1 * ld] = make_double2(m11.re, m11.im);
      M[r1 + k2 * ld] = make_double2(m12.re, m12.im);
      M[r2 + k1 * ld] = make_double2(m21.re, m21.im);
      M[r2 + k2 * ld] = make_double2(m22.re, m22.im);
    }
  }
}

cudaError_t launch_precond_assemble(int L, int64_t nblocks, const int64_t* block_off, const int64_t* mat_off,
                                    const int* perm, const void* pos, const double* tq, double k, double* mats,
                                    int64_t max_pairs, cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  if (L < 1 || L > kGMaxL) return cudaErrorInvalidValue;
  TermTableDev T;
  cudaError_t e = get_table(L, T);
  if (e != cudaSuccess) return e;
  dim3 grid(static_cast<unsigned>((max_pairs + 127) / 128), static_cast<unsigned>(nblocks));
  generic_assemble_kernel<<<grid, 128, 0, st>>>(L, T, block_off, mat_off, perm, static_cast<const Pos4*>(pos), tq, k,
                                                reinterpret_cast<double2*>(mats));
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 coupling matvec with runtime tables: one thread per receiver, source
// tiles in shared memory; writes the same +- partial layout as the unrolled
// kernels (partial [chunks][N][2][NH])
// ---------------------------------------------------------------------------
constexpr int kGBlock = 64;
constexpr int kGTJ = 16;

__global__ void __launch_bounds__(kGBlock) generic_coupling_kernel(int L, TermTableDev T, int N,
                                                                   const Pos4* __restrict__ pos,
                                                                   const double2* __restrict__ x,
                                                                   double2* __restrict__ partial, double k,
                                                                   int chunk) {
  const int NH = L * (L + 2);
  __shared__ Pos4 spos[kGTJ];
  __shared__ double2 sx[kGTJ * 2 * kGMaxNH];
  const int tid = threadIdx.x;
  const int i = blockIdx.x * kGBlock + tid;
  const int j0 = blockIdx.y * chunk;
  const int j1 = min(N, j0 + chunk);
  const bool active = i < N;
  Pos4 ri = Pos4{0, 0, 0, 0};
  if (active) ri = pos[i];
  cd acc[2 * kGMaxNH];
  for (int q = 0; q < 2 * NH; ++q) acc[q] = mkc(0.0);
  for (int jt = j0; jt < j1; jt += kGTJ) {
    const int nj = min(kGTJ, j1 - jt);
    __syncthreads();
    for (int q = tid; q < nj * NH; q += kGBlock) {
      const int jj = q / NH, r = q - jj * NH;
      const double2 a = x[(size_t)(jt + jj) * (2 * NH) + r];
      const double2 b = x[(size_t)(jt + jj) * (2 * NH) + NH + r];
      sx[jj * 2 * NH + r] = make_double2(a.x + b.x, a.y + b.y);
      sx[jj * 2 * NH + NH + r] = make_double2(a.x - b.x, a.y - b.y);
    }
    for (int q = tid; q < nj; q += kGBlock) spos[q] = pos[jt + q];
    __syncthreads();
    if (!active) continue;
    for (int jj = 0; jj < nj; ++jj) {
      if (jt + jj == i) continue;
      const Pos4 rj = spos[jj];
      cd s[kGMaxNS], e[kGMaxL + 1];
      generic_pair_functions(L, ri.x - rj.x, ri.y - rj.y, ri.z - rj.z, k, s, e);
      cd yp[2 * kGMaxNH];
      for (int q = 0; q < 2 * NH; ++q) yp[q] = mkc(0.0);
      for (int rs = 0; rs < NH; ++rs) {
        const int lp = row_l_g(rs);
        const int mp = rs - (lp * (lp + 1) - 1);
        const cd rot = eim(e, mp);
        const double2 xa = sx[jj * 2 * NH + rs], xb = sx[jj * 2 * NH + NH + rs];
        const cd xp = rot * mkc(xa.x, xa.y), xm = rot * mkc(xb.x, xb.y);
        for (int ro = 0; ro < NH; ++ro) {
          cd A, B;
          generic_entry(T, rs * NH + ro, s, A, B);
          yp[ro] = yp[ro] + (A + B) * xp;
          yp[NH + ro] = yp[NH + ro] + (A - B) * xm;
        }
      }
      for (int ro = 0; ro < NH; ++ro) {
        const int l = row_l_g(ro);
        const int m = ro - (l * (l + 1) - 1);
        const cd rot = eim(e, -m);
        acc[ro] = acc[ro] + rot * yp[ro];
        acc[NH + ro] = acc[NH + ro] + rot * yp[NH + ro];
      }
    }
  }
  if (active) {
    double2* out = partial + ((size_t)blockIdx.y * N + i) * (2 * NH);
    for (int q = 0; q < 2 * NH; ++q) out[q] = make_double2(acc[q].re, acc[q].im);
  }
}

cudaError_t launch_generic_coupling_fp64(int L, int64_t N, const void* pos, const void* x, void* partial, double k,
                                         int chunks, cudaStream_t st) {
  if (L < 1 || L > kGMaxL) return cudaErrorInvalidValue;
  if (N <= 0) return cudaSuccess;
  TermTableDev T;
  cudaError_t e = get_table(L, T);
  if (e != cudaSuccess) return e;
  if (chunks < 1) chunks = 1;
  const int64_t chunk = (N + chunks - 1) / chunks;
  dim3 grid(static_cast<unsigned>((N + kGBlock - 1) / kGBlock), static_cast<unsigned>(chunks));
  generic_coupling_kernel<<<grid, kGBlock, 0, st>>>(L, T, static_cast<int>(N), static_cast<const Pos4*>(pos),
                                                    static_cast<const double2*>(x), static_cast<double2*>(partial), k,
                                                    static_cast<int>(chunk));
  note_launch();
  return cudaGetLastError();
}

}  // namespace celes
