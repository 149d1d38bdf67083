// qa_brute.cu -- brute-force ground state (Table I, brute-force row): the
// argmin of U(n) = 1/2 (n - c)^T M (n - c) over every n in [0, n_max]^N
// (open) or every n >= 0 with sum n = N_hat (closed), in FP64.  It is the
// exact reference the default and thresholded methods are measured against
// (Sec. VII, Fig. 4) and an on-device exactness check of their maps.
//
// One warp per pixel.  With R the digit range, the free dots (all N open;
// the first N - 1 closed, the last taking N_hat minus the rest) form a
// mixed-radix number, dot 0 most significant, so numeric order of the code is
// lexicographic order of n.  The lanes split the leading (outer) digits; each
// lane walks the trailing `ni` digits in reflected mixed-radix Gray order, one
// digit +-1 per step, updating
//     E(n) = 1/2 n^T M n - n^T d,  d = M c,  y = M n,
//     E(n + s e_i) = E(n) + s (y_i - d_i) + M_ii / 2,   y += s M e_i,
// and rebuilds E and y from scratch at every outer state, so at most R^ni
// FP64 updates separate an energy from an exact evaluation.
#include "qa_launch.h"
#include "qa_prep.cuh"

namespace qa {

constexpr int kBruteThreads = 128;
constexpr int kBruteWarps = kBruteThreads / 32;

struct BruteShared {
  double M[kMaxDot * kMaxDot];
  double c[kBruteWarps][kMaxDot];
  double d[kBruteWarps][kMaxDot];
};

// Digits of code (mixed radix R, nfree digits, dot 0 most significant).
__device__ __forceinline__ void brute_digits(unsigned long long code, int R, int nfree,
                                             int* nv) {
  for (int i = nfree - 1; i >= 0; --i) {
    nv[i] = (int)(code % (unsigned long long)R);
    code /= (unsigned long long)R;
  }
}

__global__ void __launch_bounds__(kBruteThreads) k_brute(BruteLaunch L) {
  __shared__ BruteShared sh;
  const ArrayDesc& a = L.a;
  const int n = a.n;
  const bool closed = a.mt.closed != 0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) sh.M[e] = a.md->M[e];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long p = (long long)blockIdx.x * kBruteWarps + wid;
  const bool active = p < a.sc.P;
  if (active && lane < n) sh.c[wid][lane] = pixel_c_f64(a.md, a.ng, a.sc, a.mt.carrier, p, lane);
  __syncthreads();
  if (active && lane < n) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += sh.M[lane * n + j] * sh.c[wid][j];
    sh.d[wid][lane] = s;
  }
  __syncthreads();
  if (!active) return;
  const double* M = sh.M;
  const double* d = sh.d[wid];
  const int R = L.radix, nfree = L.nfree, ni = L.ni;
  const int last = n - 1;
  const int nhat = a.mt.n_charges;
  unsigned long long rpow_in = 1;  // R^ni
  for (int j = 0; j < ni; ++j) rpow_in *= (unsigned long long)R;

  double e1 = 1.0e300, e2 = 1.0e300;
  unsigned long long c1 = ~0ull;
  for (unsigned long long o = lane; o < L.nouter; o += 32) {
    int nv[kMaxDot];
    brute_digits(o * rpow_in, R, nfree, nv);
    if (closed) {
      int s = 0;
      for (int j = 0; j < nfree; ++j) s += nv[j];
      nv[last] = nhat - s;
    }
    double y[kMaxDot];
    double E = 0.0;
    for (int i = 0; i < n; ++i) {
      double r = 0.0;
      for (int j = 0; j < n; ++j) r += M[i * n + j] * (double)nv[j];
      y[i] = r;
    }
    for (int i = 0; i < n; ++i) E += (double)nv[i] * (0.5 * y[i] - d[i]);
    int dir[kMaxDot];
    for (int j = 0; j < ni; ++j) dir[j] = 1;
    unsigned long long code = o * rpow_in;
    for (;;) {
      const bool valid = !closed || nv[last] >= 0;
      if (valid) {
        if (E < e1 || (E == e1 && code < c1)) {
          e2 = e1;
          e1 = E;
          c1 = code;
        } else if (E < e2) {
          e2 = E;
        }
      }
      // next state: lowest trailing digit that can move in its direction
      int j = 0;
      unsigned long long place = 1;
      while (j < ni) {
        const int i = nfree - 1 - j;
        const int v = nv[i] + dir[j];
        if (v >= 0 && v < R) break;
        dir[j] = -dir[j];
        place *= (unsigned long long)R;
        ++j;
      }
      if (j == ni) break;
      const int i = nfree - 1 - j;
      const int sg = dir[j];
      E += (double)sg * (y[i] - d[i]) + 0.5 * M[i * n + i];
      for (int q = 0; q < n; ++q) y[q] += (double)sg * M[q * n + i];
      nv[i] += sg;
      code = sg > 0 ? code + place : code - place;
      if (closed) {  // the last dot gives the unit back
        E += (double)(-sg) * (y[last] - d[last]) + 0.5 * M[last * n + last];
        for (int q = 0; q < n; ++q) y[q] -= (double)sg * M[q * n + last];
        nv[last] -= sg;
      }
    }
  }
  // warp: best (energy, then smaller code), second-best energy
  for (int off = 16; off > 0; off >>= 1) {
    const double oe1 = __shfl_xor_sync(0xffffffffu, e1, off);
    const double oe2 = __shfl_xor_sync(0xffffffffu, e2, off);
    const unsigned long long oc1 = __shfl_xor_sync(0xffffffffu, c1, off);
    const bool take = oe1 < e1 || (oe1 == e1 && oc1 < c1);
    const double lose = take ? e1 : oe1;
    e2 = fmin(fmin(e2, oe2), lose);
    if (take) { e1 = oe1; c1 = oc1; }
  }
  if (lane != 0) return;
  unsigned flags = 0u;
  if (c1 == ~0ull) {  // no admissible state (cannot happen for valid input)
    flags |= kBruteNone;
    for (int i = 0; i < n; ++i) a.out_n[p * n + i] = 0;
    if (a.out_U) a.out_U[p] = 0.0;
    if (a.out_flags) a.out_flags[p] = (uint8_t)flags;
    return;
  }
  int nv[kMaxDot];
  brute_digits(c1, R, nfree, nv);
  if (closed) {
    int s = 0;
    for (int j = 0; j < nfree; ++j) s += nv[j];
    nv[last] = nhat - s;
  }
  double U = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = 0.0;
    for (int j = 0; j < n; ++j) r += M[i * n + j] * ((double)nv[j] - sh.c[wid][j]);
    U += ((double)nv[i] - sh.c[wid][i]) * r;
    if (!closed && nv[i] == L.n_max) flags |= kBruteAtBox;
  }
  U *= 0.5;
  if (!(e2 - e1 > 1e-9 * fmax(1.0, fabs(U)))) flags |= kBruteNearTie;
  for (int i = 0; i < n; ++i) a.out_n[p * n + i] = (int8_t)nv[i];
  if (a.out_U) a.out_U[p] = U;
  if (a.out_flags) a.out_flags[p] = (uint8_t)flags;
}

cudaError_t launch_brute(const BruteLaunch& L, cudaStream_t st) {
  if (L.a.sc.P == 0) return cudaSuccess;
  const long long blocks = (L.a.sc.P + kBruteWarps - 1) / kBruteWarps;
  k_brute<<<(unsigned)blocks, kBruteThreads, 0, st>>>(L);
  return cudaGetLastError();
}

}  // namespace qa
