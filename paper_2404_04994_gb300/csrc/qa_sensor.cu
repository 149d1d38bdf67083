// qa_sensor.cu -- charge-sensor response (Sec. IV.A), fused per pixel after
// the ground state of the non-sensing dots:
//   1. with the dots' charges n_D fixed, each sensor takes the charge that
//      minimises the full energy: the best floor / floor + 1 value around the
//      continuous sensor minimum x_S = c_S - (M_SS)^-1 M_SD (n_D - c_D)
//      (2^S candidates, S <= 4; ties to the lexicographically smaller);
//   2. the sensor potential V_S = (M (n - c))_S, Eq. "potential";
//   3. the line shape around the nearest Coulomb peak, eps = M_ss / 2 - |V_s|:
//      Lorentzian 1 / (1 + (eps / gamma)^2) or Gaussian exp(-eps^2 / 2 gamma^2);
//   4. noise along the fast axis: white, 1/f (Voss-McCartney octaves) and a
//      random telegraph, from a counter-based generator (Philox4x32-10,
//      Salmon et al. 2011), so every value is a pure function of (seed,
//      sensor, row, column).
// FP64 throughout (a few hundred operations per pixel).  One block per raster
// row: the block first marks the row's telegraph switch points in shared
// memory, then its threads take the pixels.
#include "qa_launch.h"
#include "qa_prep.cuh"

namespace qa {

constexpr int kSensorThreads = 128;
constexpr int kSensorMaxW = 8192;
constexpr int kSensorMax = 4;

// Philox4x32-10: ten rounds; each multiplies words 0 and 2 by the two round
// constants, mixes the high halves with words 1 / 3 and the key, and bumps
// the key by the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ uint4 sensor_bits(unsigned long long seed, unsigned tag,
                                             unsigned row, unsigned idx) {
  return philox10(make_uint4(tag, row, idx, 0u),
                  make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

// Box-Muller normal from the first two words.
__device__ __forceinline__ double sensor_gauss(unsigned long long seed, unsigned tag,
                                               unsigned row, unsigned idx) {
  const uint4 b = sensor_bits(seed, tag, row, idx);
  const double u1 = ((double)b.x + 1.0) * 2.3283064365386963e-10;  // (0, 1]
  const double u2 = (double)b.y * 2.3283064365386963e-10;          // [0, 1)
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

struct SensorShared {
  double M[kMaxDot * kMaxDot];
  double Mssi[kSensorMax * kSensorMax];
  unsigned flips[kSensorMax][kSensorMaxW / 32];  // telegraph switch points
  int status;
};

__global__ void __launch_bounds__(kSensorThreads) k_sensor(SensorLaunch L) {
  __shared__ SensorShared sh;
  const ArrayDesc& a = L.a;
  const int nf = a.n, S = L.S, nd = nf - S;
  const int W = a.sc.W;
  const unsigned row = blockIdx.x;
  const int words = (W + 31) / 32;
  for (int e = threadIdx.x; e < nf * nf; e += blockDim.x) sh.M[e] = a.md->M[e];
  for (int e = threadIdx.x; e < kSensorMax * words; e += blockDim.x)
    sh.flips[e / words][e % words] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    // (M_SS)^-1 by Cholesky (S <= 4), column by column
    double Lm[kSensorMax * kSensorMax] = {};
    int ok = 1;
    for (int j = 0; j < S && ok; ++j) {
      double d = sh.M[(nd + j) * nf + nd + j];
      for (int q = 0; q < j; ++q) d -= Lm[j * S + q] * Lm[j * S + q];
      if (!(d > 0.0)) { ok = 0; break; }
      Lm[j * S + j] = sqrt(d);
      for (int i = j + 1; i < S; ++i) {
        double e = sh.M[(nd + i) * nf + nd + j];
        for (int q = 0; q < j; ++q) e -= Lm[i * S + q] * Lm[j * S + q];
        Lm[i * S + j] = e / Lm[j * S + j];
      }
    }
    for (int col = 0; col < S && ok; ++col) {
      double y[kSensorMax];
      for (int i = 0; i < S; ++i) {
        double e = (i == col) ? 1.0 : 0.0;
        for (int q = 0; q < i; ++q) e -= Lm[i * S + q] * y[q];
        y[i] = e / Lm[i * S + i];
      }
      for (int i = S - 1; i >= 0; --i) {
        double e = y[i];
        for (int q = i + 1; q < S; ++q) e -= Lm[q * S + i] * sh.Mssi[q * S + col];
        sh.Mssi[i * S + col] = e / Lm[i * S + i];
      }
    }
    sh.status = ok;
  }
  if (threadIdx.x < S && L.jump_prob > 0.0) {
    // switch points of sensor s in this row: geometric gaps
    const int s = threadIdx.x;
    const double lq = log(1.0 - L.jump_prob);
    long long pos = -1;
    for (unsigned j = 0;; ++j) {
      const uint4 b = sensor_bits(L.seed, 2u | ((unsigned)s << 4), row, j);
      const double u = ((double)b.x + 1.0) * 2.3283064365386963e-10;
      const double g = 1.0 + floor(log(u) / lq);
      if (g > (double)W) break;
      pos += (long long)g;
      if (pos >= W) break;
      sh.flips[s][pos >> 5] ^= 1u << (pos & 31);
    }
  }
  __syncthreads();
  if (!sh.status) {  // M_SS of a positive definite M is positive definite: unreachable
    for (int col = threadIdx.x; col < W; col += blockDim.x)
      for (int s = 0; s < S; ++s) L.out_signal[((long long)row * W + col) * S + s] = __int_as_float(0x7fc00000);
    return;
  }
  for (int col = threadIdx.x; col < W; col += blockDim.x) {
    const long long p = (long long)row * W + col;
    double c[kMaxDot];
    int nv[kMaxDot];
    for (int i = 0; i < nf; ++i) c[i] = pixel_c_f64(a.md, a.ng, a.sc, a.mt.carrier, p, i);
    for (int i = 0; i < nd; ++i) nv[i] = (int)L.n_dots[p * nd + i];
    // b_a = (M_SD (n_D - c_D))_a - (M_SS c_S)_a : E(n_S) = 1/2 n_S M_SS n_S + n_S . b
    double g[kSensorMax], bvec[kSensorMax], xs[kSensorMax];
    for (int s = 0; s < S; ++s) {
      double acc = 0.0;
      for (int j = 0; j < nd; ++j) acc += sh.M[(nd + s) * nf + j] * ((double)nv[j] - c[j]);
      g[s] = acc;
      double mc = 0.0;
      for (int t = 0; t < S; ++t) mc += sh.M[(nd + s) * nf + nd + t] * c[nd + t];
      bvec[s] = acc - mc;
    }
    for (int s = 0; s < S; ++s) {
      double acc = 0.0;
      for (int t = 0; t < S; ++t) acc += sh.Mssi[s * S + t] * g[t];
      xs[s] = c[nd + s] - acc;
    }
    int best[kSensorMax] = {0, 0, 0, 0};
    double bestE = 0.0;
    for (int m = 0; m < (1 << S); ++m) {
      int cand[kSensorMax];
      for (int s = 0; s < S; ++s)
        cand[s] = (int)floor(xs[s] > 0.0 ? xs[s] : 0.0) + ((m >> s) & 1);
      double E = 0.0;
      for (int s = 0; s < S; ++s) {
        double q = 0.0;
        for (int t = 0; t < S; ++t) q += sh.M[(nd + s) * nf + nd + t] * (double)cand[t];
        E += (double)cand[s] * (0.5 * q + bvec[s]);
      }
      bool better = (m == 0) || E < bestE;
      if (m && E == bestE) {
        better = false;
        for (int s = 0; s < S; ++s)
          if (cand[s] != best[s]) { better = cand[s] < best[s]; break; }
      }
      if (better) {
        bestE = E;
        for (int s = 0; s < S; ++s) best[s] = cand[s];
      }
    }
    for (int s = 0; s < S; ++s) nv[nd + s] = best[s];
    for (int s = 0; s < S; ++s) {
      const int q = nd + s;
      double V = 0.0;
      for (int j = 0; j < nf; ++j) V += sh.M[q * nf + j] * ((double)nv[j] - c[j]);
      const double y = (0.5 * sh.M[q * nf + q] - fabs(V)) / L.width;
      double v = L.shape == 1 ? exp(-0.5 * y * y) : 1.0 / (1.0 + y * y);
      if (L.white_sigma > 0.0)
        v += L.white_sigma * sensor_gauss(L.seed, (unsigned)s << 4, row, (unsigned)col);
      if (L.pink_sigma > 0.0) {
        double acc = 0.0;
        for (int k = 0; k < L.K; ++k)
          acc += sensor_gauss(L.seed, 1u | ((unsigned)s << 4) | ((unsigned)k << 8), row,
                              (unsigned)col >> k);
        v += L.pink_sigma * acc / sqrt((double)L.K);
      }
      if (L.jump_prob > 0.0) {
        // telegraph state = parity of the switch points at or before col
        unsigned par = 0u;
        const int wlast = col >> 5;
        for (int w = 0; w < wlast; ++w) par ^= __popc(sh.flips[s][w]) & 1u;
        const unsigned keep = (col & 31) == 31 ? 0xffffffffu : ((2u << (col & 31)) - 1u);
        par ^= __popc(sh.flips[s][wlast] & keep) & 1u;
        if (par) v += L.jump_amplitude;
      }
      L.out_signal[p * S + s] = (float)v;
      if (L.out_n_sensor) L.out_n_sensor[p * S + s] = (int8_t)(best[s] > 127 ? 127 : best[s]);
      if (L.out_potential) L.out_potential[p * S + s] = V;
    }
  }
}

cudaError_t launch_sensor(const SensorLaunch& L, cudaStream_t st) {
  if (L.a.sc.P == 0) return cudaSuccess;
  k_sensor<<<(unsigned)L.a.sc.H, kSensorThreads, 0, st>>>(L);
  return cudaGetLastError();
}

}  // namespace qa
