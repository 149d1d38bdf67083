// qa_soft.cuh -- finite-temperature occupation (Sec. IV.B, Eq.
// "softargmin") over the method's candidate set, its gradient with the set
// frozen, and the device FP64 Cholesky inverse used when the capacitances are
// updated on the GPU.
//
// Accuracy: at kT = 0.01 an energy error dU moves <n> by up to dU / (4 kT),
// so weights are formed from differences D(b) = U(b) - U(b*) to the minimum
// b*, each a short sum over the slots where b and b* differ, with the
// gradient at b* formed in double-float.  A long incremental walk is never
// used for the weights.
#pragma once

#include "qa_launch.h"
#include "qa_prep.cuh"
#include "qa_search.cuh"

namespace qa {

constexpr unsigned kFullS = 0xffffffffu;
constexpr int kSoftThreads = 128;

__host__ __device__ constexpr int tri(int n) { return n * (n + 1) / 2; }

// length of one pixel's gradient contribution: upper triangle of dL/dM plus
// three N-vectors (sum dc, sum ix dc, sum iy dc)
__host__ __device__ inline int contrib_len(int n) { return tri(n) + 3 * n; }

struct TeamSlots {
  int dot[kMaxDot];
  float h[kMaxDot];
  float gp[kMaxDot];   // g*_s + M_ss / 2  (adding slot s to b*)
  float gm[kMaxDot];   // -g*_s + M_ss / 2 (removing slot s from b*)
  int base[kMaxDot];
  float chi[kMaxDot], clo[kMaxDot];
  unsigned mask;
  int k, w;
  unsigned bstar;
  float ustar_kT;      // U(n*) / kT  (rounded from double-float)
};

// D(b) = E(b) - E(b*) from the slots that differ from b*: the first-order
// terms gp / gm of each and the pair terms between them, read from the team's
// slot-ordered copy of M (Ms[s * KMAX + s2] = M of the dots of slots s, s2).
template <int KMAX>
__device__ __forceinline__ float delta_energy(const TeamSlots& ts, const float* Ms,
                                              unsigned b) {
  const unsigned d = b ^ ts.bstar;
  float D = 0.f;
  for (unsigned m = d; m; m &= m - 1u) {
    const int s = __ffs(m) - 1;
    const bool add = (b >> s) & 1u;
    D += add ? ts.gp[s] : ts.gm[s];
    const float* row = Ms + s * KMAX;
    for (unsigned q = d & ((1u << s) - 1u); q; q &= q - 1u) {
      const int s2 = __ffs(q) - 1;
      const bool add2 = (b >> s2) & 1u;
      const float v = row[s2];
      D += (add == add2) ? v : -v;
    }
  }
  return D;
}

// Soft occupation (forward) and, with BWD, the per-block gradient partials.
template <int L1, int L2, bool CLOSED, bool BWD, int KMAX>
__global__ void __launch_bounds__(kSoftThreads) k_soft(SoftLaunch a) {
  __shared__ ModelConsts cs;
  __shared__ TeamSlots tsm[kSoftThreads / 4 > 0 ? kSoftThreads / 4 : 1];
  // slot-ordered M per team (teams of >= 4 lanes for KMAX 8, 32 lanes beyond)
  constexpr int kMaxTeams = kSoftThreads / (KMAX > 8 ? 32 : 4);
  __shared__ float slotM[kMaxTeams][KMAX * KMAX];
  __shared__ float sQa[BWD ? kMaxTeams : 1][tri(KMAX) + KMAX + 1];  // Qa, va, sa of a team
  extern __shared__ float s_contrib[];  // BWD: [teams][contrib_len]
  const int n = a.n;
  stage_consts(&a.md->k, &cs);
  __syncthreads();
  const float* sM = cs.Mhi;
  const float* sMlo = cs.Mlo;
  const int T = a.cfg.T;  // >= 4
  const int team = threadIdx.x / T, lt = threadIdx.x % T;
  const int teams = blockDim.x / T;
  const long long p = (long long)blockIdx.x * teams + team;
  const bool active = p < a.sc.P;
  TeamSlots& ts = tsm[team];
  const float kT = (float)a.kT;

  if (active && lt == 0) {
    const PixRec& rec = a.recs[p];
    unsigned mask = rec.mask;
    int w = rec.w;
    if (rec.flags & (kFlagBoundary | kFlagQPCap)) {
      // the FP32 candidate set may differ from the exact one: redo it in FP64
      double c[kMaxDot];
      int base[kMaxDot];
      unsigned fl = 0u;
      if (prep_pixel_f64(a.md, n, a.ng, a.sc, a.mt, p, c, base, mask, w, fl) == 0) {
        for (int i = 0; i < n; ++i) {
          double h = 0.0;
          for (int j = 0; j < n; ++j) h += a.md->M[i * n + j] * ((double)base[j] - c[j]);
          ts.base[i] = base[i];
          const df cd = df_from_double(c[i]);
          ts.chi[i] = cd.hi;
          ts.clo[i] = cd.lo;
          ts.h[i] = __double2float_rn(h);
        }
      } else {
        mask = rec.mask;
        w = rec.w;
        for (int i = 0; i < n; ++i) {
          ts.base[i] = rec.base[i];
          ts.chi[i] = rec.chi[i];
          ts.clo[i] = rec.clo[i];
          ts.h[i] = rec.h[i];
        }
        atomicAdd(&a.cnt->unresolved, 1ull);
      }
    } else {
      for (int i = 0; i < n; ++i) {
        ts.base[i] = rec.base[i];
        ts.chi[i] = rec.chi[i];
        ts.clo[i] = rec.clo[i];
        ts.h[i] = rec.h[i];
      }
    }
    // slot order: h of slot s is h of its dot
    int s = 0;
    float hs[kMaxDot];
    for (unsigned m = mask; m; m &= m - 1u) {
      const int i = __ffs(m) - 1;
      ts.dot[s] = i;
      hs[s] = ts.h[i];
      ++s;
    }
    for (int q = 0; q < s; ++q) ts.h[q] = hs[q];  // reuse h[] as slot-ordered
    ts.mask = mask;
    ts.k = s;
    ts.w = CLOSED ? w : -1;
  }
  __syncwarp();
  float* Ms = slotM[team];
  if (active)
    for (int e = lt; e < KMAX * KMAX; e += T) {
      const int s = e / KMAX, s2 = e % KMAX;
      Ms[e] = (s < ts.k && s2 < ts.k) ? sM[ts.dot[s] * kLdM + ts.dot[s2]] : 0.f;
    }
  __syncwarp();

  // pass 1: the minimum-energy candidate b* (from the forward's context when
  // the backward has it)
  const bool use_ctx = BWD && a.ctx_in != nullptr;
  float m1 = kInf, m2 = kInf;
  unsigned b1 = 0u;
  unsigned long long ev = 0;
  if (use_ctx) {
    if (active) b1 = a.ctx_in[p].x;
  } else if (active) {
    SlotView sv{ts.dot, ts.h, ts.k, ts.w};
    search_lane<L1, L2, CLOSED, false>(sM, sv, lt, T, 0.f, nullptr, nullptr, 0u, m1,
                                       b1, m2, ev);
  }
  if (!use_ctx)
    for (int off = 1; off < T; off <<= 1) {
      const float om1 = __shfl_xor_sync(kFullS, m1, off);
      const unsigned ob1 = __shfl_xor_sync(kFullS, b1, off);
      const float om2 = __shfl_xor_sync(kFullS, m2, off);
      top2_merge(m1, b1, m2, om1, ob1, om2);
    }
  // gradient at b* and U(b*) in double-float; lanes split the rows
  df u = {0.f, 0.f};
  if (active) {
    if (lt == 0) ts.bstar = b1;
    int nst[kMaxDot];
#pragma unroll
    for (int i = 0; i < kMaxDot; ++i) {
      int v = 0;
      if (i < n) {
        v = ts.base[i];
        if ((ts.mask >> i) & 1u) v += (int)((b1 >> __popc(ts.mask & ((1u << i) - 1u))) & 1u);
      }
      nst[i] = v;
    }
    df r[kMaxDot];
#pragma unroll
    for (int j = 0; j < kMaxDot; ++j)
      r[j] = (j < n) ? df_sub({(float)nst[j], 0.f}, {ts.chi[j], ts.clo[j]}) : df{0.f, 0.f};
    for (int i = lt; i < n; i += T) {
      df acc = {0.f, 0.f};
#pragma unroll
      for (int j = 0; j < kMaxDot; ++j)
        if (j < n) acc = df_add(acc, df_mul({sM[i * kLdM + j], sMlo[i * kLdM + j]}, r[j]));
      u = df_add(u, df_mul(acc, r[i]));
      if ((ts.mask >> i) & 1u) {
        const int s = __popc(ts.mask & ((1u << i) - 1u));
        const float half = 0.5f * sM[i * kLdM + i];
        ts.gp[s] = (acc.hi + acc.lo) + half;
        ts.gm[s] = half - (acc.hi + acc.lo);
      }
    }
  }
  for (int off = 1; off < T; off <<= 1) {
    df o;
    o.hi = __shfl_xor_sync(kFullS, u.hi, off);
    o.lo = __shfl_xor_sync(kFullS, u.lo, off);
    u = df_add(u, o);
  }
  if (active && lt == 0) {
    const df uk = df_mul_f(u, 0.5f);
    ts.ustar_kT = (float)(df_to_double(uk) / a.kT);
  }
  __syncwarp();

  // pass 2: Boltzmann weights relative to b*
  const int k = active ? ts.k : 0;
  const unsigned total = 1u << k;
  float Z = 0.f;
  float acc[KMAX];
#pragma unroll
  for (int s = 0; s < KMAX; ++s) acc[s] = 0.f;
  const float inv_kT = 1.0f / kT;
  if (use_ctx) {
    if (active) Z = expf(__uint_as_float(a.ctx_in[p].y));
  } else {
    if (active) {
      for (unsigned b = (unsigned)lt; b < total; b += (unsigned)T) {
        if (CLOSED && __popc(b) != ts.w) continue;
        const float wgt = expf(-delta_energy<KMAX>(ts, Ms, b) * inv_kT);
        Z += wgt;
#pragma unroll
        for (int s = 0; s < KMAX; ++s)
          if ((b >> s) & 1u) acc[s] += wgt;
      }
    }
    for (int off = 1; off < T; off <<= 1) {
      Z += __shfl_xor_sync(kFullS, Z, off);
#pragma unroll
      for (int s = 0; s < KMAX; ++s) acc[s] += __shfl_xor_sync(kFullS, acc[s], off);
    }
  }
  if (!BWD) {
    if (active) {
      for (int i = lt; i < n; i += T) {
        float v = (float)ts.base[i];
        if ((ts.mask >> i) & 1u) {
          const int s = __popc(ts.mask & ((1u << i) - 1u));
#pragma unroll
          for (int q = 0; q < KMAX; ++q)
            if (q == s) v += acc[q] / Z;
        }
        a.out_mean[p * n + i] = v;
      }
      if (lt == 0 && a.out_logZ) a.out_logZ[p] = logf(Z) - ts.ustar_kT;
      if (lt == 0 && a.ctx_out) a.ctx_out[p] = make_uint2(ts.bstar, __float_as_uint(logf(Z)));
    }
    return;
  }

  // ---- backward: a_b = -(w_b / kT) (g . n_b - g . <n>), w_b normalised ----
  const int L = contrib_len(n);
  float* my = s_contrib + team * L;
  float gs[KMAX];      // g of each slot's dot
  float gmean = 0.f;   // g . <n>
  float gbase = 0.f;   // g . base
  const float invZ = 1.0f / Z;
#pragma unroll
  for (int s = 0; s < KMAX; ++s) gs[s] = 0.f;
  if (active) {
    const float* g = a.grad_mean + p * n;
    for (int i = 0; i < n; ++i) gbase += g[i] * (float)ts.base[i];
    if (use_ctx) {
      for (int i = 0; i < n; ++i) gmean += g[i] * a.mean_in[p * n + i];
    } else {
      gmean = gbase;
#pragma unroll
      for (int s = 0; s < KMAX; ++s)
        if (s < k) gmean += g[ts.dot[s]] * acc[s] * invZ;
    }
#pragma unroll
    for (int s = 0; s < KMAX; ++s)
      if (s < k) gs[s] = g[ts.dot[s]];
  }
  float sa = 0.f;
  float va[KMAX];
  float Qa[tri(KMAX)];
#pragma unroll
  for (int s = 0; s < KMAX; ++s) va[s] = 0.f;
#pragma unroll
  for (int e = 0; e < tri(KMAX); ++e) Qa[e] = 0.f;
  if (active) {
    for (unsigned b = (unsigned)lt; b < total; b += (unsigned)T) {
      if (CLOSED && __popc(b) != ts.w) continue;
      const float wgt = expf(-delta_energy<KMAX>(ts, Ms, b) * inv_kT) * invZ;
      float gn = gbase;
#pragma unroll
      for (int s = 0; s < KMAX; ++s)
        if ((b >> s) & 1u) gn += gs[s];
      const float av = -(wgt * inv_kT) * (gn - gmean);
      sa += av;
#pragma unroll
      for (int s = 0; s < KMAX; ++s) {
        if ((b >> s) & 1u) {
          va[s] += av;
#pragma unroll
          for (int s2 = s; s2 < KMAX; ++s2)
            if ((b >> s2) & 1u) Qa[s * KMAX - s * (s - 1) / 2 + (s2 - s)] += av;
        }
      }
    }
  }
  for (int off = 1; off < T; off <<= 1) {
    sa += __shfl_xor_sync(kFullS, sa, off);
#pragma unroll
    for (int s = 0; s < KMAX; ++s) va[s] += __shfl_xor_sync(kFullS, va[s], off);
#pragma unroll
    for (int e = 0; e < tri(KMAX); ++e) Qa[e] += __shfl_xor_sync(kFullS, Qa[e], off);
  }
  // pixel contribution: dM_p = 1/2 [sa r0 r0^T + r0 va^T + va r0^T + Qa],
  // rho = sa r0 + va, dc_p = -M rho (dot coordinates); the team's lanes split
  // the entries
  float* q_s = sQa[BWD ? team : 0];
  if (lt == 0) {
#pragma unroll
    for (int e = 0; e < tri(KMAX); ++e) q_s[e] = Qa[e];
#pragma unroll
    for (int s = 0; s < KMAX; ++s) q_s[tri(KMAX) + s] = va[s];
    q_s[tri(KMAX) + KMAX] = sa;
  }
  __syncwarp();
  const unsigned tmask = active ? ts.mask : 0u;
  auto slot_of = [&](int i) { return __popc(tmask & ((1u << i) - 1u)); };
  auto r0_of = [&](int i) {
    const df rr = df_sub({(float)ts.base[i], 0.f}, {ts.chi[i], ts.clo[i]});
    return rr.hi + rr.lo;
  };
  auto vd_of = [&](int i) { return ((tmask >> i) & 1u) ? q_s[tri(KMAX) + slot_of(i)] : 0.f; };
  const float sa_t = q_s[tri(KMAX) + KMAX];
  for (int e = lt; e < tri(n); e += T) {
    if (!active) { my[e] = 0.f; continue; }
    int i = 0, rem = e;
    while (rem >= n - i) { rem -= n - i; ++i; }
    const int j = i + rem;
    const float ri = r0_of(i), rj = r0_of(j);
    float q = sa_t * ri * rj + ri * vd_of(j) + vd_of(i) * rj;
    if (((tmask >> i) & 1u) && ((tmask >> j) & 1u)) {
      const int s = slot_of(i), s2 = slot_of(j);  // s <= s2: slots in dot order
      q += q_s[s * KMAX - s * (s - 1) / 2 + (s2 - s)];
    }
    my[e] = 0.5f * q;
  }
  for (int i = lt; i < n; i += T) {
    if (!active) {
      my[tri(n) + i] = my[tri(n) + n + i] = my[tri(n) + 2 * n + i] = 0.f;
      continue;
    }
    float dc = 0.f;
    for (int j = 0; j < n; ++j) dc -= sM[i * kLdM + j] * (sa_t * r0_of(j) + vd_of(j));
    const int ix = (int)(p % a.sc.W), iy = (int)(p / a.sc.W);
    my[tri(n) + i] = dc;
    my[tri(n) + n + i] = dc * (float)ix;
    my[tri(n) + 2 * n + i] = dc * (float)iy;
  }
  __syncthreads();
  // block sum over teams in fixed order (double-float), one partial per block
  float* out = a.partials + (size_t)blockIdx.x * 2 * L;
  for (int e = threadIdx.x; e < L; e += blockDim.x) {
    df sacc = {0.f, 0.f};
    for (int q = 0; q < teams; ++q) sacc = df_add(sacc, {s_contrib[q * L + e], 0.f});
    out[2 * e] = sacc.hi;
    out[2 * e + 1] = sacc.lo;
  }
}

// Second stage: one block per contribution e sums the block partials --
// thread j takes blocks j, j + 256, ... in order, then a fixed shared-memory
// tree -- so the result does not depend on scheduling.
static __global__ void __launch_bounds__(256) k_soft_reduce(SoftLaunch a, int nblocks) {
  __shared__ df red[256];
  const int e = blockIdx.x;
  const int L = contrib_len(a.n);
  df acc = {0.f, 0.f};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    const float* pb = a.partials + (size_t)b * 2 * L;
    acc = df_add(acc, {pb[2 * e], pb[2 * e + 1]});
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int half = blockDim.x / 2; half > 0; half >>= 1) {
    if ((int)threadIdx.x < half) red[threadIdx.x] = df_add(red[threadIdx.x], red[threadIdx.x + half]);
    __syncthreads();
  }
  if (threadIdx.x == 0) a.sums[e] = df_to_double(red[0]);
}

// Third stage: the chain rule through M = Cdd^-1 and c = s Cgd V:
//   dL/dCdd = -M (dL/dM) M,  dL/dCgd = s (S0 V0'^T + S1 (dx u)^T + S2 (dy w)^T)
// with V0' = V0 + x0 u + y0 w and S0, S1, S2 the sums of dc, ix dc, iy dc.
static __global__ void k_soft_finalize(SoftLaunch a) {
  __shared__ double sG[kMaxDot * kMaxDot];
  __shared__ double sS[3 * kMaxDot];
  const int n = a.n, ng = a.ng;
  const int L = contrib_len(n);
  for (int e = threadIdx.x; e < L; e += blockDim.x) {
    const double v = a.sums[e];
    if (e < tri(n)) {
      // e -> (i, j), i <= j
      int i = 0, rem = e;
      while (rem >= n - i) { rem -= n - i; ++i; }
      const int j = i + rem;
      sG[i * n + j] = v;
      sG[j * n + i] = v;
    } else {
      sS[e - tri(n)] = v;
    }
  }
  __syncthreads();
  const double* M = a.md->M;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    double s = 0.0;
    for (int p = 0; p < n; ++p) {
      double t = 0.0;
      for (int q = 0; q < n; ++q) t += sG[p * n + q] * M[q * n + j];
      s += M[i * n + p] * t;
    }
    a.dL_dCdd[e] = -s;
  }
  for (int e = threadIdx.x; e < n * ng; e += blockDim.x) {
    const int i = e / ng, g = e % ng;
    const double v0 = a.sc.V0[g] + a.sc.x0 * a.sc.u[g] + a.sc.y0 * a.sc.w[g];
    const double v = sS[i] * v0 + sS[n + i] * a.sc.dx * a.sc.u[g] +
                     sS[2 * n + i] * a.sc.dy * a.sc.w[g];
    a.dL_dCgd[e] = a.mt.carrier * v;
  }
}

inline size_t soft_partials_floats_impl(int n, long long P, const SearchCfg& cfg) {
  const int teams = kSoftThreads / cfg.T;
  const long long blocks = (P + teams - 1) / teams;
  return (size_t)blocks * 2 * (size_t)contrib_len(n);
}

template <int L1, int L2, bool CLOSED, bool BWD, int KMAX>
static cudaError_t run_soft(const SoftLaunch& a, cudaStream_t st) {
  const int teams = kSoftThreads / a.cfg.T;
  const long long P = a.sc.P;
  const unsigned grid = (unsigned)((P + teams - 1) / teams);
  const size_t smem = BWD ? (size_t)teams * contrib_len(a.n) * sizeof(float) : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_soft<L1, L2, CLOSED, BWD, KMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (a.ev) cudaEventRecord(a.ev[0], st);
  k_soft<L1, L2, CLOSED, BWD, KMAX><<<grid, kSoftThreads, smem, st>>>(a);
  if (BWD) {
    k_soft_reduce<<<contrib_len(a.n), 256, 0, st>>>(a, (int)grid);
    k_soft_finalize<<<1, 256, 0, st>>>(a);
  }
  if (a.ev) cudaEventRecord(a.ev[1], st);
  return cudaGetLastError();
}

template <bool BWD>
static cudaError_t dispatch_soft(const SoftLaunch& a, cudaStream_t st) {
  // The search here only locates b*, so two splits suffice: (4, 0) for up
  // to four dots and (5, 4) beyond (any k works with either).
  const bool cl = a.mt.closed != 0;
  if (a.n <= 4)
    return cl ? run_soft<4, 0, true, BWD, 8>(a, st) : run_soft<4, 0, false, BWD, 8>(a, st);
  if (a.n <= 8)
    return cl ? run_soft<5, 4, true, BWD, 8>(a, st) : run_soft<5, 4, false, BWD, 8>(a, st);
  return cl ? run_soft<5, 4, true, BWD, 16>(a, st) : run_soft<5, 4, false, BWD, 16>(a, st);
}

}  // namespace qa
