// qa_soft.cuh -- finite-temperature occupation (Sec. IV.B, Eq.
// "softargmin") over the method's candidate set, its gradient with the set
// frozen, and the device FP64 inverse used when the capacitances are
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

// length of one pixel's gradient contribution: upper triangle of dL/dM,
// three N-vectors (sum dc, sum ix dc, sum iy dc) and, last, the pixel's loss
// term of a fit step (0 otherwise)
__host__ __device__ inline int contrib_len(int n) { return tri(n) + 3 * n + 1; }

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

// v[s] for a runtime s, the array staying in registers.
template <int K>
__device__ __forceinline__ float pick(const float (&v)[K], int s) {
  float r = 0.f;
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (q == s) r = v[q];
  return r;
}

// Fit step: the pixel's <n> from the slot weight sums accb (slot order) and
// Z, then the MSE gradient g = dL/d<n> into gsh[0, n); returns the pixel's
// squared residual (summed over the team).  Sum target: r = sum_i <n_i> -
// target_p and g_i = scale r for every dot; per-dot target: r_i = <n_i> -
// target_pi and g_i = scale r_i.  The team's lanes take the dots; all lanes
// of the warp call.
template <int K>
__device__ __forceinline__ float fit_loss_grad_team(const SoftLaunch& a, const TeamSlots& ts,
                                                    const float (&accb)[K], float Z,
                                                    long long p, float* gsh, int lt, int T,
                                                    bool active) {
  const int n = a.n;
  float part = 0.f;
  if (active)
    for (int i = lt; i < n; i += T) {
      float v = (float)ts.base[i];
      if ((ts.mask >> i) & 1u) v += pick<K>(accb, __popc(ts.mask & ((1u << i) - 1u))) / Z;
      if (a.out_mean) a.out_mean[p * n + i] = v;
      if (a.fit_per_dot) {
        const float r = v - a.fit_target[p * n + i];
        gsh[i] = a.fit_scale * r;
        part = fmaf(r, r, part);
      } else {
        part += v;
      }
    }
  for (int off = 1; off < T; off <<= 1) part += __shfl_xor_sync(kFullS, part, off);
  float lossp = part;
  if (!a.fit_per_dot) {
    const float r = active ? part - a.fit_target[p] : 0.f;
    if (active)
      for (int i = lt; i < n; i += T) gsh[i] = a.fit_scale * r;
    lossp = r * r;
  }
  __syncwarp();
  return active ? lossp : 0.f;
}

// Lane 0 of a team: pixel p's record into the team's slots (slot order: the
// s-th ambiguous dot; h[] reused slot-ordered).  A pixel whose FP32 candidate
// set may differ from the exact one is prepared again in FP64.
template <bool CLOSED>
__device__ __noinline__ void soft_setup(const SoftLaunch& a, TeamSlots& ts, long long p) {
  const int n = a.n;
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

// The same, the team's lanes splitting the dots of the common case (the FP64
// redo of a doubtful pixel stays with lane 0); all lanes of the warp call.
template <bool CLOSED>
__device__ inline void soft_setup_team(const SoftLaunch& a, TeamSlots& ts, long long p, int lt,
                                       int T, bool active) {
  if (active) {
    const PixRec& rec = a.recs[p];
    if (rec.flags & (kFlagBoundary | kFlagQPCap)) {
      if (lt == 0) soft_setup<CLOSED>(a, ts, p);
    } else {
      const int n = a.n;
      const unsigned mask = rec.mask;
      for (int i = lt; i < n; i += T) {
        ts.base[i] = rec.base[i];
        ts.chi[i] = rec.chi[i];
        ts.clo[i] = rec.clo[i];
        if ((mask >> i) & 1u) {
          const int s = __popc(mask & ((1u << i) - 1u));
          ts.dot[s] = i;
          ts.h[s] = rec.h[i];  // h[] slot-ordered
        }
      }
      if (lt == 0) {
        ts.mask = mask;
        ts.k = __popc(mask);
        ts.w = CLOSED ? rec.w : -1;
      }
    }
  }
  __syncwarp();
}

// The gradient at b* (gp / gm of every slot) and U(b*) / kT in double-float,
// the team's lanes splitting the rows; all lanes of the warp call.
template <int ND>  // dots at most (the arrays below are unrolled to ND)
__device__ inline void soft_anchor(const SoftLaunch& a, TeamSlots& ts, const float* sM,
                                   const float* sMlo, int T, int lt, bool active, unsigned b1) {
  const int n = a.n;
  df u = {0.f, 0.f};
  if (active) {
    if (lt == 0) ts.bstar = b1;
    int nst[ND];
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      int v = 0;
      if (i < n) {
        v = ts.base[i];
        if ((ts.mask >> i) & 1u) v += (int)((b1 >> __popc(ts.mask & ((1u << i) - 1u))) & 1u);
      }
      nst[i] = v;
    }
    df r[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j)
      r[j] = (j < n) ? df_sub({(float)nst[j], 0.f}, {ts.chi[j], ts.clo[j]}) : df{0.f, 0.f};
    for (int i = lt; i < n; i += T) {
      df acc = {0.f, 0.f};
#pragma unroll
      for (int j = 0; j < ND; ++j)
        if (j < n) acc = df_add(acc, df_mul({sM[i * kLdM + j], sMlo[i * kLdM + j]}, r[j]));
      int ni = ts.base[i];
      if ((ts.mask >> i) & 1u) ni += (int)((b1 >> __popc(ts.mask & ((1u << i) - 1u))) & 1u);
      u = df_add(u, df_mul(acc, df_sub({(float)ni, 0.f}, {ts.chi[i], ts.clo[i]})));
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
}

// The pixel's gradient contribution from its candidate moments in slot
// coordinates (q_s: Qa upper triangle, va, sa; see k_soft), the team's lanes
// splitting the entries into my[], then the block's partial: the teams'
// contributions summed in a fixed order (double-float), one per block.  All
// threads of the block call.
template <int KMAX>
__device__ inline void soft_contrib(const SoftLaunch& a, TeamSlots& ts, const float* q_s,
                                    float* my, const float* s_contrib, const float* sM, int T,
                                    int lt, int teams, bool active, long long p, float lossp) {
  const int n = a.n;
  const int L = contrib_len(n);
  const unsigned tmask = active ? ts.mask : 0u;
  auto slot_of = [&](int i) { return __popc(tmask & ((1u << i) - 1u)); };
  const float sa_t = q_s[tri(KMAX) + KMAX];
  // per dot, in the team's rows that are dead by now: r0_i = base_i - c_i,
  // va_i (charge coordinates, dot order) and rho_i = sa r0_i + va_i
  float* r0 = ts.gp;
  float* vd = ts.h;
  float* rho = ts.gm;
  if (active)
    for (int i = lt; i < n; i += T) {
      const df rr = df_sub({(float)ts.base[i], 0.f}, {ts.chi[i], ts.clo[i]});
      const float ri = rr.hi + rr.lo;
      const float vi = ((tmask >> i) & 1u) ? q_s[tri(KMAX) + slot_of(i)] : 0.f;
      r0[i] = ri;
      vd[i] = vi;
      rho[i] = sa_t * ri + vi;
    }
  __syncwarp();
  // dM_ij = 1/2 (r0_i rho_j + va_i r0_j + Qa_ij)
  for (int e = lt; e < tri(n); e += T) {
    if (!active) { my[e] = 0.f; continue; }
    int i = 0, rem = e;
    while (rem >= n - i) { rem -= n - i; ++i; }
    const int j = i + rem;
    float q = r0[i] * rho[j] + vd[i] * r0[j];
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
    for (int j = 0; j < n; ++j) dc -= sM[i * kLdM + j] * rho[j];
    const int ix = (int)(p % a.sc.W), iy = (int)(p / a.sc.W);
    my[tri(n) + i] = dc;
    my[tri(n) + n + i] = dc * (float)ix;
    my[tri(n) + 2 * n + i] = dc * (float)iy;
  }
  if (lt == 0) my[L - 1] = active ? lossp : 0.f;
  __syncthreads();
  // block sum over teams in fixed order (double-float), one partial per
  // block, stored entry-major ([e][block]) so that the reduction of an entry
  // reads its partials contiguously
  float2* out = reinterpret_cast<float2*>(a.partials);
  for (int e = threadIdx.x; e < L; e += blockDim.x) {
    df sacc = {0.f, 0.f};
    for (int q = 0; q < teams; ++q) sacc = df_add(sacc, {s_contrib[q * L + e], 0.f});
    out[(size_t)e * gridDim.x + blockIdx.x] = make_float2(sacc.hi, sacc.lo);
  }
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
  __shared__ float sGf[BWD ? kMaxTeams : 1][kMaxDot];                 // fit step: g of a team
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

  soft_setup_team<CLOSED>(a, ts, p, lt, T, active);
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
  soft_anchor<kMaxDot>(a, ts, sM, sMlo, T, lt, active, b1);

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
  const bool fit = a.fit_target != nullptr;
  float lossp = 0.f;
  if (fit) lossp = fit_loss_grad_team<KMAX>(a, ts, acc, Z, p, sGf[team], lt, T, active);
  if (active) {
    const float* g = fit ? sGf[team] : a.grad_mean + p * n;
    for (int i = 0; i < n; ++i) gbase += g[i] * (float)ts.base[i];
#pragma unroll
    for (int s = 0; s < KMAX; ++s)
      if (s < k) gs[s] = g[ts.dot[s]];
    if (use_ctx) {
      for (int i = 0; i < n; ++i) gmean += g[i] * a.mean_in[p * n + i];
    } else {
      // g . <n> - g . base = sum_s g_s <b_s>, so that gn - gmean below is
      // formed without the large g . base on both sides
      gmean = 0.f;
#pragma unroll
      for (int s = 0; s < KMAX; ++s)
        if (s < k) gmean += gs[s] * acc[s] * invZ;
      gbase = 0.f;
    }
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
  soft_contrib<KMAX>(a, ts, q_s, my, s_contrib, sM, T, lt, teams, active, p, lossp);
}

// ---------------------------------------------------------------------------
// Dense soft occupation for arrays of at most 8 dots (k <= 8 ambiguous
// slots): a team of 8 lanes per pixel, lane t taking the patterns whose
// slots 5..7 are the bits of t and, for each, the 32 patterns of slots 0..4
// from a table.  Both passes evaluate a quadratic pseudo-Boolean function
//   F(d) = sum_{s in d} G_s + sum_{s < s' in d} W_ss'
// over every pattern d: the lane forms the rest value A = F(d_out) and the
// inner coefficients q_j = G_j + sum_{o in d_out} W_jo, then F(d) = A +
// sum_{j in d_in} q_j + Pw[d_in] by doubling, Pw[d_in] the pair terms among
// the inner slots -- the terms of the per-candidate sums, in another order.
//   pass 1 (b*): F = E(b) - E(base): G_s = h_s + M_ss / 2, W = M;
//   pass 2: F = D(d) = E(b* xor d) - E(b*): G_s = gp_s where b* lacks slot s
//     (adding it) or gm_s where it has it (removing it), W_ss' = sg_s sg_s'
//     M_ss' with sg_s = +1 / -1 likewise.
// The weights w(d) = exp(-D(d) / kT) of a lane go through a superset sum over
// the inner bits, Wz[S] = sum_{d_in contains S} w(d), which yields Z and the
// moments sum_d w(d) d_S in flip coordinates; with the gradient of the
// backward, a_b = -(w_b / (kT Z)) (g . n_b - g . <n>) and g . n_b = g . n* +
// sum_s gam_s d_s (gam_s = sg_s g_s), so that
//   sum_b a_b d_S = -(1 / (kT Z)) (c0 M(S) + sum_j gam_j M(S u {j})),
// M(S) = sum_d w(d) d_S, c0 = g . n* - g . <n>, for |S| <= 2; the charge
// coordinates follow from n_s = n*_s + sg_s d_s.  Per candidate this costs
// about three adds and an exponential instead of a sum over the slots that
// differ from b* and a triangle of moment updates.
// ---------------------------------------------------------------------------
constexpr int kDenseT = 8;    // lanes per pixel
constexpr int kDenseIn = 5;   // inner slots: a table of 32 patterns
constexpr int kDenseMax = 8;  // slots

constexpr int kMom = 1 + kDenseMax + tri(kDenseMax - 1);  // |S| <= 2 moments: 37
constexpr int kMomPad = 40;                                 // ... padded to 5 per lane

// Superset sum over NB bits in place: w[S] <- sum over b containing S of w[b].
template <int NB>
__device__ __forceinline__ void superset_sum(float (&w)[1 << NB]) {
#pragma unroll
  for (int j = 0; j < NB; ++j)
#pragma unroll
    for (int b = 0; b < (1 << NB); ++b)
      if (!((b >> j) & 1)) w[b] += w[b | (1 << j)];
}

// Sum of X[0, N) over a team of 8 lanes, scattered: three halving exchanges
// (partners 4, 2, 1), after which each lane holds N / 8 of the sums, written
// to out[] where the index is below nout.  All lanes of the warp call.
template <int N>
__device__ __forceinline__ void team_reduce_scatter8(float (&X)[N], int lt, float* out,
                                                     int nout) {
  static_assert(N % 8 == 0, "N must be a multiple of 8");
  constexpr int H1 = N / 2, H2 = N / 4, H3 = N / 8;
  const bool b2 = (lt >> 2) & 1, b1 = (lt >> 1) & 1, b0 = lt & 1;
#pragma unroll
  for (int i = 0; i < H1; ++i) {
    const float send = b2 ? X[i] : X[H1 + i];
    const float keep = b2 ? X[H1 + i] : X[i];
    X[i] = keep + __shfl_xor_sync(kFullS, send, 4);
  }
#pragma unroll
  for (int i = 0; i < H2; ++i) {
    const float send = b1 ? X[i] : X[H2 + i];
    const float keep = b1 ? X[H2 + i] : X[i];
    X[i] = keep + __shfl_xor_sync(kFullS, send, 2);
  }
#pragma unroll
  for (int i = 0; i < H3; ++i) {
    const float send = b0 ? X[i] : X[H3 + i];
    const float keep = b0 ? X[H3 + i] : X[i];
    X[i] = keep + __shfl_xor_sync(kFullS, send, 1);
  }
  const int base = (b2 ? H1 : 0) + (b1 ? H2 : 0) + (b0 ? H3 : 0);
#pragma unroll
  for (int i = 0; i < H3; ++i)
    if (base + i < nout) out[base + i] = X[i];
}

// F of the 32 inner patterns for the lane's outer pattern tout (slots 5..7).
// G / sg per slot, Ms the team's slot-ordered M (zero beyond the k slots,
// where G is kBig so that no pattern using such a slot counts).
__device__ __forceinline__ void dense_table(const float* G, const float* sg, const float* Ms,
                                            unsigned tout, float* F) {
  constexpr int K = kDenseMax, NI = 1 << kDenseIn, NO = K - kDenseIn;
  float po[NO];
#pragma unroll
  for (int i = 0; i < NO; ++i) po[i] = ((tout >> i) & 1u) ? 1.f : 0.f;
  // rest value and inner coefficients: 0 / 1-weighted sums over the outer
  // slots in increasing order
  float A = 0.f;
  float q[kDenseIn];
#pragma unroll
  for (int j = 0; j < kDenseIn; ++j) q[j] = G[j];
#pragma unroll
  for (int i = 0; i < NO; ++i) {
    const int o = kDenseIn + i;
    float add = G[o];
#pragma unroll
    for (int i2 = 0; i2 < i; ++i2)
      add = fmaf(po[i2], sg[o] * sg[kDenseIn + i2] * Ms[o * K + kDenseIn + i2], add);
    A = fmaf(po[i], add, A);
#pragma unroll
    for (int j = 0; j < kDenseIn; ++j) q[j] = fmaf(po[i], sg[j] * sg[o] * Ms[j * K + o], q[j]);
  }
  // pair terms among the inner slots
  float P[NI];
  P[0] = 0.f;
#pragma unroll
  for (int j = 0; j < kDenseIn; ++j) {
    float Wj[kDenseIn];
#pragma unroll
    for (int l = 0; l < j; ++l) Wj[l] = sg[j] * sg[l] * Ms[j * K + l];
#pragma unroll
    for (int b = 0; b < (1 << j); ++b) {
      float r = 0.f;
#pragma unroll
      for (int l = 0; l < j; ++l)
        if ((b >> l) & 1) r += Wj[l];
      P[b | (1 << j)] = P[b] + r;
    }
  }
  // doubling over the inner slots, then the pair terms
  F[0] = A;
#pragma unroll
  for (int j = 0; j < kDenseIn; ++j)
#pragma unroll
    for (int b = 0; b < (1 << j); ++b) F[b | (1 << j)] = F[b] + q[j];
#pragma unroll
  for (int b = 1; b < NI; ++b) F[b] += P[b];
}

// Threads per block of the dense kernel; its per-team arrays live in one
// dynamic shared buffer laid out by DenseSmem.
#ifndef QA_DENSE_THREADS
#define QA_DENSE_THREADS 128
#endif
constexpr int kDenseThreads = QA_DENSE_THREADS;
static_assert(kDenseThreads % 32 == 0 && kDenseThreads <= 1024 && kDenseThreads >= kSoftThreads,
              "dense block size (the partials are sized for kSoftThreads)");

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

struct DenseSmem {
  size_t slots, slotM, qa, qd, gf, wr, contrib, total;
  __host__ __device__ constexpr DenseSmem(bool bwd, int L)
      : slots(0),
        slotM(al16(sizeof(TeamSlots) * (kDenseThreads / kDenseT))),
        qa(slotM + al16(sizeof(float) * (kDenseThreads / kDenseT) * kDenseMax * kDenseMax)),
        qd(qa + (bwd ? al16(sizeof(float) * (kDenseThreads / kDenseT) * (tri(kDenseMax) + kDenseMax + 1)) : 0)),
        gf(qd + (bwd ? al16(sizeof(float) * (kDenseThreads / kDenseT) * kMom) : 0)),
        wr(gf + (bwd ? al16(sizeof(float) * (kDenseThreads / kDenseT) * kMaxDot) : 0)),
        contrib(wr + (bwd ? al16(sizeof(float) * kDenseThreads * ((1 << kDenseIn) + 4)) : 0)),
        total(contrib + (bwd ? al16(sizeof(float) * (kDenseThreads / kDenseT) * L) : 0)) {}
};

// what a launch of the dense kernel computes: the forward; the backward from
// grad_mean; the backward given the forward's context; the fused fit step
enum DenseMode { kDenseFwd = 0, kDenseBwd = 1, kDenseBwdCtx = 2, kDenseFit = 3 };

// five blocks of 128 threads per SM: at most 102 registers a thread
template <bool CLOSED, int MODE>
__global__ void __launch_bounds__(kDenseThreads, 640 / kDenseThreads) k_soft_dense(SoftLaunch a) {
  constexpr bool BWD = MODE != kDenseFwd;
  constexpr int K = kDenseMax, NI = 1 << kDenseIn;
  constexpr int kTeams = kDenseThreads / kDenseT;
  // of the model constants only M as double-float (hi, lo)
  __shared__ __align__(16) float sMh[kMaxDot * kLdM], sMl[kMaxDot * kLdM];
  extern __shared__ __align__(16) unsigned char s_dyn[];
  const int n = a.n;
  const DenseSmem lay(BWD, contrib_len(n));
  TeamSlots* tsm = reinterpret_cast<TeamSlots*>(s_dyn + lay.slots);
  float* slotM = reinterpret_cast<float*>(s_dyn + lay.slotM);  // [team][K * K]
  float* sQa = reinterpret_cast<float*>(s_dyn + lay.qa);       // [team][tri(K) + K + 1]: Qa, va, sa
  float* sQd = reinterpret_cast<float*>(s_dyn + lay.qd);       // [team][kMom]: the same, flip coords
  float* sGf = reinterpret_cast<float*>(s_dyn + lay.gf);       // [team][kMaxDot]: fit step g
  float* sWr = reinterpret_cast<float*>(s_dyn + lay.wr);       // [thread][NI + 4]: raw weights
  float* s_contrib = reinterpret_cast<float*>(s_dyn + lay.contrib);  // [team][contrib_len]
  static_assert((kMaxDot * kLdM) % 4 == 0, "float4 staging");
  for (int e = threadIdx.x; e < kMaxDot * kLdM / 4; e += blockDim.x) {
    reinterpret_cast<float4*>(sMh)[e] = reinterpret_cast<const float4*>(a.md->k.Mhi)[e];
    reinterpret_cast<float4*>(sMl)[e] = reinterpret_cast<const float4*>(a.md->k.Mlo)[e];
  }
  __syncthreads();
  const float* sM = sMh;
  const float* sMlo = sMl;
  const int T = kDenseT;
  const int team = threadIdx.x / T, lt = threadIdx.x % T;
  const long long p = (long long)blockIdx.x * kTeams + team;
  const bool active = p < a.sc.P;
  TeamSlots& ts = tsm[team];
  const float kT = (float)a.kT;

  soft_setup_team<CLOSED>(a, ts, p, lt, T, active);
  float* Ms = slotM + team * (K * K);
  if (active)
    for (int e = lt; e < K * K; e += T) {
      const int s = e / K, s2 = e % K;
      Ms[e] = (s < ts.k && s2 < ts.k) ? sM[ts.dot[s] * kLdM + ts.dot[s2]] : 0.f;
    }
  __syncwarp();
  const int k = active ? ts.k : 0;
  const int kout = k > kDenseIn ? k - kDenseIn : 0;
  const unsigned tout = (unsigned)lt;                 // the lane's bits of slots 5..7
  const bool lane_on = active && lt < (1 << kout);
  const int wcl = (CLOSED && active) ? ts.w : 0;

  // pass 1: b* (from the forward's context when the backward has it)
  constexpr bool use_ctx = MODE == kDenseBwdCtx;
  unsigned b1 = 0u;
  if (use_ctx) {
    if (active) b1 = a.ctx_in[p].x;
  } else {
    float G[K], sg[K], F[NI];
#pragma unroll
    for (int s = 0; s < K; ++s) {
      G[s] = s < k ? ts.h[s] + 0.5f * Ms[s * K + s] : kBig;
      sg[s] = 1.f;
    }
    dense_table(G, sg, Ms, tout, F);
    float e1 = kInf, e2 = kInf;
    unsigned bb = 0u;
    if (lane_on) {
      const int pout = __popc(tout);
#pragma unroll
      for (int b = 0; b < NI; ++b) {
        if (CLOSED && popc_c((unsigned)b) + pout != wcl) continue;
        if (F[b] < e1) { e1 = F[b]; bb = (unsigned)b; }
      }
    }
    b1 = bb | (tout << kDenseIn);
    for (int off = 1; off < T; off <<= 1) {
      const float o1 = __shfl_xor_sync(kFullS, e1, off);
      const unsigned ob = __shfl_xor_sync(kFullS, b1, off);
      const float o2 = __shfl_xor_sync(kFullS, e2, off);
      top2_merge(e1, b1, e2, o1, ob, o2);
    }
  }
  soft_anchor<kDenseMax>(a, ts, sM, sMlo, T, lt, active, b1);

  // pass 2: weights relative to b*, superset sums over the inner bits
  const unsigned bst = active ? ts.bstar : 0u;
  float w[NI];
  float sgn[K];
  {
    float G[K];
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const bool has = (bst >> s) & 1u;
      G[s] = s < k ? (has ? ts.gm[s] : ts.gp[s]) : kBig;
      sgn[s] = has ? -1.f : 1.f;
    }
    dense_table(G, sgn, Ms, tout, w);
  }
  const float c2 = -1.4426950408889634f / kT;  // exp(-D / kT) = 2^(c2 D)
  {
    const unsigned bst_in = bst & (unsigned)(NI - 1), bst_out = bst >> kDenseIn;
    const int r_need = wcl - __popc(bst_out ^ tout);
#pragma unroll
    for (int b = 0; b < NI; ++b) {
      const bool ok = lane_on && (!CLOSED || __popc(bst_in ^ (unsigned)b) == r_need);
      w[b] = ok ? exp2f(c2 * w[b]) : 0.f;
    }
  }
  // the backward needs the raw weights again once the gradient is known
  float* wraw = sWr + threadIdx.x * (NI + 4);
  if (BWD) {
#pragma unroll
    for (int b = 0; b < NI; b += 4)
      *reinterpret_cast<float4*>(wraw + b) = make_float4(w[b], w[b + 1], w[b + 2], w[b + 3]);
  }
  superset_sum<kDenseIn>(w);
  // the lane's outer slots present (1) or absent (0)
  float po[K - kDenseIn];
#pragma unroll
  for (int i = 0; i < K - kDenseIn; ++i) po[i] = (lane_on && ((tout >> i) & 1u)) ? 1.f : 0.f;

  // Z and the first moments in flip coordinates, summed over the team
  float Z = w[0];
  float md[K];
#pragma unroll
  for (int s = 0; s < K; ++s) md[s] = s < kDenseIn ? w[1 << s] : po[s - kDenseIn] * w[0];
  for (int off = 1; off < T; off <<= 1) {
    Z += __shfl_xor_sync(kFullS, Z, off);
#pragma unroll
    for (int s = 0; s < K; ++s) md[s] += __shfl_xor_sync(kFullS, md[s], off);
  }
  // sum_b w_b b_s (the weight of slot s taking its +1): Z - md where b* has s
  float accb[K];
#pragma unroll
  for (int s = 0; s < K; ++s) accb[s] = ((bst >> s) & 1u) ? Z - md[s] : md[s];
  if (!BWD) {
    if (active) {
      for (int i = lt; i < n; i += T) {
        float v = (float)ts.base[i];
        if ((ts.mask >> i) & 1u) v += pick<K>(accb, __popc(ts.mask & ((1u << i) - 1u))) / Z;
        a.out_mean[p * n + i] = v;
      }
      if (lt == 0 && a.out_logZ) a.out_logZ[p] = logf(Z) - ts.ustar_kT;
      if (lt == 0 && a.ctx_out) a.ctx_out[p] = make_uint2(ts.bstar, __float_as_uint(logf(Z)));
    }
    return;
  }

  // ---- backward: the moments of a_b in flip coordinates ----
  float gs[K];
  float gbase = 0.f, gmean = 0.f;
#pragma unroll
  for (int s = 0; s < K; ++s) gs[s] = 0.f;
  constexpr bool fit = MODE == kDenseFit;
  float lossp = 0.f;
  float* gf = sGf + team * kMaxDot;
  if (fit) lossp = fit_loss_grad_team<K>(a, ts, accb, Z, p, gf, lt, T, active);
  if (active) {
    const float* g = fit ? gf : a.grad_mean + p * n;
#pragma unroll
    for (int s = 0; s < K; ++s)
      if (s < k) gs[s] = g[ts.dot[s]];
    if (use_ctx) {
      for (int i = 0; i < n; ++i) gbase += g[i] * (float)ts.base[i];
      for (int i = 0; i < n; ++i) gmean += g[i] * a.mean_in[p * n + i];
    }
  }
  // the flip-coordinate gradient gam_s = sg_s g_s and c0 = g . n* - g . <n>:
  // from the forward's <n> with the context, else without cancellation from
  // the flip moments, n*_s - <n_s> = -sg_s md_s / Z
  float gam[K];
#pragma unroll
  for (int s = 0; s < K; ++s) gam[s] = sgn[s] * gs[s];
  float c0 = 0.f;
  if (use_ctx) {
    c0 = gbase - gmean;
#pragma unroll
    for (int s = 0; s < K; ++s)
      if ((bst >> s) & 1u) c0 += gs[s];
  } else {
#pragma unroll
    for (int s = 0; s < K; ++s) c0 = fmaf(-gam[s], md[s], c0);
    c0 = active ? c0 / Z : 0.f;
  }
  // sum_d w(d) (c0 + gam . d) d_S = c0 M(S) + Y(S): Y from y(d) = w(d) gam . d
  // by the same superset sum over the inner bits (gam . d = go + the inner
  // slots' gam by doubling); the outer slots of S count where the lane has them
  float y[NI];
  {
    float go = 0.f;
#pragma unroll
    for (int i = 0; i < K - kDenseIn; ++i) go = fmaf(po[i], gam[kDenseIn + i], go);
    y[0] = go;
#pragma unroll
    for (int j = 0; j < kDenseIn; ++j)
#pragma unroll
      for (int b = 0; b < (1 << j); ++b) y[b | (1 << j)] = y[b] + gam[j];
#pragma unroll
    for (int b = 0; b < NI; b += 4) {
      const float4 r = *reinterpret_cast<const float4*>(wraw + b);
      y[b] *= r.x;
      y[b + 1] *= r.y;
      y[b + 2] *= r.z;
      y[b + 3] *= r.w;
    }
  }
  superset_sum<kDenseIn>(y);
  // the 37 moments X(S), |S| <= 2, in the order sa, vd[K], Qd[s < s2], padded
  // to kMomPad, then summed over the team by a reduce-scatter
  float X[kMomPad];
  auto mom = [&](unsigned S) -> float {
    const unsigned si = S & (unsigned)(NI - 1), so = S >> kDenseIn;
    const float v = fmaf(c0, w[si], y[si]);
    return (so & ~tout) == 0u && lane_on ? v : 0.f;
  };
  X[0] = mom(0u);
#pragma unroll
  for (int s = 0; s < K; ++s) X[1 + s] = mom(1u << s);
#pragma unroll
  for (int s = 0; s < K; ++s)
#pragma unroll
    for (int s2 = s + 1; s2 < K; ++s2)
      X[1 + K + s * (2 * K - s - 1) / 2 + (s2 - s - 1)] = mom((1u << s) | (1u << s2));
#pragma unroll
  for (int q = kMom; q < kMomPad; ++q) X[q] = 0.f;
  float* qd = sQd + team * kMom;
  team_reduce_scatter8<kMomPad>(X, lt, qd, kMom);
  __syncwarp();
  // scale by -1 / (kT Z) and turn to charge coordinates, n_s = n*_s + sg_s d_s:
  //   va_s = bt_s sa + sg_s vd_s,  Qa_ss = va_s,
  //   Qa_ss' = bt_s bt_s' sa + bt_s sg_s' vd_s' + bt_s' sg_s vd_s + sg_s sg_s' Qd_ss'
  // (the team's lanes split the entries)
  const float alpha = active ? -1.0f / (kT * Z) : 0.f;
  float* q_s = sQa + team * (tri(K) + K + 1);
  {
    const float sa_a = alpha * qd[0];
    for (int e = lt; e < tri(K); e += T) {
      int s = 0, rem = e;
      while (rem >= K - s) { rem -= K - s; ++s; }
      const int s2 = s + rem;
      const float bts = ((bst >> s) & 1u) ? 1.f : 0.f;
      const float sgs = ((bst >> s) & 1u) ? -1.f : 1.f;
      const float vs = alpha * qd[1 + s];
      float q;
      if (s2 == s) {
        q = bts * sa_a + sgs * vs;
      } else {
        const float bt2 = ((bst >> s2) & 1u) ? 1.f : 0.f;
        const float sg2 = ((bst >> s2) & 1u) ? -1.f : 1.f;
        const float v2 = alpha * qd[1 + s2];
        q = bts * bt2 * sa_a + bts * sg2 * v2 + bt2 * sgs * vs +
            sgs * sg2 * alpha * qd[1 + K + s * (2 * K - s - 1) / 2 + (s2 - s - 1)];
      }
      q_s[e] = q;
    }
    for (int s = lt; s < K; s += T) {
      const float bts = ((bst >> s) & 1u) ? 1.f : 0.f;
      const float sgs = ((bst >> s) & 1u) ? -1.f : 1.f;
      q_s[tri(K) + s] = bts * sa_a + sgs * alpha * qd[1 + s];
    }
    if (lt == 0) q_s[tri(K) + K] = sa_a;
  }
  __syncwarp();
  const int L = contrib_len(n);
  float* my = s_contrib + team * L;
  soft_contrib<K>(a, ts, q_s, my, s_contrib, sM, T, lt, kTeams, active, p, lossp);
}

// The chain rule through M = Cdd^-1 and c = s Cgd V, from the summed
// contributions a.sums (one block, blockDim >= n^2):
//   dL/dCdd = -M (dL/dM) M,  dL/dCgd = s (S0 V0'^T + S1 (dx u)^T + S2 (dy w)^T)
// with V0' = V0 + x0 u + y0 w and S0, S1, S2 the sums of dc, ix dc, iy dc.
// Fit step: then one Adam step on every parameter with its gradient, in the
// update order of Kingma & Ba (Algorithm 1 of arXiv 1412.6980): m <- b1 m +
// (1 - b1) g, v <- b2 v + (1 - b2) g^2, p <- p - lr (m / (1 - b1^t)) /
// (sqrt(v / (1 - b2^t)) + eps), with b1^t, b2^t carried in the state; and the
// loss = summed squared residuals / count.
__device__ __forceinline__ void adam_update(const SoftLaunch& a, double* param, int e,
                                            double g, double c1, double c2) {
  const int cnt = a.n * a.n + a.n * a.ng;
  double* mo = a.fit_state + e;
  double* vo = a.fit_state + cnt + e;
  const double m1 = a.beta1 * *mo + (1.0 - a.beta1) * g;
  const double v1 = a.beta2 * *vo + (1.0 - a.beta2) * g * g;
  *mo = m1;
  *vo = v1;
  *param -= a.lr * (m1 / c1) / (sqrt(v1 / c2) + a.eps);
}

__device__ __forceinline__ void soft_finalize_block(const SoftLaunch& a) {
  __shared__ double sG[kMaxDot * kMaxDot], sMm[kMaxDot * kMaxDot], sT[kMaxDot * kMaxDot];
  __shared__ double sS[3 * kMaxDot + 1];
  const int n = a.n, ng = a.ng;
  const int L = contrib_len(n);
  const bool fit = a.fit_state != nullptr;
  const int cnt = n * n + n * ng;
  // step count and b1^t, b2^t (a zero state is step 0), read by every thread
  // before thread 0 advances them
  double tstep = 0.0, p1 = 1.0, p2 = 1.0;
  if (fit) {
    const double t0 = a.fit_state[2 * cnt];
    tstep = t0 + 1.0;
    p1 = (t0 > 0.0 ? a.fit_state[2 * cnt + 1] : 1.0) * a.beta1;
    p2 = (t0 > 0.0 ? a.fit_state[2 * cnt + 2] : 1.0) * a.beta2;
  }
  for (int e = threadIdx.x; e < L; e += blockDim.x) {
    const double v = __ldcg(a.sums + e);
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
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) sMm[e] = a.md->M[e];
  __syncthreads();
  // T = (dL/dM) M, then dL/dCdd = -M T: the same sums as -sum_p M_ip sum_q G_pq M_qj
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int p = e / n, j = e % n;
    double t = 0.0;
    for (int q = 0; q < n; ++q) t += sG[p * n + q] * sMm[q * n + j];
    sT[e] = t;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    double s = 0.0;
    for (int p = 0; p < n; ++p) s += sMm[i * n + p] * sT[p * n + j];
    if (a.dL_dCdd) a.dL_dCdd[e] = -s;
    if (fit) adam_update(a, a.fit_Cdd + e, e, -s, 1.0 - p1, 1.0 - p2);
  }
  for (int e = threadIdx.x; e < n * ng; e += blockDim.x) {
    const int i = e / ng, g = e % ng;
    const double v0 = a.sc.V0[g] + a.sc.x0 * a.sc.u[g] + a.sc.y0 * a.sc.w[g];
    const double v = sS[i] * v0 + sS[n + i] * a.sc.dx * a.sc.u[g] +
                     sS[2 * n + i] * a.sc.dy * a.sc.w[g];
    const double gv = a.mt.carrier * v;
    if (a.dL_dCgd) a.dL_dCgd[e] = gv;
    if (fit) adam_update(a, a.fit_Cgd + e, n * n + e, gv, 1.0 - p1, 1.0 - p2);
  }
  if (a.loss_out && threadIdx.x == 0) *a.loss_out = (float)(sS[3 * n] * a.fit_inv_count);
  if (fit) {
    __syncthreads();
    if (threadIdx.x == 0) {
      a.fit_state[2 * cnt] = tstep;
      a.fit_state[2 * cnt + 1] = p1;
      a.fit_state[2 * cnt + 2] = p2;
    }
  }
}

// Second stage: one block per contribution e sums the block partials --
// thread j takes blocks j, j + 256, ... in order, then a fixed shared-memory
// tree -- so the result does not depend on scheduling; the block that
// finishes last (a counter, no waiting) then runs the chain rule above.
static __global__ void __launch_bounds__(256) k_soft_reduce(SoftLaunch a, int nblocks) {
  __shared__ df red[256];
  __shared__ bool last;
  const int e = blockIdx.x;
  const float2* pe = reinterpret_cast<const float2*>(a.partials) + (size_t)e * nblocks;
  df acc = {0.f, 0.f};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    const float2 v = pe[b];
    acc = df_add(acc, {v.x, v.y});
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int half = blockDim.x / 2; half > 0; half >>= 1) {
    if ((int)threadIdx.x < half) red[threadIdx.x] = df_add(red[threadIdx.x], red[threadIdx.x + half]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.sums[e] = df_to_double(red[0]);
    __threadfence();
    last = atomicAdd(&a.cnt->soft_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  soft_finalize_block(a);
  if (threadIdx.x == 0) a.cnt->soft_done = 0u;  // zero again for the next call
}

inline size_t soft_partials_floats_impl(int n, long long P, const SearchCfg& cfg) {
  // blocks of the launch that has the most (the dense kernel's blocks hold
  // at least as many teams as the per-candidate kernel's)
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
  if (BWD) k_soft_reduce<<<contrib_len(a.n), 256, 0, st>>>(a, (int)grid);
  if (a.ev) cudaEventRecord(a.ev[1], st);
  return cudaGetLastError();
}

// Dense form (up to 8 dots; teams of kDenseT lanes, the host sizes the
// partials for cfg.T = kDenseT).
template <bool CLOSED, int MODE>
static cudaError_t run_soft_dense(const SoftLaunch& a, cudaStream_t st) {
  constexpr bool BWD = MODE != kDenseFwd;
  constexpr int teams = kDenseThreads / kDenseT;
  const long long P = a.sc.P;
  const unsigned grid = (unsigned)((P + teams - 1) / teams);
  const size_t smem = DenseSmem(BWD, contrib_len(a.n)).total;
  // the largest buffer (n = 16 does not come here: at most contrib_len(8)),
  // and the whole carveout so that as many blocks as the registers allow fit
  // an SM (once per process)
  static const cudaError_t attr = [] {
    cudaError_t e = cudaFuncSetAttribute(k_soft_dense<CLOSED, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)DenseSmem(BWD, contrib_len(kDenseMax)).total);
    if (e == cudaSuccess &&
        cudaFuncSetAttribute(k_soft_dense<CLOSED, MODE>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
      cudaGetLastError();  // the carveout is only a preference
    return e;
  }();
  if (attr != cudaSuccess) return attr;
  if (a.ev) cudaEventRecord(a.ev[0], st);
  k_soft_dense<CLOSED, MODE><<<grid, kDenseThreads, smem, st>>>(a);
  if (BWD) k_soft_reduce<<<contrib_len(a.n), 256, 0, st>>>(a, (int)grid);
  if (a.ev) cudaEventRecord(a.ev[1], st);
  return cudaGetLastError();
}

template <bool CLOSED, bool BWD>
static cudaError_t run_soft_dense_mode(const SoftLaunch& a, cudaStream_t st) {
  if constexpr (!BWD) {
    return run_soft_dense<CLOSED, kDenseFwd>(a, st);
  } else {
    if (a.fit_target) return run_soft_dense<CLOSED, kDenseFit>(a, st);
    if (a.ctx_in) return run_soft_dense<CLOSED, kDenseBwdCtx>(a, st);
    return run_soft_dense<CLOSED, kDenseBwd>(a, st);
  }
}

template <bool BWD>
static cudaError_t dispatch_soft(const SoftLaunch& a, cudaStream_t st) {
  // up to 8 dots: the dense form; beyond, the per-candidate form, whose
  // search only locates b*
  const bool cl = a.mt.closed != 0;
  if (a.n <= kDenseMax)
    return cl ? run_soft_dense_mode<true, BWD>(a, st) : run_soft_dense_mode<false, BWD>(a, st);
  return cl ? run_soft<5, 4, true, BWD, 16>(a, st) : run_soft<5, 4, false, BWD, 16>(a, st);
}

}  // namespace qa
