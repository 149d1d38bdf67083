// qa_search.cuh -- the hot loop: argmin of the candidate energies of one
// pixel over (a share of) its floor / floor + 1 hypercube (Sec. III.B).
//
// Relative to the base configuration, a candidate with ambiguous-slot bits b
// has energy
//     E(b) = sum_{j in b} (h_j + M_jj / 2) + sum_{j < l in b} M_jl,
// h = M (base - c).  The paper evaluates every candidate (2^k of them, Table
// I).  Instead of an O(k) Gray-code update per candidate, the k slots are
// split three ways:
//   inner  (L1 slots): for a fixed rest-state S the 2^L1 energies are
//          A(S) + sum_{j in b} q_j(S) + P[b], with P[b] = sum_{j<l in b} M_jl
//          a per-pixel table in registers -- two FP32 adds per candidate
//          (packed FP32x2 adds, two candidates per instruction) and half a
//          3-input minimum;
//   middle (L2 slots): a fully unrolled reflected Gray walk with compile-time
//          flip positions; one flip updates A, the L1 inner coefficients and
//          the L2 middle coefficients (L1 + L2 adds per 2^L1 candidates);
//   outer  (the rest): split across the lanes of a team and rebuilt from
//          scratch per outer state (no drift across outer states).
// Closed arrays keep one minimum per inner popcount and pick the one whose
// total matches N_hat, so they cost the same as open arrays.
//
// Near-tie detection: each lane keeps the best and second-best block minima;
// the winning block is re-evaluated once, candidate by candidate, to get the
// argmin and the in-block runner-up.
#pragma once

#include <cuda_fp16.h>

#include "qa_device.cuh"
#include "qa_launch.h"

namespace qa {

constexpr float kBig = 1.0e30f;
constexpr float kInf = __builtin_huge_valf();

// Energies of one inner block, min over all 2^L1 patterns (open).
template <int L1>
__device__ __forceinline__ float inner_min_open(float A, const float* q,
                                                const float* P) {
  constexpr int NI = 1 << L1;
  float S[NI];
  S[0] = A;
  if (L1 >= 1) S[1] = __fadd_rn(A, q[0]);
#pragma unroll
  for (int j = 1; j < L1; ++j) {
    const float2 qq = make_float2(q[j], q[j]);
#pragma unroll
    for (int b = 0; b < (1 << j); b += 2) {
      float2 r = fadd2(make_float2(S[b], S[b + 1]), qq);
      S[b + (1 << j)] = r.x;
      S[b + 1 + (1 << j)] = r.y;
    }
  }
  if (NI == 1) return S[0];
  if (NI == 2) return fminf(S[0], S[1]);
  // E = S + P (P[0] = P[1] = 0), then a 3-input min tree in two chains
  float m0 = fminf(S[0], S[1]);
  float m1 = kInf;
#pragma unroll
  for (int b = 2; b < NI; b += 4) {
    float2 e = fadd2(make_float2(S[b], S[b + 1]), make_float2(P[b], P[b + 1]));
    m0 = fmin3(m0, e.x, e.y);
    if (b + 2 < NI) {
      float2 f = fadd2(make_float2(S[b + 2], S[b + 3]),
                       make_float2(P[b + 2], P[b + 3]));
      m1 = fmin3(m1, f.x, f.y);
    }
  }
  return fminf(m0, m1);
}

// The same with the pair table P in shared memory (16-byte aligned; the
// team's lanes read the same entries, so the loads are broadcasts).
template <int L1>
__device__ __forceinline__ float inner_min_open_smem(float A, const float* q,
                                                     const float* __restrict__ P) {
  constexpr int NI = 1 << L1;
  static_assert(NI >= 8, "four-entry chunks");
  float S[NI];
  S[0] = A;
  S[1] = __fadd_rn(A, q[0]);
#pragma unroll
  for (int j = 1; j < L1; ++j) {
    const float2 qq = make_float2(q[j], q[j]);
#pragma unroll
    for (int b = 0; b < (1 << j); b += 2) {
      float2 r = fadd2(make_float2(S[b], S[b + 1]), qq);
      S[b + (1 << j)] = r.x;
      S[b + 1 + (1 << j)] = r.y;
    }
  }
  const float4* P4 = reinterpret_cast<const float4*>(P);
  float m0 = fminf(S[0], S[1]);
  float m1 = kInf;
#pragma unroll
  for (int b = 0; b < NI; b += 4) {
    const float4 p = P4[b / 4];
    if (b == 0) {
      m1 = fminf(__fadd_rn(S[2], p.z), __fadd_rn(S[3], p.w));
    } else {
      const float2 e = fadd2(make_float2(S[b], S[b + 1]), make_float2(p.x, p.y));
      const float2 f = fadd2(make_float2(S[b + 2], S[b + 3]), make_float2(p.z, p.w));
      m0 = fmin3(m0, e.x, e.y);
      m1 = fmin3(m1, f.x, f.y);
    }
  }
  return fminf(m0, m1);
}

// Closed, with the pair table P in shared memory: the minimum over the inner
// patterns with popcount r (kInf if none).
template <int L1>
__device__ __forceinline__ float inner_min_closed_smem(float A, const float* q,
                                                       const float* __restrict__ P, int r) {
  constexpr int NI = 1 << L1;
  float S[NI];
  S[0] = A;
  S[1] = __fadd_rn(A, q[0]);
#pragma unroll
  for (int j = 1; j < L1; ++j) {
    const float2 qq = make_float2(q[j], q[j]);
#pragma unroll
    for (int b = 0; b < (1 << j); b += 2) {
      const float2 e = fadd2(make_float2(S[b], S[b + 1]), qq);
      S[b + (1 << j)] = e.x;
      S[b + 1 + (1 << j)] = e.y;
    }
  }
  float acc[L1 + 1];
#pragma unroll
  for (int i = 0; i <= L1; ++i) acc[i] = kInf;
  const float4* P4 = reinterpret_cast<const float4*>(P);
#pragma unroll
  for (int b = 0; b < NI; b += 4) {
    const float4 p = P4[b / 4];
    const float2 e = fadd2(make_float2(S[b], S[b + 1]), make_float2(p.x, p.y));
    const float2 f = fadd2(make_float2(S[b + 2], S[b + 3]), make_float2(p.z, p.w));
    acc[popc_c(b)] = fminf(acc[popc_c(b)], e.x);
    acc[popc_c(b + 1)] = fminf(acc[popc_c(b + 1)], e.y);
    acc[popc_c(b + 2)] = fminf(acc[popc_c(b + 2)], f.x);
    acc[popc_c(b + 3)] = fminf(acc[popc_c(b + 3)], f.y);
  }
  float res = kInf;
#pragma unroll
  for (int i = 0; i <= L1; ++i) res = (i == r) ? acc[i] : res;
  return res;
}

// Closed: minimum over the inner patterns with popcount r (kInf if none).
template <int L1>
__device__ __forceinline__ float inner_min_closed(float A, const float* q,
                                                  const float* P, int r) {
  constexpr int NI = 1 << L1;
  float S[NI];
  S[0] = A;
  if (L1 >= 1) S[1] = __fadd_rn(A, q[0]);
#pragma unroll
  for (int j = 1; j < L1; ++j) {
    const float2 qq = make_float2(q[j], q[j]);
#pragma unroll
    for (int b = 0; b < (1 << j); b += 2) {
      float2 e = fadd2(make_float2(S[b], S[b + 1]), qq);
      S[b + (1 << j)] = e.x;
      S[b + 1 + (1 << j)] = e.y;
    }
  }
  float acc[L1 + 1];
#pragma unroll
  for (int i = 0; i <= L1; ++i) acc[i] = kInf;
#pragma unroll
  for (int b = 0; b < NI; b += 2) {
    float2 e = (b == 0) ? make_float2(S[0], S[1])
                        : fadd2(make_float2(S[b], S[b + 1]),
                                make_float2(P[b], P[b + 1]));
    if (NI == 1) { acc[0] = S[0]; break; }
    acc[popc_c(b)] = fminf(acc[popc_c(b)], e.x);
    acc[popc_c(b + 1)] = fminf(acc[popc_c(b + 1)], e.y);
  }
  float res = kInf;
#pragma unroll
  for (int i = 0; i <= L1; ++i) res = (i == r) ? acc[i] : res;
  return res;
}

// Team table of the middle-slot columns used by block-level searches: for
// middle slot m, kColStride floats holding M(inner j, m) at j < L1 and
// M(middle m', m) at L1 + m' (0 on the diagonal and for absent slots).
constexpr int kColStride = 12;  // >= L1 + L2 for every split, a multiple of 4
constexpr int kItMax = 4;       // iteration bits of a block-level search with L1 + L2 >= 9
constexpr int kItStride = 12;   // >= 1 + L1 + L2, a multiple of 4

// Per-pixel slot data staged by the team: dot of each slot, h of each slot.
struct SlotView {
  const int* dot;
  const float* h;
  int k;
  int w;  // closed weight, -1 open
};

// Rest-state (outer + middle set S) quantities from scratch:
//   A = E(S), q_j = h_j + M_jj/2 + sum_{s in S} M_{j s} for inner slots.
template <int L1>
__device__ __forceinline__ float state_from_scratch(const float* sM,
                                                    const SlotView& sv,
                                                    unsigned S_bits,
                                                    const int* dI,
                                                    const float* qb, float* q) {
#pragma unroll
  for (int j = 0; j < L1; ++j) q[j] = qb[j];
  float A = 0.f;
  for (unsigned bits = S_bits; bits; bits &= bits - 1u) {
    const int s = __ffs(bits) - 1;
    const int d = sv.dot[s];
    const float* Mrow = sM + d * kLdM;
    float add = sv.h[s] + 0.5f * Mrow[d];
    for (unsigned prev = S_bits & ((1u << s) - 1u); prev; prev &= prev - 1u)
      add += Mrow[sv.dot[__ffs(prev) - 1]];
    A += add;
#pragma unroll
    for (int j = 0; j < L1; ++j) q[j] += Mrow[dI[j]];
  }
  return A;
}

// Search of one lane's share.  Lane t of a team of T (a power of two, at
// most 2^LANEBITS) handles the outer patterns o = t, t + T, ...; results: best energy m1 with its full slot
// pattern b1, and the second-best energy m2 over the lane's candidates.
// COLLECT: instead, append every (outer, middle) block whose minimum is
// <= thr to blist (used by the FP64 recheck to shortlist candidates).
// BLOCKS: return the lane's best block minimum with its block id and the
// second-best block minimum, for a team-level finish (team_finish).
// LANEBITS: log2 of the widest team the caller uses (T <= 2^LANEBITS).
// lb_cut (COLLECT): an outer pattern whose lower bound A + sum min(0, q_j) +
// sum min(0, g_m) + qneg (qneg: the model's bound of any pair-term sum, so
// the bound holds for every candidate of the pattern) lies above lb_cut
// holds no block to collect and is skipped.
template <int L1, int L2, bool CLOSED, bool COLLECT, bool BLOCKS = false, int LANEBITS = 8>
__device__ __forceinline__ void search_lane(const float* __restrict__ sM,
                                            const SlotView sv, int t, int T,
                                            float thr, unsigned* blist,
                                            unsigned* bcount, unsigned bcap,
                                            float& m1, unsigned& b1, float& m2,
                                            unsigned long long& evaluated,
                                            const float* __restrict__ colt = nullptr,
                                            const float* __restrict__ itab = nullptr,
                                            float* __restrict__ cslot = nullptr,
                                            float lb_cut = kInf, float qneg = 0.f) {
  static_assert(L1 >= 2 && L1 <= 6 && L2 >= 0 && L2 <= 5, "search split");
  // block-level searches with at least 9 inner + middle slots take the
  // iteration slots' terms from the team table itab (iter_build): at most 7
  // outer slots, at least 3 of them lane bits, so at most kItMax iteration bits
  constexpr bool ITAB = BLOCKS && (L1 + L2 >= 9);
  constexpr int NI = 1 << L1;
  constexpr int NM = 1 << L2;
  const int k = sv.k;

  int dI[L1 > 0 ? L1 : 1];
  float qb[L1 > 0 ? L1 : 1];
#pragma unroll
  for (int j = 0; j < L1; ++j) {
    if (j < k) {
      const int d = sv.dot[j];
      dI[j] = d;
      qb[j] = sv.h[j] + 0.5f * sM[d * kLdM + d];
    } else {
      dI[j] = 0;
      qb[j] = kBig;  // dummy slot: any pattern using it never wins
    }
  }
  float P[NI];
  P[0] = 0.f;
#pragma unroll
  for (int j = 0; j < L1; ++j) {
    float Mj[L1 > 0 ? L1 : 1];
#pragma unroll
    for (int l = 0; l < j; ++l)
      Mj[l] = (j < k) ? sM[dI[j] * kLdM + dI[l]] : 0.f;
#pragma unroll
    for (int b = 0; b < (1 << j); ++b) {
      float r = 0.f;
#pragma unroll
      for (int l = 0; l < j; ++l)
        if ((b >> l) & 1) r += Mj[l];
      P[b | (1 << j)] = P[b] + r;
    }
  }

  const int nmid = min(max(k - L1, 0), L2);
  int dM[L2 > 0 ? L2 : 1];
  float gb[L2 > 0 ? L2 : 1];
  float Mmm[L2 > 0 ? L2 : 1][L2 > 0 ? L2 : 1];
  float Mim[L1 > 0 ? L1 : 1][L2 > 0 ? L2 : 1];
#pragma unroll
  for (int m = 0; m < L2; ++m) {
    const bool live = m < nmid;
    const int d = live ? sv.dot[L1 + m] : 0;
    dM[m] = d;
    gb[m] = live ? sv.h[L1 + m] + 0.5f * sM[d * kLdM + d] : 0.f;
  }
  if (!BLOCKS) {  // BLOCKS: the middle columns come from the team table colt
#pragma unroll
    for (int m = 0; m < L2; ++m)
#pragma unroll
      for (int m2 = 0; m2 < L2; ++m2)
        Mmm[m][m2] = (m != m2 && m < nmid && m2 < nmid) ? sM[dM[m] * kLdM + dM[m2]] : 0.f;
#pragma unroll
    for (int j = 0; j < L1; ++j)
#pragma unroll
      for (int m = 0; m < L2; ++m)
        Mim[j][m] = (m < nmid) ? sM[dI[j] * kLdM + dM[m]] : 0.f;
  }

  // Outer patterns o = t + T i: the low log2(T) bits of o are the lane's own
  // and fixed, so the lane-bit part of the rest state is built once and each
  // iteration only adds its iteration bits.
  const int nout = max(k - L1 - L2, 0);
  const int nlb = min(__ffs(T) - 1, nout);
  const int nit = nout - nlb;
  float g1 = kInf, g2 = kInf;
  unsigned blk = 0u;
  const int nsteps = 1 << nmid;  // Gray steps that stay inside the k slots
  const unsigned niter = ((unsigned)t < (1u << nlb)) ? (1u << nit) : 0u;
  float At = 0.f;
  float qt[L1 > 0 ? L1 : 1];
  float gt[L2 > 0 ? L2 : 1];
#pragma unroll
  for (int j = 0; j < L1; ++j) qt[j] = qb[j];
#pragma unroll
  for (int m = 0; m < L2; ++m) gt[m] = gb[m];
  // The lane-bit slots: their dots and the lane's 0 / 1 weights.  The sums
  // below run over every lane slot in increasing order with the weight as a
  // factor (fma(1, x, y) = x + y rounded, fma(0, x, y) = y exactly), so they
  // round exactly like sums over the lane's set bits alone, but with a trip
  // count that is the same for every lane of the team: no divergent,
  // load-dependent chains.
  constexpr int kLaneBits = LANEBITS;
  int dO[kLaneBits];
  float wO[kLaneBits];
#pragma unroll
  for (int i = 0; i < kLaneBits; ++i) {
    const bool live = i < nlb;
    dO[i] = live ? sv.dot[L1 + L2 + i] : 0;
    wO[i] = (live && ((t >> i) & 1)) ? 1.f : 0.f;
  }
  if (niter) {
#pragma unroll
    for (int i = 0; i < kLaneBits; ++i) {
      if (i < nlb) {
        const float* Mrow = sM + dO[i] * kLdM;
        float add = sv.h[L1 + L2 + i] + 0.5f * Mrow[dO[i]];
#pragma unroll
        for (int i2 = 0; i2 < i; ++i2) add = fmaf(wO[i2], Mrow[dO[i2]], add);
        At = fmaf(wO[i], add, At);
#pragma unroll
        for (int j = 0; j < L1; ++j) qt[j] = fmaf(wO[i], Mrow[dI[j]], qt[j]);
#pragma unroll
        for (int m = 0; m < L2; ++m) gt[m] = fmaf(wO[i], Mrow[dM[m]], gt[m]);
      }
    }
    if (ITAB) {
      // the lane's pair terms with each iteration slot (its own lane slots
      // present), kept in the lane's slot of shared memory
#pragma unroll
      for (int ii = 0; ii < kItMax; ++ii) {
        float c = 0.f;
        if (ii < nit) {
          const float* Mrow = sM + sv.dot[L1 + L2 + nlb + ii] * kLdM;
#pragma unroll
          for (int i = 0; i < kLaneBits; ++i) c = fmaf(wO[i], Mrow[dO[i]], c);
        }
        cslot[ii] = c;
      }
    }
  }

  for (unsigned it = 0; it < niter; ++it) {
    const unsigned o = (unsigned)t | (it << nlb);
    float A = At;
    float q[L1 > 0 ? L1 : 1];
    float gm[L2 > 0 ? L2 : 1];
#pragma unroll
    for (int j = 0; j < L1; ++j) q[j] = qt[j];
#pragma unroll
    for (int m = 0; m < L2; ++m) gm[m] = gt[m];
    if (ITAB) {
      // A = At + the lane's pair terms with the set iteration slots + the
      // team's terms of those slots among themselves; q, gm from the table
      const float4 cc = *reinterpret_cast<const float4*>(cslot);
      const float* row = itab + it * kItStride;
      float x = 0.f;
      x = fmaf((it & 1u) ? 1.f : 0.f, cc.x, x);
      x = fmaf((it & 2u) ? 1.f : 0.f, cc.y, x);
      x = fmaf((it & 4u) ? 1.f : 0.f, cc.z, x);
      x = fmaf((it & 8u) ? 1.f : 0.f, cc.w, x);
      A = (A + x) + row[0];
#pragma unroll
      for (int j = 0; j < L1; ++j) q[j] += row[1 + j];
#pragma unroll
      for (int m = 0; m < L2; ++m) gm[m] += row[1 + L1 + m];
    } else
    // the iteration-bit slots (the same for the whole team), each paired
    // with the lane slots and with the iteration slots below it
    for (unsigned ib = it; ib; ib &= ib - 1u) {
      const int ii = __ffs(ib) - 1;
      const int d = sv.dot[L1 + L2 + nlb + ii];
      const float* Mrow = sM + d * kLdM;
      float add = sv.h[L1 + L2 + nlb + ii] + 0.5f * Mrow[d];
#pragma unroll
      for (int i = 0; i < kLaneBits; ++i) {
        if (i < nlb) {  // reloaded here rather than kept live through the walk
          const float wi = ((t >> i) & 1) ? 1.f : 0.f;
          add = fmaf(wi, Mrow[sv.dot[L1 + L2 + i]], add);
        }
      }
      for (unsigned prev = it & ((1u << ii) - 1u); prev; prev &= prev - 1u)
        add += Mrow[sv.dot[L1 + L2 + nlb + __ffs(prev) - 1]];
      A += add;
#pragma unroll
      for (int j = 0; j < L1; ++j) q[j] += Mrow[dI[j]];
#pragma unroll
      for (int m = 0; m < L2; ++m) gm[m] += Mrow[dM[m]];
    }
    if (COLLECT) {
      float sb = 0.f;
#pragma unroll
      for (int j = 0; j < L1; ++j) sb += fminf(0.f, q[j]);
#pragma unroll
      for (int m = 0; m < L2; ++m) sb += (m < nmid) ? fminf(0.f, gm[m]) : 0.f;
      if ((A + sb) + qneg > lb_cut) continue;
    }
    const unsigned obase = o << L2;
    const int popo = __popc(o);
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      // Guarded rather than `break`: the walk must stay fully unrolled so that
      // every flip position below is a compile-time register index.
      if (s >= nsteps) continue;
      if (s > 0) {
        const int mb = ctz_c((unsigned)s);
        const bool up = (gray_c((unsigned)s) >> mb) & 1u;
        A = up ? A + gm[mb] : A - gm[mb];
        if (BLOCKS) {
          // column mb of the team table: M(inner j, mb) at j, M(mid m, mb) at L1 + m
          float col[kColStride];
#pragma unroll
          for (int e = 0; e < kColStride; e += 4) {
            const float4 c4 = *reinterpret_cast<const float4*>(colt + mb * kColStride + e);
            col[e] = c4.x; col[e + 1] = c4.y; col[e + 2] = c4.z; col[e + 3] = c4.w;
          }
#pragma unroll
          for (int m = 0; m < L2; ++m)
            if (m != mb) gm[m] = up ? gm[m] + col[L1 + m] : gm[m] - col[L1 + m];
#pragma unroll
          for (int j = 0; j < L1; ++j) q[j] = up ? q[j] + col[j] : q[j] - col[j];
        } else {
#pragma unroll
          for (int m = 0; m < L2; ++m)
            if (m != mb) gm[m] = up ? gm[m] + Mmm[m][mb] : gm[m] - Mmm[m][mb];
#pragma unroll
          for (int j = 0; j < L1; ++j)
            q[j] = up ? q[j] + Mim[j][mb] : q[j] - Mim[j][mb];
        }
      }
      float mbk;
      if (!CLOSED) {
        mbk = inner_min_open<L1>(A, q, P);
      } else {
        const int r = sv.w - popo - popc_c(gray_c((unsigned)s));
        mbk = inner_min_closed<L1>(A, q, P, r);
      }
      const unsigned id = obase | gray_c((unsigned)s);
      if (COLLECT) {
        if (mbk <= thr) {
          const unsigned at = atomicAdd(bcount, 1u);
          if (at < bcap) blist[at] = id;
        }
      } else {
        g2 = fminf(g2, fmaxf(g1, mbk));
        const bool better = mbk < g1;
        g1 = better ? mbk : g1;
        blk = better ? id : blk;
      }
    }
  }
  evaluated += (unsigned long long)niter * (unsigned)nsteps * (unsigned)NI;
  if (COLLECT) return;
  if (BLOCKS) {  // block level only: the team finishes the winning block
    m1 = g1;
    b1 = blk;
    m2 = g2;
    return;
  }

  m1 = kInf;
  b1 = 0u;
  m2 = g2;
  if (!(g1 < kInf)) return;
  // re-evaluate the winning block candidate by candidate
  const unsigned o = blk >> L2, mp = blk & (unsigned)(NM - 1);
  const unsigned Sbits = (o << (L1 + L2)) | (mp << L1);
  float q[L1 > 0 ? L1 : 1];
  const float A = state_from_scratch<L1>(sM, sv, Sbits, dI, qb, q);
  const int r = CLOSED ? sv.w - __popc(Sbits) : 0;
  float best = kInf, second = kInf;
  unsigned bb = 0u;
#pragma unroll
  for (int b = 0; b < NI; ++b) {
    if (CLOSED && popc_c((unsigned)b) != r) continue;
    float e = A;
#pragma unroll
    for (int j = 0; j < L1; ++j)
      if ((b >> j) & 1) e += q[j];
    e += P[b];
    if (e < best) { second = best; best = e; bb = (unsigned)b; }
    else if (e < second) { second = e; }
  }
  m1 = best;
  b1 = Sbits | bb;
  m2 = fminf(g2, second);
}

// Team table of the iteration slots (the outer slots above a team's lane
// bits, the same for every lane): for each iteration pattern it, kItStride
// floats holding the sum over its set slots s of h_s + M_ss / 2 plus the
// pairs among them (at 0), of M(inner j, s) (at 1 + j) and of M(middle m, s)
// (at 1 + L1 + m).  Team-cooperative (lane lt of T); sync after.
template <int L1, int L2>
__device__ __forceinline__ void iter_build(const float* sM, const SlotView& sv, int lt, int T,
                                           float* itab) {
  const int k = sv.k;
  const int nmid = min(max(k - L1, 0), L2);
  const int nout = max(k - L1 - L2, 0);
  const int nlb = min(__ffs(T) - 1, nout);
  const int nit = nout - nlb;
  const int s0 = L1 + L2 + nlb;  // the first iteration slot
  for (int e = lt; e < (1 << nit) * kItStride; e += T) {
    const unsigned it = (unsigned)(e / kItStride);
    const int v = e % kItStride;
    float acc = 0.f;
    for (unsigned ib = it; ib; ib &= ib - 1u) {
      const int ii = __ffs(ib) - 1;
      const int d = sv.dot[s0 + ii];
      const float* Mrow = sM + d * kLdM;
      if (v == 0) {
        float add = sv.h[s0 + ii] + 0.5f * Mrow[d];
        for (unsigned prev = it & ((1u << ii) - 1u); prev; prev &= prev - 1u)
          add += Mrow[sv.dot[s0 + __ffs(prev) - 1]];
        acc += add;
      } else if (v <= L1) {
        if (v - 1 < k) acc += Mrow[sv.dot[v - 1]];
      } else if (v <= L1 + L2) {
        if (v - 1 - L1 < nmid) acc += Mrow[sv.dot[v - 1]];
      }
    }
    itab[e] = acc;
  }
}

// Team-cooperative build of the column table (lane lt of T); sync after.
template <int L1, int L2>
__device__ __forceinline__ void col_build(const float* sM, const SlotView& sv, int lt, int T,
                                          float* colt) {
  const int k = sv.k;
  const int nmid = min(max(k - L1, 0), L2);
  for (int e = lt; e < L2 * kColStride; e += T) {
    const int m = e / kColStride, c = e % kColStride;
    float v = 0.f;
    if (m < nmid) {
      const int dm = sv.dot[L1 + m];
      if (c < L1) {
        const int dj = c < k ? sv.dot[c] : 0;
        v = sM[dj * kLdM + dm];
      } else if (c < L1 + L2) {
        const int m2 = c - L1;
        if (m2 != m && m2 < nmid) v = sM[sv.dot[L1 + m2] * kLdM + dm];
      }
    }
    colt[e] = v;
  }
}

// Team-level finish of a block-level search: every lane of the team (lane lt
// of T, T a power of two, all in one warp segment `tmask`) holds the winning
// block id blk (after the team's top-two merge).  Every lane named by tmask
// must call (the team reductions are shuffles); a lane whose team has no
// pixel passes an empty slot view (k = 0) and any blk.  The block's rest state
// (A, q) is summed over the team -- lane s adds slot s's terms -- and the
// lanes then evaluate the block's 2^L1 inner patterns (lane lt takes
// b = lt, lt + T, ...).  Returns the best energy e1, its full slot pattern and
// the in-block runner-up e2; ties go to the lexicographically smaller charge
// vector (bit-reversed pattern order).
template <int L1, int L2, bool CLOSED>
__device__ __forceinline__ void team_finish(const float* __restrict__ sM, const SlotView sv,
                                            int lt, int T, unsigned tmask, unsigned blk,
                                            float& e1, unsigned& bits1, float& e2) {
  constexpr int NI = 1 << L1;
  constexpr int NM = 1 << L2;
  const int k = sv.k;
  const unsigned o = blk >> L2, mp = blk & (unsigned)(NM - 1);
  const unsigned Sbits = (o << (L1 + L2)) | (mp << L1);
  float A = 0.f, q[L1 > 0 ? L1 : 1];
#pragma unroll
  for (int j = 0; j < L1; ++j) q[j] = 0.f;
  int dI[L1 > 0 ? L1 : 1];
#pragma unroll
  for (int j = 0; j < L1; ++j) dI[j] = j < k ? sv.dot[j] : 0;
  for (int s = lt; s < kMaxDot; s += T) {
    if (!((Sbits >> s) & 1u)) continue;
    const int d = sv.dot[s];
    const float* Mrow = sM + d * kLdM;
    float add = sv.h[s] + 0.5f * Mrow[d];
    // pairs with the set slots below s in increasing order, as 0 / 1
    // weighted terms over a fixed range (Sbits has no inner bits): the same
    // rounding as a loop over the set bits, without a load-dependent chain
    const unsigned below = Sbits & ((1u << s) - 1u);
#pragma unroll
    for (int s2 = L1; s2 < kMaxDot - 1; ++s2) {
      const bool on = (below >> s2) & 1u;
      const int d2 = sv.dot[s2];
      add = fmaf(on ? 1.f : 0.f, Mrow[on ? d2 : d], add);
    }
    A += add;
#pragma unroll
    for (int j = 0; j < L1; ++j)
      if (j < k) q[j] += Mrow[dI[j]];
  }
  for (int off = 1; off < T; off <<= 1) {
    A += __shfl_xor_sync(tmask, A, off, T);
#pragma unroll
    for (int j = 0; j < L1; ++j) q[j] += __shfl_xor_sync(tmask, q[j], off, T);
  }
#pragma unroll
  for (int j = 0; j < L1; ++j) {
    if (j < k) {
      const int d = sv.dot[j];
      q[j] += sv.h[j] + 0.5f * sM[d * kLdM + d];
    } else {
      q[j] = kBig;  // dummy slot: never wins
    }
  }
  const int r = CLOSED ? sv.w - __popc(Sbits) : 0;
  e1 = kInf;
  e2 = kInf;
  unsigned bb = 0xffffffffu;
  for (int b = lt; b < NI; b += T) {
    if (CLOSED && __popc((unsigned)b) != r) continue;
    // e = A + sum_{j in b} q_j + sum_{l < j in b} M(I_j, I_l), the terms in
    // increasing order with 0 / 1 weights (no lane-dependent branches)
    float e = A;
    float pb = 0.f;
#pragma unroll
    for (int j = 0; j < L1; ++j) {
      const float wj = ((b >> j) & 1) ? 1.f : 0.f;
      e = fmaf(wj, q[j], e);
      const float* Mrow = sM + dI[j] * kLdM;
#pragma unroll
      for (int l = 0; l < j; ++l) {
        const float wl = (((b >> l) & 1) && j < k) ? wj : 0.f;
        pb = fmaf(wl, Mrow[dI[l]], pb);
      }
    }
    e += pb;
    if (e < e1 || (e == e1 && __brev((unsigned)b) < __brev(bb))) {
      e2 = e1;
      e1 = e;
      bb = (unsigned)b;
    } else if (e < e2) {
      e2 = e;
    }
  }
  for (int off = 1; off < T; off <<= 1) {
    const float o1 = __shfl_xor_sync(tmask, e1, off, T);
    const float o2 = __shfl_xor_sync(tmask, e2, off, T);
    const unsigned ob = __shfl_xor_sync(tmask, bb, off, T);
    const bool take = o1 < e1 || (o1 == e1 && __brev(ob) < __brev(bb));
    const float lose = take ? e1 : o1;
    e2 = fminf(fminf(e2, o2), lose);
    if (take) { e1 = o1; bb = ob; }
  }
  bits1 = Sbits | (bb == 0xffffffffu ? 0u : bb);
}

// ---------------------------------------------------------------------------
// Pruned search: teams of 16 or 32 lanes, split L1 = 5, L2 = 2.  An exact
// branch and bound over the outer slots.
//
// With the inner and middle slots x (L1 + L2 of them) free and the outer
// pattern o fixed, a candidate's energy is
//     E(o, x) = A_o + sum_j L_oj x_j + Q(x),
// A_o the energy of o alone, L_oj = h_j + M_jj / 2 + sum_{s in o} M_js, and
// Q(x) the pair terms among the set bits of x.  Q(x) is at least qneg, the
// sum of the model's negative pair terms (0 whenever M is entrywise
// non-negative, as for every Maxwell Cdd, whose inverse is non-negative), so
//     LB_o = A_o + sum_j min(0, L_oj) + qneg
// bounds every candidate of o from below.  A closed array's candidates of o
// set exactly r = w - |o| walked slots (w the candidate weight of Sec. III.B's
// closed filter), so there the bound is A_o + (the sum of the r smallest
// lower bounds of the L_oj that hold for every pattern of the lane, sorted
// once per lane) + qneg, and +inf when no such candidate exists.  An outer pattern whose bound lies
// above an energy already known to be at least the runner-up (plus the FP32
// error margin) holds neither the argmin nor the runner-up: it is skipped,
// and the top two over the candidate set are exactly those over the patterns
// walked.  The slots come ordered so that the outer ones are the dots whose
// single-flip energy at the base, h_s + M_ss / 2, is largest in magnitude:
// a wrong setting of such a dot costs most, so its patterns are pruned first.
//
// Lane t of the team owns the outer patterns o = t + T i.  It bounds them
// all, and walks the one with the lowest bound first (every owning lane at
// once), which usually finds the argmin and a runner-up close to it; the cut
// is then the team's second-best block minimum, and the few patterns whose
// bound is still below it are collected once and walked in rounds of T, the
// cut tightening after every round.
// ---------------------------------------------------------------------------
constexpr int kBnbIn = kBnbL1 + kBnbL2;   // walked slots per outer pattern
constexpr int kBnbItBits = 5;             // iteration bits at most (k = 16, T = 16)
constexpr int kBnbStride = 8;             // iteration-table row: A part, L parts
constexpr int kBnbLane = 16;              // lane-table row: At, Lt[kBnbIn], cross[kBnbItBits]
constexpr int kBnbStates = 1 << (kMaxDot - kBnbIn);
constexpr int kBnbBuf = 64;               // patterns collected per pass

// Team-cooperative tables of the pruned search (lane lt of T; sync after):
//   pm[s][s'] = M(dot_s, dot_s') for slots s, s' < k (kLdM stride, 0 beyond)
//   vv[s]     = h_s + M_ss / 2 (slots beyond k: kBig for an inner slot, so
//               that no pattern using it wins, 0 otherwise)
// built with independent loads (one slot row per lane), so that the tables
// that follow read slot pairs directly instead of through the dot indices.
__device__ __forceinline__ void bnb_pair_build(const float* sM, const SlotView& sv, int lt, int T,
                                               float* pm, float* vv) {
  const int k = sv.k;
  for (int r = lt; r < kMaxDot; r += T) {
    const bool live = r < k;
    const int dr = live ? sv.dot[r] : 0;
    const float* Mrow = sM + dr * kLdM;
    float row[kMaxDot];
#pragma unroll
    for (int c = 0; c < kMaxDot; ++c) {
      const int dc = (live && c < k) ? sv.dot[c] : 0;
      row[c] = (live && c < k) ? Mrow[dc] : 0.f;
    }
#pragma unroll
    for (int c = 0; c < kMaxDot; ++c) pm[r * kLdM + c] = row[c];
    vv[r] = live ? sv.h[r] + 0.5f * Mrow[dr] : (r < kBnbL1 ? kBig : 0.f);
  }
}

// Team-cooperative iteration table (lane lt of T; sync after): for each
// pattern i of the nit iteration slots (slots kBnbIn + nlb + ii), the energy
// of its set slots alone (v and their pairs, at 0) and, at 1 + j, the sum of
// M(slot j, s) over its set slots s for every walked slot j (0 for j >= k).
// Fixed-range 0 / 1-weighted sums over the pair table.
__device__ __forceinline__ void bnb_iter_build(const float* pm, const float* vv, int lt, int T,
                                               int nlb, int nit, float* itab) {
  const int s0 = kBnbIn + nlb;
  for (int it = lt; it < (1 << nit); it += T) {
    float w[kBnbItBits];
#pragma unroll
    for (int ii = 0; ii < kBnbItBits; ++ii) w[ii] = (ii < nit && ((it >> ii) & 1)) ? 1.f : 0.f;
    float A = 0.f;
#pragma unroll
    for (int ii = 0; ii < kBnbItBits; ++ii) {
      const int si = min(s0 + ii, kMaxDot - 1);
      float add = vv[si];
#pragma unroll
      for (int i2 = 0; i2 < ii; ++i2) add = fmaf(w[i2], pm[si * kLdM + min(s0 + i2, kMaxDot - 1)], add);
      A = fmaf(w[ii], add, A);
    }
    float row[kBnbStride];
    row[0] = A;
#pragma unroll
    for (int j = 0; j < kBnbIn; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int ii = 0; ii < kBnbItBits; ++ii)
        acc = fmaf(w[ii], pm[j * kLdM + min(s0 + ii, kMaxDot - 1)], acc);
      row[1 + j] = acc;
    }
    float4* dst = reinterpret_cast<float4*>(itab + it * kBnbStride);
    dst[0] = make_float4(row[0], row[1], row[2], row[3]);
    dst[1] = make_float4(row[4], row[5], row[6], row[7]);
  }
}

// The team-wide top two of per-lane (a1 <= a2) pairs, by shuffles over the
// team's lanes (tmask, width T); every lane ends with the same pair.
__device__ __forceinline__ void team_top2(unsigned tmask, int T, float& a1, float& a2) {
  for (int off = 1; off < T; off <<= 1) {
    const float o1 = __shfl_xor_sync(tmask, a1, off, T);
    const float o2 = __shfl_xor_sync(tmask, a2, off, T);
    a2 = fminf(fminf(a2, o2), fmaxf(a1, o1));
    a1 = fminf(a1, o1);
  }
}

// Ascending sort of seven values (a 16-comparator network).
__device__ __forceinline__ void bnb_sort7(float* c) {
  auto cx = [&](int a, int b) {
    const float lo = fminf(c[a], c[b]), hi = fmaxf(c[a], c[b]);
    c[a] = lo;
    c[b] = hi;
  };
  cx(0, 6); cx(2, 3); cx(4, 5);
  cx(0, 2); cx(1, 4); cx(3, 6);
  cx(0, 1); cx(2, 5); cx(3, 4);
  cx(1, 2); cx(4, 6);
  cx(2, 3); cx(4, 5);
  cx(1, 2); cx(3, 4); cx(5, 6);
}

// Rest state of outer pattern o from the team tables: the lane part of its
// lane bits, the iteration part of its iteration bits, and their pair terms.
__device__ __forceinline__ void bnb_rest(const float* ltab, const float* itab, int nlb, int o,
                                         float& A, float* L) {
  const float4* lp = reinterpret_cast<const float4*>(ltab + (o & ((1 << nlb) - 1)) * kBnbLane);
  const float4* ip = reinterpret_cast<const float4*>(itab + (o >> nlb) * kBnbStride);
  const float4 l0 = lp[0], l1 = lp[1], l2 = lp[2], l3 = lp[3];
  const float4 i0 = ip[0], i1 = ip[1];
  const unsigned i = (unsigned)(o >> nlb);
  const float cr[kBnbItBits] = {l2.x, l2.y, l2.z, l2.w, l3.x};
  float x = 0.f;
#pragma unroll
  for (int ii = 0; ii < kBnbItBits; ++ii) x = fmaf(((i >> ii) & 1u) ? 1.f : 0.f, cr[ii], x);
  A = (l0.x + x) + i0.x;
  L[0] = l0.y + i0.y;
  L[1] = l0.z + i0.z;
  L[2] = l0.w + i0.w;
  L[3] = l1.x + i1.x;
  L[4] = l1.y + i1.y;
  L[5] = l1.z + i1.z;
  L[6] = l1.w + i1.w;
}

// Pruned search of one pixel by its team (every lane of the team calls it,
// lane lt of T, tmask the team's lanes).  Results per lane, for the team's
// top-two merge and team_finish: the lane's best block minimum m1 with its
// block id b1 = (o << L2) | middle pattern, and its second-best block
// minimum m2.  bound: the pixel's FP32 error bound (the cut's margin);
// qneg: the model's lower bound of any pair-term sum.  pm, vv, itab, ltab,
// lb, rbuf: the team's shared tables (kMaxDot x kLdM slot pairs, kMaxDot
// single-flip energies, (1 << kBnbItBits) kBnbStride-rows, a kBnbLane-row per
// lane, kBnbStates FP16 bounds, kBnbBuf collected patterns and their bounds,
// 2^L1 inner pair terms, 16-byte aligned).
template <bool CLOSED>
__device__ __forceinline__ void search_bnb(const float* __restrict__ sM, const SlotView sv,
                                           int lt, int T, unsigned tmask, float bound,
                                           float qneg, float* pm, float* vv, float* itab,
                                           float* ltab, __half* lb, unsigned short* rbuf,
                                           float* rlb, float* ptab,
                                           float& m1, unsigned& b1, float& m2,
                                           unsigned long long& evaluated) {
  constexpr int L1 = kBnbL1, L2 = kBnbL2, NI = 1 << L1, NM = 1 << L2;
  static_assert(kBnbIn == 7 && kBnbStride == 8 && kBnbLane >= 1 + kBnbIn + kBnbItBits,
                "pruned-search table layout");
  const int k = sv.k;
  const int nmid = min(max(k - L1, 0), L2);
  const int nout = max(k - kBnbIn, 0);
  const int nlb = min(__ffs(T) - 1, nout);
  const int nit = nout - nlb;
  const int nsteps = 1 << nmid;
  const bool own = lt < (1 << nlb);
  const int w = sv.w;                                   // closed: candidate weight
  const int lpop = __popc((unsigned)lt & ((1u << nlb) - 1u));  // the lane bits set

  // team tables: slot pairs and single-flip energies first, then the
  // iteration slots' terms and each owning lane's lane-bit part with its pair
  // terms with every iteration slot (fixed-range 0 / 1-weighted sums, the same
  // trip count in every lane)
  bnb_pair_build(sM, sv, lt, T, pm, vv);
  __syncwarp(tmask);
  bnb_iter_build(pm, vv, lt, T, nlb, nit, itab);
  float At = 0.f, Lt[kBnbIn], cr[kBnbItBits];
#pragma unroll
  for (int j = 0; j < kBnbIn; ++j) Lt[j] = vv[j];
#pragma unroll
  for (int ii = 0; ii < kBnbItBits; ++ii) cr[ii] = 0.f;
  if (own) {
    constexpr int kLB = 5;  // lane bits at most (T <= 32)
    float wO[kLB];
#pragma unroll
    for (int i = 0; i < kLB; ++i) wO[i] = (i < nlb && ((lt >> i) & 1)) ? 1.f : 0.f;
#pragma unroll
    for (int i = 0; i < kLB; ++i) {
      const int si = min(kBnbIn + i, kMaxDot - 1);
      const float* prow = pm + si * kLdM;
      float add = vv[si];
#pragma unroll
      for (int i2 = 0; i2 < i; ++i2) add = fmaf(wO[i2], prow[kBnbIn + i2], add);
      At = fmaf(wO[i], add, At);
#pragma unroll
      for (int j = 0; j < kBnbIn; ++j) Lt[j] = fmaf(wO[i], prow[j], Lt[j]);
#pragma unroll
      for (int ii = 0; ii < kBnbItBits; ++ii)
        cr[ii] = fmaf((ii < nit) ? wO[i] : 0.f, prow[min(kBnbIn + nlb + ii, kMaxDot - 1)], cr[ii]);
    }
    float4* my = reinterpret_cast<float4*>(ltab + lt * kBnbLane);
    my[0] = make_float4(At, Lt[0], Lt[1], Lt[2]);
    my[1] = make_float4(Lt[3], Lt[4], Lt[5], Lt[6]);
    my[2] = make_float4(cr[0], cr[1], cr[2], cr[3]);
    my[3] = make_float4(cr[4], 0.f, 0.f, 0.f);
  }
  // closed: the r smallest walked coefficients, bounded once per lane.  A
  // pattern's coefficient L_oj is the lane part Lt[j] plus the pair terms of
  // its iteration bits, each at least min(0, M(j, s)), so the sorted lane
  // parts with those minima added bound the sorted L_oj slot by slot; the sum
  // of their r smallest is tabulated by the iteration pattern's popcount
  // (r = w - |o|), +inf where no candidate of that weight exists
  float rsum[kBnbItBits + 1];
  if (CLOSED) {
    const int s0 = kBnbIn + nlb;
    float c[kBnbIn];
#pragma unroll
    for (int j = 0; j < kBnbIn; ++j) {
      float lo = Lt[j];
#pragma unroll
      for (int ii = 0; ii < kBnbItBits; ++ii)
        lo += (ii < nit) ? fminf(0.f, pm[j * kLdM + min(s0 + ii, kMaxDot - 1)]) : 0.f;
      c[j] = j < k ? lo : kBig;
    }
    bnb_sort7(c);
    float pre[kBnbIn + 1];
    pre[0] = 0.f;
#pragma unroll
    for (int j = 0; j < kBnbIn; ++j) pre[j + 1] = pre[j] + c[j];
    const int rmax = min(k, kBnbIn);
#pragma unroll
    for (int pc = 0; pc <= kBnbItBits; ++pc) {
      const int r = w - lpop - pc;
      float s = kInf;
#pragma unroll
      for (int j = 0; j <= kBnbIn; ++j) s = (j == r && r <= rmax) ? pre[j] : s;
      rsum[pc] = s;
    }
  }
  __syncwarp(tmask);

  // bounds of the lane's own outer patterns (all 2^kBnbItBits rows are read:
  // rows past 2^nit hold garbage that the masks below drop), and the lowest
  const int nst = own ? (1 << nit) : 0;
  float lbest = kInf;
  int ibest = 0;
#pragma unroll
  for (int i = 0; i < (1 << kBnbItBits); ++i) {
    const float4* ip = reinterpret_cast<const float4*>(itab + i * kBnbStride);
    const float4 i0 = ip[0], i1 = ip[1];
    float x = 0.f;
#pragma unroll
    for (int ii = 0; ii < kBnbItBits; ++ii)
      if ((i >> ii) & 1) x += cr[ii];
    const float A = (At + x) + i0.x;
    float v;
    if (!CLOSED) {
      const float s0 = fminf(0.f, Lt[0] + i0.y) + fminf(0.f, Lt[1] + i0.z);
      const float s1 = fminf(0.f, Lt[2] + i0.w) + fminf(0.f, Lt[3] + i1.x);
      const float s2 = fminf(0.f, Lt[4] + i1.y) + fminf(0.f, Lt[5] + i1.z);
      const float s3 = fminf(0.f, Lt[6] + i1.w);
      v = (A + ((s0 + s1) + (s2 + s3))) + qneg;
    } else {
      (void)i1;
      v = (A + rsum[popc_c((unsigned)i)]) + qneg;
    }
    // stored rounded down to FP16: still a lower bound, half the space
    if (i < nst) lb[lt | (i << nlb)] = __float2half_rd(v);
    const bool better = i < nst && v < lbest;
    lbest = better ? v : lbest;
    ibest = better ? i : ibest;
  }

  // the walk of one outer pattern: its 2^nmid middle states, each with the
  // inner table evaluated by doubling (inner_min_open)
  // the inner pair table P[b] = sum_{j < l in b} M(j, l), one entry per
  // lane at a time into the team's shared row (fixed-range 0 / 1 weights)
  for (int b = lt; b < NI; b += T) {
    float r = 0.f;
#pragma unroll
    for (int j = 1; j < L1; ++j)
#pragma unroll
      for (int l = 0; l < j; ++l)
        r = fmaf((((b >> j) & 1) && ((b >> l) & 1)) ? 1.f : 0.f, pm[j * kLdM + l], r);
    ptab[b] = r;
  }
  float Mmm[L2][L2], Mim[L1][L2];
#pragma unroll
  for (int m = 0; m < L2; ++m)
#pragma unroll
    for (int m2 = 0; m2 < L2; ++m2)
      Mmm[m][m2] = (m != m2 && m < nmid && m2 < nmid) ? pm[(L1 + m) * kLdM + L1 + m2] : 0.f;
#pragma unroll
  for (int j = 0; j < L1; ++j)
#pragma unroll
    for (int m = 0; m < L2; ++m)
      Mim[j][m] = (m < nmid) ? pm[j * kLdM + L1 + m] : 0.f;
  float g1 = kInf, g2 = kInf;
  unsigned blk = 0u;
  unsigned long long ev = 0;
  auto walk = [&](int o) {
    float A, L[kBnbIn];
    bnb_rest(ltab, itab, nlb, o, A, L);
    float q[L1], gm[L2];
#pragma unroll
    for (int j = 0; j < L1; ++j) q[j] = L[j];
#pragma unroll
    for (int m = 0; m < L2; ++m) gm[m] = L[L1 + m];
    const unsigned obase = (unsigned)o << L2;
#pragma unroll
    for (int s = 0; s < NM; ++s) {
      if (s >= nsteps) continue;
      if (s > 0) {
        const int mb = ctz_c((unsigned)s);
        const bool up = (gray_c((unsigned)s) >> mb) & 1u;
        A = up ? A + gm[mb] : A - gm[mb];
#pragma unroll
        for (int m = 0; m < L2; ++m)
          if (m != mb) gm[m] = up ? gm[m] + Mmm[m][mb] : gm[m] - Mmm[m][mb];
#pragma unroll
        for (int j = 0; j < L1; ++j) q[j] = up ? q[j] + Mim[j][mb] : q[j] - Mim[j][mb];
      }
      float mbk;
      if (!CLOSED) {
        mbk = inner_min_open_smem<L1>(A, q, ptab);
      } else {
        const int rr = w - __popc((unsigned)o) - popc_c(gray_c((unsigned)s));
        mbk = inner_min_closed_smem<L1>(A, q, ptab, rr);
      }
      const unsigned id = obase | gray_c((unsigned)s);
      g2 = fminf(g2, fmaxf(g1, mbk));
      const bool better = mbk < g1;
      g1 = better ? mbk : g1;
      blk = better ? id : blk;
    }
    ev += (unsigned long long)nsteps * NI;
  };
  __syncwarp(tmask);  // the pair table is complete

  // round one: every owning lane walks its lowest-bound pattern
  const __half taken = __ushort_as_half((unsigned short)0x7e00);  // NaN: passes no cut
  if (own) {
    const int o = lt | (ibest << nlb);
    lb[o] = taken;
    walk(o);
  }
  float cut = g1, c2 = g2;
  team_top2(tmask, T, cut, c2);
  cut = c2;
  const float slack = 2.0f * bound;

  // the patterns still below the cut, collected (lane order, at most kBnbBuf
  // per pass; a taken pattern's bound becomes NaN) and walked in rounds of
  // T, the cut re-checked and tightened every round; passes repeat until no
  // pattern is left below the cut
  const unsigned nmask = nst >= 32 ? 0xffffffffu : ((1u << nst) - 1u);
  for (;;) {
    const float thr = cut + slack;
    unsigned smask = 0u;
#pragma unroll
    for (int i = 0; i < (1 << kBnbItBits); ++i)
      smask |= (__half2float(lb[(lt | (i << nlb)) & (kBnbStates - 1)]) <= thr) ? (1u << i) : 0u;
    smask &= nmask;
    const int cnt = __popc(smask);
    int pre = cnt;  // inclusive prefix over the team's lanes
    for (int off = 1; off < T; off <<= 1) {
      const int y = __shfl_up_sync(tmask, pre, off, T);
      if (lt >= off) pre += y;
    }
    const int total = min(__shfl_sync(tmask, pre, T - 1, T), kBnbBuf);
    if (total == 0) break;
    int at = pre - cnt;
    for (unsigned mm = smask; mm && at < kBnbBuf; mm &= mm - 1u, ++at) {
      const int o = lt | ((__ffs(mm) - 1) << nlb);
      rbuf[at] = (unsigned short)o;
      rlb[at] = __half2float(lb[o]);
      lb[o] = taken;
    }
    __syncwarp(tmask);
    for (int r0 = 0; r0 < total; r0 += T) {
      const int e = r0 + lt;
      if (e < total && rlb[e] <= cut + slack) walk(rbuf[e]);
      float t1 = g1, t2 = g2;
      team_top2(tmask, T, t1, t2);
      cut = fminf(cut, t2);
    }
    __syncwarp(tmask);
  }
  evaluated += ev;
  m1 = g1;
  b1 = blk;
  m2 = g2;
}

// Top-two merge of (m1, b1, m2) triples; FP32 ties go to the pattern whose
// charge vector is lexicographically smaller (bit-reversed order).
__device__ __forceinline__ void top2_merge(float& m1, unsigned& b1, float& m2,
                                           float om1, unsigned ob1, float om2) {
  const bool take = (om1 < m1) || (om1 == m1 && __brev(ob1) < __brev(b1));
  const float hi = take ? m1 : om1;
  m2 = fminf(fminf(m2, om2), hi);
  if (take) { m1 = om1; b1 = ob1; }
}

// Per-pixel near-tie bound: the FP32 gap below which the order of the best
// two candidates is not certain.  Every energy is reached through a chain of
// at most (2^L2 + 2k + 8) FP32 additions (scratch sum of the rest-state, the
// middle Gray walk, the inner tree), each partial sum bounded by
// S = sum |h_j| + sum_j M_jj / 2 + sum_{j<l} |M_jl| over the ambiguous slots,
// and each rounding adds at most 2^-24 S.  The gap threshold is twice that.
// (The recheck shortlists by the same margin, and the parity tests check on
// every comparable pixel that no mismatch escapes it.)
__device__ __forceinline__ float near_tie_bound(float S, int k, int L2, int extra = 0) {
  return 2.0f * (float)((1 << L2) + 2 * k + 8 + extra) * 5.9604645e-8f * S;
}

}  // namespace qa
