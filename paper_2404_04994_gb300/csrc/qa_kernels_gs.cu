// qa_kernels_gs.cu -- ground-state kernels: per-pixel preparation, the
// candidate search, and the FP64 recheck of flagged pixels.
#include "qa_launch.h"
#include "qa_prep.cuh"
#include "qa_search.cuh"

namespace qa {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPrepThreads = 128;
constexpr int kSearchThreads = 128;
constexpr int kRecheckThreads = 128;
constexpr int kResolveThreads = 256;
constexpr int kRecheckL1 = 4, kRecheckL2 = 3;  // 2^9 outer states at k = 16
constexpr unsigned kBcap = 1024;

// number of k-subsets of size w (k <= 16)
__device__ __forceinline__ unsigned long long binom(int k, int w) {
  if (w < 0 || w > k) return 0ull;
  unsigned long long r = 1ull;
  for (int i = 1; i <= w; ++i) r = r * (unsigned long long)(k - w + i) / (unsigned long long)i;
  return r;
}

// ---------------------------------------------------------------------------
// (a0) raster constants of a block: c(ix, iy) = c0 + ix du + iy dw with
// c0 = s Cgd (V0 + x0 u + y0 w), du = s Cgd u dx, dw = s Cgd w dy, formed in
// double-float FP32 from FP64 inputs (one FP64 rounding per input, no FP64
// dependency chains: FP64 issues at a small fraction of the FP32 rate here).
// ---------------------------------------------------------------------------
__device__ inline void raster_consts(const ModelData* md, int n, int ng, const Scan& sc,
                                     double carrier, df* sV, df* sU, df* sW, df* c0,
                                     df* du, df* dw) {
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    sV[g] = df_from_double(sc.V0[g] + sc.x0 * sc.u[g] + sc.y0 * sc.w[g]);
    sU[g] = df_from_double(sc.u[g] * sc.dx);
    sW[g] = df_from_double(sc.w[g] * sc.dy);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 3 * n; e += blockDim.x) {
    const int i = e % n, which = e / n;
    const df* vec = which == 0 ? sV : (which == 1 ? sU : sW);
    df acc = {0.f, 0.f};
    for (int g = 0; g < ng; ++g)
      acc = df_add(acc, df_mul(df_from_double(carrier * md->Cgd[i * ng + g]), vec[g]));
    (which == 0 ? c0 : (which == 1 ? du : dw))[i] = acc;
  }
}

// Block sum of per-thread counts (all threads must call; result in thread 0).
template <typename U>
__device__ __forceinline__ U block_sum(U v, U* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  U t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// ---------------------------------------------------------------------------
// (a1)-(a4): induced charge, continuous minimum, candidate set, h = M(base-c)
//
// A team of TP lanes (a power of two >= N, at most 16) prepares one pixel,
// lane i owning dot i; team-wide sums, ballots and gathers use shuffles
// restricted to the team's lanes, so teams of one warp may diverge.
// ---------------------------------------------------------------------------
template <bool CLOSED>
__global__ void __launch_bounds__(kPrepThreads) k_prep(GsLaunch a) {
  __shared__ ModelConsts cs;
  __shared__ df sV[kMaxGate], sU[kMaxGate], sW[kMaxGate];
  __shared__ df sc0[kMaxDot], sdu[kMaxDot], sdw[kMaxDot];
  __shared__ float sx[kPrepThreads];
  __shared__ int sst[kPrepThreads];
  __shared__ unsigned long long red64[kPrepThreads / 32];
  __shared__ unsigned red32[kPrepThreads / 32];
  const int n = a.n;
  stage_consts(&a.md->k, &cs);
  if (a.sc.kind == 0) {
    if (a.rk.valid) {
      if (threadIdx.x < kMaxDot) {
        sc0[threadIdx.x] = a.rk.c0[threadIdx.x];
        sdu[threadIdx.x] = a.rk.du[threadIdx.x];
        sdw[threadIdx.x] = a.rk.dw[threadIdx.x];
      }
    } else {
      raster_consts(a.md, n, a.ng, a.sc, a.mt.carrier, sV, sU, sW, sc0, sdu, sdw);
    }
  }
  __syncthreads();
  const float* sMhi = cs.Mhi;
  const float* sMlo = cs.Mlo;
  const float bx_qp_scale = a.bx_qp_scale > 0.f ? a.bx_qp_scale : cs.bx_qp_scale;
  const bool model_bad = cs.model_bad != 0;

  const int TP = a.prep_team;
  const int lt = threadIdx.x & (TP - 1);
  const int lane = threadIdx.x & 31;
  const int tbase = lane & ~(TP - 1);                   // team's first lane
  const unsigned tmask = (TP == 32 ? 0xffffffffu : ((1u << TP) - 1u)) << tbase;
  const long long p = (long long)blockIdx.x * (kPrepThreads / TP) + threadIdx.x / TP;
  const bool active = p < a.sc.P;
  const bool live = active && lt < n;
  const int nhat = a.mt.n_charges;

  // team reductions over lanes (dead lanes contribute zero)
  auto tsum_f = [&](float v) {
    for (int off = 1; off < TP; off <<= 1) v += __shfl_xor_sync(tmask, v, off, TP);
    return v;
  };
  auto tmax_f = [&](float v) {
    for (int off = 1; off < TP; off <<= 1) v = fmaxf(v, __shfl_xor_sync(tmask, v, off, TP));
    return v;
  };
  auto tsum_i = [&](int v) {
    for (int off = 1; off < TP; off <<= 1) v += __shfl_xor_sync(tmask, v, off, TP);
    return v;
  };
  auto tsum_df = [&](df v) {
    for (int off = 1; off < TP; off <<= 1) {
      df o;
      o.hi = __shfl_xor_sync(tmask, v.hi, off, TP);
      o.lo = __shfl_xor_sync(tmask, v.lo, off, TP);
      v = df_add(v, o);
    }
    return v;
  };
  auto tballot = [&](bool pred) { return (__ballot_sync(tmask, pred) & tmask) >> tbase; };

  // (a1) c_i
  df c = {0.f, 0.f};
  if (live) {
    if (a.sc.kind == 0) {
      const int ix = (int)(p % a.sc.W), iy = (int)(p / a.sc.W);
      c = raster_c(sc0[lt], sdu[lt], sdw[lt], ix, iy);
    } else {
      c = point_c(&a.md->Cgd[lt * a.ng], &a.sc.V[p * a.ng], a.ng, a.mt.carrier);
    }
  }
  // (a2) analytic continuous minimum (Appendix C / D)
  df x = c;
  if (CLOSED) {
    const df csum = tsum_df(c);
    const df lam = df_sub({(float)nhat, 0.f}, csum);  // N_hat <= 2^24
    if (live) x = df_add(c, df_mul(lam, cs.vs[lt]));
  }
  const unsigned A =
      tballot(live && (x.hi < 0.f || (x.hi == 0.f && x.lo < 0.f)));
  unsigned flags = 0u;
  float bx = a.bx_analytic;
  const float cmax = tmax_f(live ? fabsf(c.hi + c.lo) : 0.f);
  if (A) {  // (a3) QP, solved by the team's first lane
    flags |= kFlagQP;
    if (CLOSED && nhat == 0) {
      x = {0.f, 0.f};
    } else {
      const float scale = 1.f + cmax + (float)nhat;
      bx = fmaxf(bx, bx_qp_scale * scale);
      sx[threadIdx.x] = c.hi + c.lo;
      __syncwarp(tmask);
      if (lt == 0) {
        float cf[kMaxDot], xf[kMaxDot];
        for (int j = 0; j < n; ++j) cf[j] = sx[threadIdx.x + j];
        const int st = qp_active_set<float>(n, cs.Cdd, kLdM, cf, CLOSED, (float)nhat,
                                            cs.sv, cs.s_s, A, 0.25f * bx_qp_scale * scale,
                                            4 * n + 4, xf);
        for (int j = 0; j < n; ++j) sx[threadIdx.x + j] = xf[j];
        sst[threadIdx.x] = st;
      }
      __syncwarp(tmask);
      if (live) x = {sx[threadIdx.x], 0.f};
      if (sst[threadIdx.x - lt] != 0) flags |= kFlagQPCap;
      __syncwarp(tmask);
    }
  }

  // (a4) candidate set; the closed doubling loop is team-uniform
  double tt = a.mt.t;
  unsigned mask = 0u;
  int w = -1, base = 0;
  bool amb = false;
  for (int iter = 0; iter < 40; ++iter) {
    const float th = __double2float_rn(0.5 * tt);
    bool bnd = false;
    if (live) {
      df xi = x;
      if (xi.hi < 0.f || (xi.hi == 0.f && xi.lo < 0.f)) xi = {0.f, 0.f};
      float fl = floorf(xi.hi);
      if (xi.hi == fl && xi.lo < 0.f) fl -= 1.f;
      const float fr = __fadd_rn(__fsub_rn(xi.hi, fl), xi.lo);
      amb = fabsf(fr - 0.5f) <= th;
      base = (int)fl + ((!amb && fr >= 0.5f) ? 1 : 0);
      bnd = (xi.hi >= 0.5f - bx && fminf(fr, 1.f - fr) < bx) ||
            (tt < 1.0 && fabsf(fabsf(fr - 0.5f) - th) < bx);
    }
    if (tballot(bnd)) flags |= kFlagBoundary;
    mask = tballot(live && amb);
    const int sum = tsum_i(live ? base : 0);
    if (!CLOSED) break;
    w = nhat - sum;
    if (w >= 0 && w <= __popc(mask)) break;
    if (tt >= 1.0) {  // impossible in exact arithmetic: settle in FP64
      flags |= kFlagBoundary;
      w = w < 0 ? 0 : __popc(mask);
      break;
    }
    tt = (tt <= 0.0) ? 1.0 : fmin(2.0 * tt, 1.0);
    flags |= kFlagDoubled;
  }
  if (model_bad) flags |= kFlagUnresolved;

  // h_i = (M (base - c))_i in double-float, r_j gathered from the team
  const df r = df_sub({(float)base, 0.f}, c);
  df acc = {0.f, 0.f};
  for (int j = 0; j < n; ++j) {
    df rj;
    rj.hi = __shfl_sync(tmask, r.hi, j, TP);
    rj.lo = __shfl_sync(tmask, r.lo, j, TP);
    if (live) acc = df_add(acc, df_mul({sMhi[lt * kLdM + j], sMlo[lt * kLdM + j]}, rj));
  }
  const float h = acc.hi + acc.lo;
  float Si = 0.f;
  if (live && amb) {
    Si = fabsf(h) + 0.5f * sMhi[lt * kLdM + lt];
    for (unsigned m2 = mask & ((1u << lt) - 1u); m2; m2 &= m2 - 1u)
      Si += fabsf(sMhi[lt * kLdM + (__ffs(m2) - 1)]);
  }
  const float S = tsum_f(Si);
  const int k = __popc(mask);

  PixRec* rec = a.recs + (active ? p : 0);
  if (live) {
    rec->h[lt] = h;
    rec->chi[lt] = c.hi;
    rec->clo[lt] = c.lo;
    rec->base[lt] = (short)base;
  }
  unsigned long long my_cand = 0;
  unsigned my_qp = 0, my_doubled = 0;
  if (active && lt == 0) {
    rec->mask = (unsigned short)mask;
    rec->k = (unsigned char)k;
    rec->w = (signed char)(CLOSED ? w : -1);
    rec->flags = (unsigned char)flags;
    rec->bound = near_tie_bound(S, k, a.cfg.L2);
    my_cand = CLOSED ? binom(k, w) : (1ull << k);
    my_qp = (flags & kFlagQP) ? 1u : 0u;
    my_doubled = (flags & kFlagDoubled) ? 1u : 0u;
  }
  __syncwarp();
  const unsigned long long bc = block_sum(my_cand, red64);
  const unsigned bq = block_sum(my_qp, red32);
  const unsigned bd = block_sum(my_doubled, red32);
  if (threadIdx.x == 0) {
    BlockCounts& o = a.bc_prep[blockIdx.x];
    o.candidates = bc;
    o.qp = bq;
    o.doubled = bd;
  }
}

// ---------------------------------------------------------------------------
// (a5)-(a6), (a8): candidate search, top-two selection, outputs
// ---------------------------------------------------------------------------
template <int L1, int L2, bool CLOSED>
__global__ void __launch_bounds__(kSearchThreads) k_search(GsLaunch a) {
  __shared__ ModelConsts cs;
  __shared__ int sdot[kSearchThreads][kMaxDot];
  __shared__ float sh[kSearchThreads][kMaxDot];
  __shared__ unsigned long long red64[kSearchThreads / 32];
  __shared__ unsigned red32[kSearchThreads / 32];
  const int n = a.n;
  stage_consts(&a.md->k, &cs);
  __syncthreads();
  const float* sM = cs.Mhi;
  const float* sMlo = cs.Mlo;

  const int T = a.cfg.T;
  const int team = threadIdx.x / T, lt = threadIdx.x % T;
  const int teams = blockDim.x / T;
  const long long p = (long long)blockIdx.x * teams + team;
  const bool active = p < a.sc.P;
  const PixRec* rec = a.recs + (active ? p : 0);
  const unsigned mask = active ? rec->mask : 0u;
  const int k = __popc(mask);
  if (active && lt == 0) {
    int s = 0;
    for (unsigned m = mask; m; m &= m - 1u) {
      const int i = __ffs(m) - 1;
      sdot[team][s] = i;
      sh[team][s] = rec->h[i];
      ++s;
    }
  }
  __syncwarp();
  float m1 = kInf, m2 = kInf;
  unsigned b1 = 0u;
  unsigned long long ev = 0;
  if (active) {
    SlotView sv{sdot[team], sh[team], k, (int)rec->w};
    search_lane<L1, L2, CLOSED, false>(sM, sv, lt, T, 0.f, nullptr, nullptr, 0u,
                                       m1, b1, m2, ev);
  }
  for (int off = 1; off < T; off <<= 1) {
    const float om1 = __shfl_xor_sync(kFull, m1, off);
    const unsigned ob1 = __shfl_xor_sync(kFull, b1, off);
    const float om2 = __shfl_xor_sync(kFull, m2, off);
    top2_merge(m1, b1, m2, om1, ob1, om2);
  }

  // epilogue: n* = base + bits, U(n*) = 1/2 r^T M r in double-float (team
  // lanes split the rows; no per-thread arrays, so nothing lands in local
  // memory)
  df u = {0.f, 0.f};
  unsigned flags = 0u;
  if (active) {
    for (int i = lt; i < n; i += T) {
      df acc = {0.f, 0.f};
      for (int j = 0; j < n; ++j) {
        int nj = rec->base[j];
        if ((mask >> j) & 1u) nj += (int)((b1 >> __popc(mask & ((1u << j) - 1u))) & 1u);
        const df rj = df_sub({(float)nj, 0.f}, {rec->chi[j], rec->clo[j]});
        acc = df_add(acc, df_mul({sM[i * kLdM + j], sMlo[i * kLdM + j]}, rj));
      }
      int ni = rec->base[i];
      if ((mask >> i) & 1u) ni += (int)((b1 >> __popc(mask & ((1u << i) - 1u))) & 1u);
      const df ri = df_sub({(float)ni, 0.f}, {rec->chi[i], rec->clo[i]});
      u = df_add(u, df_mul(acc, ri));
      if (ni > 127) { ni = 127; flags |= kFlagOverflow; }
      a.out_n[p * n + i] = (int8_t)ni;
    }
  }
  for (int off = 1; off < T; off <<= 1) {
    df o;
    o.hi = __shfl_xor_sync(kFull, u.hi, off);
    o.lo = __shfl_xor_sync(kFull, u.lo, off);
    u = df_add(u, o);
    flags |= __shfl_xor_sync(kFull, flags, off);
  }
  unsigned my_nt = 0, my_bd = 0, my_ov = 0;
  if (active) {
    flags |= rec->flags;
    if (!(m2 - m1 > rec->bound)) flags |= kFlagNearTie;
    if (lt == 0) {
      if (a.out_U) a.out_U[p] = 0.5 * df_to_double(u);
      if (flags & (kFlagBoundary | kFlagQPCap | kFlagUnresolved)) {
        // the candidate set itself may be wrong: FP64 recheck
        const unsigned at = atomicAdd(&a.cnt->n_flag, 1u);
        a.flag_list[at] = (int)p;
        my_bd = 1;
      } else if (flags & kFlagNearTie) {
        // right set, uncertain order: exact energies of the close candidates
        const unsigned at = atomicAdd(&a.cnt->n_tie, 1u);
        a.tie_list[at] = TieEntry{(int)p, m1};
        my_nt = 1;
      }
      my_ov = (flags & kFlagOverflow) ? 1u : 0u;
      if (a.out_flags) a.out_flags[p] = (uint8_t)flags;
    }
  }
  const unsigned long long bev = block_sum(ev, red64);
  const unsigned bnt = block_sum(my_nt, red32);
  const unsigned bbd = block_sum(my_bd, red32);
  const unsigned bov = block_sum(my_ov, red32);
  if (threadIdx.x == 0) {
    BlockCounts& o = a.bc_search[blockIdx.x];
    o.evaluated = bev;
    o.near_tie = bnt;
    o.boundary = bbd;
    o.overflow = bov;
  }
}

// ---------------------------------------------------------------------------
// (a7, near ties): a pixel whose candidate set is certain but whose FP32
// best/runner-up gap is under the error bound.  One warp per pixel re-walks
// the candidates collecting every block whose FP32 minimum is within the
// bound of the search's minimum (the exact argmin is guaranteed to be among
// them) and evaluates those candidates exactly, relative to the base state,
//     E(b) = sum_{s in b} (h_s + M_ss / 2) + sum_{s < s' in b} M_ss',
// in double-float arithmetic with h = M (base - c) in double-float (about
// 1e-13 absolute).  No FP64 instructions: GB300's FP64 rate is a small
// fraction of its FP32 rate.  A pixel whose two best exact energies are
// within 1e-10 (a true tie) or whose list overflows goes on to the FP64
// recheck, which also applies the lexicographic tie rule.
// ---------------------------------------------------------------------------
template <int L1, int L2, bool CLOSED>
__global__ void __launch_bounds__(kResolveThreads) k_resolve(GsLaunch a) {
  constexpr int NI = 1 << L1;
  constexpr int NM = 1 << L2;
  constexpr int NW = kResolveThreads / 32;
  constexpr unsigned kCap = 128;
  __shared__ ModelConsts cs;
  __shared__ int sdot[kMaxDot];
  __shared__ float sh[kMaxDot];
  __shared__ df shd[kMaxDot];
  __shared__ df sui[kMaxDot];
  __shared__ unsigned blist[kCap];
  __shared__ unsigned bcnt;
  __shared__ df rbest[NW], rsec[NW];
  __shared__ unsigned rbits[NW];
  stage_consts(&a.md->k, &cs);
  __syncthreads();
  const float* sM = cs.Mhi;
  const float* sMlo = cs.Mlo;
  const int n = a.n;
  const unsigned ntie = a.cnt->n_tie;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  unsigned my_res = 0;
  for (unsigned it = blockIdx.x; it < ntie; it += gridDim.x) {
    const TieEntry te = a.tie_list[it];
    const long long p = te.p;
    const PixRec* rec = a.recs + p;
    const unsigned mask = rec->mask;
    const int k = __popc(mask);
    const int w = rec->w;
    // h_i = (M (base - c))_i in double-float, and U(base) = r0 . h / 2
    if (tid < n) {
      df hi = {0.f, 0.f};
      for (int j = 0; j < n; ++j) {
        const df rj = df_sub({(float)rec->base[j], 0.f}, {rec->chi[j], rec->clo[j]});
        hi = df_add(hi, df_mul({sM[tid * kLdM + j], sMlo[tid * kLdM + j]}, rj));
      }
      const df r0 = df_sub({(float)rec->base[tid], 0.f}, {rec->chi[tid], rec->clo[tid]});
      sui[tid] = df_mul(hi, r0);
      if ((mask >> tid) & 1u) {
        const int s = __popc(mask & ((1u << tid) - 1u));
        sdot[s] = tid;
        sh[s] = rec->h[tid];
        shd[s] = df_add(hi, df_mul_f({sM[tid * kLdM + tid], sMlo[tid * kLdM + tid]}, 0.5f));
      }
    }
    if (tid == 0) bcnt = 0u;
    __syncthreads();
    // every block whose FP32 minimum is within the bound of the search's
    const SlotView sv{sdot, sh, k, w};
    const float thr = te.m1 + rec->bound;
    float d1, d2;
    unsigned db;
    unsigned long long ev = 0;
    search_lane<L1, L2, CLOSED, true>(sM, sv, tid, kResolveThreads, thr, blist, &bcnt,
                                      kCap, d1, db, d2, ev);
    __syncthreads();
    const unsigned nb = bcnt;
    const bool fits = nb <= kCap;
    df best = {kInf, 0.f}, second = {kInf, 0.f};
    unsigned bbits = 0xffffffffu;
    if (fits) {
      for (unsigned idx = tid; idx < nb * NI; idx += kResolveThreads) {
        const unsigned id = blist[idx / NI];
        const unsigned b = idx % NI;
        const unsigned bits = ((id >> L2) << (L1 + L2)) | ((id & (NM - 1)) << L1) | b;
        if ((bits >> k) != 0u) continue;
        if (CLOSED && __popc(bits) != w) continue;
        df E = {0.f, 0.f};
        for (unsigned m = bits; m; m &= m - 1u) {
          const int s = __ffs(m) - 1;
          const int d = sdot[s];
          E = df_add(E, shd[s]);
          for (unsigned q = bits & ((1u << s) - 1u); q; q &= q - 1u) {
            const int d2i = sdot[__ffs(q) - 1];
            E = df_add(E, {sM[d * kLdM + d2i], sMlo[d * kLdM + d2i]});
          }
        }
        const bool better = E.hi < best.hi || (E.hi == best.hi && E.lo < best.lo) ||
                            (E.hi == best.hi && E.lo == best.lo && __brev(bits) < __brev(bbits));
        if (better) { second = best; best = E; bbits = bits; }
        else if (E.hi < second.hi || (E.hi == second.hi && E.lo < second.lo)) { second = E; }
      }
    }
    auto less = [](df x, df y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); };
    auto merge = [&](df ob, df os, unsigned obb) {
      const bool take = less(ob, best) ||
                        (ob.hi == best.hi && ob.lo == best.lo && __brev(obb) < __brev(bbits));
      const df lose = take ? best : ob;
      const df s2 = less(os, second) ? os : second;
      second = less(lose, s2) ? lose : s2;
      if (take) { best = ob; bbits = obb; }
    };
    for (int off = 16; off > 0; off >>= 1) {
      df ob, os;
      ob.hi = __shfl_xor_sync(kFull, best.hi, off);
      ob.lo = __shfl_xor_sync(kFull, best.lo, off);
      os.hi = __shfl_xor_sync(kFull, second.hi, off);
      os.lo = __shfl_xor_sync(kFull, second.lo, off);
      merge(ob, os, __shfl_xor_sync(kFull, bbits, off));
    }
    if (lane == 0) { rbest[wid] = best; rsec[wid] = second; rbits[wid] = bbits; }
    __syncthreads();
    if (tid == 0) {
      for (int i = 1; i < NW; ++i) merge(rbest[i], rsec[i], rbits[i]);
      df ub = {0.f, 0.f};
      for (int i = 0; i < n; ++i) ub = df_add(ub, sui[i]);
      ub = df_mul_f(ub, 0.5f);
      const double gap = df_to_double(second) - df_to_double(best);
      const double eps = 1e-10 * (1.0 + fabs(df_to_double(ub)));
      if (!fits || bbits == 0xffffffffu || !(gap > eps)) {
        const unsigned at = atomicAdd(&a.cnt->n_flag, 1u);
        a.flag_list[at] = (int)p;
      } else {
        unsigned flags = (a.out_flags ? a.out_flags[p] : 0u) | kFlagRechecked;
        for (int i = 0; i < n; ++i) {
          int ni = rec->base[i];
          if ((mask >> i) & 1u) ni += (int)((bbits >> __popc(mask & ((1u << i) - 1u))) & 1u);
          if (ni > 127) { ni = 127; flags |= kFlagOverflow; }
          a.out_n[p * n + i] = (int8_t)ni;
        }
        if (a.out_U) a.out_U[p] = df_to_double(df_add(ub, best));
        if (a.out_flags) a.out_flags[p] = (uint8_t)flags;
        my_res += 1;
      }
      atomicMax(&a.cnt->shortlist_max, (unsigned long long)nb);
    }
    __syncthreads();
  }
  if (tid == 0 && my_res) atomicAdd(&a.cnt->resolved, (unsigned long long)my_res);
}

// ---------------------------------------------------------------------------
// (a7): FP64 recheck of flagged pixels.  One block per pixel (grid-stride
// over the list written by the search kernel):
//   1. c, the continuous minimum and the candidate set again, in FP64
//      (c and h by N threads in parallel, the minimum by one thread);
//   2. the FP32 search over that set with all threads -> m1;
//   3. the same search collecting every block whose minimum is within the
//      near-tie bound of m1 (the exact argmin is guaranteed to be there);
//   4. exact FP64 energies of those candidates, ties to the
//      lexicographically smallest charge vector.
// ---------------------------------------------------------------------------
template <bool CLOSED>
__global__ void __launch_bounds__(kRecheckThreads) k_recheck(GsLaunch a) {
  constexpr int L1 = kRecheckL1, L2 = kRecheckL2;
  constexpr int NI = 1 << L1;
  constexpr int NM = 1 << L2;
  constexpr int NW = kRecheckThreads / 32;
  __shared__ float sM[kMaxDot * kLdM];
  __shared__ int sdot[kMaxDot];
  __shared__ float sh[kMaxDot];
  __shared__ double sh64[kMaxDot], sc64[kMaxDot];
  __shared__ int sbase[kMaxDot];
  __shared__ int sk, sw, sstatus;
  __shared__ unsigned smask, sflags;
  __shared__ float sbound;
  __shared__ float rm1[NW];
  __shared__ double re[NW];
  __shared__ unsigned rbits[NW];
  __shared__ unsigned blist[kBcap];
  __shared__ unsigned bcount;
  const int n = a.n;
  for (int e = threadIdx.x; e < kMaxDot * kLdM; e += blockDim.x) sM[e] = a.md->k.Mhi[e];
  __syncthreads();
  const unsigned nflag = a.cnt->n_flag;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;

  for (unsigned it = blockIdx.x; it < nflag; it += gridDim.x) {
    const long long p = a.flag_list[it];
    if (tid < n) sc64[tid] = pixel_c_f64(a.md, a.ng, a.sc, a.mt.carrier, p, tid);
    __syncthreads();
    if (tid == 0) {
      double c[kMaxDot];
      int base[kMaxDot];
      unsigned mask = 0u, fl = 0u;
      int w = -1;
      for (int i = 0; i < n; ++i) c[i] = sc64[i];
      sstatus = (a.md->status != 0) ? -1 : settle_pixel_f64(a.md, n, a.mt, c, base, mask, w, fl);
      sflags = fl;
      smask = mask;
      sw = CLOSED ? w : -1;
      for (int i = 0; i < n; ++i) sbase[i] = base[i];
      bcount = 0u;
    }
    __syncthreads();
    if (sstatus != 0) {
      if (tid == 0) {
        if (a.out_flags) a.out_flags[p] |= (uint8_t)kFlagUnresolved;
        atomicAdd(&a.cnt->unresolved, 1ull);
      }
      __syncthreads();
      continue;
    }
    const unsigned mask = smask;
    if (tid < n && ((mask >> tid) & 1u)) {
      double h = 0.0;
      for (int j = 0; j < n; ++j) h += a.md->M[tid * n + j] * ((double)sbase[j] - sc64[j]);
      const int s = __popc(mask & ((1u << tid) - 1u));
      sdot[s] = tid;
      sh64[s] = h;
      sh[s] = __double2float_rn(h);
    }
    __syncthreads();
    if (tid == 0) {
      const int k = __popc(mask);
      float S = 0.f;
      for (int s = 0; s < k; ++s) {
        S += fabsf(sh[s]) + 0.5f * sM[sdot[s] * kLdM + sdot[s]];
        for (int q = 0; q < s; ++q) S += fabsf(sM[sdot[s] * kLdM + sdot[q]]);
      }
      sk = k;
      sbound = near_tie_bound(S, k, L2);
    }
    __syncthreads();
    const SlotView sv{sdot, sh, sk, sw};
    float m1, m2;
    unsigned b1;
    unsigned long long ev = 0;
    search_lane<L1, L2, CLOSED, false>(sM, sv, tid, kRecheckThreads, 0.f, nullptr,
                                       nullptr, 0u, m1, b1, m2, ev);
    for (int off = 16; off > 0; off >>= 1) m1 = fminf(m1, __shfl_xor_sync(kFull, m1, off));
    if (lane == 0) rm1[wid] = m1;
    __syncthreads();
    m1 = kInf;
    for (int i = 0; i < NW; ++i) m1 = fminf(m1, rm1[i]);
    const float thr = m1 + sbound;
    float d1, d2;
    unsigned db;
    search_lane<L1, L2, CLOSED, true>(sM, sv, tid, kRecheckThreads, thr, blist,
                                      &bcount, kBcap, d1, db, d2, ev);
    __syncthreads();
    const unsigned nb = bcount;
    const bool overflowed = nb > kBcap;
    const unsigned nbl = overflowed ? kBcap : nb;
    // exact FP64 energies of the shortlisted candidates
    double best = 1.0e300;
    unsigned bbits = 0xffffffffu;
    const int k = sk;
    for (unsigned idx = tid; idx < nbl * NI; idx += kRecheckThreads) {
      const unsigned id = blist[idx / NI];
      const unsigned b = idx % NI;
      const unsigned bits = ((id >> L2) << (L1 + L2)) | ((id & (NM - 1)) << L1) | b;
      if ((bits >> k) != 0u) continue;
      if (CLOSED && __popc(bits) != sw) continue;
      double E = 0.0;
      for (unsigned m = bits; m; m &= m - 1u) {
        const int s = __ffs(m) - 1;
        const int d = sdot[s];
        E += sh64[s] + 0.5 * a.md->M[d * n + d];
        for (unsigned q = bits & ((1u << s) - 1u); q; q &= q - 1u)
          E += a.md->M[d * n + sdot[__ffs(q) - 1]];
      }
      if (E < best || (E == best && __brev(bits) < __brev(bbits))) {
        best = E;
        bbits = bits;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double oe = __shfl_xor_sync(kFull, best, off);
      const unsigned ob = __shfl_xor_sync(kFull, bbits, off);
      if (oe < best || (oe == best && __brev(ob) < __brev(bbits))) { best = oe; bbits = ob; }
    }
    if (lane == 0) { re[wid] = best; rbits[wid] = bbits; }
    __syncthreads();
    if (tid == 0) {
      for (int i = 1; i < NW; ++i)
        if (re[i] < best || (re[i] == best && __brev(rbits[i]) < __brev(bbits))) {
          best = re[i];
          bbits = rbits[i];
        }
      unsigned flags = (a.out_flags ? a.out_flags[p] : 0u) | sflags | kFlagRechecked;
      if (overflowed || bbits == 0xffffffffu) {
        flags |= kFlagUnresolved;
        atomicAdd(&a.cnt->unresolved, 1ull);
      } else {
        int nst[kMaxDot];
        for (int i = 0; i < n; ++i) nst[i] = sbase[i];
        for (int s = 0; s < k; ++s)
          if ((bbits >> s) & 1u) nst[sdot[s]] += 1;
        double U = 0.0;
        for (int i = 0; i < n; ++i) {
          double row = 0.0;
          for (int j = 0; j < n; ++j) row += a.md->M[i * n + j] * ((double)nst[j] - sc64[j]);
          U += ((double)nst[i] - sc64[i]) * row;
        }
        for (int i = 0; i < n; ++i) {
          int v = nst[i];
          if (v > 127) { v = 127; flags |= kFlagOverflow; }
          a.out_n[p * n + i] = (int8_t)v;
        }
        if (a.out_U) a.out_U[p] = 0.5 * U;
      }
      if (a.out_flags) a.out_flags[p] = (uint8_t)flags;
      atomicMax(&a.cnt->shortlist_max, (unsigned long long)nb);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host-side dispatch
// ---------------------------------------------------------------------------
int prep_blocks(const GsLaunch& a) {
  const long long tpb = kPrepThreads / a.prep_team;
  return (int)((a.sc.P + tpb - 1) / tpb);
}
int search_blocks(const GsLaunch& a) {
  const int teams = kSearchThreads / a.cfg.T;
  return (int)((a.sc.P + teams - 1) / teams);
}

template <int L1, int L2, bool CLOSED>
static cudaError_t run(const GsLaunch& a, cudaStream_t st) {
  if (a.ev) cudaEventRecord(a.ev[0], st);
  cudaMemsetAsync(a.cnt, 0, sizeof(Counters), st);
  k_prep<CLOSED><<<prep_blocks(a), kPrepThreads, 0, st>>>(a);
  if (a.ev) cudaEventRecord(a.ev[1], st);
  k_search<L1, L2, CLOSED><<<search_blocks(a), kSearchThreads, 0, st>>>(a);
  if (a.ev) cudaEventRecord(a.ev[2], st);
  k_resolve<L1, L2, CLOSED><<<a.num_sms, kResolveThreads, 0, st>>>(a);
  k_recheck<CLOSED><<<a.num_sms, kRecheckThreads, 0, st>>>(a);
  if (a.ev) cudaEventRecord(a.ev[3], st);
  return cudaGetLastError();
}

cudaError_t launch_prep(const GsLaunch& a, cudaStream_t st) {
  cudaMemsetAsync(a.cnt, 0, sizeof(Counters), st);
  if (a.sc.P == 0) return cudaGetLastError();
  if (a.mt.closed)
    k_prep<true><<<prep_blocks(a), kPrepThreads, 0, st>>>(a);
  else
    k_prep<false><<<prep_blocks(a), kPrepThreads, 0, st>>>(a);
  return cudaGetLastError();
}

bool search_cfg_supported(const SearchCfg& c) {
  const bool split = (c.L1 == 2 && c.L2 == 0) || (c.L1 == 4 && c.L2 == 0) ||
                     (c.L1 == 4 && c.L2 == 3) || (c.L1 == 5 && c.L2 == 4);
  const bool team = c.T >= 1 && c.T <= 32 && (c.T & (c.T - 1)) == 0;
  return split && team;
}

cudaError_t launch_ground_state(const GsLaunch& a, cudaStream_t st) {
  const bool cl = a.mt.closed != 0;
  const int key = a.cfg.L1 * 10 + a.cfg.L2;
  switch (key) {
    case 20: return cl ? run<2, 0, true>(a, st) : run<2, 0, false>(a, st);
    case 40: return cl ? run<4, 0, true>(a, st) : run<4, 0, false>(a, st);
    case 43: return cl ? run<4, 3, true>(a, st) : run<4, 3, false>(a, st);
    case 54: return cl ? run<5, 4, true>(a, st) : run<5, 4, false>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qa
