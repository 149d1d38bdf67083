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
constexpr int kRecheckL1 = 4, kRecheckL2 = 3;  // 2^9 outer states at k = 16
constexpr unsigned kBcap = 1024;

// number of k-subsets of size w (k <= 16)
__device__ __forceinline__ unsigned long long binom(int k, int w) {
  if (w < 0 || w > k) return 0ull;
  unsigned long long r = 1ull;
  for (int i = 1; i <= w; ++i) r = r * (unsigned long long)(k - w + i) / (unsigned long long)i;
  return r;
}

// Load M (double-float split), Cdd (FP32), Cdd 1 and 1^T Cdd 1 into smem.
__device__ inline void stage_model(const ModelData* md, int n, float* sMhi,
                                   float* sMlo, float* sCdd, float* sv,
                                   float* s_s) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    if (sMhi) {
      const df m = df_from_double(md->M[e]);
      sMhi[i * kLdM + j] = m.hi;
      if (sMlo) sMlo[i * kLdM + j] = m.lo;
    }
    if (sCdd) sCdd[i * kLdM + j] = __double2float_rn(md->Cdd[e]);
  }
  if (sv) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double r = 0.0;
      for (int j = 0; j < n; ++j) r += md->Cdd[i * n + j];
      sv[i] = __double2float_rn(r);
    }
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int e = 0; e < n * n; ++e) s += md->Cdd[e];
      *s_s = __double2float_rn(s);
    }
  }
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
  __shared__ float sMhi[kMaxDot * kLdM], sMlo[kMaxDot * kLdM],
      sCdd[kMaxDot * kLdM];
  __shared__ float sv[kMaxDot];
  __shared__ float s_s;
  __shared__ df sc0[kMaxDot], sdu[kMaxDot], sdw[kMaxDot], svs[kMaxDot];
  __shared__ float sx[kPrepThreads];
  __shared__ int sst[kPrepThreads];
  const int n = a.n;
  stage_model(a.md, n, sMhi, sMlo, sCdd, sv, &s_s);
  if (a.sc.kind == 0) raster_setup(a.md, n, a.ng, a.sc, a.mt.carrier, sc0, sdu, sdw);
  for (int i = threadIdx.x; i < n; i += blockDim.x) svs[i] = df_from_double(a.md->vs[i]);
  __syncthreads();
  // decision margin of an FP32 QP minimum: 8 cond(Cdd) (n + 1) u32 per unit
  // of (1 + max|c| + N_hat)
  const float bx_qp_scale =
      a.bx_qp_scale > 0.f ? a.bx_qp_scale
                          : 8.f * (float)a.md->cond * (float)(n + 1) * 5.9604645e-8f;
  const bool model_bad = a.md->status != 0;

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

  if (!active) return;  // whole teams retire together

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
    const df cs = tsum_df(c);
    const df lam = df_sub({(float)nhat, 0.f}, cs);  // N_hat <= 2^24
    if (live) x = df_add(c, df_mul(lam, svs[lt]));
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
        const int st = qp_active_set<float>(n, sCdd, kLdM, cf, CLOSED, (float)nhat, sv,
                                            s_s, A, 0.25f * bx_qp_scale * scale,
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

  PixRec* rec = a.recs + p;
  if (live) {
    rec->h[lt] = h;
    rec->chi[lt] = c.hi;
    rec->clo[lt] = c.lo;
    rec->base[lt] = (short)base;
  }
  unsigned long long my_cand = 0, my_qp = 0, my_doubled = 0;
  if (lt == 0) {
    rec->mask = (unsigned short)mask;
    rec->k = (unsigned char)k;
    rec->w = (signed char)(CLOSED ? w : -1);
    rec->flags = (unsigned char)flags;
    rec->bound = near_tie_bound(S, k, a.cfg.L2);
    my_cand = CLOSED ? binom(k, w) : (1ull << k);
    my_qp = (flags & kFlagQP) ? 1 : 0;
    my_doubled = (flags & kFlagDoubled) ? 1 : 0;
    if (my_cand) atomicAdd(&a.cnt->candidates, my_cand);
    if (my_qp) atomicAdd(&a.cnt->qp, my_qp);
    if (my_doubled) atomicAdd(&a.cnt->doubled, my_doubled);
  }
}

// ---------------------------------------------------------------------------
// (a5)-(a6), (a8): candidate search, top-two selection, outputs
// ---------------------------------------------------------------------------
template <int L1, int L2, bool CLOSED>
__global__ void __launch_bounds__(kSearchThreads) k_search(GsLaunch a) {
  __shared__ float sM[kMaxDot * kLdM], sMlo[kMaxDot * kLdM];
  __shared__ int sdot[kSearchThreads][kMaxDot];
  __shared__ float sh[kSearchThreads][kMaxDot];
  const int n = a.n;
  stage_model(a.md, n, sM, sMlo, nullptr, nullptr, nullptr);
  __syncthreads();

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
  unsigned long long my_nt = 0, my_bd = 0, my_fl = 0, my_ov = 0;
  if (active) {
    flags |= rec->flags;
    if (!(m2 - m1 > rec->bound)) flags |= kFlagNearTie;
    if (lt == 0) {
      if (a.out_U) a.out_U[p] = 0.5 * df_to_double(u);
      if (flags & (kFlagNearTie | kFlagBoundary | kFlagQPCap)) {
        const unsigned at = atomicAdd(&a.cnt->n_flag, 1u);
        a.flag_list[at] = (int)p;
        my_fl = 1;
        my_nt = (flags & kFlagNearTie) ? 1 : 0;
        my_bd = (flags & (kFlagBoundary | kFlagQPCap)) ? 1 : 0;
      }
      my_ov = (flags & kFlagOverflow) ? 1 : 0;
      if (a.out_flags) a.out_flags[p] = (uint8_t)flags;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    ev += __shfl_xor_sync(kFull, ev, off);
    my_nt += __shfl_xor_sync(kFull, my_nt, off);
    my_bd += __shfl_xor_sync(kFull, my_bd, off);
    my_fl += __shfl_xor_sync(kFull, my_fl, off);
    my_ov += __shfl_xor_sync(kFull, my_ov, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (ev) atomicAdd(&a.cnt->evaluated, ev);
    if (my_fl) {
      atomicAdd(&a.cnt->flagged, my_fl);
      atomicAdd(&a.cnt->near_tie, my_nt);
      atomicAdd(&a.cnt->boundary, my_bd);
    }
    if (my_ov) atomicAdd(&a.cnt->overflow, my_ov);
  }
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
  for (int e = threadIdx.x; e < n * n; e += blockDim.x)
    sM[(e / n) * kLdM + (e % n)] = __double2float_rn(a.md->M[e]);
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
template <int L1, int L2, bool CLOSED>
static cudaError_t run(const GsLaunch& a, cudaStream_t st) {
  const long long P = a.sc.P;
  const long long tpb = kPrepThreads / a.prep_team;
  const unsigned gp = (unsigned)((P + tpb - 1) / tpb);
  if (a.ev) cudaEventRecord(a.ev[0], st);
  k_prep<CLOSED><<<gp, kPrepThreads, 0, st>>>(a);
  if (a.ev) cudaEventRecord(a.ev[1], st);
  const int teams = kSearchThreads / a.cfg.T;
  const unsigned gs = (unsigned)((P + teams - 1) / teams);
  k_search<L1, L2, CLOSED><<<gs, kSearchThreads, 0, st>>>(a);
  if (a.ev) cudaEventRecord(a.ev[2], st);
  k_recheck<CLOSED><<<2 * a.num_sms, kRecheckThreads, 0, st>>>(a);
  if (a.ev) cudaEventRecord(a.ev[3], st);
  return cudaGetLastError();
}

cudaError_t launch_prep(const GsLaunch& a, cudaStream_t st) {
  const long long tpb = kPrepThreads / a.prep_team;
  const unsigned gp = (unsigned)((a.sc.P + tpb - 1) / tpb);
  if (gp == 0) return cudaSuccess;
  if (a.mt.closed)
    k_prep<true><<<gp, kPrepThreads, 0, st>>>(a);
  else
    k_prep<false><<<gp, kPrepThreads, 0, st>>>(a);
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
