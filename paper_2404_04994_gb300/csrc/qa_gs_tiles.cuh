// qa_gs_tiles.cuh -- the ground-state stages as per-tile device functions,
// shared by the single-array kernels (qa_kernels_gs.cu) and the persistent
// batched kernels (qa_batch.cu).  A tile is one block's worth of pixels of one
// array; the stage functions take the array's descriptor and the tile's first
// pixel-team index, so both launch shapes run exactly the same code.
#pragma once

#include "qa_launch.h"
#include "qa_prep.cuh"
#include "qa_search.cuh"

namespace qa {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPrepThreads = 128;
constexpr int kRecheckThreads = 512;  // the tail kernel's block: resolve and recheck alike
constexpr int kResolveThreads = 512;  // the walk's 512 outer states at k = 16, one per thread
constexpr int kCheckL1 = 4, kCheckL2 = 3;  // resolve/recheck split: 2^9 outer states at k = 16
constexpr unsigned kBcap = 1024;

// One charge of the output map: int8 (saturating at 127) or int16 (at
// 32767) by the array's output width; saturation sets kFlagOverflow.
__device__ __forceinline__ void store_charge(const ArrayDesc& a, long long idx, int v,
                                             unsigned& flags) {
  if (a.out_n16) {
    if (v > 32767) { v = 32767; flags |= kFlagOverflow; }
    a.out_n16[idx] = (int16_t)v;
  } else {
    if (v > 127) { v = 127; flags |= kFlagOverflow; }
    a.out_n[idx] = (int8_t)v;
  }
}

// number of k-subsets of size w (k <= 16)
__device__ __forceinline__ unsigned long long binom(int k, int w) {
  if (w < 0 || w > k) return 0ull;
  unsigned long long r = 1ull;
  for (int i = 1; i <= w; ++i) r = r * (unsigned long long)(k - w + i) / (unsigned long long)i;
  return r;
}

// The descriptor of a list entry's array.
__device__ __forceinline__ const ArrayDesc& desc_of(const GsLaunch& L, int array) {
  return L.table ? L.table[array] : L.one;
}

// ---------------------------------------------------------------------------
// (a0) raster constants of a block: c(ix, iy) = c0 + ix du + iy dw with
// c0 = s Cgd (V0 + x0 u + y0 w), du = s Cgd u dx, dw = s Cgd w dy, formed in
// double-float FP32 from FP64 inputs (one FP64 rounding per input, no FP64
// dependency chains: FP64 issues at a small fraction of the FP32 rate here).
// Used when the host could not precompute them (model updated on the GPU).
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
// prep stage: shared state of a block and the per-array set-up
// ---------------------------------------------------------------------------
// Point lists with at most this many gates take c from a staged s Cgd and
// voltages converted once per pixel by the team (one gate per lane).
constexpr int kPointGates = 16;
struct PrepShared {
  ModelConsts cs;
  df sV[kMaxGate], sU[kMaxGate], sW[kMaxGate];
  df sc0[kMaxDot], sdu[kMaxDot], sdw[kMaxDot];
  df sG[kMaxDot][kPointGates];     // point lists of <= kPointGates gates: s Cgd
  float qK[kPrepThreads][kQPRow];  // team QP: KKT rows, active lists, unknowns, c
  int qa[kPrepThreads];
  float qz[kPrepThreads];
  float qzl[kPrepThreads];
  float qx[kPrepThreads];
  float qc[kPrepThreads];
  unsigned long long red64[kPrepThreads / 32];
  unsigned red32[kPrepThreads / 32];
  float th0;  // the threshold test's half-width t / 2 in FP32
  int tlt1;   // t < 1
};

// Stage an array's FP32 model constants and raster constants (all threads);
// one thread converts the FP64 threshold for the whole block.
__device__ inline void prep_stage_array(const ArrayDesc& a, PrepShared& sh) {
  stage_consts(&a.md->k, &sh.cs);
  if (threadIdx.x == 0) {
    sh.th0 = __double2float_rn(0.5 * a.mt.t);
    sh.tlt1 = a.mt.t < 1.0 ? 1 : 0;
  }
  if (a.sc.kind == 1 && a.ng <= kPointGates && a.prep_team >= a.ng) {
    for (int e = threadIdx.x; e < a.n * a.ng; e += blockDim.x) {
      const int i = e / a.ng, g = e - i * a.ng;
      sh.sG[i][g] = df_from_double(a.mt.carrier * a.md->Cgd[i * a.ng + g]);
    }
  }
  if (a.sc.kind == 0) {
    if (a.rk.valid) {
      if (threadIdx.x < kMaxDot) {
        sh.sc0[threadIdx.x] = a.rk.c0[threadIdx.x];
        sh.sdu[threadIdx.x] = a.rk.du[threadIdx.x];
        sh.sdw[threadIdx.x] = a.rk.dw[threadIdx.x];
      }
    } else {
      raster_consts(a.md, a.n, a.ng, a.sc, a.mt.carrier, sh.sV, sh.sU, sh.sW, sh.sc0,
                    sh.sdu, sh.sdw);
    }
  }
  __syncthreads();
}

// c of a point-list pixel by its team (out of line: the raster kernels carry
// only the call): lane g converts V_g to double-float once for the team,
// through the team's scratch rows, and each live lane sums its dot's row of
// the staged s Cgd, the same operations in the same order as point_c.
// Every lane of tmask must call; ng <= the team's lanes.
static __device__ __noinline__ df point_c_team(const double* Vp, int ng, bool active, bool live,
                                               int lt, unsigned tmask,
                                               const df (*sG)[kPointGates], float* qx,
                                               float* qz) {
  const int tq = (int)threadIdx.x - lt;
  df vg = {0.f, 0.f};
  if (active && lt < ng) vg = df_from_double(Vp[lt]);
  qx[threadIdx.x] = vg.hi;
  qz[threadIdx.x] = vg.lo;
  __syncwarp(tmask);
  df acc = {0.f, 0.f};
  if (live)
    for (int g = 0; g < ng; ++g) acc = df_add(acc, df_mul(sG[lt][g], df{qx[tq + g], qz[tq + g]}));
  __syncwarp(tmask);
  return acc;
}

// Per-block totals of the prep stage (thread 0's copy is the block's).
struct PrepAcc {
  unsigned long long candidates = 0;
  unsigned qp = 0, doubled = 0;
};

// ---------------------------------------------------------------------------
// (a1)-(a4) for one tile: induced charge, continuous minimum, candidate set,
// h = M (base - c).  A team of TP lanes (a power of two >= N, at most 16)
// prepares one pixel, lane i owning dot i; team-wide sums, ballots and gathers
// use shuffles restricted to the team's lanes, so teams of one warp may
// diverge.  Pixels team_base + threadIdx.x / TP below p_end are processed.
// All threads of the block must call (block reductions at the end).
// ---------------------------------------------------------------------------
template <bool CLOSED>
__device__ inline void prep_tile(const ArrayDesc& a, PrepShared& sh, long long team_base,
                                 long long p_end, PrepAcc& tot) {
  const int n = a.n;
  const float* sMhi = sh.cs.Mhi;
  const float* sMlo = sh.cs.Mlo;
  const float bx_qp_scale = a.bx_qp_scale > 0.f ? a.bx_qp_scale : sh.cs.bx_qp_scale;
  const bool model_bad = sh.cs.model_bad != 0;

  const int TP = a.prep_team;
  const int lt = threadIdx.x & (TP - 1);
  const int lane = threadIdx.x & 31;
  const int tbase = lane & ~(TP - 1);                   // team's first lane
  const unsigned tmask = (TP == 32 ? 0xffffffffu : ((1u << TP) - 1u)) << tbase;
  const long long p = team_base + threadIdx.x / TP;
  const bool active = p < p_end;
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

  // (a1) c_i; a point list of at most one gate per lane: lane g converts the
  // pixel's V_g to double-float once for the team (the team's scratch rows),
  // then each lane sums its dot's row of the staged s Cgd -- the same
  // operations in the same order as point_c, without the per-lane FP64
  // conversions
  df c = {0.f, 0.f};
  if (a.sc.kind == 1 && a.ng <= kPointGates && TP >= a.ng) {
    c = point_c_team(a.sc.V + (active ? p : 0) * a.ng, a.ng, active, live, lt, tmask, sh.sG,
                     sh.qx, sh.qz);
  } else if (live) {
    if (a.sc.kind == 0) {
      int ix, iy;
      if (a.sc.P <= 0xffffffffLL) {  // 32-bit division when the raster allows it
        const unsigned pu = (unsigned)p, W = (unsigned)a.sc.W;
        iy = (int)(pu / W);
        ix = (int)(pu - (unsigned)iy * W);
      } else {
        ix = (int)(p % a.sc.W);
        iy = (int)(p / a.sc.W);
      }
      c = raster_c(sh.sc0[lt], sh.sdu[lt], sh.sdw[lt], ix, iy);
    } else {
      c = point_c(&a.md->Cgd[lt * a.ng], &a.sc.V[p * a.ng], a.ng, a.mt.carrier);
    }
  }
  // (a2) analytic continuous minimum (Appendix C / D)
  df x = c;
  if (CLOSED) {
    const df csum = tsum_df(c);
    const df lam = df_sub({(float)nhat, 0.f}, csum);  // N_hat <= 2^24
    if (live) x = df_add(c, df_mul(lam, sh.cs.vs[lt]));
  }
  const unsigned A =
      tballot(live && (x.hi < 0.f || (x.hi == 0.f && x.lo < 0.f)));
  unsigned flags = 0u;
  unsigned qp_set = 0u;
  float bx = a.bx_analytic;
  // (a3) QP where the analytic minimum is infeasible, by the pixel's team
  const bool need = A != 0u && !(CLOSED && nhat == 0);  // team-uniform
  const int tb = threadIdx.x - lt;
  float scale = 1.f;
  if (A) {
    flags |= kFlagQP;
    const float cmax = tmax_f(live ? fabsf(c.hi + c.lo) : 0.f);
    if (need) {
      scale = 1.f + cmax + (float)nhat;
      bx = fmaxf(bx, bx_qp_scale * scale);
    } else {
      x = {0.f, 0.f};
    }
  }
  float xf = 0.f;
  unsigned Af = 0u;
  int st = 0;
  // open array with one negative c_a (every QP pixel of the 16-dot diagram):
  // the active set {a} solved in place -- z_a = -c_a / Cdd_aa through the
  // same reciprocal square root, x_i = c_i + Cdd_ia z_a -- with the same
  // operations, results and shared state (factor, active list, multiplier)
  // as the team QP's first iteration; it stands when no other x_i is below
  // -tol, else the team QP runs from {a}
  bool solved = false;
  if (!CLOSED && need && __popc(A) == 1) {
    const int ad = __ffs(A) - 1;
    const float cl = live ? c.hi + c.lo : 0.f;
    const float ca = __shfl_sync(tmask, cl, ad, TP);
    const float caa = sh.cs.Cdd[ad * kLdM + ad];
    const float r = caa > 0.f ? rsqrtf(caa) : 0.f;
    const float zf = (-ca * r) * r;
    float xi = 0.f;
    if (live && lt != ad) xi = cl + sh.cs.Cdd[lt * kLdM + ad] * zf;
    const float tolq = 0.25f * bx_qp_scale * scale;
    solved = r > 0.f && tballot(live && lt != ad && xi < -tolq) == 0u;
    if (solved) {
      if (lt == 0) {
        sh.qa[tb] = ad;
        sh.qz[tb] = zf;
        sh.qK[tb][0] = caa * r;
        sh.qK[tb][kQPRow - 1] = r;
      }
      xf = (live && lt != ad) ? (xi > 0.f ? xi : 0.f) : 0.f;
      Af = A;
      __syncwarp(tmask);
    }
  }
  if (need && !solved)
    st = qp_team<float, CLOSED>(n, lt, TP, tmask, tb, sh.cs.Cdd, kLdM, sh.cs.sv, sh.cs.s_s,
                                live ? c.hi + c.lo : 0.f, (float)nhat, A,
                                0.25f * bx_qp_scale * scale, 4 * n + 4, sh.qK, sh.qa, sh.qz,
                                sh.qc, xf, Af);
  if (need) {
    // the FP32 solution stands when its active set is certain at FP32
    // precision (every free x_i and every multiplier more than twice the
    // FP32 margin above zero) and no floor or threshold decision lies
    // within that margin; otherwise one double-float refinement follows
    bool sure = st == 0;
    if (sure && live) {
      if ((Af >> lt) & 1u) {
        sure = sh.qz[tb + __popc(Af & ((1u << lt) - 1u))] > 2.f * bx;
      } else {
        const float fr = xf - floorf(xf);
        sure = xf > 2.f * bx && !(xf >= 0.5f - bx && fminf(fr, 1.f - fr) < bx) &&
               !(sh.tlt1 && fabsf(fabsf(fr - 0.5f) - sh.th0) < bx);
      }
    }
    sure = tballot(!sure) == 0u;
    if (st != 0) {
      flags |= kFlagQPCap;
      if (live) x = {xf, 0.f};
    } else if (sure) {
      if (live) x = {xf, 0.f};
      qp_set = Af;
    } else {
      // one double-float refinement: the margin shrinks to the square of
      // the FP32 one; a multiplier or free x_i below -margin at that
      // precision leaves the active set (and x) to the FP64 recheck
      const float bx2 = fmaxf(a.bx_analytic, sh.cs.bx_qp_scale2 * scale);
      df xr;
      unsigned flip = 0u;
      int bad = qp_team_refine<CLOSED>(n, lt, TP, tmask, tb, sh.cs.Cdd, sh.cs.CddLo, sh.cs.sv2,
                                       live ? c : df{0.f, 0.f}, (float)nhat, Af, 0.25f * bx2,
                                       sh.qK, sh.qa, sh.qz, sh.qzl, sh.qx, xr, flip);
      // a sign violation below FP32 resolution (a nearly degenerate vertex:
      // a multiplier or free x_i within rounding of zero): one more round
      // with those constraints toggled -- the FP32 factor and solve of that
      // active set, and its double-float refinement -- before the FP64
      // recheck is left to settle the pixel
      const unsigned A2 = (Af ^ flip) & ((n < 32 ? (1u << n) : 0u) - 1u);
      if (bad && flip && A2 != Af && !(CLOSED && __popc(A2) == n)) {
        float xf2 = 0.f;
        unsigned Af2 = 0u;
        const int st2 = qp_team<float, CLOSED>(n, lt, TP, tmask, tb, sh.cs.Cdd, kLdM, sh.cs.sv,
                                               sh.cs.s_s, live ? c.hi + c.lo : 0.f, (float)nhat,
                                               A2, 0.25f * bx_qp_scale * scale, 1, sh.qK, sh.qa,
                                               sh.qz, sh.qc, xf2, Af2);
        if (st2 == 0) {
          Af = Af2;
          bad = qp_team_refine<CLOSED>(n, lt, TP, tmask, tb, sh.cs.Cdd, sh.cs.CddLo, sh.cs.sv2,
                                       live ? c : df{0.f, 0.f}, (float)nhat, Af, 0.25f * bx2,
                                       sh.qK, sh.qa, sh.qz, sh.qzl, sh.qx, xr, flip);
        }
      }
      if (live) x = xr;
      if (bad) flags |= kFlagBoundary;
      else bx = bx2;
      // closed with every dot but one active: the sum constraint makes the
      // relaxed minimum the vertex N_hat e_j exactly, so once every
      // multiplier is certainly positive no rounding error is left in x
      // and the floor decisions need no margin
      if (CLOSED && !bad && __popc(Af) == n - 1) {
        const bool zpos = lt >= n - 1 || sh.qz[tb + lt] + sh.qzl[tb + lt] > 0.25f * bx2;
        if (tballot(!zpos) == 0u) {
          if (live) x = ((Af >> lt) & 1u) ? df{0.f, 0.f} : df{(float)nhat, 0.f};
          bx = 0.f;
        }
      }
      qp_set = Af;
    }
    __syncwarp(tmask);
  }

  // (a4) candidate set; the closed doubling loop is team-uniform (its first
  // pass takes t / 2 and t < 1 from the block's staging, later ones double t
  // in FP64)
  double tt = a.mt.t;
  float th = sh.th0;
  bool tlt1 = sh.tlt1 != 0;
  unsigned mask = 0u;
  int w = -1, base = 0;
  bool amb = false;
  for (int iter = 0; iter < 40; ++iter) {
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
            (tlt1 && fabsf(fabsf(fr - 0.5f) - th) < bx);
    }
    if (tballot(bnd)) flags |= kFlagBoundary;
    mask = tballot(live && amb);
    if (!CLOSED) break;
    const int sum = tsum_i(live ? base : 0);
    w = nhat - sum;
    if (w >= 0 && w <= __popc(mask)) break;
    if (!tlt1) {  // t = 1 and still infeasible: impossible in exact arithmetic, settle in FP64
      flags |= kFlagBoundary;
      w = w < 0 ? 0 : __popc(mask);
      break;
    }
    tt = (tt <= 0.0) ? 1.0 : fmin(2.0 * tt, 1.0);
    th = __double2float_rn(0.5 * tt);
    tlt1 = tt < 1.0;
    flags |= kFlagDoubled;
  }
  if (model_bad) flags |= kFlagUnresolved;

  // h_i = (M (base - c))_i, r = base - c in double-float staged in the
  // team's rows of qx / qz (free after the QP); the products' high parts are
  // summed error-free and their low parts and rounding errors in plain FP32
  // (error O(u^2) of sum |M_ij r_j|, far below the final rounding of h to
  // FP32).  Four columns per step with their loads issued together and two
  // independent sums (even and odd columns), joined error-free at the end.
  const df r = df_sub({(float)base, 0.f}, c);
  const int tb0 = threadIdx.x - lt;
  __syncwarp(tmask);
  sh.qx[threadIdx.x] = r.hi;
  sh.qz[threadIdx.x] = r.lo;
  __syncwarp(tmask);
  const float* Mrow = sMhi + lt * kLdM;
  const float* Mrowl = sMlo + lt * kLdM;
  float h = 0.f;
  if (live) {
    float shi[2] = {0.f, 0.f}, slo[2] = {0.f, 0.f};
    for (int j0 = 0; j0 < n; j0 += 4) {
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int j = j0 + jj;
        const bool on = j < n;
        const int jc = on ? j : 0;
        const float mh = on ? Mrow[jc] : 0.f, ml = on ? Mrowl[jc] : 0.f;
        const float xh = sh.qx[tb0 + jc], xl = sh.qz[tb0 + jc];
        const df pr = two_prod(mh, xh);
        const float small = __fmaf_rn(mh, xl, __fmaf_rn(ml, xh, pr.lo));
        const df sm = two_sum(shi[jj & 1], pr.hi);
        shi[jj & 1] = sm.hi;
        slo[jj & 1] = __fadd_rn(slo[jj & 1], __fadd_rn(sm.lo, small));
      }
    }
    const df st = two_sum(shi[0], shi[1]);
    h = st.hi + (st.lo + (slo[0] + slo[1]));
  }
  // S_i = |h_i| + M_ii / 2 + sum over the ambiguous j < i of |M_ij|: the
  // row's precomputed prefix when every j < i is ambiguous, else four columns
  // per step with two independent sums
  float Si = 0.f;
  const unsigned below = mask & ((1u << lt) - 1u);
  if (live && amb && below == (1u << lt) - 1u) {
    Si = fabsf(h) + sh.cs.absl[lt];
  } else if (live && amb) {
    float sp[2] = {fabsf(h) + 0.5f * Mrow[lt], 0.f};
    for (int j0 = 0; j0 < n; j0 += 4) {
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int j = j0 + jj;
        sp[jj & 1] += ((below >> j) & 1u) ? fabsf(Mrow[j < n ? j : 0]) : 0.f;
      }
    }
    Si = sp[0] + sp[1];
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
    rec->qpA = (unsigned short)qp_set;
    // the pruned search walks a shallower middle level than the resolve's
    // re-walk (kCheckL2), which shortlists by this bound, and forms each
    // rest state from up to kBnbItBits + 2 more table sums
    rec->bound = bnb_search(a.cfg.L1, a.cfg.L2)
                     ? near_tie_bound(S, k, max(a.cfg.L2, kCheckL2), kBnbItBits + 2)
                     : near_tie_bound(S, k, a.cfg.L2);
    my_cand = CLOSED ? binom(k, w) : (1ull << k);
    my_qp = (flags & kFlagQP) ? 1u : 0u;
    my_doubled = (flags & kFlagDoubled) ? 1u : 0u;
  }
  __syncwarp();
  // one block sum of the three counts packed in 64 bits: candidates in the
  // low 32 (a block prepares 128 / TP pixels of at most 2^N candidates with
  // TP >= N, below 2^20 in all), QP and doubled pixels (<= 128) above
  const unsigned long long packed = block_sum(
      my_cand | ((unsigned long long)my_qp << 32) | ((unsigned long long)my_doubled << 48),
      sh.red64);
  if (threadIdx.x == 0) {
    tot.candidates += packed & 0xffffffffull;
    tot.qp += (unsigned)((packed >> 32) & 0xffffu);
    tot.doubled += (unsigned)(packed >> 48);
  }
}

// ---------------------------------------------------------------------------
// search stage: shared state of a block
// ---------------------------------------------------------------------------
// Three layouts share the space: teams narrower than kTeamFinishMin keep a
// slot table per thread; block-level teams one per team with their walk
// tables; the pruned search (teams of kBnbMinT+ lanes) its bound tables.
constexpr int kTeamsTF = kSearchThreads / kTeamFinishMin;
constexpr int kTeamsBnb = kSearchThreads / kBnbMinT;
struct SearchShared {
  ModelConsts cs;
  union {
    struct {
      int sdot[kSearchThreads][kMaxDot];
      float sh[kSearchThreads][kMaxDot];
    } lane;
    struct {
      int sdot[kTeamsTF][kMaxDot];
      float sh[kTeamsTF][kMaxDot];
      __align__(16) float colt[kTeamsTF][4 * kColStride];
      __align__(16) float itab[kTeamsTF][(1 << kItMax) * kItStride];
      __align__(16) float cslot[kSearchThreads][kItMax];
    } team;
    struct {
      int sdot[kTeamsBnb][kMaxDot];
      float sh[kTeamsBnb][kMaxDot];
      int slot_of[kTeamsBnb][kMaxDot];  // slot of each ambiguous dot
      float pm[kTeamsBnb][kMaxDot * kLdM];
      float vv[kTeamsBnb][kMaxDot];
      __align__(16) float itab[kTeamsBnb][(1 << kBnbItBits) * kBnbStride];
      __align__(16) float ltab[kSearchThreads][kBnbLane];
      __half lb[kTeamsBnb][kBnbStates];
      unsigned short rbuf[kTeamsBnb][kBnbBuf];
      float rlb[kTeamsBnb][kBnbBuf];
      __align__(16) float ptab[kTeamsBnb][1 << kBnbL1];
    } bnb;
  } u;
  unsigned long long red64[kSearchThreads / 32];
  unsigned red32[kSearchThreads / 32];
};

struct SearchAcc {
  unsigned long long evaluated = 0;
  unsigned near_tie = 0, boundary = 0, overflow = 0;
};

// A block that prepares and then searches its own tile holds the two stages'
// scratch in one place; the model constants, first in both, are staged once.
union GsShared {
  PrepShared p;
  SearchShared s;
};
static_assert(offsetof(PrepShared, cs) == 0 && offsetof(SearchShared, cs) == 0,
              "the model constants open both stages' shared state");
static_assert(kPrepThreads == kSearchThreads, "one block size for both stages");

// ---------------------------------------------------------------------------
// (a5)-(a6), (a8) for one tile: candidate search, top-two selection, outputs.
// A team of T lanes (the array's cfg.T) searches one pixel; pixels
// team_base + threadIdx.x / T below p_end.  Pixels whose candidate set is in
// doubt go on the FP64 recheck list, near ties on the resolve list.  All
// threads of the block must call.
// ---------------------------------------------------------------------------
template <int L1, int L2, bool CLOSED, bool TF>
__device__ inline void search_tile(const GsLaunch& L, const ArrayDesc& a, SearchShared& sh,
                                   int array, long long team_base, long long p_end,
                                   SearchAcc& acc) {
  const int n = a.n;
  const float* sM = sh.cs.Mhi;
  const float* sMlo = sh.cs.Mlo;

  const int T = a.cfg.T;
  const int team = threadIdx.x / T, lt = threadIdx.x % T;
  const long long p = team_base + team;
  const bool active = p < p_end;
  const PixRec* rec = a.recs + (active ? p : 0);
  const unsigned mask = active ? rec->mask : 0u;
  const int k = __popc(mask);
  // BNB: the pruned search (5 + 2 split, teams of kBnbMinT+ lanes, which
  // the host guarantees for this split)
  constexpr bool BNB = TF && bnb_search(L1, L2);
  int* sdot = BNB ? sh.u.bnb.sdot[team] : TF ? sh.u.team.sdot[team] : sh.u.lane.sdot[team];
  float* sht = BNB ? sh.u.bnb.sh[team] : TF ? sh.u.team.sh[team] : sh.u.lane.sh[team];
  int* slot_of = BNB ? sh.u.bnb.slot_of[team] : nullptr;
  if (BNB) {
    // slot s = the ambiguous dot of rank s by |h_i + M_ii / 2|, ascending
    // (ties by dot index): the least certain dots are walked, the most
    // certain ones are the outer slots the bounds prune
    if (active)
      for (int i = lt; i < n; i += T)
        sht[i] = ((mask >> i) & 1u) ? fabsf(rec->h[i] + 0.5f * sM[i * kLdM + i]) : 0.f;
    __syncwarp();
    int rank = -1;
    if (active && lt < n && ((mask >> lt) & 1u)) {
      const float key = sht[lt];
      rank = 0;
      for (int j = 0; j < n; ++j) {
        const float kj = sht[j];
        rank += (((mask >> j) & 1u) && (kj < key || (kj == key && j < lt))) ? 1 : 0;
      }
    }
    __syncwarp();
    if (rank >= 0) {
      sdot[rank] = lt;
      sht[rank] = rec->h[lt];
      slot_of[lt] = rank;
    }
  } else if (active) {
    // slot table of the pixel: slot s = the s-th ambiguous dot (lanes in parallel)
    for (int i = lt; i < n; i += T)
      if ((mask >> i) & 1u) {
        const int s = __popc(mask & ((1u << i) - 1u));
        sdot[s] = i;
        sht[s] = rec->h[i];
      }
  }
  __syncwarp();
  float m1 = kInf, m2 = kInf;
  unsigned b1 = 0u;
  unsigned long long ev = 0;
  const SlotView sv{sdot, sht, active ? k : 0, active ? (int)rec->w : -1};
  // TF (teams of 8 or more lanes): search at block level and finish the
  // winning block together; smaller teams finish each lane's best block in
  // the lane.
  float* colt = (TF && !BNB) ? sh.u.team.colt[team] : nullptr;
  float* itab = (TF && !BNB) ? sh.u.team.itab[team] : nullptr;
  if (TF && !BNB) {
    static_assert(L2 <= 4 && L1 + L2 <= kColStride, "column table layout");
    if (active) {
      col_build<L1, L2>(sM, sv, lt, T, colt);
      if (L1 + L2 >= 9) iter_build<L1, L2>(sM, sv, lt, T, itab);
    }
    __syncwarp();
  }
  if (active) {
    if constexpr (BNB) {
      const unsigned wl = threadIdx.x & 31u;
      const unsigned tmask =
          T >= 32 ? kFull : (((1u << T) - 1u) << (wl & ~(unsigned)(T - 1)));
      search_bnb<CLOSED>(sM, sv, lt, T, tmask, rec->bound, sh.cs.qneg, sh.u.bnb.pm[team],
                 sh.u.bnb.vv[team], sh.u.bnb.itab[team],
                 sh.u.bnb.ltab[team * T], sh.u.bnb.lb[team], sh.u.bnb.rbuf[team],
                 sh.u.bnb.rlb[team], sh.u.bnb.ptab[team], m1, b1, m2, ev);
    } else {
      search_lane<L1, L2, CLOSED, false, TF>(sM, sv, lt, T, 0.f, nullptr, nullptr, 0u, m1, b1,
                                             m2, ev, colt, itab,
                                             TF ? sh.u.team.cslot[threadIdx.x] : nullptr);
    }
  }
  // best (block or candidate) with its id, and the second-best minimum
  for (int off = 1; off < T; off <<= 1) {
    const float om1 = __shfl_xor_sync(kFull, m1, off);
    const unsigned ob1 = __shfl_xor_sync(kFull, b1, off);
    const float om2 = __shfl_xor_sync(kFull, m2, off);
    top2_merge(m1, b1, m2, om1, ob1, om2);
  }
  // candidate level inside the winning block, by the whole team; every lane
  // of the warp takes part (the finish shuffles over the full warp), teams
  // without a pixel or without a block keep their result
  if (TF) {
    float e1, e2;
    unsigned bits;
    team_finish<L1, L2, CLOSED>(sM, sv, lt, T, kFull, m1 < kInf ? b1 : 0u, e1, bits, e2);
    if (m1 < kInf) {
      m1 = e1;
      b1 = bits;
      m2 = fminf(m2, e2);
    }
  }

  // epilogue: n* = base + bits and r = n* - c in double-float, one lane per
  // dot, kept in the team's slot-table rows (dead after the finish: r.hi in
  // sh, the bits of r.lo in sdot); then U(n*) = 1/2 r^T M r with the team's
  // lanes splitting the rows.  A row's products M_ij r_j are summed with
  // error-free sums of their high parts and plain FP32 sums of the rounding
  // errors and low-order parts, whose own error is O(u^2) of the row's
  // magnitude, then renormalised to double-float.
  df u = {0.f, 0.f};
  unsigned flags = 0u;
  __syncwarp();
  float* rhi = sht;
  int* rlo = sdot;
  // int8 maps of 4, 8 or 16 dots with a lane per dot: the team's charges go
  // out as one 4-, 8- or 16-byte store per pixel (the same for every team of
  // the launch, so the shuffles below are warp-uniform)
  const bool vec = !a.out_n16 && (n == 4 || n == 8 || n == 16) && T >= n &&
                   (reinterpret_cast<uintptr_t>(a.out_n) & (uintptr_t)(n - 1)) == 0;
  unsigned word = 0u;
  // the record's flags and bound, and the lane's dots' base and c, four dots
  // at a time: their loads are issued together (one round trip to L2)
  const unsigned rflags = active ? rec->flags : 0u;
  const float rbound = active ? rec->bound : 0.f;
  if (active) {
    for (int i0 = lt; i0 < n; i0 += 4 * T) {
      int bq[4];
      float chq[4], clq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + q * T;
        const int ic = i < n ? i : i0;
        bq[q] = rec->base[ic];
        chq[q] = rec->chi[ic];
        clq[q] = rec->clo[ic];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + q * T;
        if (i >= n) continue;
        int ni = bq[q];
        if ((mask >> i) & 1u) {
          const int si = BNB ? slot_of[i] : __popc(mask & ((1u << i) - 1u));
          ni += (int)((b1 >> si) & 1u);
        }
        const df ri = df_sub({(float)ni, 0.f}, {chq[q], clq[q]});
        rhi[i] = ri.hi;
        rlo[i] = __float_as_int(ri.lo);
        if (vec) {
          if (ni > 127) { ni = 127; flags |= kFlagOverflow; }
          word = (unsigned)ni << (8 * (lt & 3));
        } else {
          store_charge(a, p * n + i, ni, flags);
        }
      }
    }
  }
  if (vec) {
    // bytes of lanes 4q .. 4q + 3 into word q (held by all four), then lane 0
    // of the team gathers the words and stores them
    word |= __shfl_xor_sync(kFull, word, 1);
    word |= __shfl_xor_sync(kFull, word, 2);
    const int tb = (int)(threadIdx.x & 31u) & ~(T - 1);
    const unsigned w1 = __shfl_sync(kFull, word, (tb + 4) & 31);
    const unsigned w2 = __shfl_sync(kFull, word, (tb + 8) & 31);
    const unsigned w3 = __shfl_sync(kFull, word, (tb + 12) & 31);
    if (active && lt == 0) {
      int8_t* dst = a.out_n + p * n;
      if (n == 16) *reinterpret_cast<int4*>(dst) = make_int4((int)word, (int)w1, (int)w2, (int)w3);
      else if (n == 8) *reinterpret_cast<int2*>(dst) = make_int2((int)word, (int)w1);
      else *reinterpret_cast<int*>(dst) = (int)word;
    }
  }
  __syncwarp();
  // U = r^T M r.  The pruned search's wide teams (a row per lane) sum full
  // rows, M_ij r_j over j, scaled by r_i.  Narrower teams, whose lanes take
  // several rows each, use the symmetry: U = sum_i r_i S_i with
  // S_i = M_ii r_i + 2 sum_{j > i} M_ij r_j (the upper triangle, 136 products
  // at N = 16 instead of 256); rows i and N - 1 - i pair up to N + 1
  // products, one pair per task, or half a pair when the team has lanes for
  // that; a task's part of each row is summed, scaled by r_i and added to
  // the lane's u.  (Measured: the shorter sums do not pay at 16 lanes, where
  // the pair tasks' extra code costs more than the products they save.)
  if (active && BNB) {
    const int nc = T >= 2 * n ? T / n : 1;
    const int cw = (n + nc - 1) / nc;
    for (int task = lt; task < n * nc; task += T) {
      const int i = task / nc, j0 = (task % nc) * cw, j1 = min(n, j0 + cw);
      float shi = 0.f, slo = 0.f;
      for (int j = j0; j < j1; ++j) {
        const float mh = sM[i * kLdM + j], ml = sMlo[i * kLdM + j];
        const float xh = rhi[j], xl = __int_as_float(rlo[j]);
        const df pr = two_prod(mh, xh);
        const float small = __fmaf_rn(mh, xl, __fmaf_rn(ml, xh, pr.lo));
        const df sm = two_sum(shi, pr.hi);
        shi = sm.hi;
        slo = __fadd_rn(slo, __fadd_rn(sm.lo, small));
      }
      const df acc = fast_two_sum(shi, slo);
      u = df_add(u, df_mul(acc, {rhi[i], __int_as_float(rlo[i])}));
    }
  } else if (active) {
    const int npair = (n + 1) >> 1;
    const int nt = T >= 2 * npair ? 2 : 1;
    for (int task = lt; task < npair * nt; task += T) {
      const int pp = task / nt, hh = task - pp * nt;
      const int q = n - 1 - pp;
      const int len1 = n - pp, len = len1 + (q != pp ? pp + 1 : 0);
      const int mid = (len + 1) >> 1;
      const int e0 = (nt == 2 && hh) ? mid : 0;
      const int e1 = (nt == 2 && !hh) ? mid : len;
      for (int seg = 0; seg < 2; ++seg) {
        const int i = seg ? q : pp;
        const int sa = seg ? max(e0 - len1, 0) : e0;
        const int sb = seg ? e1 - len1 : min(e1, len1);
        if (sb <= sa) continue;
        const int ja = i + sa, jb = i + sb;
        // four columns per step with their loads issued together and two
        // independent sums (even and odd columns), joined error-free at the
        // end; a column past the range adds exact zeros, the off-diagonal
        // ones count twice (an exact scaling)
        float shi[2] = {0.f, 0.f}, slo[2] = {0.f, 0.f};
        for (int jb4 = ja; jb4 < jb; jb4 += 4) {
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int j = jb4 + jj;
            const bool on = j < jb;
            const int jc = on ? j : ja;
            const float wt = !on ? 0.f : (j == i ? 1.f : 2.f);
            const float mh = wt * sM[i * kLdM + jc], ml = wt * sMlo[i * kLdM + jc];
            const float xh = rhi[jc], xl = __int_as_float(rlo[jc]);
            const df pr = two_prod(mh, xh);
            const float small = __fmaf_rn(mh, xl, __fmaf_rn(ml, xh, pr.lo));
            const df sm = two_sum(shi[jj & 1], pr.hi);
            shi[jj & 1] = sm.hi;
            slo[jj & 1] = __fadd_rn(slo[jj & 1], __fadd_rn(sm.lo, small));
          }
        }
        const df st = two_sum(shi[0], shi[1]);
        const df acc = two_sum(st.hi, __fadd_rn(st.lo, __fadd_rn(slo[0], slo[1])));
        u = df_add(u, df_mul(acc, {rhi[i], __int_as_float(rlo[i])}));
      }
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
    flags |= rflags;
    if (!(m2 - m1 > rbound)) flags |= kFlagNearTie;
    if (lt == 0) {
      if (a.out_U) a.out_U[p] = 0.5 * df_to_double(u);
      if (flags & (kFlagBoundary | kFlagQPCap | kFlagUnresolved)) {
        // the candidate set itself may be wrong: FP64 recheck
        const unsigned at = atomicAdd(&L.cnt->n_flag, 1u);
        L.flag_list[at] = ListEntry{array, (int)p, m1, (flags & kFlagNearTie) ? 1 : 0};
        my_bd = 1;
      } else if (flags & kFlagNearTie) {
        // right set, uncertain order: exact energies of the close candidates
        const unsigned at = atomicAdd(&L.cnt->n_tie, 1u);
        L.tie_list[at] = ListEntry{array, (int)p, m1, 0};
        my_nt = 1;
      }
      my_ov = (flags & kFlagOverflow) ? 1u : 0u;
      if (a.out_flags) a.out_flags[p] = (uint8_t)flags;
    }
  }
  // one block sum of the four counts packed in 64 bits: evaluated slots in
  // the low 32 (at most 128 pixels of 2^16 slots per block, 2^23), near-tie,
  // recheck and overflow pixels (<= 128 each) in 10 bits apiece above
  const unsigned long long packed = block_sum(
      ev | ((unsigned long long)my_nt << 32) | ((unsigned long long)my_bd << 42) |
          ((unsigned long long)my_ov << 52),
      sh.red64);
  if (threadIdx.x == 0) {
    acc.evaluated += packed & 0xffffffffull;
    acc.near_tie += (unsigned)((packed >> 32) & 0x3ffu);
    acc.boundary += (unsigned)((packed >> 42) & 0x3ffu);
    acc.overflow += (unsigned)(packed >> 52);
  }
}

// ---------------------------------------------------------------------------
// (a7, near ties) for one list entry: a pixel whose candidate set is certain
// but whose FP32 best/runner-up gap is under the error bound.  The block
// re-walks the candidates collecting every block of the split whose FP32
// minimum is within the bound of the search's minimum (the exact argmin is
// guaranteed to be among them) and evaluates those candidates exactly,
// relative to the base state,
//     E(b) = sum_{s in b} (h_s + M_ss / 2) + sum_{s < s' in b} M_ss',
// in double-float arithmetic with h = M (base - c) in double-float (about
// 1e-13 absolute).  No FP64 instructions: GB300's FP64 rate is a small
// fraction of its FP32 rate.  A pixel whose two best exact energies are
// within 1e-10 (a true tie) or whose list overflows goes on to the FP64
// recheck, which also applies the lexicographic tie rule.  The resolve split
// is kCheckL1 / kCheckL2 for every array; the search's bound covers it (it
// was derived for a middle level at least as deep).  A block runs an entry's
// code once per launch, on cold instruction caches, so the small reductions
// and sums below stay rolled loops: their bodies are fetched once.
// ---------------------------------------------------------------------------
struct ResolveShared {
  ModelConsts cs;
  int sdot[kMaxDot];
  float sh[kMaxDot];
  df shd[kMaxDot];
  df sui[kMaxDot];
  float pk[kMaxDot][kMaxDot + 1];   // pair terms of the pixel's slots, M_{dot(s) dot(s2)}
  float pkl[kMaxDot][kMaxDot + 1];  // ... and their low parts
  unsigned blist[128];
  unsigned bcnt;
  df rbest[kResolveThreads / 32], rsec[kResolveThreads / 32];
  unsigned rbits[kResolveThreads / 32];
  unsigned dbits;   // the decision of warp 0, for the whole block
  int dok;
  unsigned dflags;
  df ub;            // U(base)
};

template <bool CLOSED>
__device__ inline void resolve_entry(const GsLaunch& L, const ArrayDesc& a, ResolveShared& S,
                                     ListEntry te, unsigned& my_res, unsigned& my_slmax) {
  constexpr int L1 = kCheckL1, L2 = kCheckL2;
  constexpr int NI = 1 << L1;
  constexpr int NM = 1 << L2;
  constexpr int NW = kResolveThreads / 32;
  constexpr unsigned kCap = 128;
  const float* sM = S.cs.Mhi;
  const float* sMlo = S.cs.Mlo;
  const int n = a.n;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  int* sdot = S.sdot;
  float* sh = S.sh;
  df* shd = S.shd;
  df* sui = S.sui;
  unsigned* blist = S.blist;
  unsigned& bcnt = S.bcnt;
  df* rbest = S.rbest;
  df* rsec = S.rsec;
  unsigned* rbits = S.rbits;
  const long long p = te.p;
  const PixRec* rec = a.recs + p;
  const unsigned mask = rec->mask;
  const int k = __popc(mask);
  const int w = rec->w;
  // the pixel's flags, read while the walk runs
  const unsigned char flags0 = (tid == 0 && a.out_flags) ? a.out_flags[p] : 0;
  // h_i = (M (base - c))_i in double-float, and U(base) = r0 . h / 2: one
  // product M_ij r_j per thread of the first 256 (row i = tid / 16), summed
  // over the row's 16 threads
  {
    static_assert(kResolveThreads >= kMaxDot * kMaxDot, "one thread per matrix entry");
    const int i = tid >> 4, j = tid & 15;
    df prod = {0.f, 0.f};
    if (i < n && j < n) {
      const df rj = df_sub({(float)rec->base[j], 0.f}, {rec->chi[j], rec->clo[j]});
      prod = df_mul({sM[i * kLdM + j], sMlo[i * kLdM + j]}, rj);
    }
#pragma unroll 1
    for (int off = 1; off < 16; off <<= 1) {
      df o;
      o.hi = __shfl_xor_sync(kFull, prod.hi, off, 16);
      o.lo = __shfl_xor_sync(kFull, prod.lo, off, 16);
      prod = df_add(prod, o);
    }
    if (j == 0 && i < n) {
      const df hi = prod;
      const df r0 = df_sub({(float)rec->base[i], 0.f}, {rec->chi[i], rec->clo[i]});
      sui[i] = df_mul(hi, r0);
      if ((mask >> i) & 1u) {
        const int s = __popc(mask & ((1u << i) - 1u));
        sdot[s] = i;
        sh[s] = rec->h[i];
        shd[s] = df_add(hi, df_mul_f({sM[i * kLdM + i], sMlo[i * kLdM + i]}, 0.5f));
      }
    }
  }
  if (tid == 0) bcnt = 0u;
  __syncthreads();
  // U(base) = sum_i r0_i h_i / 2, a 16-lane double-float sum in warp 0
  if (wid == 0) {
    df u = (lane < n) ? sui[lane] : df{0.f, 0.f};
#pragma unroll 1
    for (int off = 8; off > 0; off >>= 1) {
      df o;
      o.hi = __shfl_xor_sync(kFull, u.hi, off, 16);
      o.lo = __shfl_xor_sync(kFull, u.lo, off, 16);
      u = df_add(u, o);
    }
    if (lane == 0) S.ub = df_mul_f(u, 0.5f);
  }
  // the slots' pair terms, one per thread (zero outside the k slots), for
  // the shortlist's sums
  {
    const int s1 = tid >> 4, s2 = tid & 15;
    if (s1 < kMaxDot) {
      const bool on = s1 < k && s2 < k;
      const int e = on ? sdot[s1] * kLdM + sdot[s2] : 0;
      S.pk[s1][s2] = on ? sM[e] : 0.f;
      S.pkl[s1][s2] = on ? sMlo[e] : 0.f;
    }
  }
  // every block whose FP32 minimum is within the bound of the search's
  const SlotView sv{sdot, sh, k, w};
  const float thr = te.m1 + rec->bound;
  float d1, d2;
  unsigned db;
  unsigned long long ev = 0;
  static_assert(kResolveThreads <= 512, "the walk's team is the block: at most 9 lane bits");
  // (outer patterns whose lower bound is above the threshold plus the FP32
  // margin hold no block within the threshold)
  search_lane<L1, L2, CLOSED, true, false, 9>(sM, sv, tid, kResolveThreads, thr, blist, &bcnt,
                                    kCap, d1, db, d2, ev, nullptr, nullptr, nullptr,
                                    thr + 2.0f * rec->bound, S.cs.qneg);
  __syncthreads();
  const unsigned nb = bcnt;
  const bool fits = nb <= kCap;
  df best = {kInf, 0.f}, second = {kInf, 0.f};
  unsigned bbits = 0xffffffffu;
  if (fits) {
    // sixteen threads per shortlisted candidate, thread `sub` taking slot
    // sub when it is set: h_s + M_ss / 2 plus the pair terms with the set
    // slots below s, over a fixed range of slots with zero terms for the
    // others (no data-dependent chains); the high parts are summed
    // error-free, the low parts and rounding errors in plain FP32 (their own
    // error is O(u^2) of the magnitudes); the group then sums its slots
    constexpr int kSub = kMaxDot;
    const int sub = tid & (kSub - 1), grp = tid / kSub;
    const unsigned ncand = nb * NI;
    for (unsigned base_idx = 0; base_idx < ncand; base_idx += kResolveThreads / kSub) {
      const unsigned idx = base_idx + (unsigned)grp;
      bool ok = idx < ncand;
      unsigned bits = 0u;
      if (ok) {
        const unsigned id = blist[idx / NI];
        const unsigned b = idx % NI;
        bits = ((id >> L2) << (L1 + L2)) | ((id & (NM - 1)) << L1) | b;
        ok = (bits >> k) == 0u && (!CLOSED || __popc(bits) == w);
      }
      df E = {0.f, 0.f};
      if (ok && ((bits >> sub) & 1u)) {
        const float* Pr = S.pk[sub];
        const float* Pl = S.pkl[sub];
        const unsigned below = bits & ((1u << sub) - 1u);
        float hi = shd[sub].hi, lo = shd[sub].lo;
#pragma unroll 1
        for (int s2 = 0; s2 < kMaxDot - 1; ++s2) {
          const bool on = (below >> s2) & 1u;
          const df t = two_sum(hi, on ? Pr[s2] : 0.f);
          hi = t.hi;
          lo = __fadd_rn(lo, __fadd_rn(t.lo, on ? Pl[s2] : 0.f));
        }
        E = two_sum(hi, lo);
      }
#pragma unroll 1
      for (int off = 1; off < kSub; off <<= 1) {
        df o;
        o.hi = __shfl_xor_sync(kFull, E.hi, off, kSub);
        o.lo = __shfl_xor_sync(kFull, E.lo, off, kSub);
        E = df_add(E, o);
      }
      if (!ok || sub != 0) continue;
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
  // only the group leaders (sub = 0: lanes 0 and 16) hold candidates, so
  // one exchange merges a warp
  static_assert(kMaxDot == 16, "two candidate groups of kMaxDot threads per warp");
  {
    df ob, os;
    ob.hi = __shfl_xor_sync(kFull, best.hi, 16);
    ob.lo = __shfl_xor_sync(kFull, best.lo, 16);
    os.hi = __shfl_xor_sync(kFull, second.hi, 16);
    os.lo = __shfl_xor_sync(kFull, second.lo, 16);
    merge(ob, os, __shfl_xor_sync(kFull, bbits, 16));
  }
  if (lane == 0) { rbest[wid] = best; rsec[wid] = second; rbits[wid] = bbits; }
  __syncthreads();
  // warp 0 merges the warps' results as a shuffle tree (the order by energy,
  // then by the reversed bits, is total, so any merge order gives the same
  // best and second); lane 0 decides
  static_assert((NW & (NW - 1)) == 0 && NW <= 32, "warps of the block: a power of two");
  if (wid == 0) {
    const bool have = lane < NW;
    best = have ? rbest[lane] : df{kInf, 0.f};
    second = have ? rsec[lane] : df{kInf, 0.f};
    bbits = have ? rbits[lane] : 0xffffffffu;
#pragma unroll 1
    for (int off = NW / 2; off > 0; off >>= 1) {
      df ob, os;
      ob.hi = __shfl_xor_sync(kFull, best.hi, off);
      ob.lo = __shfl_xor_sync(kFull, best.lo, off);
      os.hi = __shfl_xor_sync(kFull, second.hi, off);
      os.lo = __shfl_xor_sync(kFull, second.lo, off);
      merge(ob, os, __shfl_xor_sync(kFull, bbits, off));
    }
  }
  if (tid == 0) {
    const df ub = S.ub;
    // exact-tie test in double-float: second - best against
    // 1e-10 (1 + |U(base)|) (no FP64 instructions on this path)
    const float gap = second.hi < kInf ? df_add(second, df_neg(best)).hi : kInf;
    const float eps = 1e-10f * (1.f + fabsf(ub.hi));
    const bool ok = fits && bbits != 0xffffffffu && gap > eps;
    S.dok = ok ? 1 : 0;  // not ok: the caller rechecks the pixel in FP64 next
    S.dbits = bbits;
    S.dflags = 0u;
    if (ok && a.out_U) a.out_U[p] = df_to_double(df_add(ub, best));
    // the shortlist length goes to the counters once per block, at the end
    // of the kernel (an atomic here would hold up the barrier below)
    my_slmax = nb > my_slmax ? nb : my_slmax;
  }
  __syncthreads();
  // the charges, one dot per thread
  if (S.dok) {
    unsigned fl = 0u;
    if (tid < n) {
      int ni = rec->base[tid];
      if ((mask >> tid) & 1u) ni += (int)((S.dbits >> __popc(mask & ((1u << tid) - 1u))) & 1u);
      store_charge(a, p * n + tid, ni, fl);
      if (fl) atomicOr(&S.dflags, fl);
    }
    __syncthreads();
    if (tid == 0) {
      if (a.out_flags) a.out_flags[p] = (uint8_t)(flags0 | kFlagRechecked | S.dflags);
      my_res += 1;
    }
  }
}

// ---------------------------------------------------------------------------
// (a7) FP64 recheck of one list entry (one block per pixel):
//   1. c, the continuous minimum and the candidate set again, in FP64
//      (c and h by N threads in parallel, the minimum by one thread); when
//      that set is the one the FP32 path searched and the FP32 order of the
//      best two was certain, the search's result stands and the pixel is
//      done;
//   2. the FP32 search over that set with all threads -> m1;
//   3. the same search collecting every block whose minimum is within the
//      near-tie bound of m1 (the exact argmin is guaranteed to be there);
//   4. exact FP64 energies of those candidates, ties to the
//      lexicographically smallest charge vector.
// ---------------------------------------------------------------------------
struct RecheckShared {
  double qK[32][kQPRow];  // FP64 team QP of warp 0
  int qa[32];
  double qz[32], qc[32], v64[kMaxDot], sx64[kMaxDot];
  int sqp;
  float sM[kMaxDot * kLdM];
  int sdot[kMaxDot];
  float sh[kMaxDot];
  double sh64[kMaxDot], sc64[kMaxDot];
  int sbase[kMaxDot];
  int sk, sw, sstatus;
  unsigned smask, sflags;
  float sbound;
  float rm1[kRecheckThreads / 32];
  double re[kRecheckThreads / 32];
  unsigned rbits[kRecheckThreads / 32];
  unsigned blist[kBcap];
  unsigned bcount;
};

template <bool CLOSED>
__device__ inline void recheck_entry(const GsLaunch& L, const ArrayDesc& a, RecheckShared& S,
                                     ListEntry fe) {
  constexpr int L1 = kCheckL1, L2 = kCheckL2;
  constexpr int NI = 1 << L1;
  constexpr int NM = 1 << L2;
  constexpr int NW = kRecheckThreads / 32;
  const int n = a.n;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const float* sM = S.sM;
  int* sdot = S.sdot;
  float* sh = S.sh;
  double* sh64 = S.sh64;
  double* sc64 = S.sc64;
  int* sbase = S.sbase;
  int& sk = S.sk;
  int& sw = S.sw;
  int& sstatus = S.sstatus;
  unsigned& smask = S.smask;
  unsigned& sflags = S.sflags;
  float& sbound = S.sbound;
  float* rm1 = S.rm1;
  double* re = S.re;
  unsigned* rbits = S.rbits;
  unsigned* blist = S.blist;
  unsigned& bcount = S.bcount;
  const long long p = fe.p;
  if (tid < n) sc64[tid] = pixel_c_f64(a.md, a.ng, a.sc, a.mt.carrier, p, tid);
  __syncthreads();
  if (tid < 32) {
    // continuous minimum in FP64 by warp 0, lane i owning dot i: analytic
    // (Appendix C / D), else the team active-set QP
    const int lt = tid;
    const bool live = lt < n;
    const double ci = live ? sc64[lt] : 0.0;
    double csum = ci, cmax = live ? fabs(ci) : 0.0;
    for (int off = 1; off < 32; off <<= 1) {
      csum += __shfl_xor_sync(kFull, csum, off);
      cmax = fmax(cmax, __shfl_xor_sync(kFull, cmax, off));
    }
    const double nh = (double)a.mt.n_charges;
    double x = CLOSED ? ci + (nh - csum) * (live ? a.md->vs[lt] : 0.0) : ci;
    const unsigned A = __ballot_sync(kFull, live && x < 0.0);
    int st = 0;
    if (A) {
      if (CLOSED && a.mt.n_charges == 0) {
        x = 0.0;
      } else {
        double vi = 0.0;
        if (live)
          for (int j = 0; j < n; ++j) vi += a.md->Cdd[lt * n + j];
        if (lt < kMaxDot) S.v64[lt] = vi;
        double s = vi;
        for (int off = 1; off < 32; off <<= 1) s += __shfl_xor_sync(kFull, s, off);
        __syncwarp();
        unsigned Af = 0u;
        const double tol = 1e-12 * (fmax(cmax, 1.0) + nh);
        // warm start from the active set the FP32 QP settled on, if any
        const unsigned A0 = a.recs[p].qpA ? (unsigned)a.recs[p].qpA : A;
        st = qp_team<double, CLOSED>(n, lt, 32, kFull, 0, a.md->Cdd, n, S.v64, s, ci, nh, A0,
                                     tol, 8 * n + 8, S.qK, S.qa, S.qz, S.qc, x, Af);
      }
    }
    if (live) S.sx64[lt] = x;
    if (lt == 0) S.sqp = (A ? 1 : 0) | (st != 0 ? 2 : 0);
  }
  __syncthreads();
  if (wid == 0) {
    // the candidate set in FP64 (the rules of candidate_set_f64), lane i
    // deciding dot i, the closed doubling loop warp-uniform
    const bool live = lane < n;
    unsigned fl = (S.sqp & 1) ? kFlagQP : 0u;
    unsigned mask = 0u;
    int st = -1, w = -1, bi = 0;
    if (a.md->status == 0 && !(S.sqp & 2)) {
      const double xl = live ? S.sx64[lane] : 0.0;
      const double xi = xl > 0.0 ? xl : 0.0;
      const double fli = floor(xi);
      const double fr = xi - fli;
      double tt = a.mt.t;
      for (int iter = 0; iter < 40; ++iter) {
        const bool am = live && fabs(fr - 0.5) <= 0.5 * tt;
        bi = live ? (int)fli + ((!am && fr >= 0.5) ? 1 : 0) : 0;
        mask = __ballot_sync(kFull, am);
        if (!CLOSED) { st = 0; break; }
        int sum = bi;
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(kFull, sum, off);
        w = a.mt.n_charges - sum;
        if (w >= 0 && w <= __popc(mask)) { st = 0; break; }
        if (tt >= 1.0) break;
        tt = (tt <= 0.0) ? 1.0 : fmin(2.0 * tt, 1.0);
        fl |= kFlagDoubled;
      }
    }
    if (live) sbase[lane] = bi;
    // same candidate set as the FP32 search and a certain order: keep its result
    const PixRec* rec = a.recs + p;
    const bool same = st == 0 && fe.tie == 0 && mask == (unsigned)rec->mask &&
                      (!CLOSED || w == (int)rec->w) &&
                      __all_sync(kFull, !live || bi == (int)rec->base[lane]);
    if (lane == 0) {
      sflags = fl;
      smask = mask;
      sw = CLOSED ? w : -1;
      bcount = 0u;
      sstatus = st;
      if (same) {
        if (a.out_flags) a.out_flags[p] = (uint8_t)(a.out_flags[p] | fl | kFlagRechecked);
        sstatus = 1;
      }
    }
  }
  __syncthreads();
  if (sstatus == 1) return;
  if (sstatus != 0) {
    if (tid == 0) {
      if (a.out_flags) a.out_flags[p] |= (uint8_t)kFlagUnresolved;
      atomicAdd(&L.cnt->unresolved, 1ull);
    }
    return;
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
  static_assert(kRecheckThreads <= 512, "the walk's team is the block: at most 9 lane bits");
  search_lane<L1, L2, CLOSED, false, false, 9>(sM, sv, tid, kRecheckThreads, 0.f, nullptr,
                                     nullptr, 0u, m1, b1, m2, ev);
  for (int off = 16; off > 0; off >>= 1) m1 = fminf(m1, __shfl_xor_sync(kFull, m1, off));
  if (lane == 0) rm1[wid] = m1;
  __syncthreads();
  m1 = kInf;
  for (int i = 0; i < NW; ++i) m1 = fminf(m1, rm1[i]);
  const float thr = m1 + sbound;
  float d1, d2;
  unsigned db;
  search_lane<L1, L2, CLOSED, true, false, 9>(sM, sv, tid, kRecheckThreads, thr, blist,
                                    &bcount, kBcap, d1, db, d2, ev, nullptr, nullptr, nullptr,
                                    thr + 2.0f * sbound, a.md->k.qneg);
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
    const bool settled = !overflowed && bbits != 0xffffffffu;
    if (!settled) {
      flags |= kFlagUnresolved;
      atomicAdd(&L.cnt->unresolved, 1ull);
      if (a.out_flags) a.out_flags[p] = (uint8_t)flags;
    }
    sflags = flags;
    rbits[0] = bbits;
    sstatus = settled ? 2 : 3;
    atomicMax(&L.cnt->shortlist_max, (unsigned long long)nb);
  }
  __syncthreads();
  // the charges and U(n*) = 1/2 r^T M r, r = n* - c, by warp 0: lane i its
  // dot's charge and row of M r, then a shuffle sum
  if (sstatus == 2 && wid == 0) {
    const unsigned bb = rbits[0];
    const bool live = lane < n;
    int ni = live ? sbase[lane] : 0;
    if (live && ((mask >> lane) & 1u)) ni += (int)((bb >> __popc(mask & ((1u << lane) - 1u))) & 1u);
    double row = 0.0;
    for (int j = 0; j < n; ++j) {
      const int nj = __shfl_sync(kFull, ni, j);
      if (live) row += a.md->M[lane * n + j] * ((double)nj - sc64[j]);
    }
    double u = live ? ((double)ni - sc64[lane]) * row : 0.0;
    for (int off = 16; off > 0; off >>= 1) u += __shfl_xor_sync(kFull, u, off);
    unsigned fl = 0u;
    if (live) store_charge(a, p * n + lane, ni, fl);
    fl = __reduce_or_sync(kFull, fl);
    if (lane == 0) {
      if (a.out_U) a.out_U[p] = 0.5 * u;
      if (a.out_flags) a.out_flags[p] = (uint8_t)(sflags | fl);
    }
  }
}

}  // namespace qa
