// qa_prep.cuh -- per-pixel preparation: continuous minimum (Sec. III.A) and
// the floor / threshold candidate set (Sec. III.B, Eq. "threshold").
#pragma once

#include "qa_device.cuh"

namespace qa {

constexpr int kQPRow = kMaxDot + 1;  // row length of the team QP's shared KKT rows

// ---------------------------------------------------------------------------
// Continuous minimum when the analytic one is infeasible (Sec. III.A.2).
//
// The paper hands min 1/2 (x - c)^T M (x - c), x >= 0 [, 1^T x = N_hat] to
// OSQP.  Here the KKT system is solved exactly for a working active set A
// (x_A = 0).  Stationarity M (x - c) = z + lambda 1 gives
//     x = c + Cdd (z + lambda 1),  z_F = 0,
// so for a fixed A only a small system in Cdd (not M) is solved:
//     [Cdd_AA        (Cdd 1)_A ] [z_A   ]   [ -c_A          ]
//     [(Cdd 1)_A^T   1^T Cdd 1 ] [lambda] = [ N_hat - 1^T c ]   (closed)
// (open: the first block row alone).  The bordered matrix is P^T Cdd P with
// P = [E_A, 1], hence SPD whenever A is not every dot.  A grows by the
// indices with x_i < 0 and shrinks by the most negative z_i, at most `cap`
// times; failure to settle is reported (never a loop without bound).
// T = float for the search path, double for the FP64 recheck.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ int qp_active_set(int n, const T* Cdd, int ldc,
                                          const T* c, bool closed, T nhat,
                                          const T* v, T s, unsigned A, T tol,
                                          int cap, T* x) {
  for (int it = 0; it < cap; ++it) {
    int a[kMaxDot];
    int m = 0;
    for (int i = 0; i < n; ++i)
      if ((A >> i) & 1u) a[m++] = i;
    if (closed && m == n) return -1;
    const int ms = m + (closed ? 1 : 0);
    T K[(kMaxDot + 1) * (kMaxDot + 1)];
    T z[kMaxDot + 1];
    T csum = 0;
    for (int i = 0; i < n; ++i) csum += c[i];
    for (int p = 0; p < m; ++p) {
      for (int q = 0; q <= p; ++q) K[p * ms + q] = Cdd[a[p] * ldc + a[q]];
      z[p] = -c[a[p]];
    }
    if (closed) {
      for (int q = 0; q < m; ++q) K[m * ms + q] = v[a[q]];
      K[m * ms + m] = s;
      z[m] = nhat - csum;
    }
    // Cholesky (lower triangle) and two triangular solves, in place
    bool ok = true;
    for (int j = 0; j < ms && ok; ++j) {
      T d = K[j * ms + j];
      for (int q = 0; q < j; ++q) d -= K[j * ms + q] * K[j * ms + q];
      if (!(d > (T)0)) { ok = false; break; }
      T ljj = sqrt(d);
      K[j * ms + j] = ljj;
      for (int i = j + 1; i < ms; ++i) {
        T e = K[i * ms + j];
        for (int q = 0; q < j; ++q) e -= K[i * ms + q] * K[j * ms + q];
        K[i * ms + j] = e / ljj;
      }
    }
    if (!ok) return -1;
    for (int i = 0; i < ms; ++i) {
      T e = z[i];
      for (int q = 0; q < i; ++q) e -= K[i * ms + q] * z[q];
      z[i] = e / K[i * ms + i];
    }
    for (int i = ms - 1; i >= 0; --i) {
      T e = z[i];
      for (int q = i + 1; q < ms; ++q) e -= K[q * ms + i] * z[q];
      z[i] = e / K[i * ms + i];
    }
    const T lam = closed ? z[m] : (T)0;
    unsigned neg = 0u;
    for (int i = 0; i < n; ++i) {
      if ((A >> i) & 1u) { x[i] = 0; continue; }
      T e = c[i] + lam * (closed ? v[i] : (T)0);
      for (int p = 0; p < m; ++p) e += Cdd[i * ldc + a[p]] * z[p];
      x[i] = e;
      if (e < -tol) neg |= 1u << i;
    }
    if (neg) { A |= neg; continue; }
    int worst = -1;
    T zw = -tol;
    for (int p = 0; p < m; ++p)
      if (z[p] < zw) { zw = z[p]; worst = a[p]; }
    if (worst >= 0) { A &= ~(1u << worst); continue; }
    for (int i = 0; i < n; ++i)
      if (x[i] < (T)0) x[i] = 0;
    return 0;
  }
  return -1;
}

// ---------------------------------------------------------------------------
// The same active-set method, run by a team of TP lanes (TP a power of two,
// TP >= n; lane i owns dot i; `tmask` the team's lanes of the warp, `tbase`
// the index of the team's first thread in the block).  Row p of the bordered
// KKT matrix lives in the shared row Ks[tbase + p][.] and is owned by lane p:
// the Cholesky factor is built column by column (lane j the pivot, lanes
// below it their entries, a dot product each), and both triangular solves
// proceed one unknown at a time with a shuffle broadcast, so the serial chain
// is O(m^2) instead of O(m^3).  Active-set decisions are team ballots.
// Returns 0 with x_i in lane i, or -1 (no PD system, or no settling within
// cap iterations).  T = float (prep) or double (FP64 recheck); Cdd has row
// stride ldc.  Every lane of tmask must call.  Out of line, as is the
// refinement below: few pixels need the QP, and inlined it spreads the
// prep's common path over more instruction-cache lines, which the prep
// shares with the search's walk in the one-kernel form.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float qrsqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double qrsqrt(double v) { return rsqrt(v); }

template <typename T, bool CLOSED>
__device__ __noinline__ int qp_team(int n, int lt, int TP, unsigned tmask, int tbase,
                                       const T* Cdd, int ldc, const T* v, T s, T ci, T nhat,
                                       unsigned A, T tol, int cap, T (*Ks)[kQPRow], int* alist,
                                       T* zs, T* cs, T& x, unsigned& Afinal) {
  const bool live = lt < n;
  cs[tbase + lt] = live ? ci : (T)0;
  T csum = live ? ci : (T)0;
  for (int off = 1; off < TP; off <<= 1) csum += __shfl_xor_sync(tmask, csum, off, TP);
  for (int it = 0; it < cap; ++it) {
    const int m = __popc(A);
    if (CLOSED && m == n) return -1;
    const int ms = m + (CLOSED ? 1 : 0);
    const bool act = live && ((A >> lt) & 1u);
    if (act) alist[tbase + __popc(A & ((1u << lt) - 1u))] = lt;
    __syncwarp(tmask);
    // row lt of K and its right-hand side
    T y = 0;
    if (lt < m) {
      const int ap = alist[tbase + lt];
      for (int q = 0; q <= lt; ++q) Ks[tbase + lt][q] = Cdd[ap * ldc + alist[tbase + q]];
      y = -cs[tbase + ap];
    } else if (CLOSED && lt == m) {
      for (int q = 0; q < m; ++q) Ks[tbase + lt][q] = v[alist[tbase + q]];
      Ks[tbase + lt][m] = s;
      y = nhat - csum;
    }
    __syncwarp(tmask);
    // Cholesky, column by column; the pivot's reciprocal 1 / L_jj (one
    // reciprocal square root) is kept in the row's spare last column, so the
    // column and both solves multiply instead of dividing
    bool ok = true;
    for (int j = 0; j < ms; ++j) {
      if (lt == j) {
        T d = Ks[tbase + j][j];
        for (int q = 0; q < j; ++q) d -= Ks[tbase + j][q] * Ks[tbase + j][q];
        const T r = d > (T)0 ? qrsqrt(d) : (T)0;
        Ks[tbase + j][j] = d * r;
        Ks[tbase + j][kQPRow - 1] = r;
      }
      __syncwarp(tmask);
      const T rjj = Ks[tbase + j][kQPRow - 1];
      if (!(rjj > (T)0)) { ok = false; break; }
      if (lt > j && lt < ms) {
        T e = Ks[tbase + lt][j];
        for (int q = 0; q < j; ++q) e -= Ks[tbase + lt][q] * Ks[tbase + j][q];
        Ks[tbase + lt][j] = e * rjj;
      }
      __syncwarp(tmask);
    }
    if (!ok) return -1;
    // L y = rhs, then L^T z = y (lane p holds unknown p)
    for (int q = 0; q < ms; ++q) {
      if (lt == q) y *= Ks[tbase + q][kQPRow - 1];
      const T yq = __shfl_sync(tmask, y, tbase % 32 + q);
      if (lt > q && lt < ms) y -= Ks[tbase + lt][q] * yq;
    }
    for (int q = ms - 1; q >= 0; --q) {
      if (lt == q) y *= Ks[tbase + q][kQPRow - 1];
      const T zq = __shfl_sync(tmask, y, tbase % 32 + q);
      if (lt < q) y -= Ks[tbase + q][lt] * zq;
    }
    if (lt < ms) zs[tbase + lt] = y;
    __syncwarp(tmask);
    const T lam = CLOSED ? zs[tbase + m] : (T)0;
    T xi = 0;
    if (live && !act) {
      xi = ci + (CLOSED ? lam * v[lt] : (T)0);
      for (int p = 0; p < m; ++p) xi += Cdd[lt * ldc + alist[tbase + p]] * zs[tbase + p];
    }
    const unsigned neg =
        (__ballot_sync(tmask, live && !act && xi < -tol) & tmask) >> (tbase % 32);
    __syncwarp(tmask);
    if (neg) { A |= neg; continue; }
    // most negative multiplier leaves the active set
    T zw = (lt < m) ? zs[tbase + lt] : (T)0;
    int wdot = (lt < m && zw < -tol) ? alist[tbase + lt] : -1;
    if (wdot < 0) zw = 0;
    for (int off = 1; off < TP; off <<= 1) {
      const T oz = __shfl_xor_sync(tmask, zw, off, TP);
      const int od = __shfl_xor_sync(tmask, wdot, off, TP);
      if (od >= 0 && (wdot < 0 || oz < zw || (oz == zw && od < wdot))) { zw = oz; wdot = od; }
    }
    __syncwarp(tmask);
    if (wdot >= 0) { A &= ~(1u << wdot); continue; }
    x = (live && !act) ? (xi > (T)0 ? xi : (T)0) : (T)0;
    Afinal = A;
    return 0;
  }
  return -1;
}

// One step of iterative refinement of a settled team QP (active set A, FP32
// multipliers in zs, the FP32 Cholesky factor of the bordered KKT matrix
// still in Ks): x is formed in double-float from c, Cdd (hi + lo) and the
// multipliers; the KKT residual (x_a for active a, N_hat - 1^T x closed) is
// solved for a correction with the same factor; x is formed again from the
// corrected multipliers (double-float).  The error of x drops from about
// cond(Cdd) u to (cond(Cdd) u)^2.  Returns nonzero when, at this precision,
// a free x_i or a multiplier is below -tol (the active set is then in doubt);
// `flip` then holds the dots whose constraint that suggests toggling (free
// dots with x_i < -tol, active dots with a multiplier below -tol).  Every
// lane of tmask must call; lane i returns x_i (0 for active dots).
template <bool CLOSED>
__device__ __noinline__ int qp_team_refine(int n, int lt, int TP, unsigned tmask, int tbase,
                                              const float* CddHi, const float* CddLo,
                                              const df* v2, df ci, float nhat, unsigned A,
                                              float tol, float (*Ks)[kQPRow], const int* alist,
                                              float* zs, float* zl, float* xr, df& x,
                                              unsigned& flip) {
  const bool live = lt < n;
  const int m = __popc(A);
  const int ms = m + (CLOSED ? 1 : 0);
  const bool act = live && ((A >> lt) & 1u);
  auto form_x = [&](bool with_lo) {
    df xi = live ? ci : df{0.f, 0.f};
    if (live) {
      if (CLOSED) {
        const df lam = {zs[tbase + m], with_lo ? zl[tbase + m] : 0.f};
        xi = df_add(xi, df_mul(v2[lt], lam));
      }
      for (int p = 0; p < m; ++p) {
        const int ap = alist[tbase + p];
        const df cd = {CddHi[lt * kLdM + ap], CddLo[lt * kLdM + ap]};
        const df zp = {zs[tbase + p], with_lo ? zl[tbase + p] : 0.f};
        xi = df_add(xi, df_mul(cd, zp));
      }
    }
    return xi;
  };
  df xi = form_x(false);
  xr[tbase + lt] = xi.hi + xi.lo;
  df xsum = xi;
  for (int off = 1; off < TP; off <<= 1) {
    df o;
    o.hi = __shfl_xor_sync(tmask, xsum.hi, off, TP);
    o.lo = __shfl_xor_sync(tmask, xsum.lo, off, TP);
    xsum = df_add(xsum, o);
  }
  __syncwarp(tmask);
  float y = 0.f;
  if (lt < m) y = -xr[tbase + alist[tbase + lt]];
  else if (CLOSED && lt == m) {
    const df r = df_sub({nhat, 0.f}, xsum);
    y = r.hi + r.lo;
  }
  for (int q = 0; q < ms; ++q) {
    if (lt == q) y *= Ks[tbase + q][kQPRow - 1];
    const float yq = __shfl_sync(tmask, y, tbase % 32 + q);
    if (lt > q && lt < ms) y -= Ks[tbase + lt][q] * yq;
  }
  for (int q = ms - 1; q >= 0; --q) {
    if (lt == q) y *= Ks[tbase + q][kQPRow - 1];
    const float zq = __shfl_sync(tmask, y, tbase % 32 + q);
    if (lt < q) y -= Ks[tbase + q][lt] * zq;
  }
  if (lt < ms) {
    const df zc = two_sum(zs[tbase + lt], y);
    zs[tbase + lt] = zc.hi;
    zl[tbase + lt] = zc.lo;
  }
  __syncwarp(tmask);
  xi = act ? df{0.f, 0.f} : form_x(true);
  const bool xbad = live && !act && xi.hi + xi.lo < -tol;
  const bool zbad = lt < m && zs[tbase + lt] + zl[tbase + lt] < -tol;
  const bool bad = xbad || zbad;
  const unsigned anybad = __ballot_sync(tmask, bad) & tmask;
  flip = __reduce_or_sync(tmask, (xbad ? (1u << lt) : 0u) |
                                     (zbad ? (1u << alist[tbase + lt]) : 0u));
  __syncwarp(tmask);
  if (xi.hi < 0.f || (xi.hi == 0.f && xi.lo < 0.f)) xi = {0.f, 0.f};
  x = xi;
  return anybad != 0u;
}

// ---------------------------------------------------------------------------
// Candidate set of the default / thresholded method for a double-float x.
// Dot i keeps both floor and floor + 1 iff |frac(x_i) - 1/2| <= t/2, else it
// takes the nearest integer; x_i is clamped to >= 0 first.  A closed array
// whose set holds no state with the right total doubles t (0 -> 1) and
// retries.  Any decision closer than bx to flipping sets kFlagBoundary.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void candidate_set_df(int n, const df* x, double t,
                                                 bool closed, int nhat,
                                                 float bx, int* base,
                                                 unsigned& mask, int& w,
                                                 unsigned& flags) {
  double tt = t;
  for (int iter = 0; iter < 40; ++iter) {
    const float th = __double2float_rn(0.5 * tt);
    unsigned mk = 0u;
    int sum = 0;
#pragma unroll
    for (int i = 0; i < kMaxDot; ++i) {
      if (i < n) {
        df xi = x[i];
        if (xi.hi < 0.f || (xi.hi == 0.f && xi.lo < 0.f)) xi = {0.f, 0.f};
        float fl = floorf(xi.hi);
        if (xi.hi == fl && xi.lo < 0.f) fl -= 1.f;
        const float fr = __fadd_rn(__fsub_rn(xi.hi, fl), xi.lo);
        const bool a = fabsf(fr - 0.5f) <= th;
        const int b = (int)fl + ((!a && fr >= 0.5f) ? 1 : 0);
        base[i] = b;
        sum += b;
        if (a) mk |= 1u << i;
        if (xi.hi >= 0.5f - bx && fminf(fr, 1.f - fr) < bx) flags |= kFlagBoundary;
        if (tt < 1.0 && fabsf(fabsf(fr - 0.5f) - th) < bx) flags |= kFlagBoundary;
      }
    }
    mask = mk;
    if (!closed) { w = -1; return; }
    w = nhat - sum;
    if (w >= 0 && w <= __popc(mk)) return;
    if (tt >= 1.0) {  // impossible in exact arithmetic: settle in FP64
      flags |= kFlagBoundary;
      w = w < 0 ? 0 : __popc(mk);
      return;
    }
    tt = (tt <= 0.0) ? 1.0 : fmin(2.0 * tt, 1.0);
    flags |= kFlagDoubled;
  }
}

// The same rules in FP64 (recheck path).
__device__ __forceinline__ int candidate_set_f64(int n, const double* x,
                                                 double t, bool closed,
                                                 int nhat, int* base,
                                                 unsigned& mask, int& w,
                                                 unsigned& flags) {
  double tt = t;
  for (int iter = 0; iter < 40; ++iter) {
    unsigned mk = 0u;
    int sum = 0;
    for (int i = 0; i < n; ++i) {
      const double xi = x[i] > 0.0 ? x[i] : 0.0;
      const double fl = floor(xi);
      const double fr = xi - fl;
      const bool a = fabs(fr - 0.5) <= 0.5 * tt;
      base[i] = (int)fl + ((!a && fr >= 0.5) ? 1 : 0);
      sum += base[i];
      if (a) mk |= 1u << i;
    }
    mask = mk;
    if (!closed) { w = -1; return 0; }
    w = nhat - sum;
    if (w >= 0 && w <= __popc(mk)) return 0;
    if (tt >= 1.0) return -1;
    tt = (tt <= 0.0) ? 1.0 : fmin(2.0 * tt, 1.0);
    flags |= kFlagDoubled;
  }
  return -1;
}

// ---------------------------------------------------------------------------
// FP64 preparation of one pixel (recheck path).
// ---------------------------------------------------------------------------
// Voltage of pixel p at gate g.
__device__ __forceinline__ double scan_voltage(const Scan& sc, int ng, long long p,
                                               int g) {
  if (sc.kind == 0) {
    const int ix = (int)(p % sc.W), iy = (int)(p / sc.W);
    return sc.V0[g] + (sc.x0 + ix * sc.dx) * sc.u[g] + (sc.y0 + iy * sc.dy) * sc.w[g];
  }
  return sc.V[p * ng + g];
}

// c_i = s (Cgd V(p))_i in FP64 (the raster position found once, not per gate;
// the voltages as in scan_voltage)
__device__ __forceinline__ double pixel_c_f64(const ModelData* md, int ng,
                                              const Scan& sc, double carrier,
                                              long long p, int i) {
  double a = 0.0;
  if (sc.kind == 0) {
    const long long iy = p / sc.W, ix = p - iy * sc.W;
    const double xs = sc.x0 + (int)ix * sc.dx, ys = sc.y0 + (int)iy * sc.dy;
    for (int g = 0; g < ng; ++g) a += md->Cgd[i * ng + g] * (sc.V0[g] + xs * sc.u[g] + ys * sc.w[g]);
  } else {
    for (int g = 0; g < ng; ++g) a += md->Cgd[i * ng + g] * sc.V[p * ng + g];
  }
  return carrier * a;
}

// Continuous minimum and candidate set in FP64 from a given c (one thread).
__device__ inline int settle_pixel_f64(const ModelData* md, int n, const Method& mt,
                                       const double* c, int* base, unsigned& mask,
                                       int& w, unsigned& flags) {
  double x[kMaxDot];
  const bool closed = mt.closed != 0;
  unsigned A = 0u;
  if (closed) {
    double cs = 0.0;
    for (int i = 0; i < n; ++i) cs += c[i];
    for (int i = 0; i < n; ++i) x[i] = c[i] + ((double)mt.n_charges - cs) * md->vs[i];
  } else {
    for (int i = 0; i < n; ++i) x[i] = c[i];
  }
  for (int i = 0; i < n; ++i)
    if (x[i] < 0.0) A |= 1u << i;
  if (A) {
    flags |= kFlagQP;
    if (closed && mt.n_charges == 0) {
      for (int i = 0; i < n; ++i) x[i] = 0.0;
    } else {
      double v[kMaxDot], s = 0.0, cmax = 1.0;
      for (int i = 0; i < n; ++i) {
        double r = 0.0;
        for (int j = 0; j < n; ++j) r += md->Cdd[i * n + j];
        v[i] = r;
        s += r;
        cmax = fmax(cmax, fabs(c[i]));
      }
      const double tol = 1e-12 * (cmax + (double)mt.n_charges);
      if (qp_active_set<double>(n, md->Cdd, n, c, closed, (double)mt.n_charges,
                                v, s, A, tol, 8 * n + 8, x) != 0)
        return -1;
    }
  }
  return candidate_set_f64(n, x, mt.t, closed, mt.n_charges, base, mask, w, flags);
}

__device__ inline int prep_pixel_f64(const ModelData* md, int n, int ng,
                                     const Scan& sc, const Method& mt,
                                     long long p, double* c, int* base,
                                     unsigned& mask, int& w, unsigned& flags) {
  for (int i = 0; i < n; ++i) c[i] = pixel_c_f64(md, ng, sc, mt.carrier, p, i);
  return settle_pixel_f64(md, n, mt, c, base, mask, w, flags);
}

}  // namespace qa
