// qa_prep.cuh -- per-pixel preparation: continuous minimum (Sec. III.A) and
// the floor / threshold candidate set (Sec. III.B, Eq. "threshold").
#pragma once

#include "qa_device.cuh"

namespace qa {

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

// c_i = s (Cgd V(p))_i in FP64
__device__ __forceinline__ double pixel_c_f64(const ModelData* md, int ng,
                                              const Scan& sc, double carrier,
                                              long long p, int i) {
  double a = 0.0;
  for (int g = 0; g < ng; ++g) a += md->Cgd[i * ng + g] * scan_voltage(sc, ng, p, g);
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
