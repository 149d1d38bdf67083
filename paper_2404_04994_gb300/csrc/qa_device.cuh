// qa_device.cuh -- device-side building blocks of libqarray (sm_103a).
//
// Method (arXiv 2404.04994, Sec. III): per pixel, the continuous minimum of
// U(x) = 1/2 (x - c)^T M (x - c), M = Cdd^-1, subject to x >= 0 (and
// 1^T x = N_hat for a closed array), then the argmin of U over the floor /
// floor + 1 neighbours of that minimum, pruned by Eq. "threshold".
//
// Precision plan: c, the analytic minimum and the linear coefficients
// h = M (base - c) are formed in double-float FP32 arithmetic (error-free
// transformations, Dekker 1971 / Knuth TAOCP Vol. 2 4.2.2); candidate energies
// are summed in plain FP32 with a per-pixel error bound; pixels whose decisions
// fall inside the bound are re-evaluated in FP64 by the list kernel.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace qa {

constexpr int kMaxDot = 16;
constexpr int kMaxGate = 64;
constexpr int kLdM = 17;  // padded smem stride of N x N matrices

enum : unsigned {
  kFlagNearTie = 1u, kFlagBoundary = 2u, kFlagQP = 4u, kFlagQPCap = 8u,
  kFlagRechecked = 16u, kFlagDoubled = 32u, kFlagUnresolved = 64u,
  kFlagOverflow = 128u
};

// ---------------------------------------------------------------------------
// double-float arithmetic (value = hi + lo, |lo| <= ulp(hi) / 2)
// ---------------------------------------------------------------------------
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ df df_mul(df x, df y) {
  df p = two_prod(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
  return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ df df_mul_f(df x, float b) {
  df p = two_prod(x.hi, b);
  float e = __fmaf_rn(x.lo, b, p.lo);
  return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ df df_from_double(double v) {
  float hi = __double2float_rn(v);
  float lo = __double2float_rn(v - (double)hi);
  return {hi, lo};
}
__device__ __forceinline__ double df_to_double(df x) {
  return (double)x.hi + (double)x.lo;
}

// ---------------------------------------------------------------------------
// shared per-pixel record written by the prep kernel, read by the search
// ---------------------------------------------------------------------------
struct __align__(16) PixRec {
  float h[kMaxDot];     // FP32 of h = M (base - c), formed in double-float
  float chi[kMaxDot];   // c = s Cgd V as double-float
  float clo[kMaxDot];
  short base[kMaxDot];  // floor / rounded charges before the ambiguous +1s
  unsigned short mask;  // ambiguous dots (both floor and floor + 1 kept)
  unsigned char k;      // popcount(mask)
  signed char w;        // closed: number of ambiguous dots taking +1; open: -1
  unsigned char flags;  // QA flag bits from the prep stage
  unsigned char pad0;
  unsigned short qpA;   // QP pixels: the active set the FP32 QP settled on
  float bound;          // FP32 gap below which the pixel is a near-tie
};

// FP32 / double-float constants of a model, derived once from the FP64
// matrices whenever they change (host set-up or the device inverse) and
// staged by every block with plain 16-byte loads.
struct __align__(16) ModelConsts {
  float Mhi[kMaxDot * kLdM];   // M = Cdd^-1 as double-float (hi, lo)
  float Mlo[kMaxDot * kLdM];
  float Cdd[kMaxDot * kLdM];   // FP32 Cdd for the QP
  float sv[kMaxDot];           // Cdd 1
  df vs[kMaxDot];              // Cdd 1 / (1^T Cdd 1)   (Appendix D)
  float s_s;                   // 1^T Cdd 1
  float bx_qp_scale;           // QP decision margin per unit of (1+|c|+N_hat)
  int model_bad;               // device inverse of an updated Cdd failed (not PD)
  int pad;
  float CddLo[kMaxDot * kLdM]; // Cdd - hi part (Cdd as double-float with Cdd above)
  df sv2[kMaxDot];             // Cdd 1 as double-float
  float absl[kMaxDot];         // M_ii / 2 + sum_{j < i} |M_ij| (FP32 hi parts, j increasing)
  float bx_qp_scale2;          // ... after one double-float refinement of the QP
  float qneg;                  // sum of the negative off-diagonal M_ij, i < j (0 for Maxwell Cdd)
  int pad2[2];
};

// Device copy of a model (written by the host or by the device update).
struct __align__(16) ModelData {
  double Cdd[kMaxDot * kMaxDot];
  double M[kMaxDot * kMaxDot];        // Cdd^-1
  double Cgd[kMaxDot * kMaxGate];
  double vs[kMaxDot];                 // Cdd 1 / (1^T Cdd 1)   (Appendix D)
  double cond;                        // ||Cdd||_1 ||M||_1
  int status;                         // 0 ok; nonzero: Cdd not PD on update
  int pad;
  ModelConsts k;                      // FP32 forms of the above
};

// Where the voltages come from: a raster (by value) or a device list.
struct Scan {
  int kind;          // 0 raster, 1 points
  int W, H;
  long long P;
  double x0, dx, y0, dy;
  double V0[kMaxGate], u[kMaxGate], w[kMaxGate];
  const double* V;   // points: [P, n_gate]
};

// Raster induced-charge constants c0, du, dw (double-float), computed on the
// host when the host copy of the model is current.
struct RasterK {
  int valid;
  int pad;
  df c0[kMaxDot], du[kMaxDot], dw[kMaxDot];
};

struct Method {
  double t;          // threshold
  int closed;
  int n_charges;
  double carrier;    // +1 / -1
};

struct Counters {
  unsigned long long candidates, evaluated, qp, flagged, near_tie, boundary,
      unresolved, overflow, doubled, shortlist_max, resolved;
  unsigned int n_flag;  // length of the FP64 recheck list
  unsigned int n_tie;   // length of the near-tie list
  unsigned int q_prep;  // batched launch: work-queue heads
  unsigned int q_search;
  unsigned int q_var[20];  // batched launch: the search queue of each kernel variant
  unsigned int lists_done; // blocks of the list kernel that have finished
  unsigned int soft_done;  // blocks of the soft gradient reduction that have finished
};

// A single-array call's first kernel clears every counter but the two list
// heads, which its own blocks append to while others are still starting; the
// last block of the call's list kernel clears those (and lists_done)
// instead, so the heads are zero whenever a call starts.
__device__ __forceinline__ void zero_accumulators(Counters* c) {
  constexpr int nw = (int)(sizeof(Counters) / sizeof(unsigned));
  constexpr int k0 = (int)(offsetof(Counters, n_flag) / sizeof(unsigned));
  constexpr int k1 = (int)(offsetof(Counters, n_tie) / sizeof(unsigned));
  constexpr int k2 = (int)(offsetof(Counters, lists_done) / sizeof(unsigned));
  for (int e = threadIdx.x; e < nw; e += blockDim.x)
    if (e != k0 && e != k1 && e != k2) reinterpret_cast<unsigned*>(c)[e] = 0u;
}

// A pixel queued for the near-tie resolve or the FP64 recheck: its array (0
// for a single-array call), its index and the FP32 minimum of its search.
struct ListEntry {
  int array;
  int p;
  float m1;
  int tie;  // 1 when the order of the best two candidates is in doubt
};

// Copy the model's FP32 constants into shared memory (16-byte vectors).
__device__ __forceinline__ void stage_consts(const ModelConsts* g, ModelConsts* s) {
  const int4* src = reinterpret_cast<const int4*>(g);
  int4* dst = reinterpret_cast<int4*>(s);
  constexpr int nvec = (int)(sizeof(ModelConsts) / sizeof(int4));
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = src[i];
}

// Per-block counters written without atomics (summed on the host on demand).
struct BlockCounts {
  unsigned long long candidates;  // prep: admissible candidates
  unsigned long long evaluated;   // search: candidate energies evaluated
  unsigned int qp, doubled;       // prep
  unsigned int near_tie, boundary, overflow, pad;  // search
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
// Bit helpers written as straight-line code so that, inside fully unrolled
// loops, they fold to constants (a recursive form is not folded and turns
// register-array indices into local-memory accesses).
__host__ __device__ constexpr int ctz_c(unsigned v) {
  return (v & 0x1u) ? 0 : (v & 0x2u) ? 1 : (v & 0x4u) ? 2 : (v & 0x8u) ? 3
       : (v & 0x10u) ? 4 : (v & 0x20u) ? 5 : (v & 0x40u) ? 6 : (v & 0x80u) ? 7
       : (v & 0x100u) ? 8 : (v & 0x200u) ? 9 : 10;
}
__host__ __device__ constexpr unsigned gray_c(unsigned s) { return s ^ (s >> 1); }
__host__ __device__ constexpr int popc_c(unsigned v) {
  return (int)(v & 1u) + (int)((v >> 1) & 1u) + (int)((v >> 2) & 1u) +
         (int)((v >> 3) & 1u) + (int)((v >> 4) & 1u) + (int)((v >> 5) & 1u) +
         (int)((v >> 6) & 1u) + (int)((v >> 7) & 1u) + (int)((v >> 8) & 1u) +
         (int)((v >> 9) & 1u);
}

// 3-input minimum (PTX ISA 8.8+, sm_100+).
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the previous kernel of the stream finishes;
// it waits here before touching that kernel's results.  The previous kernel
// lets it start once every block has signalled (or exited).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_signal() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  return __fadd2_rn(a, b);
}

// ---------------------------------------------------------------------------
// stage (a1): the induced charge c(p) = s Cgd V(p) in double-float
// ---------------------------------------------------------------------------
// Block-level setup for a raster: c(ix, iy) = c0 + ix du + iy dw with
// c0 = s Cgd (V0 + x0 u + y0 w), du = s Cgd u dx, dw = s Cgd w dy (FP64, split).
struct RasterC {
  df c0[kMaxDot], du[kMaxDot], dw[kMaxDot];
};

__device__ inline void raster_setup(const ModelData* md, int n, int ng,
                                    const Scan& sc, double carrier,
                                    df* c0, df* du, df* dw) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int g = 0; g < ng; ++g) {
      double G = md->Cgd[i * ng + g];
      a += G * (sc.V0[g] + sc.x0 * sc.u[g] + sc.y0 * sc.w[g]);
      b += G * sc.u[g];
      c += G * sc.w[g];
    }
    c0[i] = df_from_double(carrier * a);
    du[i] = df_from_double(carrier * b * sc.dx);
    dw[i] = df_from_double(carrier * c * sc.dy);
  }
}

__device__ __forceinline__ df raster_c(df c0, df du, df dw, int ix, int iy) {
  df a = df_mul_f(du, (float)ix);   // ix, iy < 2^24: exact as floats
  df b = df_mul_f(dw, (float)iy);
  return df_add(c0, df_add(a, b));
}

// c for a point list: s * sum_g Cgd_ig V_g in double-float
__device__ inline df point_c(const double* Cgd_row, const double* Vp, int ng,
                             double carrier) {
  df acc = {0.f, 0.f};
  for (int g = 0; g < ng; ++g) {
    df G = df_from_double(carrier * Cgd_row[g]);
    df v = df_from_double(Vp[g]);
    acc = df_add(acc, df_mul(G, v));
  }
  return acc;
}

}  // namespace qa
