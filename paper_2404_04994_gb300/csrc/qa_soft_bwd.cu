// qa_soft_bwd.cu -- soft occupation backward pass (instantiations) and the
// device model update.
#include "qa_soft.cuh"

namespace qa {

cudaError_t launch_soft_backward(const SoftLaunch& a, cudaStream_t st) {
  return dispatch_soft<true>(a, st);
}

// ---------------------------------------------------------------------------
// FP64 inverse of a device Cdd (model update on the GPU) by the symmetric
// sweep operator (Gauss-Jordan elimination on diagonal pivots; Goodnight,
// The American Statistician 33 (1979) 149).  Sweeping pivot k of a symmetric
// matrix A with D = a_kk:
//   a_kk <- -1/D,   a_ik = a_ki <- a_ik / D,   a_ij <- a_ij - a_ik a_kj / D,
// and once every pivot is swept A holds -A^-1.  On a positive definite matrix
// each pivot is a diagonal entry of a Schur complement, so D > 0; a pivot
// <= 0 means Cdd is not positive definite.  One thread per entry (n^2 <=
// 256) and two shared buffers, one barrier per pivot; the product a_ik a_kj
// is the same for (i, j) and (j, i), so the result is exactly symmetric.
// Warp 0 then forms the row sums Cdd 1, the 1-norm condition number and the
// per-dot constants with shuffles; the block fills the FP32 / double-float
// forms (same definitions as the host set-up).
// ---------------------------------------------------------------------------
constexpr int kUpdThreads = kMaxDot * kMaxDot;

__global__ void __launch_bounds__(kUpdThreads) k_model_update(ModelData* md, int n, int ng,
                                                              const double* Cdd,
                                                              const double* Cgd) {
  __shared__ double A[2][kMaxDot * kMaxDot];
  __shared__ double C[kMaxDot * kMaxDot];
  const int tid = threadIdx.x;
  const int nn = n * n;
  const int i = tid / n, j = tid % n;  // this thread's entry when tid < nn
  if (tid < nn) {
    const double v = 0.5 * (Cdd[i * n + j] + Cdd[j * n + i]);
    C[tid] = v;
    A[0][tid] = v;
    md->Cdd[tid] = v;
  }
  for (int e = tid; e < n * ng; e += blockDim.x) md->Cgd[e] = Cgd[e];
  __syncthreads();
  bool ok = true;
  for (int k = 0; k < n; ++k) {
    const double* a = A[k & 1];
    double* b = A[(k + 1) & 1];
    const double D = a[k * n + k];  // the same value in every thread
    if (!(D > 0.0)) {
      ok = false;
      break;
    }
    if (tid < nn) {
      const double r = 1.0 / D;
      double v;
      if (i == k && j == k) v = -r;
      else if (i == k) v = a[k * n + j] * r;
      else if (j == k) v = a[i * n + k] * r;
      else v = fma(-(a[i * n + k] * a[k * n + j]), r, a[i * n + j]);
      b[tid] = v;
    }
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) {
      md->status = 1;
      md->k.model_bad = 1;
    }
    return;
  }
  // M = -(swept A) into the buffer the last pivot read
  double* Ms = A[(n + 1) & 1];
  if (tid < nn) {
    const double m = -A[n & 1][tid];
    Ms[tid] = m;
    md->M[tid] = m;
  }
  __syncthreads();
  ModelConsts& kc = md->k;
  for (int e = tid; e < kMaxDot * kLdM; e += blockDim.x) {
    const int r = e / kLdM, c = e % kLdM;
    df m = {0.f, 0.f}, cd = {0.f, 0.f};
    if (r < n && c < n) {
      m = df_from_double(Ms[r * n + c]);
      cd = df_from_double(C[r * n + c]);
    }
    kc.Mhi[e] = m.hi;
    kc.Mlo[e] = m.lo;
    kc.Cdd[e] = cd.hi;
    kc.CddLo[e] = cd.lo;
  }
  if (tid < 32) {
    const bool live = tid < n;
    double r = 0.0, sc = 0.0, sm = 0.0;
    if (live)
      for (int q = 0; q < n; ++q) {
        r += C[tid * n + q];
        sc += fabs(C[q * n + tid]);
        sm += fabs(Ms[q * n + tid]);
      }
    double tot = r, n1c = sc, n1m = sm;
    for (int off = 16; off > 0; off >>= 1) {
      tot += __shfl_xor_sync(0xffffffffu, tot, off);
      n1c = fmax(n1c, __shfl_xor_sync(0xffffffffu, n1c, off));
      n1m = fmax(n1m, __shfl_xor_sync(0xffffffffu, n1m, off));
    }
    const double cond = n1c * n1m;
    const double vsi = live ? r / tot : 0.0;
    if (live) md->vs[tid] = vsi;
    // the same FP32 sums as the host set-up, from the same FP32 roundings
    float al = 0.f, qn = 0.f;
    if (live) {
      al = 0.5f * __double2float_rn(Ms[tid * n + tid]);
      for (int q = 0; q < tid; ++q) {
        const float mij = __double2float_rn(Ms[tid * n + q]);
        al += fabsf(mij);
        qn += fminf(0.f, mij);
      }
    }
    if (tid < kMaxDot) {
      kc.sv[tid] = __double2float_rn(r);
      kc.sv2[tid] = live ? df_from_double(r) : df{0.f, 0.f};
      kc.vs[tid] = live ? df_from_double(vsi) : df{0.f, 0.f};
      kc.absl[tid] = al;
    }
    for (int off = 16; off > 0; off >>= 1) qn += __shfl_xor_sync(0xffffffffu, qn, off);
    if (tid == 0) {
      md->cond = cond;
      md->status = 0;
      kc.s_s = __double2float_rn(tot);
      const double e1 = cond * (n + 1) * 5.9604644775390625e-8;
      kc.bx_qp_scale = __double2float_rn(8.0 * e1);
      kc.bx_qp_scale2 = __double2float_rn(8.0 * e1 * e1);
      kc.qneg = qn;
      kc.pad2[0] = kc.pad2[1] = 0;
      kc.model_bad = 0;
      kc.pad = 0;
    }
  }
}

cudaError_t launch_model_update(ModelData* md, int n, int ng, const double* Cdd_dev,
                                const double* Cgd_dev, cudaStream_t st) {
  k_model_update<<<1, kUpdThreads, 0, st>>>(md, n, ng, Cdd_dev, Cgd_dev);
  return cudaGetLastError();
}

}  // namespace qa
