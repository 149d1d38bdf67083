// qa_soft_bwd.cu -- soft occupation backward pass (instantiations) and the
// device model update.
#include "qa_soft.cuh"

namespace qa {

cudaError_t launch_soft_backward(const SoftLaunch& a, cudaStream_t st) {
  return dispatch_soft<true>(a, st);
}

// ---------------------------------------------------------------------------
// FP64 Cholesky inverse of a device Cdd (model update on the GPU).  One block,
// everything staged in shared memory: warp 0 factors column by column (lane j
// the pivot, the lanes below it one dot product each; the pivot's reciprocal
// once, products after), threads j < n solve for column j of the inverse, and the symmetrisation, Cdd 1 and the 1-norm
// condition number are spread over the block.
// ---------------------------------------------------------------------------
__global__ void k_model_update(ModelData* md, int n, int ng, const double* Cdd,
                               const double* Cgd) {
  __shared__ double C[kMaxDot * kMaxDot], L[kMaxDot * kMaxDot], Ms[kMaxDot * kMaxDot];
  __shared__ double rowsum[kMaxDot], colc[kMaxDot], colm[kMaxDot];
  __shared__ double inv_diag[kMaxDot];  // 1 / L_jj: one FP64 division per column
  __shared__ int ok;
  const int tid = threadIdx.x;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    const double v = 0.5 * (Cdd[i * n + j] + Cdd[j * n + i]);
    C[e] = v;
    md->Cdd[e] = v;
    L[e] = 0.0;
  }
  for (int e = tid; e < n * ng; e += blockDim.x) md->Cgd[e] = Cgd[e];
  if (tid == 0) ok = 1;
  __syncthreads();
  if (tid < 32) {
    for (int j = 0; j < n; ++j) {
      if (tid == j) {
        double d = C[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        const double ljj = d > 0.0 ? sqrt(d) : 0.0;
        L[j * n + j] = ljj;
        inv_diag[j] = d > 0.0 ? 1.0 / ljj : 0.0;
        if (!(d > 0.0)) ok = 0;
      }
      __syncwarp();
      if (!(L[j * n + j] > 0.0)) break;
      const double rjj = inv_diag[j];
      if (tid > j && tid < n) {
        double t = C[tid * n + j];
        for (int k = 0; k < j; ++k) t -= L[tid * n + k] * L[j * n + k];
        L[tid * n + j] = t * rjj;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (!ok) {
    if (tid == 0) {
      md->status = 1;
      md->k.model_bad = 1;
    }
    return;
  }
  if (tid < n) {
    const int col = tid;
    double z[kMaxDot], y[kMaxDot];
    for (int i = 0; i < n; ++i) {
      double t = (i == col) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) t -= L[i * n + k] * z[k];
      z[i] = t * inv_diag[i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = z[i];
      for (int k = i + 1; k < n; ++k) t -= L[k * n + i] * y[k];
      y[i] = t * inv_diag[i];
    }
    for (int i = 0; i < n; ++i) Ms[i * n + col] = y[i];
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    md->M[e] = 0.5 * (Ms[i * n + j] + Ms[j * n + i]);
  }
  if (tid < n) {
    double r = 0.0, sc = 0.0, sm = 0.0;
    for (int j = 0; j < n; ++j) {
      r += C[tid * n + j];
      sc += fabs(C[j * n + tid]);
      sm += fabs(0.5 * (Ms[j * n + tid] + Ms[tid * n + j]));
    }
    rowsum[tid] = r;
    colc[tid] = sc;
    colm[tid] = sm;
  }
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0, n1c = 0.0, n1m = 0.0;
    for (int i = 0; i < n; ++i) {
      tot += rowsum[i];
      n1c = fmax(n1c, colc[i]);
      n1m = fmax(n1m, colm[i]);
    }
    for (int i = 0; i < n; ++i) md->vs[i] = rowsum[i] / tot;
    md->cond = n1c * n1m;
    md->status = 0;
  }
  __syncthreads();
  // FP32 / double-float forms (same definitions as the host set-up)
  ModelConsts& k = md->k;
  for (int e = tid; e < kMaxDot * kLdM; e += blockDim.x) {
    const int i = e / kLdM, j = e % kLdM;
    const bool live = i < n && j < n;
    const df m = live ? df_from_double(md->M[i * n + j]) : df{0.f, 0.f};
    k.Mhi[e] = m.hi;
    k.Mlo[e] = m.lo;
    const df cd = live ? df_from_double(md->Cdd[i * n + j]) : df{0.f, 0.f};
    k.Cdd[e] = cd.hi;
    k.CddLo[e] = cd.lo;
  }
  if (tid < kMaxDot) {
    double r = 0.0;
    for (int j = 0; j < n && tid < n; ++j) r += md->Cdd[tid * n + j];
    k.sv[tid] = __double2float_rn(r);
    k.sv2[tid] = tid < n ? df_from_double(r) : df{0.f, 0.f};
    k.vs[tid] = tid < n ? df_from_double(md->vs[tid]) : df{0.f, 0.f};
    // the same FP32 sum as the host set-up, from the same FP32 roundings
    float al = 0.f;
    if (tid < n) {
      al = 0.5f * __double2float_rn(md->M[tid * n + tid]);
      for (int j = 0; j < tid; ++j) al += fabsf(__double2float_rn(md->M[tid * n + j]));
    }
    k.absl[tid] = al;
  }
  if (tid == 0) {
    double tot = 0.0;
    for (int e = 0; e < n * n; ++e) tot += md->Cdd[e];
    k.s_s = __double2float_rn(tot);
    k.bx_qp_scale = __double2float_rn(8.0 * md->cond * (n + 1) * 5.9604644775390625e-8);
    const double e1 = md->cond * (n + 1) * 5.9604644775390625e-8;
    k.bx_qp_scale2 = __double2float_rn(8.0 * e1 * e1);
    float qn = 0.f;  // from M itself (the other lanes' Mhi stores are not ordered yet)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) qn += fminf(0.f, __double2float_rn(md->M[i * n + j]));
    k.qneg = qn;
    k.pad2[0] = k.pad2[1] = 0;
    k.model_bad = md->status != 0;
    k.pad = 0;
  }
}

cudaError_t launch_model_update(ModelData* md, int n, int ng, const double* Cdd_dev,
                                const double* Cgd_dev, cudaStream_t st) {
  k_model_update<<<1, 32, 0, st>>>(md, n, ng, Cdd_dev, Cgd_dev);
  return cudaGetLastError();
}

}  // namespace qa
