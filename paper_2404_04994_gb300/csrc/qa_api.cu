// qa_api.cu -- host implementation of the C ABI declared in include/qarray.h.
//
// Argument validation, the FP64 model set-up (Cholesky inverse of Cdd,
// Appendix B positive-definiteness check), workspace management and kernel
// dispatch.  No pixel work happens on the host.
#include <algorithm>
#include <memory>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "qarray.h"
#include "qa_launch.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(QA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool finite_all(const double* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// Cholesky inverse in FP64; returns false if A is not positive definite.
bool spd_inverse(int n, const double* A, double* Ainv) {
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / ljj;
    }
  }
  for (int col = 0; col < n; ++col) {
    std::vector<double> z(n), y(n);
    for (int i = 0; i < n; ++i) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * z[k];
      z[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = z[i];
      for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * y[k];
      y[i] = s / L[i * n + i];
    }
    for (int i = 0; i < n; ++i) Ainv[i * n + col] = y[i];
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double s = 0.5 * (Ainv[i * n + j] + Ainv[j * n + i]);
      Ainv[i * n + j] = Ainv[j * n + i] = s;
    }
  return true;
}

double norm1(int n, const double* A) {
  double best = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += std::fabs(A[i * n + j]);
    best = s > best ? s : best;
  }
  return best;
}

}  // namespace

struct qa_model {
  int n = 0, ng = 0, form = 0;
  double carrier = 1.0;
  int device = 0, num_sms = 0;
  qa::ModelData host;            // host mirror (stale after update_dev)
  bool host_stale = false;
  qa::ModelData* d_md = nullptr; // device copy
  void* ws = nullptr;            // workspace
  size_t ws_bytes = 0;
  qa::Counters* d_cnt = nullptr;
  qa::SearchCfg last_cfg{0, 0, 0};
  long long last_P = 0;
  bool timing = false;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int last_kind = 0;  // 1 ground state, 2 soft
  qa::BlockCounts* d_bc_prep = nullptr;
  qa::BlockCounts* d_bc_search = nullptr;
  int n_bc_prep = 0, n_bc_search = 0;
  qa::ModelData* staging = nullptr;   // pinned, for asynchronous updates
  cudaEvent_t staged = nullptr;       // last copy out of `staging`
  // Model generation (bumped by every update) and the key of the records the
  // last soft-occupation prep left in the workspace: a backward with the
  // forward's context on the same model, raster and method reuses them.
  unsigned long long gen = 0;
  struct {
    bool valid;
    const void* recs;
    qa::Scan sc;
    double t;
    int closed, n_charges;
    unsigned long long gen;
  } soft_recs = {};
};

namespace {

qa::df split(double v) {
  const float hi = (float)v;
  return {hi, (float)(v - (double)hi)};
}

// FP32 / double-float forms of the model used by every kernel.
void fill_consts(int n, qa::ModelData* md) {
  qa::ModelConsts& k = md->k;
  std::memset(&k, 0, sizeof(k));
  double tot = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = 0.0;
    for (int j = 0; j < n; ++j) {
      const qa::df m = split(md->M[i * n + j]);
      k.Mhi[i * qa::kLdM + j] = m.hi;
      k.Mlo[i * qa::kLdM + j] = m.lo;
      const qa::df cd = split(md->Cdd[i * n + j]);
      k.Cdd[i * qa::kLdM + j] = cd.hi;
      k.CddLo[i * qa::kLdM + j] = cd.lo;
      r += md->Cdd[i * n + j];
    }
    k.sv[i] = (float)r;
    k.sv2[i] = split(r);
    k.vs[i] = split(md->vs[i]);
    tot += r;
    float al = 0.5f * k.Mhi[i * qa::kLdM + i];
    for (int j = 0; j < i; ++j) al += std::fabs(k.Mhi[i * qa::kLdM + j]);
    k.absl[i] = al;
  }
  k.s_s = (float)tot;
  // decision margin of an FP32 QP minimum: 8 cond(Cdd) (n + 1) u32 per unit
  // of (1 + max|c| + N_hat)
  k.bx_qp_scale = (float)(8.0 * md->cond * (n + 1) * 5.9604644775390625e-8);
  // after one refinement step with double-float residuals the error is the
  // square of the FP32 one (per unit of the same scale)
  const double e1 = md->cond * (n + 1) * 5.9604644775390625e-8;
  k.bx_qp_scale2 = (float)(8.0 * e1 * e1);
  // lower bound of any set of pair terms (the pruned search's bounds)
  float qn = 0.f;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) qn += std::fmin(0.f, k.Mhi[i * qa::kLdM + j]);
  k.qneg = qn;
  k.model_bad = md->status != 0;
}

// Validate + convert host matrices into a ModelData (Maxwell form).
int build_model(int n, int ng, int form, const double* Cdd_in,
                const double* Cgd_in, qa::ModelData* md) {
  if (!Cdd_in || !Cgd_in) return fail(QA_ERR_INVALID, "null capacitance matrix");
  if (n < 1 || n > QA_MAX_DOT) return fail(QA_ERR_SHAPE, "n_dot=%d outside [1, %d]", n, QA_MAX_DOT);
  if (ng < 1 || ng > QA_MAX_GATE) return fail(QA_ERR_SHAPE, "n_gate=%d outside [1, %d]", ng, QA_MAX_GATE);
  if (!finite_all(Cdd_in, (size_t)n * n) || !finite_all(Cgd_in, (size_t)n * ng))
    return fail(QA_ERR_INVALID, "non-finite capacitance");
  std::memset(md, 0, sizeof(*md));
  double amax = 0.0;
  for (int e = 0; e < n * n; ++e) amax = std::fmax(amax, std::fabs(Cdd_in[e]));
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (std::fabs(Cdd_in[i * n + j] - Cdd_in[j * n + i]) > 1e-12 * amax)
        return fail(QA_ERR_NOT_SYMMETRIC, "Cdd is not symmetric at (%d, %d)", i, j);
  if (form == QA_FORM_MAXWELL) {
    for (int e = 0; e < n * n; ++e) md->Cdd[e] = Cdd_in[e];
  } else if (form == QA_FORM_COUPLING) {
    // Appendix B: Maxwell diagonal = total capacitance of the node, off-
    // diagonals = minus the coupling.
    for (int i = 0; i < n; ++i) {
      double tot = 0.0;
      for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        if (Cdd_in[i * n + j] < 0.0) return fail(QA_ERR_INVALID, "negative coupling Cdd[%d,%d]", i, j);
        tot += Cdd_in[i * n + j];
        md->Cdd[i * n + j] = -Cdd_in[i * n + j];
      }
      for (int g = 0; g < ng; ++g) {
        if (Cgd_in[i * ng + g] < 0.0) return fail(QA_ERR_INVALID, "negative coupling Cgd[%d,%d]", i, g);
        tot += Cgd_in[i * ng + g];
      }
      md->Cdd[i * n + i] = tot;
    }
  } else {
    return fail(QA_ERR_INVALID, "unknown form %d", form);
  }
  for (int e = 0; e < n * ng; ++e) md->Cgd[e] = Cgd_in[e];
  if (!spd_inverse(n, md->Cdd, md->M))
    return fail(QA_ERR_NOT_PD, "Cdd is not positive definite");
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = 0.0;
    for (int j = 0; j < n; ++j) r += md->Cdd[i * n + j];
    md->vs[i] = r;
    s += r;
  }
  if (!(s > 0.0)) return fail(QA_ERR_NOT_PD, "1^T Cdd 1 <= 0");
  for (int i = 0; i < n; ++i) md->vs[i] /= s;
  md->cond = norm1(n, md->Cdd) * norm1(n, md->M);
  md->status = 0;
  fill_consts(n, md);
  return QA_OK;
}

// Moore-Penrose pseudo-inverse of the m x k row-major A into the k x m
// row-major P, by one-sided Jacobi SVD (Hestenes 1958): plane rotations of
// the columns of W = A (accumulated in V) until every pair is orthogonal to
// working precision; then W = U S, A = U S V^T and
//     A^+ = sum_{s_j > tol} V e_j (W e_j)^T / s_j^2,
// with tol = max(m, k) eps max_j s_j (singular values below are treated as
// zero).  Host FP64; m, k <= 64.
void pinv(int m, int k, const double* A, double* P) {
  std::vector<double> W((size_t)m * k), V((size_t)k * k, 0.0);
  for (int e = 0; e < m * k; ++e) W[(size_t)e] = A[e];
  for (int j = 0; j < k; ++j) V[(size_t)j * k + j] = 1.0;
  const double eps = 2.220446049250313e-16;
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = 0; i < m; ++i) {
          const double wp = W[(size_t)i * k + p], wq = W[(size_t)i * k + q];
          a += wp * wp;
          b += wq * wq;
          c += wp * wq;
        }
        if (c == 0.0 || std::fabs(c) <= eps * std::sqrt(a * b)) continue;
        rotated = true;
        const double zeta = (b - a) / (2.0 * c);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int i = 0; i < m; ++i) {
          const double wp = W[(size_t)i * k + p], wq = W[(size_t)i * k + q];
          W[(size_t)i * k + p] = cs * wp - sn * wq;
          W[(size_t)i * k + q] = sn * wp + cs * wq;
        }
        for (int i = 0; i < k; ++i) {
          const double vp = V[(size_t)i * k + p], vq = V[(size_t)i * k + q];
          V[(size_t)i * k + p] = cs * vp - sn * vq;
          V[(size_t)i * k + q] = sn * vp + cs * vq;
        }
      }
    if (!rotated) break;
  }
  std::vector<double> s2((size_t)k, 0.0);
  double smax = 0.0;
  for (int j = 0; j < k; ++j) {
    double a = 0.0;
    for (int i = 0; i < m; ++i) a += W[(size_t)i * k + j] * W[(size_t)i * k + j];
    s2[(size_t)j] = a;
    smax = std::fmax(smax, std::sqrt(a));
  }
  const double tol = (double)std::max(m, k) * eps * smax;
  for (int e = 0; e < k * m; ++e) P[e] = 0.0;
  for (int j = 0; j < k; ++j) {
    if (!(std::sqrt(s2[(size_t)j]) > tol)) continue;
    for (int r = 0; r < k; ++r) {
      const double vr = V[(size_t)r * k + j] / s2[(size_t)j];
      for (int i = 0; i < m; ++i) P[(size_t)r * m + i] += vr * W[(size_t)i * k + j];
    }
  }
}

int ensure_workspace(qa_model* m, size_t bytes) {
  if (bytes <= m->ws_bytes) return QA_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  if (m->ws) cudaFree(m->ws);
  m->ws = nullptr;
  m->ws_bytes = 0;
  m->soft_recs.valid = false;
  const size_t want = bytes + bytes / 2 + (1u << 20);
  e = cudaMalloc(&m->ws, want);
  if (e != cudaSuccess) return fail(QA_ERR_NOMEM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
  m->ws_bytes = want;
  // the counters open the workspace; a ground-state call expects its list
  // heads at zero
  e = cudaMemset(m->ws, 0, sizeof(qa::Counters));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "workspace counters");
  return QA_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device id check: every call runs on the model's device.
int select_device(const qa_model* m) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != m->device) {
    e = cudaSetDevice(m->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  }
  return QA_OK;
}

qa::SearchCfg choose_cfg(int n, double t, long long P, int num_sms, bool closed) {
  const double kexp = (t >= 1.0) ? (double)n : (double)n * std::log2(1.0 + t);
  // closed arrays below t = 1 double t for the pixels whose candidate set
  // misses the total charge, and those pixels can reach every dot ambiguous:
  // they get a split whose outer states cover 2^9 candidates (the 16-dot
  // diagram at t = 0 took 2.4 ms with the 4 + 0 split the expected count picks)
  const int ke0 = (int)std::ceil(kexp - 1e-9);
  const int ke = (closed && t < 1.0) ? std::max(ke0, std::min(n, 10)) : ke0;
  qa::SearchCfg c;
  if (n <= 2) c = {2, 0, 1};
  else if (ke <= 4) c = {4, 0, 1};
  else if (ke <= 7) c = {4, 3, 1};
  else if (ke >= 15) {
    // nearly every dot ambiguous among 15 or 16: the pruned search, 16-lane
    // teams (two pixels per warp), 32 on rasters too small to fill the GPU
    // (below that the exhaustive search costs less than the pruned search's
    // fixed per-pixel set-up: measured on 128 x 128 rasters of 10 to 16 dots)
    c = {qa::kBnbL1, qa::kBnbL2, qa::kBnbMinT};
    if (P * c.T < (long long)num_sms * 128 * 4) c.T = 32;
    return c;
  } else {
    c = {5, 4, 1};
    const int rest = ke - 9;
    // two pixels per warp at most: a 16-lane team halves the per-pixel
    // set-up, merge and finish per warp against a 32-lane one, and small
    // rasters are widened below
    c.T = rest <= 0 ? 1 : (rest >= 4 ? 16 : (1 << rest));
  }
  // small rasters of many dots: a pixel's slot tables, finish and energy are
  // spread over its team's lanes, so four lanes at least even where the walk
  // leaves some of them idle (16-dot 100 x 100 diagram at t = 0.25, split
  // 4 + 3: 1, 2, 4, 16 lanes 105, 48, 36, 39 us; at t = 0.5 four lanes are
  // the widening below anyway)
  if (n >= 12 && c.T < 4 && P * 4 < (long long)num_sms * 128 * 4) c.T = 4;
  // spread a small raster over more lanes while each lane keeps >= 2 outer
  // states of work at the expected ambiguous count (>= 1 below t = 1, where
  // the count varies from pixel to pixel and the pixels above it set the
  // time: 4-lane teams instead of 2 on the 16-dot diagram at t = 0.5, 0.049
  // -> 0.043 ms)
  const int spare = ke - c.L1 - c.L2;
  const int keep = t < 1.0 ? 1 : 4;
  while (c.T < 32 && P * c.T < (long long)num_sms * 128 * 4 && spare > 0 &&
         (1 << spare) >= keep * c.T)
    c.T *= 2;
  return c;
}

// c0 = s Cgd (V0 + x0 u + y0 w), du = s Cgd u dx, dw = s Cgd w dy in FP64 on
// the host, split into double-float; only when the host copy is current.
qa::RasterK raster_constants(const qa_model* m, const qa::Scan& sc) {
  qa::RasterK rk;
  std::memset(&rk, 0, sizeof(rk));
  if (sc.kind != 0 || m->host_stale) return rk;
  const int n = m->n, ng = m->ng;
  for (int i = 0; i < n; ++i) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int g = 0; g < ng; ++g) {
      const double G = m->carrier * m->host.Cgd[i * ng + g];
      a += G * (sc.V0[g] + sc.x0 * sc.u[g] + sc.y0 * sc.w[g]);
      b += G * (sc.u[g] * sc.dx);
      c += G * (sc.w[g] * sc.dy);
    }
    rk.c0[i] = split(a);
    rk.du[i] = split(b);
    rk.dw[i] = split(c);
  }
  rk.valid = 1;
  return rk;
}

int prep_team(int n) {
  int t = 1;
  while (t < n) t <<= 1;
  return t;
}

struct ScanIn {
  const qa_raster* r = nullptr;
  const double* V = nullptr;
  long long P = 0;
};

int make_scan(const qa_model* m, const ScanIn& in, qa::Scan* sc) {
  std::memset(sc, 0, sizeof(*sc));
  if (in.r) {
    const qa_raster* r = in.r;
    if (!r->V0 || !r->u || !r->w) return fail(QA_ERR_INVALID, "raster vectors must be non-null");
    if (r->W < 1 || r->H < 1 || (long long)r->W * r->H > 2147483647LL)
      return fail(QA_ERR_SHAPE, "raster %d x %d out of range", r->W, r->H);
    if (!std::isfinite(r->x0) || !std::isfinite(r->x1) || !std::isfinite(r->y0) ||
        !std::isfinite(r->y1) || !finite_all(r->V0, m->ng) || !finite_all(r->u, m->ng) ||
        !finite_all(r->w, m->ng))
      return fail(QA_ERR_INVALID, "non-finite raster");
    sc->kind = 0;
    sc->W = r->W;
    sc->H = r->H;
    sc->P = (long long)r->W * r->H;
    sc->x0 = r->x0;
    sc->dx = r->W > 1 ? (r->x1 - r->x0) / (double)(r->W - 1) : 0.0;
    sc->y0 = r->y0;
    sc->dy = r->H > 1 ? (r->y1 - r->y0) / (double)(r->H - 1) : 0.0;
    for (int g = 0; g < m->ng; ++g) {
      sc->V0[g] = r->V0[g];
      sc->u[g] = r->u[g];
      sc->w[g] = r->w[g];
    }
  } else {
    if (in.P < 0 || in.P > 2147483647LL) return fail(QA_ERR_SHAPE, "P=%lld out of range", in.P);
    if (in.P > 0 && !in.V) return fail(QA_ERR_INVALID, "null voltage list");
    sc->kind = 1;
    sc->P = in.P;
    sc->V = in.V;
  }
  return QA_OK;
}

// Brute force (Table I): every state of the box (open) or every composition
// of N_hat (closed), FP64, one warp per pixel.
int run_brute(qa_model* m, const qa_raster* r, int closed, int bound, int8_t* out_n,
              double* out_U, uint8_t* out_flags, void* stream) {
  if (!m) return fail(QA_ERR_INVALID, "null model");
  if (!r) return fail(QA_ERR_INVALID, "null raster");
  if (bound < 0 || bound > 127)
    return fail(QA_ERR_RANGE, "%s=%d outside [0, 127]", closed ? "n_charges" : "n_max", bound);
  ScanIn in;
  in.r = r;
  qa::Scan sc;
  int rc = make_scan(m, in, &sc);
  if (rc) return rc;
  if (!out_n) return fail(QA_ERR_INVALID, "null out_n");
  const int R = bound + 1;
  const int nfree = closed ? m->n - 1 : m->n;
  double states = 1.0;
  for (int j = 0; j < nfree; ++j) states *= (double)R;
  if (states > 1099511627776.0)  // 2^40 per pixel
    return fail(QA_ERR_RANGE, "%d^%d brute-force states per pixel is too many", R, nfree);
  int ni = 0;
  double outer = states;
  while (ni < nfree && outer / R >= 32.0) { outer /= R; ++ni; }
  if ((rc = select_device(m))) return rc;
  qa::BruteLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.a.md = m->d_md;
  L.a.n = m->n;
  L.a.ng = m->ng;
  L.a.sc = sc;
  L.a.mt.t = 1.0;
  L.a.mt.closed = closed ? 1 : 0;
  L.a.mt.n_charges = closed ? bound : 0;
  L.a.mt.carrier = m->carrier;
  L.a.out_n = out_n;
  L.a.out_U = out_U;
  L.a.out_flags = out_flags;
  L.radix = R;
  L.nfree = nfree;
  L.ni = ni;
  L.n_max = closed ? -1 : bound;
  L.nouter = (unsigned long long)(outer + 0.5);
  cudaError_t e = qa::launch_brute(L, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "brute-force launch");
  return QA_OK;
}

int run_ground_state(qa_model* m, const ScanIn& in, double t, int closed,
                     int n_charges, int8_t* out_n, double* out_U,
                     uint8_t* out_flags, void* stream, int16_t* out_n16 = nullptr) {
  if (!m) return fail(QA_ERR_INVALID, "null model");
  if (!(t >= 0.0 && t <= 1.0)) return fail(QA_ERR_RANGE, "threshold %g outside [0, 1]", t);
  if (closed && (n_charges < 0 || n_charges > 100000))
    return fail(QA_ERR_RANGE, "n_charges=%d out of range", n_charges);
  qa::Scan sc;
  int rc = make_scan(m, in, &sc);
  if (rc) return rc;
  if (sc.P > 0 && !out_n && !out_n16) return fail(QA_ERR_INVALID, "null out_n");
  if ((rc = select_device(m))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const long long P = sc.P;
  const size_t Pn = (size_t)(P > 0 ? P : 1);
  const size_t nbp = (size_t)P + 1, nbs = (size_t)P + 1;  // >= block counts
  const size_t off_list = align_up(sizeof(qa::Counters), 256);
  const size_t off_tie = align_up(off_list + sizeof(qa::ListEntry) * Pn, 256);
  const size_t off_bcp = align_up(off_tie + sizeof(qa::ListEntry) * Pn, 256);
  const size_t off_bcs = align_up(off_bcp + sizeof(qa::BlockCounts) * nbp, 256);
  const size_t off_recs = align_up(off_bcs + sizeof(qa::BlockCounts) * nbs, 256);
  const size_t total = off_recs + sizeof(qa::PixRec) * Pn;
  if ((rc = ensure_workspace(m, total))) return rc;
  char* ws = (char*)m->ws;
  m->soft_recs.valid = false;  // this call's records replace any soft prep's
  m->d_cnt = (qa::Counters*)ws;
  m->last_P = P;
  m->n_bc_prep = m->n_bc_search = 0;
  m->d_bc_prep = (qa::BlockCounts*)(ws + off_bcp);
  m->d_bc_search = (qa::BlockCounts*)(ws + off_bcs);
  if (P == 0) {
    cudaError_t e0 = cudaMemsetAsync(m->d_cnt, 0, sizeof(qa::Counters), st);
    if (e0 != cudaSuccess) return cuda_fail(e0, "cudaMemsetAsync");
    return QA_OK;
  }
  cudaError_t e;

  qa::GsLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.one.md = m->d_md;
  a.one.n = m->n;
  a.one.ng = m->ng;
  a.one.sc = sc;
  a.one.mt.t = t;
  a.one.mt.closed = closed ? 1 : 0;
  a.one.mt.n_charges = closed ? n_charges : 0;
  a.one.mt.carrier = m->carrier;
  a.one.cfg = choose_cfg(m->n, t, P, m->num_sms, closed);
  a.one.klass = qa::search_klass(a.one.cfg);
  a.one.prep_team = prep_team(m->n);
  a.one.rk = raster_constants(m, sc);
  a.one.bx_analytic = 4.0e-7f;
  a.one.bx_qp_scale = 0.f;  // derived from the device model's condition number
  a.one.recs = (qa::PixRec*)(ws + off_recs);
  a.flag_list = (qa::ListEntry*)(ws + off_list);
  a.tie_list = (qa::ListEntry*)(ws + off_tie);
  a.bc_prep = m->d_bc_prep;
  a.bc_search = m->d_bc_search;
  a.cnt = m->d_cnt;
  a.one.out_n = out_n;
  a.one.out_n16 = out_n16;
  a.one.out_U = out_U;
  a.one.out_flags = out_flags;
  a.num_sms = m->num_sms;
  m->last_cfg = a.one.cfg;
  m->last_P = P;
  a.ev = m->timing ? m->ev : nullptr;
  m->last_kind = 1;
  m->n_bc_prep = qa::fused_tiles(a) ? qa::search_blocks(a) : qa::prep_blocks(a);
  m->n_bc_search = qa::search_blocks(a);
  e = qa::launch_ground_state(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "ground-state launch");
  return QA_OK;
}

// the fit step's extra arguments (qa_fit_step)
struct FitArgs {
  const float* target;
  int per_dot;
  float* loss;
  double* Cdd;
  double* Cgd;
  double* state;
  qa_adam opt;
};

int run_soft(qa_model* m, const qa_raster* r, double kT, double t, int closed,
             int n_charges, float* out_mean, float* out_logZ,
             const float* grad_mean, double* dCdd, double* dCgd, void* stream,
             uint2* ctx_out = nullptr, const uint2* ctx_in = nullptr,
             const float* mean_in = nullptr, const FitArgs* fit = nullptr) {
  const bool bwd = grad_mean != nullptr || fit != nullptr;
  if (!m) return fail(QA_ERR_INVALID, "null model");
  if (!r) return fail(QA_ERR_INVALID, "null raster");
  if (!(kT > 0.0) || !std::isfinite(kT)) return fail(QA_ERR_RANGE, "kT=%g must be > 0", kT);
  if (!(t >= 0.0 && t <= 1.0)) return fail(QA_ERR_RANGE, "threshold %g outside [0, 1]", t);
  if (closed && (n_charges < 0 || n_charges > 100000))
    return fail(QA_ERR_RANGE, "n_charges=%d out of range", n_charges);
  if (!bwd && !out_mean) return fail(QA_ERR_INVALID, "null out_mean");
  if (bwd && !fit && (!dCdd || !dCgd)) return fail(QA_ERR_INVALID, "null gradient output");
  ScanIn in;
  in.r = r;
  qa::Scan sc;
  int rc = make_scan(m, in, &sc);
  if (rc) return rc;
  if ((rc = select_device(m))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const long long P = sc.P;
  qa::SearchCfg cfg;
  if (m->n <= 8) cfg = {5, 4, 8};  // the dense form: teams of 8 lanes
  else cfg = {5, 4, 32};
  const size_t off_list = align_up(sizeof(qa::Counters), 256);
  const size_t off_bcp = align_up(off_list + sizeof(qa::ListEntry) * (size_t)P, 256);
  const size_t off_recs = align_up(off_bcp + sizeof(qa::BlockCounts) * ((size_t)P + 1), 256);
  const size_t off_part = align_up(off_recs + sizeof(qa::PixRec) * (size_t)P, 256);
  const size_t off_sums =
      align_up(off_part + (bwd ? sizeof(float) * qa::soft_partials_floats(m->n, P, cfg) : 0), 256);
  const size_t total = off_sums + (bwd ? sizeof(double) * (size_t)(qa::kMaxDot * qa::kMaxDot + 3 * qa::kMaxDot) : 0);
  if ((rc = ensure_workspace(m, total))) return rc;
  char* ws = (char*)m->ws;
  m->d_cnt = (qa::Counters*)ws;
  m->d_bc_prep = (qa::BlockCounts*)(ws + off_bcp);
  m->n_bc_search = 0;
  cudaError_t e;

  qa::GsLaunch g;
  std::memset(&g, 0, sizeof(g));
  g.one.md = m->d_md;
  g.one.n = m->n;
  g.one.ng = m->ng;
  g.one.sc = sc;
  g.one.mt.t = t;
  g.one.mt.closed = closed ? 1 : 0;
  g.one.mt.n_charges = closed ? n_charges : 0;
  g.one.mt.carrier = m->carrier;
  g.one.cfg = cfg;
  g.one.klass = qa::search_klass(cfg);
  g.one.prep_team = prep_team(m->n);
  g.one.rk = raster_constants(m, sc);
  g.one.bx_analytic = 4.0e-7f;
  g.one.recs = (qa::PixRec*)(ws + off_recs);
  g.flag_list = (qa::ListEntry*)(ws + off_list);
  g.bc_prep = m->d_bc_prep;
  g.cnt = m->d_cnt;
  g.num_sms = m->num_sms;
  if (m->timing) cudaEventRecord(m->ev[0], st);
  // the backward with the forward's context skips the prep when the records
  // of that forward (same model generation, raster and method) are in place
  const bool same_recs = m->soft_recs.valid && m->soft_recs.recs == (const void*)g.one.recs &&
                         std::memcmp(&m->soft_recs.sc, &sc, sizeof(sc)) == 0 &&
                         m->soft_recs.t == t && m->soft_recs.closed == (closed ? 1 : 0) &&
                         m->soft_recs.n_charges == g.one.mt.n_charges && m->soft_recs.gen == m->gen;
  if (!(bwd && ctx_in && same_recs)) {
    m->n_bc_prep = qa::prep_blocks(g);
    e = qa::launch_prep(g, st);
    if (e != cudaSuccess) return cuda_fail(e, "prep launch");
    m->soft_recs.valid = true;
    m->soft_recs.recs = g.one.recs;
    m->soft_recs.sc = sc;
    m->soft_recs.t = t;
    m->soft_recs.closed = closed ? 1 : 0;
    m->soft_recs.n_charges = g.one.mt.n_charges;
    m->soft_recs.gen = m->gen;
  }

  qa::SoftLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.md = m->d_md;
  a.n = m->n;
  a.ng = m->ng;
  a.sc = sc;
  a.mt = g.one.mt;
  a.cfg = cfg;
  a.kT = kT;
  a.recs = g.one.recs;
  a.cnt = m->d_cnt;
  a.out_mean = out_mean;
  a.out_logZ = out_logZ;
  a.grad_mean = grad_mean;
  a.ctx_out = ctx_out;
  a.ctx_in = ctx_in;
  a.mean_in = mean_in;
  a.partials = bwd ? (float*)(ws + off_part) : nullptr;
  a.sums = bwd ? (double*)(ws + off_sums) : nullptr;
  a.dL_dCdd = dCdd;
  a.dL_dCgd = dCgd;
  a.num_sms = m->num_sms;
  if (fit) {
    const double terms = (double)P * (fit->per_dot ? m->n : 1);
    a.fit_target = fit->target;
    a.fit_per_dot = fit->per_dot ? 1 : 0;
    a.fit_scale = (float)(2.0 / terms);
    a.fit_inv_count = 1.0 / terms;
    a.loss_out = fit->loss;
    a.fit_Cdd = fit->Cdd;
    a.fit_Cgd = fit->Cgd;
    a.fit_state = fit->state;
    a.lr = fit->opt.lr;
    a.beta1 = fit->opt.beta1;
    a.beta2 = fit->opt.beta2;
    a.eps = fit->opt.eps;
  }
  m->last_cfg = cfg;
  m->last_P = P;
  a.ev = m->timing ? m->ev + 4 : nullptr;
  m->last_kind = 2;
  e = bwd ? qa::launch_soft_backward(a, st) : qa::launch_soft_forward(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "soft launch");
  return QA_OK;
}

}  // namespace

extern "C" {

const char* qa_last_error(void) { return g_err.c_str(); }

int qa_model_create(const double* Cdd, const double* Cgd, int n_dot, int n_gate,
                    int form, double carrier_sign, qa_model** out) {
  if (!out) return fail(QA_ERR_INVALID, "null out");
  *out = nullptr;
  if (!(carrier_sign == 1.0 || carrier_sign == -1.0))
    return fail(QA_ERR_INVALID, "carrier_sign must be +1 or -1");
  qa_model* m = new qa_model();
  int rc = build_model(n_dot, n_gate, form, Cdd, Cgd, &m->host);
  if (rc) { delete m; return rc; }
  m->n = n_dot;
  m->ng = n_gate;
  m->form = form;
  m->carrier = carrier_sign;
  cudaError_t e = cudaGetDevice(&m->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_md, sizeof(qa::ModelData));
  if (e == cudaSuccess)
    e = cudaMemcpy(m->d_md, &m->host, sizeof(qa::ModelData), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (m->d_md) cudaFree(m->d_md);
    delete m;
    return cuda_fail(e, "model upload");
  }
  *out = m;
  return QA_OK;
}

int qa_model_update(qa_model* m, const double* Cdd, const double* Cgd) {
  if (!m) return fail(QA_ERR_INVALID, "null model");
  qa::ModelData md;
  int rc = build_model(m->n, m->ng, m->form, Cdd, Cgd, &md);
  if (rc) return rc;
  if ((rc = select_device(m))) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(m->d_md, &md, sizeof(qa::ModelData), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "model update");
  m->host = md;
  m->host_stale = false;
  ++m->gen;
  return QA_OK;
}

int qa_model_update_async(qa_model* m, const double* Cdd, const double* Cgd, void* stream) {
  if (!m) return fail(QA_ERR_INVALID, "null model");
  int rc = select_device(m);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (!m->staging) {
    e = cudaMallocHost(&m->staging, sizeof(qa::ModelData));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->staged, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "staging buffer");
  } else {
    e = cudaEventSynchronize(m->staged);  // the previous copy has left the buffer
    if (e != cudaSuccess) return cuda_fail(e, "staging buffer");
  }
  if ((rc = build_model(m->n, m->ng, m->form, Cdd, Cgd, m->staging))) return rc;
  e = cudaMemcpyAsync(m->d_md, m->staging, sizeof(qa::ModelData), cudaMemcpyHostToDevice,
                      (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaEventRecord(m->staged, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "model update");
  m->host = *m->staging;
  m->host_stale = false;
  ++m->gen;
  return QA_OK;
}

int qa_model_update_dev(qa_model* m, const double* Cdd_dev, const double* Cgd_dev,
                        void* stream) {
  if (!m || !Cdd_dev || !Cgd_dev) return fail(QA_ERR_INVALID, "null argument");
  int rc = select_device(m);
  if (rc) return rc;
  cudaError_t e = qa::launch_model_update(m->d_md, m->n, m->ng, Cdd_dev, Cgd_dev,
                                          (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "model update launch");
  m->host_stale = true;
  ++m->gen;
  return QA_OK;
}

int qa_model_destroy(qa_model* m) {
  if (!m) return QA_OK;
  select_device(m);
  cudaDeviceSynchronize();
  if (m->ws) cudaFree(m->ws);
  if (m->d_md) cudaFree(m->d_md);
  if (m->staging) cudaFreeHost(m->staging);
  if (m->staged) cudaEventDestroy(m->staged);
  for (cudaEvent_t& e : m->ev)
    if (e) cudaEventDestroy(e);
  delete m;
  return QA_OK;
}

int qa_model_set_timing(qa_model* m, int enable) {
  if (!m) return fail(QA_ERR_INVALID, "null model");
  int rc = select_device(m);
  if (rc) return rc;
  if (enable && !m->ev[0]) {
    for (cudaEvent_t& e : m->ev) {
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return cuda_fail(err, "cudaEventCreate");
    }
  }
  m->timing = enable != 0;
  return QA_OK;
}

int qa_model_shape(const qa_model* m, int* n_dot, int* n_gate) {
  if (!m) return fail(QA_ERR_INVALID, "null model");
  if (n_dot) *n_dot = m->n;
  if (n_gate) *n_gate = m->ng;
  return QA_OK;
}

int qa_model_get(const qa_model* m, double* Cdd, double* M, double* Cgd) {
  if (!m) return fail(QA_ERR_INVALID, "null model");
  qa::ModelData md;
  int rc = select_device(m);
  if (rc) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&md, m->d_md, sizeof(md), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "model read");
  const int n = m->n, ng = m->ng;
  if (Cdd) std::memcpy(Cdd, md.Cdd, sizeof(double) * n * n);
  if (M) std::memcpy(M, md.M, sizeof(double) * n * n);
  if (Cgd) std::memcpy(Cgd, md.Cgd, sizeof(double) * n * ng);
  if (md.status != 0) return fail(QA_ERR_NOT_PD, "device update: Cdd is not positive definite");
  return QA_OK;
}

int qa_ground_state_open(qa_model* m, const qa_raster* r, double threshold,
                         int8_t* out_n, double* out_U, uint8_t* out_flags,
                         void* stream) {
  if (!r) return fail(QA_ERR_INVALID, "null raster");
  ScanIn in;
  in.r = r;
  return run_ground_state(m, in, threshold, 0, 0, out_n, out_U, out_flags, stream);
}

int qa_ground_state_closed(qa_model* m, const qa_raster* r, double threshold,
                           int n_charges, int8_t* out_n, double* out_U,
                           uint8_t* out_flags, void* stream) {
  if (!r) return fail(QA_ERR_INVALID, "null raster");
  ScanIn in;
  in.r = r;
  return run_ground_state(m, in, threshold, 1, n_charges, out_n, out_U, out_flags,
                          stream);
}

int qa_ground_state_i16(qa_model* m, const qa_raster* r, double threshold, int closed,
                        int n_charges, int16_t* out_n, double* out_U, uint8_t* out_flags,
                        void* stream) {
  if (!r) return fail(QA_ERR_INVALID, "null raster");
  if (!out_n) return fail(QA_ERR_INVALID, "null out_n");
  ScanIn in;
  in.r = r;
  return run_ground_state(m, in, threshold, closed ? 1 : 0, n_charges, nullptr, out_U,
                          out_flags, stream, out_n);
}

int qa_ground_state_points(qa_model* m, const double* V_dev, long long P,
                           double threshold, int closed, int n_charges,
                           int8_t* out_n, double* out_U, uint8_t* out_flags,
                           void* stream) {
  ScanIn in;
  in.V = V_dev;
  in.P = P;
  return run_ground_state(m, in, threshold, closed ? 1 : 0, n_charges, out_n, out_U,
                          out_flags, stream);
}

int qa_optimal_gate_voltages(const double* Cdd, const double* Cgd, int n_dot, int n_gate,
                             int form, double carrier_sign, const double* Q, double* V) {
  if (!Q || !V) return fail(QA_ERR_INVALID, "null Q or V");
  if (!(carrier_sign == 1.0 || carrier_sign == -1.0))
    return fail(QA_ERR_INVALID, "carrier_sign must be +1 or -1");
  std::unique_ptr<qa::ModelData> md(new qa::ModelData());
  int rc = build_model(n_dot, n_gate, form, Cdd, Cgd, md.get());
  if (rc) return rc;
  const int n = n_dot, ng = n_gate;
  // R upper triangular with R^T R = M: R^T is the Cholesky factor of M
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = md->M[j * n + j];
    for (int q = 0; q < j; ++q) d -= L[(size_t)j * n + q] * L[(size_t)j * n + q];
    if (!(d > 0.0)) return fail(QA_ERR_NOT_PD, "Cdd^-1 is not positive definite");
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double e = md->M[i * n + j];
      for (int q = 0; q < j; ++q) e -= L[(size_t)i * n + q] * L[(size_t)j * n + q];
      L[(size_t)i * n + j] = e / ljj;
    }
  }
  std::vector<double> A((size_t)n * ng, 0.0), b((size_t)n, 0.0), P((size_t)ng * n);
  for (int i = 0; i < n; ++i) {   // (R A)_ig = sum_j L_ji Cgd_jg, (R Q)_i = sum_j L_ji Q_j
    for (int j = i; j < n; ++j) {
      const double rij = L[(size_t)j * n + i];
      for (int g = 0; g < ng; ++g) A[(size_t)i * ng + g] += rij * md->Cgd[j * ng + g];
      b[(size_t)i] += rij * Q[j];
    }
  }
  pinv(n, ng, A.data(), P.data());
  for (int g = 0; g < ng; ++g) {
    double v = 0.0;
    for (int i = 0; i < n; ++i) v += P[(size_t)g * n + i] * b[(size_t)i];
    V[g] = carrier_sign * v;
  }
  return QA_OK;
}

int qa_virtual_gate_matrix(const double* Cdd, const double* Cgd, int n_dot, int n_gate,
                           int form, double* alpha) {
  if (!alpha) return fail(QA_ERR_INVALID, "null alpha");
  std::unique_ptr<qa::ModelData> md(new qa::ModelData());
  int rc = build_model(n_dot, n_gate, form, Cdd, Cgd, md.get());
  if (rc) return rc;
  const int n = n_dot, ng = n_gate;
  std::vector<double> A((size_t)n * ng, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int g = 0; g < ng; ++g) A[(size_t)i * ng + g] += md->M[i * n + j] * md->Cgd[j * ng + g];
  pinv(n, ng, A.data(), alpha);
  return QA_OK;
}

int qa_charge_sensor(qa_model* m, const qa_raster* r, const int8_t* n_dots,
                     const qa_sensor_params* sp, float* out_signal, int8_t* out_n_sensor,
                     double* out_potential, void* stream) {
  if (!m || !r || !sp) return fail(QA_ERR_INVALID, "null argument");
  if (sp->n_sensor < 1 || sp->n_sensor > 4 || sp->n_sensor >= m->n)
    return fail(QA_ERR_RANGE, "n_sensor=%d outside [1, min(4, n_dot - 1)]", sp->n_sensor);
  if (sp->shape != QA_SENSOR_LORENTZIAN && sp->shape != QA_SENSOR_GAUSSIAN)
    return fail(QA_ERR_INVALID, "unknown sensor shape %d", sp->shape);
  if (!(sp->width > 0.0) || !(sp->white_sigma >= 0.0) || !(sp->pink_sigma >= 0.0) ||
      !std::isfinite(sp->width) || !std::isfinite(sp->white_sigma) ||
      !std::isfinite(sp->pink_sigma) || !std::isfinite(sp->jump_amplitude))
    return fail(QA_ERR_RANGE, "sensor width must be > 0 and noise levels >= 0");
  if (!(sp->jump_prob >= 0.0 && sp->jump_prob < 1.0))
    return fail(QA_ERR_RANGE, "jump_prob %g outside [0, 1)", sp->jump_prob);
  ScanIn in;
  in.r = r;
  qa::Scan sc;
  int rc = make_scan(m, in, &sc);
  if (rc) return rc;
  if (sc.W > 8192) return fail(QA_ERR_SHAPE, "sensor rasters hold at most 8192 columns");
  if (!n_dots || !out_signal) return fail(QA_ERR_INVALID, "null n_dots or out_signal");
  if ((rc = select_device(m))) return rc;
  qa::SensorLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.a.md = m->d_md;
  L.a.n = m->n;
  L.a.ng = m->ng;
  L.a.sc = sc;
  L.a.mt.carrier = m->carrier;
  L.S = sp->n_sensor;
  L.shape = sp->shape;
  L.K = 1;
  while ((1 << (L.K - 1)) < sc.W) ++L.K;
  L.width = sp->width;
  L.white_sigma = sp->white_sigma;
  L.pink_sigma = sp->pink_sigma;
  L.jump_amplitude = sp->jump_amplitude;
  L.jump_prob = sp->jump_prob;
  L.seed = sp->seed;
  L.n_dots = n_dots;
  L.out_signal = out_signal;
  L.out_n_sensor = out_n_sensor;
  L.out_potential = out_potential;
  cudaError_t e = qa::launch_sensor(L, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sensor launch");
  return QA_OK;
}

int qa_brute_force_open(qa_model* m, const qa_raster* r, int n_max, int8_t* out_n,
                        double* out_U, uint8_t* out_flags, void* stream) {
  return run_brute(m, r, 0, n_max, out_n, out_U, out_flags, stream);
}

int qa_brute_force_closed(qa_model* m, const qa_raster* r, int n_charges, int8_t* out_n,
                          double* out_U, uint8_t* out_flags, void* stream) {
  return run_brute(m, r, 1, n_charges, out_n, out_U, out_flags, stream);
}

int qa_soft_occupation(qa_model* m, const qa_raster* r, double kT,
                       double threshold, int closed, int n_charges,
                       float* out_mean, float* out_logZ, void* stream) {
  return run_soft(m, r, kT, threshold, closed, n_charges, out_mean, out_logZ,
                  nullptr, nullptr, nullptr, stream);
}

int qa_soft_occupation_backward(qa_model* m, const qa_raster* r, double kT,
                                double threshold, int closed, int n_charges,
                                const float* grad_mean, double* dL_dCdd,
                                double* dL_dCgd, void* stream) {
  if (!grad_mean) return fail(QA_ERR_INVALID, "null grad_mean");
  return run_soft(m, r, kT, threshold, closed, n_charges, nullptr, nullptr,
                  grad_mean, dL_dCdd, dL_dCgd, stream);
}

int qa_soft_occupation_ctx(qa_model* m, const qa_raster* r, double kT, double threshold,
                           int closed, int n_charges, float* out_mean, float* out_logZ,
                           void* out_ctx, void* stream) {
  if (!out_ctx) return fail(QA_ERR_INVALID, "null out_ctx");
  return run_soft(m, r, kT, threshold, closed, n_charges, out_mean, out_logZ, nullptr,
                  nullptr, nullptr, stream, (uint2*)out_ctx);
}

int qa_soft_occupation_backward_ctx(qa_model* m, const qa_raster* r, double kT,
                                    double threshold, int closed, int n_charges,
                                    const float* grad_mean, const float* mean,
                                    const void* ctx, double* dL_dCdd, double* dL_dCgd,
                                    void* stream) {
  if (!grad_mean || !mean || !ctx) return fail(QA_ERR_INVALID, "null grad_mean, mean or ctx");
  return run_soft(m, r, kT, threshold, closed, n_charges, nullptr, nullptr, grad_mean,
                  dL_dCdd, dL_dCgd, stream, nullptr, (const uint2*)ctx, mean);
}

int qa_fit_step(qa_model* m, const qa_raster* r, double kT, double threshold, int closed,
                int n_charges, const float* target, int per_dot, double* Cdd, double* Cgd,
                double* opt_state, const qa_adam* opt, float* loss, double* dL_dCdd,
                double* dL_dCgd, float* out_mean, void* stream) {
  if (!m || !r || !target || !Cdd || !Cgd || !opt_state || !opt)
    return fail(QA_ERR_INVALID, "null argument");
  if (!(opt->lr > 0.0) || !std::isfinite(opt->lr))
    return fail(QA_ERR_RANGE, "Adam lr=%g must be > 0", opt->lr);
  if (!(opt->beta1 >= 0.0 && opt->beta1 < 1.0) || !(opt->beta2 >= 0.0 && opt->beta2 < 1.0))
    return fail(QA_ERR_RANGE, "Adam betas (%g, %g) outside [0, 1)", opt->beta1, opt->beta2);
  if (!(opt->eps > 0.0) || !std::isfinite(opt->eps))
    return fail(QA_ERR_RANGE, "Adam eps=%g must be > 0", opt->eps);
  if (!(kT > 0.0) || !std::isfinite(kT)) return fail(QA_ERR_RANGE, "kT=%g must be > 0", kT);
  int rc = select_device(m);
  if (rc) return rc;
  cudaError_t e = qa::launch_model_update(m->d_md, m->n, m->ng, Cdd, Cgd, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "model update launch");
  m->host_stale = true;
  ++m->gen;
  FitArgs f{target, per_dot ? 1 : 0, loss, Cdd, Cgd, opt_state, *opt};
  return run_soft(m, r, kT, threshold, closed, n_charges, out_mean, nullptr, nullptr, dL_dCdd,
                  dL_dCgd, stream, nullptr, nullptr, nullptr, &f);
}

int qa_model_stats(qa_model* m, void* stream, qa_stats* out) {
  if (!m || !out) return fail(QA_ERR_INVALID, "null argument");
  std::memset(out, 0, sizeof(*out));
  int rc = select_device(m);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (!m->d_cnt) return QA_OK;
  qa::Counters c;
  e = cudaMemcpy(&c, m->d_cnt, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "counters read");
  // per-block counters: summed here, in block order
  std::vector<qa::BlockCounts> bc;
  if (m->n_bc_prep > 0) {
    bc.resize((size_t)m->n_bc_prep);
    e = cudaMemcpy(bc.data(), m->d_bc_prep, sizeof(qa::BlockCounts) * bc.size(),
                   cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "block counters read");
    for (const auto& b : bc) {
      c.candidates += b.candidates;
      c.qp += b.qp;
      c.doubled += b.doubled;
    }
  }
  if (m->n_bc_search > 0) {
    bc.resize((size_t)m->n_bc_search);
    e = cudaMemcpy(bc.data(), m->d_bc_search, sizeof(qa::BlockCounts) * bc.size(),
                   cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "block counters read");
    for (const auto& b : bc) {
      c.evaluated += b.evaluated;
      c.near_tie += b.near_tie;
      c.boundary += b.boundary;
      c.overflow += b.overflow;
    }
  }
  c.flagged = c.near_tie + c.boundary;
  out->candidates = (long long)c.candidates;
  out->evaluated = (long long)c.evaluated;
  out->qp_pixels = (long long)c.qp;
  out->flagged = (long long)c.flagged;
  out->near_tie = (long long)c.near_tie;
  out->boundary = (long long)c.boundary;
  out->unresolved = (long long)c.unresolved;
  out->overflow = (long long)c.overflow;
  out->doubled = (long long)c.doubled;
  out->shortlist_max = (long long)c.shortlist_max;
  out->resolved = (long long)c.resolved;
  out->pixels = m->last_P;
  if (m->timing && m->last_kind != 0) {
    float t0 = 0.f, t1 = 0.f, t2 = 0.f;
    if (m->last_kind == 1 &&
        cudaEventElapsedTime(&t0, m->ev[0], m->ev[1]) == cudaSuccess &&
        cudaEventElapsedTime(&t1, m->ev[1], m->ev[2]) == cudaSuccess &&
        cudaEventElapsedTime(&t2, m->ev[2], m->ev[3]) == cudaSuccess) {
      out->timed = 1;
      out->ms_prep = t0;
      out->ms_search = t1;
      out->ms_recheck = t2;
    } else if (m->last_kind == 2 &&
               cudaEventElapsedTime(&t0, m->ev[0], m->ev[4]) == cudaSuccess &&
               cudaEventElapsedTime(&t1, m->ev[4], m->ev[5]) == cudaSuccess) {
      out->timed = 1;
      out->ms_prep = t0;
      out->ms_soft = t1;
    }
  }
  out->team = m->last_cfg.T;
  out->inner_bits = m->last_cfg.L1;
  out->middle_bits = m->last_cfg.L2;
  return QA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// qa_ground_state_open_static: the open ground-state call for callers that
// must not allocate GPU memory while they run (see include/qarray.h).  Its
// scratch -- the per-pixel records, the recheck lists and the counters that
// qa_ground_state_open keeps in a cudaMalloc'd model workspace -- lives in
// the file-scope array below instead, sized for QA_STATIC_MAX_PIXELS pixels.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticPixels = (size_t)QA_STATIC_MAX_PIXELS;
constexpr size_t al256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kStOffList = al256(sizeof(qa::Counters));
constexpr size_t kStOffTie = al256(kStOffList + sizeof(qa::ListEntry) * kStaticPixels);
constexpr size_t kStOffBcp = al256(kStOffTie + sizeof(qa::ListEntry) * kStaticPixels);
constexpr size_t kStOffBcs = al256(kStOffBcp + sizeof(qa::BlockCounts) * (kStaticPixels + 1));
constexpr size_t kStOffRecs = al256(kStOffBcs + sizeof(qa::BlockCounts) * (kStaticPixels + 1));
constexpr size_t kStaticBytes = al256(kStOffRecs + sizeof(qa::PixRec) * kStaticPixels);

// Device address of the array below, looked up once per device.
constexpr int kStaticMaxDevices = 64;
void* g_static_ptr[kStaticMaxDevices] = {};
std::mutex g_static_mu;

}  // namespace

// Scratch of qa_ground_state_open_static.  Every GPU that loads this library
// holds it (about 5.4 MB) until the process exits; all calls on a device share
// it, so calls that overlap on that device race.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

extern "C" int qa_ground_state_open_static(qa_model* m, const qa_raster* r,
                                           double threshold, int8_t* out_n,
                                           double* out_U, uint8_t* out_flags,
                                           void* stream) {
  if (!m) return fail(QA_ERR_INVALID, "null model");
  if (!r) return fail(QA_ERR_INVALID, "null raster");
  if (!(threshold >= 0.0 && threshold <= 1.0))
    return fail(QA_ERR_RANGE, "threshold %g outside [0, 1]", threshold);
  ScanIn in;
  in.r = r;
  qa::Scan sc;
  int rc = make_scan(m, in, &sc);
  if (rc) return rc;
  const long long P = sc.P;
  if (P > (long long)kStaticPixels)
    return fail(QA_ERR_SHAPE, "raster of %lld pixels exceeds the static scratch of %lld "
                "pixels (QA_STATIC_MAX_PIXELS); use qa_ground_state_open", P,
                (long long)kStaticPixels);
  if (!out_n) return fail(QA_ERR_INVALID, "null out_n");
  if ((rc = select_device(m))) return rc;

  // In host code g_static_scratch names a host-side stand-in, not device
  // memory: its device address comes from the runtime, once per device, with
  // that device current (this first call must precede any stream capture).
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (m->device < 0 || m->device >= kStaticMaxDevices)
      return fail(QA_ERR_INVALID, "device %d out of range", m->device);
    if (!g_static_ptr[m->device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
      g_static_ptr[m->device] = p;
    }
    base = g_static_ptr[m->device];
  }
  char* ws = (char*)base;
  cudaStream_t st = (cudaStream_t)stream;
  qa::Counters* cnt = (qa::Counters*)ws;
  // the list counters must start at zero on every call (the array keeps the
  // last call's contents); the records and block counts are overwritten
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(qa::Counters), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if (P == 0) return QA_OK;

  qa::GsLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.one.md = m->d_md;
  a.one.n = m->n;
  a.one.ng = m->ng;
  a.one.sc = sc;
  a.one.mt.t = threshold;
  a.one.mt.closed = 0;
  a.one.mt.n_charges = 0;
  a.one.mt.carrier = m->carrier;
  a.one.cfg = choose_cfg(m->n, threshold, P, m->num_sms, false);
  a.one.klass = qa::search_klass(a.one.cfg);
  a.one.prep_team = prep_team(m->n);
  a.one.rk = raster_constants(m, sc);
  a.one.bx_analytic = 4.0e-7f;
  a.one.bx_qp_scale = 0.f;
  a.one.recs = (qa::PixRec*)(ws + kStOffRecs);
  a.flag_list = (qa::ListEntry*)(ws + kStOffList);
  a.tie_list = (qa::ListEntry*)(ws + kStOffTie);
  a.bc_prep = (qa::BlockCounts*)(ws + kStOffBcp);
  a.bc_search = (qa::BlockCounts*)(ws + kStOffBcs);
  a.cnt = cnt;
  a.one.out_n = out_n;
  a.one.out_U = out_U;
  a.one.out_flags = out_flags;
  a.num_sms = m->num_sms;
  a.ev = nullptr;
  e = qa::launch_ground_state(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "ground-state launch");
  return QA_OK;
}

// ---------------------------------------------------------------------------
// batched ground state
// ---------------------------------------------------------------------------
struct qa_batch {
  int device = 0, num_sms = 0, count = 0;
  long long pixels = 0;
  qa::GsLaunch L;
  void* mem = nullptr;  // one allocation: table, units, scratch
  std::vector<long long> P;
  std::vector<qa::SearchCfg> cfg;
};

namespace {

// Estimated candidate evaluations per pixel of an array (for unit sizing and
// the largest-first order).
double unit_cost(const qa::ArrayDesc& d) {
  const double kexp = d.mt.t >= 1.0 ? d.n : d.n * std::log2(1.0 + d.mt.t);
  return std::pow(2.0, kexp) + 64.0;
}

}  // namespace

extern "C" {

int qa_batch_create(const qa_batch_item* items, int count, qa_batch** out) {
  if (!out) return fail(QA_ERR_INVALID, "null out");
  *out = nullptr;
  if (!items || count < 1) return fail(QA_ERR_SHAPE, "empty batch");
  qa_batch* b = new qa_batch();
  std::vector<qa::ArrayDesc> table((size_t)count);
  int rc = QA_OK;
  for (int i = 0; i < count && rc == QA_OK; ++i) {
    const qa_batch_item& it = items[i];
    qa_model* m = it.model;
    if (!m) { rc = fail(QA_ERR_INVALID, "item %d: null model", i); break; }
    if (i == 0) { b->device = m->device; b->num_sms = m->num_sms; }
    if (m->device != b->device) { rc = fail(QA_ERR_SHAPE, "item %d: models on different devices", i); break; }
    if (!(it.threshold >= 0.0 && it.threshold <= 1.0)) { rc = fail(QA_ERR_RANGE, "item %d: threshold %g", i, it.threshold); break; }
    if (it.closed && (it.n_charges < 0 || it.n_charges > 100000)) { rc = fail(QA_ERR_RANGE, "item %d: n_charges %d", i, it.n_charges); break; }
    if (it.team != 0 && (it.team < 1 || it.team > 32 || (it.team & (it.team - 1)))) { rc = fail(QA_ERR_RANGE, "item %d: team %d", i, it.team); break; }
    ScanIn in;
    in.r = &it.raster;
    qa::Scan sc;
    if ((rc = make_scan(m, in, &sc))) break;
    if (!it.out_n) { rc = fail(QA_ERR_INVALID, "item %d: null out_n", i); break; }
    qa::ArrayDesc& d = table[(size_t)i];
    std::memset(&d, 0, sizeof(d));
    d.md = m->d_md;
    d.n = m->n;
    d.ng = m->ng;
    d.sc = sc;
    d.rk = raster_constants(m, sc);
    d.mt.t = it.threshold;
    d.mt.closed = it.closed ? 1 : 0;
    d.mt.n_charges = it.closed ? it.n_charges : 0;
    d.mt.carrier = m->carrier;
    d.cfg = choose_cfg(m->n, it.threshold, 1LL << 40, m->num_sms,
                       it.closed != 0);  // no small-raster spreading
    if (it.team) d.cfg.T = it.team;
    // the pruned search needs teams of kBnbMinT lanes or more
    if (qa::bnb_search(d.cfg.L1, d.cfg.L2) && d.cfg.T < qa::kBnbMinT)
      d.cfg.T = qa::kBnbMinT;
    d.klass = qa::search_klass(d.cfg);
    d.prep_team = prep_team(m->n);
    d.bx_analytic = 4.0e-7f;
    d.bx_qp_scale = 0.f;
    d.out_n = it.out_n;
    d.out_U = it.out_U;
    d.out_flags = it.out_flags;
    b->P.push_back(sc.P);
    b->cfg.push_back(d.cfg);
    b->pixels += sc.P;
  }
  if (rc) { delete b; return rc; }
  b->count = count;
  // work units, sized so that the persistent grids get several units per
  // block however the pixels are spread over the arrays: prep in runs of at
  // most 4096 pixels, search in runs of about an equal share of the total
  // candidate work (2^14 to 2^18 evaluations, at most 64 tiles), largest first
  if ((rc = select_device(items[0].model))) { delete b; return rc; }
  int pps = 1, sps = 1;
  qa::batch_occupancy(&pps, &sps);
  const double unit_target = 8.0;  // units per resident block
  double total_cost = 0.0;
  for (int i = 0; i < count; ++i) total_cost += unit_cost(table[(size_t)i]) * (double)b->P[(size_t)i];
  const long long prep_share =
      (long long)std::ceil((double)b->pixels / (unit_target * b->num_sms * pps));
  const double search_share =
      std::min(262144.0, std::max(16384.0, total_cost / (unit_target * b->num_sms * sps)));
  std::vector<qa::WorkUnit> pu, su;
  std::vector<double> scost;
  for (int i = 0; i < count; ++i) {
    const qa::ArrayDesc& d = table[(size_t)i];
    const long long P = b->P[(size_t)i];
    const long long tpb = 128 / d.prep_team;
    const long long pchunk = std::max(tpb, std::min(4096LL / tpb, (prep_share + tpb - 1) / tpb) * tpb);
    for (long long f = 0; f < P; f += pchunk)
      pu.push_back({i, (int)std::min(pchunk, P - f), f});
    const long long teams = 128 / d.cfg.T;
    const double c = unit_cost(d);
    long long k = (long long)std::max(1.0, std::floor(search_share / (c * (double)teams)));
    k = std::min(k, 64LL);
    const long long schunk = teams * k;
    for (long long f = 0; f < P; f += schunk) {
      const long long cnt = std::min(schunk, P - f);
      su.push_back({i, (int)cnt, f});
      scost.push_back(c * (double)cnt);
    }
  }
  // group the search units by kernel variant (4 klass + 2 closed + team
  // finish), largest first within a group; one persistent grid per variant
  auto variant = [&](const qa::WorkUnit& w) {
    const qa::ArrayDesc& d = table[(size_t)w.array];
    return 4 * d.klass + 2 * (d.mt.closed ? 1 : 0) + (d.cfg.T >= qa::kTeamFinishMin ? 1 : 0);
  };
  std::vector<size_t> order(su.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
    const int vx = variant(su[x]), vy = variant(su[y]);
    return vx != vy ? vx < vy : scost[x] > scost[y];
  });
  std::vector<qa::WorkUnit> su_sorted(su.size());
  for (size_t i = 0; i < order.size(); ++i) su_sorted[i] = su[order[i]];
  int var_first[qa::kBatchVariants] = {}, var_count[qa::kBatchVariants] = {},
      var_grid[qa::kBatchVariants] = {}, var_bc[qa::kBatchVariants] = {};
  for (size_t i = 0; i < su_sorted.size(); ++i) {
    const int v = variant(su_sorted[i]);
    if (var_count[v]++ == 0) var_first[v] = (int)i;
  }
  int grid_search = 0;
  for (int v = 0; v < qa::kBatchVariants; ++v) {
    if (!var_count[v]) continue;
    var_bc[v] = grid_search;
    var_grid[v] = std::min(var_count[v], b->num_sms * qa::batch_search_occupancy(v));
    grid_search += var_grid[v];
  }
  const int grid_prep = b->num_sms * pps;
  const size_t Ptot = (size_t)std::max(1LL, b->pixels);
  const size_t off_cnt = 0;
  const size_t off_tab = align_up(sizeof(qa::Counters), 256);
  const size_t off_pu = align_up(off_tab + sizeof(qa::ArrayDesc) * (size_t)count, 256);
  const size_t off_su = align_up(off_pu + sizeof(qa::WorkUnit) * pu.size(), 256);
  const size_t off_fl = align_up(off_su + sizeof(qa::WorkUnit) * su_sorted.size(), 256);
  const size_t off_tl = align_up(off_fl + sizeof(qa::ListEntry) * Ptot, 256);
  const size_t off_bcp = align_up(off_tl + sizeof(qa::ListEntry) * Ptot, 256);
  const size_t off_bcs = align_up(off_bcp + sizeof(qa::BlockCounts) * (size_t)grid_prep, 256);
  const size_t off_rec = align_up(off_bcs + sizeof(qa::BlockCounts) * (size_t)grid_search, 256);
  const size_t total = off_rec + sizeof(qa::PixRec) * Ptot;
  cudaError_t e = cudaMalloc(&b->mem, total);
  if (e != cudaSuccess) {
    delete b;
    return fail(QA_ERR_NOMEM, "batch scratch of %zu bytes: %s", total, cudaGetErrorString(e));
  }
  char* mem = (char*)b->mem;
  long long roff = 0;
  for (int i = 0; i < count; ++i) {
    table[(size_t)i].recs = (qa::PixRec*)(mem + off_rec) + roff;
    roff += b->P[(size_t)i];
  }
  e = cudaMemcpy(mem + off_tab, table.data(), sizeof(qa::ArrayDesc) * (size_t)count,
                 cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !pu.empty())
    e = cudaMemcpy(mem + off_pu, pu.data(), sizeof(qa::WorkUnit) * pu.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !su_sorted.empty())
    e = cudaMemcpy(mem + off_su, su_sorted.data(), sizeof(qa::WorkUnit) * su_sorted.size(),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(b->mem);
    delete b;
    return cuda_fail(e, "batch upload");
  }
  qa::GsLaunch& L = b->L;
  std::memset(&L, 0, sizeof(L));
  L.table = (const qa::ArrayDesc*)(mem + off_tab);
  L.prep_units = (const qa::WorkUnit*)(mem + off_pu);
  L.n_prep_units = (int)pu.size();
  L.search_units = (const qa::WorkUnit*)(mem + off_su);
  L.n_search_units = (int)su_sorted.size();
  L.flag_list = (qa::ListEntry*)(mem + off_fl);
  L.tie_list = (qa::ListEntry*)(mem + off_tl);
  L.cnt = (qa::Counters*)(mem + off_cnt);
  L.bc_prep = (qa::BlockCounts*)(mem + off_bcp);
  L.bc_search = (qa::BlockCounts*)(mem + off_bcs);
  L.grid_prep = grid_prep;
  L.grid_search = grid_search;
  for (int v = 0; v < qa::kBatchVariants; ++v) {
    L.var_first[v] = var_first[v];
    L.var_count[v] = var_count[v];
    L.var_grid[v] = var_grid[v];
    L.var_bc[v] = var_bc[v];
  }
  L.num_sms = b->num_sms;
  L.ev = nullptr;
  *out = b;
  return QA_OK;
}

int qa_batch_run(qa_batch* b, void* stream) {
  if (!b) return fail(QA_ERR_INVALID, "null batch");
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != b->device) e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return cuda_fail(e, "device");
  e = qa::launch_ground_state_batch(b->L, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return QA_OK;
}

int qa_batch_stats(qa_batch* b, void* stream, qa_stats* out) {
  if (!b || !out) return fail(QA_ERR_INVALID, "null argument");
  std::memset(out, 0, sizeof(*out));
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  qa::Counters c;
  if (e == cudaSuccess) e = cudaMemcpy(&c, b->L.cnt, sizeof(c), cudaMemcpyDeviceToHost);
  std::vector<qa::BlockCounts> bp((size_t)b->L.grid_prep), bs((size_t)b->L.grid_search);
  if (e == cudaSuccess)
    e = cudaMemcpy(bp.data(), b->L.bc_prep, sizeof(qa::BlockCounts) * bp.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(bs.data(), b->L.bc_search, sizeof(qa::BlockCounts) * bs.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "batch counters read");
  for (const auto& x : bp) { c.candidates += x.candidates; c.qp += x.qp; c.doubled += x.doubled; }
  for (const auto& x : bs) {
    c.evaluated += x.evaluated;
    c.near_tie += x.near_tie;
    c.boundary += x.boundary;
    c.overflow += x.overflow;
  }
  out->pixels = b->pixels;
  out->candidates = (long long)c.candidates;
  out->evaluated = (long long)c.evaluated;
  out->qp_pixels = (long long)c.qp;
  out->near_tie = (long long)c.near_tie;
  out->boundary = (long long)c.boundary;
  out->flagged = out->near_tie + out->boundary;
  out->unresolved = (long long)c.unresolved;
  out->overflow = (long long)c.overflow;
  out->doubled = (long long)c.doubled;
  out->shortlist_max = (long long)c.shortlist_max;
  out->resolved = (long long)c.resolved;
  return QA_OK;
}

int qa_batch_destroy(qa_batch* b) {
  if (!b) return QA_OK;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->mem) cudaFree(b->mem);
  delete b;
  return QA_OK;
}

}  // extern "C"
