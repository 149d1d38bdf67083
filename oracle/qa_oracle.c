/*
 * qa_oracle.c -- FP64 CPU oracle (test infrastructure only; see qa_oracle.h).
 *
 * Plain and slow on purpose: every energy is evaluated directly from its
 * definition, every candidate is enumerated, the QP is solved by trying active
 * sets in order of size.  Compiled with -ffp-contract=off so that x86-64 and
 * aarch64 hosts give identical results.
 */
#include "qa_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define N QO_MAX_DOT

/* ------------------------------------------------------------------------ */
/* small dense linear algebra                                               */
/* ------------------------------------------------------------------------ */

/* Cholesky A = L L^T of an m x m SPD matrix (row-major, leading dim m).
 * Returns 0 on success, -1 if a pivot is not positive. */
static int cholesky(int m, const double* A, double* L)
{
    for (int i = 0; i < m * m; ++i) L[i] = 0.0;
    for (int j = 0; j < m; ++j) {
        double d = A[j * m + j];
        for (int k = 0; k < j; ++k) d -= L[j * m + k] * L[j * m + k];
        if (!(d > 0.0)) return -1;
        double ljj = sqrt(d);
        L[j * m + j] = ljj;
        for (int i = j + 1; i < m; ++i) {
            double s = A[i * m + j];
            for (int k = 0; k < j; ++k) s -= L[i * m + k] * L[j * m + k];
            L[i * m + j] = s / ljj;
        }
    }
    return 0;
}

/* Solve L L^T y = b. */
static void chol_solve(int m, const double* L, const double* b, double* y)
{
    double z[N];
    for (int i = 0; i < m; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * m + k] * z[k];
        z[i] = s / L[i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
        double s = z[i];
        for (int k = i + 1; k < m; ++k) s -= L[k * m + i] * y[k];
        y[i] = s / L[i * m + i];
    }
}

int qo_inverse_spd(int n, const double* A, double* Ainv)
{
    double L[N * N];
    if (n < 1 || n > N) return -1;
    if (cholesky(n, A, L) != 0) return -1;
    for (int j = 0; j < n; ++j) {
        double e[N] = {0}, col[N];
        e[j] = 1.0;
        chol_solve(n, L, e, col);
        for (int i = 0; i < n; ++i) Ainv[i * n + j] = col[i];
    }
    /* symmetrise the round-off */
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double s = 0.5 * (Ainv[i * n + j] + Ainv[j * n + i]);
            Ainv[i * n + j] = s;
            Ainv[j * n + i] = s;
        }
    return 0;
}

/* U(n) = 1/2 (n - c)^T M (n - c): Eq. "free_energy" with the n-independent
 * constant 1/2 c^T M c added back. */
double qo_energy(int n, const double* M, const int* nvec, const double* c)
{
    double r[N], U = 0.0;
    for (int i = 0; i < n; ++i) r[i] = (double)nvec[i] - c[i];
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += M[i * n + j] * r[j];
        U += r[i] * s;
    }
    return 0.5 * U;
}

/* ------------------------------------------------------------------------ */
/* continuous minimum (Sec. III.A)                                          */
/* ------------------------------------------------------------------------ */

/* Try one active set A (bit i set <=> x_i fixed at 0) for
 *   minimise 1/2 (x - c)^T M (x - c)  s.t.  x >= 0  [and 1^T x = Nhat].
 * KKT: M (x - c) = z + lambda 1, z >= 0, z_F = 0, x_A = 0, x_F >= 0.
 * Returns 1 and fills x, cert when the KKT conditions hold within tol. */
static int try_active_set(int n, const double* M, const double* c,
                          unsigned A, int closed, int n_charges, double tol,
                          double* x, double* cert)
{
    int F[N], nf = 0;
    for (int i = 0; i < n; ++i)
        if (!((A >> i) & 1u)) F[nf++] = i;

    double Mc[N];
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += M[i * n + j] * c[j];
        Mc[i] = s;
    }

    double xs[N] = {0};
    double lambda = 0.0;
    if (nf == 0) {
        if (closed && n_charges != 0) return 0;  /* sum x = 0 != Nhat */
        /* x = 0; with closed Nhat = 0 pick lambda so that z >= 0 */
        if (closed) {
            lambda = INFINITY;
            for (int i = 0; i < n; ++i)
                if (-Mc[i] < lambda) lambda = -Mc[i];
        }
    } else {
        double MFF[N * N], L[N * N], rhs[N], y1[N];
        for (int a = 0; a < nf; ++a) {
            for (int b = 0; b < nf; ++b) MFF[a * nf + b] = M[F[a] * n + F[b]];
            rhs[a] = Mc[F[a]];
        }
        if (cholesky(nf, MFF, L) != 0) return 0;
        chol_solve(nf, L, rhs, y1);                 /* M_FF x_F = (M c)_F */
        if (closed) {
            /* stationarity on F gives M_FF x_F = (Mc)_F + lambda 1; the sum
             * constraint fixes lambda (the Lagrangian of Appendix D with
             * x_A = 0). */
            double ones[N] = {0}, y2[N], s1 = 0.0, s2 = 0.0;
            for (int a = 0; a < nf; ++a) ones[a] = 1.0;
            chol_solve(nf, L, ones, y2);
            for (int a = 0; a < nf; ++a) { s1 += y1[a]; s2 += y2[a]; }
            lambda = ((double)n_charges - s1) / s2;
            for (int a = 0; a < nf; ++a) y1[a] += lambda * y2[a];
        }
        for (int a = 0; a < nf; ++a) xs[F[a]] = y1[a];
    }

    /* check primal feasibility and the multipliers of the active bounds */
    double res = 0.0;
    for (int i = 0; i < n; ++i) {
        double g = 0.0;
        for (int j = 0; j < n; ++j) g += M[i * n + j] * (xs[j] - c[j]);
        double zi = g - lambda;              /* multiplier of x_i >= 0 */
        if ((A >> i) & 1u) {
            if (zi < -tol) return 0;
            if (-zi > res) res = -zi;
        } else {
            if (xs[i] < -tol) return 0;
            if (fabs(zi) > res) res = fabs(zi);       /* stationarity on F */
            if (-xs[i] > res) res = -xs[i];
        }
    }
    for (int i = 0; i < n; ++i) x[i] = xs[i];
    *cert = res;
    return 1;
}

int qo_continuous_min(int n, const double* Cdd, const double* M, const double* c,
                      int closed, int n_charges, double* x, int* qp_used,
                      double* cert)
{
    /* analytic minimum: open x = c (Appendix C); closed
     * x = c + (Nhat - 1^T c) Cdd 1 / (1^T Cdd 1) (Appendix D). */
    if (!closed) {
        for (int i = 0; i < n; ++i) x[i] = c[i];
    } else {
        double Cdd1[N], s = 0.0, sc = 0.0;
        for (int i = 0; i < n; ++i) {
            double r = 0.0;
            for (int j = 0; j < n; ++j) r += Cdd[i * n + j];
            Cdd1[i] = r;
            s += r;
            sc += c[i];
        }
        for (int i = 0; i < n; ++i)
            x[i] = c[i] + ((double)n_charges - sc) * Cdd1[i] / s;
    }
    int feasible = 1;
    for (int i = 0; i < n; ++i)
        if (x[i] < 0.0) feasible = 0;
    *qp_used = 0;
    *cert = 0.0;
    if (feasible) return 0;

    /* numerical QP: exact KKT active-set enumeration, smallest sets first */
    *qp_used = 1;
    double cmax = 1.0, mmax = 1.0;
    for (int i = 0; i < n; ++i) {
        if (fabs(c[i]) > cmax) cmax = fabs(c[i]);
        for (int j = 0; j < n; ++j)
            if (fabs(M[i * n + j]) > mmax) mmax = fabs(M[i * n + j]);
    }
    double tol = 1e-11 * cmax * mmax;
    for (int size = 0; size <= n; ++size) {
        if (size == 0) {
            if (try_active_set(n, M, c, 0u, closed, n_charges, tol, x, cert)) return 0;
            continue;
        }
        /* all masks with popcount == size, increasing (Gosper's successor) */
        unsigned m = (1u << size) - 1u;
        unsigned lim = 1u << n;
        while (m < lim) {
            if (try_active_set(n, M, c, m, closed, n_charges, tol, x, cert)) return 0;
            unsigned lo = m & (0u - m);
            unsigned hi = m + lo;
            m = (((hi ^ m) >> 2) / lo) | hi;
        }
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* candidate set (Sec. III.B)                                               */
/* ------------------------------------------------------------------------ */

/* Default/thresholded neighbourhood of x.  amb[i] = 1 when both floor and
 * floor + 1 are candidates for dot i (Eq. "threshold"), else base[i] is the
 * rounding to the nearest integer. */
static void candidate_set(int n, const double* x, double t, int* base, int* amb,
                          double* margin_floor, double* margin_thresh)
{
    for (int i = 0; i < n; ++i) {
        double xi = x[i] > 0.0 ? x[i] : 0.0;
        double fl = floor(xi);
        double fr = xi - fl;
        int a = fabs(fr - 0.5) <= 0.5 * t;
        amb[i] = a;
        base[i] = (int)fl + ((!a && fr >= 0.5) ? 1 : 0);
        if (xi >= 0.5) {
            double d = fabs(xi - floor(xi + 0.5));
            if (d < *margin_floor) *margin_floor = d;
        }
        if (t < 1.0) {
            double d = fabs(fabs(fr - 0.5) - 0.5 * t);
            if (d < *margin_thresh) *margin_thresh = d;
        }
    }
}

/* lexicographic order on charge vectors, for exact energy ties */
static int lex_less(int n, const int* a, const int* b)
{
    for (int i = 0; i < n; ++i)
        if (a[i] != b[i]) return a[i] < b[i];
    return 0;
}

typedef struct {
    int base[N];
    int slot[N];   /* dot index of each ambiguous slot, increasing */
    int k;         /* number of ambiguous dots */
    int w;         /* closed: number of slots taking floor + 1; open: -1 */
    double t_used, margin_floor, margin_thresh;
} cand_set;

static int build_candidates(int n, const double* x, double t, int closed,
                            int n_charges, cand_set* cs)
{
    cs->margin_floor = INFINITY;
    cs->margin_thresh = INFINITY;
    for (int iter = 0; iter < 64; ++iter) {
        int amb[N];
        candidate_set(n, x, t, cs->base, amb, &cs->margin_floor, &cs->margin_thresh);
        cs->k = 0;
        int sum = 0;
        for (int i = 0; i < n; ++i) {
            if (amb[i]) cs->slot[cs->k++] = i;
            sum += cs->base[i];
        }
        cs->t_used = t;
        if (!closed) { cs->w = -1; return 0; }
        cs->w = n_charges - sum;
        if (cs->w >= 0 && cs->w <= cs->k) return 0;
        if (t >= 1.0) return -1;
        /* no admissible candidate: double the threshold and recompute */
        t = (t <= 0.0) ? 1.0 : (2.0 * t < 1.0 ? 2.0 * t : 1.0);
    }
    return -1;
}

static int popcount_u(unsigned v)
{
    int s = 0;
    while (v) { s += (int)(v & 1u); v >>= 1; }
    return s;
}

static void candidate_vector(int n, const cand_set* cs, unsigned m, int* nv)
{
    for (int i = 0; i < N; ++i) nv[i] = i < n ? cs->base[i] : 0;
    for (int j = 0; j < cs->k; ++j)
        if ((m >> j) & 1u) nv[cs->slot[j]] += 1;
}

int qo_ground_state_c(int n, const double* Cdd, const double* M, const double* c,
                      double t, int closed, int n_charges, qo_pixel* out)
{
    memset(out, 0, sizeof(*out));
    int st = qo_continuous_min(n, Cdd, M, c, closed, n_charges, out->x,
                               &out->qp_used, &out->qp_cert);
    if (st != 0) { out->status = -1; return -1; }
    cand_set cs;
    if (build_candidates(n, out->x, t, closed, n_charges, &cs) != 0) {
        out->status = -2;
        return -2;
    }
    out->t_used = cs.t_used;
    out->margin_floor = cs.margin_floor;
    out->margin_thresh = cs.margin_thresh;

    double best = INFINITY, second = INFINITY;
    int nbest[N] = {0};
    int count = 0;
    unsigned total = 1u << cs.k;
    for (unsigned m = 0; m < total; ++m) {
        if (closed && popcount_u(m) != cs.w) continue;
        int nv[N];
        candidate_vector(n, &cs, m, nv);
        double U = qo_energy(n, M, nv, c);
        ++count;
        if (U < best || (U == best && lex_less(n, nv, nbest))) {
            if (count > 1) second = best < second ? best : second;
            best = U;
            memcpy(nbest, nv, sizeof(nbest));
        } else if (U < second) {
            second = U;
        }
    }
    memcpy(out->n, nbest, sizeof(nbest));
    out->U = best;
    out->U2 = second;
    out->n_cand = count;
    out->status = 0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* voltages                                                                 */
/* ------------------------------------------------------------------------ */

static double lin(double a, double b, int n, int i)
{
    return n > 1 ? a + (double)i * (b - a) / (double)(n - 1) : a;
}

static void pixel_c(int n_dot, int n_gate, const double* Cgd, double carrier,
                    const qo_raster* r, const double* V, long p, double* c)
{
    double Vp[256];
    if (r) {
        int ix = (int)(p % r->W), iy = (int)(p / r->W);
        double xs = lin(r->x0, r->x1, r->W, ix);
        double ys = lin(r->y0, r->y1, r->H, iy);
        for (int g = 0; g < n_gate; ++g)
            Vp[g] = r->V0[g] + xs * r->u[g] + ys * r->w[g];
    } else {
        for (int g = 0; g < n_gate; ++g) Vp[g] = V[p * n_gate + g];
    }
    for (int i = 0; i < n_dot; ++i) {
        double s = 0.0;
        for (int g = 0; g < n_gate; ++g) s += Cgd[i * n_gate + g] * Vp[g];
        c[i] = carrier * s;
    }
}

void qo_raster_c(int n_dot, int n_gate, const double* Cgd, double carrier,
                 const qo_raster* r, long p, double* c)
{
    pixel_c(n_dot, n_gate, Cgd, carrier, r, NULL, p, c);
}

static void pixel_voltage(int n_gate, const qo_raster* r, const double* V, long p,
                          double* Vp)
{
    if (r) {
        int ix = (int)(p % r->W), iy = (int)(p / r->W);
        double xs = lin(r->x0, r->x1, r->W, ix);
        double ys = lin(r->y0, r->y1, r->H, iy);
        for (int g = 0; g < n_gate; ++g)
            Vp[g] = r->V0[g] + xs * r->u[g] + ys * r->w[g];
    } else {
        for (int g = 0; g < n_gate; ++g) Vp[g] = V[p * n_gate + g];
    }
}

/* ------------------------------------------------------------------------ */
/* threaded drivers                                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    int kind;                  /* 0 ground state, 1 soft, 2 grad */
    int n_dot, n_gate;
    const double *Cdd, *M, *Cgd;
    double carrier;
    const qo_raster* r;
    const double* V;
    long p0, p1;
    long off;                  /* pixel index of out[0] / mean[0] / gbar[0] */
    double kT, t;
    int closed, n_charges;
    qo_pixel* out;
    double *mean, *logZ;
    const double* gbar;
    double dM[N * N];
    double dc0[N * 256];       /* per-thread sum of dL/dc_p V_p^T */
    int status;
} job;

/* Boltzmann weights over the method's candidate set for one pixel; fills the
 * mean occupation and log Z; when gbar != NULL accumulates the frozen-set
 * gradient into dM (N x N) and returns dL/dc in dc. */
static int soft_pixel(int n, const double* Cdd, const double* M, const double* c,
                      double kT, double t, int closed, int n_charges,
                      double* mean, double* logZ, const double* gbar,
                      double* dM, double* dc)
{
    double x[N], cert;
    int qp;
    if (qo_continuous_min(n, Cdd, M, c, closed, n_charges, x, &qp, &cert) != 0)
        return -1;
    cand_set cs;
    if (build_candidates(n, x, t, closed, n_charges, &cs) != 0) return -2;
    unsigned total = 1u << cs.k;
    double Umin = INFINITY;
    for (unsigned m = 0; m < total; ++m) {
        if (closed && popcount_u(m) != cs.w) continue;
        int nv[N];
        candidate_vector(n, &cs, m, nv);
        double U = qo_energy(n, M, nv, c);
        if (U < Umin) Umin = U;
    }
    double Z = 0.0, acc[N] = {0};
    for (unsigned m = 0; m < total; ++m) {
        if (closed && popcount_u(m) != cs.w) continue;
        int nv[N];
        candidate_vector(n, &cs, m, nv);
        double wgt = exp(-(qo_energy(n, M, nv, c) - Umin) / kT);
        Z += wgt;
        for (int i = 0; i < n; ++i) acc[i] += wgt * nv[i];
    }
    for (int i = 0; i < n; ++i) mean[i] = acc[i] / Z;
    *logZ = -Umin / kT + log(Z);
    if (!gbar) return 0;

    /* dL/dU_c = a_c = -(w_c / kT) (gbar . n_c - gbar . <n>), w_c normalised;
     * U_c = 1/2 r^T M r with r = n_c - c:  dU/dM = 1/2 r r^T, dU/dc = -M r. */
    double gm = 0.0;
    for (int i = 0; i < n; ++i) gm += gbar[i] * mean[i];
    double sr[N] = {0};
    for (unsigned m = 0; m < total; ++m) {
        if (closed && popcount_u(m) != cs.w) continue;
        int nv[N];
        candidate_vector(n, &cs, m, nv);
        double wgt = exp(-(qo_energy(n, M, nv, c) - Umin) / kT) / Z;
        double gn = 0.0;
        for (int i = 0; i < n; ++i) gn += gbar[i] * nv[i];
        double a = -(wgt / kT) * (gn - gm);
        double r[N];
        for (int i = 0; i < n; ++i) r[i] = nv[i] - c[i];
        for (int i = 0; i < n; ++i) {
            sr[i] += a * r[i];
            for (int j = 0; j < n; ++j) dM[i * n + j] += 0.5 * a * r[i] * r[j];
        }
    }
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += M[i * n + j] * sr[j];
        dc[i] = -s;
    }
    return 0;
}

static void* run_job(void* arg)
{
    job* jb = (job*)arg;
    int n = jb->n_dot;
    jb->status = 0;
    for (long p = jb->p0; p < jb->p1; ++p) {
        double c[N];
        pixel_c(n, jb->n_gate, jb->Cgd, jb->carrier, jb->r, jb->V, p, c);
        if (jb->kind == 0) {
            if (qo_ground_state_c(n, jb->Cdd, jb->M, c, jb->t, jb->closed,
                                  jb->n_charges, &jb->out[p - jb->off]) != 0)
                jb->status = -1;
        } else if (jb->kind == 1) {
            if (soft_pixel(n, jb->Cdd, jb->M, c, jb->kT, jb->t, jb->closed,
                           jb->n_charges, &jb->mean[(p - jb->off) * n],
                           &jb->logZ[p - jb->off],
                           NULL, NULL, NULL) != 0)
                jb->status = -1;
        } else {
            double mean[N], lz, dc[N], Vp[256];
            if (soft_pixel(n, jb->Cdd, jb->M, c, jb->kT, jb->t, jb->closed,
                           jb->n_charges, mean, &lz,
                           &jb->gbar[(p - jb->off) * n], jb->dM,
                           dc) != 0) {
                jb->status = -1;
                continue;
            }
            /* c = carrier Cgd V  =>  dL/dCgd += carrier dL/dc V^T */
            pixel_voltage(jb->n_gate, jb->r, jb->V, p, Vp);
            for (int i = 0; i < n; ++i)
                for (int g = 0; g < jb->n_gate; ++g)
                    jb->dc0[i * jb->n_gate + g] += jb->carrier * dc[i] * Vp[g];
        }
    }
    return NULL;
}

static int run_threads(job* proto, int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    long P = proto->p1 - proto->p0;
    if (P < n_threads) n_threads = P > 0 ? (int)P : 1;
    job* jobs = (job*)calloc((size_t)n_threads, sizeof(job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -3; }
    for (int k = 0; k < n_threads; ++k) {
        jobs[k] = *proto;
        memset(jobs[k].dM, 0, sizeof(jobs[k].dM));
        memset(jobs[k].dc0, 0, sizeof(jobs[k].dc0));
        jobs[k].p0 = proto->p0 + P * k / n_threads;
        jobs[k].p1 = proto->p0 + P * (k + 1) / n_threads;
    }
    for (int k = 1; k < n_threads; ++k)
        pthread_create(&th[k], NULL, run_job, &jobs[k]);
    run_job(&jobs[0]);
    for (int k = 1; k < n_threads; ++k) pthread_join(th[k], NULL);
    int status = 0;
    memset(proto->dM, 0, sizeof(proto->dM));
    memset(proto->dc0, 0, sizeof(proto->dc0));
    for (int k = 0; k < n_threads; ++k) {   /* fixed order: deterministic */
        if (jobs[k].status) status = jobs[k].status;
        for (int i = 0; i < N * N; ++i) proto->dM[i] += jobs[k].dM[i];
        for (int i = 0; i < N * 256; ++i) proto->dc0[i] += jobs[k].dc0[i];
    }
    free(jobs);
    free(th);
    return status;
}

static int setup(job* jb, int n_dot, int n_gate, const double* Cdd,
                 const double* Cgd, double carrier, const qo_raster* r,
                 const double* V, long p0, long p1, double* Mbuf)
{
    if (n_dot < 1 || n_dot > N || n_gate < 1 || n_gate > 256) return -1;
    if (qo_inverse_spd(n_dot, Cdd, Mbuf) != 0) return -2;
    memset(jb, 0, sizeof(*jb));
    jb->n_dot = n_dot;
    jb->n_gate = n_gate;
    jb->Cdd = Cdd;
    jb->M = Mbuf;
    jb->Cgd = Cgd;
    jb->carrier = carrier;
    jb->r = r;
    jb->V = V;
    jb->p0 = p0;
    jb->p1 = p1;
    jb->off = p0;
    return 0;
}

int qo_ground_state(int n_dot, int n_gate, const double* Cdd, const double* Cgd,
                    double carrier, const qo_raster* r, const double* V,
                    long p0, long p1, double t, int closed, int n_charges,
                    int n_threads, qo_pixel* out)
{
    static __thread job jb;
    double M[N * N];
    int st = setup(&jb, n_dot, n_gate, Cdd, Cgd, carrier, r, V, p0, p1, M);
    if (st) return st;
    jb.kind = 0;
    jb.t = t;
    jb.closed = closed;
    jb.n_charges = n_charges;
    jb.out = out;
    return run_threads(&jb, n_threads);
}

int qo_soft(int n_dot, int n_gate, const double* Cdd, const double* Cgd,
            double carrier, const qo_raster* r, const double* V,
            long p0, long p1, double kT, double t, int closed, int n_charges,
            int n_threads, double* out_mean, double* out_logZ)
{
    static __thread job jb;
    double M[N * N];
    int st = setup(&jb, n_dot, n_gate, Cdd, Cgd, carrier, r, V, p0, p1, M);
    if (st) return st;
    if (!(kT > 0.0)) return -1;
    jb.kind = 1;
    jb.kT = kT;
    jb.t = t;
    jb.closed = closed;
    jb.n_charges = n_charges;
    jb.mean = out_mean;
    jb.logZ = out_logZ;
    return run_threads(&jb, n_threads);
}

int qo_soft_grad(int n_dot, int n_gate, const double* Cdd, const double* Cgd,
                 double carrier, const qo_raster* r, const double* V,
                 long p0, long p1, double kT, double t, int closed,
                 int n_charges, const double* grad_mean, int n_threads,
                 double* dL_dM, double* dL_dCdd, double* dL_dCgd)
{
    static __thread job jb;
    double M[N * N];
    int st = setup(&jb, n_dot, n_gate, Cdd, Cgd, carrier, r, V, p0, p1, M);
    if (st) return st;
    if (!(kT > 0.0)) return -1;
    jb.kind = 2;
    jb.kT = kT;
    jb.t = t;
    jb.closed = closed;
    jb.n_charges = n_charges;
    jb.gbar = grad_mean;
    st = run_threads(&jb, n_threads);
    int n = n_dot;
    for (int i = 0; i < n * n; ++i) dL_dM[i] = jb.dM[i];
    /* M = Cdd^-1  =>  dL/dCdd = -M^T (dL/dM) M^T */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b)
                    s += M[a * n + i] * jb.dM[a * n + b] * M[j * n + b];
            dL_dCdd[i * n + j] = -s;
        }
    for (int i = 0; i < n * n_gate; ++i) dL_dCgd[i] = jb.dc0[i];
    return st;
}

/* ------------------------------------------------------------------------ */
/* brute force (Table I)                                                    */
/* ------------------------------------------------------------------------ */

long qo_brute_force(int n, const double* M, const double* c, int closed,
                    int n_charges, int n_max, int* out_n, double* out_U,
                    int* hit_nmax)
{
    double second;
    return qo_brute_force2(n, M, c, closed, n_charges, n_max, out_n, out_U,
                           &second, hit_nmax);
}

long qo_brute_force2(int n, const double* M, const double* c, int closed,
                     int n_charges, int n_max, int* out_n, double* out_U,
                     double* out_U2, int* hit_nmax)
{
    int hi = closed ? n_charges : n_max;
    int nv[N] = {0};
    double best = INFINITY, second = INFINITY;
    long count = 0;
    *hit_nmax = 0;
    for (;;) {
        int ok = 1;
        ++count;                 /* states visited: (hi + 1)^n in total */
        if (closed) {
            int s = 0;
            for (int i = 0; i < n; ++i) s += nv[i];
            ok = (s == n_charges);
        }
        if (ok) {
            double U = qo_energy(n, M, nv, c);
            if (U < best || (U == best && lex_less(n, nv, out_n))) {
                second = best;
                best = U;
                memcpy(out_n, nv, sizeof(int) * (size_t)n);
            } else if (U < second) {
                second = U;
            }
        }
        /* odometer over [0, hi]^n in lexicographic order */
        int i = n - 1;
        while (i >= 0 && nv[i] == hi) { nv[i] = 0; --i; }
        if (i < 0) break;
        ++nv[i];
    }
    *out_U = best;
    *out_U2 = second;
    if (!closed)
        for (int i = 0; i < n; ++i)
            if (out_n[i] == n_max) *hit_nmax = 1;
    return count;
}

/* ------------------------------------------------------------------------ */
/* Charge sensors (Sec. IV.A)                                               */
/* ------------------------------------------------------------------------ */

void qo_philox4x32_10(const unsigned* ctr, const unsigned* key, unsigned* out)
{
    unsigned c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    unsigned k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        unsigned n0 = (unsigned)(p1 >> 32) ^ c1 ^ k0;
        unsigned n1 = (unsigned)p1;
        unsigned n2 = (unsigned)(p0 >> 32) ^ c3 ^ k1;
        unsigned n3 = (unsigned)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void sensor_draw(unsigned long long seed, unsigned tag, unsigned row,
                        unsigned idx, unsigned* out)
{
    unsigned ctr[4] = {tag, row, idx, 0u};
    unsigned key[2] = {(unsigned)seed, (unsigned)(seed >> 32)};
    qo_philox4x32_10(ctr, key, out);
}

static double sensor_normal(unsigned long long seed, unsigned tag, unsigned row,
                            unsigned idx)
{
    unsigned x[4];
    sensor_draw(seed, tag, row, idx, x);
    double u1 = ((double)x[0] + 1.0) / 4294967296.0;
    double u2 = (double)x[1] / 4294967296.0;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
}

/* telegraph state (0/1) at every index < len of one row */
static void sensor_telegraph(unsigned long long seed, unsigned tag, unsigned row,
                             double prob, int len, unsigned char* state)
{
    for (int i = 0; i < len; ++i) state[i] = 0;
    if (!(prob > 0.0)) return;
    long pos = -1;
    unsigned j = 0;
    for (;;) {
        unsigned x[4];
        sensor_draw(seed, tag, row, j++, x);
        double u = ((double)x[0] + 1.0) / 4294967296.0;
        double g = prob >= 1.0 ? 1.0 : 1.0 + floor(log(u) / log(1.0 - prob));
        if (g > (double)len) break;
        pos += (long)g;
        if (pos >= len) break;
        for (long i = pos; i < len; ++i) state[i] ^= 1u;
    }
}

int qo_charge_sensor(int n_full, int n_gate, const double* Cdd_full,
                     const double* Cgd_full, double carrier, const qo_raster* r,
                     const int* n_dots, const qo_sensor_params* sp,
                     double* signal, int* n_sensor, double* potential)
{
    int S = sp->n_sensor, nd = n_full - S;
    if (S < 1 || S > 4 || nd < 1 || n_full > N || !(sp->width > 0.0)) return -1;
    if (!(sp->jump_prob >= 0.0 && sp->jump_prob < 1.0)) return -1;
    double M[N * N];
    if (qo_inverse_spd(n_full, Cdd_full, M)) return -1;
    /* (M_SS)^-1 */
    double Mss[16], Mssi[16];
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) Mss[a * S + b] = M[(nd + a) * n_full + nd + b];
    if (qo_inverse_spd(S, Mss, Mssi)) return -1;
    int K = 1;
    while ((1 << (K - 1)) < r->W) ++K;
    unsigned char* tel = (unsigned char*)malloc((size_t)r->W);
    long P = (long)r->W * r->H;
    for (int s = 0; s < S; ++s) {
        for (int row = 0; row < r->H; ++row) {
            sensor_telegraph(sp->seed, 2u | ((unsigned)s << 4), (unsigned)row, sp->jump_prob,
                             r->W, tel);
            for (int col = 0; col < r->W; ++col) {
                long p = (long)row * r->W + col;
                /* computed per sensor from scratch: steps 1-2 */
                double c[N];
                pixel_c(n_full, n_gate, Cgd_full, carrier, r, NULL, p, c);
                int nv[N];
                for (int i = 0; i < nd; ++i) nv[i] = n_dots[p * nd + i];
                double g[4], xs[4];
                for (int a = 0; a < S; ++a) {
                    double acc = 0.0;
                    for (int j = 0; j < nd; ++j)
                        acc += M[(nd + a) * n_full + j] * ((double)nv[j] - c[j]);
                    g[a] = acc;
                }
                for (int a = 0; a < S; ++a) {
                    double acc = 0.0;
                    for (int b = 0; b < S; ++b) acc += Mssi[a * S + b] * g[b];
                    xs[a] = c[nd + a] - acc;
                }
                int best[4] = {0, 0, 0, 0}, have = 0;
                double bestU = 0.0;
                for (int m = 0; m < (1 << S); ++m) {
                    int cand[N];
                    for (int i = 0; i < nd; ++i) cand[i] = nv[i];
                    for (int a = 0; a < S; ++a) {
                        double xa = xs[a] > 0.0 ? xs[a] : 0.0;
                        cand[nd + a] = (int)floor(xa) + ((m >> a) & 1);
                    }
                    double U = qo_energy(n_full, M, cand, c);
                    int better = !have || U < bestU;
                    if (have && U == bestU) {
                        int lt = 0;
                        for (int a = 0; a < S; ++a)
                            if (cand[nd + a] != best[a]) { lt = cand[nd + a] < best[a]; break; }
                        better = lt;
                    }
                    if (better) {
                        have = 1;
                        bestU = U;
                        for (int a = 0; a < S; ++a) best[a] = cand[nd + a];
                    }
                }
                for (int a = 0; a < S; ++a) nv[nd + a] = best[a];
                /* step 2: potential of sensor s */
                int q = nd + s;
                double V = 0.0;
                for (int j = 0; j < n_full; ++j) V += M[q * n_full + j] * ((double)nv[j] - c[j]);
                /* step 3: line shape */
                double eps = 0.5 * M[q * n_full + q] - fabs(V);
                double y = eps / sp->width;
                double resp = sp->shape == 1 ? exp(-0.5 * y * y) : 1.0 / (1.0 + y * y);
                /* step 4: noise */
                double noise = 0.0;
                if (sp->white_sigma > 0.0)
                    noise += sp->white_sigma *
                             sensor_normal(sp->seed, 0u | ((unsigned)s << 4), (unsigned)row, (unsigned)col);
                if (sp->pink_sigma > 0.0) {
                    double acc = 0.0;
                    for (int k = 0; k < K; ++k)
                        acc += sensor_normal(sp->seed, 1u | ((unsigned)s << 4) | ((unsigned)k << 8),
                                             (unsigned)row, (unsigned)col >> k);
                    noise += sp->pink_sigma * acc / sqrt((double)K);
                }
                if (tel[col]) noise += sp->jump_amplitude;
                signal[p * S + s] = resp + noise;
                n_sensor[p * S + s] = nv[q];
                potential[p * S + s] = V;
            }
        }
    }
    free(tel);
    return 0;
}
