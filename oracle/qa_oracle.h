/*
 * qa_oracle.h -- plain, slow, FP64 CPU oracle for the constant-capacitance-model
 * ground-state method of "QArray" (arXiv 2404.04994).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py use it.  It shares no code, header, table or
 * constant with the CUDA library in paper_2404_04994_gb300/csrc.
 *
 * Every routine follows the paper's own statement of the method, step by step,
 * in double precision, with direct (non-incremental) energy evaluation:
 *   Sec. II   (Eq. 1-2, Eq. "potential", Eq. "free_energy", Eq. "argmin"):
 *             Maxwell matrices, U(n) = 1/2 (n - c)^T Cdd^-1 (n - c), c = Cgd V.
 *   Sec. III.A: continuous minimum, analytic first (open: x = c;
 *             closed: Appendix D), numerical QP only if some x_i < 0.
 *   Sec. III.B: default (all floor/ceil) and thresholded candidate sets
 *             (Eq. "threshold"), closed-array filtering and threshold doubling.
 *   Sec. IV.B (Eq. "softargmin"): Boltzmann-weighted occupation.
 *   Table I:  brute-force enumeration over [0, n_max]^N.
 *
 * Readings of points where the paper is silent:
 *   - x_i is clamped to >= 0 before the floor; the pair of a dot is always
 *     {floor, floor + 1} (two distinct values, as Table I's 2^N count needs).
 *   - the threshold test is inclusive (<= t/2) as printed.
 *   - closed threshold doubling is done per pixel; t = 0 doubles to 1.
 *   - exact energy ties go to the lexicographically smallest n.
 *   - the QP is solved exactly by KKT active-set enumeration in order of
 *     increasing active-set size (the paper uses OSQP, an iterative solver).
 */
#ifndef QA_ORACLE_H
#define QA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define QO_MAX_DOT 16

/* A 2-D raster V(ix, iy) = V0 + xs[ix] * u + ys[iy] * w with
 * xs = linspace(x0, x1, W), ys = linspace(y0, y1, H); pixel p = iy * W + ix.
 * (the GateVoltageComposer meshgrid of Sec. V, generalised to virtual-gate
 * directions u, w). */
typedef struct {
    const double* V0;
    const double* u;
    const double* w;
    double x0, x1, y0, y1;
    int W, H;
} qo_raster;

/* Per-pixel result of the ground-state method. */
typedef struct {
    int    n[QO_MAX_DOT];   /* argmin charge configuration                  */
    double x[QO_MAX_DOT];   /* continuous minimum (Sec. III.A)              */
    double U;               /* U(n*)                                        */
    double U2;              /* runner-up energy in the candidate set        */
    double margin_floor;    /* min_i |x_i - round(x_i)| over x_i >= 1/2     */
    double margin_thresh;   /* min_i ||frac(x_i) - 1/2| - t/2| (t < 1)      */
    double t_used;          /* threshold after closed doubling              */
    double qp_cert;         /* KKT residual of the QP (0 when analytic)     */
    int    qp_used;         /* 1 when the analytic minimum was infeasible   */
    int    n_cand;          /* candidates evaluated                         */
    int    status;          /* 0 ok; < 0 failure                            */
} qo_pixel;

/* M = A^-1 for symmetric positive-definite A (Cholesky).  0 ok, -1 not PD. */
int qo_inverse_spd(int n, const double* A, double* Ainv);

/* U(n) = 1/2 (n - c)^T M (n - c)  (Eq. "free_energy" plus a constant). */
double qo_energy(int n, const double* M, const int* nvec, const double* c);

/* Continuous minimum (Sec. III.A): analytic form, else exact QP.
 * Returns 0 ok, -1 when no active set satisfies the KKT conditions. */
int qo_continuous_min(int n, const double* Cdd, const double* M, const double* c,
                      int closed, int n_charges, double* x, int* qp_used,
                      double* cert);

/* The whole method for one induced-charge vector c. */
int qo_ground_state_c(int n, const double* Cdd, const double* M, const double* c,
                      double t, int closed, int n_charges, qo_pixel* out);

/* c = carrier * Cgd . V(p) for raster pixel p. */
void qo_raster_c(int n_dot, int n_gate, const double* Cgd, double carrier,
                 const qo_raster* r, long p, double* c);

/* Ground state over pixels [p0, p1) of a raster (or of a point list when
 * r == NULL and V is a [P, n_gate] array).  Runs on n_threads host threads. */
int qo_ground_state(int n_dot, int n_gate, const double* Cdd, const double* Cgd,
                    double carrier, const qo_raster* r, const double* V,
                    long p0, long p1, double t, int closed, int n_charges,
                    int n_threads, qo_pixel* out);

/* Soft occupation (Sec. IV.B) over the candidate set of the method.
 * out_mean: [P, n_dot], out_logZ: [P].  Returns 0 ok. */
int qo_soft(int n_dot, int n_gate, const double* Cdd, const double* Cgd,
            double carrier, const qo_raster* r, const double* V,
            long p0, long p1, double kT, double t, int closed, int n_charges,
            int n_threads, double* out_mean, double* out_logZ);

/* Gradient of L through the soft occupation with the candidate set frozen.
 * grad_mean: dL/d<n>, [P, n_dot].  Outputs (accumulated over the pixels):
 * dL_dM [n_dot^2], dL_dCdd [n_dot^2] = -M dL_dM M, dL_dCgd [n_dot * n_gate].
 * Returns 0 ok. */
int qo_soft_grad(int n_dot, int n_gate, const double* Cdd, const double* Cgd,
                 double carrier, const qo_raster* r, const double* V,
                 long p0, long p1, double kT, double t, int closed,
                 int n_charges, const double* grad_mean, int n_threads,
                 double* dL_dM, double* dL_dCdd, double* dL_dCgd);

/* Brute force (Table I): open over [0, n_max]^N, closed over all
 * compositions with sum N_hat (visiting [0, N_hat]^N).  hit_nmax is set when
 * an open argmin touches n_max in some dot.  Returns the number of states
 * visited, (n_max + 1)^N or (N_hat + 1)^N, the count Table I quotes. */
long qo_brute_force(int n, const double* M, const double* c, int closed,
                    int n_charges, int n_max, int* out_n, double* out_U,
                    int* hit_nmax);

/* The same, also returning the second-lowest energy over the admissible
 * states (INFINITY when there is only one). */
long qo_brute_force2(int n, const double* M, const double* c, int closed,
                     int n_charges, int n_max, int* out_n, double* out_U,
                     double* out_U2, int* hit_nmax);

/* ------------------------------------------------------------------------ */
/* Charge sensors (Sec. IV.A)                                               */
/* ------------------------------------------------------------------------ */

/* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11): ten rounds of the
 * published round function (multipliers 0xD2511F53 and 0xCD9E8D57, key
 * schedule bumped by 0x9E3779B9 and 0xBB67AE85 between rounds). */
void qo_philox4x32_10(const unsigned* ctr, const unsigned* key, unsigned* out);

typedef struct {
    int n_sensor;             /* the last n_sensor dots of the model        */
    int shape;                /* 0 Lorentzian, 1 Gaussian                   */
    double width;             /* gamma > 0                                  */
    double white_sigma, pink_sigma, jump_amplitude, jump_prob;
    unsigned long long seed;
} qo_sensor_params;

/* Sensor response on every pixel of a raster (Sec. IV.A), given the dots'
 * ground state n_dots [P, n_full - S] (int):
 *   1. with the dots fixed, each sensor takes the charge minimising the full
 *      energy U: the best of the floor / floor + 1 values around the
 *      continuous sensor minimum x_S = c_S - (M_SS)^-1 M_SD (n_D - c_D)
 *      (2^S candidates, direct energies, lexicographic ties);
 *   2. the sensor potential V_S = (M (n - c))_S (Eq. "potential");
 *   3. the distance to the nearest Coulomb peak eps = M_ss / 2 - |V_s| and
 *      the line shape 1 / (1 + (eps / gamma)^2) or exp(-eps^2 / (2 gamma^2));
 *   4. noise: white (one normal deviate per pixel), 1/f along the fast axis
 *      (Voss-McCartney: octave k redrawn every 2^k pixels, K octaves with
 *      2^(K-1) >= W, sum / sqrt(K)) and a random telegraph of amplitude
 *      jump_amplitude switching with probability jump_prob per pixel
 *      (geometric gaps), all drawn from Philox4x32-10 with key = seed and
 *      counter (kind | sensor << 4 | octave << 8, row, index, 0); normals by
 *      Box-Muller from u1 = (x0 + 1) / 2^32, u2 = x1 / 2^32.
 * Outputs [P, S]: signal, sensor charges, potentials.  Returns 0, or -1 on
 * bad input. */
int qo_charge_sensor(int n_full, int n_gate, const double* Cdd_full,
                     const double* Cgd_full, double carrier, const qo_raster* r,
                     const int* n_dots, const qo_sensor_params* sp,
                     double* signal, int* n_sensor, double* potential);

#ifdef __cplusplus
}
#endif
#endif
