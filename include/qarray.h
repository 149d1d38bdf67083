/*
 * qarray.h -- C ABI of libqarray.so, the GB300 (sm_103a) implementation of the
 * constant-capacitance-model ground-state method of "QArray" (arXiv 2404.04994).
 *
 * Problem (Sec. II): for dot-dot Maxwell block Cdd (N x N, symmetric positive
 * definite), gate-dot block Cgd (N x N_g) and gate voltages V, the charge
 * state of an open array is
 *     n* = argmin_{n in Z^N, n >= 0} U(n),  U(n) = 1/2 (n - c)^T Cdd^-1 (n - c),
 *     c = s * Cgd V   (s = +1, or -1 for the opposite carrier sign, Sec. II),
 * (Eq. "free_energy" plus the n-independent constant 1/2 c^T Cdd^-1 c), and a
 * closed array adds sum(n) = N_hat (constraint iii).  The method (Sec. III):
 * continuous minimum of the relaxed problem (analytic, else a QP with x >= 0),
 * then the argmin over the floor/floor+1 neighbours of that minimum, pruned by
 * the threshold t of Eq. "threshold" (t = 1 is the default algorithm, t < 1
 * the thresholded algorithm; a closed array whose pruned set holds no state
 * with the right total doubles t per pixel).
 *
 * Conventions shared by every call:
 *  - Return value: QA_OK (0) or a negative QA_ERR_* code; the message of the
 *    last failure on the calling thread is qa_last_error().  No call throws.
 *  - Host pointers are read during the call and never retained.  Device
 *    pointers (suffix _dev, or documented as device) must stay valid until the
 *    work enqueued on `stream` has completed; they are never freed here.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued asynchronously; errors detected on the host are returned
 *    before anything is enqueued.  Calls that share one model must not overlap
 *    on the GPU (the model owns one scratch workspace); use one model per
 *    concurrent stream.
 *  - Matrices are row-major FP64.  Charge maps are channel-last [H, W, N]
 *    (pixel p = iy * W + ix), the (100, 100, 2) layout of Sec. V.
 *  - Every call runs on the device that was current at qa_model_create.
 */
#ifndef QARRAY_H
#define QARRAY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QA_MAX_DOT 16
#define QA_MAX_GATE 64

enum {
    QA_OK = 0,
    QA_ERR_INVALID = -1,       /* null pointer, NaN/Inf input, bad enum      */
    QA_ERR_SHAPE = -2,         /* n_dot / n_gate / raster size out of range  */
    QA_ERR_NOT_SYMMETRIC = -3, /* |Cdd - Cdd^T| > 1e-12 max|Cdd|             */
    QA_ERR_NOT_PD = -4,        /* Cholesky of Cdd failed (Appendix B)         */
    QA_ERR_RANGE = -5,         /* threshold outside [0, 1], kT <= 0, N_hat<0  */
    QA_ERR_OVERFLOW = -6,      /* a charge does not fit the output type       */
    QA_ERR_CUDA = -7,          /* a CUDA runtime call failed                  */
    QA_ERR_TIMEOUT = -8,       /* a bounded device wait expired               */
    QA_ERR_NOMEM = -9,         /* workspace allocation failed                 */
    QA_ERR_UNRESOLVED = -10    /* a pixel the FP64 recheck could not settle   */
};

/* Input form of the capacitances (Sec. V, DotArray keyword arguments). */
enum {
    QA_FORM_MAXWELL = 0,  /* cdd, cgd: Maxwell blocks (lower-case in the paper) */
    QA_FORM_COUPLING = 1  /* Cdd, Cgd: non-negative couplings (upper-case);
                             converted by Appendix B: cdd_ii = sum of dot i's
                             couplings to dots and gates, cdd_ij = -C_ij,
                             cgd = Cgd (gate couplings are the induced charge
                             per volt). */
};

/* Per-pixel status bits written to out_flags (uint8 per pixel). */
enum {
    QA_FLAG_NEAR_TIE = 1,    /* FP32 best/runner-up gap under the error bound */
    QA_FLAG_BOUNDARY = 2,    /* continuous minimum within the error bound of a
                                floor or threshold decision                   */
    QA_FLAG_QP = 4,          /* analytic minimum infeasible: QP was solved    */
    QA_FLAG_QP_CAP = 8,      /* FP32 active-set iteration hit its cap          */
    QA_FLAG_RECHECKED = 16,  /* pixel re-evaluated in FP64                     */
    QA_FLAG_DOUBLED = 32,    /* closed threshold doubled at least once         */
    QA_FLAG_UNRESOLVED = 64, /* FP64 recheck could not settle the pixel        */
    QA_FLAG_OVERFLOW = 128   /* a charge exceeds the int8 output               */
};

typedef struct qa_model qa_model;

/* A 2-D gate-voltage raster (the meshgrid of Sec. V, with arbitrary virtual
 * gate directions):  V(ix, iy) = V0 + xs[ix] u + ys[iy] w,
 * xs = linspace(x0, x1, W), ys = linspace(y0, y1, H).  V0, u, w are HOST
 * arrays of length n_gate.  1 <= W, H and W * H <= 2^31 - 1. */
typedef struct {
    const double* V0;
    const double* u;
    const double* w;
    double x0, x1, y0, y1;
    int W, H;
} qa_raster;

/* Counters of the last ground-state / soft call on a model (read back with a
 * stream synchronisation by qa_model_stats). */
typedef struct {
    long long pixels;          /* pixels processed                            */
    long long candidates;      /* admissible candidates (2^k or C(k, w))      */
    long long evaluated;       /* candidate energies evaluated by the kernels */
    long long qp_pixels;       /* pixels that needed the QP                   */
    long long flagged;         /* pixels re-evaluated exactly: the two below  */
    long long near_tie;        /* FP32 top-two gap under the bound (resolve)  */
    long long boundary;        /* decision boundary / QP cap (FP64 recheck)   */
    long long unresolved;      /* pixels the recheck could not settle         */
    long long overflow;        /* pixels whose charges exceed int8            */
    long long doubled;         /* closed pixels whose threshold was doubled   */
    long long shortlist_max;   /* largest near-tie shortlist (blocks)         */
    long long resolved;        /* near ties settled by exact double-float    */
    int team;                  /* lanes per pixel used by the search kernel   */
    int inner_bits;            /* unrolled inner / middle bits of the search  */
    int middle_bits;
    int timed;                 /* 1 when the ms_* fields below are valid      */
    double ms_prep;            /* device time of each kernel of the last call */
    double ms_search;          /* (qa_model_set_timing)                       */
    double ms_recheck;
    double ms_soft;
} qa_stats;

/* Create a model from HOST matrices Cdd [n_dot x n_dot] and Cgd
 * [n_dot x n_gate] (copied).  Validates 1 <= n_dot <= 16, 1 <= n_gate <= 64,
 * finiteness, symmetry and positive definiteness (Appendix B; Sec. V
 * validation), computes M = Cdd^-1 in FP64 and uploads the model to the
 * current device.  carrier_sign = +1 (c = Cgd V) or -1 (c = -Cgd V, Q = +-eN,
 * Sec. II).  *out receives a handle owned by the caller (qa_model_destroy).
 * Errors: QA_ERR_INVALID, QA_ERR_SHAPE, QA_ERR_NOT_SYMMETRIC, QA_ERR_NOT_PD,
 * QA_ERR_CUDA, QA_ERR_NOMEM. */
int qa_model_create(const double* Cdd, const double* Cgd, int n_dot, int n_gate,
                    int form, double carrier_sign, qa_model** out);

/* Replace the capacitances of a model from HOST matrices (same shape and form
 * as at creation); same checks as qa_model_create.  Synchronous. */
int qa_model_update(qa_model* m, const double* Cdd, const double* Cgd);

/* The same, asynchronously on `stream`: the host checks and the FP64
 * Cholesky inverse run before the call returns (errors as qa_model_update),
 * the result is copied from the model's pinned staging buffer to the device
 * in stream order, so calls on `stream` after it see the new model.  Work on
 * other streams that reads the model must be ordered by the caller.  A second
 * update waits for the first one's copy to finish before reusing the staging
 * buffer. */
int qa_model_update_async(qa_model* m, const double* Cdd, const double* Cgd, void* stream);

/* Replace the capacitances from DEVICE FP64 Maxwell matrices (same shape) and
 * recompute M = Cdd^-1 on the GPU in FP64 (symmetric sweeps, i.e. Gauss-Jordan
 * on diagonal pivots), asynchronously on `stream`.  A non-positive pivot (Cdd
 * not positive definite) is recorded on the device; the next call that
 * reads the model on that stream writes QA_FLAG_UNRESOLVED for every pixel and
 * qa_model_stats reports it (host checks are impossible without a sync).
 * Used by the capacitance-fitting loop. */
int qa_model_update_dev(qa_model* m, const double* Cdd_dev,
                        const double* Cgd_dev, void* stream);

/* Release the model and its device memory (synchronises the device). */
int qa_model_destroy(qa_model* m);

/* Shape of a model: *n_dot, *n_gate (either may be NULL). */
int qa_model_shape(const qa_model* m, int* n_dot, int* n_gate);

/* Copy the model's current FP64 Cdd, M = Cdd^-1 and Cgd to HOST arrays (any
 * may be NULL); synchronises the device. */
int qa_model_get(const qa_model* m, double* Cdd, double* M, double* Cgd);

/* Ground state of an OPEN array on every raster pixel (Sec. III, constraints
 * i-ii).  threshold t in [0, 1] (Eq. "threshold"; 1 = default algorithm).
 * DEVICE outputs, caller-owned:
 *   out_n     int8  [H, W, n_dot]  charge configuration n*;
 *   out_U     FP64  [H, W]         U(n*) (nullable);
 *   out_flags uint8 [H, W]         QA_FLAG_* bits (nullable).
 * Errors: QA_ERR_INVALID, QA_ERR_SHAPE, QA_ERR_RANGE, QA_ERR_CUDA,
 * QA_ERR_NOMEM.  Charges above 127 saturate and set QA_FLAG_OVERFLOW. */
int qa_ground_state_open(qa_model* m, const qa_raster* r, double threshold,
                         int8_t* out_n, double* out_U, uint8_t* out_flags,
                         void* stream);

/* Ground state of a CLOSED array holding n_charges carriers (constraint iii;
 * Appendix D continuous minimum; per-pixel threshold doubling of Sec. III.B).
 * Outputs as qa_ground_state_open.  n_charges >= 0, else QA_ERR_RANGE. */
int qa_ground_state_closed(qa_model* m, const qa_raster* r, double threshold,
                           int n_charges, int8_t* out_n, double* out_U,
                           uint8_t* out_flags, void* stream);

/* Ground state of an open (closed = 0) or closed (closed = 1, n_charges
 * carriers) array with an int16 charge map out_n [H, W, n_dot] (DEVICE,
 * caller-owned), for scans whose charges exceed int8; charges above 32767
 * saturate and set QA_FLAG_OVERFLOW.  Otherwise as qa_ground_state_open /
 * qa_ground_state_closed. */
int qa_ground_state_i16(qa_model* m, const qa_raster* r, double threshold, int closed,
                        int n_charges, int16_t* out_n, double* out_U, uint8_t* out_flags,
                        void* stream);

/* Ground state at an arbitrary list of P gate-voltage vectors V_dev (DEVICE,
 * FP64 [P, n_gate]), the random-voltage workload of Sec. VII.  closed = 0/1.
 * Outputs as above with H * W replaced by P. */
int qa_ground_state_points(qa_model* m, const double* V_dev, long long P,
                           double threshold, int closed, int n_charges,
                           int8_t* out_n, double* out_U, uint8_t* out_flags,
                           void* stream);

/* Optimal gate voltages for a charge state (Sec. IV.C, Eq.
 * "optimal_gate_voltages"; proof in Appendix H): the V that minimises
 * 1/2 (Q - s Cgd V)^T Cdd^-1 (Q - s Cgd V), i.e. the least-squares problem
 * min ||R Q - s R Cgd V||_2 with R^T R = Cdd^-1 (Cholesky), solved by the
 * Moore-Penrose pseudo-inverse: V = s (R Cgd)^+ R Q (minimum-norm V when the
 * gates outnumber the dots).  HOST arrays: Cdd [n_dot, n_dot] and Cgd
 * [n_dot, n_gate] row-major in `form` (QA_FORM_*), Q [n_dot] (charges, in
 * units of e), V [n_gate] output; s = carrier_sign (+1 or -1).  No GPU is
 * used.  Errors as qa_model_create, QA_ERR_INVALID for null pointers. */
int qa_optimal_gate_voltages(const double* Cdd, const double* Cgd, int n_dot, int n_gate,
                             int form, double carrier_sign, const double* Q, double* V);

/* Virtual gate matrix (Sec. IV.C; Appendix I): alpha = (Cdd^-1 Cgd)^+,
 * HOST output [n_gate, n_dot] row-major.  Column i is the gate-voltage change
 * that moves the potential of dot i by one unit and leaves the other dots'
 * potentials unchanged (exactly when Cdd^-1 Cgd has full row rank; the
 * least-squares best otherwise); it is the raster direction u or w of a
 * virtual-gate sweep.  Pseudo-inverse by one-sided Jacobi SVD, singular
 * values below max(n_dot, n_gate) eps s_max treated as zero.  No GPU is
 * used. */
int qa_virtual_gate_matrix(const double* Cdd, const double* Cgd, int n_dot, int n_gate,
                           int form, double* alpha);

/* Charge-sensor response (Sec. IV.A).  `m` is the FULL system: its last
 * n_sensor dots are the sensing dots (1 <= n_sensor <= 4, fewer than n_dot).
 * n_dots (DEVICE int8 [H, W, n_dot - n_sensor]) is the ground state of the
 * other dots, computed by the caller without the sensors but with every gate
 * (so the sensor gates' cross-talk is included), e.g. by
 * qa_ground_state_open/closed on the model made of the leading blocks of Cdd
 * and Cgd.  Per pixel, with those charges fixed:
 *   1. each sensor takes the charge minimising U (floor / floor + 1 around the
 *      continuous sensor minimum c_S - (M_SS)^-1 M_SD (n_D - c_D); 2^S
 *      candidates, ties to the lexicographically smaller);
 *   2. its potential V_s = (M (n - c))_s (Eq. "potential");
 *   3. the response at detuning eps = M_ss / 2 - |V_s| from the nearest
 *      Coulomb peak: 1 / (1 + (eps / width)^2) (QA_SENSOR_LORENTZIAN, weak
 *      coupling) or exp(-eps^2 / (2 width^2)) (QA_SENSOR_GAUSSIAN, strong);
 *   4. plus noise along each raster row: white (white_sigma), 1/f
 *      (pink_sigma; Voss-McCartney octaves) and a random telegraph of
 *      jump_amplitude switching with probability jump_prob per pixel; all
 *      drawn from Philox4x32-10 keyed by `seed`, so a result depends only on
 *      the inputs.
 * DEVICE outputs, caller-owned: out_signal float [H, W, n_sensor];
 * out_n_sensor int8 and out_potential FP64 [H, W, n_sensor] (nullable).
 * W <= 8192.  FP64 arithmetic.  Errors: QA_ERR_INVALID, QA_ERR_RANGE,
 * QA_ERR_SHAPE, QA_ERR_CUDA. */
#define QA_SENSOR_LORENTZIAN 0
#define QA_SENSOR_GAUSSIAN   1
typedef struct {
    int n_sensor;
    int shape;
    double width;
    double white_sigma;
    double pink_sigma;
    double jump_amplitude;
    double jump_prob;
    unsigned long long seed;
} qa_sensor_params;
int qa_charge_sensor(qa_model* m, const qa_raster* r, const int8_t* n_dots,
                     const qa_sensor_params* sp, float* out_signal, int8_t* out_n_sensor,
                     double* out_potential, void* stream);

/* Brute-force ground state (Table I, brute-force row; the reference the
 * default and thresholded methods are measured against in Sec. VII, Fig. 4):
 * the exact argmin of U over every n in [0, n_max]^n_dot, in FP64, ties to
 * the lexicographically smallest n.  (n_max + 1)^n_dot states per pixel (at
 * most 2^40, else QA_ERR_RANGE); 0 <= n_max <= 127.  Outputs as
 * qa_ground_state_open, with out_flags holding QA_BF_* bits:
 *   QA_BF_NEAR_TIE  the best two energies are within 1e-9 max(1, |U|);
 *   QA_BF_AT_BOX    some n_i = n_max (the box may cut off the true minimum). */
#define QA_BF_NEAR_TIE 1
#define QA_BF_AT_BOX   2
int qa_brute_force_open(qa_model* m, const qa_raster* r, int n_max, int8_t* out_n,
                        double* out_U, uint8_t* out_flags, void* stream);

/* Brute-force ground state of a CLOSED array: every n >= 0 with
 * sum n = n_charges (constraint iii), in FP64; 0 <= n_charges <= 127 and at
 * most 2^40 states (n_charges + 1)^(n_dot - 1) per pixel.  Outputs and flags
 * as qa_brute_force_open (QA_BF_AT_BOX never set). */
int qa_brute_force_closed(qa_model* m, const qa_raster* r, int n_charges, int8_t* out_n,
                          double* out_U, uint8_t* out_flags, void* stream);

/* Finite-temperature occupation (Sec. IV.B, Eq. "softargmin") over the
 * method's candidate set at threshold t (closed: states with sum N_hat only):
 *   <n> = sum_c n_c exp(-U_c / kT) / Z,  log Z = log sum_c exp(-U_c / kT),
 * kT in the units of U (e^2 / Cdd_ii with Cdd_ii = 1).  DEVICE outputs:
 * out_mean FP32 [H, W, n_dot], out_logZ FP32 [H, W] (nullable).
 * kT > 0, else QA_ERR_RANGE. */
int qa_soft_occupation(qa_model* m, const qa_raster* r, double kT,
                       double threshold, int closed, int n_charges,
                       float* out_mean, float* out_logZ, void* stream);

/* Gradient of a loss L through qa_soft_occupation with the candidate set of
 * every pixel frozen (the set is piecewise constant in the parameters).  The
 * paper has no gradient (Sec. VI notes that its JAX core cannot
 * differentiate); this follows from differentiating Eq. "softargmin":
 *   a_c = -(w_c / kT) (g . n_c - g . <n>),  g = dL/d<n> of the pixel,
 *   dL/dM   = 1/2 sum_p sum_c a_c r_c r_c^T,   r_c = n_c - c,
 *   dL/dc_p = -M sum_c a_c r_c,   dL/dCgd = s sum_p dL/dc_p V_p^T,
 *   dL/dCdd = -M (dL/dM) M.
 * grad_mean: DEVICE FP32 [H, W, n_dot].  Outputs: DEVICE FP64 dL_dCdd
 * [n_dot x n_dot] and dL_dCgd [n_dot x n_gate], overwritten (not
 * accumulated).  The reduction over pixels is deterministic. */
int qa_soft_occupation_backward(qa_model* m, const qa_raster* r, double kT,
                                double threshold, int closed, int n_charges,
                                const float* grad_mean, double* dL_dCdd,
                                double* dL_dCgd, void* stream);

/* qa_soft_occupation that also writes, for the backward pass, an opaque
 * per-pixel context out_ctx (DEVICE, caller-owned, 8 bytes per pixel: the
 * anchor candidate and the log of the pixel's partition sum relative to it). */
int qa_soft_occupation_ctx(qa_model* m, const qa_raster* r, double kT, double threshold,
                           int closed, int n_charges, float* out_mean, float* out_logZ,
                           void* out_ctx, void* stream);

/* qa_soft_occupation_backward given the forward's <n> (mean) and context
 * from qa_soft_occupation_ctx with the same model, raster and settings: the
 * anchor search and the partition sum are not redone.  Same outputs. */
int qa_soft_occupation_backward_ctx(qa_model* m, const qa_raster* r, double kT,
                                    double threshold, int closed, int n_charges,
                                    const float* grad_mean, const float* mean,
                                    const void* ctx, double* dL_dCdd, double* dL_dCgd,
                                    void* stream);

/* Adam hyper-parameters (Kingma & Ba, arXiv 1412.6980, Algorithm 1). */
typedef struct {
    double lr;      /* step size, > 0                  */
    double beta1;   /* first-moment decay, [0, 1)      */
    double beta2;   /* second-moment decay, [0, 1)     */
    double eps;     /* denominator offset, > 0         */
} qa_adam;

/* One capacitance-fitting step on the GPU, fused: the capacitances Cdd, Cgd
 * (DEVICE FP64, [n_dot x n_dot] and [n_dot x n_gate], the parameters) go into
 * the model (FP64 Cholesky on the GPU, as qa_model_update_dev), the soft
 * occupation <n> of Eq. "softargmin" is formed on the raster, the mean squared
 * error against `target` and its gradient dL/d<n> are formed per pixel inside
 * the same kernel, the gradient goes back to (Cdd, Cgd) as in
 * qa_soft_occupation_backward, and one Adam step updates Cdd and Cgd in place.
 *   per_dot = 0: target DEVICE FP32 [H, W], L = mean_p (sum_i <n_i> - target_p)^2
 *   per_dot = 1: target DEVICE FP32 [H, W, n_dot], L = mean_{p,i} (<n_i> - target_pi)^2
 * opt_state: DEVICE FP64 [2 (n_dot^2 + n_dot n_gate) + 3], caller-owned and
 * zeroed before the first step (first moments, second moments, then the step
 * count t, beta1^t and beta2^t).
 * loss (DEVICE FP32 scalar), dL_dCdd, dL_dCgd (DEVICE FP64) and out_mean
 * (DEVICE FP32 [H, W, n_dot]) are optional outputs (NULL to skip), all taken
 * at the parameters before the update.  Everything is enqueued on `stream`
 * with no host synchronisation, so a warmed-up step can be captured in a CUDA
 * graph.  Cdd must stay positive definite; a non-positive pivot is handled as in
 * qa_model_update_dev. */
int qa_fit_step(qa_model* m, const qa_raster* r, double kT, double threshold, int closed,
                int n_charges, const float* target, int per_dot, double* Cdd, double* Cgd,
                double* opt_state, const qa_adam* opt, float* loss, double* dL_dCdd,
                double* dL_dCgd, float* out_mean, void* stream);

/* Record CUDA events around each kernel that later calls on this model
 * enqueue (enable = 1) or stop doing so (0, the default).  The device time of
 * each kernel of the last call is then reported by qa_model_stats.  Events
 * are recorded on the call's stream; they add no synchronisation. */
int qa_model_set_timing(qa_model* m, int enable);

/* Counters of the last call on this model; synchronises `stream` first. */
int qa_model_stats(qa_model* m, void* stream, qa_stats* out);

/* One array of a batched call (qa_batch_create). */
typedef struct {
    qa_model* model;      /* from qa_model_create; all models on one device   */
    qa_raster raster;     /* host vectors, read by qa_batch_create            */
    double threshold;     /* Eq. "threshold", [0, 1]                          */
    int closed;           /* 0 open, 1 closed with n_charges carriers         */
    int n_charges;
    int team;             /* lanes per pixel of the search (1..32, power of
                             two); 0 = the library's choice                   */
    int8_t* out_n;        /* DEVICE [H, W, n_dot]                              */
    double* out_U;        /* DEVICE [H, W] (nullable)                          */
    uint8_t* out_flags;   /* DEVICE [H, W] (nullable)                          */
} qa_batch_item;

typedef struct qa_batch qa_batch;

/* Prepare a batch of `count` independent arrays of any dot count, raster size
 * and open/closed form: validates every item (as the single-array calls do),
 * uploads one descriptor per array, builds the work-unit queues (runs of
 * pixels of one array, ordered by estimated cost, largest first) and
 * allocates the scratch (per-pixel records for all pixels, the recheck lists).
 * Synchronous; *out is owned by the caller (qa_batch_destroy).  The models
 * and output buffers must outlive the batch; model capacitances may change
 * between runs only through qa_model_update (same shapes).
 * Errors: as qa_ground_state_open, plus QA_ERR_SHAPE for count < 1 or items on
 * different devices. */
int qa_batch_create(const qa_batch_item* items, int count, qa_batch** out);

/* Run the batch on `stream`: one persistent prep launch and one persistent
 * search launch whose blocks take work units from a device queue, then the
 * list kernel (near-tie resolve, FP64 recheck) over all arrays.  Asynchronous, allocates
 * nothing and synchronises nothing, so it can be captured in a CUDA graph.
 * Runs of one batch must not overlap on the GPU. */
int qa_batch_run(qa_batch* b, void* stream);

/* Counters of the last run (synchronises `stream`). */
int qa_batch_stats(qa_batch* b, void* stream, qa_stats* out);

/* Release the batch (synchronises the device). */
int qa_batch_destroy(qa_batch* b);

/* Largest raster qa_ground_state_open_static accepts (128 x 128 pixels). */
#define QA_STATIC_MAX_PIXELS 16384

/* The open ground state of qa_ground_state_open, for callers that cannot
 * allocate GPU memory while they run -- a control loop that drives an
 * instrument in real time and must not stall on, or fail in, an allocation,
 * or a host process whose GPU memory is already fully handed to another
 * allocator.  (The paper has no counterpart; this is a property of this
 * library only.)  It allocates nothing: where qa_ground_state_open keeps its
 * per-pixel scratch in a workspace it grows with cudaMalloc, this call uses a
 * fixed array of static device memory for at most QA_STATIC_MAX_PIXELS
 * pixels; larger rasters are rejected with QA_ERR_SHAPE.  The model must come
 * from qa_model_create (run it during set-up); inputs, outputs and errors are
 * otherwise those of qa_ground_state_open.
 *  - The first call on a device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *    With CUDA's lazy module loading (the default) that lookup may be what
 *    loads the library's module on the device, and so what allocates the
 *    array: make the first call during set-up, where an allocation is
 *    acceptable; later calls allocate nothing.
 *  - Every call on a device shares the one array, which keeps the previous
 *    call's contents: calls that overlap on the GPU race, so serialise them
 *    (one stream, or events).
 *  - qa_model_stats does not report these calls.
 *  - The array (about 5.4 MB) is held on every GPU that loads the library
 *    until the process exits. */
int qa_ground_state_open_static(qa_model* m, const qa_raster* r, double threshold,
                                int8_t* out_n, double* out_U, uint8_t* out_flags,
                                void* stream);

/* Message of the last error on the calling thread ("" if none). */
const char* qa_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
