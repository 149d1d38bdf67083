// qa_launch.h -- internal interface between the host ABI (qa_api.cu) and the
// kernel translation units.  Not part of the public header.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qa_device.cuh"

namespace qa {

// Split of the candidate hypercube used by the search kernel.
struct SearchCfg {
  int L1;  // unrolled inner slots (register table of 2^L1 pair terms)
  int L2;  // unrolled middle slots (compile-time Gray walk)
  int T;   // lanes per pixel (1..32)
};

// One array of a ground-state call: its model, voltages, method settings,
// scratch records and outputs.
struct ArrayDesc {
  const ModelData* md;
  int n, ng;
  Scan sc;
  RasterK rk;          // host-computed raster constants (rk.valid = 0: device)
  Method mt;
  SearchCfg cfg;
  int prep_team;       // lanes per pixel in the prep stage (pow2 >= n, <= 16)
  int klass;           // search split class: 0 (2,0), 1 (4,0), 2 (4,3), 3 (5,4)
  float bx_analytic;   // decision margin for double-float continuous minima
  float bx_qp_scale;   // ... per unit of (1 + max|c| + N_hat) for FP32 QP minima
  PixRec* recs;        // scratch [P]
  int8_t* out_n;
  int16_t* out_n16;    // int16 charge map instead of out_n when non-null
  double* out_U;
  uint8_t* out_flags;
};

constexpr int kSearchThreads = 128;  // threads of a search block
constexpr int kTeamFinishMin = 8;    // teams at least this wide finish the winning block together
// The pruned search (branch and bound over the outer slots, qa_search.cuh):
// arrays with the 5 + 2 split, teams of kBnbMinT or 32 lanes.
constexpr int kBnbL1 = 5, kBnbL2 = 2;
constexpr int kBnbMinT = 16;
constexpr int kBnbBlocks = 5;  // resident blocks per SM its kernels are built for
// Batched search kernel variants: 4 per split class (closed, team finish).
constexpr int kBatchVariants = 20;
static_assert(sizeof(((Counters*)nullptr)->q_var) / sizeof(unsigned) == kBatchVariants,
              "one queue head per batched search variant");
__host__ __device__ constexpr bool bnb_search(int L1, int L2) {
  return L1 == kBnbL1 && L2 == kBnbL2;
}

// Pixels [first, first + count) of one array of a batched call.
struct WorkUnit {
  int array;
  int count;
  long long first;
};

struct GsLaunch {
  ArrayDesc one;               // single-array call
  const ArrayDesc* table;      // batched call: descriptors (null: use `one`)
  const WorkUnit* prep_units;  // batched call: work queues, largest first
  int n_prep_units;
  const WorkUnit* search_units;
  int n_search_units;
  ListEntry* flag_list;        // scratch: pixels for the FP64 recheck
  ListEntry* tie_list;         // scratch: near-tie pixels for the list kernel's resolve
  Counters* cnt;               // scratch; list heads zero at the start of each call
  BlockCounts* bc_prep;        // scratch [prep blocks]
  BlockCounts* bc_search;      // scratch [search blocks]
  int grid_prep, grid_search;  // batched call: persistent grid sizes
  // batched call: the search units grouped by kernel variant v = 4 klass +
  // 2 closed + team finish (units [var_first, var_first + var_count) of
  // search_units, largest first within a group), one persistent grid of
  // var_grid blocks per variant, its block counts from bc_search + var_bc
  int var_first[kBatchVariants], var_count[kBatchVariants], var_grid[kBatchVariants],
      var_bc[kBatchVariants];
  int num_sms;
  cudaEvent_t* ev;     // optional: events around prep / search / resolve+recheck
};

// Brute-force ground state (Table I): digit range R, free digits (N open,
// N - 1 closed), trailing digits walked per outer state, outer states.
struct BruteLaunch {
  ArrayDesc a;                 // model, voltages, method (closed, N_hat), outputs
  int radix;                   // n_max + 1 (open) or N_hat + 1 (closed)
  int nfree;
  int ni;
  int n_max;                   // open: box bound reported by kBruteAtBox
  unsigned long long nouter;   // radix^(nfree - ni)
};
enum : unsigned { kBruteNearTie = 1u, kBruteAtBox = 2u, kBruteNone = 4u };
cudaError_t launch_brute(const BruteLaunch& L, cudaStream_t st);

// Charge-sensor response (Sec. IV.A) over a raster: the model is the full
// system, its last S dots the sensors; n_dots holds the other dots' ground
// state [P, n - S].
struct SensorLaunch {
  ArrayDesc a;                 // full model, raster, carrier
  int S;                       // sensors (1..4)
  int shape;                   // 0 Lorentzian, 1 Gaussian
  int K;                       // 1/f octaves: 2^(K-1) >= W
  double width, white_sigma, pink_sigma, jump_amplitude, jump_prob;
  unsigned long long seed;
  const int8_t* n_dots;
  float* out_signal;           // [P, S]
  int8_t* out_n_sensor;        // [P, S] (nullable)
  double* out_potential;       // [P, S] (nullable)
};
cudaError_t launch_sensor(const SensorLaunch& L, cudaStream_t st);

// prep + search (one kernel or two) -> resolve -> FP64 recheck of one array,
// enqueued on `st`; the counters' list heads must be zero on entry and are on
// exit.
cudaError_t launch_ground_state(const GsLaunch& a, cudaStream_t st);
// The same for a batch (persistent kernels over the work queues).
cudaError_t launch_ground_state_batch(const GsLaunch& a, cudaStream_t st);
// prep alone (candidate-set records), for the soft path.
cudaError_t launch_prep(const GsLaunch& a, cudaStream_t st);
// resolve + FP64 recheck over the lists of a call (single or batched).
cudaError_t launch_lists(const GsLaunch& a, cudaStream_t st);
int prep_blocks(const GsLaunch& a);
int search_blocks(const GsLaunch& a);
// true: one kernel prepares and searches each tile (block counts of both
// stages per search block); false: k_prep then k_search
bool fused_tiles(const GsLaunch& a);
bool search_cfg_supported(const SearchCfg& c);
int search_klass(const SearchCfg& c);
// Resident blocks per SM of the persistent batched kernels.
void batch_occupancy(int* prep_per_sm, int* search_per_sm);
int batch_search_occupancy(int variant);  // resident blocks per SM of a variant's kernel

struct SoftLaunch {
  const ModelData* md;
  int n, ng;
  Scan sc;
  Method mt;
  SearchCfg cfg;
  float bx_analytic, bx_qp_scale;
  double kT;
  PixRec* recs;
  Counters* cnt;
  float* out_mean;      // forward outputs
  float* out_logZ;
  const float* grad_mean;  // backward input
  uint2* ctx_out;          // forward, optional: per pixel (b* bits, log sum exp(-D/kT))
  const uint2* ctx_in;     // backward, optional: the forward's context ...
  const float* mean_in;    // ... and its <n>, so passes 1 and 2 are not redone
  float* partials;      // backward scratch: [blocks][2 * L] double-float sums
  double* sums;         // backward scratch: [L] block partials summed
  double* dL_dCdd;      // backward outputs
  double* dL_dCgd;
  int num_sms;
  cudaEvent_t* ev;     // optional: events around the soft kernel(s)
  // fit step: the kernel forms the MSE gradient of each pixel from its own
  // <n> (no grad_mean input), the last stage adds up the loss and applies
  // one Adam step to the parameters in place
  const float* fit_target;  // [P] (target of sum_i <n_i>) or [P, n] (per dot); null otherwise
  int fit_per_dot;
  float fit_scale;          // 2 / (number of loss terms)
  double fit_inv_count;     // 1 / (number of loss terms)
  float* loss_out;          // device float, may be null
  double* fit_Cdd;          // [n * n] parameters
  double* fit_Cgd;          // [n * ng]
  double* fit_state;        // [2 (n n + n ng) + 1]: first moments, second moments, step
  double lr, beta1, beta2, eps;
};

cudaError_t launch_soft_forward(const SoftLaunch& a, cudaStream_t st);
cudaError_t launch_soft_backward(const SoftLaunch& a, cudaStream_t st);
size_t soft_partials_floats(int n, long long P, const SearchCfg& cfg);

// FP64 inverse (symmetric sweeps) of a device Cdd into the model (update_dev).
cudaError_t launch_model_update(ModelData* md, int n, int ng,
                                const double* Cdd_dev, const double* Cgd_dev,
                                cudaStream_t st);

}  // namespace qa
