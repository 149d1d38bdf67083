// qa_batch.cu -- the batched ground state: many arrays (any N, raster size,
// open or closed) in one persistent prep launch and one persistent search
// launch per kernel variant present (split, form, team finish).  Blocks take
// work units -- a run of pixels of one array -- from a device queue (an
// atomic counter over a unit table ordered largest first), stage that array's
// constants when it changes, and run the same tile code as the single-array
// kernels.  The near-tie and FP64 lists are then settled by the list kernels
// shared with the single-array path.
#include "qa_gs_tiles.cuh"

namespace qa {

__global__ void __launch_bounds__(kPrepThreads) k_prep_batch(GsLaunch L) {
  __shared__ PrepShared sh;
  __shared__ int s_unit;
  int staged = -1;
  PrepAcc acc;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = (int)atomicAdd(&L.cnt->q_prep, 1u);
    __syncthreads();
    const int u = s_unit;
    if (u >= L.n_prep_units) break;
    const WorkUnit wu = L.prep_units[u];
    const ArrayDesc& a = L.table[wu.array];
    if (wu.array != staged) {
      prep_stage_array(a, sh);
      staged = wu.array;
    }
    const int tpb = kPrepThreads / a.prep_team;
    const long long end = wu.first + wu.count;
    for (long long tb = wu.first; tb < end; tb += tpb) {
      if (a.mt.closed)
        prep_tile<true>(a, sh, tb, end, acc);
      else
        prep_tile<false>(a, sh, tb, end, acc);
    }
  }
  if (threadIdx.x == 0) {
    BlockCounts& o = L.bc_prep[blockIdx.x];
    o.candidates = acc.candidates;
    o.qp = acc.qp;
    o.doubled = acc.doubled;
  }
}

// The search of one kernel variant (split, form, team finish): a persistent
// grid over that variant's units, so that every variant runs with its own
// register count (one kernel over all of them needs the largest).
template <int L1, int L2, bool CLOSED, bool TF>
__device__ __forceinline__ void search_batch_units(const GsLaunch& L, int v) {
  __shared__ SearchShared sh;
  __shared__ int s_unit;
  int staged = -1;
  SearchAcc acc;
  const int first = L.var_first[v], count = L.var_count[v];
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = (int)atomicAdd(&L.cnt->q_var[v], 1u);
    __syncthreads();
    const int u = s_unit;
    if (u >= count) break;
    const WorkUnit wu = L.search_units[first + u];
    const ArrayDesc& a = L.table[wu.array];
    if (wu.array != staged) {
      stage_consts(&a.md->k, &sh.cs);
      __syncthreads();
      staged = wu.array;
    }
    const int tpb = kSearchThreads / a.cfg.T;
    const long long end = wu.first + wu.count;
    for (long long tb = wu.first; tb < end; tb += tpb)
      search_tile<L1, L2, CLOSED, TF>(L, a, sh, wu.array, tb, end, acc);
  }
  if (threadIdx.x == 0) {
    BlockCounts& o = L.bc_search[L.var_bc[v] + blockIdx.x];
    o.evaluated = acc.evaluated;
    o.near_tie = acc.near_tie;
    o.boundary = acc.boundary;
    o.overflow = acc.overflow;
  }
}

template <int L1, int L2, bool CLOSED, bool TF>
__global__ void __launch_bounds__(kSearchThreads) k_search_batch(GsLaunch L, int v) {
  search_batch_units<L1, L2, CLOSED, TF>(L, v);
}

// The pruned search's variants (5 + 2 split, teams of kBnbMinT+ lanes),
// built for kBnbBlocks resident blocks per SM.
template <bool CLOSED>
__global__ void __launch_bounds__(kSearchThreads, kBnbBlocks) k_search_batch_bnb(GsLaunch L, int v) {
  search_batch_units<kBnbL1, kBnbL2, CLOSED, true>(L, v);
}

// The kernel of variant v = 4 klass + 2 closed + team finish.
typedef void (*BatchSearchKernel)(GsLaunch, int);
static BatchSearchKernel batch_search_kernel(int v) {
#define QA_V(l1, l2)                                                                   \
  k_search_batch<l1, l2, false, false>, k_search_batch<l1, l2, false, true>,          \
      k_search_batch<l1, l2, true, false>, k_search_batch<l1, l2, true, true>
  static const BatchSearchKernel table[kBatchVariants] = {
      QA_V(2, 0), QA_V(4, 0), QA_V(4, 3), QA_V(5, 4),
      k_search_batch<5, 2, false, false>, k_search_batch_bnb<false>,
      k_search_batch<5, 2, true, false>, k_search_batch_bnb<true>};
  static_assert(bnb_search(kBnbL1, kBnbL2) && kBnbL1 == 5 && kBnbL2 == 2,
                "the block-level variants of klass 4 are the pruned search");
#undef QA_V
  return (v >= 0 && v < kBatchVariants) ? table[v] : nullptr;
}

int batch_search_occupancy(int v) {
  int nb = 0;
  const BatchSearchKernel k = batch_search_kernel(v);
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kSearchThreads, 0) != cudaSuccess)
    return 1;
  return nb < 1 ? 1 : nb;
}

// Resident blocks per SM of the persistent prep kernel and of the search of
// the large arrays' variant (the pruned search, 5 + 2 split, open), for unit
// sizing.
void batch_occupancy(int* prep_per_sm, int* search_per_sm) {
  *prep_per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(prep_per_sm, k_prep_batch, kPrepThreads, 0);
  if (*prep_per_sm < 1) *prep_per_sm = 1;
  *search_per_sm = batch_search_occupancy(4 * 4 + 1);
}

cudaError_t launch_ground_state_batch(const GsLaunch& L, cudaStream_t st) {
  if (L.ev) cudaEventRecord(L.ev[0], st);
  cudaMemsetAsync(L.cnt, 0, sizeof(Counters), st);
  k_prep_batch<<<L.grid_prep, kPrepThreads, 0, st>>>(L);
  if (L.ev) cudaEventRecord(L.ev[1], st);
  for (int v = 0; v < kBatchVariants; ++v)
    if (L.var_count[v] > 0) batch_search_kernel(v)<<<L.var_grid[v], kSearchThreads, 0, st>>>(L, v);
  if (L.ev) cudaEventRecord(L.ev[2], st);
  launch_lists(L, st);
  if (L.ev) cudaEventRecord(L.ev[3], st);
  return cudaGetLastError();
}

}  // namespace qa
