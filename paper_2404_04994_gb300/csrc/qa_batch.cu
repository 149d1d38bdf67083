// qa_batch.cu -- the batched ground state: many arrays (any N, raster size,
// open or closed) in one persistent prep launch and one persistent search
// launch.  Blocks take work units -- a run of pixels of one array -- from a
// device queue (an atomic counter over a unit table ordered largest first),
// stage that array's constants when it changes, and run the same tile code as
// the single-array kernels.  The near-tie and FP64 lists are then settled by
// the list kernels shared with the single-array path.
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

template <int L1, int L2>
__device__ __forceinline__ void search_any(const GsLaunch& L, const ArrayDesc& a,
                                           SearchShared& sh, int array, long long tb,
                                           long long end, SearchAcc& acc) {
  const bool tf = a.cfg.T >= kTeamFinishMin;
  if (a.mt.closed) {
    if (tf) search_tile<L1, L2, true, true>(L, a, sh, array, tb, end, acc);
    else search_tile<L1, L2, true, false>(L, a, sh, array, tb, end, acc);
  } else {
    if (tf) search_tile<L1, L2, false, true>(L, a, sh, array, tb, end, acc);
    else search_tile<L1, L2, false, false>(L, a, sh, array, tb, end, acc);
  }
}

__global__ void __launch_bounds__(kSearchThreads) k_search_batch(GsLaunch L) {
  __shared__ SearchShared sh;
  __shared__ int s_unit;
  int staged = -1;
  SearchAcc acc;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = (int)atomicAdd(&L.cnt->q_search, 1u);
    __syncthreads();
    const int u = s_unit;
    if (u >= L.n_search_units) break;
    const WorkUnit wu = L.search_units[u];
    const ArrayDesc& a = L.table[wu.array];
    if (wu.array != staged) {
      stage_consts(&a.md->k, &sh.cs);
      __syncthreads();
      staged = wu.array;
    }
    const int tpb = kSearchThreads / a.cfg.T;
    const long long end = wu.first + wu.count;
    for (long long tb = wu.first; tb < end; tb += tpb) {
      switch (a.klass) {
        case 0: search_any<2, 0>(L, a, sh, wu.array, tb, end, acc); break;
        case 1: search_any<4, 0>(L, a, sh, wu.array, tb, end, acc); break;
        case 2: search_any<4, 3>(L, a, sh, wu.array, tb, end, acc); break;
        default: search_any<5, 4>(L, a, sh, wu.array, tb, end, acc); break;
      }
    }
  }
  if (threadIdx.x == 0) {
    BlockCounts& o = L.bc_search[blockIdx.x];
    o.evaluated = acc.evaluated;
    o.near_tie = acc.near_tie;
    o.boundary = acc.boundary;
    o.overflow = acc.overflow;
  }
}

// Resident blocks per SM of the two persistent kernels.
void batch_occupancy(int* prep_per_sm, int* search_per_sm) {
  *prep_per_sm = *search_per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(prep_per_sm, k_prep_batch, kPrepThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(search_per_sm, k_search_batch,
                                                kSearchThreads, 0);
  if (*prep_per_sm < 1) *prep_per_sm = 1;
  if (*search_per_sm < 1) *search_per_sm = 1;
}

cudaError_t launch_ground_state_batch(const GsLaunch& L, cudaStream_t st) {
  if (L.ev) cudaEventRecord(L.ev[0], st);
  cudaMemsetAsync(L.cnt, 0, sizeof(Counters), st);
  k_prep_batch<<<L.grid_prep, kPrepThreads, 0, st>>>(L);
  if (L.ev) cudaEventRecord(L.ev[1], st);
  k_search_batch<<<L.grid_search, kSearchThreads, 0, st>>>(L);
  if (L.ev) cudaEventRecord(L.ev[2], st);
  launch_lists(L, st);
  if (L.ev) cudaEventRecord(L.ev[3], st);
  return cudaGetLastError();
}

}  // namespace qa
