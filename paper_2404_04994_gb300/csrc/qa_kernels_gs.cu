// qa_kernels_gs.cu -- ground-state kernels for one array: one tile per block
// for prep and search, grid-stride over the lists for resolve and recheck.
// The stages themselves live in qa_gs_tiles.cuh (shared with the batch).
#include "qa_gs_tiles.cuh"

namespace qa {

template <bool CLOSED>
__global__ void __launch_bounds__(kPrepThreads) k_prep(GsLaunch L) {
  __shared__ PrepShared sh;
  const ArrayDesc& a = L.one;
  // the search may launch now: it stages its constants and then waits for
  // this grid's results in grid_dep_wait
  grid_dep_signal();
  if (L.prep_zeroes_counters && blockIdx.x == 0)
    for (int e = threadIdx.x; e < (int)(sizeof(Counters) / sizeof(unsigned)); e += blockDim.x)
      reinterpret_cast<unsigned*>(L.cnt)[e] = 0u;
  prep_stage_array(a, sh);
  PrepAcc acc;
  const long long team_base = (long long)blockIdx.x * (kPrepThreads / a.prep_team);
  prep_tile<CLOSED>(a, sh, team_base, a.sc.P, acc);
  if (threadIdx.x == 0) {
    BlockCounts& o = L.bc_prep[blockIdx.x];
    o.candidates = acc.candidates;
    o.qp = acc.qp;
    o.doubled = acc.doubled;
  }
}

template <int L1, int L2, bool CLOSED, bool TF>
__global__ void __launch_bounds__(kSearchThreads) k_search(GsLaunch L) {
  __shared__ SearchShared sh;
  const ArrayDesc& a = L.one;
  stage_consts(&a.md->k, &sh.cs);
  grid_dep_wait();  // the records come from k_prep
  __syncthreads();
  // every block of this grid is resident or done once all have passed here:
  // the resolve grid may launch into the slots that free up, stage its
  // constants and wait for this grid's results
  grid_dep_signal();
  SearchAcc acc;
  const long long team_base = (long long)blockIdx.x * (kSearchThreads / a.cfg.T);
  search_tile<L1, L2, CLOSED, TF>(L, a, sh, 0, team_base, a.sc.P, acc);
  if (threadIdx.x == 0) {
    BlockCounts& o = L.bc_search[blockIdx.x];
    o.evaluated = acc.evaluated;
    o.near_tie = acc.near_tie;
    o.boundary = acc.boundary;
    o.overflow = acc.overflow;
  }
}

// Near-tie list: one block per entry, grid-stride.  In a batched call the
// entries belong to different arrays; the model is restaged when it changes.
__global__ void __launch_bounds__(kResolveThreads) k_resolve(GsLaunch L) {
  __shared__ ResolveShared S;
  int staged = -1;
  if (!L.table) {  // one array: its model is known before the search ends
    stage_consts(&L.one.md->k, &S.cs);
    staged = 0;
  }
  grid_dep_signal();  // the recheck may launch and stage likewise
  grid_dep_wait();    // the tie list comes from the search
  const unsigned ntie = L.cnt->n_tie;
  unsigned my_res = 0;
  for (unsigned it = blockIdx.x; it < ntie; it += gridDim.x) {
    const ListEntry te = L.tie_list[it];
    const ArrayDesc& a = desc_of(L, te.array);
    if (te.array != staged) {
      stage_consts(&a.md->k, &S.cs);
      staged = te.array;
    }
    if (threadIdx.x == 0) S.bcnt = 0u;
    __syncthreads();
    if (a.mt.closed)
      resolve_entry<true>(L, a, S, te, my_res);
    else
      resolve_entry<false>(L, a, S, te, my_res);
    __syncthreads();
  }
  if (threadIdx.x == 0 && my_res) atomicAdd(&L.cnt->resolved, (unsigned long long)my_res);
}

// FP64 recheck list: one block per entry, grid-stride.
__global__ void __launch_bounds__(kRecheckThreads) k_recheck(GsLaunch L) {
  __shared__ RecheckShared S;
  int staged = -1;
  if (!L.table) {  // one array: its model is known before the resolve ends
    for (int e = threadIdx.x; e < kMaxDot * kLdM; e += blockDim.x) S.sM[e] = L.one.md->k.Mhi[e];
    staged = 0;
  }
  grid_dep_wait();  // the FP64 list is complete once the resolve has run
  const unsigned nflag = L.cnt->n_flag;
  for (unsigned it = blockIdx.x; it < nflag; it += gridDim.x) {
    const ListEntry fe = L.flag_list[it];
    const ArrayDesc& a = desc_of(L, fe.array);
    if (fe.array != staged) {
      for (int e = threadIdx.x; e < kMaxDot * kLdM; e += blockDim.x) S.sM[e] = a.md->k.Mhi[e];
      staged = fe.array;
    }
    if (threadIdx.x == 0) S.bcount = 0u;
    __syncthreads();
    if (a.mt.closed)
      recheck_entry<true>(L, a, S, fe);
    else
      recheck_entry<false>(L, a, S, fe);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host-side dispatch
// ---------------------------------------------------------------------------
int prep_blocks(const GsLaunch& L) {
  const long long tpb = kPrepThreads / L.one.prep_team;
  return (int)((L.one.sc.P + tpb - 1) / tpb);
}
int search_blocks(const GsLaunch& L) {
  const int teams = kSearchThreads / L.one.cfg.T;
  return (int)((L.one.sc.P + teams - 1) / teams);
}

// Launch with programmatic stream serialisation (the kernel waits for its
// predecessor's results with grid_dep_wait).
template <typename... KArgs>
static cudaError_t launch_dependent(void (*kern)(KArgs...), unsigned grid, unsigned block,
                                    cudaStream_t st, KArgs... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_lists(const GsLaunch& L, cudaStream_t st) {
  cudaError_t e = launch_dependent(k_resolve, (unsigned)L.num_sms, kResolveThreads, st, L);
  if (e == cudaSuccess) e = launch_dependent(k_recheck, (unsigned)L.num_sms, kRecheckThreads, st, L);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int L1, int L2, bool CLOSED>
static cudaError_t run(const GsLaunch& Lin, cudaStream_t st) {
  // k_prep clears the counters (no memset node); search, resolve and recheck
  // start early behind their predecessor (programmatic dependent launch)
  GsLaunch L = Lin;
  L.prep_zeroes_counters = 1;
  if (L.ev) cudaEventRecord(L.ev[0], st);
  k_prep<CLOSED><<<prep_blocks(L), kPrepThreads, 0, st>>>(L);
  if (L.ev) cudaEventRecord(L.ev[1], st);
  cudaError_t e;
  if (L.one.cfg.T >= kTeamFinishMin)
    e = launch_dependent(k_search<L1, L2, CLOSED, true>, (unsigned)search_blocks(L),
                         kSearchThreads, st, L);
  else
    e = launch_dependent(k_search<L1, L2, CLOSED, false>, (unsigned)search_blocks(L),
                         kSearchThreads, st, L);
  if (e != cudaSuccess) return e;
  if (L.ev) cudaEventRecord(L.ev[2], st);
  e = launch_lists(L, st);
  if (L.ev) cudaEventRecord(L.ev[3], st);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_prep(const GsLaunch& L, cudaStream_t st) {
  cudaMemsetAsync(L.cnt, 0, sizeof(Counters), st);
  if (L.one.sc.P == 0) return cudaGetLastError();
  if (L.one.mt.closed)
    k_prep<true><<<prep_blocks(L), kPrepThreads, 0, st>>>(L);
  else
    k_prep<false><<<prep_blocks(L), kPrepThreads, 0, st>>>(L);
  return cudaGetLastError();
}

int search_klass(const SearchCfg& c) {
  const int key = c.L1 * 10 + c.L2;
  return key == 20 ? 0 : key == 40 ? 1 : key == 43 ? 2 : key == 54 ? 3 : -1;
}

bool search_cfg_supported(const SearchCfg& c) {
  const bool team = c.T >= 1 && c.T <= 32 && (c.T & (c.T - 1)) == 0;
  return search_klass(c) >= 0 && team;
}

cudaError_t launch_ground_state(const GsLaunch& L, cudaStream_t st) {
  const bool cl = L.one.mt.closed != 0;
  switch (search_klass(L.one.cfg)) {
    case 0: return cl ? run<2, 0, true>(L, st) : run<2, 0, false>(L, st);
    case 1: return cl ? run<4, 0, true>(L, st) : run<4, 0, false>(L, st);
    case 2: return cl ? run<4, 3, true>(L, st) : run<4, 3, false>(L, st);
    case 3: return cl ? run<5, 4, true>(L, st) : run<5, 4, false>(L, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qa
