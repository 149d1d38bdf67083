// qa_kernels_gs.cu -- ground-state kernels for one array: one tile per block
// for prep and search (one kernel or two), grid-stride over the lists for
// resolve and recheck.
// The stages themselves live in qa_gs_tiles.cuh (shared with the batch).
#include "qa_gs_tiles.cuh"

namespace qa {

// Prep alone: the soft path's candidate-set records, and the first stage of a
// ground-state call whose tiling keeps prep and search apart (it clears the
// accumulating counters; the list heads are zero on entry).
template <bool CLOSED>
__global__ void __launch_bounds__(kPrepThreads) k_prep(GsLaunch L) {
  __shared__ PrepShared sh;
  const ArrayDesc& a = L.one;
  // the search may launch now: it stages its constants and then waits for
  // this grid's results
  grid_dep_signal();
  if (blockIdx.x == 0) zero_accumulators(L.cnt);
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

// Prep and search of one tile: the block prepares the pixels it then searches
// (their records go to global memory for the list kernels and come back from
// L1 / L2 for the search), so no grid-wide wait separates the two stages and
// the prep of later tiles overlaps the search of earlier ones.
template <int L1, int L2, bool CLOSED, bool TF>
__device__ __forceinline__ void ground_state_tile(const GsLaunch& L) {
  __shared__ GsShared sh;
  const ArrayDesc& a = L.one;
  // the resolve may launch once every block has passed here (all are then
  // resident or done): it stages its constants and waits for this grid
  grid_dep_signal();
  if (blockIdx.x == 0) zero_accumulators(L.cnt);
  prep_stage_array(a, sh.p);
  const long long per = kSearchThreads / a.cfg.T;
  const long long first = (long long)blockIdx.x * per;
  const long long last = first + per < a.sc.P ? first + per : a.sc.P;
  PrepAcc pacc;
  for (long long b = first; b < last; b += kPrepThreads / a.prep_team)
    prep_tile<CLOSED>(a, sh.p, b, last, pacc);
  if (threadIdx.x == 0) {
    BlockCounts& o = L.bc_prep[blockIdx.x];
    o.candidates = pacc.candidates;
    o.qp = pacc.qp;
    o.doubled = pacc.doubled;
  }
  __syncthreads();  // the tile's records are written; the prep scratch is free
  SearchAcc acc;
  search_tile<L1, L2, CLOSED, TF>(L, a, sh.s, 0, first, a.sc.P, acc);
  if (threadIdx.x == 0) {
    BlockCounts& o = L.bc_search[blockIdx.x];
    o.evaluated = acc.evaluated;
    o.near_tie = acc.near_tie;
    o.boundary = acc.boundary;
    o.overflow = acc.overflow;
  }
}

template <int L1, int L2, bool CLOSED, bool TF>
__global__ void __launch_bounds__(kSearchThreads) k_ground_state(GsLaunch L) {
  ground_state_tile<L1, L2, CLOSED, TF>(L);
}

// The pruned search's tiles, built for kBnbBlocks resident blocks per SM.
template <bool CLOSED>
__global__ void __launch_bounds__(kSearchThreads, kBnbBlocks) k_ground_state_bnb(GsLaunch L) {
  ground_state_tile<kBnbL1, kBnbL2, CLOSED, true>(L);
}

// Search alone, behind k_prep (programmatic dependent launch): for tilings
// where one search block covers several prep blocks' pixels, which a block
// preparing its own tile would prepare one pass after another.
template <int L1, int L2, bool CLOSED, bool TF>
__device__ __forceinline__ void search_only_tile(const GsLaunch& L) {
  __shared__ SearchShared sh;
  const ArrayDesc& a = L.one;
  stage_consts(&a.md->k, &sh.cs);
  grid_dep_wait();  // the records come from k_prep
  __syncthreads();
  // every block of this grid is resident or done once all have passed here:
  // the resolve grid may launch into the slots that free up
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

template <int L1, int L2, bool CLOSED, bool TF>
__global__ void __launch_bounds__(kSearchThreads) k_search(GsLaunch L) {
  search_only_tile<L1, L2, CLOSED, TF>(L);
}

template <bool CLOSED>
__global__ void __launch_bounds__(kSearchThreads, kBnbBlocks) k_search_bnb(GsLaunch L) {
  search_only_tile<kBnbL1, kBnbL2, CLOSED, true>(L);
}

// The lists after the search, in one launch: near ties (resolve_entry) and
// the FP64 recheck list (recheck_entry), grid-stride over both; a near tie
// the resolve cannot settle is rechecked next by the same block.  The two
// entries' shared layouts overlap, so each restages its model constants when
// the other ran last.
static_assert(kResolveThreads == kRecheckThreads, "one block size for both lists");
__global__ void __launch_bounds__(kResolveThreads) k_lists(GsLaunch L) {
  __shared__ union ListShared {
    ResolveShared r;
    RecheckShared c;
  } S;
  int staged_r = -1, staged_c = -1;  // the array whose constants each layout holds
  if (!L.table) {  // one array: its model is known before the search ends
    stage_consts(&L.one.md->k, &S.r.cs);
    staged_r = 0;
  }
  grid_dep_wait();  // the lists come from the search
  // one array: the block's first near-tie entry is read together with the
  // list heads instead of after them (the list has room for P entries, so
  // the index lies inside it; the entry is used only below the head)
  const bool pf = !L.table && (long long)blockIdx.x < L.one.sc.P;
  ListEntry first{};
  if (pf) first = L.tie_list[blockIdx.x];
  const unsigned ntie = L.cnt->n_tie;
  const unsigned nflag = L.cnt->n_flag;
  unsigned my_res = 0, my_slmax = 0;
  for (unsigned it = blockIdx.x; it < ntie + nflag; it += gridDim.x) {
    ListEntry e = (pf && it == blockIdx.x && it < ntie)
                      ? first
                      : (it < ntie ? L.tie_list[it] : L.flag_list[it - ntie]);
    const ArrayDesc& a = desc_of(L, e.array);
    bool check = it >= ntie;
    if (!check) {
      if (e.array != staged_r) {
        __syncthreads();
        stage_consts(&a.md->k, &S.r.cs);
        staged_r = e.array;
        staged_c = -1;
      }
      if (threadIdx.x == 0) S.r.bcnt = 0u;
      __syncthreads();
      if (a.mt.closed)
        resolve_entry<true>(L, a, S.r, e, my_res, my_slmax);
      else
        resolve_entry<false>(L, a, S.r, e, my_res, my_slmax);
      __syncthreads();
      check = S.r.dok == 0;
      e.tie = 1;
      __syncthreads();
    }
    if (check) {
      if (e.array != staged_c) {
        for (int q = threadIdx.x; q < kMaxDot * kLdM; q += blockDim.x) S.c.sM[q] = a.md->k.Mhi[q];
        staged_c = e.array;
        staged_r = -1;
      }
      if (threadIdx.x == 0) S.c.bcount = 0u;
      __syncthreads();
      if (a.mt.closed)
        recheck_entry<true>(L, a, S.c, e);
      else
        recheck_entry<false>(L, a, S.c, e);
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && my_res) atomicAdd(&L.cnt->resolved, (unsigned long long)my_res);
  if (threadIdx.x == 0 && my_slmax)
    atomicMax(&L.cnt->shortlist_max, (unsigned long long)my_slmax);
  // the list heads start the next call at zero: the last block to finish
  // clears them (every block has read both by then)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&L.cnt->lists_done, 1u) == gridDim.x - 1) {
      L.cnt->n_flag = 0u;
      L.cnt->n_tie = 0u;
      L.cnt->lists_done = 0u;
    }
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
  cudaError_t e = launch_dependent(k_lists, (unsigned)L.num_sms, kResolveThreads, st, L);
  return e != cudaSuccess ? e : cudaGetLastError();
}

bool fused_tiles(const GsLaunch& L) {
  // a block preparing its own tile makes (prep_team / T) prep passes over it
  return L.one.prep_team <= 2 * L.one.cfg.T;
}

template <int L1, int L2, bool CLOSED>
static cudaError_t run(const GsLaunch& L, cudaStream_t st) {
  // prep + search in one kernel where a search tile is at most two prep
  // passes, else k_prep and k_search (programmatic dependent launch); the
  // first kernel clears the accumulating counters, the list heads are zero
  // on entry; resolve and recheck start early behind their predecessor
  cudaError_t e = cudaSuccess;
  if (L.ev) cudaEventRecord(L.ev[0], st);
  // the pruned search (5 + 2 split; teams of kBnbMinT+ lanes) has kernels
  // of its own, built for kBnbBlocks resident blocks per SM
  constexpr bool kBnb = bnb_search(L1, L2);
  const bool tf = L.one.cfg.T >= kTeamFinishMin;
  if (fused_tiles(L)) {
    if (L.ev) cudaEventRecord(L.ev[1], st);
    if (kBnb && tf)
      k_ground_state_bnb<CLOSED><<<search_blocks(L), kSearchThreads, 0, st>>>(L);
    else if (tf)
      k_ground_state<L1, L2, CLOSED, !kBnb><<<search_blocks(L), kSearchThreads, 0, st>>>(L);
    else
      k_ground_state<L1, L2, CLOSED, false><<<search_blocks(L), kSearchThreads, 0, st>>>(L);
    e = cudaGetLastError();
  } else {
    k_prep<CLOSED><<<prep_blocks(L), kPrepThreads, 0, st>>>(L);
    e = cudaGetLastError();
    if (L.ev) cudaEventRecord(L.ev[1], st);
    if (e == cudaSuccess) {
      if (kBnb && tf)
        e = launch_dependent(k_search_bnb<CLOSED>, (unsigned)search_blocks(L), kSearchThreads, st, L);
      else if (tf)
        e = launch_dependent(k_search<L1, L2, CLOSED, !kBnb>, (unsigned)search_blocks(L),
                             kSearchThreads, st, L);
      else
        e = launch_dependent(k_search<L1, L2, CLOSED, false>, (unsigned)search_blocks(L),
                             kSearchThreads, st, L);
    }
  }
  if (L.ev) cudaEventRecord(L.ev[2], st);
  if (e == cudaSuccess) e = launch_lists(L, st);
  if (L.ev) cudaEventRecord(L.ev[3], st);
  if (e == cudaSuccess) e = cudaGetLastError();
  // a chain cut short leaves the list heads set: clear them for the next call
  if (e != cudaSuccess) cudaMemsetAsync(L.cnt, 0, sizeof(Counters), st);
  return e;
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
  return key == 20 ? 0 : key == 40 ? 1 : key == 43 ? 2 : key == 54 ? 3 : key == 52 ? 4 : -1;
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
    case 4: return cl ? run<5, 2, true>(L, st) : run<5, 2, false>(L, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qa
