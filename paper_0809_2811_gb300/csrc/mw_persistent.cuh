// mw_persistent.cuh -- persistent engine: one cooperative launch advances
// every box nsteps MD steps, with grid-wide barriers between the phases of
// mw_device.cuh (kick1 | [bin | scan | scan | scatter | copy + neighbour
// list] | force | kick2 + thermostat in the last block to arrive).  All blocks are
// co-resident (cooperative launch), every barrier wait is bounded in wall
// time, and the release of each barrier carries one status snapshot so that
// all blocks take the same decision to stop.  Data written in one phase is
// read by other blocks in a later phase of the same launch, so those reads
// are coherent loads (no ld.global.nc / __ldg anywhere in the phase bodies).
#pragma once

#include "mw_device.cuh"

namespace mw {

constexpr int kPersThreads = kFThreads;
// Co-resident blocks per SM the engine is compiled for (96 registers a
// thread): 7 or 8 (72 or 64 registers) measured slower on the two-box
// 32768-atom workload, and left to itself ptxas may take 128 (4 blocks).
constexpr int kPersBlocksPerSm = 5;

// Phase mark k of step s (block 0, thread 0; the SM clock): 0 step start,
// 1 kick1 done, 2 its barrier passed, 3 rebuild done, 4 force done, 5 its
// barrier passed, 6 kick2 done, 7 the last barrier passed (a launch's last
// step has none: block 0's arrival); on rebuild steps
// also 8 binning, 9 local scan, 10 scan offsets, 11 scatter, 12 copy-back,
// 13 neighbour lists done (each before its barrier).
__device__ __forceinline__ void phase_mark(const Dev& d, int s, int k) {
  if (d.marks && s < d.marks_cap && blockIdx.x == 0 && threadIdx.x == 0) d.marks[s * kPhaseMarks + k] = clock64();
}
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // default wait limit, 2 s (mw_set_wait_limit)

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier (one counter: a two-level counter tree measured slower on
// GB300, where the L2 round trips, ~3 us per barrier, dominate rather than
// atomic contention).  gen is this block's count of barriers passed (all
// blocks start from the same value).  Returns the status snapshot of the
// release (identical in every block), or ST_TIMEOUT if this block gave up
// waiting.
//
// Memory order (PTX memory model, gpu scope, no fences): __syncthreads orders
// every thread's writes of the phase before thread 0's arrival, an acq_rel
// add on the counter; the last arrival thus acquires all blocks' writes and
// publishes them again with a release store of the next generation, which
// the waiters read with acquire loads; the closing __syncthreads hands that
// order to the rest of each block.  In a barrier-only microbenchmark this
// took ~0.45 us less per barrier than __threadfence around relaxed atomics.

// The last arrival's release: reset the counter, snapshot the status, open
// generation gen + 1.  Returns the snapshot.
__device__ __forceinline__ int bar_release(Global* g, unsigned gen) {
  g->bar_count = 0u;
  const int st = *(volatile int*)&g->status;
  g->bar_stat[gen & 1u] = st;
  st_release(&g->bar_gen, gen + 1u);
  return st;
}

// A waiter: spin (bounded by limit_ns of wall time; a limit of 0 gives up at
// once) until generation gen is closed, then read its status snapshot.
__device__ __forceinline__ int bar_wait(Global* g, unsigned gen, unsigned long long limit_ns) {
  const unsigned long long t0 = globaltimer_ns();
  while (ld_acquire(&g->bar_gen) == gen) {
    if (globaltimer_ns() - t0 >= limit_ns) {
      set_status(g, ST_TIMEOUT);
      return ST_TIMEOUT;
    }
    __nanosleep(100);
  }
  return *(volatile int*)&g->bar_stat[gen & 1u];
}

__device__ int grid_barrier(Global* g, unsigned& gen, unsigned long long limit_ns) {
  __shared__ int s_status;
  __syncthreads();
  if (threadIdx.x == 0)
    s_status = (bar_arrive(&g->bar_count) == gridDim.x) ? bar_release(g, gen) : bar_wait(g, gen, limit_ns);
  __syncthreads();
  gen += 1u;
  return s_status;
}

// Grid barrier whose last arriving block runs fn() (all its threads) before
// the release, so that work that needs every block's results and that every
// block needs next costs no barrier of its own.  Same bounded waits, status
// snapshot and memory order as grid_barrier (fn's threads see the other
// blocks' writes through thread 0's acquire and the __syncthreads after it).
template <class Fn>
__device__ int grid_barrier_last(Global* g, unsigned& gen, unsigned long long limit_ns, Fn fn) {
  __shared__ int s_status;
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) s_last = (bar_arrive(&g->bar_count) == gridDim.x);
  __syncthreads();
  if (s_last) {
    fn();
    __syncthreads();
    if (threadIdx.x == 0) s_status = bar_release(g, gen);
  } else if (threadIdx.x == 0) {
    s_status = bar_wait(g, gen, limit_ns);
  }
  __syncthreads();
  gen += 1u;
  return s_status;
}

// The end of a launch: the last block to arrive runs fn() and resets the
// arrival count; the others return without waiting (no wait, so no limit).
// The launch's end publishes fn's writes to whatever runs next on the stream.
template <class Fn>
__device__ void end_arrive_last(Global* g, Fn fn) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) s_last = (bar_arrive(&g->bar_count) == gridDim.x);
  __syncthreads();
  if (s_last) {
    fn();
    __syncthreads();
    if (threadIdx.x == 0) g->bar_count = 0u;
  }
}

// Two-level exclusive scan of the cell counts over the grid: each block scans
// a contiguous chunk of cells (local prefix + chunk total), then adds the
// totals of the chunks before it.
__device__ void scan_chunk_local(const Dev& d) {
  __shared__ int wsum[kPersThreads / 32];
  __shared__ int carry;
  const int per = (d.ncell + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * per, c1 = min(d.ncell, c0 + per);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = c0; base < c1; base += kPersThreads) {
    const int c = base + threadIdx.x;
    const int v = (c < c1) ? d.cell_cnt[c] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int before = carry;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    if (c < c1) d.cell_start[c] = before + incl - v;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < kPersThreads / 32; ++w) tot += wsum[w];
      carry += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && blockIdx.x < d.chunk_cap) d.chunk[blockIdx.x] = carry;
}

__device__ void scan_chunk_offsets(const Dev& d) {
  __shared__ int red[kPersThreads / 32];
  const int per = (d.ncell + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * per, c1 = min(d.ncell, c0 + per);
  int part = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += kPersThreads) part += d.chunk[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(kFull, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  int off = 0;
  for (int w = 0; w < kPersThreads / 32; ++w) off += red[w];
  for (int c = c0 + threadIdx.x; c < c1; c += kPersThreads) {
    d.cell_start[c] += off;
    d.cell_cnt[c] = 0;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) d.cell_start[d.ncell] = off + d.chunk[blockIdx.x];
  __syncthreads();
}

// The same two halves as separate kernels, for the per-phase engines (the
// graph's rebuild body and the host-launched rebuilds): a grid of blocks in
// place of the single block of k_scan, whose one-block pass over every cell
// took tens of microseconds at 10^5 cells.  Grid size <= chunk_cap.
__global__ void __launch_bounds__(kPersThreads) k_scan_local(Dev d) {
  if (!d.g->any_rebuild || d.g->status) return;
  scan_chunk_local(d);
}
__global__ void __launch_bounds__(kPersThreads) k_scan_offsets(Dev d) {
  if (!d.g->any_rebuild || d.g->status) return;
  scan_chunk_offsets(d);
}

template <bool kCount, bool kNpt = false>
__global__ void __launch_bounds__(kPersThreads, kPersBlocksPerSm) k_persistent(const __grid_constant__ Dev d, const __grid_constant__ FParams P, int nsteps,
                                                                                        unsigned long long wait_ns) {
  __shared__ LegTable T;
  __shared__ unsigned s_gen;
  Global* g = d.g;
  if (threadIdx.x == 0) s_gen = *(volatile unsigned*)&g->bar_gen;
  __syncthreads();
  unsigned gen = s_gen;
  const Integ I = *d.integ;
  const unsigned long long step0 = g->step;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const int gw = tid >> 5, nwarps = nth >> 5;
  const int nblk = (d.N + kFAtoms - 1) / kFAtoms;
  for (int s = 0; s < nsteps; ++s) {
    const unsigned long long step = step0 + (unsigned long long)s;
    const int par = (int)(step & 1ull);
    phase_mark(d, s, 0);
    // a1 + a7 first half, a8 displacement check
    const int pend = *(volatile int*)&g->pend;  // stable: written only at the end of the kick2 phase
    if (tid == 0) g->n_over = 0;
    for (int i = tid; i < d.N; i += nth) kick1_atom<kNpt>(d, I, i, par, pend);
    phase_mark(d, s, 1);
    if constexpr (kNpt) {  // the new edges once every block has drifted with the old
      if (grid_barrier_last(g, gen, wait_ns, [&] {
            for (int b = threadIdx.x; b < d.nbox; b += blockDim.x) npt_commit_box(d, b);
          }))
        return;
    } else {
      if (grid_barrier(g, gen, wait_ns)) return;
    }
    phase_mark(d, s, 2);
    // a2 + a3: cell binning and neighbour list, when due (flag is stable until kick2)
    if (*(volatile int*)&g->any_rebuild) {
      if (tid == 0) g->max_count = 0;
      for (int i = tid; i < d.N; i += nth) bin_item(d, i);
      phase_mark(d, s, 8);
      if (grid_barrier(g, gen, wait_ns)) return;
      scan_chunk_local(d);
      phase_mark(d, s, 9);
      if (grid_barrier(g, gen, wait_ns)) return;
      scan_chunk_offsets(d);
      phase_mark(d, s, 10);
      if (grid_barrier(g, gen, wait_ns)) return;
      for (int i = tid; i < d.N; i += nth) scatter_item(d, i);
      phase_mark(d, s, 11);
      if (grid_barrier(g, gen, wait_ns)) return;
      for (int i = tid; i < d.N; i += nth) copyback_item(d, i);
      phase_mark(d, s, 12);
      {  // the warp's candidate staging slice aliases the leg table (idle until the force phase)
        static_assert(sizeof(LegTable) >= (kPersThreads / 32) * kNStage * sizeof(float4), "staging slices");
        float4* stg = reinterpret_cast<float4*>(&T) + (threadIdx.x >> 5) * kNStage;
        for (int c = gw; c < d.ncell; c += nwarps) neigh_cell_warp(d, d.tq, stg, c, P.rl2);
      }
      phase_mark(d, s, 13);
      if (tid < d.nbox && box_flagged(d, tid)) {
        d.bst[tid].rebuilds += 1;
        d.bst[tid].Lb = d.box[tid].L[0];
      }
      if (tid == 0) g->rebuild_steps += 1;
      if (grid_barrier(g, gen, wait_ns)) return;
    }
    phase_mark(d, s, 3);
    // a4 - a6: fused two- + three-body force, energy, virial
    if (tid == 0) g->wpar = par;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) force_block<kCount>(d, P, T, blk, par);
    phase_mark(d, s, 4);
    if (grid_barrier(g, gen, wait_ns)) return;
    phase_mark(d, s, 5);
    // a7 second half: kinetic energy of v + a per box; the rebuild (if any) is consumed
    if (blockIdx.x == 0) {
      for (int k = threadIdx.x; k < d.nbox; k += blockDim.x) d.bst[k].rebuild = 0;
      if (threadIdx.x == 0) g->any_rebuild = 0;
    }
    for (int i0 = blockIdx.x * kPersThreads; i0 < d.N; i0 += nth) {  // block-uniform
      float ke[1] = {0.f};
      int b = -1;
      ke[0] = kick2_atom(d, I, i0 + (int)threadIdx.x, b);
      box_accumulate<1>(ke, b, [&](int bb) { return &d.bst[bb].ke_acc[par]; });
    }
    phase_mark(d, s, 6);
    // the last block to arrive runs the thermostat halves of every box (end of
    // this step, start of the next) before releasing the others
    auto tail = [&] {
      for (int b = threadIdx.x; b < d.nbox; b += blockDim.x) end_of_step_box<kNpt>(d, I, b, par);
      if (threadIdx.x == 0) {
        g->pend = 1;
        g->step = step + 1ull;
      }
    };
    if (s == nsteps - 1) {
      // the launch's last step: nothing follows in this launch, so the other
      // blocks leave at once and the last one to arrive runs the tail (the
      // arrival count goes back to 0 as at a barrier)
      phase_mark(d, s, 7);
      end_arrive_last(g, tail);
      return;
    }
    if (grid_barrier_last(g, gen, wait_ns, tail)) return;
    phase_mark(d, s, 7);
  }
}

}  // namespace mw
