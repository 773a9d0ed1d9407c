// lb_batch.cu -- many independent lattices ("replicas") advanced together.  Each kernel of the
// coupled step runs once per step for ALL replicas of a batch: the lattice kernels walk a table
// of site tiles (every tile belongs to one replica and carries that replica's parameters), the
// particle kernels walk one concatenated particle array, and the particle sort works on one
// row space in which each replica owns a contiguous range of rows.  The kernels are persistent
// (a fixed grid walks the tables), and every count and pointer they need lives in device
// memory, so one CUDA graph of k steps stays valid while replicas join and leave; only the
// tables change.  A per-replica step budget lets replicas that finish freeze mid-graph.
//
// The arithmetic per site and per particle is the one of a single lattice (lb_site.cuh), and a
// replica's particles keep their relative order in the shared sort, so a replica gives the
// same bits alone and in any mix.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "lb_site.cuh"

using namespace lbmd;

namespace {

constexpr int kBThreads = 256;   // lattice kernels
constexpr int kBPThreads = 128;  // particle and row kernels
constexpr int kPairGrid = 4;     // the coupling's and the pair forces' grid, in particle grids

// ------------------------------------------------------------------ device tables

struct RepDev {      // per slot, written by the host when the replica's parameters change
  StepParams P;      // P.np = the replica's particle count
  void *pop[2];      // population buffers (element type P.storage); pop[state.cur] = current
  float *rest;       // 16-bit storage: FP32 rest populations [2][N]; NULL for FP32
  float *rho, *jp;   // [N][2] densities, [3][N] j'
  int diag_every;    // FP64 drift check every diag_every steps (0: off)
  double drift_tol;
};

struct RepState {    // per slot, advanced by the device at the end of each step
  int cur;           // which population buffer holds the current state
  unsigned err;      // device error bits of this replica
  unsigned long long step;  // steps taken (the particle noise counter)
  unsigned long long checked;  // step count of the last drift check (or of the reference)
  unsigned ref_req;  // set by the host: take the current totals as the drift reference
  unsigned pad;
};

struct RepLayout {   // per slot, written by the host at each repack
  int tile0;         // first tile of the replica in the tile table
  int row0;          // first row of the replica in the shared row space (-1: no particles)
  int p0;            // first slot of the replica in the particle arrays
  int pad;
};

struct BatchDev {
  int nrep, ntiles, nrows, np;
  int tile_sites;        // sites per tile
  const int *rep_slot;   // [nrep] slot of each replica in the tables
  const int *tile_slot;  // [ntiles] slot owning each tile
  const int *pslot;      // [np] slot owning each particle (constant between repacks)
  const RepDev *rep;     // [max_slots]
  RepState *state;       // [max_slots]
  const RepLayout *lay;  // [max_slots]
  int *left;             // [max_slots] steps still to take in the current lbmd_batch_step
  ParticleArrays U;      // particle state between steps
  ParticleArrays S;      // the same particles sorted by (row, x cell, id) during a step
  ParticleForces pf;     // forces, indexed like S (and like U after the update)
  int *row_of, *row_count, *row_start, *row_cursor, *bsum, *perm;
  double *tile_sums;     // [ntiles][5] FP64 sums of the drift check
  double *drift;         // [max_slots][10]: reference totals [5], last check {step, dA, dB, dP, n}
};

// ------------------------------------------------------------------ lattice kernels

// tuning != 0: time the update without side effects on the state -- no particle coupling (the
// sorted particle arrays are only valid inside a step) and, with 16-bit storage, the FP32 rest
// populations are not written (f_0 goes to the output buffer, which is scratch between steps).
// Per-block copy of what the kernels need for one replica's tile.  Kept in shared memory (and
// re-read there for every site) so that it takes no registers across the site update and is
// not reloaded from global memory after every store.
template <class T>
struct TileCtx {
  StepParams P;
  const T *fin;
  T *fout;
  const float *rest_in;
  float *rest_out;
  float *rho, *jp;
  unsigned *err;
  const int *row_start;  // the replica's rows in the shared row space; NULL: no particle coupling
  long long base;        // first site of the tile
  unsigned long long step;  // the replica's step count (noise counter)
  ParticleArrays pa;     // the sorted particles of the batch
  ParticleForces pf;
};

// The first tile at or after t, in steps of the grid, that this launch updates (ntiles if none):
// uniform across the block.
__device__ __forceinline__ int next_update_tile(const BatchDev *__restrict__ B, int t, bool mrt) {
  for (; t < B->ntiles; t += gridDim.x) {
    const int slot = B->tile_slot[t];
    if (B->left[slot] > 0 && (B->rep[slot].P.collision == LBMD_COLLISION_MRT) == mrt) break;
  }
  return t;
}

// Fill c for tile t of `slot` (all threads call it; the parameters are copied when the slot
// differs from `have`, the one c held).  No barrier: the caller orders it.
template <class T>
__device__ __forceinline__ void fill_tile(TileCtx<T> &c, const BatchDev *__restrict__ B, int t, int slot, int &have,
                                          int tuning) {
  if (slot != have) {
    const int *src = reinterpret_cast<const int *>(&B->rep[slot].P);
    int *dst = reinterpret_cast<int *>(&c.P);
    for (int k = threadIdx.x; k < (int)(sizeof(StepParams) / sizeof(int)); k += kBThreads) dst[k] = src[k];
  }
  if (threadIdx.x == 0) {
    const RepDev &R = B->rep[slot];
    const RepLayout &L = B->lay[slot];
    const int cur = B->state[slot].cur;
    c.fin = static_cast<const T *>(R.pop[cur]);
    c.fout = static_cast<T *>(R.pop[cur ^ 1]);
    c.rest_in = R.rest;
    c.rest_out = tuning ? nullptr : R.rest;
    c.rho = R.rho;
    c.jp = R.P.np > 0 ? R.jp : nullptr;
    c.err = &B->state[slot].err;
    c.row_start = (!tuning && R.P.np > 0) ? B->row_start + L.row0 : nullptr;
    c.base = (long long)(t - L.tile0) * B->tile_sites;
    c.step = B->state[slot].step;
    c.pa = B->S;
    c.pf = B->pf;
  }
  have = slot;
}

// The density pass over the tiles of the replicas still taking steps, with the tile contexts
// double-buffered like the update's.
__device__ __forceinline__ int next_live_tile(const BatchDev *__restrict__ B, int t) {
  for (; t < B->ntiles; t += gridDim.x)
    if (B->left[B->tile_slot[t]] > 0) break;
  return t;
}

template <class T>
__global__ void __launch_bounds__(kBThreads, 4) kb_moments(const BatchDev *__restrict__ B) {
  __shared__ TileCtx<T> cb[2];
  const int ts = B->tile_sites;
  int have0 = -1, have1 = -1;  // the slots whose parameters cb[0], cb[1] hold
  int t = next_live_tile(B, blockIdx.x);
  if (t >= B->ntiles) return;  // uniform across the block
  fill_tile(cb[0], B, t, B->tile_slot[t], have0, 0);
  __syncthreads();
  for (int b = 0; t < B->ntiles; b ^= 1) {
    const int tn = next_live_tile(B, t + gridDim.x);
    if (tn < B->ntiles) fill_tile(cb[b ^ 1], B, tn, B->tile_slot[tn], b ? have0 : have1, 0);
    const TileCtx<T> &c = cb[b];
    for (int k = threadIdx.x; k < ts; k += kBThreads) {
      const long long s = c.base + k;
      if (s >= c.P.N) break;
      site::moments<T>(c.P, s, c.fin, c.rest_in, c.rho, c.jp);
    }
    __syncthreads();  // the next context is complete; this one is free for the tile after it
    t = tn;
  }
}

// kMinBlocks: blocks per SM the register budget is sized for (3: 80 registers, some spilled; 2:
// up to 128 registers, none spilled) -- the autotuner picks.
// kMRT: this launch updates the replicas with the fluctuating MRT collision (and skips the BGK
// ones); the step runs both, each with its own register budget.
// The tile contexts are double-buffered: the next tile's is filled before this tile's sites are
// updated, and one barrier per tile publishes it (and frees this one).
template <class T, int kMinBlocks, bool kMRT>
__global__ void __launch_bounds__(kBThreads, kMinBlocks) kb_collide(const BatchDev *__restrict__ B, int tuning) {
  __shared__ TileCtx<T> cb[2];
  const int ts = B->tile_sites;
  int have0 = -1, have1 = -1;  // the slots whose parameters cb[0], cb[1] hold
  int t = next_update_tile(B, blockIdx.x, kMRT);
  if (t >= B->ntiles) return;  // uniform across the block
  fill_tile(cb[0], B, t, B->tile_slot[t], have0, tuning);
  __syncthreads();
  for (int b = 0; t < B->ntiles; b ^= 1) {
    const int tn = next_update_tile(B, t + gridDim.x, kMRT);
    if (tn < B->ntiles) fill_tile(cb[b ^ 1], B, tn, B->tile_slot[tn], b ? have0 : have1, tuning);
    const TileCtx<T> &c = cb[b];
    for (int k = threadIdx.x; k < ts; k += kBThreads) {
      const long long s = c.base + k;
      if (s >= c.P.N) break;
      if (c.row_start)
        site::collide<T, true, kMRT>(c.P, s, c.step, c.fin, c.fout, c.rho, c.pa, c.pf, CellIndex{c.row_start},
                                     c.err, c.rest_in, c.rest_out);
      else
        site::collide<T, false, kMRT>(c.P, s, c.step, c.fin, c.fout, c.rho, c.pa, c.pf, CellIndex{nullptr},
                                      c.err, c.rest_in, c.rest_out);
    }
    __syncthreads();  // the next context is complete; this one is free for the tile after it
    t = tn;
  }
}

// ------------------------------------------------------------------ particle sort

__global__ void __launch_bounds__(kBPThreads) kb_bin(const BatchDev *__restrict__ B) {
  const int np = B->np;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    const int slot = B->pslot[p];
    const StepParams &P = B->rep[slot].P;
    int4 c = B->U.cell[p];
    if (c.x < 0 || c.x >= P.nx || c.y < 0 || c.y >= P.ny || c.z < 0 || c.z >= P.nz) {
      atomicOr(&B->state[slot].err, kErrParticle);  // cannot happen for states written by this library
      c.x = wrapi(c.x, P.nx); c.y = wrapi(c.y, P.ny); c.z = wrapi(c.z, P.nz);
      B->U.cell[p] = c;
    }
    const int row = B->lay[slot].row0 + c.z * P.ny + c.y;
    B->row_of[p] = row;
    atomicAdd(B->row_count + row, 1);
  }
}

using site::block_exclusive_scan;
using site::kScanPerThread;
using site::kScanRows;
using site::kScanThreads;

// Exclusive scan of the row histogram in three passes (block sums of kScanRows rows, a scan of
// the block sums, in-block scans), each walking the blocks of rows with a fixed grid.  The final
// pass also clears the histogram for the next step.
__global__ void __launch_bounds__(kScanThreads) kb_scan_partial(const BatchDev *__restrict__ B) {
  __shared__ int wt[kScanThreads / 32];
  const int nrows = B->nrows, nb = (nrows + kScanRows - 1) / kScanRows;
  for (int blk = blockIdx.x; blk < nb; blk += gridDim.x) {
    const int base = blk * kScanRows + threadIdx.x * kScanPerThread;
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k)
      if (base + k < nrows) sum += B->row_count[base + k];
    int total;
    block_exclusive_scan(sum, wt, total);
    if (threadIdx.x == 0) B->bsum[blk] = total;
    __syncthreads();  // wt is reused by the next block of rows
  }
}

__global__ void __launch_bounds__(kScanThreads) kb_scan_top(const BatchDev *__restrict__ B) {
  __shared__ int wt[kScanThreads / 32];
  const int nb = (B->nrows + kScanRows - 1) / kScanRows;
  int *bsum = B->bsum;
  const int per = (nb + kScanThreads - 1) / kScanThreads;
  const int b = threadIdx.x * per;
  int sum = 0;
  for (int k = 0; k < per; ++k)
    if (b + k < nb) sum += bsum[b + k];
  int total;
  int run = block_exclusive_scan(sum, wt, total);
  for (int k = 0; k < per; ++k)
    if (b + k < nb) {
      const int c = bsum[b + k];
      bsum[b + k] = run;
      run += c;
    }
  if (threadIdx.x == 0) bsum[nb] = total;
}

__global__ void __launch_bounds__(kScanThreads) kb_scan_final(const BatchDev *__restrict__ B) {
  __shared__ int wt[kScanThreads / 32];
  const int nrows = B->nrows, nb = (nrows + kScanRows - 1) / kScanRows;
  int *count = B->row_count, *start = B->row_start, *cursor = B->row_cursor;
  for (int blk = blockIdx.x; blk < nb; blk += gridDim.x) {
    const int base = blk * kScanRows + threadIdx.x * kScanPerThread;
    int c[kScanPerThread];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
      c[k] = base + k < nrows ? count[base + k] : 0;
      sum += c[k];
    }
    int total;
    int run = B->bsum[blk] + block_exclusive_scan(sum, wt, total);
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k)
      if (base + k < nrows) {
        start[base + k] = run;
        cursor[base + k] = run;
        count[base + k] = 0;
        run += c[k];
      }
    if (blk == nb - 1 && threadIdx.x == 0) start[nrows] = B->bsum[nb];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kBPThreads) kb_scatter(const BatchDev *__restrict__ B) {
  const int np = B->np;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x)
    B->perm[atomicAdd(B->row_cursor + B->row_of[p], 1)] = p;
}

// Order each row by (x cell, particle id) -- ids are the replica's own, unique within a row.
__global__ void __launch_bounds__(kBPThreads) kb_row_sort(const BatchDev *__restrict__ B) {
  const int nrows = B->nrows;
  const int *start = B->row_start;
  int *perm = B->perm;
  const int4 *cell = B->U.cell;
  const int *pid = B->U.pid;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < nrows; row += gridDim.x * blockDim.x) {
    const int b = start[row], e = start[row + 1];
    for (int i = b + 1; i < e; ++i) {
      const int v = perm[i];
      const long long kv = ((long long)cell[v].x << 32) | (unsigned)pid[v];
      int j = i - 1;
      while (j >= b) {
        const int w = perm[j];
        const long long kw = ((long long)cell[w].x << 32) | (unsigned)pid[w];
        if (kw <= kv) break;
        perm[j + 1] = w;
        --j;
      }
      perm[j + 1] = v;
    }
  }
}

// S[j] = U[perm[j]].  A frozen replica's particles move too (their order can change once, in
// the first step after their last update), so their last total force travels with them, parked
// in the friction array, which no kernel computes for them.
__global__ void __launch_bounds__(kBPThreads) kb_permute(const BatchDev *__restrict__ B) {
  const int np = B->np;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < np; j += gridDim.x * blockDim.x) {
    const int p = B->perm[j];
    B->S.cell[j] = B->U.cell[p];
    B->S.frac[j] = B->U.frac[p];
    B->S.vel[j] = B->U.vel[p];
    B->S.pid[j] = B->U.pid[p];
    if (B->left[B->pslot[j]] <= 0) B->pf.fric[j] = B->pf.total[p];
  }
}

// ------------------------------------------------------------------ particle forces, update

// 8 lanes per particle (site::couple8); the 8 lanes of a particle stay together through the loop
__global__ void __launch_bounds__(kBPThreads) kb_couple(const BatchDev *__restrict__ B) {
  const int np = B->np;
  const int k = threadIdx.x & 7;
  const unsigned mask = 0xFFu << (threadIdx.x & 24);
  const int stride = (gridDim.x * blockDim.x) >> 3;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 3; p < np; p += stride) {
    const int slot = B->pslot[p];
    if (B->left[slot] <= 0) continue;
    const RepDev &R = B->rep[slot];
    const CellIndex ci{B->row_start + B->lay[slot].row0};
    site::couple8(R.P, B->state[slot].step, p, k, mask, B->S, B->S, ci, R.rho, R.jp, B->pf);
  }
}

// 8 lanes per particle (site::pairs8); the 8 lanes of a particle stay together through the loop
__global__ void __launch_bounds__(kBPThreads) kb_pairs(const BatchDev *__restrict__ B) {
  const int np = B->np;
  const int k = threadIdx.x & 7;
  const unsigned mask = 0xFFu << (threadIdx.x & 24);
  const int stride = (gridDim.x * blockDim.x) >> 3;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 3; p < np; p += stride) {
    const int slot = B->pslot[p];
    if (B->left[slot] <= 0) continue;
    const RepDev &R = B->rep[slot];
    const CellIndex ci{B->row_start + B->lay[slot].row0};
    site::pairs8(R.P, p, k, mask, B->S, ci, nullptr, nullptr, nullptr, B->pf, &B->state[slot].err);
  }
}

// S -> U: the update for replicas still stepping, a plain copy for frozen ones.
__global__ void __launch_bounds__(kBPThreads) kb_integrate(const BatchDev *__restrict__ B) {
  const int np = B->np;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    const int slot = B->pslot[p];
    if (B->left[slot] <= 0) {
      B->U.cell[p] = B->S.cell[p];
      B->U.frac[p] = B->S.frac[p];
      B->U.vel[p] = B->S.vel[p];
      B->U.pid[p] = B->S.pid[p];
      B->pf.total[p] = B->pf.fric[p];
      continue;
    }
    site::integrate(B->rep[slot].P, p, B->S, B->U, B->pf, &B->state[slot].err);
  }
}

// End of a step: replicas that stepped swap buffers and count the step; a replica with a device
// error stops (its remaining steps are dropped).
__global__ void kb_advance(const BatchDev *__restrict__ B) {
  for (int r = threadIdx.x; r < B->nrep; r += blockDim.x) {
    const int slot = B->rep_slot[r];
    if (B->left[slot] <= 0) continue;
    RepState &S = B->state[slot];
    S.cur ^= 1;
    S.step += 1;
    B->left[slot] = S.err ? 0 : B->left[slot] - 1;
  }
}

// ------------------------------------------------------------------ FP64 drift check

// A replica's totals are taken when the host asked for a reference, or after every diag_every
// steps (once per step count).  Both kernels below decide the same way from the same state.
__device__ __forceinline__ bool drift_due(const RepDev &R, const RepState &S) {
  return R.diag_every > 0 &&
         (S.ref_req || (S.step % (unsigned long long)R.diag_every == 0 && S.step != S.checked));
}

// FP64 sums [M_A, M_B, Px, Py, Pz] of every tile of the replicas due for a drift check, over
// the current buffer (streaming permutes populations, so the stored values sum alike).
template <class T>
__global__ void __launch_bounds__(kBThreads) kb_drift_sums(const BatchDev *__restrict__ B) {
  __shared__ double sh[5][kBThreads];
  // most steps have no replica due: one look at all replicas in parallel, instead of a chain of
  // dependent loads per tile
  bool any = false;
  for (int r = threadIdx.x; r < B->nrep; r += blockDim.x) {
    const int slot = B->rep_slot[r];
    any = any || drift_due(B->rep[slot], B->state[slot]);
  }
  if (!__syncthreads_or(any)) return;
  const int ts = B->tile_sites;
  for (int t = blockIdx.x; t < B->ntiles; t += gridDim.x) {
    const int slot = B->tile_slot[t];
    const RepDev &R = B->rep[slot];
    const RepState &S = B->state[slot];
    if (!drift_due(R, S)) continue;  // uniform across the block
    const StepParams &P = R.P;
    const T *f = static_cast<const T *>(R.pop[S.cur]);
    const long long base = (long long)(t - B->lay[slot].tile0) * ts;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < ts; k += kBThreads) {
      const long long s = base + k;
      if (s >= P.N) break;
      site::FloatPair m[5];  // the node's sums without rounding error; FP64 over nodes
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const float a = site::pop_read(P, f, R.rest, 0, i, s);
        const float b = site::pop_read(P, f, R.rest, 1, i, s);
        m[0].add(a);
        m[1].add(b);
        if (kCx[i]) { m[2].add(kCx[i] > 0 ? a : -a); m[2].add(kCx[i] > 0 ? b : -b); }
        if (kCy[i]) { m[3].add(kCy[i] > 0 ? a : -a); m[3].add(kCy[i] > 0 ? b : -b); }
        if (kCz[i]) { m[4].add(kCz[i] > 0 ? a : -a); m[4].add(kCz[i] > 0 ? b : -b); }
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) acc[q] += m[q].value();
    }
    __syncthreads();  // sh is free (previous tile)
#pragma unroll
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kBThreads / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w)
#pragma unroll
        for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < 5; ++k) B->tile_sums[(long long)t * 5 + k] = sh[k][0];
  }
}

// Per replica due: its tiles' sums plus the momentum of its particles, in a fixed order; then
// either the new reference or the comparison with it (kErrDrift beyond the tolerance: the
// replica takes no further step, like after any device error).
__global__ void __launch_bounds__(kBThreads) kb_drift_finish(const BatchDev *__restrict__ B) {
  __shared__ double sh[5][kBThreads];
  for (int r = blockIdx.x; r < B->nrep; r += gridDim.x) {
    const int slot = B->rep_slot[r];
    const RepDev &R = B->rep[slot];
    RepState &S = B->state[slot];
    if (!drift_due(R, S)) continue;  // uniform across the block
    const RepLayout &L = B->lay[slot];
    const int nt = (int)((R.P.N + B->tile_sites - 1) / B->tile_sites);
    double acc[5] = {0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < nt; t += kBThreads)
#pragma unroll
      for (int k = 0; k < 5; ++k) acc[k] += B->tile_sums[(long long)(L.tile0 + t) * 5 + k];
    for (int p = threadIdx.x; p < R.P.np; p += kBThreads) {
      const int q = L.p0 + p;
      const float4 v = B->U.vel[q];
      const double m = (double)R.P.types[B->U.cell[q].w].mass;
      acc[2] += m * v.x;
      acc[3] += m * v.y;
      acc[4] += m * v.z;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kBThreads / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w)
#pragma unroll
        for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double *ref = B->drift + (long long)slot * 10, *last = ref + 5;
      if (S.ref_req) {
        for (int k = 0; k < 5; ++k) ref[k] = sh[k][0];
        last[0] = -1.0;
        last[1] = last[2] = last[3] = last[4] = 0.0;
        S.ref_req = 0;
      } else {
        const double dA = fabs(sh[0][0] - ref[0]) / fabs(ref[0]), dB = fabs(sh[1][0] - ref[1]) / fabs(ref[1]);
        const double px = sh[2][0] - ref[2], py = sh[3][0] - ref[3], pz = sh[4][0] - ref[4];
        const double dP = sqrt(px * px + py * py + pz * pz) / (fabs(ref[0]) + fabs(ref[1]));
        last[0] = (double)S.step;
        last[1] = dA;
        last[2] = dB;
        last[3] = dP;
        last[4] += 1.0;
        if (!(dA <= R.drift_tol) || !(dB <= R.drift_tol) || !(dP <= R.drift_tol)) {
          S.err |= kErrDrift;
          B->left[slot] = 0;  // no further step in this call (kb_advance stops it for good)
        }
      }
      S.checked = S.step;
    }
  }
}

// Repack: dst[j] = src[src_of[j]] for src_of[j] >= 0 (the other slots are uploaded).
__global__ void kb_gather(int n, const int *__restrict__ src_of, ParticleArrays from, ParticleArrays to,
                          const float4 *__restrict__ tot_from, float4 *__restrict__ tot_to) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int p = src_of[j];
    if (p < 0) continue;
    to.cell[j] = from.cell[p];
    to.frac[j] = from.frac[p];
    to.vel[j] = from.vel[p];
    to.pid[j] = from.pid[p];
    tot_to[j] = tot_from[p];
  }
}

// ------------------------------------------------------------------ host side

struct Slot {
  bool used = false, fluid_ready = false, types_set = false;
  lbmd_params prm{};
  StepParams P{};
  unsigned char *pop[2] = {nullptr, nullptr};
  float *rest = nullptr, *rho = nullptr, *jp = nullptr;
  size_t bytes = 0;      // accounted against the batch budget
  int np_max = 0, np = 0;
  int64_t total = 0;     // requested number of steps
  int64_t queued = 0;    // steps enqueued so far (the device may stop earlier on an error)
  RepState mirror{};     // last state read from the device
  bool on_device = false;  // particles live in U at p0 (else pending on the host)
  std::vector<int4> hc;
  std::vector<float4> hf, hv;
  std::vector<int> hid;
  RepLayout lay{-1, -1, 0, 0};
  bool ref_pending = false;  // a drift reference is requested and not yet taken
};

constexpr size_t kParticleBytes = 2 * (16 + 16 + 16 + 4) + 6 * 16 + 3 * 4;  // U, S, forces, row_of/perm/pslot

size_t lattice_bytes(const StepParams &P, size_t elem) {
  const size_t N = (size_t)P.N;
  size_t b = 2 * (2 * kQ * N * elem);  // two population buffers
  if (elem == 2) b += 2 * N * 4;      // FP32 rest populations
  b += 2 * N * 4 + 3 * N * 4;         // densities, j'
  b += ((N + 255) / 256) * 4;         // tile table share (smallest tile)
  return b;
}

size_t particle_bytes(const StepParams &P, int np_max) {
  if (np_max <= 0) return 0;
  return (size_t)np_max * kParticleBytes * 5 / 4 + ((size_t)P.nrows + 1) * 3 * 4;  // 25 % capacity slack; rows
}

}  // namespace

struct lbmd_batch {
  int dev = 0, sms = 0;
  cudaStream_t st = nullptr;
  // the particle sort and the pair forces run on a side stream beside the density pass (joined
  // into st within every captured step; see enqueue_step)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_sorted = nullptr, ev_pairs = nullptr;
  bool own_stream = false;
  size_t budget = 0, used = 0;
  int storage = 0;
  size_t elem = 4;
  int max_slots = 0;
  cudaMemPool_t pool = nullptr;
  std::vector<Slot> slots;
  // device tables
  RepDev *d_rep = nullptr;
  RepState *d_state = nullptr;
  RepLayout *d_lay = nullptr;
  int *d_left = nullptr, *d_rep_slot = nullptr;
  BatchDev *d_batch = nullptr;
  BatchDev hb{};  // host copy of *d_batch
  int *d_tile_slot = nullptr;
  size_t tile_cap = 0;
  int pcap = 0;  // capacity of the particle arrays (U, S, forces, row_of, perm, pslot)
  int *d_pslot = nullptr;
  int rcap = 0;  // capacity of the row arrays (rows + 1)
  int bcap = 0;  // capacity of the block sums
  double *diag_partial = nullptr, *diag_out = nullptr;
  int diag_cap = 0;
  double *d_drift = nullptr;  // [max_slots][10] (BatchDev::drift)
  double *d_tile_sums = nullptr;  // [tile_cap][5] (BatchDev::tile_sums)
  bool dirty = true;
  // launch shape (autotuned)
  int tile_sites = 1024, grid_moments = 0, grid_collide = 0, grid_particles = 0;
  int collide_blocks = 3;  // register budget of the update kernel: blocks per SM
  // collisions among the replicas of the tables: bit 0 BGK, bit 1 MRT (the update launches only
  // the variants in use)
  int mix = 0;
  std::map<int, cudaGraphExec_t> graphs;  // by steps per graph and mix: 4 n + mix
  int64_t launches = 0;
  std::string msg;
};

namespace {

int bfail(lbmd_batch *b, int code, const std::string &m) {
  if (b) b->msg = m;
  else set_context_free_error(m);
  return code;
}

int bcuda(lbmd_batch *b, cudaError_t e, const char *where) {
  return bfail(b, e == cudaErrorMemoryAllocation ? LBMD_E_NOMEM : LBMD_E_CUDA,
               std::string(where) + ": " + cudaGetErrorString(e));
}

#define BK(call, where)                          \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return bcuda(b, e_, where); \
  } while (0)

template <class T>
cudaError_t palloc(lbmd_batch *b, T **p, size_t n) {
  *p = nullptr;
  if (n == 0) return cudaSuccess;
  return cudaMallocFromPoolAsync((void **)p, n * sizeof(T), b->pool, b->st);
}

template <class T>
void pfree(lbmd_batch *b, T *&p) {
  if (p) cudaFreeAsync((void *)p, b->st);
  p = nullptr;
}

void free_particle_set(lbmd_batch *b, ParticleArrays &a) {
  pfree(b, a.cell); pfree(b, a.frac); pfree(b, a.vel); pfree(b, a.pid);
}

void free_forces(lbmd_batch *b, ParticleForces &f) {
  pfree(b, f.fric); pfree(b, f.psA); pfree(b, f.psB); pfree(b, f.fsr); pfree(b, f.pair); pfree(b, f.total);
}

cudaError_t alloc_particle_set(lbmd_batch *b, ParticleArrays &a, int n) {
  cudaError_t e;
  if ((e = palloc(b, &a.cell, n)) != cudaSuccess) return e;
  if ((e = palloc(b, &a.frac, n)) != cudaSuccess) return e;
  if ((e = palloc(b, &a.vel, n)) != cudaSuccess) return e;
  return palloc(b, &a.pid, n);
}

cudaError_t alloc_forces(lbmd_batch *b, ParticleForces &f, int n) {
  cudaError_t e;
  if ((e = palloc(b, &f.fric, n)) != cudaSuccess) return e;
  if ((e = palloc(b, &f.psA, n)) != cudaSuccess) return e;
  if ((e = palloc(b, &f.psB, n)) != cudaSuccess) return e;
  if ((e = palloc(b, &f.fsr, n)) != cudaSuccess) return e;
  if ((e = palloc(b, &f.pair, n)) != cudaSuccess) return e;
  return palloc(b, &f.total, n);
}

int upload_rep(lbmd_batch *b, int slot) {
  Slot &s = b->slots[slot];
  RepDev r{};
  r.P = s.P;
  r.pop[0] = s.pop[0];
  r.pop[1] = s.pop[1];
  r.rest = s.rest;
  r.rho = s.rho;
  r.jp = s.jp;
  r.diag_every = s.prm.diag_every;
  r.drift_tol = s.prm.drift_tol;
  BK(cudaMemcpyAsync(b->d_rep + slot, &r, sizeof(RepDev), cudaMemcpyHostToDevice, b->st), "upload replica");
  return LBMD_OK;
}

int check_slot(lbmd_batch *b, int slot) {
  if (!b) return LBMD_E_INVALID_ARG;
  if (slot < 0 || slot >= b->max_slots || !b->slots[slot].used)
    return bfail(b, LBMD_E_INVALID_ARG, "slot " + std::to_string(slot) + " is not in use");
  cudaSetDevice(b->dev);
  return LBMD_OK;
}

// Wait for the stream and read every replica's device state.
int refresh(lbmd_batch *b) {
  BK(cudaStreamSynchronize(b->st), "cudaStreamSynchronize");
  std::vector<RepState> h(b->max_slots);
  BK(cudaMemcpy(h.data(), b->d_state, sizeof(RepState) * b->max_slots, cudaMemcpyDeviceToHost), "read states");
  for (int i = 0; i < b->max_slots; ++i)
    if (b->slots[i].used) b->slots[i].mirror = h[i];
  return LBMD_OK;
}

int slot_error_code(unsigned bits) {
  if (bits & kErrNonFinite) return LBMD_E_NONFINITE;
  if (bits & kErrNegDensity) return LBMD_E_NEGATIVE_DENSITY;
  if (bits & kErrBond) return LBMD_E_BOND_BROKEN;
  if (bits & kErrParticle) return LBMD_E_NONFINITE;
  if (bits & kErrDrift) return LBMD_E_DRIFT;
  return LBMD_OK;
}

// Rebuild the tile table for the replicas in `act` with the current tile size.
int build_tiles(lbmd_batch *b, const std::vector<int> &act) {
  std::vector<int> tiles;
  for (int s : act) {
    Slot &sl = b->slots[s];
    sl.lay.tile0 = (int)tiles.size();
    const long long nt = (sl.P.N + b->tile_sites - 1) / b->tile_sites;
    tiles.insert(tiles.end(), (size_t)nt, s);
  }
  if (tiles.size() > 0x7fffffffull) return bfail(b, LBMD_E_INVALID_ARG, "too many tiles");
  if (tiles.size() > b->tile_cap) {
    pfree(b, b->d_tile_slot);
    pfree(b, b->d_tile_sums);
    const size_t cap = tiles.size() + tiles.size() / 4;
    BK(palloc(b, &b->d_tile_slot, cap), "tile table");
    BK(palloc(b, &b->d_tile_sums, 5 * cap), "tile sums");
    b->tile_cap = cap;
  }
  if (!tiles.empty())
    BK(cudaMemcpyAsync(b->d_tile_slot, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice, b->st),
       "upload tiles");
  b->hb.ntiles = (int)tiles.size();
  b->hb.tile_sites = b->tile_sites;
  b->hb.tile_slot = b->d_tile_slot;
  b->hb.tile_sums = b->d_tile_sums;
  return LBMD_OK;
}

int upload_tables(lbmd_batch *b) {
  std::vector<RepLayout> lay(b->max_slots);
  for (int i = 0; i < b->max_slots; ++i) lay[i] = b->slots[i].lay;
  BK(cudaMemcpyAsync(b->d_lay, lay.data(), sizeof(RepLayout) * b->max_slots, cudaMemcpyHostToDevice, b->st),
     "upload layout");
  BK(cudaMemcpyAsync(b->d_batch, &b->hb, sizeof(BatchDev), cudaMemcpyHostToDevice, b->st), "upload batch");
  return LBMD_OK;
}

std::vector<int> active_slots(const lbmd_batch *b) {
  std::vector<int> act;
  for (int i = 0; i < b->max_slots; ++i)
    if (b->slots[i].used && b->slots[i].fluid_ready) act.push_back(i);
  return act;
}

// Lay the tables out again after replicas joined or left or changed their particles: particle
// ranges (moving the particles that stay, uploading new ones), row ranges, tiles.
int repack(lbmd_batch *b) {
  const std::vector<int> act = active_slots(b);
  // particles
  int np = 0;
  for (int s : act) np += b->slots[s].np;
  std::vector<int> src_of((size_t)np), pslot((size_t)np);
  {
    int j = 0;
    for (int s : act) {
      Slot &sl = b->slots[s];
      for (int k = 0; k < sl.np; ++k, ++j) {
        src_of[j] = sl.on_device ? sl.lay.p0 + k : -1;
        pslot[j] = s;
      }
    }
  }
  ParticleArrays dst = b->hb.S;
  float4 *dst_total = b->hb.pf.fric;  // scratch between steps
  const bool grow = np > b->pcap;
  BatchDev nb = b->hb;
  int *perm = b->hb.perm;
  if (grow) {
    const int cap = np + np / 4;
    nb.U = ParticleArrays{};
    nb.S = ParticleArrays{};
    nb.pf = ParticleForces{};
    nb.row_of = nb.perm = nullptr;
    int *pslot_new = nullptr;
    cudaError_t e;
    if ((e = alloc_particle_set(b, nb.U, cap)) != cudaSuccess || (e = alloc_particle_set(b, nb.S, cap)) != cudaSuccess ||
        (e = alloc_forces(b, nb.pf, cap)) != cudaSuccess || (e = palloc(b, &nb.row_of, cap)) != cudaSuccess ||
        (e = palloc(b, &nb.perm, cap)) != cudaSuccess || (e = palloc(b, &pslot_new, cap)) != cudaSuccess) {
      free_particle_set(b, nb.U); free_particle_set(b, nb.S); free_forces(b, nb.pf);
      pfree(b, nb.row_of); pfree(b, nb.perm); pfree(b, pslot_new);
      return bcuda(b, e, "particle arrays");
    }
    dst = nb.U;
    dst_total = nb.pf.total;
    perm = nb.perm;
    pfree(b, b->d_pslot);
    b->d_pslot = pslot_new;
  }
  if (np > 0) {
    BK(cudaMemcpyAsync(perm, src_of.data(), sizeof(int) * np, cudaMemcpyHostToDevice, b->st), "upload map");
    kb_gather<<<std::max(1, std::min(b->grid_particles, (np + kBPThreads - 1) / kBPThreads)), kBPThreads, 0, b->st>>>(
        np, perm, b->hb.U, dst, b->hb.pf.total, dst_total);
    BK(cudaGetLastError(), "gather");
    b->launches++;
  }
  if (grow) {
    free_particle_set(b, b->hb.U); free_particle_set(b, b->hb.S); free_forces(b, b->hb.pf);
    pfree(b, b->hb.row_of); pfree(b, b->hb.perm);
    b->hb.U = nb.U; b->hb.S = nb.S; b->hb.pf = nb.pf; b->hb.row_of = nb.row_of; b->hb.perm = nb.perm;
    b->pcap = np + np / 4;
  } else {
    std::swap(b->hb.U, b->hb.S);
    std::swap(b->hb.pf.total, b->hb.pf.fric);
  }
  // new particles, pslot, p0
  {
    int j = 0;
    for (int s : act) {
      Slot &sl = b->slots[s];
      sl.lay.p0 = j;
      if (!sl.on_device && sl.np > 0) {
        const ParticleArrays &U = b->hb.U;
        BK(cudaMemcpyAsync(U.cell + j, sl.hc.data(), sizeof(int4) * sl.np, cudaMemcpyHostToDevice, b->st), "upload");
        BK(cudaMemcpyAsync(U.frac + j, sl.hf.data(), sizeof(float4) * sl.np, cudaMemcpyHostToDevice, b->st), "upload");
        BK(cudaMemcpyAsync(U.vel + j, sl.hv.data(), sizeof(float4) * sl.np, cudaMemcpyHostToDevice, b->st), "upload");
        BK(cudaMemcpyAsync(U.pid + j, sl.hid.data(), sizeof(int) * sl.np, cudaMemcpyHostToDevice, b->st), "upload");
        BK(cudaMemsetAsync(b->hb.pf.total + j, 0, sizeof(float4) * sl.np, b->st), "clear forces");
      }
      sl.on_device = true;
      j += sl.np;
    }
    if (np > 0)
      BK(cudaMemcpyAsync(b->d_pslot, pslot.data(), sizeof(int) * np, cudaMemcpyHostToDevice, b->st), "upload pslot");
  }
  // rows (replicas with particles only)
  int nrows = 0;
  for (int s : act) {
    Slot &sl = b->slots[s];
    if (sl.np > 0) {
      sl.lay.row0 = nrows;
      nrows += sl.P.nrows;
    } else {
      sl.lay.row0 = 0;
    }
  }
  const int nbs = site::kScanRows;
  const int nblk = (nrows + nbs - 1) / nbs;
  if (nrows + 1 > b->rcap || nblk + 1 > b->bcap) {
    pfree(b, b->hb.row_count); pfree(b, b->hb.row_start); pfree(b, b->hb.row_cursor); pfree(b, b->hb.bsum);
    const int cap = nrows + 1 + nrows / 4;
    const int bcap = (cap + nbs - 1) / nbs + 1;
    BK(palloc(b, &b->hb.row_count, cap), "row arrays");
    BK(palloc(b, &b->hb.row_start, cap), "row arrays");
    BK(palloc(b, &b->hb.row_cursor, cap), "row arrays");
    BK(palloc(b, &b->hb.bsum, bcap), "row arrays");
    b->rcap = cap;
    b->bcap = bcap;
  }
  BK(cudaMemsetAsync(b->hb.row_count, 0, sizeof(int) * (nrows + 1), b->st), "clear rows");
  // replicas, tiles
  std::vector<int> rep_slot(act.begin(), act.end());
  if (!rep_slot.empty())
    BK(cudaMemcpyAsync(b->d_rep_slot, rep_slot.data(), sizeof(int) * rep_slot.size(), cudaMemcpyHostToDevice, b->st),
       "upload replicas");
  int r = build_tiles(b, act);
  if (r) return r;
  b->mix = 0;
  for (int s : act) b->mix |= b->slots[s].P.collision == LBMD_COLLISION_MRT ? 2 : 1;
  b->hb.nrep = (int)act.size();
  b->hb.np = np;
  b->hb.nrows = nrows;
  b->hb.pslot = b->d_pslot;
  r = upload_tables(b);
  if (r) return r;
  b->dirty = false;
  return LBMD_OK;
}

template <class F>
void with_batch_storage(int storage, F f) {
  switch (storage) {
    case LBMD_STORAGE_FP16_SHIFTED: f((__half *)nullptr); break;
    case LBMD_STORAGE_BF16_SHIFTED: f((__nv_bfloat16 *)nullptr); break;
    default: f((float *)nullptr); break;
  }
}

void launch_batched_moments(lbmd_batch *b, int grid) {
  with_batch_storage(b->storage, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    kb_moments<T><<<grid, kBThreads, 0, b->st>>>(b->d_batch);
  });
}

// The BGK replicas with the tuned shape, then the MRT ones (two blocks of 256 per SM: at three the
// tile context spills heavily); a variant no replica uses is not launched.  Returns the number of
// launches.
int launch_batched_collide(lbmd_batch *b, int grid, int min_blocks, int tuning) {
  int n = 0;
  with_batch_storage(b->storage, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    if (b->mix & 1) {
      if (min_blocks == 2)
        kb_collide<T, 2, false><<<grid, kBThreads, 0, b->st>>>(b->d_batch, tuning);
      else
        kb_collide<T, 3, false><<<grid, kBThreads, 0, b->st>>>(b->d_batch, tuning);
      ++n;
    }
    if (b->mix & 2) {
      kb_collide<T, 2, true><<<2 * b->sms, kBThreads, 0, b->st>>>(b->d_batch, tuning);
      ++n;
    }
  });
  return n;
}

// The drift check of the replicas due (two launches; a replica not due costs its tiles a test).
void launch_drift(lbmd_batch *b) {
  with_batch_storage(b->storage, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    kb_drift_sums<T><<<b->grid_moments, kBThreads, 0, b->st>>>(b->d_batch);
  });
  kb_drift_finish<<<2 * b->sms, kBThreads, 0, b->st>>>(b->d_batch);
}

// Enqueues one step; returns the number of kernel launches.
// The particle sort and the pair forces depend on the particles only: they run on the side
// stream beside the density pass, forked from st at the start of the step and joined before the
// coupling (sorted rows) and before the particle update (pair forces).
int enqueue_step(lbmd_batch *b) {
  const BatchDev *B = b->d_batch;
  const int gp = b->grid_particles;
  cudaStream_t sd = b->side;
  cudaEventRecord(b->ev_fork, b->st);
  cudaStreamWaitEvent(sd, b->ev_fork, 0);
  kb_bin<<<gp, kBPThreads, 0, sd>>>(B);
  kb_scan_partial<<<gp, site::kScanThreads, 0, sd>>>(B);
  kb_scan_top<<<1, site::kScanThreads, 0, sd>>>(B);
  kb_scan_final<<<gp, site::kScanThreads, 0, sd>>>(B);
  kb_scatter<<<gp, kBPThreads, 0, sd>>>(B);
  kb_row_sort<<<gp, kBPThreads, 0, sd>>>(B);
  kb_permute<<<gp, kBPThreads, 0, sd>>>(B);
  cudaEventRecord(b->ev_sorted, sd);
  launch_batched_moments(b, b->grid_moments);
  cudaStreamWaitEvent(b->st, b->ev_sorted, 0);
  // the coupling and the pair forces walk chains of dependent loads per particle: a grid of
  // kPairGrid times the particle grid (blocks beyond the resident ones queue) leaves each of their
  // threads about one particle instead of a few in a row
  kb_couple<<<kPairGrid * gp, kBPThreads, 0, b->st>>>(B);
  kb_pairs<<<kPairGrid * gp, kBPThreads, 0, sd>>>(B);
  cudaEventRecord(b->ev_pairs, sd);
  const int nc = launch_batched_collide(b, b->grid_collide, b->collide_blocks, 0);
  cudaStreamWaitEvent(b->st, b->ev_pairs, 0);
  kb_integrate<<<gp, kBPThreads, 0, b->st>>>(B);
  kb_advance<<<1, 256, 0, b->st>>>(B);
  launch_drift(b);
  return 14 + nc;
}

void drop_graphs(lbmd_batch *b) {
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
  b->graphs.clear();
}

// The graph of n steps for the current mix of collisions (captured once per n and mix);
// *launches receives its kernel launches.
int graph_for(lbmd_batch *b, int n, cudaGraphExec_t *out, int *launches) {
  const int key = 4 * n + b->mix;
  auto it = b->graphs.find(key);
  int per_step = 0;
  if (it != b->graphs.end()) {
    *out = it->second;
    *launches = n * (14 + ((b->mix & 1) != 0) + ((b->mix & 2) != 0));
    return LBMD_OK;
  }
  cudaGraph_t g = nullptr;
  BK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal), "begin capture");
  for (int k = 0; k < n; ++k) per_step = enqueue_step(b);
  cudaError_t e = cudaStreamEndCapture(b->st, &g);
  if (e != cudaSuccess) return bcuda(b, e, "end capture");
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bcuda(b, e, "instantiate graph");
  b->graphs[key] = x;
  *out = x;
  *launches = n * per_step;
  return LBMD_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

const char *lbmd_batch_last_error(const lbmd_batch *b) { return b ? b->msg.c_str() : lbmd_last_error(nullptr); }

void lbmd_batch_destroy(lbmd_batch *b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  cudaStreamSynchronize(b->st);
  drop_graphs(b);
  for (Slot &s : b->slots) {
    pfree(b, s.pop[0]); pfree(b, s.pop[1]); pfree(b, s.rest); pfree(b, s.rho); pfree(b, s.jp);
  }
  free_particle_set(b, b->hb.U); free_particle_set(b, b->hb.S); free_forces(b, b->hb.pf);
  pfree(b, b->hb.row_of); pfree(b, b->hb.perm); pfree(b, b->d_pslot);
  pfree(b, b->hb.row_count); pfree(b, b->hb.row_start); pfree(b, b->hb.row_cursor); pfree(b, b->hb.bsum);
  pfree(b, b->d_tile_slot);
  cudaStreamSynchronize(b->st);
  if (b->pool) cudaMemPoolDestroy(b->pool);
  cudaFree(b->d_rep); cudaFree(b->d_state); cudaFree(b->d_lay); cudaFree(b->d_left); cudaFree(b->d_rep_slot);
  pfree(b, b->d_tile_sums);
  cudaStreamSynchronize(b->st);
  cudaFree(b->d_batch); cudaFree(b->diag_partial); cudaFree(b->diag_out); cudaFree(b->d_drift);
  if (b->own_stream) cudaStreamDestroy(b->st);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_sorted) cudaEventDestroy(b->ev_sorted);
  if (b->ev_pairs) cudaEventDestroy(b->ev_pairs);
  delete b;
}

int lbmd_batch_create(size_t mem_budget, int storage, int max_slots, void *stream, lbmd_batch **out) {
  lbmd_batch *b = nullptr;
  if (!out) return bfail(b, LBMD_E_INVALID_ARG, "null output");
  *out = nullptr;
  if (storage != LBMD_STORAGE_FP32 && storage != LBMD_STORAGE_FP16_SHIFTED && storage != LBMD_STORAGE_BF16_SHIFTED)
    return bfail(b, LBMD_E_INVALID_ARG, "unknown storage");
  if (max_slots < 1 || max_slots > 65536) return bfail(b, LBMD_E_INVALID_ARG, "max_slots must be in [1, 65536]");
  b = new lbmd_batch();
  cudaGetDevice(&b->dev);
  cudaError_t e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev);
  if (e == cudaSuccess && !stream) {
    e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);  // capturable, unlike the legacy stream
    b->own_stream = e == cudaSuccess;
  } else {
    b->st = (cudaStream_t)stream;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_sorted, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_pairs, cudaEventDisableTiming);
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e == cudaSuccess) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = b->dev;
    e = cudaMemPoolCreate(&b->pool, &props);
  }
  if (e == cudaSuccess) {
    uint64_t keep = UINT64_MAX;  // keep freed blocks in the pool for the next replicas
    e = cudaMemPoolSetAttribute(b->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_rep, sizeof(RepDev) * max_slots);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_state, sizeof(RepState) * max_slots);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_lay, sizeof(RepLayout) * max_slots);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_left, sizeof(int) * max_slots);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_rep_slot, sizeof(int) * max_slots);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_batch, sizeof(BatchDev));
  if (e == cudaSuccess) e = cudaMalloc(&b->diag_partial, sizeof(double) * 8 * 1024);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_drift, sizeof(double) * 10 * max_slots);
  if (e == cudaSuccess) e = cudaMalloc(&b->diag_out, sizeof(double) * 8);
  if (e == cudaSuccess) e = cudaMemset(b->d_state, 0, sizeof(RepState) * max_slots);
  if (e == cudaSuccess) e = cudaMemset(b->d_left, 0, sizeof(int) * max_slots);
  if (e == cudaSuccess) e = cudaMemset(b->d_rep, 0, sizeof(RepDev) * max_slots);
  if (e != cudaSuccess) {
    cudaGetLastError();
    const std::string m = std::string("batch set-up: ") + cudaGetErrorString(e);
    lbmd_batch_destroy(b);
    return bfail(nullptr, e == cudaErrorMemoryAllocation ? LBMD_E_NOMEM : LBMD_E_CUDA, m);
  }
  b->budget = mem_budget ? mem_budget : (size_t)(0.9 * (double)free_b);
  b->storage = storage;
  b->elem = storage == LBMD_STORAGE_FP32 ? 4 : 2;
  b->max_slots = max_slots;
  b->slots.resize(max_slots);
  b->grid_moments = 4 * b->sms;
  b->grid_collide = 3 * b->sms;
  b->grid_particles = 8 * b->sms;
  b->hb = BatchDev{};
  b->hb.rep = b->d_rep;
  b->hb.state = b->d_state;
  b->hb.lay = b->d_lay;
  b->hb.left = b->d_left;
  b->hb.rep_slot = b->d_rep_slot;
  b->hb.tile_sites = b->tile_sites;
  b->hb.drift = b->d_drift;
  b->dirty = true;
  *out = b;
  return LBMD_OK;
}

int lbmd_batch_add(lbmd_batch *b, const lbmd_params *prm, int np_max, int64_t total_steps, int *slot,
                   unsigned *warnings) {
  if (!b || !prm || !slot) return b ? bfail(b, LBMD_E_INVALID_ARG, "null argument") : LBMD_E_INVALID_ARG;
  cudaSetDevice(b->dev);
  *slot = -1;
  if (warnings) *warnings = 0;
  std::string why;
  int r = check_params(prm, why);
  if (r) return bfail(b, r, why);
  if (prm->storage != b->storage) return bfail(b, LBMD_E_INVALID_ARG, "replica storage differs from the batch's");
  if (prm->md_substeps != 1) return bfail(b, LBMD_E_INVALID_ARG, "batches take md_substeps = 1 only");
  if (np_max < 0 || total_steps < 0) return bfail(b, LBMD_E_INVALID_ARG, "np_max and total_steps must be >= 0");
  StepParams P;
  fill_step_params(prm, P);
  const size_t need = lattice_bytes(P, b->elem) + particle_bytes(P, np_max);
  if (b->used + need > b->budget)
    return bfail(b, LBMD_E_NOMEM, "replica needs " + std::to_string(need) + " bytes; " + std::to_string(b->used) +
                                      " of the budget of " + std::to_string(b->budget) + " are in use");
  int s = -1;
  for (int i = 0; i < b->max_slots; ++i)
    if (!b->slots[i].used) {
      s = i;
      break;
    }
  if (s < 0) return bfail(b, LBMD_E_NOMEM, "all " + std::to_string(b->max_slots) + " slots are in use");
  Slot &sl = b->slots[s];
  sl = Slot{};
  sl.prm = *prm;
  sl.P = P;
  const size_t npop = (size_t)2 * kQ * P.N * b->elem;
  cudaError_t e;
  if ((e = palloc(b, &sl.pop[0], npop)) != cudaSuccess || (e = palloc(b, &sl.pop[1], npop)) != cudaSuccess ||
      (e = palloc(b, &sl.rho, (size_t)2 * P.N)) != cudaSuccess || (e = palloc(b, &sl.jp, (size_t)3 * P.N)) != cudaSuccess ||
      (b->elem == 2 && (e = palloc(b, &sl.rest, (size_t)2 * P.N)) != cudaSuccess)) {
    cudaGetLastError();
    pfree(b, sl.pop[0]); pfree(b, sl.pop[1]); pfree(b, sl.rho); pfree(b, sl.jp); pfree(b, sl.rest);
    sl = Slot{};
    return bfail(b, LBMD_E_NOMEM, std::string("replica allocation: ") + cudaGetErrorString(e));
  }
  sl.used = true;
  sl.bytes = need;
  sl.np_max = np_max;
  sl.total = total_steps;
  BK(cudaMemsetAsync(b->d_state + s, 0, sizeof(RepState), b->st), "clear state");
  BK(cudaMemsetAsync(b->d_left + s, 0, sizeof(int), b->st), "clear budget");
  r = upload_rep(b, s);
  if (r) return r;
  b->used += need;
  *slot = s;
  if (warnings) *warnings = param_warnings(prm);
  return LBMD_OK;
}

int lbmd_batch_remove(lbmd_batch *b, int slot) {
  int r = check_slot(b, slot);
  if (r) return r;
  Slot &sl = b->slots[slot];
  pfree(b, sl.pop[0]); pfree(b, sl.pop[1]); pfree(b, sl.rest); pfree(b, sl.rho); pfree(b, sl.jp);
  BK(cudaMemsetAsync(b->d_left + slot, 0, sizeof(int), b->st), "clear budget");
  b->used -= sl.bytes;
  const bool active = sl.fluid_ready;
  sl = Slot{};
  if (active) b->dirty = true;
  return LBMD_OK;
}

int lbmd_batch_set_types(lbmd_batch *b, int slot, int ntypes, const lbmd_ptype *types, int npairs,
                         const lbmd_pair *pairs, unsigned *warnings) {
  int r = check_slot(b, slot);
  if (r) return r;
  Slot &sl = b->slots[slot];
  unsigned w = 0;
  std::string why;
  if ((r = apply_types(sl.P, sl.prm.kT, sl.prm.dt, ntypes, types, npairs, pairs, w, why))) return bfail(b, r, why);
  sl.types_set = true;
  if (warnings) *warnings = w;
  return upload_rep(b, slot);
}

int lbmd_batch_set_debye_hueckel(lbmd_batch *b, int slot, double lB, double kappa_D, double rc) {
  int r = check_slot(b, slot);
  if (r) return r;
  std::string why;
  if ((r = apply_debye_hueckel(b->slots[slot].P, lB, kappa_D, rc, why))) return bfail(b, r, why);
  return upload_rep(b, slot);
}

int lbmd_batch_init_fluid(lbmd_batch *b, int slot, const float *rhoA, const float *rhoB, const float *u) {
  int r = check_slot(b, slot);
  if (r) return r;
  if (!rhoA || !rhoB) return bfail(b, LBMD_E_INVALID_ARG, "null density");
  Slot &sl = b->slots[slot];
  const long long N = sl.P.N;
  if (!densities_valid(rhoA, rhoB, N))
    return bfail(b, LBMD_E_INVALID_ARG, "densities must be finite and > 0");
  if (sl.fluid_ready && (r = refresh(b))) return r;  // the current buffer
  const int cur = sl.fluid_ready ? sl.mirror.cur : 0;
  float *stage = reinterpret_cast<float *>(sl.pop[1 - cur]);
  const size_t bytes = sizeof(float) * (size_t)N;
  BK(cudaMemcpyAsync(stage, rhoA, bytes, cudaMemcpyHostToDevice, b->st), "upload rhoA");
  BK(cudaMemcpyAsync(stage + N, rhoB, bytes, cudaMemcpyHostToDevice, b->st), "upload rhoB");
  const float *du = nullptr;
  if (u) {
    BK(cudaMemcpyAsync(stage + 2 * N, u, 3 * bytes, cudaMemcpyHostToDevice, b->st), "upload u");
    du = stage + 2 * N;
  }
  launch_init_equilibrium(sl.P, stage, stage + N, du, sl.pop[cur], sl.rest, b->st);
  BK(cudaGetLastError(), "init_equilibrium");
  b->launches++;
  const RepState st0{cur, 0u, 0ull, 0ull, sl.prm.diag_every > 0 ? 1u : 0u, 0u};
  sl.ref_pending = sl.prm.diag_every > 0;
  BK(cudaMemcpyAsync(b->d_state + slot, &st0, sizeof(RepState), cudaMemcpyHostToDevice, b->st), "reset state");
  // no check yet (lbmd_batch_get_drift before the first step: step -1, no checks)
  static const double kNoCheck[5] = {-1, 0, 0, 0, 0};
  BK(cudaMemcpyAsync(b->d_drift + (size_t)slot * 10 + 5, kNoCheck, sizeof(kNoCheck), cudaMemcpyHostToDevice, b->st),
     "reset drift");
  sl.mirror = st0;
  sl.queued = 0;
  if (!sl.fluid_ready) b->dirty = true;
  sl.fluid_ready = true;
  return LBMD_OK;
}

int lbmd_batch_set_particles(lbmd_batch *b, int slot, int n, const double *x, const double *v, const int *type,
                             const double *q) {
  int r = check_slot(b, slot);
  if (r) return r;
  Slot &sl = b->slots[slot];
  if (n < 0 || (n > 0 && (!x || !v || !type))) return bfail(b, LBMD_E_INVALID_ARG, "bad particle arrays");
  if (n > sl.np_max)
    return bfail(b, LBMD_E_INVALID_ARG, "n exceeds the np_max reserved when the replica was added");
  if (n > 0 && !sl.types_set) return bfail(b, LBMD_E_STATE, "set the particle types first");
  std::string why;
  std::vector<int4> hc;
  std::vector<float4> hf, hv;
  std::vector<int> hid;
  if ((r = convert_particles(sl.P, n, x, v, type, q, hc, hf, hv, hid, why))) return bfail(b, r, why);
  sl.hc.swap(hc); sl.hf.swap(hf); sl.hv.swap(hv); sl.hid.swap(hid);
  sl.np = n;
  sl.P.np = n;
  sl.on_device = false;
  b->dirty = true;
  if (sl.prm.diag_every > 0 && sl.fluid_ready) {  // the reference includes the new particles
    const unsigned one = 1u;
    BK(cudaMemcpyAsync(&b->d_state[slot].ref_req, &one, sizeof(unsigned), cudaMemcpyHostToDevice, b->st),
       "drift reference");
    sl.ref_pending = true;
  }
  return upload_rep(b, slot);
}

int lbmd_batch_step(lbmd_batch *b, int nsteps) {
  if (!b) return LBMD_E_INVALID_ARG;
  if (nsteps < 0) return bfail(b, LBMD_E_INVALID_ARG, "nsteps < 0");
  cudaSetDevice(b->dev);
  int r;
  if (b->dirty && (r = repack(b))) return r;
  std::vector<int> left(b->max_slots, 0);
  int most = 0;
  for (int i = 0; i < b->max_slots; ++i) {
    Slot &sl = b->slots[i];
    if (!sl.used || !sl.fluid_ready || sl.mirror.err) continue;  // a failed replica takes no more steps
    const int64_t k = std::min<int64_t>(nsteps, std::max<int64_t>(0, sl.total - sl.queued));
    left[i] = (int)k;
    sl.queued += k;
    most = std::max(most, (int)k);
  }
  if (most == 0) return LBMD_OK;
  // drift references asked for since the last step: taken on the state as it is now
  bool pending = false;
  for (Slot &sl : b->slots)
    if (sl.used && sl.ref_pending) {
      pending = true;
      sl.ref_pending = false;
    }
  if (pending) {
    launch_drift(b);
    BK(cudaGetLastError(), "drift reference");
    b->launches += 2;
  }
  BK(cudaMemcpyAsync(b->d_left, left.data(), sizeof(int) * b->max_slots, cudaMemcpyHostToDevice, b->st), "budgets");
  constexpr int kMaxGraphSteps = 16;
  const int chunk = std::min(most, kMaxGraphSteps);
  cudaGraphExec_t g = nullptr;
  int nl = 0;
  if ((r = graph_for(b, chunk, &g, &nl))) return r;
  for (int k = 0; k + chunk <= most; k += chunk) {
    BK(cudaGraphLaunch(g, b->st), "graph launch");
    b->launches += nl;
  }
  if (most % chunk) {
    if ((r = graph_for(b, most % chunk, &g, &nl))) return r;
    BK(cudaGraphLaunch(g, b->st), "graph launch");
    b->launches += nl;
  }
  return LBMD_OK;
}

int lbmd_batch_poll(lbmd_batch *b, int *status) {
  if (!b) return LBMD_E_INVALID_ARG;
  cudaSetDevice(b->dev);
  int r = refresh(b);
  if (r) return r;
  if (status)
    for (int i = 0; i < b->max_slots; ++i) {
      const Slot &sl = b->slots[i];
      if (!sl.used) status[i] = LBMD_SLOT_EMPTY;
      else if (sl.mirror.err) status[i] = LBMD_SLOT_FAILED;
      else if (sl.fluid_ready && (int64_t)sl.mirror.step >= sl.total) status[i] = LBMD_SLOT_DONE;
      else status[i] = LBMD_SLOT_ACTIVE;
    }
  return LBMD_OK;
}

int lbmd_batch_slot_error(const lbmd_batch *b, int slot) {
  if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot].used) return LBMD_E_INVALID_ARG;
  return slot_error_code(b->slots[slot].mirror.err);
}

int64_t lbmd_batch_step_count(const lbmd_batch *b, int slot) {
  if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot].used) return -1;
  return (int64_t)b->slots[slot].mirror.step;
}

int lbmd_batch_get_populations(lbmd_batch *b, int slot, int comp, float *f) {
  int r = check_slot(b, slot);
  if (r) return r;
  Slot &sl = b->slots[slot];
  if (!f || comp < 0 || comp > 1) return bfail(b, LBMD_E_INVALID_ARG, "bad arguments");
  if (!sl.fluid_ready) return bfail(b, LBMD_E_STATE, "fluid not initialised");
  if ((r = refresh(b))) return r;
  const int cur = sl.mirror.cur;
  float *stage = reinterpret_cast<float *>(sl.pop[1 - cur]);
  launch_unstream(sl.P, sl.pop[cur], sl.rest, comp, stage, b->st);
  BK(cudaGetLastError(), "unstream");
  BK(cudaMemcpyAsync(f, stage, sizeof(float) * kQ * (size_t)sl.P.N, cudaMemcpyDeviceToHost, b->st), "download f");
  BK(cudaStreamSynchronize(b->st), "sync");
  return LBMD_OK;
}

int lbmd_batch_get_fields(lbmd_batch *b, int slot, float *rhoA, float *rhoB, float *u) {
  int r = check_slot(b, slot);
  if (r) return r;
  Slot &sl = b->slots[slot];
  if (!sl.fluid_ready) return bfail(b, LBMD_E_STATE, "fluid not initialised");
  if ((r = refresh(b))) return r;
  const int cur = sl.mirror.cur;
  const long long N = sl.P.N;
  float *stage = reinterpret_cast<float *>(sl.pop[1 - cur]);
  launch_moments(sl.P, sl.pop[cur], sl.rest, sl.rho, nullptr, b->st);
  launch_fields(sl.P, sl.pop[cur], sl.rest, sl.rho, stage, stage + N, stage + 2 * N, b->st);
  BK(cudaGetLastError(), "fields");
  const size_t bytes = sizeof(float) * (size_t)N;
  if (rhoA) BK(cudaMemcpyAsync(rhoA, stage, bytes, cudaMemcpyDeviceToHost, b->st), "download");
  if (rhoB) BK(cudaMemcpyAsync(rhoB, stage + N, bytes, cudaMemcpyDeviceToHost, b->st), "download");
  if (u) BK(cudaMemcpyAsync(u, stage + 2 * N, 3 * bytes, cudaMemcpyDeviceToHost, b->st), "download");
  BK(cudaStreamSynchronize(b->st), "sync");
  return LBMD_OK;
}

int lbmd_batch_get_particles(lbmd_batch *b, int slot, double *x, double *v, double *f) {
  int r = check_slot(b, slot);
  if (r) return r;
  Slot &sl = b->slots[slot];
  const int n = sl.np;
  if (n == 0) return LBMD_OK;
  std::vector<int4> hc;
  std::vector<float4> hf, hv, ht;
  std::vector<int> hid;
  if (!sl.on_device) {  // not yet stepped: the values as set
    hc = sl.hc; hf = sl.hf; hv = sl.hv; hid = sl.hid;
    ht.assign(n, make_float4(0.f, 0.f, 0.f, 0.f));
  } else {
    if ((r = refresh(b))) return r;
    hc.resize(n); hf.resize(n); hv.resize(n); ht.resize(n); hid.resize(n);
    const ParticleArrays &U = b->hb.U;
    const int p0 = sl.lay.p0;
    BK(cudaMemcpyAsync(hc.data(), U.cell + p0, sizeof(int4) * n, cudaMemcpyDeviceToHost, b->st), "download");
    BK(cudaMemcpyAsync(hf.data(), U.frac + p0, sizeof(float4) * n, cudaMemcpyDeviceToHost, b->st), "download");
    BK(cudaMemcpyAsync(hv.data(), U.vel + p0, sizeof(float4) * n, cudaMemcpyDeviceToHost, b->st), "download");
    BK(cudaMemcpyAsync(ht.data(), b->hb.pf.total + p0, sizeof(float4) * n, cudaMemcpyDeviceToHost, b->st), "download");
    BK(cudaMemcpyAsync(hid.data(), U.pid + p0, sizeof(int) * n, cudaMemcpyDeviceToHost, b->st), "download");
    BK(cudaStreamSynchronize(b->st), "sync");
  }
  for (int j = 0; j < n; ++j) {
    const int id = hid[j];
    if (id < 0 || id >= n) return bfail(b, LBMD_E_CUDA, "corrupt particle ids");
    if (x) {
      x[3 * id] = hc[j].x + (double)hf[j].x;
      x[3 * id + 1] = hc[j].y + (double)hf[j].y;
      x[3 * id + 2] = hc[j].z + (double)hf[j].z;
    }
    if (v) {
      v[3 * id] = hv[j].x; v[3 * id + 1] = hv[j].y; v[3 * id + 2] = hv[j].z;
    }
    if (f) {
      f[3 * id] = ht[j].x; f[3 * id + 1] = ht[j].y; f[3 * id + 2] = ht[j].z;
    }
  }
  return LBMD_OK;
}

int lbmd_batch_diagnostics(lbmd_batch *b, int slot, double out[8]) {
  int r = check_slot(b, slot);
  if (r) return r;
  Slot &sl = b->slots[slot];
  if (!out) return bfail(b, LBMD_E_INVALID_ARG, "null output");
  if (!sl.fluid_ready) return bfail(b, LBMD_E_STATE, "fluid not initialised");
  if (b->dirty && (r = repack(b))) return r;
  if ((r = refresh(b))) return r;
  const int cur = sl.mirror.cur;
  const int nb = fluid_sum_blocks(sl.P);
  launch_fluid_sums(sl.P, sl.pop[cur], sl.rest, b->diag_partial, nb, b->st);
  launch_finish_sums(b->diag_partial, nb, 5, b->diag_out, b->st);
  double h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (sl.np > 0) {
    StepParams P = sl.P;
    const ParticleArrays &U = b->hb.U;
    const int p0 = sl.lay.p0;
    const ParticleArrays view{U.cell + p0, U.frac + p0, U.vel + p0, U.pid + p0};
    const int pb = std::min(1024, (sl.np + 255) / 256);
    launch_particle_momentum(P, view, b->diag_partial + 5 * 1024, pb, b->st);
    launch_finish_sums(b->diag_partial + 5 * 1024, pb, 3, b->diag_out + 5, b->st);
    BK(cudaGetLastError(), "sums");
    BK(cudaMemcpyAsync(h, b->diag_out, sizeof(double) * 8, cudaMemcpyDeviceToHost, b->st), "download");
  } else {
    BK(cudaGetLastError(), "sums");
    BK(cudaMemcpyAsync(h, b->diag_out, sizeof(double) * 5, cudaMemcpyDeviceToHost, b->st), "download");
  }
  BK(cudaStreamSynchronize(b->st), "sync");
  std::memcpy(out, h, sizeof(h));
  return LBMD_OK;
}

int lbmd_batch_get_drift(lbmd_batch *b, int slot, double out[5]) {
  int r = check_slot(b, slot);
  if (r) return r;
  if (!out) return bfail(b, LBMD_E_INVALID_ARG, "null output");
  if (!b->slots[slot].prm.diag_every) return bfail(b, LBMD_E_STATE, "the replica has no drift check (diag_every = 0)");
  double h[5];
  BK(cudaMemcpyAsync(h, b->d_drift + (size_t)slot * 10 + 5, sizeof(h), cudaMemcpyDeviceToHost, b->st), "download");
  BK(cudaStreamSynchronize(b->st), "sync");
  std::memcpy(out, h, sizeof(h));
  return LBMD_OK;
}

int lbmd_batch_set_config(lbmd_batch *b, int tile_sites, int grid_moments, int grid_collide, int collide_blocks) {
  if (!b) return LBMD_E_INVALID_ARG;
  if (collide_blocks != 2 && collide_blocks != 3) return bfail(b, LBMD_E_INVALID_ARG, "collide_blocks must be 2 or 3");
  if (tile_sites < kBThreads || tile_sites > 65536 || tile_sites % kBThreads)
    return bfail(b, LBMD_E_INVALID_ARG, "tile_sites must be a multiple of 256 in [256, 65536]");
  if (grid_moments < 1 || grid_collide < 1 || grid_moments > 64 * b->sms || grid_collide > 64 * b->sms)
    return bfail(b, LBMD_E_INVALID_ARG, "grid sizes must be in [1, 64 x SM count]");
  cudaSetDevice(b->dev);
  if (tile_sites != b->tile_sites) b->dirty = true;
  b->tile_sites = tile_sites;
  b->grid_moments = grid_moments;
  b->grid_collide = grid_collide;
  b->collide_blocks = collide_blocks;
  drop_graphs(b);
  return LBMD_OK;
}

int lbmd_batch_get_config(const lbmd_batch *b, int cfg[5]) {
  if (!b || !cfg) return LBMD_E_INVALID_ARG;
  cfg[0] = b->tile_sites;
  cfg[1] = b->grid_moments;
  cfg[2] = b->grid_collide;
  cfg[3] = b->collide_blocks;
  cfg[4] = b->grid_particles;
  return LBMD_OK;
}

int lbmd_batch_tune(lbmd_batch *b, int cfg[5], double ms[2]) {
  if (!b) return LBMD_E_INVALID_ARG;
  cudaSetDevice(b->dev);
  int r;
  if (b->dirty && (r = repack(b))) return r;
  const std::vector<int> act = active_slots(b);
  if (act.empty()) return bfail(b, LBMD_E_STATE, "no initialised replica to tune on");
  if ((r = refresh(b))) return r;
  std::vector<int> one(b->max_slots, 0);
  for (int s : act) one[s] = 1;
  BK(cudaMemcpyAsync(b->d_left, one.data(), sizeof(int) * b->max_slots, cudaMemcpyHostToDevice, b->st), "budgets");
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0), "event");
  BK(cudaEventCreate(&e1), "event");
  auto time_it = [&](auto launch) -> float {
    launch();  // warm-up
    cudaEventRecord(e0, b->st);
    constexpr int kReps = 3;
    for (int k = 0; k < kReps; ++k) launch();
    cudaEventRecord(e1, b->st);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    return t / kReps;
  };
  const int tiles[] = {256, 1024, 4096};
  const int gms[] = {2, 3, 4};
  static const int gcs_v[][2] = {{3, 1}, {3, 2}, {3, 3}, {2, 1}, {2, 2}};  // (blocks per SM budget, grid / SMs)
  const int *gcs[] = {gcs_v[0], gcs_v[1], gcs_v[2], gcs_v[3], gcs_v[4]};
  float best = 1e30f, best_m = 0.f, best_c = 0.f;
  int bt = b->tile_sites, bm = b->grid_moments, bc = b->grid_collide, bb = b->collide_blocks;
  const int saved_tile = b->tile_sites;
  for (int ts : tiles) {
    b->tile_sites = ts;
    if ((r = build_tiles(b, act)) || (r = upload_tables(b))) break;
    float tm = 1e30f, tc = 1e30f;
    int gm = 0, gc = 0, gb = 3;
    for (int g : gms) {
      const int grid = g * b->sms;
      const float t = time_it([&] { launch_batched_moments(b, grid); });
      if (t < tm) tm = t, gm = grid;
    }
    for (const int *v : gcs) {
      const int grid = v[1] * b->sms;
      const float t = time_it([&] { launch_batched_collide(b, grid, v[0], 1); });
      if (t < tc) tc = t, gc = grid, gb = v[0];
    }
    if (tm + tc < best) {
      best = tm + tc;
      best_m = tm;
      best_c = tc;
      bt = ts;
      bm = gm;
      bc = gc;
      bb = gb;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t e = cudaGetLastError();
  cudaMemsetAsync(b->d_left, 0, sizeof(int) * b->max_slots, b->st);
  if (r || e != cudaSuccess) {
    b->tile_sites = saved_tile;
    b->dirty = true;
    return r ? r : bcuda(b, e, "tuning launches");
  }
  b->tile_sites = bt;
  b->grid_moments = bm;
  b->grid_collide = bc;
  b->collide_blocks = bb;
  drop_graphs(b);
  if ((r = build_tiles(b, act)) || (r = upload_tables(b))) return r;
  BK(cudaStreamSynchronize(b->st), "sync");
  if (cfg) lbmd_batch_get_config(b, cfg);
  if (ms) {
    ms[0] = best_m;
    ms[1] = best_c;
  }
  return LBMD_OK;
}

int lbmd_batch_info(const lbmd_batch *b, size_t *budget, size_t *used, int *active, int *max_slots) {
  if (!b) return LBMD_E_INVALID_ARG;
  int n = 0;
  for (const Slot &s : b->slots) n += s.used ? 1 : 0;
  if (budget) *budget = b->budget;
  if (used) *used = b->used;
  if (active) *active = n;
  if (max_slots) *max_slots = b->max_slots;
  return LBMD_OK;
}

int64_t lbmd_batch_launch_count(const lbmd_batch *b) { return b ? b->launches : -1; }

}  // extern "C"
