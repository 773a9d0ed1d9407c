// lb_particles.cu -- particle kernels of the coupled Shan-Chen LB / MD step (sm_103a):
// deterministic counting sort by lattice row, coupling forces (Eqs. NEWTON,
// solvation_kappa, solvation_lambda with trilinear interpolation), short-range pair and
// bonded forces (owner computes, no atomics), and the particle update.
#include "lb_site.cuh"

namespace lbmd {

namespace {

constexpr int kPBlock = 128;

inline unsigned pgrid(long long n) { return (unsigned)((n + kPBlock - 1) / kPBlock); }

// Lattice row (z, y) of each particle and the row histogram.
__global__ void k_bin(StepParams P, ParticleArrays pa, int *__restrict__ row_of, int *__restrict__ row_count,
                      unsigned *err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  int4 c = pa.cell[p];
  if (c.x < 0 || c.x >= P.nx || c.y < 0 || c.y >= P.ny || c.z < 0 || c.z >= P.nz) {
    atomicOr(err, kErrParticle);  // cannot happen for states written by this library
    c.x = wrapi(c.x, P.nx); c.y = wrapi(c.y, P.ny); c.z = wrapi(c.z, P.nz);
    pa.cell[p] = c;
  }
  const int row = c.z * P.ny + c.y;
  row_of[p] = row;
  atomicAdd(row_count + row, 1);
}

// Exclusive scan of the row histogram (rows -> first sorted slot) in three passes: per-block
// sums of 2048 rows, a scan of the block sums, and the in-block scans.  Also primes the
// scatter cursors.
using site::block_exclusive_scan;
using site::kScanThreads;
using site::kScanPerThread;
using site::kScanRows;

__global__ void __launch_bounds__(kScanThreads) k_scan_partial(int nrows, const int *__restrict__ count,
                                                               int *__restrict__ bsum) {
  __shared__ int wt[kScanThreads / 32];
  const int base = blockIdx.x * kScanRows + threadIdx.x * kScanPerThread;
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k)
    if (base + k < nrows) sum += count[base + k];
  int total;
  block_exclusive_scan(sum, wt, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int nb, int *__restrict__ bsum) {
  __shared__ int wt[kScanThreads / 32];
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

__global__ void __launch_bounds__(kScanThreads) k_scan_final(int nrows, int nb, const int *__restrict__ count,
                                                             const int *__restrict__ bsum, int *__restrict__ start,
                                                             int *__restrict__ cursor) {
  __shared__ int wt[kScanThreads / 32];
  const int base = blockIdx.x * kScanRows + threadIdx.x * kScanPerThread;
  int c[kScanPerThread];
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    c[k] = base + k < nrows ? count[base + k] : 0;
    sum += c[k];
  }
  int total;
  int run = bsum[blockIdx.x] + block_exclusive_scan(sum, wt, total);
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k)
    if (base + k < nrows) {
      start[base + k] = run;
      cursor[base + k] = run;
      run += c[k];
    }
  if (blockIdx.x == nb - 1 && threadIdx.x == 0) start[nrows] = bsum[nb];
}

__global__ void k_scatter(int np, const int *__restrict__ row_of, int *__restrict__ cursor, int *__restrict__ perm) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  perm[atomicAdd(cursor + row_of[p], 1)] = p;
}

// Order each row by (x cell, particle id) so the sort, and every gather after it, is
// deterministic.  Rows hold few particles: insertion sort, one thread per row.
__global__ void k_row_sort(StepParams P, const int *__restrict__ start, ParticleArrays pa, int *__restrict__ perm) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= P.nrows) return;
  const int b = start[row], e = start[row + 1];
  for (int i = b + 1; i < e; ++i) {
    const int v = perm[i];
    const long long kv = ((long long)pa.cell[v].x << 32) | (unsigned)pa.pid[v];
    int j = i - 1;
    while (j >= b) {
      const int w = perm[j];
      const long long kw = ((long long)pa.cell[w].x << 32) | (unsigned)pa.pid[w];
      if (kw <= kv) break;
      perm[j + 1] = w;
      --j;
    }
    perm[j + 1] = v;
  }
}

__global__ void k_permute(int np, const int *__restrict__ perm, ParticleArrays src, ParticleArrays dst,
                          int *__restrict__ slot_of_id) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  const int p = perm[j];
  dst.cell[j] = src.cell[p];
  dst.frac[j] = src.frac[p];
  dst.vel[j] = src.vel[p];
  const int id = src.pid[p];
  dst.pid[j] = id;
  slot_of_id[id] = j;
}

// The whole counting sort of a small system in one block: the steps of k_bin ... k_permute
// (histogram with the same range check, exclusive scan, scatter, order by (x cell, id) within a
// row, permutation) with the counts and the permutation in shared memory, one launch instead of
// a chain of seven that a step of a small lattice would wait for.  The order is unique, so the
// result is that of the chain.
constexpr int kSortSmallRows = 4096, kSortSmallNp = 2048;

__global__ void __launch_bounds__(kScanThreads) k_sort_small(StepParams P, ParticleArrays src, ParticleArrays dst,
                                                             int *__restrict__ start, int *__restrict__ slot_of_id,
                                                             unsigned *err) {
  __shared__ int count[kSortSmallRows];  // histogram, then the scatter cursors (= row ends)
  __shared__ int row_of[kSortSmallNp];
  __shared__ int perm[kSortSmallNp];
  __shared__ int wt[kScanThreads / 32];
  const int np = P.np, nrows = P.nrows;
  for (int r = threadIdx.x; r < nrows; r += kScanThreads) count[r] = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < np; p += kScanThreads) {
    int4 c = src.cell[p];
    if (c.x < 0 || c.x >= P.nx || c.y < 0 || c.y >= P.ny || c.z < 0 || c.z >= P.nz) {
      atomicOr(err, kErrParticle);  // cannot happen for states written by this library
      c.x = wrapi(c.x, P.nx); c.y = wrapi(c.y, P.ny); c.z = wrapi(c.z, P.nz);
      src.cell[p] = c;
    }
    const int row = c.z * P.ny + c.y;
    row_of[p] = row;
    atomicAdd(&count[row], 1);
  }
  __syncthreads();
  const int per = (nrows + kScanThreads - 1) / kScanThreads;  // consecutive rows of a thread
  const int b = threadIdx.x * per;
  int sum = 0;
  for (int k = 0; k < per; ++k)
    if (b + k < nrows) sum += count[b + k];
  int total;
  int run = block_exclusive_scan(sum, wt, total);
  for (int k = 0; k < per; ++k)
    if (b + k < nrows) {
      const int n = count[b + k];
      start[b + k] = run;
      count[b + k] = run;
      run += n;
    }
  if (threadIdx.x == 0) start[nrows] = total;
  __syncthreads();
  for (int p = threadIdx.x; p < np; p += kScanThreads) perm[atomicAdd(&count[row_of[p]], 1)] = p;
  __syncthreads();
  for (int r = threadIdx.x; r < nrows; r += kScanThreads) {  // row r holds slots [end of r-1, end of r)
    const int b0 = r == 0 ? 0 : count[r - 1], e0 = count[r];
    for (int i = b0 + 1; i < e0; ++i) {
      const int v = perm[i];
      const long long kv = ((long long)src.cell[v].x << 32) | (unsigned)src.pid[v];
      int j = i - 1;
      while (j >= b0) {
        const int w = perm[j];
        const long long kw = ((long long)src.cell[w].x << 32) | (unsigned)src.pid[w];
        if (kw <= kv) break;
        perm[j + 1] = w;
        --j;
      }
      perm[j + 1] = v;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < np; j += kScanThreads) {
    const int p = perm[j];
    dst.cell[j] = src.cell[p];
    dst.frac[j] = src.frac[p];
    dst.vel[j] = src.vel[p];
    const int id = src.pid[p];
    dst.pid[j] = id;
    slot_of_id[id] = j;
  }
}

// Coupling forces of every particle (site::couple).
__global__ void __launch_bounds__(kPBlock) k_couple(StepParams P, ParticleArrays pa, CellIndex ci,
                                                    const float *__restrict__ rho, const float *__restrict__ jp,
                                                    ParticleForces pf) {
  // 8 lanes per particle (site::couple8): the group of a particle returns together
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = (int)(t >> 3), k = (int)(t & 7);
  if (p >= P.np) return;
  site::couple8(P, noise_step(P, P.step), p, k, 0xFFu << (threadIdx.x & 24), pa, pa, ci, rho, jp, pf);
}

// k_couple with j' at each corner already formed (jc, 8 float4 per particle id).
__global__ void __launch_bounds__(kPBlock) k_couple_jc(StepParams P, ParticleArrays pa, CellIndex ci,
                                                       const float *__restrict__ rho, const float4 *__restrict__ jc,
                                                       ParticleForces pf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = (int)(t >> 3), k = (int)(t & 7);
  if (p >= P.np) return;
  site::couple8(P, noise_step(P, P.step), p, k, 0xFFu << (threadIdx.x & 24), pa, pa, ci, rho, nullptr, pf, true,
                jc);
}

// j' = sum_z sum_i f_zi c_i of the populations `store` at the 8 corners of every particle's cell,
// into jc[pid * 8 + corner] (the values k_couple_jc reads).
template <class T>
__global__ void __launch_bounds__(kPBlock) k_corner_jprime(StepParams P, ParticleArrays pa, int np,
                                                           const T *__restrict__ store, float4 *__restrict__ jc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 8LL * np) return;
  const int p = (int)(t >> 3), k = (int)(t & 7);
  const site::Coord cc = site::cell_corner(P, __ldg(pa.cell + p), k);
  const float3 j = site::jprime_at<T>(P, store, cc.x, cc.y, cc.z);
  jc[(long long)__ldg(pa.pid + p) * 8 + k] = make_float4(j.x, j.y, j.z, 0.f);
}

// Pair and bonded forces of every particle (site::pairs).
__global__ void __launch_bounds__(kPBlock) k_pairs(StepParams P, ParticleArrays pa, CellIndex ci,
                                                   const int *__restrict__ bond_start,
                                                   const int *__restrict__ bond_other,
                                                   const int *__restrict__ slot_of_id, ParticleForces pf,
                                                   unsigned *err) {
  // 8 lanes per particle (site::pairs8): the group of a particle returns together
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = (int)(t >> 3), k = (int)(t & 7);
  if (p >= P.np) return;
  site::pairs8(P, p, k, 0xFFu << (threadIdx.x & 24), pa, ci, bond_start, bond_other, slot_of_id, pf, err);
}

// Particle update (site::integrate) from src into dst, in the same order (dst may be src).
__global__ void k_integrate(StepParams P, ParticleArrays src, ParticleArrays dst, ParticleForces pf, unsigned *err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  site::integrate(P, p, src, dst, pf, err);
}

// ------------------------------------------------------------------ MD sub-stepping

// Coupling forces of substep `sub` at the particles' current positions C (in the order of the
// step's sorted list S, whose fluid-side solvation force stays frozen), then the substep's
// reaction record: position, friction and solvation forces over K, and the substep index in
// the cell's w (the fluid-side solvation force is taken from substep 0's records only).
__global__ void __launch_bounds__(kPBlock) k_couple_sub(StepParams P, ParticleArrays C, ParticleArrays S,
                                                        CellIndex ci, const float *__restrict__ rho,
                                                        const float *__restrict__ jp, ParticleForces pf, int sub,
                                                        ReactionRecords rec) {
  // 8 lanes per particle (site::couple8); lane 0, which wrote the forces, writes the records
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = (int)(t >> 3), k = (int)(t & 7);
  if (p >= P.np) return;
  site::couple8(P, noise_step(P, P.step), p, k, 0xFFu << (threadIdx.x & 24), C, S, ci, rho, jp, pf, sub == 0);
  if (k != 0) return;
  const float invK = 1.f / (float)P.substeps;
  const int r = sub * P.np + p;
  const int4 c = C.cell[p];
  rec.cell[r] = make_int4(c.x, c.y, c.z, c.w | (sub << 8));
  rec.frac[r] = C.frac[p];
  rec.key[r] = sub * P.np + C.pid[p];
  const float4 a = pf.fric[p], b = pf.psA[p], d = pf.psB[p];
  rec.fric[r] = make_float4(a.x * invK, a.y * invK, a.z * invK, 0.f);
  rec.psA[r] = make_float4(b.x * invK, b.y * invK, b.z * invK, 0.f);
  rec.psB[r] = make_float4(d.x * invK, d.y * invK, d.z * invK, 0.f);
}

// Particle update of one substep (P.dt = dt / K), in place, and the check that each particle
// is still within one cell of where the step started (the cell list of the step relies on it).
__global__ void k_integrate_sub(StepParams P, ParticleArrays C, ParticleArrays S, ParticleForces pf, unsigned *err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  site::integrate(P, p, C, C, pf, err);
  const int4 a = C.cell[p], b = S.cell[p];
  const int dx = site::min_image_cells(a.x - b.x, P.nx), dy = site::min_image_cells(a.y - b.y, P.ny),
            dz = site::min_image_cells(a.z - b.z, P.nz);
  if (dx > 1 || dx < -1 || dy > 1 || dy < -1 || dz > 1 || dz < -1) atomicOr(err, kErrTooFast);
}

__global__ void k_rec_permute(int n, const int *__restrict__ perm, ReactionRecords src, ReactionRecords dst) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int p = perm[j];
  dst.cell[j] = src.cell[p];
  dst.frac[j] = src.frac[p];
  dst.key[j] = src.key[p];
  dst.fric[j] = src.fric[p];
  dst.psA[j] = src.psA[p];
  dst.psB[j] = src.psB[p];
}

constexpr int kMomBlock = 256;
__global__ void __launch_bounds__(kMomBlock) k_particle_momentum(StepParams P, ParticleArrays pa,
                                                                 double *__restrict__ partial) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.np; p += gridDim.x * blockDim.x) {
    const float4 v = pa.vel[p];
    const double m = (double)P.types[pa.cell[p].w].mass;
    acc[0] += m * v.x;
    acc[1] += m * v.y;
    acc[2] += m * v.z;
  }
  __shared__ double sh[3][kMomBlock];
  for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kMomBlock / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) partial[(long long)blockIdx.x * 3 + k] = sh[k][0];
}

// Particle state in the caller's order: entry j of the sorted arrays is particle pa.pid[j], and
// total force j is that of particle tid_of[j].  The ids are a permutation of 0..n-1; an id out of
// range (which no step writes) is skipped rather than written out of bounds.
__global__ void __launch_bounds__(kPBlock) k_particles_out(int n, ParticleArrays pa, const int *__restrict__ tid_of,
                                                           const float4 *__restrict__ total, double *__restrict__ x,
                                                           double *__restrict__ v, double *__restrict__ f) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int id = pa.pid[j];
  if (id >= 0 && id < n) {
    if (x) {
      const int4 c = pa.cell[j];
      const float4 q = pa.frac[j];
      x[3LL * id] = c.x + (double)q.x;  // exact: an integer plus an FP32 fraction fits FP64
      x[3LL * id + 1] = c.y + (double)q.y;
      x[3LL * id + 2] = c.z + (double)q.z;
    }
    if (v) {
      const float4 w = pa.vel[j];
      v[3LL * id] = w.x;
      v[3LL * id + 1] = w.y;
      v[3LL * id + 2] = w.z;
    }
  }
  if (f) {
    const int t = tid_of[j];
    if (t >= 0 && t < n) {
      const float4 g = total[j];
      f[3LL * t] = g.x;
      f[3LL * t + 1] = g.y;
      f[3LL * t + 2] = g.z;
    }
  }
}

}  // namespace

void launch_bin(const StepParams &P, const ParticleArrays &pa, int *row_of, int *row_count, unsigned *err,
                cudaStream_t st) {
  k_bin<<<pgrid(P.np), kPBlock, 0, st>>>(P, pa, row_of, row_count, err);
}
int scan_blocks(int nrows) { return (nrows + kScanRows - 1) / kScanRows; }
void launch_scan_rows(int nrows, const int *row_count, int *row_start, int *row_cursor, int *bsum, cudaStream_t st) {
  const int nb = scan_blocks(nrows);
  k_scan_partial<<<nb, kScanThreads, 0, st>>>(nrows, row_count, bsum);
  k_scan_top<<<1, kScanThreads, 0, st>>>(nb, bsum);
  k_scan_final<<<nb, kScanThreads, 0, st>>>(nrows, nb, row_count, bsum, row_start, row_cursor);
}
bool sort_fits_one_block(int nrows, int np) { return nrows <= kSortSmallRows && np <= kSortSmallNp; }

void launch_sort_small(const StepParams &P, const ParticleArrays &src, const ParticleArrays &dst, int *row_start,
                       int *slot_of_id, unsigned *err, cudaStream_t st) {
  k_sort_small<<<1, kScanThreads, 0, st>>>(P, src, dst, row_start, slot_of_id, err);
}

void launch_scatter(int np, const int *row_of, int *row_cursor, int *perm, cudaStream_t st) {
  k_scatter<<<pgrid(np), kPBlock, 0, st>>>(np, row_of, row_cursor, perm);
}
void launch_row_sort(const StepParams &P, const int *row_start, const ParticleArrays &pa, int *perm,
                     cudaStream_t st) {
  k_row_sort<<<pgrid(P.nrows), kPBlock, 0, st>>>(P, row_start, pa, perm);
}
void launch_permute(int np, const int *perm, const ParticleArrays &src, const ParticleArrays &dst, int *slot_of_id,
                    cudaStream_t st) {
  k_permute<<<pgrid(np), kPBlock, 0, st>>>(np, perm, src, dst, slot_of_id);
}
void launch_couple(const StepParams &P, const ParticleArrays &pa, CellIndex ci, const float *rho, const float *jp,
                   const ParticleForces &pf, cudaStream_t st) {
  k_couple<<<pgrid(8LL * P.np), kPBlock, 0, st>>>(P, pa, ci, rho, jp, pf);
}
void launch_couple_jc(const StepParams &P, const ParticleArrays &pa, CellIndex ci, const float *rho,
                      const float4 *jc, const ParticleForces &pf, cudaStream_t st) {
  k_couple_jc<<<pgrid(8LL * P.np), kPBlock, 0, st>>>(P, pa, ci, rho, jc, pf);
}
void launch_corner_jprime(const StepParams &P, const ParticleArrays &pa, int np, const void *store, float4 *jc,
                          cudaStream_t st) {
  if (np <= 0) return;
  switch (P.storage) {
    case LBMD_STORAGE_FP16_SHIFTED:
      k_corner_jprime<__half><<<pgrid(8LL * np), kPBlock, 0, st>>>(P, pa, np, static_cast<const __half *>(store), jc);
      break;
    case LBMD_STORAGE_BF16_SHIFTED:
      k_corner_jprime<__nv_bfloat16><<<pgrid(8LL * np), kPBlock, 0, st>>>(
          P, pa, np, static_cast<const __nv_bfloat16 *>(store), jc);
      break;
    default:
      k_corner_jprime<float><<<pgrid(8LL * np), kPBlock, 0, st>>>(P, pa, np, static_cast<const float *>(store), jc);
  }
}
void launch_pairs(const StepParams &P, const ParticleArrays &pa, CellIndex ci, const int *bond_start,
                  const int *bond_other, const int *slot_of_id, const ParticleForces &pf, unsigned *err,
                  cudaStream_t st) {
  k_pairs<<<pgrid(8LL * P.np), kPBlock, 0, st>>>(P, pa, ci, bond_start, bond_other, slot_of_id, pf, err);
}
void launch_integrate(const StepParams &P, const ParticleArrays &src, const ParticleArrays &dst,
                      const ParticleForces &pf, unsigned *err, cudaStream_t st) {
  k_integrate<<<pgrid(P.np), kPBlock, 0, st>>>(P, src, dst, pf, err);
}
void launch_couple_sub(const StepParams &P, const ParticleArrays &C, const ParticleArrays &S, CellIndex ci,
                       const float *rho, const float *jp, const ParticleForces &pf, int sub,
                       const ReactionRecords &rec, cudaStream_t st) {
  k_couple_sub<<<pgrid(8LL * P.np), kPBlock, 0, st>>>(P, C, S, ci, rho, jp, pf, sub, rec);
}
void launch_integrate_sub(const StepParams &P, const ParticleArrays &C, const ParticleArrays &S,
                          const ParticleForces &pf, unsigned *err, cudaStream_t st) {
  k_integrate_sub<<<pgrid(P.np), kPBlock, 0, st>>>(P, C, S, pf, err);
}
void launch_rec_permute(int n, const int *perm, const ReactionRecords &src, const ReactionRecords &dst,
                        cudaStream_t st) {
  k_rec_permute<<<pgrid(n), kPBlock, 0, st>>>(n, perm, src, dst);
}
void launch_particle_momentum(const StepParams &P, const ParticleArrays &pa, double *partial, int nblocks,
                              cudaStream_t st) {
  k_particle_momentum<<<nblocks, kMomBlock, 0, st>>>(P, pa, partial);
}
void launch_particles_out(int n, const ParticleArrays &pa, const int *tid_of, const float4 *total, double *x,
                          double *v, double *f, cudaStream_t st) {
  k_particles_out<<<pgrid(n), kPBlock, 0, st>>>(n, pa, tid_of, total, x, v, f);
}

}  // namespace lbmd
