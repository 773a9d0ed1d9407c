// lbmd_internal.cuh -- device-side types, lattice constants and helpers shared by the
// sm_103a kernels of the coupled Shan-Chen LB / MD step.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fastdiv.h"
#include "lbmd.h"

namespace lbmd {

constexpr int kQ = 19;

// D3Q19 velocities (Eq. velo) in the ABI order: rest; +x,-x,+y,-y,+z,-z; then the xy, xz, yz
// face diagonals with opposite directions adjacent.
__device__ constexpr int kCx[kQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__device__ constexpr int kCy[kQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__device__ constexpr int kCz[kQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
// Weights (Eq. weights): 1/3, 1/18 (axis), 1/36 (diagonal).
__device__ constexpr float kW[kQ] = {1.f / 3.f,  1.f / 18.f, 1.f / 18.f, 1.f / 18.f, 1.f / 18.f,
                                     1.f / 18.f, 1.f / 18.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f,
                                     1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f,
                                     1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};
constexpr float kCs2 = 1.f / 3.f;

// device error word bits
constexpr unsigned kErrNegDensity = 1u << 0;
constexpr unsigned kErrNonFinite = 1u << 1;
constexpr unsigned kErrBond = 1u << 2;
constexpr unsigned kErrParticle = 1u << 3;
constexpr unsigned kErrTooFast = 1u << 4;  // a particle left its cell's neighbourhood within one sub-stepped step
constexpr unsigned kErrDrift = 1u << 5;    // the FP64 drift check found a conserved total beyond its tolerance

struct TypeParams {
  float kappa[2];   // Eq. (solvation_kappa)
  float lam[2];     // Eq. (solvation_lambda)
  float gamma;      // Eq. (NEWTON)
  float inv_mass;
  float noise_amp;  // sqrt(2 kT gamma / dt)
  float mass;
};

struct PairParams {
  float eps, sigma2, rc2, pad;  // WCA: epsilon, sigma^2, (2^(1/6) sigma)^2; eps = 0 -> none
};

// Everything a step needs, passed by value to every kernel.
struct StepParams {
  int nx, ny, nz;
  int nrows;             // ny * nz
  long long N;           // nx * ny * nz
  FastDiv divx, divy;    // division by nx and by ny (site index -> coordinates)
  float inv_tau;         // 1 / tau_r
  float force_pref;      // 1 - 1/(2 tau_r)  (the (2 + lambda)/2 factor of the forcing term)
  float gAB, gBA;
  float dt;
  int storage;           // LBMD_STORAGE_*
  float rho0[2];         // shift reference of the 16-bit storages (f_i - w_i rho0_z is stored)
  int np, ntypes;
  float dh_lB, dh_kappa, dh_rc2;
  int bond_kind;
  float bond_k, bond_r;
  int reach;             // cells to scan for pair forces: ceil(max interaction range)
  // fluctuating MRT (collision == LBMD_COLLISION_MRT): per mode k, relax[k] = 1 + lambda_k,
  // force[k] the factor of the forcing moment ((2 + lambda)/2 for the momenta, 2 + lambda for
  // the bulk and the normal shear modes, (2 + lambda)/2 for the off-diagonal ones), noise[k]
  // the amplitude over sqrt(rho_z) (over sqrt(rho_A rho_B / rho) for the momenta, k = 1..3)
  int collision;
  bool fluct;            // kT > 0: draw the mode noise
  // MD sub-stepping: K particle substeps per lattice step; the particle noise amplitude of a
  // substep is that of dt times sqrt(K) (noise_scale, 1 for K = 1)
  int substeps;
  float noise_scale;
  float relax[kQ], force[kQ], noise[kQ];
  unsigned long long seed, step;
  // the round keys of the fluid noise's generator (Philox4x32-10 under the key (seed lo, seed hi)):
  // round r uses the key plus r times the Weyl increments.  The same for every draw of a run, so
  // they are formed once on the host instead of per draw.
  uint2 noise_keys[10];
  // replayed step graphs: the particle kernels' noise counter is step + *step_base * step_mul,
  // the device-resident base being the lattice step at the replay's start (null: step alone);
  // the lattice update keeps its counter in `step` (patched into its graph node per replay)
  const unsigned long long *step_base;
  unsigned long long step_mul;
  TypeParams types[LBMD_MAX_TYPES];
  PairParams pairs[LBMD_MAX_TYPES * LBMD_MAX_TYPES];
};

// Particle state in sorted order (by lattice row (z, y), then x cell, then id).
struct ParticleArrays {
  int4 *cell;    // cx, cy, cz, type
  float4 *frac;  // fractional position in the cell (x, y, z) and charge q (w)
  float4 *vel;   // vx, vy, vz, 0
  int *pid;      // caller's particle index
};

// Per-particle forces of the current step (sorted order).
struct ParticleForces {
  float4 *fric;   // friction + noise (Eq. NEWTON)
  float4 *psA;    // -kappa_A grad rho_A
  float4 *psB;    // -kappa_B grad rho_B
  float4 *fsr;    // reaction of the fluid-side solvation force (minus what the particle exerts)
  float4 *pair;   // WCA + screened Coulomb + bonds
  float4 *total;  // sum, written by the integrator
};

// Momentum-return records of MD sub-stepping, one per particle and substep: position (cell with
// type | substep << 8 in w, fraction), a unique sort key (substep * np + id), and the friction
// and solvation forces divided by the number of substeps.
struct ReactionRecords {
  int4 *cell;
  float4 *frac;
  int *key;
  float4 *fric, *psA, *psB;
};

struct CellIndex {
  const int *row_start;  // [nrows + 1] offsets into the sorted particle arrays
};

// The one-pass lattice update: a block's warps own 8 consecutive rows (y) of a column tile of 32
// x nodes (one per lane) and the block marches along z through one chunk of planes of that tile;
// the blocks of a chunk cover neighbouring tiles and run together.  A node whose sources lie in
// other blocks gets its density from partial sums: each block writes what it holds for the node,
// and a second kernel adds the parts.  Where a lattice is too thin for that (edge rows of tiles
// with fewer than 3 rows or 2 columns; the planes of a lattice one plane deep) the second kernel
// pulls the node's populations instead, from a list of (row, x0, count) runs.
constexpr int kOnePassRows = 8;
constexpr int kOnePassCols = 32;
struct OnePassGeom {
  int ntx, nty;  // column tiles along x (kOnePassCols columns each) and y (kOnePassRows rows)
  int nchunks;   // z-chunks per tile: block b takes chunk b / (ntx nty) of tile b % (ntx nty)
  int ypart;     // every tile has >= 3 rows and >= 2 columns: the edge rows are finished from
                 // partial sums (else their densities are pulled)
  int zpart;     // nz >= 2: the first and last plane of each chunk are finished from partial sums
                 // (else pulled)
};
// Partial sums the update writes for nodes whose sources lie in other blocks.  A chunk-edge plane
// (the plane zs - 1 or zs at the boundary between the chunk below and the chunk starting at zs)
// gets its sources from two chunks: the upper chunk's part goes where an inner plane's does
// (rho_next, edge, yedge at the plane's index), the lower chunk's into the z arrays, at the slot
// 2 b + (0 for zs - 1, 1 for zs) of the boundary b = the upper chunk's index.
struct OnePassOut {
  float *edge;   // [nz][ny][ntx][2] float2: what leaves a tile row along x (side 0: -x, 1: +x)
  float *yedge;  // [2][nz][nty][ntx * 32] float2: what leaves a tile across its bottom (0) / top (1) row
  float *diag;   // [nz][nty][ntx][4] float2: the one value leaving each corner diagonally
  float *zown;   // [2 nchunks][ny][nx] float2: the lower chunk's sums at its own nodes
  float *zedge;  // [2 nchunks][ny][ntx][2] float2: its edge sums
  float *zyedge; // [2][2 nchunks][nty][ntx * 32] float2: its y-edge sums
};
struct BoundaryRun {
  int row;   // z * ny + y
  int x0;    // first node
  int n;     // nodes (at most kOnePassCols)
};

__host__ __device__ __forceinline__ int wrapi(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// The noise counter of a particle kernel given its own counter `step` (StepParams::step_base).
__device__ __forceinline__ unsigned long long noise_step(const StepParams &P, unsigned long long step) {
  return P.step_base ? step + *P.step_base * P.step_mul : step;
}

__device__ __forceinline__ long long site_index(const StepParams &P, int x, int y, int z) {
  return ((long long)z * P.ny + y) * P.nx + x;
}

// Geometric factor of Eq. (solvation_lambda): sum over the 18 neighbours of
// Theta[d_hat . c_hat] c / |c|^2 with Theta(x) = 1 for 0 < x < 1, tested exactly as
// d.c > 0 and d not parallel to c (d.c_hat = |d| iff parallel).
__device__ __forceinline__ float3 fs_geometry(float dx, float dy, float dz) {
  float3 s = make_float3(0.f, 0.f, 0.f);
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const float c2 = (float)(kCx[i] * kCx[i] + kCy[i] * kCy[i] + kCz[i] * kCz[i]);
    const float dc = dx * kCx[i] + dy * kCy[i] + dz * kCz[i];
    const float crx = dy * kCz[i] - dz * kCy[i];
    const float cry = dz * kCx[i] - dx * kCz[i];
    const float crz = dx * kCy[i] - dy * kCx[i];
    const bool parallel = (crx == 0.f) && (cry == 0.f) && (crz == 0.f);
    if (dc > 0.f && !parallel) {
      const float inv = 1.f / c2;
      s.x += kCx[i] * inv;
      s.y += kCy[i] * inv;
      s.z += kCz[i] * inv;
    }
  }
  return s;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): multipliers 0xD2511F53, 0xCD9E8D57,
// Weyl key increments 0x9E3779B9, 0xBB67AE85, ten rounds.
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = 0xD2511F53ull * c.x;
    const unsigned long long p1 = 0xCD9E8D57ull * c.z;
    const unsigned hi0 = (unsigned)(p0 >> 32), lo0 = (unsigned)p0;
    const unsigned hi1 = (unsigned)(p1 >> 32), lo1 = (unsigned)p1;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// The same generator with its ten round keys given (k_r of philox4x32_10's key schedule, r = 0 .. 9):
// for many draws under one key, with no key schedule per draw.
__device__ __forceinline__ uint4 philox4x32_10_keyed(uint4 c, const uint2 *__restrict__ rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = 0xD2511F53ull * c.x;
    const unsigned long long p1 = 0xCD9E8D57ull * c.z;
    const unsigned hi0 = (unsigned)(p0 >> 32), lo0 = (unsigned)p0;
    const unsigned hi1 = (unsigned)(p1 >> 32), lo1 = (unsigned)p1;
    c = make_uint4(hi1 ^ c.y ^ rk[r].x, lo1, hi0 ^ c.w ^ rk[r].y, lo0);
  }
  return c;
}

// Three standard normals for (seed, step, particle id): counter (id, step lo, step hi,
// 0x4c42), key (seed lo, seed hi); uniforms from the top 24 bits; Box-Muller.
__device__ __forceinline__ float3 particle_normals(unsigned long long seed, unsigned long long step,
                                                   unsigned id) {
  const uint4 r = philox4x32_10(make_uint4(id, (unsigned)step, (unsigned)(step >> 32), 0x4c42u),
                                make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  const float s = 1.f / 16777216.f;
  const float u0 = ((float)(r.x >> 8) + 0.5f) * s, u1 = ((float)(r.y >> 8) + 0.5f) * s;
  const float u2 = ((float)(r.z >> 8) + 0.5f) * s, u3 = ((float)(r.w >> 8) + 0.5f) * s;
  const float a = sqrtf(-2.f * logf(u0)), b = sqrtf(-2.f * logf(u2));
  float s1, c1, s3, c3;
  sincospif(2.f * u1, &s1, &c1);
  sincospif(2.f * u3, &s3, &c3);
  return make_float3(a * c1, a * s1, b * c3);
}

// Message returned by lbmd_last_error(NULL) (calls made without a context).
void set_context_free_error(const std::string &m);

// Argument handling shared by single contexts and batches (lbmd_api.cu).  Each returns LBMD_OK or
// an LBMD_E_* code with the reason in `why`; nothing is changed on failure.
int check_params(const lbmd_params *prm, std::string &why);
void fill_step_params(const lbmd_params *prm, StepParams &P);
unsigned param_warnings(const lbmd_params *prm);
// Every density of both fields finite and > 0 (one branch-free pass the host compiler vectorises).
bool densities_valid(const float *rhoA, const float *rhoB, long long n);
int apply_types(StepParams &P, double kT, double dt, int ntypes, const lbmd_ptype *types, int npairs,
                const lbmd_pair *pairs, unsigned &warnings, std::string &why);
int apply_debye_hueckel(StepParams &P, double lB, double kappa_D, double rc, std::string &why);
int convert_particles(const StepParams &P, int n, const double *x, const double *v, const int *type,
                      const double *q, std::vector<int4> &cell, std::vector<float4> &frac,
                      std::vector<float4> &vel, std::vector<int> &id, std::string &why);

// ------------------------------------------------------------------ launch wrappers
// lattice (lb_fluid.cu); population buffers are void*: their element type is P.storage.  With
// 16-bit storage `rest` is the FP32 array [2][N] of the rest populations (NULL for FP32).
void launch_init_equilibrium(const StepParams &P, const float *rhoA, const float *rhoB, const float *u,
                             void *store, float *rest, cudaStream_t st);
void launch_restream(const StepParams &P, const float *post, int comp, void *store, float *rest, cudaStream_t st);
void launch_unstream(const StepParams &P, const void *store, const float *rest, int comp, float *post,
                     cudaStream_t st);
void launch_moments(const StepParams &P, const void *store, const float *rest, float *rho, float *jp,
                    cudaStream_t st);
void launch_collide(const StepParams &P, const void *fin, void *fout, float *rest, const float *rho,
                    const ParticleArrays &pa, const ParticleForces &pf, CellIndex ci, unsigned *err,
                    cudaStream_t st);
// One-pass update (BGK, md_substeps = 1): writes the populations of the next step, the densities
// rho_next of the nodes whose sources are all in one block, and the partial sums of `out` for the
// others; launch_boundary_densities then finishes those.
void launch_collide_onepass(const StepParams &P, const void *fin, void *fout, float *rest, const float *rho,
                            float *rho_next, OnePassOut out, const ParticleArrays &pa, const ParticleForces &pf,
                            CellIndex ci, unsigned *err, OnePassGeom G, int grid, cudaStream_t st);
// Adds the partial sums of `out` where they belong and pulls the densities of the listed boundary
// runs from the new populations, in one launch.  zslot[z]: -1 where z is neither the first nor the
// last plane of its chunk, else its slot in the z arrays of `out`.  With jc (not NULL), the same
// launch also forms j' of the new populations at the 8 corners of the cells of the np particles
// pn, into jc[pid * 8 + corner] (what launch_couple_jc reads).
void launch_boundary_densities(const StepParams &P, OnePassGeom G, const void *store, const float *rest,
                               float *rho_next, const BoundaryRun *runs, int nruns, OnePassOut out,
                               const int *zslot, const ParticleArrays &pn, int np, float4 *jc, cudaStream_t st);
// Blocks of the one-pass update resident on one SM (its persistent grid is this times the SMs).
int onepass_blocks_per_sm();
void launch_fields(const StepParams &P, const void *store, const float *rest, const float *rho, float *rhoA,
                   float *rhoB, float *u, cudaStream_t st);
void launch_fluid_sums(const StepParams &P, const void *store, const float *rest, double *partial, int nblocks,
                       cudaStream_t st);
void launch_finish_sums(const double *partial, int nblocks, int nvals, double *out, cudaStream_t st);
// Replayed step graphs.  The lattice update with the fluctuating MRT collision draws its noise
// with the counter in its parameter bank (a counter read from memory would hold a register pair
// through the update and spill): is_noisy_update tells its kernels, set_update_step writes the
// counter into a node of an instantiated graph.  The particle kernels read the device-resident
// step base, set or advanced by the two launches below.
bool is_noisy_update(const void *fn);
cudaError_t set_update_step(cudaGraphExec_t exec, cudaGraphNode_t node, unsigned long long step);
void launch_set_step(unsigned long long *base, unsigned long long value, cudaStream_t st);
void launch_advance_step(unsigned long long *base, unsigned long long n, cudaStream_t st);
int fluid_sum_blocks(const StepParams &P);
// The FP64 drift check: compares the totals [M_A, M_B, Px, Py, Pz] of the fluid (sums[0..4])
// plus the particle momentum (psum[0..2], NULL: no particles) with ref[5].  set_ref != 0: take
// them as the new reference (last[4] = 0).  Otherwise last[] = {step, drift of M_A, of M_B,
// momentum drift per unit mass, checks so far} and kErrDrift goes to err when a drift exceeds
// tol.  One thread; reads and writes device memory only.
void launch_drift_check(const double *sums, const double *psum, double *ref, double *last, unsigned *err,
                        long long step, double tol, int set_ref, cudaStream_t st);

// particles (lb_particles.cu)
void launch_bin(const StepParams &P, const ParticleArrays &pa, int *row_of, int *row_count,
                unsigned *err, cudaStream_t st);
int scan_blocks(int nrows);  // size of the block-sum scratch is scan_blocks(nrows) + 1
void launch_scan_rows(int nrows, const int *row_count, int *row_start, int *row_cursor, int *bsum, cudaStream_t st);
void launch_scatter(int np, const int *row_of, int *row_cursor, int *perm, cudaStream_t st);
// The particle sort of a small system (nrows and np within one block's shared memory) in one
// launch: row_start and the sorted copy dst of src, as the chain bin ... permute gives them.
bool sort_fits_one_block(int nrows, int np);
void launch_sort_small(const StepParams &P, const ParticleArrays &src, const ParticleArrays &dst, int *row_start,
                       int *slot_of_id, unsigned *err, cudaStream_t st);
void launch_row_sort(const StepParams &P, const int *row_start, const ParticleArrays &pa, int *perm,
                     cudaStream_t st);
void launch_permute(int np, const int *perm, const ParticleArrays &src, const ParticleArrays &dst,
                    int *slot_of_id, cudaStream_t st);
void launch_couple(const StepParams &P, const ParticleArrays &pa, CellIndex ci, const float *rho,
                   const float *jp, const ParticleForces &pf, cudaStream_t st);
// The same with j' at the corners from jc (8 float4 per particle id, launch_corner_jprime or the
// one-pass update's boundary kernel).
void launch_couple_jc(const StepParams &P, const ParticleArrays &pa, CellIndex ci, const float *rho,
                      const float4 *jc, const ParticleForces &pf, cudaStream_t st);
// j' of the populations `store` (element type P.storage) at the 8 corners of the cells of the np
// particles pa, into jc[pid * 8 + corner].
void launch_corner_jprime(const StepParams &P, const ParticleArrays &pa, int np, const void *store, float4 *jc,
                          cudaStream_t st);
void launch_pairs(const StepParams &P, const ParticleArrays &pa, CellIndex ci, const int *bond_start,
                  const int *bond_other, const int *slot_of_id, const ParticleForces &pf, unsigned *err,
                  cudaStream_t st);
void launch_integrate(const StepParams &P, const ParticleArrays &src, const ParticleArrays &dst,
                      const ParticleForces &pf, unsigned *err, cudaStream_t st);
// Positions (cell + fraction, in FP64), velocities and the total forces of the last step of n
// particles into device arrays [n][3] in the caller's particle order; any output may be null.
// tid_of: the caller's index of each entry of total (the order the particle update wrote them).
void launch_particles_out(int n, const ParticleArrays &pa, const int *tid_of, const float4 *total, double *x,
                          double *v, double *f, cudaStream_t st);
// True if [p, p + bytes) is device (or managed) memory inside one allocation of the current
// context (checked with the runtime's pointer attributes and the driver's allocation extent).
bool device_buffer_ok(const void *p, size_t bytes);
void launch_particle_momentum(const StepParams &P, const ParticleArrays &pa, double *partial, int nblocks,
                              cudaStream_t st);
// MD sub-stepping (lb_particles.cu)
void launch_couple_sub(const StepParams &P, const ParticleArrays &C, const ParticleArrays &S, CellIndex ci,
                       const float *rho, const float *jp, const ParticleForces &pf, int sub,
                       const ReactionRecords &rec, cudaStream_t st);
void launch_integrate_sub(const StepParams &P, const ParticleArrays &C, const ParticleArrays &S,
                          const ParticleForces &pf, unsigned *err, cudaStream_t st);
void launch_rec_permute(int n, const int *perm, const ReactionRecords &src, const ReactionRecords &dst,
                        cudaStream_t st);

}  // namespace lbmd
