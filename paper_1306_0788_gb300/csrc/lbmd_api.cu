// lbmd_api.cu -- the C ABI (include/lbmd.h): context, device memory, argument checks and the
// launch sequence of one coupled step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbmd_internal.cuh"

using namespace lbmd;

namespace {
constexpr int kGraphSteps = 2;  // steps per replayed graph: both buffer pairs return to their start

// A recorded sequence of kGraphSteps coupled steps (lbmd_set_graphs).
struct StepGraph {
  cudaGraph_t graph = nullptr;  // kept for the event nodes' handles
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;                            // kernels per replay
  cudaGraphNode_t ev_node[2 * kGraphSteps] = {};  // k_collide timing events, retargeted per replay
  // the noisy MRT update of each step: its node and the counter offset it was recorded with
  // (its counter is patched per replay; see is_noisy_update)
  cudaGraphNode_t upd_node[kGraphSteps] = {};
  unsigned long long upd_off[kGraphSteps] = {};
  int n_upd = 0;
};
constexpr int kGraphUnavailable = 1;  // record_steps: take the steps one by one instead
}  // namespace

struct lbmd_ctx {
  lbmd_params prm{};
  cudaStream_t st = nullptr;
  // the particle sort and the pair forces depend on the particles only, so they run on a side
  // stream: the pair forces beside the coupling, the particle update (waiting for the coupling,
  // ev_coupled) beside the lattice update that gathers from the sorted copy, and the sort of the
  // updated particles once the lattice update has read that copy (ev_collided), beside the kernels
  // that follow it on st; st waits for the sort (ev_sorted) at the end of a launch sequence or
  // before the next coupling.  ev_int and ev_pairs order the substeps of MD sub-stepping.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_int = nullptr, ev_sorted = nullptr, ev_pairs = nullptr, ev_coupled = nullptr;
  // the particle sort of the next step runs on side right after the lattice update (ev_collided),
  // beside what follows it on st; sort_pending: st has not waited for it yet
  cudaEvent_t ev_collided = nullptr;
  bool sort_pending = false;
  // one pass with particles: ev_integrated (the particle update done, on side) orders the boundary
  // kernel, which forms the next step's corner j' (jc) at the updated positions, after it
  cudaEvent_t ev_integrated = nullptr;
  // the device-memory getters: the caller's stream's queued work before their writes (dev_in),
  // and their writes before what the caller queues next (dev_out); created on first use
  cudaEvent_t ev_dev_in = nullptr, ev_dev_out = nullptr;
  int dev = 0;
  StepParams P{};
  unsigned char *pop[2] = {nullptr, nullptr};  // population buffers, element type P.storage
  size_t pop_elem = 4;
  float *rest = nullptr;  // 16-bit storage: FP32 rest populations [2][N] (not double-buffered: local)
  int cur = 0;
  // [N][2] interleaved rho_A, rho_B: rho_buf[cur] holds the densities of pop[cur] while
  // rho_valid (after init_fluid, set_populations and one-pass steps; the two-pass update
  // recomputes them at the start of its step)
  float *rho_buf[2] = {nullptr, nullptr};
  bool rho_valid = false;
  float *jp = nullptr;   // [3][N]
  // [cap][8] j' at the corners of each particle's cell (by particle id), for the coupling of the
  // one-pass update; jc_valid: formed from the current populations and positions
  float4 *jc = nullptr;
  bool jc_valid = false;
  // the lattice update: 0 = chosen by the lattice size, 1 = one pass (densities of the next step
  // formed by the update), 2 = two passes (density pass, then the update)
  int passes = 0;
  OnePassGeom op_geom{};
  int op_grid = 0;
  BoundaryRun *op_runs = nullptr;
  int op_nruns = 0;
  OnePassOut op_out{};     // partial sums (all buffers owned by the context)
  int *op_zslot = nullptr;  // [nz]: -1, or the chunk-edge plane's slot in op_out's z arrays
  // particles
  int np = 0, cap = 0;
  ParticleArrays pa[2]{};
  int pcur = 0;
  ParticleForces pf{};
  int *slot_of_id = nullptr;
  int *row_of = nullptr, *row_count = nullptr, *row_start = nullptr, *row_cursor = nullptr, *perm = nullptr;
  int *row_bsum = nullptr;  // block sums of the row scan
  int *bond_start = nullptr, *bond_other = nullptr;
  int nbonds = 0, bond_np = 0;  // bonds index particles 0..bond_np-1
  // MD sub-stepping: momentum-return records per (substep, particle), unsorted and sorted
  ReactionRecords rec[2]{};
  int *rec_row_of = nullptr, *rec_perm = nullptr;
  long long rec_cap = 0;
  unsigned *err = nullptr;
  double *diag_partial = nullptr, *diag_out = nullptr;
  int diag_blocks = 0;
  // the FP64 drift check: reference totals [M_A, M_B, Px, Py, Pz] and the last check's
  // {step, drift A, drift B, momentum drift, checks} (device memory, 10 doubles)
  double *drift = nullptr;
  int64_t steps = 0, launches = 0;
  bool fluid_ready = false, types_set = false;
  unsigned sticky = 0;
  std::string msg;
  bool prof = false;
  std::vector<cudaEvent_t> ev;  // pairs (start, stop)
  size_t ev_used = 0;
  double prof_ms = 0.0;
  int64_t prof_launches = 0;
  // replayed step graphs: recorded on gst (never on the caller's stream, which may carry other
  // work), one per parity of (cur, pcur) at the replay's start, launched into st; the kernels
  // read their noise counter's base from step_base, which holds dev_step once the work
  // enqueued so far has run (-1: not known)
  bool graphs = true;
  cudaStream_t gst = nullptr;
  StepGraph graph[2][2];
  unsigned long long *step_base = nullptr;
  int64_t dev_step = -1;
  cudaEvent_t ph[2 * kGraphSteps] = {};  // stand-ins for the timing events while recording
};

namespace {

thread_local std::string g_create_error;

int fail(lbmd_ctx *c, int code, const std::string &m) {
  if (c)
    c->msg = m;
  else
    g_create_error = m;
  return code;
}

int cuda_fail(lbmd_ctx *c, cudaError_t e, const char *where) {
  return fail(c, LBMD_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                          \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t n) {
  *p = nullptr;
  if (n == 0) return cudaSuccess;
  return cudaMalloc((void **)p, n * sizeof(T));
}

template <class T>
void dfree(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

int launched(lbmd_ctx *c, const char *where, int n = 1) {
  c->launches += n;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  return LBMD_OK;
}

int map_device_error(lbmd_ctx *c, unsigned bits) {
  if (bits & kErrNonFinite) return fail(c, LBMD_E_NONFINITE, "non-finite density or particle state");
  if (bits & kErrNegDensity) return fail(c, LBMD_E_NEGATIVE_DENSITY, "negative fluid density");
  if (bits & kErrBond) return fail(c, LBMD_E_BOND_BROKEN, "FENE bond stretched to or beyond R0");
  if (bits & kErrParticle) return fail(c, LBMD_E_NONFINITE, "particle position out of range");
  if (bits & kErrTooFast)
    return fail(c, LBMD_E_PARTICLE_TOO_FAST,
                "with md_substeps > 1 a particle moved more than one cell away within one lattice step");
  if (bits & kErrDrift) {
    double d[5] = {0, 0, 0, 0, 0};
    char m[256];
    if (cudaMemcpy(d, c->drift + 5, sizeof(d), cudaMemcpyDeviceToHost) != cudaSuccess) cudaGetLastError();
    std::snprintf(m, sizeof(m),
                  "FP64 drift check at step %.0f: mass drift A %.3e, B %.3e, momentum drift %.3e per unit mass "
                  "(tolerance %.3e)",
                  d[0], d[1], d[2], d[3], c->prm.drift_tol);
    return fail(c, LBMD_E_DRIFT, m);
  }
  return LBMD_OK;
}

int sync_and_check(lbmd_ctx *c) {
  CK(cudaStreamSynchronize(c->st), "cudaStreamSynchronize");
  unsigned bits = 0;
  CK(cudaMemcpy(&bits, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read error word");
  c->sticky |= bits;
  return map_device_error(c, c->sticky);
}

void free_records(lbmd_ctx *c) {
  for (int b = 0; b < 2; ++b) {
    dfree(c->rec[b].cell); dfree(c->rec[b].frac); dfree(c->rec[b].key);
    dfree(c->rec[b].fric); dfree(c->rec[b].psA); dfree(c->rec[b].psB);
  }
  dfree(c->rec_row_of); dfree(c->rec_perm);
  c->rec_cap = 0;
}

int ensure_records(lbmd_ctx *c, long long n) {
  if (n <= c->rec_cap) return LBMD_OK;
  free_records(c);
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    ReactionRecords &r = c->rec[b];
    if ((e = dalloc(&r.cell, n)) != cudaSuccess || (e = dalloc(&r.frac, n)) != cudaSuccess ||
        (e = dalloc(&r.key, n)) != cudaSuccess || (e = dalloc(&r.fric, n)) != cudaSuccess ||
        (e = dalloc(&r.psA, n)) != cudaSuccess)
      break;
    e = dalloc(&r.psB, n);
  }
  if (e == cudaSuccess) e = dalloc(&c->rec_row_of, n);
  if (e == cudaSuccess) e = dalloc(&c->rec_perm, n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_records(c);
    return fail(c, LBMD_E_NOMEM, std::string("sub-stepping records: ") + cudaGetErrorString(e));
  }
  c->rec_cap = n;
  return LBMD_OK;
}

void free_particles(lbmd_ctx *c) {
  for (int b = 0; b < 2; ++b) {
    dfree(c->pa[b].cell);
    dfree(c->pa[b].frac);
    dfree(c->pa[b].vel);
    dfree(c->pa[b].pid);
  }
  dfree(c->pf.fric); dfree(c->pf.psA); dfree(c->pf.psB); dfree(c->pf.fsr); dfree(c->pf.pair); dfree(c->pf.total);
  dfree(c->slot_of_id); dfree(c->row_of); dfree(c->perm); dfree(c->jc);
  c->jc_valid = false;
  c->cap = 0;
}

// One-pass update: BGK, one particle update per lattice step.  Chosen by the lattice size
// unless set (lbmd_set_lattice_passes): when the blocks of the full persistent grid march at least
// kOnePassAutoPlanes planes each; smaller lattices (set to one pass) take a grid of stretches of
// kOnePassMinPlanes planes.
constexpr int kOnePassMinPlanes = 8;
constexpr int kOnePassAutoPlanes = 16;
constexpr int kOnePassChunkPlanes = 16;

bool onepass_allowed(const lbmd_ctx *c) {
  return c->P.collision == LBMD_COLLISION_BGK && c->P.substeps == 1;
}

long long onepass_units(const StepParams &P) {
  const long long ntx = (P.nx + kOnePassCols - 1) / kOnePassCols, nty = (P.ny + kOnePassRows - 1) / kOnePassRows;
  return ntx * nty * P.nz;
}

int onepass_full_grid(const lbmd_ctx *c) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 1;
  }
  return sms * onepass_blocks_per_sm();
}

bool uses_onepass(const lbmd_ctx *c) {
  if (!onepass_allowed(c) || c->passes == 2) return false;
  if (c->passes == 1) return true;
  return c->op_grid > 0;  // auto: prepare_onepass decided from the size
}

// Frees what prepare_onepass set up.
void free_onepass(lbmd_ctx *c) {
  dfree(c->op_runs);
  dfree(c->op_out.edge);
  dfree(c->op_out.yedge);
  dfree(c->op_out.diag);
  dfree(c->op_out.zown);
  dfree(c->op_out.zedge);
  dfree(c->op_out.zyedge);
  dfree(c->op_zslot);
  c->op_nruns = 0;
  c->op_grid = 0;
}

// Sets up the one-pass update (persistent grid, boundary runs) once per context; in the automatic
// mode only for lattices large enough.  Allocates: call it before any capture.
int prepare_onepass(lbmd_ctx *c) {
  // set up already (op_grid; the run list may be empty: every node finished from partial sums)
  if (!onepass_allowed(c) || c->passes == 2 || c->op_grid > 0) return LBMD_OK;
  const StepParams &P = c->P;
  const long long U = onepass_units(P);
  const int full = onepass_full_grid(c);
  // automatic: one pass for FP32 storage on lattices large enough (the 16-bit update is bound by
  // instruction issue, and the one-pass update's extra instructions cost it more than the second
  // pass over half the bytes)
  if (c->passes == 0 && (P.storage != LBMD_STORAGE_FP32 || U < (long long)kOnePassAutoPlanes * full))
    return LBMD_OK;  // two passes
  free_onepass(c);  // what an earlier attempt that failed part-way left
  const int ntx = (P.nx + kOnePassCols - 1) / kOnePassCols, nty = (P.ny + kOnePassRows - 1) / kOnePassRows;
  // chunks of about kOnePassChunkPlanes planes, one block each, neighbouring column tiles of a
  // chunk launched together (they march in step, so the sectors they share meet in L2)
  const int nchunks = std::max(1, (P.nz + kOnePassChunkPlanes / 2) / kOnePassChunkPlanes);
  const int grid = ntx * nty * nchunks;
  std::vector<unsigned char> edge((size_t)ntx * nty * P.nz, 0);
  for (int col = 0; col < ntx * nty; ++col)
    for (int ch = 0; ch < nchunks; ++ch) {
      const int zs = (int)((long long)ch * P.nz / nchunks), ze = (int)((long long)(ch + 1) * P.nz / nchunks);
      if (ze <= zs) continue;
      edge[(size_t)col * P.nz + zs] = edge[(size_t)col * P.nz + ze - 1] = 1;
    }
  // edge rows from partial sums when every tile has at least 3 rows and 2 columns; chunk-edge
  // planes when the lattice is at least 2 planes deep
  const int ry = P.ny % kOnePassRows, rx = P.nx % kOnePassCols;
  const int ypart = (P.ny >= 3 && (ry == 0 || ry >= 3) && P.nx >= 2 && (rx == 0 || rx >= 2)) ? 1 : 0;
  const int zpart = P.nz >= 2 ? 1 : 0;
  std::vector<BoundaryRun> runs;
  for (int col = 0; col < ntx * nty; ++col) {
    const int tx = col % ntx, ty = col / ntx;
    const int x0 = tx * kOnePassCols, nown = std::min(kOnePassCols, P.nx - x0);
    const int y0 = ty * kOnePassRows, rows = std::min(kOnePassRows, P.ny - y0);
    for (int z = 0; z < P.nz; ++z)
      for (int w = 0; w < rows; ++w)
        if ((!zpart && edge[(size_t)col * P.nz + z]) || (!ypart && (w == 0 || w == rows - 1)))
          runs.push_back(BoundaryRun{z * P.ny + y0 + w, x0, nown});
  }
  if (runs.size() > 0x7fffffffull) return fail(c, LBMD_E_INVALID_ARG, "too many boundary runs");
  CK(dalloc(&c->op_out.edge, (size_t)P.nz * P.ny * ntx * 4), "edge sums");
  {
    // slot 2 b (plane zs - 1) and 2 b + 1 (plane zs) of the boundary below chunk b
    std::vector<int> zslot((size_t)P.nz, -1);
    for (int ch = 0; ch < nchunks; ++ch) {
      const int zs = (int)((long long)ch * P.nz / nchunks);
      zslot[(size_t)(zs == 0 ? P.nz - 1 : zs - 1)] = 2 * ch;
      zslot[(size_t)zs] = 2 * ch + 1;
    }
    CK(dalloc(&c->op_zslot, zslot.size()), "plane table");
    CK(cudaMemcpy(c->op_zslot, zslot.data(), sizeof(int) * zslot.size(), cudaMemcpyHostToDevice), "plane table");
  }
  if (ypart) {
    CK(dalloc(&c->op_out.yedge, (size_t)2 * P.nz * nty * ntx * kOnePassCols * 2), "edge sums");
    CK(dalloc(&c->op_out.diag, (size_t)P.nz * nty * ntx * 4 * 2), "edge sums");
  }
  if (zpart) {
    CK(dalloc(&c->op_out.zown, (size_t)2 * nchunks * P.ny * P.nx * 2), "chunk-edge sums");
    CK(dalloc(&c->op_out.zedge, (size_t)2 * nchunks * P.ny * ntx * 4), "chunk-edge sums");
    if (ypart) CK(dalloc(&c->op_out.zyedge, (size_t)2 * 2 * nchunks * nty * ntx * kOnePassCols * 2), "chunk-edge sums");
  }
  CK(dalloc(&c->op_runs, runs.size()), "boundary runs");
  CK(cudaMemcpy(c->op_runs, runs.data(), sizeof(BoundaryRun) * runs.size(), cudaMemcpyHostToDevice), "boundary runs");
  c->op_nruns = (int)runs.size();
  c->op_geom = OnePassGeom{ntx, nty, nchunks, ypart, zpart};
  c->op_grid = grid;
  return LBMD_OK;
}

// The densities of the current state into rho_buf[cur] (a density pass), if not there already.
int ensure_densities(lbmd_ctx *c) {
  if (c->rho_valid) return LBMD_OK;
  launch_moments(c->P, c->pop[c->cur], c->rest, c->rho_buf[c->cur], nullptr, c->st);
  const int r = launched(c, "moments");
  if (!r) c->rho_valid = true;
  return r;
}

// One pass with particles (one particle update per step): the corner j' of the current state
// into jc, if not there already.
int ensure_corner_j(lbmd_ctx *c) {
  if (c->jc_valid || c->np == 0 || c->P.substeps > 1 || !uses_onepass(c)) return LBMD_OK;
  if (c->sort_pending) {  // the arrays read here are the ones the pending sort writes
    CK(cudaStreamWaitEvent(c->st, c->ev_sorted, 0), "stream wait");
    c->sort_pending = false;
  }
  launch_corner_jprime(c->P, c->pa[c->pcur], c->np, c->pop[c->cur], c->jc, c->st);
  const int r = launched(c, "corner j'");
  if (!r) c->jc_valid = true;
  return r;
}

int sort_particles(lbmd_ctx *c, cudaStream_t st) {
  const StepParams &P = c->P;
  if (sort_fits_one_block(P.nrows, P.np)) {
    launch_sort_small(P, c->pa[c->pcur], c->pa[1 - c->pcur], c->row_start, c->slot_of_id, c->err, st);
    c->pcur = 1 - c->pcur;
    return launched(c, "particle sort");
  }
  CK(cudaMemsetAsync(c->row_count, 0, sizeof(int) * (P.nrows + 1), st), "memset rows");
  launch_bin(P, c->pa[c->pcur], c->row_of, c->row_count, c->err, st);
  launch_scan_rows(P.nrows, c->row_count, c->row_start, c->row_cursor, c->row_bsum, st);
  launch_scatter(P.np, c->row_of, c->row_cursor, c->perm, st);
  launch_row_sort(P, c->row_start, c->pa[c->pcur], c->perm, st);
  launch_permute(P.np, c->perm, c->pa[c->pcur], c->pa[1 - c->pcur], c->slot_of_id, st);
  c->pcur = 1 - c->pcur;
  return launched(c, "particle sort", 7);  // bin, three scan passes, scatter, row order, permute
}

// FP64 totals of the current state into diag_out: [M_A, M_B, Px, Py, Pz] of the fluid and,
// with particles, [5..7] = sum m v (K9 of the step; appendix and Sec. 2 for what they conserve).
int enqueue_totals(lbmd_ctx *c) {
  launch_fluid_sums(c->P, c->pop[c->cur], c->rest, c->diag_partial, c->diag_blocks, c->st);
  launch_finish_sums(c->diag_partial, c->diag_blocks, 5, c->diag_out, c->st);
  int r = launched(c, "fluid sums", 2);
  if (r || c->np == 0) return r;
  StepParams P = c->P;
  P.np = c->np;
  const int nb = std::min(c->diag_blocks, (c->np + 255) / 256);
  double *part = c->diag_partial + (size_t)5 * c->diag_blocks - 3 * (size_t)nb;
  launch_particle_momentum(P, c->pa[c->pcur], part, nb, c->st);
  launch_finish_sums(part, nb, 3, c->diag_out + 5, c->st);
  return launched(c, "particle momentum", 2);
}

// The drift check on the device (set_ref: take the totals as the reference instead).
// The drift table before any reference: no reference, no check yet (step -1, no checks).
const double kDriftNone[10] = {0, 0, 0, 0, 0, -1, 0, 0, 0, 0};

int enqueue_drift(lbmd_ctx *c, int set_ref) {
  int r = enqueue_totals(c);
  if (r) return r;
  launch_drift_check(c->diag_out, c->np > 0 ? c->diag_out + 5 : nullptr, c->drift, c->drift + 5, c->err,
                     (long long)c->steps, c->prm.drift_tol, set_ref, c->st);
  return launched(c, "drift check");
}

}  // namespace

namespace {

// MD sub-stepping of one lattice step (K = P.substeps > 1): the sorted particles S of the step's
// start stay frozen (cell list, fluid-side solvation force); a working copy C takes K substeps
// of coupling forces (writing one momentum-return record per particle and substep), pair
// forces over S's rows with one more cell of reach, and updates of dt / K; the records are
// then sorted by row for the update's node-side gather.  On return C is the particle state and
// (pa, pf, ci) describe the records.
int substep_particles(lbmd_ctx *c, ParticleArrays &pa, ParticleForces &pf, CellIndex &ci) {
  const StepParams &P = c->P;
  const int K = P.substeps, np = P.np;
  const long long nrec = (long long)K * np;
  if (nrec > 0x7fffffffLL) return fail(c, LBMD_E_INVALID_ARG, "md_substeps x particles exceeds 2^31");
  int r = ensure_records(c, nrec);
  if (r) return r;
  const ParticleArrays &S = c->pa[c->pcur];
  const ParticleArrays &C = c->pa[1 - c->pcur];
  CK(cudaMemcpyAsync(C.cell, S.cell, sizeof(int4) * np, cudaMemcpyDeviceToDevice, c->st), "copy particles");
  CK(cudaMemcpyAsync(C.frac, S.frac, sizeof(float4) * np, cudaMemcpyDeviceToDevice, c->st), "copy particles");
  CK(cudaMemcpyAsync(C.vel, S.vel, sizeof(float4) * np, cudaMemcpyDeviceToDevice, c->st), "copy particles");
  CK(cudaMemcpyAsync(C.pid, S.pid, sizeof(int) * np, cudaMemcpyDeviceToDevice, c->st), "copy particles");
  const CellIndex rows{c->row_start};
  for (int sub = 0; sub < K; ++sub) {
    StepParams Q = P;
    Q.step = P.step * (unsigned long long)K + (unsigned long long)sub;
    Q.step_mul = (unsigned long long)K;
    Q.dt = P.dt / (float)K;
    // the pair forces (side stream) and the coupling read the same positions and write
    // different forces; the update of the substep waits for both
    CK(cudaEventRecord(c->ev_int, c->st), "event");
    CK(cudaStreamWaitEvent(c->side, c->ev_int, 0), "stream wait");
    StepParams Qp = Q;
    Qp.reach = P.reach + 1;  // particles may have left their row by one cell
    launch_pairs(Qp, C, rows, c->nbonds ? c->bond_start : nullptr, c->bond_other, c->slot_of_id, c->pf, c->err,
                 c->side);
    CK(cudaEventRecord(c->ev_pairs, c->side), "event");
    launch_couple_sub(Q, C, S, rows, c->rho_buf[c->cur], c->jp, c->pf, sub, c->rec[0], c->st);
    CK(cudaStreamWaitEvent(c->st, c->ev_pairs, 0), "stream wait");
    launch_integrate_sub(Q, C, S, c->pf, c->err, c->st);
    if ((r = launched(c, "particle substep", 3))) return r;
  }
  // sort the records by (row, x cell, substep * np + id): the same counting sort as particles
  StepParams R = P;
  R.np = (int)nrec;
  const ParticleArrays view{c->rec[0].cell, c->rec[0].frac, nullptr, c->rec[0].key};
  CK(cudaMemsetAsync(c->row_count, 0, sizeof(int) * (P.nrows + 1), c->st), "memset rows");
  launch_bin(R, view, c->rec_row_of, c->row_count, c->err, c->st);
  launch_scan_rows(P.nrows, c->row_count, c->row_start, c->row_cursor, c->row_bsum, c->st);
  launch_scatter(R.np, c->rec_row_of, c->row_cursor, c->rec_perm, c->st);
  launch_row_sort(R, c->row_start, view, c->rec_perm, c->st);
  launch_rec_permute(R.np, c->rec_perm, c->rec[0], c->rec[1], c->st);
  if ((r = launched(c, "record sort", 7))) return r;
  pa = ParticleArrays{c->rec[1].cell, c->rec[1].frac, nullptr, c->rec[1].key};
  pf = c->pf;
  pf.fric = c->rec[1].fric;
  pf.psA = c->rec[1].psA;
  pf.psB = c->rec[1].psB;
  ci = CellIndex{c->row_start};
  return LBMD_OK;
}

// Timing events of k_collide (lbmd_profile_enable): the pool holds at least n unused ones.
int reserve_events(lbmd_ctx *c, size_t n) {
  while (c->ev.size() < c->ev_used + n) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e), "event");
    c->ev.push_back(e);
  }
  return LBMD_OK;
}

// One coupled step on st and side.  `step` is the noise counter the kernels get: the lattice
// step, or, while a graph is recorded, the step's offset in it (the kernels add the base).
// t0, t1 (or null): events recorded around the lattice update, with `flags`.
// The particles are kept sorted between steps: every step ends by sorting the updated particles
// for the next one, on the side stream once the lattice update has read the sorted arrays, so that
// the sort runs beside the kernels that follow the update on st (the boundary densities, or the
// next step's density pass).  join: st waits for that sort before returning (else the next step
// does, before its particle coupling).
int one_step(lbmd_ctx *c, unsigned long long step, cudaEvent_t t0, cudaEvent_t t1, unsigned flags, bool join) {
  StepParams &P = c->P;
  P.step = step;
  const CellIndex ci{c->row_start};
  const void *fin = c->pop[c->cur];
  void *fout = c->pop[1 - c->cur];
  float *rho = c->rho_buf[c->cur];
  int r;
  const bool sub = P.np > 0 && P.substeps > 1;
  const bool onepass = uses_onepass(c);
  if (P.np > 0 && !sub) {
    // fork the side stream from the step's start (while st records a graph, this is also what
    // makes the side stream's work part of the graph)
    CK(cudaEventRecord(c->ev_int, c->st), "event");
    CK(cudaStreamWaitEvent(c->side, c->ev_int, 0), "stream wait");
  }
  if (onepass) {
    if (!c->rho_valid) return fail(c, LBMD_E_STATE, "one-pass update without the densities of the current state");
  } else {
    // densities (and j' for the particle coupling) of this step's populations
    launch_moments(P, fin, c->rest, rho, P.np > 0 ? c->jp : nullptr, c->st);
    if ((r = launched(c, "moments"))) return r;
  }
  if (P.np > 0 && c->sort_pending) {  // the previous step's sort of these particles
    CK(cudaStreamWaitEvent(c->st, c->ev_sorted, 0), "stream wait");
    c->sort_pending = false;
  }
  ParticleArrays gpa = c->pa[c->pcur];  // what the update gathers the momentum return from
  ParticleForces gpf = c->pf;
  CellIndex gci = ci;
  if (sub) {
    if ((r = substep_particles(c, gpa, gpf, gci))) return r;
  } else if (P.np > 0) {
    if (onepass) {  // no density pass stored j': the previous step's boundary kernel formed it at the corners
      if (!c->jc_valid) return fail(c, LBMD_E_STATE, "one-pass coupling without the corner j' of the current state");
      launch_couple_jc(P, c->pa[c->pcur], ci, rho, c->jc, c->pf, c->st);
    } else
      launch_couple(P, c->pa[c->pcur], ci, rho, c->jp, c->pf, c->st);
    CK(cudaEventRecord(c->ev_coupled, c->st), "event");
    launch_pairs(P, c->pa[c->pcur], ci, c->nbonds ? c->bond_start : nullptr, c->bond_other, c->slot_of_id, c->pf,
                 c->err, c->side);
    CK(cudaStreamWaitEvent(c->side, c->ev_coupled, 0), "stream wait");
    launch_integrate(P, c->pa[c->pcur], c->pa[1 - c->pcur], c->pf, c->err, c->side);
    if ((r = launched(c, "particle forces and update", 3))) return r;
    if (onepass) CK(cudaEventRecord(c->ev_integrated, c->side), "event");
  }
  if (t0) CK(cudaEventRecordWithFlags(t0, c->st, flags), "event");
  if (onepass)
    launch_collide_onepass(P, fin, fout, c->rest, rho, c->rho_buf[1 - c->cur],
                           c->op_out, gpa, gpf, gci, c->err, c->op_geom,
                           c->op_grid, c->st);
  else
    launch_collide(P, fin, fout, c->rest, rho, gpa, gpf, gci, c->err, c->st);
  if ((r = launched(c, "collide"))) return r;
  if (t1) CK(cudaEventRecordWithFlags(t1, c->st, flags), "event");
  if (P.np > 0) CK(cudaEventRecord(c->ev_collided, c->st), "event");
  const bool corner_j = onepass && P.np > 0 && !sub;  // the boundary kernel forms the next step's jc
  if (onepass) {
    if (corner_j) CK(cudaStreamWaitEvent(c->st, c->ev_integrated, 0), "stream wait");
    launch_boundary_densities(P, c->op_geom, fout, c->rest, c->rho_buf[1 - c->cur], c->op_runs, c->op_nruns,
                              c->op_out, c->op_zslot, c->pa[1 - c->pcur], corner_j ? P.np : 0,
                              corner_j ? c->jc : nullptr, c->st);
    if ((r = launched(c, "boundary densities"))) return r;
  }
  if (P.np > 0) {
    // the updated particles (the working copy that took the substeps, or the update's output) are
    // the state; sort them for the next step into the arrays the lattice update has just read
    c->pcur = 1 - c->pcur;
    CK(cudaStreamWaitEvent(c->side, c->ev_collided, 0), "stream wait");
    if ((r = sort_particles(c, c->side))) return r;
    CK(cudaEventRecord(c->ev_sorted, c->side), "event");
    c->sort_pending = true;
    if (join) {
      CK(cudaStreamWaitEvent(c->st, c->ev_sorted, 0), "stream wait");
      c->sort_pending = false;
    }
  }
  c->cur = 1 - c->cur;
  c->steps++;
  c->rho_valid = onepass;  // the two-pass update leaves the new state's densities to its next step
  c->jc_valid = corner_j;
  return LBMD_OK;
}

void drop_graphs(lbmd_ctx *c) {
  for (auto &row : c->graph)
    for (StepGraph &g : row) {
      if (g.exec) cudaGraphExecDestroy(g.exec);  // a launch in flight completes first
      if (g.graph) cudaGraphDestroy(g.graph);
      g = StepGraph{};
    }
}

// Records kGraphSteps steps from the current buffers into g: on the private stream gst, with
// the noise counters relative to the device-resident step base, the base advanced at the end.
// Nothing runs; the context's host state is left as it was.
int record_steps(lbmd_ctx *c, StepGraph &g) {
  const StepParams &P = c->P;
  int r;
  if (P.np > 0 && P.substeps > 1 && (r = ensure_records(c, (long long)P.substeps * P.np)))
    return r;  // no allocation while recording
  if ((r = prepare_onepass(c))) return r;
  if (!c->gst) CK(cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking), "graph stream");
  if (!c->step_base) CK(dalloc(&c->step_base, 1), "alloc step base");
  if (c->prof)
    for (cudaEvent_t &e : c->ph)
      if (!e) CK(cudaEventCreate(&e), "event");
  const int cur0 = c->cur, pcur0 = c->pcur;
  const bool rho_valid0 = c->rho_valid, sort_pending0 = c->sort_pending, jc_valid0 = c->jc_valid;
  const int64_t steps0 = c->steps, launches0 = c->launches;
  cudaStream_t user = c->st;
  CK(cudaStreamBeginCapture(c->gst, cudaStreamCaptureModeThreadLocal), "begin capture");
  c->st = c->gst;
  c->P.step_base = c->step_base;
  r = LBMD_OK;
  for (int j = 0; j < kGraphSteps && !r; ++j)
    r = one_step(c, (unsigned long long)j, c->prof ? c->ph[2 * j] : nullptr, c->prof ? c->ph[2 * j + 1] : nullptr,
                 cudaEventRecordExternal, j == kGraphSteps - 1);
  if (!r) {
    launch_advance_step(c->step_base, kGraphSteps, c->gst);
    r = launched(c, "step counter");
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->gst, &graph);
  const bool back = c->cur == cur0 && c->pcur == pcur0;
  c->st = user;
  c->P.step_base = nullptr;
  c->cur = cur0;
  c->pcur = pcur0;
  c->rho_valid = rho_valid0;
  c->sort_pending = sort_pending0;
  c->jc_valid = jc_valid0;
  c->steps = steps0;
  g.launches = c->launches - launches0;
  c->launches = launches0;
  if (r || e != cudaSuccess || !back) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (r) return r;
    if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
    return fail(c, LBMD_E_STATE, "recorded steps do not return to their buffers");
  }
  g.graph = graph;
  cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  const bool noisy = c->P.collision == LBMD_COLLISION_MRT && c->P.fluct;
  if (ei == cudaSuccess && (c->prof || noisy)) {  // find the timing stand-ins and the noisy updates
    size_t n = 0;
    ei = cudaGraphGetNodes(graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (ei == cudaSuccess) ei = cudaGraphGetNodes(graph, nodes.data(), &n);
    for (size_t k = 0; k < n && ei == cudaSuccess; ++k) {
      cudaGraphNodeType t;
      if ((ei = cudaGraphNodeGetType(nodes[k], &t)) != cudaSuccess) break;
      if (t == cudaGraphNodeTypeEventRecord) {
        cudaEvent_t ev = nullptr;
        if ((ei = cudaGraphEventRecordNodeGetEvent(nodes[k], &ev)) != cudaSuccess) break;
        for (int q = 0; q < 2 * kGraphSteps; ++q)
          if (ev == c->ph[q]) g.ev_node[q] = nodes[k];
      } else if (t == cudaGraphNodeTypeKernel && noisy) {
        cudaKernelNodeParams kp;
        if ((ei = cudaGraphKernelNodeGetParams(nodes[k], &kp)) != cudaSuccess) break;
        if (!is_noisy_update(kp.func) || !kp.kernelParams || g.n_upd == kGraphSteps) continue;
        StepParams Q;
        std::memcpy(&Q, kp.kernelParams[0], sizeof(Q));
        g.upd_node[g.n_upd] = nodes[k];
        g.upd_off[g.n_upd++] = Q.step;
      }
    }
    for (int q = 0; q < 2 * kGraphSteps && ei == cudaSuccess && c->prof; ++q)
      if (!g.ev_node[q]) ei = cudaErrorInvalidValue;
  }
  if (ei != cudaSuccess) {
    drop_graphs(c);
    cudaGetLastError();
    return cuda_fail(c, ei, "graph instantiation");
  }
  if (noisy && g.n_upd != kGraphSteps) {  // the update's nodes were not recognised
    drop_graphs(c);
    c->graphs = false;
    return kGraphUnavailable;
  }
  return LBMD_OK;
}

// kGraphSteps steps by one launch of the graph recorded for the current buffers.
int replay_steps(lbmd_ctx *c) {
  StepGraph &g = c->graph[c->cur][c->pcur];
  int r;
  if ((r = prepare_onepass(c))) return r;
  if (uses_onepass(c) && ((r = ensure_densities(c)) || (r = ensure_corner_j(c))))
    return r;  // before recording: not in the graph
  if (!g.exec && (r = record_steps(c, g))) return r;
  if (c->dev_step != c->steps) {  // steps were taken without the graph since it last ran
    launch_set_step(c->step_base, (unsigned long long)c->steps, c->st);
    if ((r = launched(c, "step counter"))) return r;
  }
  if (c->prof) {
    if ((r = reserve_events(c, 2 * kGraphSteps))) return r;
    for (int q = 0; q < 2 * kGraphSteps; ++q)
      CK(cudaGraphExecEventRecordNodeSetEvent(g.exec, g.ev_node[q], c->ev[c->ev_used + q]), "timing event");
  }
  for (int q = 0; q < g.n_upd; ++q)
    CK(set_update_step(g.exec, g.upd_node[q], (unsigned long long)c->steps + g.upd_off[q]), "update counter");
  CK(cudaGraphLaunch(g.exec, c->st), "graph launch");
  if (c->prof) c->ev_used += 2 * kGraphSteps;
  c->launches += g.launches;
  c->steps += kGraphSteps;
  c->dev_step = c->steps;
  c->rho_valid = uses_onepass(c);
  c->jc_valid = c->rho_valid && c->np > 0 && c->P.substeps == 1;
  return LBMD_OK;
}

}  // namespace

void lbmd::set_context_free_error(const std::string &m) { g_create_error = m; }

extern "C" {

const char *lbmd_last_error(const lbmd_ctx *c) { return c ? c->msg.c_str() : g_create_error.c_str(); }

int lbmd_create(const lbmd_params *prm, void *stream, lbmd_ctx **out, unsigned *warnings) {
  lbmd_ctx *c = nullptr;
  if (!prm || !out) return fail(c, LBMD_E_INVALID_ARG, "null argument");
  *out = nullptr;
  if (warnings) *warnings = 0;
  {
    std::string why;
    const int r = check_params(prm, why);
    if (r) return fail(c, r, why);
  }
  c = new lbmd_ctx();
  c->prm = *prm;
  c->st = (cudaStream_t)stream;
  cudaGetDevice(&c->dev);
  StepParams &P = c->P;
  fill_step_params(prm, P);
  c->pop_elem = prm->storage == LBMD_STORAGE_FP32 ? 4 : 2;
  cudaError_t e = cudaSuccess;
  const size_t npop = (size_t)2 * kQ * P.N * c->pop_elem;  // bytes; >= 19 N floats of staging
  if ((e = dalloc(&c->pop[0], npop)) != cudaSuccess || (e = dalloc(&c->pop[1], npop)) != cudaSuccess ||
      (e = dalloc(&c->rho_buf[0], (size_t)2 * P.N)) != cudaSuccess ||
      (e = dalloc(&c->rho_buf[1], (size_t)2 * P.N)) != cudaSuccess || (e = dalloc(&c->jp, (size_t)3 * P.N)) != cudaSuccess ||
      (e = dalloc(&c->err, 1)) != cudaSuccess ||
      (c->pop_elem == 2 && (e = dalloc(&c->rest, (size_t)2 * P.N)) != cudaSuccess)) {
    cudaGetLastError();
    lbmd_destroy(c);
    return fail(nullptr, e == cudaErrorMemoryAllocation ? LBMD_E_NOMEM : LBMD_E_CUDA,
                std::string("device allocation: ") + cudaGetErrorString(e));
  }
  if ((e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_int, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_sorted, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_pairs, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_coupled, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_collided, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_integrated, cudaEventDisableTiming)) != cudaSuccess) {
    cudaGetLastError();
    lbmd_destroy(c);
    return fail(nullptr, LBMD_E_CUDA, std::string("stream / event creation: ") + cudaGetErrorString(e));
  }
  c->diag_blocks = fluid_sum_blocks(P);
  if ((e = dalloc(&c->diag_partial, (size_t)5 * c->diag_blocks)) != cudaSuccess ||
      (e = dalloc(&c->diag_out, 8)) != cudaSuccess || (e = dalloc(&c->drift, 10)) != cudaSuccess ||
      (e = cudaMemcpy(c->drift, kDriftNone, sizeof(kDriftNone), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(c->err, 0, sizeof(unsigned))) != cudaSuccess) {
    cudaGetLastError();
    lbmd_destroy(c);
    return fail(nullptr, LBMD_E_NOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
  }
  const unsigned w = param_warnings(prm);
  if (warnings) *warnings = w;
  *out = c;
  return LBMD_OK;
}

void lbmd_destroy(lbmd_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_int) cudaEventDestroy(c->ev_int);
  if (c->ev_sorted) cudaEventDestroy(c->ev_sorted);
  if (c->ev_pairs) cudaEventDestroy(c->ev_pairs);
  if (c->ev_coupled) cudaEventDestroy(c->ev_coupled);
  if (c->ev_collided) cudaEventDestroy(c->ev_collided);
  if (c->ev_integrated) cudaEventDestroy(c->ev_integrated);
  if (c->ev_dev_in) cudaEventDestroy(c->ev_dev_in);
  if (c->ev_dev_out) cudaEventDestroy(c->ev_dev_out);
  drop_graphs(c);
  if (c->gst) cudaStreamDestroy(c->gst);
  for (cudaEvent_t e : c->ph)
    if (e) cudaEventDestroy(e);
  dfree(c->step_base);
  dfree(c->pop[0]); dfree(c->pop[1]); dfree(c->rho_buf[0]); dfree(c->rho_buf[1]); dfree(c->jp); dfree(c->err);
  dfree(c->rest);
  free_onepass(c);
  dfree(c->diag_partial); dfree(c->diag_out); dfree(c->drift);
  free_particles(c);
  free_records(c);
  dfree(c->row_count); dfree(c->row_start); dfree(c->row_cursor); dfree(c->row_bsum);
  dfree(c->bond_start); dfree(c->bond_other);
  for (cudaEvent_t ev : c->ev) cudaEventDestroy(ev);
  delete c;
}

int lbmd_set_types(lbmd_ctx *c, int ntypes, const lbmd_ptype *types, int npairs, const lbmd_pair *pairs,
                   unsigned *warnings) {
  if (!c) return LBMD_E_INVALID_ARG;
  drop_graphs(c);  // every setter: the recorded steps hold the old parameters and buffers
  if (warnings) *warnings = 0;
  unsigned w = 0;
  std::string why;
  const int r = apply_types(c->P, c->prm.kT, c->prm.dt, ntypes, types, npairs, pairs, w, why);
  if (r) return fail(c, r, why);
  c->types_set = true;
  if (warnings) *warnings = w;
  return LBMD_OK;
}

int lbmd_set_debye_hueckel(lbmd_ctx *c, double lB, double kappa_D, double rc) {
  if (!c) return LBMD_E_INVALID_ARG;
  drop_graphs(c);
  std::string why;
  const int r = apply_debye_hueckel(c->P, lB, kappa_D, rc, why);
  return r ? fail(c, r, why) : LBMD_OK;
}

int lbmd_init_fluid(lbmd_ctx *c, const float *rhoA, const float *rhoB, const float *u) {
  if (!c || !rhoA || !rhoB) return c ? fail(c, LBMD_E_INVALID_ARG, "null density") : LBMD_E_INVALID_ARG;
  cudaSetDevice(c->dev);
  drop_graphs(c);
  const long long N = c->P.N;
  if (!densities_valid(rhoA, rhoB, N))
    return fail(c, LBMD_E_INVALID_ARG, "densities must be finite and > 0");
  // stage through the (not yet used) second population buffer
  float *stage = reinterpret_cast<float *>(c->pop[1 - c->cur]);
  const size_t bytes = sizeof(float) * (size_t)N;
  CK(cudaMemcpyAsync(stage, rhoA, bytes, cudaMemcpyHostToDevice, c->st), "upload rhoA");
  CK(cudaMemcpyAsync(stage + N, rhoB, bytes, cudaMemcpyHostToDevice, c->st), "upload rhoB");
  const float *du = nullptr;
  if (u) {
    CK(cudaMemcpyAsync(stage + 2 * N, u, 3 * bytes, cudaMemcpyHostToDevice, c->st), "upload u");
    du = stage + 2 * N;
  }
  launch_init_equilibrium(c->P, stage, stage + N, du, c->pop[c->cur], c->rest, c->st);
  int r = launched(c, "init_equilibrium");
  if (r) return r;
  c->steps = 0;
  c->rho_valid = false;
  c->jc_valid = false;
  if ((r = ensure_densities(c))) return r;
  // the drift check's reference (a context that never checks takes it only when asked)
  if (c->prm.diag_every > 0 && (r = enqueue_drift(c, 1))) return r;
  CK(cudaStreamSynchronize(c->st), "sync");
  c->fluid_ready = true;
  return LBMD_OK;
}

int lbmd_set_populations(lbmd_ctx *c, int comp, const float *f) {
  if (!c || !f || comp < 0 || comp > 1) return c ? fail(c, LBMD_E_INVALID_ARG, "bad arguments") : LBMD_E_INVALID_ARG;
  cudaSetDevice(c->dev);
  drop_graphs(c);
  float *stage = reinterpret_cast<float *>(c->pop[1 - c->cur]);
  CK(cudaMemcpyAsync(stage, f, sizeof(float) * kQ * (size_t)c->P.N, cudaMemcpyHostToDevice, c->st), "upload f");
  launch_restream(c->P, stage, comp, c->pop[c->cur], c->rest, c->st);
  int r = launched(c, "restream");
  if (r) return r;
  c->rho_valid = false;
  c->jc_valid = false;
  if ((r = ensure_densities(c))) return r;
  CK(cudaStreamSynchronize(c->st), "sync");
  c->fluid_ready = true;
  return LBMD_OK;
}

int lbmd_get_populations(lbmd_ctx *c, int comp, float *f) {
  if (!c || !f || comp < 0 || comp > 1) return c ? fail(c, LBMD_E_INVALID_ARG, "bad arguments") : LBMD_E_INVALID_ARG;
  if (!c->fluid_ready) return fail(c, LBMD_E_STATE, "fluid not initialised");
  cudaSetDevice(c->dev);
  float *stage = reinterpret_cast<float *>(c->pop[1 - c->cur]);
  launch_unstream(c->P, c->pop[c->cur], c->rest, comp, stage, c->st);
  int r = launched(c, "unstream");
  if (r) return r;
  CK(cudaMemcpyAsync(f, stage, sizeof(float) * kQ * (size_t)c->P.N, cudaMemcpyDeviceToHost, c->st), "download f");
  return sync_and_check(c);
}

int lbmd_set_particles(lbmd_ctx *c, int n, const double *x, const double *v, const int *type, const double *q) {
  if (!c) return LBMD_E_INVALID_ARG;
  if (n < 0 || (n > 0 && (!x || !v || !type))) return fail(c, LBMD_E_INVALID_ARG, "bad particle arrays");
  if (n > 0 && !c->types_set) return fail(c, LBMD_E_STATE, "set the particle types first");
  cudaSetDevice(c->dev);
  drop_graphs(c);
  StepParams &P = c->P;
  std::vector<int4> hc;
  std::vector<float4> hf, hv;
  std::vector<int> hid;
  {
    std::string why;
    const int r = convert_particles(P, n, x, v, type, q, hc, hf, hv, hid, why);
    if (r) return fail(c, r, why);
  }
  if (n > c->cap) {
    free_particles(c);
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      if ((e = dalloc(&c->pa[b].cell, n)) != cudaSuccess) break;
      if ((e = dalloc(&c->pa[b].frac, n)) != cudaSuccess) break;
      if ((e = dalloc(&c->pa[b].vel, n)) != cudaSuccess) break;
      e = dalloc(&c->pa[b].pid, n);
    }
    if (e == cudaSuccess) e = dalloc(&c->pf.fric, n);
    if (e == cudaSuccess) e = dalloc(&c->pf.psA, n);
    if (e == cudaSuccess) e = dalloc(&c->pf.psB, n);
    if (e == cudaSuccess) e = dalloc(&c->pf.fsr, n);
    if (e == cudaSuccess) e = dalloc(&c->pf.pair, n);
    if (e == cudaSuccess) e = dalloc(&c->pf.total, n);
    if (e == cudaSuccess) e = dalloc(&c->slot_of_id, n);
    if (e == cudaSuccess) e = dalloc(&c->row_of, n);
    if (e == cudaSuccess) e = dalloc(&c->perm, n);
    if (e == cudaSuccess) e = dalloc(&c->jc, (size_t)n * 8);
    if (e == cudaSuccess && !c->row_count) e = dalloc(&c->row_count, (size_t)P.nrows + 1);
    if (e == cudaSuccess && !c->row_start) e = dalloc(&c->row_start, (size_t)P.nrows + 1);
    if (e == cudaSuccess && !c->row_cursor) e = dalloc(&c->row_cursor, (size_t)P.nrows + 1);
    if (e == cudaSuccess && !c->row_bsum) e = dalloc(&c->row_bsum, (size_t)scan_blocks(P.nrows) + 1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_particles(c);
      c->np = 0;
      P.np = 0;
      return fail(c, LBMD_E_NOMEM, std::string("particle allocation: ") + cudaGetErrorString(e));
    }
    c->cap = n;
  }
  if (!c->row_count) {  // rows are needed by the lattice kernels' gather even without particles
    CK(dalloc(&c->row_count, (size_t)P.nrows + 1), "alloc rows");
    CK(dalloc(&c->row_start, (size_t)P.nrows + 1), "alloc rows");
    CK(dalloc(&c->row_cursor, (size_t)P.nrows + 1), "alloc rows");
    CK(dalloc(&c->row_bsum, (size_t)scan_blocks(P.nrows) + 1), "alloc rows");
  }
  c->np = n;
  P.np = n;
  c->pcur = 0;
  c->jc_valid = false;
  if (n > 0) {
    CK(cudaMemcpyAsync(c->pa[0].cell, hc.data(), sizeof(int4) * n, cudaMemcpyHostToDevice, c->st), "upload");
    CK(cudaMemcpyAsync(c->pa[0].frac, hf.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, c->st), "upload");
    CK(cudaMemcpyAsync(c->pa[0].vel, hv.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, c->st), "upload");
    CK(cudaMemcpyAsync(c->pa[0].pid, hid.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st), "upload");
    CK(cudaMemsetAsync(c->pf.total, 0, sizeof(float4) * n, c->st), "memset");
    int r = sort_particles(c, c->st);
    if (r) return r;
  }
  c->sort_pending = false;
  if (c->fluid_ready && c->prm.diag_every > 0) {  // the drift check's reference includes the new particles' momentum
    const int r = enqueue_drift(c, 1);
    if (r) return r;
  }
  CK(cudaStreamSynchronize(c->st), "sync");
  return LBMD_OK;
}

int lbmd_set_bonds(lbmd_ctx *c, int nb, const int *pairs, int kind, double k, double r) {
  if (!c) return LBMD_E_INVALID_ARG;
  drop_graphs(c);
  if (nb < 0 || (nb > 0 && !pairs)) return fail(c, LBMD_E_INVALID_ARG, "bad bond list");
  if (kind != LBMD_BOND_FENE && kind != LBMD_BOND_HARMONIC) return fail(c, LBMD_E_INVALID_ARG, "unknown bond kind");
  if (nb > 0 && (!(k >= 0.0) || !(r > 0.0 || kind == LBMD_BOND_HARMONIC)))
    return fail(c, LBMD_E_INVALID_ARG, "bad bond parameters");
  cudaSetDevice(c->dev);
  dfree(c->bond_start);
  dfree(c->bond_other);
  c->nbonds = 0;
  if (nb == 0) return LBMD_OK;
  const int n = c->np;
  std::vector<int> deg(n + 1, 0), other(2 * (size_t)nb);
  for (int b = 0; b < nb; ++b) {
    const int i = pairs[2 * b], j = pairs[2 * b + 1];
    if (i < 0 || i >= n || j < 0 || j >= n || i == j) return fail(c, LBMD_E_INVALID_ARG, "bond index out of range");
    deg[i + 1]++;
    deg[j + 1]++;
  }
  for (int i = 0; i < n; ++i) deg[i + 1] += deg[i];
  std::vector<int> fill(deg.begin(), deg.end() - 1);
  for (int b = 0; b < nb; ++b) {
    const int i = pairs[2 * b], j = pairs[2 * b + 1];
    other[fill[i]++] = j;
    other[fill[j]++] = i;
  }
  CK(dalloc(&c->bond_start, (size_t)n + 1), "alloc bonds");
  CK(dalloc(&c->bond_other, 2 * (size_t)nb), "alloc bonds");
  CK(cudaMemcpy(c->bond_start, deg.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice), "upload bonds");
  CK(cudaMemcpy(c->bond_other, other.data(), sizeof(int) * 2 * nb, cudaMemcpyHostToDevice), "upload bonds");
  c->nbonds = nb;
  c->bond_np = n;
  c->P.bond_kind = kind;
  c->P.bond_k = (float)k;
  c->P.bond_r = (float)r;
  return LBMD_OK;
}

int lbmd_step(lbmd_ctx *c, int nsteps) {
  if (!c) return LBMD_E_INVALID_ARG;
  if (nsteps < 0) return fail(c, LBMD_E_INVALID_ARG, "nsteps < 0");
  if (!c->fluid_ready) return fail(c, LBMD_E_STATE, "fluid not initialised");
  cudaSetDevice(c->dev);
  if (c->nbonds > 0 && c->bond_np != c->np)
    return fail(c, LBMD_E_STATE, "bonds refer to a different particle set; call lbmd_set_bonds again");
  c->P.np = c->np;
  const int64_t K = c->prm.diag_every;
  int left = nsteps, r;
  while (left > 0) {
    // steps up to the next multiple of diag_every (the drift check runs after it), or all
    int n = left;
    if (K > 0) n = (int)std::min<int64_t>(left, K - c->steps % K);
    left -= n;
    int s = 0;
    if (c->graphs)
      for (; s + kGraphSteps <= n; s += kGraphSteps)
        if ((r = replay_steps(c))) {
          if (r != kGraphUnavailable) return r;
          break;
        }
    if (s < n) {
      if ((r = prepare_onepass(c))) return r;
      if (uses_onepass(c) && ((r = ensure_densities(c)) || (r = ensure_corner_j(c)))) return r;
    }
    for (; s < n; ++s) {
      cudaEvent_t t0 = nullptr, t1 = nullptr;
      if (c->prof) {
        if ((r = reserve_events(c, 2))) return r;
        t0 = c->ev[c->ev_used];
        t1 = c->ev[c->ev_used + 1];
      }
      if ((r = one_step(c, (unsigned long long)c->steps, t0, t1, cudaEventRecordDefault, true))) return r;
      if (c->prof) c->ev_used += 2;
    }
    if (K > 0 && c->steps % K == 0 && (r = enqueue_drift(c, 0))) return r;
  }
  return LBMD_OK;
}

int lbmd_set_graphs(lbmd_ctx *c, int on) {
  if (!c) return LBMD_E_INVALID_ARG;
  cudaSetDevice(c->dev);
  drop_graphs(c);
  c->graphs = on != 0;
  return LBMD_OK;
}

int lbmd_set_lattice_passes(lbmd_ctx *c, int passes) {
  if (!c) return LBMD_E_INVALID_ARG;
  if (passes < 0 || passes > 2) return fail(c, LBMD_E_INVALID_ARG, "passes must be 0 (by size), 1 or 2");
  if (passes == 1 && !onepass_allowed(c))
    return fail(c, LBMD_E_INVALID_ARG, "the one-pass update takes the BGK collision with md_substeps = 1");
  cudaSetDevice(c->dev);
  drop_graphs(c);
  if (passes != c->passes) {
    free_onepass(c);  // set up again for the new choice at the next step
    c->jc_valid = false;
  }
  c->passes = passes;
  return LBMD_OK;
}

int lbmd_get_lattice_passes(lbmd_ctx *c) {
  if (!c) return LBMD_E_INVALID_ARG;
  cudaSetDevice(c->dev);
  const int r = prepare_onepass(c);
  if (r) return r;
  return uses_onepass(c) ? 1 : 2;
}

int lbmd_sync(lbmd_ctx *c) {
  if (!c) return LBMD_E_INVALID_ARG;
  cudaSetDevice(c->dev);
  return sync_and_check(c);
}

int lbmd_clear_error(lbmd_ctx *c) {
  if (!c) return LBMD_E_INVALID_ARG;
  cudaSetDevice(c->dev);
  CK(cudaStreamSynchronize(c->st), "sync");
  CK(cudaMemset(c->err, 0, sizeof(unsigned)), "clear error word");
  c->sticky = 0;
  c->msg.clear();
  return LBMD_OK;
}

int lbmd_get_fields(lbmd_ctx *c, float *rhoA, float *rhoB, float *u) {
  if (!c) return LBMD_E_INVALID_ARG;
  if (!c->fluid_ready) return fail(c, LBMD_E_STATE, "fluid not initialised");
  cudaSetDevice(c->dev);
  const long long N = c->P.N;
  float *stage = reinterpret_cast<float *>(c->pop[1 - c->cur]);
  int r = ensure_densities(c);
  if (r) return r;
  launch_fields(c->P, c->pop[c->cur], c->rest, c->rho_buf[c->cur], stage, stage + N, stage + 2 * N, c->st);
  if ((r = launched(c, "fields"))) return r;
  const size_t bytes = sizeof(float) * (size_t)N;
  if (rhoA) CK(cudaMemcpyAsync(rhoA, stage, bytes, cudaMemcpyDeviceToHost, c->st), "download");
  if (rhoB) CK(cudaMemcpyAsync(rhoB, stage + N, bytes, cudaMemcpyDeviceToHost, c->st), "download");
  if (u) CK(cudaMemcpyAsync(u, stage + 2 * N, 3 * bytes, cudaMemcpyDeviceToHost, c->st), "download");
  return sync_and_check(c);
}

int lbmd_get_particles(lbmd_ctx *c, double *x, double *v, double *f) {
  if (!c) return LBMD_E_INVALID_ARG;
  cudaSetDevice(c->dev);
  const int n = c->np;
  if (n == 0) return sync_and_check(c);
  std::vector<int4> hc(n);
  std::vector<float4> hf(n), hv(n), ht(n);
  std::vector<int> hid(n), htid(n);
  const ParticleArrays &pa = c->pa[c->pcur];
  // the total forces are in the order of the copy the particle update wrote, which the sort for
  // the next step leaves in the other buffer
  const ParticleArrays &pt = c->pa[1 - c->pcur];
  CK(cudaMemcpyAsync(hc.data(), pa.cell, sizeof(int4) * n, cudaMemcpyDeviceToHost, c->st), "download");
  CK(cudaMemcpyAsync(hf.data(), pa.frac, sizeof(float4) * n, cudaMemcpyDeviceToHost, c->st), "download");
  CK(cudaMemcpyAsync(hv.data(), pa.vel, sizeof(float4) * n, cudaMemcpyDeviceToHost, c->st), "download");
  CK(cudaMemcpyAsync(ht.data(), c->pf.total, sizeof(float4) * n, cudaMemcpyDeviceToHost, c->st), "download");
  CK(cudaMemcpyAsync(hid.data(), pa.pid, sizeof(int) * n, cudaMemcpyDeviceToHost, c->st), "download");
  CK(cudaMemcpyAsync(htid.data(), pt.pid, sizeof(int) * n, cudaMemcpyDeviceToHost, c->st), "download");
  int r = sync_and_check(c);
  for (int j = 0; j < n; ++j) {
    const int id = hid[j], tid = htid[j];
    if (id < 0 || id >= n || tid < 0 || tid >= n) return fail(c, LBMD_E_CUDA, "corrupt particle ids");
    if (x) {
      x[3 * id] = hc[j].x + (double)hf[j].x;
      x[3 * id + 1] = hc[j].y + (double)hf[j].y;
      x[3 * id + 2] = hc[j].z + (double)hf[j].z;
    }
    if (v) {
      v[3 * id] = hv[j].x; v[3 * id + 1] = hv[j].y; v[3 * id + 2] = hv[j].z;
    }
    if (f) {
      f[3 * tid] = ht[j].x; f[3 * tid + 1] = ht[j].y; f[3 * tid + 2] = ht[j].z;
    }
  }
  return r;
}

// The device-memory getters write into caller buffers on the context's stream, ordered after the
// work already queued on the caller's stream and before the work the caller queues there next.
static int dev_getter_begin(lbmd_ctx *c, cudaStream_t caller) {
  if (!c->ev_dev_in) CK(cudaEventCreateWithFlags(&c->ev_dev_in, cudaEventDisableTiming), "event");
  if (!c->ev_dev_out) CK(cudaEventCreateWithFlags(&c->ev_dev_out, cudaEventDisableTiming), "event");
  if (caller != c->st) {
    CK(cudaEventRecord(c->ev_dev_in, caller), "event");
    CK(cudaStreamWaitEvent(c->st, c->ev_dev_in, 0), "stream wait");
  }
  return LBMD_OK;
}

static int dev_getter_end(lbmd_ctx *c, cudaStream_t caller) {
  if (caller != c->st) {
    CK(cudaEventRecord(c->ev_dev_out, c->st), "event");
    CK(cudaStreamWaitEvent(caller, c->ev_dev_out, 0), "stream wait");
  }
  return LBMD_OK;
}

static int dev_buffers_ok(lbmd_ctx *c, const char *name, const void *p, size_t bytes) {
  if (p && !device_buffer_ok(p, bytes))
    return fail(c, LBMD_E_INVALID_ARG,
                std::string(name) + " is not device memory of this context's device holding " +
                    std::to_string(bytes) + " bytes");
  return LBMD_OK;
}

int lbmd_get_fields_dev(lbmd_ctx *c, float *rhoA, float *rhoB, float *u, void *stream) {
  if (!c) return LBMD_E_INVALID_ARG;
  if (!c->fluid_ready) return fail(c, LBMD_E_STATE, "fluid not initialised");
  cudaSetDevice(c->dev);
  const long long N = c->P.N;
  const size_t bytes = sizeof(float) * (size_t)N;
  int r;
  if ((r = dev_buffers_ok(c, "rhoA_dev", rhoA, bytes)) || (r = dev_buffers_ok(c, "rhoB_dev", rhoB, bytes)) ||
      (r = dev_buffers_ok(c, "u_dev", u, 3 * bytes)))
    return r;
  if (!rhoA && !rhoB && !u) return LBMD_OK;
  const cudaStream_t caller = static_cast<cudaStream_t>(stream);
  if ((r = dev_getter_begin(c, caller))) return r;
  // outputs the caller does not want go to the spare population buffer, as in lbmd_get_fields
  float *stage = reinterpret_cast<float *>(c->pop[1 - c->cur]);
  if ((r = ensure_densities(c))) return r;
  launch_fields(c->P, c->pop[c->cur], c->rest, c->rho_buf[c->cur], rhoA ? rhoA : stage, rhoB ? rhoB : stage + N,
                u ? u : stage + 2 * N, c->st);
  if ((r = launched(c, "fields"))) return r;
  return dev_getter_end(c, caller);
}

int lbmd_get_populations_dev(lbmd_ctx *c, int comp, float *f, void *stream) {
  if (!c || !f || comp < 0 || comp > 1) return c ? fail(c, LBMD_E_INVALID_ARG, "bad arguments") : LBMD_E_INVALID_ARG;
  if (!c->fluid_ready) return fail(c, LBMD_E_STATE, "fluid not initialised");
  cudaSetDevice(c->dev);
  int r;
  if ((r = dev_buffers_ok(c, "f_dev", f, sizeof(float) * kQ * (size_t)c->P.N))) return r;
  const cudaStream_t caller = static_cast<cudaStream_t>(stream);
  if ((r = dev_getter_begin(c, caller))) return r;
  launch_unstream(c->P, c->pop[c->cur], c->rest, comp, f, c->st);
  if ((r = launched(c, "unstream"))) return r;
  return dev_getter_end(c, caller);
}

int lbmd_get_particles_dev(lbmd_ctx *c, double *x, double *v, double *f, void *stream) {
  if (!c) return LBMD_E_INVALID_ARG;
  cudaSetDevice(c->dev);
  const int n = c->np;
  const size_t bytes = sizeof(double) * 3 * (size_t)n;
  int r;
  if ((r = dev_buffers_ok(c, "x_dev", x, bytes)) || (r = dev_buffers_ok(c, "v_dev", v, bytes)) ||
      (r = dev_buffers_ok(c, "f_dev", f, bytes)))
    return r;
  if (n == 0 || (!x && !v && !f)) return LBMD_OK;
  const cudaStream_t caller = static_cast<cudaStream_t>(stream);
  if ((r = dev_getter_begin(c, caller))) return r;
  if (c->sort_pending) {  // the arrays read here are the ones the pending sort writes
    CK(cudaStreamWaitEvent(c->st, c->ev_sorted, 0), "stream wait");
    c->sort_pending = false;
  }
  // the total forces are in the order of the copy the particle update wrote (as in lbmd_get_particles)
  launch_particles_out(n, c->pa[c->pcur], c->pa[1 - c->pcur].pid, c->pf.total, x, v, f, c->st);
  if ((r = launched(c, "particles out"))) return r;
  return dev_getter_end(c, caller);
}

int lbmd_diagnostics(lbmd_ctx *c, double out[8]) {
  if (!c || !out) return c ? fail(c, LBMD_E_INVALID_ARG, "null output") : LBMD_E_INVALID_ARG;
  if (!c->fluid_ready) return fail(c, LBMD_E_STATE, "fluid not initialised");
  cudaSetDevice(c->dev);
  int r = enqueue_totals(c);
  if (r) return r;
  double h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  CK(cudaMemcpyAsync(h, c->diag_out, sizeof(double) * (c->np > 0 ? 8 : 5), cudaMemcpyDeviceToHost, c->st),
     "download");
  r = sync_and_check(c);
  std::memcpy(out, h, sizeof(h));
  return r;
}

int lbmd_set_drift_reference(lbmd_ctx *c) {
  if (!c) return LBMD_E_INVALID_ARG;
  if (!c->fluid_ready) return fail(c, LBMD_E_STATE, "fluid not initialised");
  cudaSetDevice(c->dev);
  return enqueue_drift(c, 1);
}

int lbmd_get_drift(lbmd_ctx *c, double out[5]) {
  if (!c || !out) return c ? fail(c, LBMD_E_INVALID_ARG, "null output") : LBMD_E_INVALID_ARG;
  if (!c->fluid_ready) return fail(c, LBMD_E_STATE, "fluid not initialised");
  cudaSetDevice(c->dev);
  double h[5];
  CK(cudaMemcpyAsync(h, c->drift + 5, sizeof(h), cudaMemcpyDeviceToHost, c->st), "download");
  CK(cudaStreamSynchronize(c->st), "sync");
  std::memcpy(out, h, sizeof(h));
  return LBMD_OK;
}

int64_t lbmd_step_count(const lbmd_ctx *c) { return c ? c->steps : -1; }
int64_t lbmd_launch_count(const lbmd_ctx *c) { return c ? c->launches : -1; }

int lbmd_profile_enable(lbmd_ctx *c, int on) {
  if (!c) return LBMD_E_INVALID_ARG;
  if (c->prof != (on != 0)) drop_graphs(c);  // profiled graphs carry the timing events
  c->prof = on != 0;
  return LBMD_OK;
}

int lbmd_profile_read(lbmd_ctx *c, double *ms, int64_t *nl, int reset) {
  if (!c) return LBMD_E_INVALID_ARG;
  cudaSetDevice(c->dev);
  CK(cudaStreamSynchronize(c->st), "sync");
  for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->ev[k], c->ev[k + 1]), "event time");
    c->prof_ms += t;
    c->prof_launches++;
  }
  c->ev_used = 0;
  if (ms) *ms = c->prof_ms;
  if (nl) *nl = c->prof_launches;
  if (reset) {
    c->prof_ms = 0.0;
    c->prof_launches = 0;
  }
  return LBMD_OK;
}

}  // extern "C"
