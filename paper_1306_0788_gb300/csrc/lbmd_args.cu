// lbmd_args.cu -- argument checks and conversions shared by single contexts (lbmd_api.cu) and
// batches (lb_batch.cu): model parameters, particle types and pairs, screened Coulomb, and the
// host-side conversion of particle positions to (cell, fraction).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "lb_modes.h"
#include "lbmd_internal.cuh"

namespace lbmd {

bool densities_valid(const float *rhoA, const float *rhoB, long long n) {
  // x > 0 and x <= FLT_MAX: false for NaN, infinities, zero and negative values
  constexpr float kMax = 3.402823466e38f;
  unsigned ok = 1u;
  for (long long s = 0; s < n; ++s)
    ok &= (unsigned)(rhoA[s] > 0.f) & (unsigned)(rhoA[s] <= kMax) & (unsigned)(rhoB[s] > 0.f) &
          (unsigned)(rhoB[s] <= kMax);
  return ok != 0u;
}

int check_params(const lbmd_params *prm, std::string &why) {
  if (prm->nx < 1 || prm->ny < 1 || prm->nz < 1) return why = "lattice sizes must be >= 1", LBMD_E_INVALID_ARG;
  if ((double)prm->nx * prm->ny * prm->nz * kQ >= 4294967296.0)  // 32-bit population offsets
    return why = "lattice too large: nx*ny*nz must be below 2^32/19", LBMD_E_INVALID_ARG;
  if (!(prm->tau_r > 0.5)) return why = "tau_r must exceed 1/2", LBMD_E_INVALID_ARG;
  if (prm->dt != 1.0) return why = "dt must equal the lattice time step 1", LBMD_E_INVALID_ARG;
  if (!(prm->kT >= 0.0)) return why = "kT must be >= 0", LBMD_E_INVALID_ARG;
  if (prm->storage != LBMD_STORAGE_FP32 && prm->storage != LBMD_STORAGE_FP16_SHIFTED &&
      prm->storage != LBMD_STORAGE_BF16_SHIFTED)
    return why = "unknown storage", LBMD_E_INVALID_ARG;
  if (!(prm->rho0_A >= 0.0) || !(prm->rho0_B >= 0.0) || !std::isfinite(prm->rho0_A) || !std::isfinite(prm->rho0_B))
    return why = "rho0_A, rho0_B must be finite and >= 0", LBMD_E_INVALID_ARG;
  if (prm->md_substeps < 1 || prm->md_substeps > 256) return why = "md_substeps must be in [1, 256]", LBMD_E_INVALID_ARG;
  if (prm->diag_every < 0) return why = "diag_every must be >= 0", LBMD_E_INVALID_ARG;
  if (prm->diag_every > 0 && !(prm->drift_tol > 0.0 && std::isfinite(prm->drift_tol)))
    return why = "with diag_every > 0, drift_tol must be finite and > 0", LBMD_E_INVALID_ARG;
  if (prm->collision != LBMD_COLLISION_BGK && prm->collision != LBMD_COLLISION_MRT)
    return why = "unknown collision", LBMD_E_INVALID_ARG;
  if (prm->collision == LBMD_COLLISION_MRT)
    for (double l : {prm->lambda_bulk, prm->lambda_mom, prm->lambda_ghost})
      if (!(l > -2.0 && l < 0.0)) return why = "MRT eigenvalues must lie in (-2, 0)", LBMD_E_INVALID_ARG;
  return LBMD_OK;
}

void fill_step_params(const lbmd_params *prm, StepParams &P) {
  P = StepParams{};
  P.nx = prm->nx;
  P.ny = prm->ny;
  P.nz = prm->nz;
  P.nrows = prm->ny * prm->nz;
  P.N = (long long)prm->nx * prm->ny * prm->nz;
  P.divx = make_fastdiv((uint32_t)prm->nx);
  P.divy = make_fastdiv((uint32_t)prm->ny);
  P.inv_tau = (float)(1.0 / prm->tau_r);
  P.force_pref = (float)(1.0 - 0.5 / prm->tau_r);
  P.gAB = (float)prm->g_AB;
  P.gBA = (float)prm->g_BA;
  P.dt = (float)prm->dt;
  P.storage = prm->storage;
  P.rho0[0] = prm->storage == LBMD_STORAGE_FP32 ? 0.f : (float)prm->rho0_A;
  P.rho0[1] = prm->storage == LBMD_STORAGE_FP32 ? 0.f : (float)prm->rho0_B;
  P.seed = prm->seed;
  {
    uint2 k = make_uint2((unsigned)prm->seed, (unsigned)(prm->seed >> 32));
    for (int r = 0; r < 10; ++r) {
      P.noise_keys[r] = k;
      k.x += 0x9E3779B9u;  // the Weyl increments of philox4x32_10's key schedule
      k.y += 0xBB67AE85u;
    }
  }
  P.ntypes = 0;
  P.bond_kind = LBMD_BOND_FENE;
  // fluctuating MRT factors (Eq. MODES): eigenvalue per mode, forcing moments of the paper's
  // forcing term, noise amplitudes from the equilibrium mode variances (kT/c_s^2) rho_z b_k
  P.substeps = prm->md_substeps;
  P.step_mul = 1;
  P.noise_scale = (float)std::sqrt((double)prm->md_substeps);
  P.collision = prm->collision;
  const bool mrt = prm->collision == LBMD_COLLISION_MRT;
  P.fluct = mrt && prm->kT > 0.0;
  const double ls = -1.0 / prm->tau_r;
  const double lb = mrt ? prm->lambda_bulk : ls, lm = mrt ? prm->lambda_mom : ls, lg = mrt ? prm->lambda_ghost : ls;
  for (int k = 0; k < kQ; ++k) {
    const double l = k == 0 ? 0.0 : k <= 3 ? lm : k == 4 ? lb : k <= 9 ? ls : lg;
    P.relax[k] = (float)(1.0 + l);
    P.force[k] = (float)(k == 0 ? 0.0 : k <= 3 ? 0.5 * (2.0 + lm) : k == 4 ? 2.0 + lb : k <= 6 ? 2.0 + ls
                                        : k <= 9 ? 0.5 * (2.0 + ls) : 0.0);
    const double keep = 1.0 - (1.0 + l) * (1.0 + l);
    const double bk = mode_norm9(k) / 9.0;
    P.noise[k] = (float)(k == 0 ? 0.0 : k <= 3 ? std::sqrt(prm->kT * keep) : std::sqrt(3.0 * prm->kT * bk * keep));
  }
}

unsigned param_warnings(const lbmd_params *prm) {
  unsigned w = 0;
  if (1.0 / 3.0 * (prm->tau_r - 0.5) < 1e-3) w |= LBMD_WARN_VISCOSITY;
  if (prm->g_AB != prm->g_BA) w |= LBMD_WARN_ASYMMETRIC_G;
  const double r0 = prm->rho0_A + prm->rho0_B;
  if (prm->kT > 0.0 && r0 > 0.0 && std::sqrt(prm->kT / (r0 / 3.0)) > 0.5) w |= LBMD_WARN_BOLTZMANN;
  return w;
}

namespace {
// largest interaction range of the WCA pairs and the screened Coulomb cut-off
double max_range(const StepParams &P) {
  double r = 0.0;
  for (int i = 0; i < P.ntypes; ++i)
    for (int j = 0; j < P.ntypes; ++j) {
      const PairParams &pp = P.pairs[i * LBMD_MAX_TYPES + j];
      if (pp.eps > 0.f) r = std::fmax(r, std::sqrt((double)pp.rc2));
    }
  if (P.dh_lB != 0.f) r = std::fmax(r, std::sqrt((double)P.dh_rc2));
  return r;
}
}  // namespace

int apply_types(StepParams &P, double kT, double dt, int ntypes, const lbmd_ptype *types, int npairs,
                const lbmd_pair *pairs, unsigned &w, std::string &why) {
  w = 0;
  if (ntypes < 1 || ntypes > LBMD_MAX_TYPES || !types || npairs < 0 || (npairs > 0 && !pairs))
    return why = "bad type table", LBMD_E_INVALID_ARG;
  StepParams Q = P;  // applied only if every entry is valid
  for (int t = 0; t < ntypes; ++t) {
    const lbmd_ptype &T = types[t];
    if (!(T.mass > 0.0) || !(T.gamma >= 0.0)) return why = "mass must be > 0, gamma >= 0", LBMD_E_INVALID_ARG;
    TypeParams &D = Q.types[t];
    D.kappa[0] = (float)T.kappa_A;
    D.kappa[1] = (float)T.kappa_B;
    D.lam[0] = (float)T.lambda_A;
    D.lam[1] = (float)T.lambda_B;
    D.gamma = (float)T.gamma;
    D.inv_mass = (float)(1.0 / T.mass);
    D.mass = (float)T.mass;
    D.noise_amp = (float)std::sqrt(2.0 * kT * T.gamma / dt);
    if (T.gamma * dt / T.mass > 0.5) w |= LBMD_WARN_GAMMA_DT;
  }
  for (int i = 0; i < LBMD_MAX_TYPES * LBMD_MAX_TYPES; ++i) Q.pairs[i] = PairParams{0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < npairs; ++k) {
    const lbmd_pair &pp = pairs[k];
    if (pp.type_i < 0 || pp.type_i >= ntypes || pp.type_j < 0 || pp.type_j >= ntypes || pp.wca_eps < 0 ||
        !(pp.wca_sigma > 0))
      return why = "bad pair entry", LBMD_E_INVALID_ARG;
    const double rc = std::pow(2.0, 1.0 / 6.0) * pp.wca_sigma;
    if (2.0 * rc >= std::min(Q.nx, std::min(Q.ny, Q.nz)))
      return why = "WCA range must be below half the smallest box edge", LBMD_E_INVALID_ARG;
    PairParams d{(float)pp.wca_eps, (float)(pp.wca_sigma * pp.wca_sigma), (float)(rc * rc), 0.f};
    Q.pairs[pp.type_i * LBMD_MAX_TYPES + pp.type_j] = d;
    Q.pairs[pp.type_j * LBMD_MAX_TYPES + pp.type_i] = d;
  }
  Q.ntypes = ntypes;
  Q.reach = (int)std::ceil(max_range(Q));
  P = Q;
  return LBMD_OK;
}

int apply_debye_hueckel(StepParams &P, double lB, double kappa_D, double rc, std::string &why) {
  if (lB != 0.0) {
    if (!(rc > 0.0) || !(kappa_D >= 0.0)) return why = "bad Debye-Hueckel parameters", LBMD_E_INVALID_ARG;
    if (2.0 * rc >= std::min(P.nx, std::min(P.ny, P.nz)))
      return why = "cut-off must be below half the smallest box edge", LBMD_E_INVALID_ARG;
  }
  P.dh_lB = (float)lB;
  P.dh_kappa = (float)kappa_D;
  P.dh_rc2 = (float)(rc * rc);
  P.reach = (int)std::ceil(max_range(P));
  return LBMD_OK;
}

int convert_particles(const StepParams &P, int n, const double *x, const double *v, const int *type,
                      const double *q, std::vector<int4> &hc, std::vector<float4> &hf, std::vector<float4> &hv,
                      std::vector<int> &hid, std::string &why) {
  const int L[3] = {P.nx, P.ny, P.nz};
  hc.resize(n);
  hf.resize(n);
  hv.resize(n);
  hid.resize(n);
  for (int p = 0; p < n; ++p) {
    if (type[p] < 0 || type[p] >= P.ntypes) return why = "particle type out of range", LBMD_E_INVALID_ARG;
    int ci[3];
    float fr[3];
    for (int a = 0; a < 3; ++a) {
      const double xa = x[3 * p + a];
      if (!std::isfinite(xa) || !std::isfinite(v[3 * p + a])) return why = "non-finite particle", LBMD_E_INVALID_ARG;
      double w = xa - L[a] * std::floor(xa / L[a]);
      if (w >= L[a]) w = 0.0;
      int cell = (int)std::floor(w);
      float f = (float)(w - cell);
      if (f >= 1.f) {
        f = 0.f;
        cell = (cell + 1) % L[a];
      }
      ci[a] = cell;
      fr[a] = f;
    }
    hc[p] = make_int4(ci[0], ci[1], ci[2], type[p]);
    hf[p] = make_float4(fr[0], fr[1], fr[2], q ? (float)q[p] : 0.f);
    hv[p] = make_float4((float)v[3 * p], (float)v[3 * p + 1], (float)v[3 * p + 2], 0.f);
    hid[p] = p;
  }
  return LBMD_OK;
}

}  // namespace lbmd
