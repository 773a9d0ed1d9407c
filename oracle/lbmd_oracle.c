/*
 * lbmd_oracle.c -- plain FP64 CPU oracle of one coupled time step of the
 * two-component Shan-Chen D3Q19 lattice Boltzmann fluid with friction-coupled
 * off-lattice particles and solvation forces (Sega, Sbragaglia, Kantorovich,
 * Ivanov, "Mesoscale Structures at Complex Fluid-Fluid Interfaces: a Novel
 * Lattice Boltzmann / Molecular Dynamics Coupling", arXiv:1306.0788).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or call
 * this file: only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant with the CUDA
 * implementation; it is written straight from the paper's equations, in the
 * paper's order and notation, with loops over sites, directions, components and
 * particles, in IEEE double precision, compiled without FMA contraction.
 *
 * Readings of passages the paper leaves open (each one is listed in the design
 * notes of the repository):
 *   R1  Shan-Chen force, Eq. (SCforce): the link vector (r'-r) is weighted with the
 *       isotropy weights w_i, g_z(r) = -rho_z(r) sum_z' g_zz' sum_i w_i rho_z'(r+c_i) c_i,
 *       so that its continuum limit is -c_s^2 rho_z g grad rho_z' (Eq. Taylor with
 *       the c_s^2 of Eq. fbulk).  psi = rho, g_AA = g_BB = 0.
 *   R2  Eq. (feq): the identity in uu:(c c - 1) is read as c_s^2 times the identity
 *       (the only reading with sum_i f^eq = rho).
 *   R3  BGK: all relaxation eigenvalues lambda_k = -1/tau_r (lattice time step 1).
 *   R4  Forcing (appendix, last two equations): G_z is built from g_z and the common
 *       barycentric velocity u.
 *   R5  The velocity that the particles see (Eq. NEWTON) is the pre-collision
 *       barycentric velocity of Eq. (momentum_definition) built with the Shan-Chen and
 *       fluid-side solvation forces only: u_cpl = (j' + (1/2) sum_z (g^SC_z + F^fs_z)) / rho.
 *   R6  grad rho_z at a particle (Eq. solvation_kappa) is the trilinear interpolation
 *       of the node gradient S_z / c_s^2, S_z = sum_i w_i rho_z(r+c_i) c_i.
 *   R7  Momentum return (Sec. 2, last paragraphs): the friction + noise reaction is
 *       spread with the trilinear weights and split over components in proportion
 *       rho_z/rho at each node; the reaction of the kappa_z term goes to component z;
 *       the particle receives minus the total fluid-side solvation force it exerts.
 *   R8  Eq. (solvation_lambda): r' runs over the 18 lattice neighbours of r, Theta is
 *       open at both ends, particles are those of the 8 unit cells with corner r, no
 *       interpolation weight; a particle exactly on a node contributes nothing.
 *   R9  Integrator (not given by the paper): v += F dt/m, x += v dt with dt = 1; noise
 *       R_a = sqrt(2 kT gamma / dt) N(0,1), N drawn with Philox4x32-10 (Salmon et al.,
 *       SC'11) and the Box-Muller transform.
 *   R10 D3Q19 order: 0; +x,-x,+y,-y,+z,-z; then the xy, xz, yz diagonals with
 *       opposite directions adjacent.
 *   R13 Fluctuating MRT (Eq. MODES, appendix): mode basis = the orthogonal polynomials of
 *       Duenweg, Schiller and Ladd in c (the paper's citation for its mode space); eigenvalues
 *       lambda_M (component momenta), lambda_b (bulk), lambda_s = -1/tau_r (shear), lambda_g
 *       (kinetic modes); m*_k = m^eq_k + (1 + lambda_k)(m_k - m^eq_k) + m^g_k + phi_k r_k with
 *       m^eq, m^g the projections of f^eq and of the forcing term.  Noise amplitudes from the
 *       equilibrium mode variances <m_k^2> = (kT/c_s^2) rho_z b_k (b_k = sum_i w_i e_ki^2):
 *       phi = sqrt((kT/c_s^2) rho_z b_k (1 - (1+lambda_k)^2)) for the stress and kinetic modes,
 *       one Gaussian per component; the momentum modes share one Gaussian per direction with
 *       opposite signs for A and B (Sec. 2), amplitude sqrt(kT (rho_A rho_B / rho)
 *       (1 - (1+lambda_M)^2)), the equilibrium variance of the interdiffusion flux
 *       (rho_B j_A - rho_A j_B) / rho of two ideal components.  Gaussians from Philox4x32-10
 *       with counter (site, step low, step high, 0x464c0000 + k), k = 0..8, Box-Muller on both
 *       uniform pairs of each draw: normals 0-2 are the momentum ones (x, y, z), 3-17 the
 *       modes 4-18 of A, 18-32 those of B.
 *   R15 MD sub-stepping (Sec. 3, gamma dt / m << 1): with K = md_substeps > 1 the particle
 *       forces, the momentum return and the particle update (steps 5, 6 and 9 below) run K
 *       times with dt / K while the fluid fields of the step stay frozen: the coupling velocity
 *       field u_cpl and the node gradients are those of step 4, the fluid-side solvation force
 *       and its reaction on the particles those of x(n); the friction noise of substep k draws
 *       with the counter step K + k and has the amplitude sqrt(2 kT gamma K / dt); the momentum
 *       return of every substep is spread with that substep's trilinear weights and divided by
 *       K, and the collision uses the sum.  K = 1 is the step above.
 *   R14 Bulk viscosity of that collision: eta_b = -(2/3) rho c_s^2 (1/lambda_b + 1/2), from the
 *       trace equation of the Chapman-Enskog expansion with the traceless shear stress of
 *       Eq. (comp_Pi); Eq. (TRANSPORTCOEFF) prints it without the 2/3 (which at BGK would
 *       contradict the known eta_b = 2/3 eta_s of D3Q19).  Nothing in the collision depends on
 *       this reading; only the pin of the sound damping does.
 *
 * Threads: the loops over sites whose iterations are independent (each writes only its own
 * site's values, summed in the same order) may run on several host threads (OpenMP, set by
 * orc_set_threads; one thread by default).  The arithmetic and its order per site do not
 * change, so every result is bitwise the same for any thread count; the global reductions
 * (orc_fluid_moments) and the particle loops stay serial.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q 19
#define ORC_CS2 (1.0 / 3.0)

static int orc_nthreads = 1;

/* Host threads of the per-site loops (see the header; n < 1 means 1). */
void orc_set_threads(int n) { orc_nthreads = n < 1 ? 1 : n; }

/* Eq. (velo), ordered per reading R10. */
static const int orc_c[ORC_Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
};

/* Eq. (weights). */
static double orc_w(int i) {
  if (i == 0) return 1.0 / 3.0;
  if (i <= 6) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

void orc_lattice(int *c_out, double *w_out) {
  for (int i = 0; i < ORC_Q; ++i) {
    for (int a = 0; a < 3; ++a) c_out[3 * i + a] = orc_c[i][a];
    w_out[i] = orc_w(i);
  }
}

static long orc_wrap(long a, long n) {
  long r = a % n;
  return r < 0 ? r + n : r;
}

static long orc_site(const int *dim, long x, long y, long z) {
  return (orc_wrap(z, dim[2]) * dim[1] + orc_wrap(y, dim[1])) * dim[0] + orc_wrap(x, dim[0]);
}

/* Eq. (feq), reading R2: f^eq_i = w_i rho [1 + u.c_i/cs2 + uu:(c_i c_i - cs2 1)/(2 cs2^2)]. */
void orc_feq(double rho, const double *u, double *out) {
  for (int i = 0; i < ORC_Q; ++i) {
    double uc = 0.0;
    for (int a = 0; a < 3; ++a) uc += u[a] * orc_c[i][a];
    double second = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        second += u[a] * u[b] * (orc_c[i][a] * orc_c[i][b] - (a == b ? ORC_CS2 : 0.0));
    out[i] = orc_w(i) * rho * (1.0 + uc / ORC_CS2 + second / (2.0 * ORC_CS2 * ORC_CS2));
  }
}

/* Forcing source term of the appendix (last two equations), lattice time step tau = 1:
 *   Delta^g_i = (w_i/cs2) ((2+lM)/2) g.c_i + (w_i/cs2) (1/(2 cs2)) G:(c_i c_i - cs2 1),
 *   G_ab = ((2+ls)/2)(u_a g_b + g_a u_b - (2/3) u.g d_ab) + ((2+lb)/3) u.g d_ab. */
void orc_forcing(const double *g, const double *u, double lM, double ls, double lb, double *out) {
  double ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
  double G[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      G[a][b] = 0.5 * (2.0 + ls) * (u[a] * g[b] + g[a] * u[b] - (a == b ? 2.0 / 3.0 * ug : 0.0)) +
                (a == b ? (2.0 + lb) / 3.0 * ug : 0.0);
  for (int i = 0; i < ORC_Q; ++i) {
    double gc = 0.0;
    for (int a = 0; a < 3; ++a) gc += g[a] * orc_c[i][a];
    double Gcc = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Gcc += G[a][b] * (orc_c[i][a] * orc_c[i][b] - (a == b ? ORC_CS2 : 0.0));
    out[i] = orc_w(i) / ORC_CS2 * (0.5 * (2.0 + lM)) * gc + orc_w(i) / ORC_CS2 * (Gcc / (2.0 * ORC_CS2));
  }
}

/* Node gradient sum S(r) = sum_i w_i rho(r + c_i) c_i (the lattice sum inside Eq. SCforce,
 * reading R1) for every site.  S has layout [N][3]. */
void orc_stencil_sum(const int *dim, const double *rho, double *S) {
#pragma omp parallel for num_threads(orc_nthreads) schedule(static)
  for (long z = 0; z < dim[2]; ++z)
    for (long y = 0; y < dim[1]; ++y)
      for (long x = 0; x < dim[0]; ++x) {
        long s = orc_site(dim, x, y, z);
        for (int a = 0; a < 3; ++a) S[3 * s + a] = 0.0;
        for (int i = 1; i < ORC_Q; ++i) {
          double r2 = rho[orc_site(dim, x + orc_c[i][0], y + orc_c[i][1], z + orc_c[i][2])];
          for (int a = 0; a < 3; ++a) S[3 * s + a] += orc_w(i) * r2 * orc_c[i][a];
        }
      }
}

/* Eq. (SCforce) with psi = rho and g_AA = g_BB = 0 (readings R1):
 *   g^SC_A = -g_AB rho_A S_B,  g^SC_B = -g_BA rho_B S_A. */
void orc_sc_force(const int *dim, const double *rhoA, const double *rhoB, double gAB, double gBA,
                  double *gA, double *gB, double *SA, double *SB) {
  long N = (long)dim[0] * dim[1] * dim[2];
  orc_stencil_sum(dim, rhoA, SA);
  orc_stencil_sum(dim, rhoB, SB);
#pragma omp parallel for num_threads(orc_nthreads) schedule(static)
  for (long s = 0; s < N; ++s)
    for (int a = 0; a < 3; ++a) {
      gA[3 * s + a] = -gAB * rhoA[s] * SB[3 * s + a];
      gB[3 * s + a] = -gBA * rhoB[s] * SA[3 * s + a];
    }
}

/* ---------------------------------------------------------------------------
 * Philox4x32-10 counter-based generator, written from its published definition
 * (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64 multiplies with
 * multipliers 0xD2511F53 / 0xCD9E8D57 and a Weyl key schedule 0x9E3779B9 / 0xBB67AE85.
 * ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three unit normals for (seed, step, particle id), reading R9.  Counter = (id, step low,
 * step high, 0x4c42), key = (seed low, seed high); uniforms u = (top 24 bits + 1/2) / 2^24;
 * Box-Muller on (u0,u1) gives n0, n1 and on (u2,u3) gives n2. */
void orc_normals(uint64_t seed, uint64_t step, uint32_t id, double *n) {
  uint32_t ctr[4] = {id, (uint32_t)step, (uint32_t)(step >> 32), 0x4c42u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  orc_philox4x32_10(ctr, key, r);
  double u[4];
  for (int k = 0; k < 4; ++k) u[k] = ((double)(r[k] >> 8) + 0.5) / 16777216.0;
  const double two_pi = 6.283185307179586;
  double a = sqrt(-2.0 * log(u[0])), b = sqrt(-2.0 * log(u[2]));
  n[0] = a * cos(two_pi * u[1]);
  n[1] = a * sin(two_pi * u[1]);
  n[2] = b * cos(two_pi * u[3]);
}

/* Mode basis (R13): e_k(c_i) for k = 0..18 -- density; momentum x, y, z; bulk c^2 - 1; the
 * five shear modes 3c_x^2 - c^2, c_y^2 - c_z^2, c_x c_y, c_y c_z, c_z c_x; the kinetic modes
 * (3c^2 - 5) c_a, (c_y^2 - c_z^2) c_x, (c_z^2 - c_x^2) c_y, (c_x^2 - c_y^2) c_z, 3c^4 - 6c^2 + 1,
 * (2c^2 - 3)(3c_x^2 - c^2), (2c^2 - 3)(c_y^2 - c_z^2).  e has layout [k][i]; b_k = sum_i w_i e_ki^2. */
static double orc_mode_poly(int k, const int *c) {
  const double x = c[0], y = c[1], z = c[2], c2 = x * x + y * y + z * z;
  switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return c2 - 1.0;
    case 5: return 3.0 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return z * x;
    case 10: return (3.0 * c2 - 5.0) * x;
    case 11: return (3.0 * c2 - 5.0) * y;
    case 12: return (3.0 * c2 - 5.0) * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
    case 17: return (2.0 * c2 - 3.0) * (3.0 * x * x - c2);
    case 18: return (2.0 * c2 - 3.0) * (y * y - z * z);
  }
  return 0.0;
}

void orc_mode_basis(double *e, double *b) {
  for (int k = 0; k < ORC_Q; ++k) {
    b[k] = 0.0;
    for (int i = 0; i < ORC_Q; ++i) {
      e[k * ORC_Q + i] = orc_mode_poly(k, orc_c[i]);
      b[k] += orc_w(i) * e[k * ORC_Q + i] * e[k * ORC_Q + i];
    }
  }
}

/* The 36 unit normals of one node and step for the fluid noise (R13). */
void orc_fluid_normals(uint64_t seed, uint64_t step, uint32_t site, double *n) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const double two_pi = 6.283185307179586;
  for (uint32_t k = 0; k < 9; ++k) {
    uint32_t ctr[4] = {site, (uint32_t)step, (uint32_t)(step >> 32), 0x464c0000u + k};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    double u[4];
    for (int j = 0; j < 4; ++j) u[j] = ((double)(r[j] >> 8) + 0.5) / 16777216.0;
    double a = sqrt(-2.0 * log(u[0])), bb = sqrt(-2.0 * log(u[2]));
    n[4 * k + 0] = a * cos(two_pi * u[1]);
    n[4 * k + 1] = a * sin(two_pi * u[1]);
    n[4 * k + 2] = bb * cos(two_pi * u[3]);
    n[4 * k + 3] = bb * sin(two_pi * u[3]);
  }
}

/* Geometric factor of Eq. (solvation_lambda) for one particle seen from one node, readings R8:
 *   sum over the 18 neighbours r' = r + c_i of Theta[d_hat . c_hat_i] c_i / |c_i|^2,
 * with d = r_particle - r and Theta(x) = 1 for 0 < x < 1.  By Cauchy-Schwarz d_hat . c_hat <= 1
 * with equality iff d is parallel to c_i, so 0 < x < 1 is tested exactly as
 * (d . c_i > 0 and d x c_i != 0), free of rounding in the normalisation. */
void orc_fs_geometry(const double *d, double *out) {
  out[0] = out[1] = out[2] = 0.0;
  for (int i = 1; i < ORC_Q; ++i) {
    const int *c = orc_c[i];
    double c2 = (double)(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    double dc = d[0] * c[0] + d[1] * c[1] + d[2] * c[2];
    double cross[3] = {d[1] * c[2] - d[2] * c[1], d[2] * c[0] - d[0] * c[2], d[0] * c[1] - d[1] * c[0]};
    int parallel = cross[0] == 0.0 && cross[1] == 0.0 && cross[2] == 0.0;
    if (dc > 0.0 && !parallel)
      for (int a = 0; a < 3; ++a) out[a] += c[a] / c2;
  }
}

/* Pair potentials: WCA (Examples, Eq. for U^WCA) and screened Coulomb (Eq. for U^DH).
 * kind 0 = WCA(eps, sigma), kind 1 = DH(q_i q_j lB, kappa_D, rc), kind 2 = FENE(k, R0)
 * (Kremer-Grest form), kind 3 = harmonic(k, d).  Energy and the scalar -dU/dr. */
double orc_pair_energy(int kind, double p0, double p1, double p2, double r) {
  switch (kind) {
    case 0: {
      if (r >= pow(2.0, 1.0 / 6.0) * p1) return 0.0;
      double s6 = pow(p1 / r, 6.0);
      return 4.0 * p0 * (s6 * s6 - s6);
    }
    case 1:
      if (r >= p2) return 0.0;
      return p0 * exp(-p1 * r) / r;
    case 2:
      return -0.5 * p0 * p1 * p1 * log(1.0 - (r / p1) * (r / p1));
    case 3:
      return 0.5 * p0 * (r - p1) * (r - p1);
  }
  return 0.0;
}

double orc_pair_force(int kind, double p0, double p1, double p2, double r) {
  switch (kind) {
    case 0: {
      if (r >= pow(2.0, 1.0 / 6.0) * p1) return 0.0;
      double s6 = pow(p1 / r, 6.0);
      return 24.0 * p0 / r * (2.0 * s6 * s6 - s6);
    }
    case 1:
      if (r >= p2) return 0.0;
      return p0 * exp(-p1 * r) * (1.0 / (r * r) + p1 / r);
    case 2:
      return -p0 * r / (1.0 - (r / p1) * (r / p1));
    case 3:
      return -p0 * (r - p1);
  }
  return 0.0;
}

/* --------------------------------------------------------------------------
 * The coupled step.
 * ------------------------------------------------------------------------ */
typedef struct {
  int dim[3];
  double tau_r;          /* BGK relaxation time, lambda = -1/tau_r (R3) */
  double g_AB, g_BA;     /* Shan-Chen couplings (R1) */
  double kT;             /* thermal energy of the particle noise */
  double dt;             /* particle time step (lattice units, R9) */
  uint64_t seed;
  int ntypes;
  const double *kappa;   /* [ntypes][2]  Eq. solvation_kappa */
  const double *lam;     /* [ntypes][2]  Eq. solvation_lambda */
  const double *gamma;   /* [ntypes]     Eq. NEWTON */
  const double *mass;    /* [ntypes] */
  const double *wca_eps; /* [ntypes][ntypes] */
  const double *wca_sig; /* [ntypes][ntypes] */
  double dh_lB, dh_kappa, dh_rc; /* Debye-Hueckel (dh_lB = 0 switches it off) */
  int np;
  const int *type;       /* [np] */
  const double *q;       /* [np] charges */
  const int *pid;        /* [np] particle ids (noise counter) */
  int nbonds;
  const int *bonds;      /* [nbonds][2] */
  int bond_kind;         /* 2 = FENE, 3 = harmonic */
  double bond_k, bond_r;
  int collision;         /* 0 = BGK (R3), 1 = fluctuating MRT (R13) */
  double lam_bulk, lam_mom, lam_ghost; /* MRT eigenvalues; the shear one is -1/tau_r */
  int md_substeps;       /* K >= 1 particle substeps per lattice step (R15) */
} orc_system;

typedef struct {         /* optional outputs, each may be NULL */
  double *rho;           /* [2][N]       densities at the start of the step */
  double *u_cpl;         /* [N][3]       coupling velocity (R5) */
  double *g;             /* [2][N][3]    total force density per component */
  double *f_fric;        /* [np][3]      friction + noise force */
  double *f_ps;          /* [np][3]      sum_z F^ps_z */
  double *f_fs;          /* [np][3]      reaction of the fluid-side solvation force */
  double *f_pair;        /* [np][3]      pair forces */
  double *f_bond;        /* [np][3]      bond forces */
  double *f_total;       /* [np][3] */
} orc_trace;

static double orc_min_image(double d, double L) { return d - L * floor(d / L + 0.5); }

/* Trilinear weights and corner nodes of the unit cell that contains x (Sec. 2, "usually
 * employing a linear scheme").  corner k = (k&1, (k>>1)&1, (k>>2)&1). */
static void orc_trilinear(const int *dim, const double *x, long *cell, double *frac, long *node, double *w) {
  for (int a = 0; a < 3; ++a) {
    cell[a] = (long)floor(x[a]);
    frac[a] = x[a] - (double)cell[a];
  }
  for (int k = 0; k < 8; ++k) {
    int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
    double wk = 1.0;
    for (int a = 0; a < 3; ++a) wk *= o[a] ? frac[a] : 1.0 - frac[a];
    w[k] = wk;
    node[k] = orc_site(dim, cell[0] + o[0], cell[1] + o[1], cell[2] + o[2]);
  }
}

/* One time step n -> n+1.  f holds the post-streaming populations f_zi(r, t) with layout
 * [2][19][nz][ny][nx]; x, v are [np][3] and are advanced in place.  Returns 0, or -1 if a
 * density is non-positive, -2 if a FENE bond is stretched beyond R0.  Steps follow the
 * order: densities and momentum, Shan-Chen force, fluid-side solvation force, coupling
 * velocity, particle forces, momentum return, particle update (these three once per particle
 * substep, reading R15), collision with forcing, streaming. */
int orc_step(const orc_system *sys, double *f, double *x, double *v, uint64_t step, orc_trace *tr) {
  const int *dim = sys->dim;
  const long N = (long)dim[0] * dim[1] * dim[2];
  const int np = sys->np;
  int status = 0;
  double *rho = calloc(2 * N, sizeof(double));
  double *jp = calloc(3 * N, sizeof(double));
  double *S = calloc(2 * 3 * N, sizeof(double));
  double *gsc = calloc(2 * 3 * N, sizeof(double));
  double *ffs = calloc(2 * 3 * N, sizeof(double));
  double *gcp = calloc(2 * 3 * N, sizeof(double));
  double *ucpl = calloc(3 * N, sizeof(double));
  double *fnew = calloc(2 * ORC_Q * N, sizeof(double));
  double *P = calloc(11 * (size_t)(np > 0 ? np : 1) * 3, sizeof(double));
  double *pf_fric = P, *pf_psA = P + 3 * np, *pf_psB = P + 6 * np, *pf_fs = P + 9 * np;
  double *pf_pair = P + 12 * np, *pf_bond = P + 15 * np, *pf_tot = P + 18 * np;
  double *pu = P + 21 * np, *pgA = P + 24 * np, *pgB = P + 27 * np;

  /* 1. rho_z = sum_i f_zi (appendix, zeroth mode) and j' = sum_z sum_i f_zi c_i. */
#pragma omp parallel for num_threads(orc_nthreads) schedule(static)
  for (long s = 0; s < N; ++s)
    for (int z = 0; z < 2; ++z)
      for (int i = 0; i < ORC_Q; ++i) {
        double fi = f[((long)z * ORC_Q + i) * N + s];
        rho[z * N + s] += fi;
        for (int a = 0; a < 3; ++a) jp[3 * s + a] += fi * orc_c[i][a];
      }
  for (long s = 0; s < 2 * N; ++s)
    if (!(rho[s] > 0.0)) status = -1;

  /* 2. Shan-Chen force, Eq. (SCforce). */
  orc_sc_force(dim, rho, rho + N, sys->g_AB, sys->g_BA, gsc, gsc + 3 * N, S, S + 3 * N);

  /* 3. Fluid-side solvation force, Eq. (solvation_lambda), readings R8.  A node r sees the
   * particles of the 8 cells with corner r, i.e. a particle acts on the 8 corners of its own
   * cell; it receives minus what it exerts (R7). */
  for (int p = 0; p < np; ++p) {
    long cell[3], node[8];
    double frac[3], w[8];
    orc_trilinear(dim, x + 3 * p, cell, frac, node, w);
    int t = sys->type[p];
    for (int k = 0; k < 8; ++k) {
      double d[3] = {frac[0] - (k & 1), frac[1] - ((k >> 1) & 1), frac[2] - ((k >> 2) & 1)};
      double geo[3];
      orc_fs_geometry(d, geo);
      for (int z = 0; z < 2; ++z) {
        double lz = sys->lam[2 * t + z];
        for (int a = 0; a < 3; ++a) {
          double fz = -lz * rho[z * N + node[k]] * geo[a];
          ffs[3 * (z * N + node[k]) + a] += fz;
          pf_fs[3 * p + a] -= fz;
        }
      }
    }
  }

  /* 4. Coupling velocity, reading R5 (Eq. momentum_definition without the particle term). */
#pragma omp parallel for num_threads(orc_nthreads) schedule(static)
  for (long s = 0; s < N; ++s) {
    double r = rho[s] + rho[N + s];
    for (int a = 0; a < 3; ++a)
      ucpl[3 * s + a] = (jp[3 * s + a] + 0.5 * (gsc[3 * s + a] + gsc[3 * (N + s) + a] +
                                                 ffs[3 * s + a] + ffs[3 * (N + s) + a])) / r;
  }

  /* Steps 5, 6 and 9 run once per particle substep (reading R15; K = 1: once, with dt). */
  const int K = sys->md_substeps > 1 ? sys->md_substeps : 1;
  const double dts = sys->dt / K, wK = 1.0 / K;
  for (int sub = 0; sub < K; ++sub) {
  if (sub > 0) {
    memset(pu, 0, sizeof(double) * 9 * np);   /* pu, pgA, pgB */
    memset(pf_pair, 0, sizeof(double) * 6 * np); /* pf_pair, pf_bond */
  }

  /* 5. Particle forces at x(n), v(n): friction and noise (Eq. NEWTON), solvation
   * (Eq. solvation_kappa, reading R6), pair forces (WCA, DH) and bonds. */
  for (int p = 0; p < np; ++p) {
    long cell[3], node[8];
    double frac[3], w[8];
    orc_trilinear(dim, x + 3 * p, cell, frac, node, w);
    int t = sys->type[p];
    for (int k = 0; k < 8; ++k)
      for (int a = 0; a < 3; ++a) {
        pu[3 * p + a] += w[k] * ucpl[3 * node[k] + a];
        pgA[3 * p + a] += w[k] * S[3 * node[k] + a] / ORC_CS2;
        pgB[3 * p + a] += w[k] * S[3 * (N + node[k]) + a] / ORC_CS2;
      }
    double noise[3] = {0.0, 0.0, 0.0};
    if (sys->kT > 0.0) {
      double nrm[3];
      orc_normals(sys->seed, step * (uint64_t)K + (uint64_t)sub, (uint32_t)sys->pid[p], nrm);
      double amp = sqrt(2.0 * sys->kT * sys->gamma[t] / dts);
      for (int a = 0; a < 3; ++a) noise[a] = amp * nrm[a];
    }
    for (int a = 0; a < 3; ++a) {
      pf_fric[3 * p + a] = -sys->gamma[t] * (v[3 * p + a] - pu[3 * p + a]) + noise[a];
      pf_psA[3 * p + a] = -sys->kappa[2 * t + 0] * pgA[3 * p + a];
      pf_psB[3 * p + a] = -sys->kappa[2 * t + 1] * pgB[3 * p + a];
    }
  }
  for (int p = 0; p < np; ++p)
    for (int q2 = p + 1; q2 < np; ++q2) {
      double d[3], r2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        d[a] = orc_min_image(x[3 * p + a] - x[3 * q2 + a], (double)dim[a]);
        r2 += d[a] * d[a];
      }
      double r = sqrt(r2), fr = 0.0;
      int tp = sys->type[p], tq = sys->type[q2];
      double eps = sys->wca_eps[tp * sys->ntypes + tq], sig = sys->wca_sig[tp * sys->ntypes + tq];
      if (eps != 0.0 && sig > 0.0) fr += orc_pair_force(0, eps, sig, 0.0, r);
      if (sys->dh_lB != 0.0 && sys->q[p] != 0.0 && sys->q[q2] != 0.0)
        fr += orc_pair_force(1, sys->q[p] * sys->q[q2] * sys->dh_lB, sys->dh_kappa, sys->dh_rc, r);
      for (int a = 0; a < 3; ++a) {
        pf_pair[3 * p + a] += fr * d[a] / r;
        pf_pair[3 * q2 + a] -= fr * d[a] / r;
      }
    }
  for (int b = 0; b < sys->nbonds; ++b) {
    int p = sys->bonds[2 * b], q2 = sys->bonds[2 * b + 1];
    double d[3], r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      d[a] = orc_min_image(x[3 * p + a] - x[3 * q2 + a], (double)dim[a]);
      r2 += d[a] * d[a];
    }
    double r = sqrt(r2);
    if (sys->bond_kind == 2 && r >= sys->bond_r) status = -2;
    double fr = orc_pair_force(sys->bond_kind, sys->bond_k, sys->bond_r, 0.0, r);
    for (int a = 0; a < 3; ++a) {
      pf_bond[3 * p + a] += fr * d[a] / r;
      pf_bond[3 * q2 + a] -= fr * d[a] / r;
    }
  }

  /* 6. Momentum return onto the 8 corners (Sec. 2, reading R7). */
  for (int p = 0; p < np; ++p) {
    long cell[3], node[8];
    double frac[3], w[8];
    orc_trilinear(dim, x + 3 * p, cell, frac, node, w);
    for (int k = 0; k < 8; ++k) {
      long s = node[k];
      double r = rho[s] + rho[N + s];
      double sA = rho[s] / r, sB = rho[N + s] / r;
      for (int a = 0; a < 3; ++a) {
        gcp[3 * s + a] += wK * (w[k] * (-sA * pf_fric[3 * p + a] - pf_psA[3 * p + a]));
        gcp[3 * (N + s) + a] += wK * (w[k] * (-sB * pf_fric[3 * p + a] - pf_psB[3 * p + a]));
      }
    }
  }

  /* 9. Particle update (reading R9) with the substep dt / K (reading R15); the collision
   * below does not depend on the particle state any more. */
  for (int p = 0; p < np; ++p) {
    int t = sys->type[p];
    for (int a = 0; a < 3; ++a) {
      double F = pf_fric[3 * p + a] + pf_psA[3 * p + a] + pf_psB[3 * p + a] + pf_fs[3 * p + a] +
                 pf_pair[3 * p + a] + pf_bond[3 * p + a];
      pf_tot[3 * p + a] = F;
      v[3 * p + a] += F * dts / sys->mass[t];
      x[3 * p + a] += v[3 * p + a] * dts;
      x[3 * p + a] -= dim[a] * floor(x[3 * p + a] / dim[a]);
      if (x[3 * p + a] >= dim[a]) x[3 * p + a] = 0.0;
    }
  }
  }  /* substeps */

  /* 7. Collision with forcing (Eqs. EQ:LBapp, collis, feq, momentum_definition and the
   * forcing term), BGK reading R3 or fluctuating MRT (Eq. MODES, reading R13), then
   * 8. streaming f(r + c_i, t+1) = f*(r, t). */
  const double lam = -1.0 / sys->tau_r;
  const int mrt = sys->collision == 1;
  double E[ORC_Q * ORC_Q], bk[ORC_Q], lk[ORC_Q];
  orc_mode_basis(E, bk);
  for (int k = 0; k < ORC_Q; ++k)
    lk[k] = k == 0 ? 0.0 : k <= 3 ? sys->lam_mom : k == 4 ? sys->lam_bulk : k <= 9 ? lam : sys->lam_ghost;
#pragma omp parallel for num_threads(orc_nthreads) schedule(static)
  for (long zz = 0; zz < dim[2]; ++zz)
    for (long yy = 0; yy < dim[1]; ++yy)
      for (long xx = 0; xx < dim[0]; ++xx) {
        long s = orc_site(dim, xx, yy, zz);
        double gz[2][3], gt[3], u[3];
        double r = rho[s] + rho[N + s];
        for (int a = 0; a < 3; ++a) {
          for (int z = 0; z < 2; ++z)
            gz[z][a] = gsc[3 * (z * N + s) + a] + ffs[3 * (z * N + s) + a] + gcp[3 * (z * N + s) + a];
          gt[a] = gz[0][a] + gz[1][a];
          u[a] = (jp[3 * s + a] + 0.5 * gt[a]) / r;
        }
        if (tr && tr->g)
          for (int z = 0; z < 2; ++z)
            for (int a = 0; a < 3; ++a) tr->g[3 * (z * N + s) + a] = gz[z][a];
        double nrm[36];
        if (mrt && sys->kT > 0.0) orc_fluid_normals(sys->seed, step, (uint32_t)s, nrm);
        for (int z = 0; z < 2; ++z) {
          double feq[ORC_Q], dg[ORC_Q], fstar[ORC_Q];
          orc_feq(rho[z * N + s], u, feq);
          if (!mrt) {
            orc_forcing(gz[z], u, lam, lam, lam, dg);
            for (int i = 0; i < ORC_Q; ++i) {
              double fi = f[((long)z * ORC_Q + i) * N + s];
              fstar[i] = fi + lam * (fi - feq[i]) + dg[i];
            }
          } else {
            /* modes m_k = sum_i e_ki f_i, their equilibria and forcing moments, Eq. MODES */
            orc_forcing(gz[z], u, sys->lam_mom, lam, sys->lam_bulk, dg);
            double ms[ORC_Q];
            for (int k = 0; k < ORC_Q; ++k) {
              double m = 0.0, meq = 0.0, mg = 0.0;
              for (int i = 0; i < ORC_Q; ++i) {
                m += E[k * ORC_Q + i] * f[((long)z * ORC_Q + i) * N + s];
                meq += E[k * ORC_Q + i] * feq[i];
                mg += E[k * ORC_Q + i] * dg[i];
              }
              double noise = 0.0;
              if (sys->kT > 0.0 && k > 0) {
                const double rz = rho[z * N + s];
                if (k <= 3) {
                  double rr = rho[s] * rho[N + s] / r;
                  double phi = sqrt(sys->kT * rr * (1.0 - (1.0 + lk[k]) * (1.0 + lk[k])));
                  noise = (z == 0 ? 1.0 : -1.0) * phi * nrm[k - 1];
                } else {
                  double phi = sqrt(sys->kT / ORC_CS2 * rz * bk[k] * (1.0 - (1.0 + lk[k]) * (1.0 + lk[k])));
                  noise = phi * nrm[3 + 15 * z + (k - 4)];
                }
              }
              ms[k] = meq + (1.0 + lk[k]) * (m - meq) + mg + noise;
            }
            /* back to populations: f*_i = w_i sum_k e_ki m*_k / b_k */
            for (int i = 0; i < ORC_Q; ++i) {
              double acc = 0.0;
              for (int k = 0; k < ORC_Q; ++k) acc += E[k * ORC_Q + i] * ms[k] / bk[k];
              fstar[i] = orc_w(i) * acc;
            }
          }
          for (int i = 0; i < ORC_Q; ++i) {
            long dst = orc_site(dim, xx + orc_c[i][0], yy + orc_c[i][1], zz + orc_c[i][2]);
            fnew[((long)z * ORC_Q + i) * N + dst] = fstar[i];
          }
        }
      }
  memcpy(f, fnew, sizeof(double) * 2 * ORC_Q * N);

  if (tr) {
    if (tr->rho) memcpy(tr->rho, rho, sizeof(double) * 2 * N);
    if (tr->u_cpl) memcpy(tr->u_cpl, ucpl, sizeof(double) * 3 * N);
    for (int p = 0; p < np; ++p)
      for (int a = 0; a < 3; ++a) {
        if (tr->f_fric) tr->f_fric[3 * p + a] = pf_fric[3 * p + a];
        if (tr->f_ps) tr->f_ps[3 * p + a] = pf_psA[3 * p + a] + pf_psB[3 * p + a];
        if (tr->f_fs) tr->f_fs[3 * p + a] = pf_fs[3 * p + a];
        if (tr->f_pair) tr->f_pair[3 * p + a] = pf_pair[3 * p + a];
        if (tr->f_bond) tr->f_bond[3 * p + a] = pf_bond[3 * p + a];
        if (tr->f_total) tr->f_total[3 * p + a] = pf_tot[3 * p + a];
      }
  }
  free(rho); free(jp); free(S); free(gsc); free(ffs); free(gcp); free(ucpl); free(fnew); free(P);
  return status;
}

/* Equilibrium initialisation f_zi = f^eq_i(rho_z, u) (Eq. feq); u may be NULL (rest). */
void orc_init_equilibrium(const int *dim, const double *rhoA, const double *rhoB, const double *u, double *f) {
  long N = (long)dim[0] * dim[1] * dim[2];
#pragma omp parallel for num_threads(orc_nthreads) schedule(static)
  for (long s = 0; s < N; ++s) {
    double us[3] = {0.0, 0.0, 0.0};
    if (u)
      for (int a = 0; a < 3; ++a) us[a] = u[3 * s + a];
    double feq[ORC_Q];
    for (int z = 0; z < 2; ++z) {
      orc_feq(z == 0 ? rhoA[s] : rhoB[s], us, feq);
      for (int i = 0; i < ORC_Q; ++i) f[((long)z * ORC_Q + i) * N + s] = feq[i];
    }
  }
}

/* Global diagnostics: out = [M_A, M_B, Px, Py, Pz] with M_z = sum_r rho_z and
 * P = sum_r j'(r) (appendix: zeroth and first moments). */
void orc_fluid_moments(const int *dim, const double *f, double *out) {
  long N = (long)dim[0] * dim[1] * dim[2];
  for (int k = 0; k < 5; ++k) out[k] = 0.0;
  for (int z = 0; z < 2; ++z)
    for (int i = 0; i < ORC_Q; ++i)
      for (long s = 0; s < N; ++s) {
        double fi = f[((long)z * ORC_Q + i) * N + s];
        out[z] += fi;
        for (int a = 0; a < 3; ++a) out[2 + a] += fi * orc_c[i][a];
      }
}
