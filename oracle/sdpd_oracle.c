/*
 * sdpd_oracle.c -- plain, slow FP64 reference of one SDPD time step with the
 * Shardlow-like fluctuation/dissipation sweep and its Metropolis corrections
 * (Faure & Stoltz, "Stable and accurate schemes for Smoothed Dissipative
 * Particle Dynamics").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  It shares no code,
 * header, table or constant with the CUDA library, and the library never
 * calls it.
 *
 * Every pair quantity is computed by brute force over all N(N-1)/2 pairs with
 * the periodic minimum image; cell indices are used only to define the order
 * of the sequential sweep (owner block and colour of a pair).
 *
 * Readings of points the paper leaves open (they are also listed in the
 * design notes of the repository):
 *  R1  kernel: the cubic spline of Eq. (sdpd-cubic-w) and the Lucy kernel are
 *      both provided; the outer branch of the cubic F(r) is read as
 *      48/(pi h^5) (h/r)(1 - r/h)^2, which equals -W'(r)/r.
 *  R3  the density sum runs over j = 1..N and includes the self term m W(0).
 *  R4  ideal-gas entropy S = C_K ln(eps) - c_rho ln(rho), C_K = 3/2 (K-1) kB,
 *      c_rho = (K-1)/2 taken literally (a parameter here).
 *  R6  the pairwise OU update of Section 3.2 keeps the centre-of-mass
 *      momentum: p_i' = p_i + (m/2)(v' - v), p_j' = p_j - (m/2)(v' - v).
 *  R7  the noise amplitude of the relative-velocity proposal (Eq. proposal)
 *      is zt = (2/m) zeta, so that Eq. (proposal) is the relative-velocity
 *      form of Eq. (ssa-ou); the Metropolis ratio uses B = sum zt P.
 *  R10 pairs are r_ij < h strictly; a pair at r_ij = 0 is skipped.
 *  R11 one step = Velocity Verlet (Eq. sdpd-verlet) with the entropies held
 *      fixed, then one fluctuation/dissipation sweep; the first kick of every
 *      step is recomputed with the current (post-sweep) pressures.
 *  R12 sweep order: colour 0..7, owner cells of that colour by linear index,
 *      then, inside the owner's 2x2x2 block of cells, pairs by
 *      (rank(j) - rank(i), rank(i)), where rank(x) is the position of x's id
 *      among the ids of all particles in the block's 8 cells and i is the
 *      lower id.  Colour and owner are defined in orc_pair_owner below: along
 *      an axis where the two cells coincide, three bits drawn from the lower
 *      id choose which of the two blocks holding that coordinate owns the
 *      pair, which spreads a particle's pairs over the colours.
 *  R13 the energy bound of Eq. (energy-bound) rejects iff the smaller new
 *      internal energy is <= 0; the Metropolis step rejects iff U > exp(a).
 *      The internal-energy change is -1/2 of the change of the pair's kinetic
 *      energy computed from the updated momenta (Section 3.2), equal to
 *      -(m/8)(|v'|^2 - |v|^2) of Eq. (proposal-update).
 *  R14 random numbers: Philox4x64-10 (Salmon et al., SC'11) with
 *      key (seed, 0) and counter (fd_step, id_min, id_max, 0); the four
 *      64-bit words give G0, G1 (Box-Muller on two 53-bit uniforms), G2
 *      (Box-Muller on two 32-bit uniforms taken from word 2) and U (53 bits
 *      of word 3).
 *  R15 gradients: reverse mode of the Velocity Verlet dynamics of Section 3.1
 *      with the entropies as its constants (eps = E(S, rho(q))), by the chain
 *      rule through Eq. (pg-eos) and the density gradient of Eq.
 *      (gradient-rho); parameters theta = (h, c_rho, C_K) with kB, m and the
 *      box held fixed; the scalar observable is the virial pressure
 *      (1/3V)[sum |p|^2/m + sum_{i<j} r_ij . F_ij].  The sweep is not
 *      differentiated.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_KERNEL_CUBIC 0
#define ORC_KERNEL_LUCY 1

#define ORC_SCHEME_SSA 0
#define ORC_SCHEME_AMS 1
#define ORC_SCHEME_EMS 2
#define ORC_SCHEME_NONE 3 /* Velocity Verlet only */

#define ORC_OK 0
#define ORC_ERR_NEGATIVE_ENERGY 4
#define ORC_ERR_NOT_ADJACENT 9
#define ORC_ERR_ALLOC 10

#define ORC_ACCEPT 0
#define ORC_REJECT_BOUND 1
#define ORC_REJECT_METROPOLIS 2

typedef struct {
  int64_t N;
  double L[3];  /* periodic box sides */
  double m, h;  /* particle mass, smoothing length */
  double kB;
  double eta, zeta; /* shear and bulk viscosities */
  double C_K;   /* heat capacity 3/2 (K-1) kB (Section 4) */
  double c_rho; /* density coefficient of the entropy (Eq. pg-eos) */
  int kernel;
  int scheme;
  int n_c[3];   /* cells per axis (even, >= 4) */
  double cs[3]; /* cell side L / n_c (>= h) */
} orc_params;

typedef struct {
  int64_t n_pairs, n_accept, n_reject_bound, n_reject_metropolis, n_negative;
} orc_fd_stats;

typedef struct {
  int64_t id_i, id_j;  /* id_i < id_j */
  int32_t colour, owner;
  int32_t decision;
  int32_t pad;
  double margin;       /* EMS: a - ln U; AMS/bound: min new energy */
} orc_pair_rec;

/* ------------------------------------------------------------------------ */
/* Smoothing kernels, Section 2.1.1                                          */
/* ------------------------------------------------------------------------ */

/* W(r): cubic spline of Eq. (sdpd-cubic-w), or Lucy's kernel
 * W = 105/(16 pi h^3) (1 + 3x)(1 - x)^3 with x = r/h.  Both integrate to 1
 * over R^3 and vanish for r >= h. */
double orc_W(int kernel, double r, double h) {
  double x = r / h;
  if (x >= 1.0) return 0.0;
  if (kernel == ORC_KERNEL_CUBIC) {
    double c = 8.0 / (M_PI * h * h * h);
    if (x <= 0.5) return c * (1.0 - 6.0 * x * x + 6.0 * x * x * x);
    double y = 1.0 - x;
    return 2.0 * c * y * y * y;
  } else {
    double c = 105.0 / (16.0 * M_PI * h * h * h);
    double y = 1.0 - x;
    return c * (1.0 + 3.0 * x) * y * y * y;
  }
}

/* F(r) defined by grad W(r) = -F(|r|) r (Section 2.1.1).  Cubic spline:
 * 48/(pi h^5)(2 - 3x) for x <= 1/2 and 48/(pi h^5)(h/r)(1 - x)^2 for
 * 1/2 <= x <= 1 (reading R1).  Lucy: 315/(4 pi h^5)(1 - x)^2. */
double orc_F(int kernel, double r, double h) {
  double x = r / h;
  if (x >= 1.0) return 0.0;
  double h5 = h * h * h * h * h;
  if (kernel == ORC_KERNEL_CUBIC) {
    double c = 48.0 / (M_PI * h5);
    if (x <= 0.5) return c * (2.0 - 3.0 * x);
    double y = 1.0 - x;
    return c * (h / r) * y * y;
  } else {
    double c = 315.0 / (4.0 * M_PI * h5);
    double y = 1.0 - x;
    return c * y * y;
  }
}

/* ------------------------------------------------------------------------ */
/* Thermodynamic closure, Section 2.1.2, with the ideal gas of Eq. (pg-eos)  */
/* ------------------------------------------------------------------------ */

/* S(eps, rho) = C_K ln eps - c_rho ln rho */
double orc_S(const orc_params* P, double eps, double rho) {
  return P->C_K * log(eps) - P->c_rho * log(rho);
}
/* partial derivatives of S */
static double dS_deps(const orc_params* P, double eps) { return P->C_K / eps; }
static double d2S_deps2(const orc_params* P, double eps) { return -P->C_K / (eps * eps); }
static double dS_drho(const orc_params* P, double rho) { return -P->c_rho / rho; }

/* T = 1 / (dS/deps) */
double orc_T(const orc_params* P, double eps) { return 1.0 / dS_deps(P, eps); }
/* P = -(rho^2/m) (dS/drho)/(dS/deps) */
double orc_P(const orc_params* P, double eps, double rho) {
  return -(rho * rho / P->m) * dS_drho(P, rho) / dS_deps(P, eps);
}
/* C = -(dS/deps)^2 / (d2S/deps2) */
double orc_C(const orc_params* P, double eps) {
  double g = dS_deps(P, eps);
  return -(g * g) / d2S_deps2(P, eps);
}
/* Energy function E(S, rho): the inverse of S in eps at fixed rho
 * (Section 3.1), eps = exp((S + c_rho ln rho) / C_K). */
double orc_E_of_S(const orc_params* P, double S, double rho) {
  return exp((S + P->c_rho * log(rho)) / P->C_K);
}

/* ------------------------------------------------------------------------ */
/* Geometry: periodic minimum image, neighbour predicate, cells              */
/* ------------------------------------------------------------------------ */

double orc_min_image(double d, double L) {
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

/* r^2 of a displacement, with the two fused multiply-adds written out so the
 * neighbour predicate r^2 < h^2 is a fixed sequence of correctly rounded
 * operations. */
double orc_r2(double dx, double dy, double dz) {
  return fma(dz, dz, fma(dy, dy, dx * dx));
}

static void displacement(const orc_params* P, const double* q, int64_t i, int64_t j, double d[3]) {
  for (int k = 0; k < 3; ++k) d[k] = orc_min_image(q[3 * i + k] - q[3 * j + k], P->L[k]);
}

/* Periodic wrap of a coordinate into [0, L). */
double orc_wrap(double x, double L) {
  if (x >= L) x -= L;
  else if (x < 0.0) x += L;
  if (x >= L) x = 0.0; /* x < 0 by less than half an ulp of L */
  return x;
}

/* Cell index of a coordinate along one axis: floor(x / cs), clamped. */
int orc_cell_1d(const orc_params* P, int axis, double x) {
  int c = (int)floor(x / P->cs[axis]);
  if (c >= P->n_c[axis]) c = P->n_c[axis] - 1;
  if (c < 0) c = 0;
  return c;
}

void orc_cells(const orc_params* P, const double* q, int32_t* cell_xyz /* [N][3] */) {
  for (int64_t i = 0; i < P->N; ++i)
    for (int k = 0; k < 3; ++k) cell_xyz[3 * i + k] = orc_cell_1d(P, k, q[3 * i + k]);
}

/* 3-D Morton code of cell coordinates (bit interleave x, y, z; x lowest). */
uint64_t orc_morton3(uint32_t x, uint32_t y, uint32_t z) {
  uint64_t code = 0;
  for (int b = 0; b < 21; ++b) {
    code |= (uint64_t)((x >> b) & 1u) << (3 * b);
    code |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
    code |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
  }
  return code;
}

typedef struct { uint64_t key; int64_t id; } orc_key;
static int cmp_key(const void* a, const void* b) {
  const orc_key* x = (const orc_key*)a; const orc_key* y = (const orc_key*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->id < y->id ? -1 : (x->id > y->id);
}

/* Storage order of the particles: ascending (Morton code of the cell, id). */
int orc_sorted_order(const orc_params* P, const double* q, int64_t* order_ids) {
  orc_key* k = (orc_key*)malloc(sizeof(orc_key) * (size_t)(P->N ? P->N : 1));
  if (!k) return ORC_ERR_ALLOC;
  for (int64_t i = 0; i < P->N; ++i) {
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = orc_cell_1d(P, a, q[3 * i + a]);
    k[i].key = orc_morton3((uint32_t)c[0], (uint32_t)c[1], (uint32_t)c[2]);
    k[i].id = i;
  }
  qsort(k, (size_t)P->N, sizeof(orc_key), cmp_key);
  for (int64_t i = 0; i < P->N; ++i) order_ids[i] = k[i].id;
  free(k);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Density, Eq. (sdpd-rho-v), and conservative forces, Eq. (cons-forces)     */
/* ------------------------------------------------------------------------ */

/* rho_i = sum_{j=1..N} m W(r_ij), self term included (reading R3). */
void orc_density(const orc_params* P, const double* q, double* rho) {
  const double h2 = P->h * P->h;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < P->N; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < P->N; ++j) {
      double d[3];
      displacement(P, q, i, j, d);
      double r2 = orc_r2(d[0], d[1], d[2]);
      if (r2 < h2) s += P->m * orc_W(P->kernel, sqrt(r2), P->h);
    }
    rho[i] = s;
  }
}

/* Number of neighbours j != i with r_ij < h (for the neighbour-set check). */
void orc_neighbour_counts(const orc_params* P, const double* q, int32_t* count) {
  const double h2 = P->h * P->h;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < P->N; ++i) {
    int32_t c = 0;
    for (int64_t j = 0; j < P->N; ++j) {
      if (j == i) continue;
      double d[3];
      displacement(P, q, i, j, d);
      if (orc_r2(d[0], d[1], d[2]) < h2) ++c;
    }
    count[i] = c;
  }
}

/* F_i = sum_{j != i} m^2 (P_i/rho_i^2 + P_j/rho_j^2) F(r_ij) r_ij. */
void orc_forces(const orc_params* P, const double* q, const double* rho, const double* eps,
                double* force) {
  const double h2 = P->h * P->h;
  const double m2 = P->m * P->m;
  double* pi = (double*)malloc(sizeof(double) * (size_t)(P->N ? P->N : 1));
  for (int64_t i = 0; i < P->N; ++i) pi[i] = orc_P(P, eps[i], rho[i]) / (rho[i] * rho[i]);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < P->N; ++i) {
    double f[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < P->N; ++j) {
      if (j == i) continue;
      double d[3];
      displacement(P, q, i, j, d);
      double r2 = orc_r2(d[0], d[1], d[2]);
      if (r2 < h2) {
        double c = m2 * (pi[i] + pi[j]) * orc_F(P->kernel, sqrt(r2), P->h);
        for (int k = 0; k < 3; ++k) f[k] += c * d[k];
      }
    }
    for (int k = 0; k < 3; ++k) force[3 * i + k] = f[k];
  }
  free(pi);
}

/* Density of selected particles only (the same sum as orc_density, one
 * particle at a time): rho[k] = rho_{idx[k]}. */
void orc_density_at(const orc_params* P, const double* q, const int64_t* idx, int64_t n, double* rho) {
  const double h2 = P->h * P->h;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < n; ++k) {
    int64_t i = idx[k];
    double s = 0.0;
    for (int64_t j = 0; j < P->N; ++j) {
      double d[3];
      displacement(P, q, i, j, d);
      double r2 = orc_r2(d[0], d[1], d[2]);
      if (r2 < h2) s += P->m * orc_W(P->kernel, sqrt(r2), P->h);
    }
    rho[k] = s;
  }
}

/* Neighbour count (j != i, r_ij < h) of selected particles only. */
void orc_neighbour_count_at(const orc_params* P, const double* q, const int64_t* idx, int64_t n, int32_t* count) {
  const double h2 = P->h * P->h;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < n; ++k) {
    int64_t i = idx[k];
    int32_t c = 0;
    for (int64_t j = 0; j < P->N; ++j) {
      if (j == i) continue;
      double d[3];
      displacement(P, q, i, j, d);
      if (orc_r2(d[0], d[1], d[2]) < h2) ++c;
    }
    count[k] = c;
  }
}

/* Conservative force on selected particles (Eq. cons-forces), with the
 * densities of the particle and of each of its neighbours recomputed by the
 * full sum: force[3k..3k+2] = F_{idx[k]}. */
void orc_forces_at(const orc_params* P, const double* q, const double* eps, const int64_t* idx, int64_t n,
                   double* force) {
  const double h2 = P->h * P->h;
  const double m2 = P->m * P->m;
  for (int64_t k = 0; k < n; ++k) {
    int64_t i = idx[k];
    double rho_i;
    orc_density_at(P, q, &i, 1, &rho_i);
    double pi_i = orc_P(P, eps[i], rho_i) / (rho_i * rho_i);
    double f[3] = {0.0, 0.0, 0.0};
#pragma omp parallel
    {
      double fl[3] = {0.0, 0.0, 0.0};
#pragma omp for schedule(dynamic, 4096)
      for (int64_t j = 0; j < P->N; ++j) {
        if (j == i) continue;
        double d[3];
        displacement(P, q, i, j, d);
        double r2 = orc_r2(d[0], d[1], d[2]);
        if (r2 < h2) {
          double rho_j = 0.0;
          for (int64_t l = 0; l < P->N; ++l) {
            double e[3];
            displacement(P, q, j, l, e);
            double s2 = orc_r2(e[0], e[1], e[2]);
            if (s2 < h2) rho_j += P->m * orc_W(P->kernel, sqrt(s2), P->h);
          }
          double pi_j = orc_P(P, eps[j], rho_j) / (rho_j * rho_j);
          double c = m2 * (pi_i + pi_j) * orc_F(P->kernel, sqrt(r2), P->h);
          for (int a = 0; a < 3; ++a) fl[a] += c * d[a];
        }
      }
#pragma omp critical
      for (int a = 0; a < 3; ++a) f[a] += fl[a];
    }
    for (int a = 0; a < 3; ++a) force[3 * k + a] = f[a];
  }
}

/* Hamiltonian of Section 3.1 at fixed entropies:
 * H = sum |p_i|^2/(2m) + sum E(S_i, rho_i(q)). */
double orc_hamiltonian(const orc_params* P, const double* q, const double* p, const double* S) {
  double* rho = (double*)malloc(sizeof(double) * (size_t)(P->N ? P->N : 1));
  orc_density(P, q, rho);
  double H = 0.0;
  for (int64_t i = 0; i < P->N; ++i) {
    double p2 = p[3 * i] * p[3 * i] + p[3 * i + 1] * p[3 * i + 1] + p[3 * i + 2] * p[3 * i + 2];
    H += p2 / (2.0 * P->m) + orc_E_of_S(P, S[i], rho[i]);
  }
  free(rho);
  return H;
}

/* ------------------------------------------------------------------------ */
/* Velocity Verlet with fixed entropies, Eq. (sdpd-verlet) and Section 3.1   */
/* ------------------------------------------------------------------------ */

void orc_verlet(const orc_params* P, double* q, double* p, double* eps, double dt) {
  int64_t N = P->N;
  double* rho = (double*)malloc(sizeof(double) * (size_t)(N ? N : 1));
  double* S = (double*)malloc(sizeof(double) * (size_t)(N ? N : 1));
  double* f = (double*)malloc(sizeof(double) * 3 * (size_t)(N ? N : 1));
  /* entropies of the current state; they are invariants of this sub-step */
  orc_density(P, q, rho);
  for (int64_t i = 0; i < N; ++i) S[i] = orc_S(P, eps[i], rho[i]);
  /* p^{n+1/2} = p^n + F^n dt/2 */
  orc_forces(P, q, rho, eps, f);
  for (int64_t i = 0; i < 3 * N; ++i) p[i] += f[i] * (0.5 * dt);
  /* q^{n+1} = q^n + p^{n+1/2} dt / m, wrapped into the periodic box */
  for (int64_t i = 0; i < N; ++i)
    for (int k = 0; k < 3; ++k) q[3 * i + k] = orc_wrap(q[3 * i + k] + p[3 * i + k] * dt / P->m, P->L[k]);
  /* rho^{n+1}, then eps^{n+1} = E(S, rho^{n+1}) */
  orc_density(P, q, rho);
  for (int64_t i = 0; i < N; ++i) eps[i] = orc_E_of_S(P, S[i], rho[i]);
  /* p^{n+1} = p^{n+1/2} + F^{n+1} dt/2 */
  orc_forces(P, q, rho, eps, f);
  for (int64_t i = 0; i < 3 * N; ++i) p[i] += f[i] * (0.5 * dt);
  free(rho); free(S); free(f);
}

/* ------------------------------------------------------------------------ */
/* Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)         */
/* ------------------------------------------------------------------------ */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 prod = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(prod >> 64);
  *lo = (uint64_t)prod;
}

/* Ten rounds of the Philox S-box on a 4x64-bit counter with a 2x64-bit key.
 * Round: multiply words 0 and 2 by the two round multipliers, exchange the
 * high halves (xored with the other words and the key) and the low halves;
 * the key is bumped by the two Weyl increments between rounds. */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, x0, &hi0, &lo0);
    mulhilo64(M1, x2, &hi1, &lo1);
    uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static double u53(uint64_t w) { return ((double)(w >> 11) + 0.5) * 0x1.0p-53; }
static double u32(uint32_t w) { return ((double)w + 0.5) * 0x1.0p-32; }

/* The pair's random numbers for one fluctuation/dissipation step (R14):
 * G ~ N(0, I_3) and U ~ U(0, 1). */
void orc_pair_randoms(uint64_t seed, uint64_t fd_step, uint64_t id_i, uint64_t id_j, double G[3],
                      double* U) {
  uint64_t ctr[4] = {fd_step, id_i, id_j, 0};
  uint64_t key[2] = {seed, 0};
  uint64_t w[4];
  orc_philox4x64_10(ctr, key, w);
  double R = sqrt(-2.0 * log(u53(w[0])));
  double th = 2.0 * M_PI * u53(w[1]);
  G[0] = R * cos(th);
  G[1] = R * sin(th);
  double R2 = sqrt(-2.0 * log(u32((uint32_t)(w[2] >> 32))));
  G[2] = R2 * cos(2.0 * M_PI * u32((uint32_t)(w[2] & 0xffffffffULL)));
  *U = u53(w[3]);
}

/* ------------------------------------------------------------------------ */
/* Fluctuation/dissipation of one pair, Sections 2.2.2, 3.2 and 3.3         */
/* ------------------------------------------------------------------------ */

/* Coefficients of one pair at internal energies (eps_i, eps_j):
 * kappa (Section 2.2.2), d, gamma, sigma (Eq. sdpd-gamma-sigma), the OU
 * contraction alpha = exp(-2 gamma dt / m) and the relative-velocity noise
 * amplitude zt = (2/m) sigma sqrt(m (1 - alpha^2) / (4 gamma)) (R7), for
 * theta = parallel (index 0) and perpendicular (index 1). */
static void pair_coefficients(const orc_params* P, double kpar, double kperp, double eps_i,
                              double eps_j, double dt, double alpha[2], double zt[2]) {
  double Ti = orc_T(P, eps_i), Tj = orc_T(P, eps_j);
  double Ci = orc_C(P, eps_i), Cj = orc_C(P, eps_j);
  double d = P->kB * Ti * Tj / ((Ti + Tj) * (Ti + Tj)) * (1.0 / Ci + 1.0 / Cj);
  double kap[2] = {kpar, kperp};
  for (int t = 0; t < 2; ++t) {
    double gamma = kap[t] * (1.0 - d);
    double sigma = 2.0 * sqrt(kap[t] * P->kB * Ti * Tj / (Ti + Tj));
    alpha[t] = exp(-2.0 * gamma * dt / P->m);
    double one_m_a2 = -expm1(-4.0 * gamma * dt / P->m); /* 1 - alpha^2 */
    double zeta = sigma * sqrt(P->m * one_m_a2 / (4.0 * gamma));
    zt[t] = 2.0 * zeta / P->m;
  }
}

/* Split w into its component along e and the rest. */
static void split(const double e[3], const double w[3], double par[3], double perp[3]) {
  double s = e[0] * w[0] + e[1] * w[1] + e[2] * w[2];
  for (int k = 0; k < 3; ++k) { par[k] = s * e[k]; perp[k] = w[k] - par[k]; }
}

/* One pairwise fluctuation/dissipation update of (p_i, p_j, eps_i, eps_j)
 * for i = min id, j = max id, with r = q_i - q_j (minimum image) and the
 * densities at the current positions.  Returns ORC_ACCEPT or a rejection
 * code; *margin receives a - ln U (EMS) or the smaller new energy. */
int orc_fd_pair(const orc_params* P, const double r[3], double rho_i, double rho_j, double* p_i,
                double* p_j, double* eps_i, double* eps_j, double dt, const double G[3], double U,
                double* margin, int* negative) {
  const double m = P->m;
  double rr = sqrt(orc_r2(r[0], r[1], r[2]));
  double e[3] = {r[0] / rr, r[1] / rr, r[2] / rr};
  double Fij = orc_F(P->kernel, rr, P->h);
  /* kappa^par = (10/3 eta + 4 zeta) m^2 F / (rho_i rho_j),
   * kappa^perp = (5/3 eta - zeta) m^2 F / (rho_i rho_j) */
  double base = m * m * Fij / (rho_i * rho_j);
  double kpar = (10.0 / 3.0 * P->eta + 4.0 * P->zeta) * base;
  double kperp = (5.0 / 3.0 * P->eta - P->zeta) * base;

  /* current relative velocity v = (p_i - p_j)/m */
  double v[3];
  for (int k = 0; k < 3; ++k) v[k] = (p_i[k] - p_j[k]) / m;

  /* proposal, Eq. (proposal): v' = sum_theta P^theta (alpha v + zt G) */
  double alpha[2], zt[2];
  pair_coefficients(P, kpar, kperp, *eps_i, *eps_j, dt, alpha, zt);
  double vpar[3], vperp[3], Gpar[3], Gperp[3], vn[3];
  split(e, v, vpar, vperp);
  split(e, G, Gpar, Gperp);
  for (int k = 0; k < 3; ++k)
    vn[k] = alpha[0] * vpar[k] + alpha[1] * vperp[k] + zt[0] * Gpar[k] + zt[1] * Gperp[k];

  /* momenta of Eq. (proposal-update) and the energy redistributed equally */
  double pin[3], pjn[3];
  for (int k = 0; k < 3; ++k) {
    double dp = 0.5 * m * (vn[k] - v[k]);
    pin[k] = p_i[k] + dp;
    pjn[k] = p_j[k] - dp;
  }
  double ke_old = 0.0, ke_new = 0.0;
  for (int k = 0; k < 3; ++k) {
    ke_old += p_i[k] * p_i[k] + p_j[k] * p_j[k];
    ke_new += pin[k] * pin[k] + pjn[k] * pjn[k];
  }
  double deps = -0.5 * (ke_new - ke_old) / (2.0 * m);
  double ein = *eps_i + deps, ejn = *eps_j + deps;
  double emin = ein < ejn ? ein : ejn;

  int decision = ORC_ACCEPT;
  *margin = emin;
  if (P->scheme == ORC_SCHEME_SSA) {
    if (!(emin > 0.0)) *negative = 1;
  } else {
    /* energy bound, Eq. (energy-bound) */
    if (!(emin > 0.0)) {
      decision = ORC_REJECT_BOUND;
    } else if (P->scheme == ORC_SCHEME_EMS) {
      /* Metropolis ratio, Eq. (metropolis-ratio), with the reverse move
       * evaluated at the proposed energies */
      double alpha_r[2], zt_r[2];
      pair_coefficients(P, kpar, kperp, ein, ejn, dt, alpha_r, zt_r);
      double back[3];
      double vnpar[3], vnperp[3];
      split(e, vn, vnpar, vnperp);
      for (int k = 0; k < 3; ++k) back[k] = v[k] - (alpha_r[0] * vnpar[k] + alpha_r[1] * vnperp[k]);
      double bpar[3], bperp[3];
      split(e, back, bpar, bperp);
      double quad = 0.0, g2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        double w = bpar[k] / zt_r[0] + bperp[k] / zt_r[1];
        quad += w * w;
        g2 += G[k] * G[k];
      }
      double logdetB = log(zt[0]) + 2.0 * log(zt[1]);
      double logdetB_r = log(zt_r[0]) + 2.0 * log(zt_r[1]);
      double dS = (orc_S(P, ein, rho_i) - orc_S(P, *eps_i, rho_i) + orc_S(P, ejn, rho_j) -
                   orc_S(P, *eps_j, rho_j)) / P->kB;
      double dlogT = log(orc_T(P, ein)) - log(orc_T(P, *eps_i)) + log(orc_T(P, ejn)) -
                     log(orc_T(P, *eps_j));
      double a = 0.5 * g2 + logdetB - 0.5 * quad - logdetB_r + dS - dlogT;
      *margin = a - log(U);
      if (U > exp(a)) decision = ORC_REJECT_METROPOLIS;
    }
  }
  if (decision == ORC_ACCEPT) {
    for (int k = 0; k < 3; ++k) { p_i[k] = pin[k]; p_j[k] = pjn[k]; }
    *eps_i = ein;
    *eps_j = ejn;
  }
  return decision;
}

/* ------------------------------------------------------------------------ */
/* Pair colouring of the sequential sweep (reading R12)                      */
/* ------------------------------------------------------------------------ */

/* Three bits of a particle id: a multiply / xor-shift mix of the id as a
 * 32-bit unsigned integer, top three bits (bit k for axis k). */
unsigned orc_owner_bits(int64_t id) {
  uint32_t x = (uint32_t)id;
  x *= 2654435761u;
  x ^= x >> 15;
  x *= 2246822519u;
  x ^= x >> 13;
  x *= 3266489917u;
  x ^= x >> 16;
  return x >> 29;
}

/* The owner cell of a pair whose lower-id particle (id_lo) sits in cell a
 * and whose other particle sits in cell b.  Along each axis a and b are equal
 * or adjacent (the cell side is >= h).  Where they are adjacent the owner
 * takes the lower of the two in the periodic sense.  Where they are equal
 * the pair lies in the two blocks starting at a_k and a_k - 1; bit k of
 * orc_owner_bits(id_lo) picks a_k (0) or a_k - 1 (1).  Both cells then lie in
 * the 2x2x2 block of cells starting at the owner.  The pair's colour is the
 * parity pattern of the owner, (ox & 1) | (oy & 1) << 1 | (oz & 1) << 2.
 * Owners of one colour have disjoint blocks when every n_c is even and >= 4,
 * so the pairs of one colour touch disjoint particles. */
int orc_pair_owner(const orc_params* P, const int32_t ca[3], const int32_t cb[3], int64_t id_lo, int32_t o[3]) {
  const unsigned bits = orc_owner_bits(id_lo);
  for (int k = 0; k < 3; ++k) {
    int n = P->n_c[k];
    int diff = ((cb[k] - ca[k]) % n + n) % n;
    if (diff == 0) o[k] = (ca[k] - (int)((bits >> k) & 1u) + n) % n;
    else if (diff == 1) o[k] = ca[k];
    else if (diff == n - 1) o[k] = cb[k];
    else return ORC_ERR_NOT_ADJACENT;
  }
  return ORC_OK;
}

typedef struct {
  int64_t i, j;
  int32_t colour, owner;
  int32_t rank_i, rank_j; /* ranks of the ids inside the owner's block */
} orc_pair;

static int cmp_pair(const void* a, const void* b) {
  const orc_pair* x = (const orc_pair*)a; const orc_pair* y = (const orc_pair*)b;
  if (x->colour != y->colour) return x->colour < y->colour ? -1 : 1;
  if (x->owner != y->owner) return x->owner < y->owner ? -1 : 1;
  int32_t dx = x->rank_j - x->rank_i, dy = y->rank_j - y->rank_i;
  if (dx != dy) return dx < dy ? -1 : 1;
  if (x->rank_i != y->rank_i) return x->rank_i < y->rank_i ? -1 : 1;
  return 0;
}

/* Cells of all particles as linear indices, and per cell its member ids in
 * ascending order (cell_off[c] .. cell_off[c+1] in cell_mem). */
typedef struct {
  int64_t* cell_off;
  int64_t* cell_mem;
} orc_cell_lists;

static int build_cell_lists(const orc_params* P, const double* q, orc_cell_lists* cl) {
  int64_t ncell = (int64_t)P->n_c[0] * P->n_c[1] * P->n_c[2];
  cl->cell_off = (int64_t*)calloc((size_t)(ncell + 1), sizeof(int64_t));
  cl->cell_mem = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P->N ? P->N : 1));
  int64_t* lin = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P->N ? P->N : 1));
  if (!cl->cell_off || !cl->cell_mem || !lin) return ORC_ERR_ALLOC;
  for (int64_t k = 0; k < P->N; ++k) {
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = orc_cell_1d(P, a, q[3 * k + a]);
    lin[k] = c[0] + (int64_t)P->n_c[0] * (c[1] + (int64_t)P->n_c[1] * c[2]);
    cl->cell_off[lin[k] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) cl->cell_off[c + 1] += cl->cell_off[c];
  int64_t* fill = (int64_t*)calloc((size_t)(ncell ? ncell : 1), sizeof(int64_t));
  for (int64_t k = 0; k < P->N; ++k) /* ids ascending -> each list sorted */
    cl->cell_mem[cl->cell_off[lin[k]] + fill[lin[k]]++] = k;
  free(fill);
  free(lin);
  return ORC_OK;
}

/* rank of id among the particles of the 2x2x2 block of cells starting at the
 * owner cell: the number of particles in those 8 cells with a smaller id. */
static int32_t block_rank(const orc_params* P, const orc_cell_lists* cl, int64_t owner, int64_t id) {
  int o[3] = {(int)(owner % P->n_c[0]), (int)((owner / P->n_c[0]) % P->n_c[1]),
              (int)(owner / ((int64_t)P->n_c[0] * P->n_c[1]))};
  int32_t r = 0;
  for (int d = 0; d < 8; ++d) {
    int c[3] = {(o[0] + (d & 1)) % P->n_c[0], (o[1] + ((d >> 1) & 1)) % P->n_c[1],
                (o[2] + ((d >> 2) & 1)) % P->n_c[2]};
    int64_t lc = c[0] + (int64_t)P->n_c[0] * (c[1] + (int64_t)P->n_c[1] * c[2]);
    /* members of cell lc with an id below id: binary search of the sorted list */
    int64_t lo = cl->cell_off[lc], hi = cl->cell_off[lc + 1];
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (cl->cell_mem[mid] < id) lo = mid + 1;
      else hi = mid;
    }
    r += (int32_t)(lo - cl->cell_off[lc]);
  }
  return r;
}

/* All pairs i < j with r_ij < h, in sweep order.  Caller frees *out. */
int orc_enumerate_pairs(const orc_params* P, const double* q, orc_pair** out, int64_t* npairs) {
  int64_t N = P->N;
  const double h2 = P->h * P->h;
  int64_t* cnt = (int64_t*)calloc((size_t)(N + 1), sizeof(int64_t));
  if (!cnt) return ORC_ERR_ALLOC;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < N; ++i) {
    int64_t c = 0;
    for (int64_t j = i + 1; j < N; ++j) {
      double d[3];
      displacement(P, q, i, j, d);
      double r2 = orc_r2(d[0], d[1], d[2]);
      if (r2 < h2 && r2 > 0.0) ++c;
    }
    cnt[i + 1] = c;
  }
  for (int64_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
  int64_t np = cnt[N];
  orc_pair* pr = (orc_pair*)malloc(sizeof(orc_pair) * (size_t)(np ? np : 1));
  if (!pr) { free(cnt); return ORC_ERR_ALLOC; }
  int err = ORC_OK;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < N; ++i) {
    int64_t w = cnt[i];
    int32_t ci[3];
    for (int k = 0; k < 3; ++k) ci[k] = orc_cell_1d(P, k, q[3 * i + k]);
    for (int64_t j = i + 1; j < N; ++j) {
      double d[3];
      displacement(P, q, i, j, d);
      double r2 = orc_r2(d[0], d[1], d[2]);
      if (!(r2 < h2 && r2 > 0.0)) continue;
      int32_t cj[3], o[3];
      for (int k = 0; k < 3; ++k) cj[k] = orc_cell_1d(P, k, q[3 * j + k]);
      if (orc_pair_owner(P, ci, cj, i, o) != ORC_OK) {  /* i < j: i is the lower id */
#pragma omp atomic write
        err = ORC_ERR_NOT_ADJACENT;
        o[0] = o[1] = o[2] = 0;
      }
      pr[w].i = i;
      pr[w].j = j;
      pr[w].colour = (o[0] & 1) | ((o[1] & 1) << 1) | ((o[2] & 1) << 2);
      pr[w].owner = o[0] + P->n_c[0] * (o[1] + P->n_c[1] * o[2]);
      ++w;
    }
  }
  free(cnt);
  /* ranks of the two ids inside the owner's block */
  orc_cell_lists cl;
  if (build_cell_lists(P, q, &cl) != ORC_OK) { free(pr); return ORC_ERR_ALLOC; }
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t k = 0; k < np; ++k) {
    pr[k].rank_i = block_rank(P, &cl, pr[k].owner, pr[k].i);
    pr[k].rank_j = block_rank(P, &cl, pr[k].owner, pr[k].j);
  }
  free(cl.cell_off);
  free(cl.cell_mem);
  qsort(pr, (size_t)np, sizeof(orc_pair), cmp_pair);
  *out = pr;
  *npairs = np;
  return err;
}

/* One fluctuation/dissipation sweep over all pairs in sweep order, at fixed
 * positions (Sections 3.2-3.3).  The temperatures and heat capacities seen by
 * a pair are those of the energies left by the previous pairs. */
int orc_fd_sweep(const orc_params* P, const double* q, double* p, double* eps, double dt,
                 uint64_t seed, uint64_t fd_step, orc_fd_stats* st, orc_pair_rec* recs,
                 int64_t rec_cap) {
  int64_t N = P->N;
  double* rho = (double*)malloc(sizeof(double) * (size_t)(N ? N : 1));
  if (!rho) return ORC_ERR_ALLOC;
  orc_density(P, q, rho);
  orc_pair* pr = NULL;
  int64_t np = 0;
  int err = orc_enumerate_pairs(P, q, &pr, &np);
  if (err != ORC_OK && err != ORC_ERR_NOT_ADJACENT) { free(rho); return err; }
  int negative = 0;
  for (int64_t k = 0; k < np; ++k) {
    int64_t i = pr[k].i, j = pr[k].j;
    double r[3], G[3], U, margin;
    displacement(P, q, i, j, r);
    orc_pair_randoms(seed, fd_step, (uint64_t)i, (uint64_t)j, G, &U);
    int neg = 0;
    int dcs = orc_fd_pair(P, r, rho[i], rho[j], &p[3 * i], &p[3 * j], &eps[i], &eps[j], dt, G, U,
                          &margin, &neg);
    negative |= neg;
    if (st) {
      st->n_pairs++;
      if (dcs == ORC_ACCEPT) st->n_accept++;
      else if (dcs == ORC_REJECT_BOUND) st->n_reject_bound++;
      else st->n_reject_metropolis++;
      st->n_negative += neg;
    }
    if (recs && k < rec_cap) {
      recs[k].id_i = i; recs[k].id_j = j;
      recs[k].colour = pr[k].colour; recs[k].owner = pr[k].owner;
      recs[k].decision = dcs; recs[k].pad = 0; recs[k].margin = margin;
    }
  }
  free(pr);
  free(rho);
  if (err != ORC_OK) return err;
  return negative ? ORC_ERR_NEGATIVE_ENERGY : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Full steps: single time step (theta = 1) or multiple time step            */
/* ------------------------------------------------------------------------ */

/* nsteps Velocity Verlet steps of size dt; after every theta of them one
 * fluctuation/dissipation sweep with step theta*dt (Section 4.2; theta = 1 is
 * the plain splitting).  fd_only skips Velocity Verlet (Section 4.1).  The
 * sweep counter *fd_step numbers the sweeps and advances by one per sweep. */
int orc_run(const orc_params* P, double* q, double* p, double* eps, double dt, int64_t nsteps,
            int theta, int fd_only, uint64_t seed, uint64_t* fd_step, orc_fd_stats* st) {
  int status = ORC_OK;
  if (theta < 1) theta = 1;
  for (int64_t n = 0; n < nsteps; ++n) {
    if (!fd_only) orc_verlet(P, q, p, eps, dt);
    if (P->scheme != ORC_SCHEME_NONE && ((n + 1) % theta == 0)) {
      int s = orc_fd_sweep(P, q, p, eps, theta * dt, seed, *fd_step, st, NULL, 0);
      (*fd_step)++;
      if (s != ORC_OK && status == ORC_OK) status = s;
    }
  }
  return status;
}

/* ------------------------------------------------------------------------ */
/* Observables                                                               */
/* ------------------------------------------------------------------------ */

/* out[0] E = sum eps + |p|^2/2m, out[1] sum eps, out[2] kinetic energy,
 * out[3..5] total momentum, out[6] T_kin = sum |p|^2 / (3 (N-1) m),
 * out[7] mean internal temperature. */
void orc_observables(const orc_params* P, const double* p, const double* eps, double out[8]) {
  double se = 0.0, ke = 0.0, px = 0.0, py = 0.0, pz = 0.0, st = 0.0;
  for (int64_t i = 0; i < P->N; ++i) {
    const double* pi = &p[3 * i];
    se += eps[i];
    ke += (pi[0] * pi[0] + pi[1] * pi[1] + pi[2] * pi[2]) / (2.0 * P->m);
    px += pi[0]; py += pi[1]; pz += pi[2];
    st += orc_T(P, eps[i]);
  }
  out[0] = se + ke; out[1] = se; out[2] = ke;
  out[3] = px; out[4] = py; out[5] = pz;
  out[6] = P->N > 1 ? 2.0 * ke / (3.0 * (double)(P->N - 1)) : 0.0;
  out[7] = P->N > 0 ? st / (double)P->N : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Reverse-mode gradients of the conservative dynamics (Section 3.1)         */
/* ------------------------------------------------------------------------ */
/* A gradient here is the vector-Jacobian product of a map with a given
 * cotangent of its outputs; every routine ADDS its contribution to the
 * gradient arrays it is given.  The parameters differentiated are
 * theta = (h, c_rho, C_K) (kB, m and the box are held fixed).  Entropies are
 * the constants of the Velocity Verlet dynamics (the energies follow
 * eps = E(S, rho(q)) as in Section 3.1). */

/* dF/dr of the kernel function F(r) (grad W = -F r): Lucy -2c(1-x)/h; cubic
 * -3c/h for x <= 1/2 and -(c/h)(1-x)(1+x)/x^2 above (c = the F prefactor). */
double orc_dF_dr(int kernel, double r, double h) {
  double x = r / h;
  if (x >= 1.0) return 0.0;
  double h5 = h * h * h * h * h;
  if (kernel == ORC_KERNEL_CUBIC) {
    double c = 48.0 / (M_PI * h5);
    if (x <= 0.5) return -3.0 * c / h;
    return -(c / h) * (1.0 - x) * (1.0 + x) / (x * x);
  }
  double c = 315.0 / (4.0 * M_PI * h5);
  return -2.0 * c * (1.0 - x) / h;
}

/* dW/dh and dF/dh at fixed r.  W = h^-3 w(r/h), F = h^-5 phi(r/h) and
 * dW/dr = -r F give dW/dh = (r^2 F - 3 W)/h and dF/dh = -(5 F + r dF/dr)/h. */
double orc_dW_dh(int kernel, double r, double h) {
  return (r * r * orc_F(kernel, r, h) - 3.0 * orc_W(kernel, r, h)) / h;
}
double orc_dF_dh(int kernel, double r, double h) {
  return -(5.0 * orc_F(kernel, r, h) + r * orc_dF_dr(kernel, r, h)) / h;
}

/* Virial pressure of a state, (1/3V) [sum_i |p_i|^2/m + sum_{i<j} r_ij . F_ij]
 * with the pair forces of Eq. (cons-forces) and pi_i = P_i/rho_i^2 from
 * Eq. (pg-eos) at the state's own energies. */
double orc_virial_pressure(const orc_params* P, const double* q, const double* p, const double* eps) {
  int64_t N = P->N;
  const double h2 = P->h * P->h, m2 = P->m * P->m;
  double* rho = (double*)malloc(sizeof(double) * (size_t)(N ? N : 1));
  orc_density(P, q, rho);
  double kin = 0.0, vir = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    kin += (p[3 * i] * p[3 * i] + p[3 * i + 1] * p[3 * i + 1] + p[3 * i + 2] * p[3 * i + 2]) / P->m;
    double pi_i = orc_P(P, eps[i], rho[i]) / (rho[i] * rho[i]);
    for (int64_t j = i + 1; j < N; ++j) {
      double d[3];
      displacement(P, q, i, j, d);
      double r2 = orc_r2(d[0], d[1], d[2]);
      if (r2 < h2) {
        double pi_j = orc_P(P, eps[j], rho[j]) / (rho[j] * rho[j]);
        vir += m2 * (pi_i + pi_j) * orc_F(P->kernel, sqrt(r2), P->h) * r2;
      }
    }
  }
  free(rho);
  return (kin + vir) / (3.0 * P->L[0] * P->L[1] * P->L[2]);
}

/* Gradient through the density sum of Eq. (sdpd-rho-v): given rbar_i =
 * dL/drho_i, adds dL/dq (Eq. gradient-rho: d rho_i/d q_i = -m sum_j F r_ij,
 * d rho_j/d q_i = -m F r_ij) and dL/dh (the self term m W(0) included). */
void orc_density_vjp(const orc_params* P, const double* q, const double* rbar, double* gq, double gth[3]) {
  int64_t N = P->N;
  const double h = P->h, h2 = h * h, m = P->m;
  for (int64_t i = 0; i < N; ++i) gth[0] += rbar[i] * m * orc_dW_dh(P->kernel, 0.0, h);
  for (int64_t i = 0; i < N; ++i)
    for (int64_t j = i + 1; j < N; ++j) {
      double d[3];
      displacement(P, q, i, j, d);
      double r2 = orc_r2(d[0], d[1], d[2]);
      if (!(r2 < h2)) continue;
      double r = sqrt(r2);
      double f = orc_F(P->kernel, r, h);
      for (int k = 0; k < 3; ++k) {
        gq[3 * i + k] -= m * f * (rbar[i] + rbar[j]) * d[k];
        gq[3 * j + k] += m * f * (rbar[i] + rbar[j]) * d[k];
      }
      gth[0] += m * orc_dW_dh(P->kernel, r, h) * (rbar[i] + rbar[j]);
    }
}

/* Gradient of the pair sum
 *   Phi(q) = weight * sum_{i<j} m^2 (pi_i + pi_j) F(r_ij) t_ij
 * with t_ij = (v_i - v_j) . r_ij (mode 0: Phi = weight * sum_i v_i . F_i, the
 * pull-back of a kick) or t_ij = |r_ij|^2 (mode 1: the virial sum).
 * The pressures pi_i = c_rho eps_i / (C_K m rho_i) follow Eq. (pg-eos), with
 * x = the entropies S (fixed_S = 1, eps = E(S, rho(q))) or x = the energies
 * (fixed_S = 0).  Adds dPhi/dq to gq, dPhi/dx to gx and dPhi/dtheta to gth. */
void orc_pair_vjp(const orc_params* P, const double* q, const double* x, int fixed_S, int mode, const double* v,
                  double weight, double* gq, double* gx, double gth[3]) {
  int64_t N = P->N;
  const double h = P->h, h2 = h * h, m2 = P->m * P->m;
  const double CK = P->C_K, cr = P->c_rho;
  size_t n1 = (size_t)(N ? N : 1);
  double* rho = (double*)malloc(sizeof(double) * n1);
  double* pi = (double*)malloc(sizeof(double) * n1);
  double* A = (double*)calloc(n1, sizeof(double));
  double* rbar = (double*)malloc(sizeof(double) * n1);
  orc_density(P, q, rho);
  for (int64_t i = 0; i < N; ++i) {
    double eps = fixed_S ? orc_E_of_S(P, x[i], rho[i]) : x[i];
    pi[i] = orc_P(P, eps, rho[i]) / (rho[i] * rho[i]);
  }
  /* dPhi/dpi_i = weight * A_i, A_i = m^2 sum_{j != i} F(r_ij) t_ij */
  for (int64_t i = 0; i < N; ++i)
    for (int64_t j = i + 1; j < N; ++j) {
      double d[3];
      displacement(P, q, i, j, d);
      double r2 = orc_r2(d[0], d[1], d[2]);
      if (!(r2 < h2)) continue;
      double t = 0.0;
      for (int k = 0; k < 3; ++k) t += (mode == 0 ? v[3 * i + k] - v[3 * j + k] : d[k]) * d[k];
      double a = m2 * orc_F(P->kernel, sqrt(r2), h) * t;
      A[i] += a;
      A[j] += a;
    }
  /* pi = c_rho eps / (C_K m rho).  At fixed S, eps = exp((S + c_rho ln rho)/C_K):
   *   dpi/drho = pi (c_rho/C_K - 1)/rho, dpi/dS = pi/C_K,
   *   dpi/dc_rho = pi (1/c_rho + ln(rho)/C_K), dpi/dC_K = -pi (1 + ln(eps))/C_K.
   * At fixed eps: dpi/drho = -pi/rho, dpi/deps = pi/eps, dpi/dc_rho = pi/c_rho,
   *   dpi/dC_K = -pi/C_K. */
  for (int64_t i = 0; i < N; ++i) {
    double g = weight * A[i] * pi[i];
    if (fixed_S) {
      double eps = orc_E_of_S(P, x[i], rho[i]);
      rbar[i] = g * (cr / CK - 1.0) / rho[i];
      gx[i] += g / CK;
      gth[1] += g * (1.0 / cr + log(rho[i]) / CK);
      gth[2] -= g * (1.0 + log(eps)) / CK;
    } else {
      rbar[i] = -g / rho[i];
      gx[i] += g / x[i];
      gth[1] += g / cr;
      gth[2] -= g / CK;
    }
  }
  orc_density_vjp(P, q, rbar, gq, gth);
  /* the explicit dependence of each pair term on q and h */
  for (int64_t i = 0; i < N; ++i)
    for (int64_t j = i + 1; j < N; ++j) {
      double d[3];
      displacement(P, q, i, j, d);
      double r2 = orc_r2(d[0], d[1], d[2]);
      if (!(r2 < h2)) continue;
      double r = sqrt(r2);
      double f = orc_F(P->kernel, r, h), fp = orc_dF_dr(P->kernel, r, h);
      /* d(F(r) r_ij)/dq_i = F I + (F'/r) r_ij r_ij^T; at r = 0 (coincident
       * particles) the second term vanishes (t is O(r) or O(r^2)) */
      double fpr = r2 > 0.0 ? fp / r : 0.0;
      double c = weight * m2 * (pi[i] + pi[j]);
      double t = 0.0, dt_dqi[3];
      for (int k = 0; k < 3; ++k) {
        double u = mode == 0 ? v[3 * i + k] - v[3 * j + k] : d[k];
        t += u * d[k];
        dt_dqi[k] = mode == 0 ? u : 2.0 * d[k];
      }
      for (int k = 0; k < 3; ++k) {
        double g = c * (fpr * t * d[k] + f * dt_dqi[k]);
        gq[3 * i + k] += g;
        gq[3 * j + k] -= g;
      }
      gth[0] += c * t * orc_dF_dh(P->kernel, r, h);
    }
  free(rho); free(pi); free(A); free(rbar);
}

/* Gradient of the virial pressure of a state (q, p, eps) at its own
 * energies; adds dP/dq, dP/dp, dP/deps, dP/dtheta and returns P. */
double orc_virial_vjp(const orc_params* P, const double* q, const double* p, const double* eps, double* gq,
                      double* gp, double* geps, double gth[3]) {
  const double V3 = 3.0 * P->L[0] * P->L[1] * P->L[2];
  for (int64_t k = 0; k < 3 * P->N; ++k) gp[k] += 2.0 * p[k] / (V3 * P->m);
  orc_pair_vjp(P, q, eps, 0, 1, NULL, 1.0 / V3, gq, geps, gth);
  return orc_virial_pressure(P, q, p, eps);
}

/* Gradient of nsteps Velocity Verlet steps (Eq. sdpd-verlet, no sweep) from
 * (q0, p0, eps0) with the entropies S_i = S(eps0_i, rho_i(q0)) held fixed.
 * Given the cotangents (gqn, gpn, gepsn) of the final state, writes those of
 * the initial state and of theta (overwriting gq0, gp0, geps0, gth). */
void orc_vv_vjp(const orc_params* P, const double* q0, const double* p0, const double* eps0, double dt,
                int nsteps, const double* gqn, const double* gpn, const double* gepsn, double* gq0, double* gp0,
                double* geps0, double gth[3]) {
  int64_t N = P->N;
  size_t n1 = (size_t)(N ? N : 1), n3 = 3 * n1;
  double* qs = (double*)malloc(sizeof(double) * n3 * (size_t)(nsteps + 1));
  double* p = (double*)malloc(sizeof(double) * n3);
  double* eps = (double*)malloc(sizeof(double) * n1);
  double* rho = (double*)malloc(sizeof(double) * n1);
  double* S = (double*)malloc(sizeof(double) * n1);
  double* gS = (double*)calloc(n1, sizeof(double));
  double* rbar = (double*)malloc(sizeof(double) * n1);
  double* v = (double*)malloc(sizeof(double) * n3);
  orc_density(P, q0, rho);
  for (int64_t i = 0; i < N; ++i) S[i] = orc_S(P, eps0[i], rho[i]);
  /* forward, keeping every position */
  memcpy(qs, q0, sizeof(double) * 3 * (size_t)N);
  memcpy(p, p0, sizeof(double) * 3 * (size_t)N);
  memcpy(eps, eps0, sizeof(double) * (size_t)N);
  for (int n = 0; n < nsteps; ++n) {
    memcpy(qs + n3 * (size_t)(n + 1), qs + n3 * (size_t)n, sizeof(double) * 3 * (size_t)N);
    orc_verlet(P, qs + n3 * (size_t)(n + 1), p, eps, dt);
  }
  gth[0] = gth[1] = gth[2] = 0.0;
  double* gq = gq0;
  double* gp = gp0;
  memcpy(gq, gqn, sizeof(double) * 3 * (size_t)N);
  memcpy(gp, gpn, sizeof(double) * 3 * (size_t)N);
  /* final energies eps_n = E(S, rho(q_n)): dE/dS = eps/C_K,
   * dE/drho = eps c_rho/(C_K rho), dE/dc_rho = eps ln(rho)/C_K,
   * dE/dC_K = -eps ln(eps)/C_K */
  const double* qn = qs + n3 * (size_t)nsteps;
  orc_density(P, qn, rho);
  for (int64_t i = 0; i < N; ++i) {
    double e = orc_E_of_S(P, S[i], rho[i]), ge = gepsn[i] * e / P->C_K;
    gS[i] += ge;
    rbar[i] = ge * P->c_rho / rho[i];
    gth[1] += ge * log(rho[i]);
    gth[2] -= ge * log(e);
  }
  orc_density_vjp(P, qn, rbar, gq, gth);
  /* each step backwards: p1 = ph + dt/2 F(q1), q1 = q + dt ph/m,
   * ph = p + dt/2 F(q) */
  for (int n = nsteps - 1; n >= 0; --n) {
    for (size_t k = 0; k < 3 * (size_t)N; ++k) v[k] = 0.5 * dt * gp[k];
    orc_pair_vjp(P, qs + n3 * (size_t)(n + 1), S, 1, 0, v, 1.0, gq, gS, gth);
    for (size_t k = 0; k < 3 * (size_t)N; ++k) gp[k] += dt / P->m * gq[k];
    for (size_t k = 0; k < 3 * (size_t)N; ++k) v[k] = 0.5 * dt * gp[k];
    orc_pair_vjp(P, qs + n3 * (size_t)n, S, 1, 0, v, 1.0, gq, gS, gth);
  }
  /* S_i = C_K ln eps0_i - c_rho ln rho_i(q0) */
  orc_density(P, q0, rho);
  for (int64_t i = 0; i < N; ++i) {
    geps0[i] = gS[i] * P->C_K / eps0[i];
    rbar[i] = -gS[i] * P->c_rho / rho[i];
    gth[1] -= gS[i] * log(rho[i]);
    gth[2] += gS[i] * log(eps0[i]);
  }
  orc_density_vjp(P, q0, rbar, gq, gth);
  free(qs); free(p); free(eps); free(rho); free(S); free(gS); free(rbar); free(v);
}

/* Trajectory with the sweeps frozen: n steps of x_{k+1} = VV(x_k) + D_k,
 * where D_k = (dp_k [N][3], deps_k [N]) are given increments of the momenta
 * and internal energies (those that step k's fluctuation/dissipation sweep
 * produced, held fixed); NULL increments are zero.  Velocity Verlet
 * recomputes the entropies at every step from the current energies
 * (Section 3.1).  Updates (q, p, eps) in place. */
void orc_frozen_run(const orc_params* P, double* q, double* p, double* eps, double dt, int nsteps,
                    const double* dp, const double* deps) {
  int64_t N = P->N;
  for (int k = 0; k < nsteps; ++k) {
    orc_verlet(P, q, p, eps, dt);
    if (dp)
      for (int64_t i = 0; i < 3 * N; ++i) p[i] += dp[(size_t)k * 3 * (size_t)N + (size_t)i];
    if (deps)
      for (int64_t i = 0; i < N; ++i) eps[i] += deps[(size_t)k * (size_t)N + (size_t)i];
  }
}

/* Reverse mode of orc_frozen_run: given the cotangents (gqn, gpn, gepsn) of
 * the final state, writes those of (q0, p0, eps0) and of theta = (h, c_rho,
 * C_K).  Step k backwards: the increments pass cotangents through; the
 * final energies eps' = E(S_k, rho(q_{k+1})) and the two kicks at fixed S_k
 * are pulled back; then S_k = C_K ln eps_k - c_rho ln rho(q_k) carries the
 * entropy cotangent to the energies and positions at the start of step k. */
void orc_frozen_vjp(const orc_params* P, const double* q0, const double* p0, const double* eps0, double dt,
                    int nsteps, const double* dp, const double* deps, const double* gqn, const double* gpn,
                    const double* gepsn, double* gq0, double* gp0, double* geps0, double gth[3]) {
  int64_t N = P->N;
  size_t n1 = (size_t)(N ? N : 1), n3 = 3 * n1;
  double* qs = (double*)malloc(sizeof(double) * n3 * (size_t)(nsteps + 1));
  double* es = (double*)malloc(sizeof(double) * n1 * (size_t)(nsteps + 1));
  double* p = (double*)malloc(sizeof(double) * n3);
  double* rho = (double*)malloc(sizeof(double) * n1);
  double* S = (double*)malloc(sizeof(double) * n1);
  double* gS = (double*)malloc(sizeof(double) * n1);
  double* ge = (double*)malloc(sizeof(double) * n1);
  double* rbar = (double*)malloc(sizeof(double) * n1);
  double* v = (double*)malloc(sizeof(double) * n3);
  /* forward, keeping the positions and energies at every step start */
  memcpy(qs, q0, sizeof(double) * 3 * (size_t)N);
  memcpy(es, eps0, sizeof(double) * (size_t)N);
  memcpy(p, p0, sizeof(double) * 3 * (size_t)N);
  for (int k = 0; k < nsteps; ++k) {
    double* q = qs + n3 * (size_t)(k + 1);
    double* e = es + n1 * (size_t)(k + 1);
    memcpy(q, qs + n3 * (size_t)k, sizeof(double) * 3 * (size_t)N);
    memcpy(e, es + n1 * (size_t)k, sizeof(double) * (size_t)N);
    orc_frozen_run(P, q, p, e, dt, 1, dp ? dp + (size_t)k * 3 * (size_t)N : NULL,
                   deps ? deps + (size_t)k * (size_t)N : NULL);
  }
  gth[0] = gth[1] = gth[2] = 0.0;
  double* gq = gq0;
  double* gp = gp0;
  memcpy(gq, gqn, sizeof(double) * 3 * (size_t)N);
  memcpy(gp, gpn, sizeof(double) * 3 * (size_t)N);
  memcpy(ge, gepsn, sizeof(double) * (size_t)N);
  for (int k = nsteps - 1; k >= 0; --k) {
    const double* qk = qs + n3 * (size_t)k;
    const double* q1 = qs + n3 * (size_t)(k + 1);
    const double* ek = es + n1 * (size_t)k;
    orc_density(P, qk, rho);
    for (int64_t i = 0; i < N; ++i) {
      S[i] = orc_S(P, ek[i], rho[i]);
      gS[i] = 0.0;
    }
    /* eps' = E(S_k, rho(q_{k+1})) at the end of the Verlet step */
    orc_density(P, q1, rho);
    for (int64_t i = 0; i < N; ++i) {
      double e = orc_E_of_S(P, S[i], rho[i]), g = ge[i] * e / P->C_K;
      gS[i] += g;
      rbar[i] = g * P->c_rho / rho[i];
      gth[1] += g * log(rho[i]);
      gth[2] -= g * log(e);
    }
    orc_density_vjp(P, q1, rbar, gq, gth);
    /* second kick at q_{k+1}, drift, first kick at q_k (fixed S_k) */
    for (size_t j = 0; j < 3 * (size_t)N; ++j) v[j] = 0.5 * dt * gp[j];
    orc_pair_vjp(P, q1, S, 1, 0, v, 1.0, gq, gS, gth);
    for (size_t j = 0; j < 3 * (size_t)N; ++j) gp[j] += dt / P->m * gq[j];
    for (size_t j = 0; j < 3 * (size_t)N; ++j) v[j] = 0.5 * dt * gp[j];
    orc_pair_vjp(P, qk, S, 1, 0, v, 1.0, gq, gS, gth);
    /* S_k = C_K ln eps_k - c_rho ln rho(q_k) */
    orc_density(P, qk, rho);
    for (int64_t i = 0; i < N; ++i) {
      ge[i] = gS[i] * P->C_K / ek[i];
      rbar[i] = -gS[i] * P->c_rho / rho[i];
      gth[1] -= gS[i] * log(rho[i]);
      gth[2] += gS[i] * log(ek[i]);
    }
    orc_density_vjp(P, qk, rbar, gq, gth);
  }
  memcpy(geps0, ge, sizeof(double) * (size_t)N);
  free(qs); free(es); free(p); free(rho); free(S); free(gS); free(ge); free(rbar); free(v);
}

int orc_sizeof_params(void) { return (int)sizeof(orc_params); }
int orc_sizeof_pair_rec(void) { return (int)sizeof(orc_pair_rec); }
