/*
 * FP64 oracle for the two-component Shan-Chen D3Q19 step with the evaporation
 * boundary (arXiv:1701.03637, Sec. II). TEST INFRASTRUCTURE ONLY: the product
 * never links it. Plain loops, in the order the paper states the method:
 *
 *   densities       rho^c = sum_i f_i^c                        (Sec. II A, after Eq. 2)
 *   pseudopotential Psi(rho) = 1 - exp(-rho/rho0), rho0 = 1    (Eq. 4)
 *   force           F^c = -Psi^c(x) sum_cbar g^{c cbar} sum_i w_i Psi^cbar(x+e_i) e_i   (Eq. 3),
 *                   the sum over cbar in {r, b} with g^{rb} = g^{br} = G and the self
 *                   couplings g^{rr}, g^{bb} (0 in the paper's runs; g^{cc} < 0 is the
 *                   multiphase pseudopotential model the paper names as an extension)
 *   common velocity u' = sum_c (m^c/tau_c) / sum_c (rho^c/tau_c) (reduces to the
 *                   paper's mass-weighted u_eq when tau_r = tau_b)   (Sec. II A)
 *   shifted velocity u^c_eq = u' + tau_c F^c / rho^c             (Sec. II B)
 *   BGK collision toward f^eq(rho^c, u^c_eq)                     (Eqs. 1, 2)
 *   streaming with periodic wrap, halfway bounce-back at solid sites (Sec. II A)
 *   evaporation boundary: at sink sites f^r_i = w_i rho_H and
 *   f^b_i = w_i (rho^r + rho^b - rho_H) from the populations that arrived
 *   (Sec. II C, the two fixed-density equations and the mass-conserving
 *   complement).
 *
 * Readings where the paper is silent (stated in the design notes too):
 *   - canonical state = post-stream, post-sink-reset populations;
 *   - sink sites are neither forced nor collided (forces act in the bulk only);
 *   - solid sites have Psi = 0 and hold no populations;
 *   - the evaporated mass counts sum over sink sites of (rho^r_arrived - rho_H).
 */
#include "sc_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* D3Q19: rest, 6 axis, 12 face diagonals; opposite pairs adjacent (i odd <-> i+1). */
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static double W[Q];
static int OPP[Q];
static int tables_ready = 0;
static int n_threads = 1;

static void make_tables(void) {
  if (tables_ready) return;
  for (int i = 0; i < Q; ++i) {
    int c2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
    W[i] = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0); /* weights, Sec. II A */
    for (int j = 0; j < Q; ++j)
      if (CX[j] == -CX[i] && CY[j] == -CY[i] && CZ[j] == -CZ[i]) OPP[i] = j;
  }
  tables_ready = 1;
}

struct orc_lattice {
  orc_params p;
  int64_t n;
  double* f;      /* [2][Q][n] canonical */
  double* ftmp;   /* [2][Q][n] post-collision */
  double* rho;    /* [2][n] */
  double* psi;    /* [2][n] */
  int8_t* cls;    /* 0 fluid, 1 sink, 2 solid */
  int64_t step;
  double evaporated, flux_last;
};

static int64_t wrapi(int64_t v, int64_t n) { v %= n; return v < 0 ? v + n : v; }

static int classify(const orc_params* p, int x, int y, int z) {
  if (p->wall_thickness > 0 && z >= p->wall_z0 && z < p->wall_z0 + p->wall_thickness) return 2;
  if (p->geometry == 1) {
    if (wrapi((int64_t)z - p->sink_z0, p->nz) < p->sink_layers) return 1;
  } else if (p->geometry == 2) {
    double dx = x - p->sphere_cx, dy = y - p->sphere_cy, dz = z - p->sphere_cz;
    if (dx * dx + dy * dy + dz * dz >= p->R_H * p->R_H) return 1;
  }
  return 0;
}

void orc_set_threads(int n) { n_threads = n < 1 ? 1 : n; }
int orc_threads(void) { return n_threads; }

int orc_create(const orc_params* p, orc_lattice** out) {
  make_tables();
  if (!p || !out || p->nx < 1 || p->ny < 1 || p->nz < 1 || p->tau_r <= 0.5 || p->tau_b <= 0.5) return -1;
  orc_lattice* L = (orc_lattice*)calloc(1, sizeof(orc_lattice));
  L->p = *p;
  L->n = (int64_t)p->nx * p->ny * p->nz;
  L->f = (double*)calloc((size_t)(2 * Q * L->n), sizeof(double));
  L->ftmp = (double*)calloc((size_t)(2 * Q * L->n), sizeof(double));
  L->rho = (double*)calloc((size_t)(2 * L->n), sizeof(double));
  L->psi = (double*)calloc((size_t)(2 * L->n), sizeof(double));
  L->cls = (int8_t*)calloc((size_t)L->n, 1);
  if (!L->f || !L->ftmp || !L->rho || !L->psi || !L->cls) { orc_destroy(L); return -2; }
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x)
        L->cls[x + (int64_t)p->nx * (y + (int64_t)p->ny * z)] = (int8_t)classify(p, x, y, z);
  *out = L;
  return 0;
}

void orc_destroy(orc_lattice* L) {
  if (!L) return;
  free(L->f); free(L->ftmp); free(L->rho); free(L->psi); free(L->cls); free(L);
}

#define F(L, c, i, s) ((L)->f[((int64_t)(c) * Q + (i)) * (L)->n + (s)])

/* Evaporation boundary (Sec. II C): returns rho^r_arrived - rho_H summed over sinks. */
static double sink_reset(orc_lattice* L) {
  double evap = 0.0;
  for (int64_t s = 0; s < L->n; ++s) {
    if (L->cls[s] != 1) continue;
    double rr = 0.0, rb = 0.0;
    for (int i = 0; i < Q; ++i) { rr += F(L, 0, i, s); rb += F(L, 1, i, s); }
    double rb_new = rr + rb - L->p.rho_H;
    for (int i = 0; i < Q; ++i) {
      F(L, 0, i, s) = W[i] * L->p.rho_H;   /* f^eq(rho_H, u = 0) */
      F(L, 1, i, s) = W[i] * rb_new;       /* f^eq(rho^cbar_H, u = 0) */
    }
    evap += rr - L->p.rho_H;
  }
  return evap;
}

void orc_lattice_tables(int32_t* c, double* w, int32_t* opp) {
  make_tables();
  for (int i = 0; i < Q; ++i) {
    if (c) { c[3 * i] = CX[i]; c[3 * i + 1] = CY[i]; c[3 * i + 2] = CZ[i]; }
    if (w) w[i] = W[i];
    if (opp) opp[i] = OPP[i];
  }
}

/* Second-order equilibrium, Eq. (2), c_s^2 = 1/3. */
void orc_feq(double rho, const double* u, double* feq) {
  make_tables();
  const double cs2 = 1.0 / 3.0;
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
    feq[i] = W[i] * rho * (1.0 + cu / cs2 - uu / (2.0 * cs2) + cu * cu / (2.0 * cs2 * cs2));
  }
}

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the k-th output of the
   generator seeded with `seed` is the finaliser applied to seed + k*gamma. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double orc_uniform(uint64_t seed, uint64_t k) {
  return (double)(orc_splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

int orc_init_fields(orc_lattice* L, const double* rho_r, const double* rho_b) {
  make_tables();
  for (int64_t s = 0; s < L->n; ++s)
    for (int i = 0; i < Q; ++i) {
      int solid = L->cls[s] == 2;
      F(L, 0, i, s) = solid ? 0.0 : W[i] * rho_r[s];
      F(L, 1, i, s) = solid ? 0.0 : W[i] * rho_b[s];
    }
  sink_reset(L);
  L->step = 0; L->evaporated = 0.0; L->flux_last = 0.0;
  return 0;
}

int orc_init_shape(orc_lattice* L, const orc_init* in) {
  const orc_params* p = &L->p;
  double* rr = (double*)malloc(sizeof(double) * (size_t)L->n);
  double* rb = (double*)malloc(sizeof(double) * (size_t)L->n);
  if (!rr || !rb) { free(rr); free(rb); return -2; }
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        int64_t s = x + (int64_t)p->nx * (y + (int64_t)p->ny * z);
        int rich;
        if (in->shape == 0) rich = z < in->film_z;
        else {
          double dx = x - in->cx, dy = y - in->cy, dz = z - in->cz;
          rich = dx * dx + dy * dy + dz * dz < in->radius * in->radius;
        }
        double nr = in->noise_amp * (2.0 * orc_uniform(in->seed, 1 + (uint64_t)s) - 1.0);
        double nb = in->noise_amp * (2.0 * orc_uniform(in->seed, 1 + (uint64_t)L->n + (uint64_t)s) - 1.0);
        rr[s] = (rich ? in->rho_hi : in->rho_lo) + nr;
        rb[s] = (rich ? in->rho_lo : in->rho_hi) + nb;
      }
  int rc = orc_init_fields(L, rr, rb);
  free(rr); free(rb);
  return rc;
}

int orc_set_populations(orc_lattice* L, const double* f) {
  memcpy(L->f, f, sizeof(double) * (size_t)(2 * Q * L->n));
  for (int64_t s = 0; s < L->n; ++s)
    if (L->cls[s] == 2)
      for (int c = 0; c < 2; ++c)
        for (int i = 0; i < Q; ++i) F(L, c, i, s) = 0.0;
  sink_reset(L);
  return 0;
}

void orc_get_populations(const orc_lattice* L, double* f) {
  memcpy(f, L->f, sizeof(double) * (size_t)(2 * Q * L->n));
}

static void densities(orc_lattice* L) {
  const int64_t n = L->n;
#pragma omp parallel for num_threads(n_threads) schedule(static)
  for (int64_t s = 0; s < n; ++s) {
    for (int c = 0; c < 2; ++c) {
      double r = 0.0;
      if (L->cls[s] != 2)
        for (int i = 0; i < Q; ++i) r += F(L, c, i, s);
      L->rho[c * n + s] = r;
      L->psi[c * n + s] = (L->cls[s] == 2) ? 0.0 : 1.0 - exp(-r); /* Eq. (4) */
    }
  }
}

/* Eq. (3) at fluid site (x, y, z) from the current Psi: for each component c,
   F^c = -Psi^c(x) sum_cbar g^{c cbar} sum_{i>=1} w_i Psi^cbar(x + e_i) e_i, periodic
   neighbours (solid ones have Psi = 0). The cross term is evaluated first, as
   -Psi^c(x) G a^cbar; the self term -Psi^c(x) g^{cc} a^c is added to it. */
static void force(const orc_lattice* L, int x, int y, int z, double Fc[2][3]) {
  const orc_params* p = &L->p;
  const int64_t n = L->n;
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const int64_t s = x + (int64_t)nx * (y + (int64_t)ny * z);
  const double gself[2] = {p->G_rr, p->G_bb};
  double a[2][3] = {{0, 0, 0}, {0, 0, 0}};  /* a^cbar = sum_i w_i Psi^cbar(x + e_i) e_i */
  for (int cb = 0; cb < 2; ++cb)
    for (int i = 1; i < Q; ++i) {
      int64_t xn = wrapi(x + CX[i], nx), yn = wrapi(y + CY[i], ny), zn = wrapi(z + CZ[i], nz);
      double pn = L->psi[cb * n + xn + (int64_t)nx * (yn + (int64_t)ny * zn)];
      a[cb][0] += W[i] * pn * CX[i];
      a[cb][1] += W[i] * pn * CY[i];
      a[cb][2] += W[i] * pn * CZ[i];
    }
  for (int c = 0; c < 2; ++c)
    for (int d = 0; d < 3; ++d) {
      Fc[c][d] = -L->psi[c * n + s] * p->G * a[1 - c][d];
      if (gself[c] != 0.0) Fc[c][d] += -L->psi[c * n + s] * gself[c] * a[c][d];
    }
}

static void one_step(orc_lattice* L) {
  const orc_params* p = &L->p;
  const int64_t n = L->n;
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const double tau[2] = {p->tau_r, p->tau_b};
  densities(L);

  /* Force, shifted velocities and BGK collision into ftmp. */
#pragma omp parallel for num_threads(n_threads) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t s = x + (int64_t)nx * (y + (int64_t)ny * z);
        if (L->cls[s] != 0) {  /* sink and solid sites are not collided */
          for (int c = 0; c < 2; ++c)
            for (int i = 0; i < Q; ++i) L->ftmp[((int64_t)c * Q + i) * n + s] = F(L, c, i, s);
          continue;
        }
        double Fc[2][3];
        force(L, x, y, z, Fc);
        double m[2][3] = {{0, 0, 0}, {0, 0, 0}};
        for (int c = 0; c < 2; ++c)
          for (int i = 0; i < Q; ++i) {
            double fi = F(L, c, i, s);
            m[c][0] += fi * CX[i]; m[c][1] += fi * CY[i]; m[c][2] += fi * CZ[i];
          }
        double den = L->rho[s] / tau[0] + L->rho[n + s] / tau[1];
        double up[3] = {0, 0, 0};
        if (den > 0)
          for (int d = 0; d < 3; ++d) up[d] = (m[0][d] / tau[0] + m[1][d] / tau[1]) / den;
        for (int c = 0; c < 2; ++c) {
          double r = L->rho[c * n + s];
          double ueq[3];
          for (int d = 0; d < 3; ++d) ueq[d] = up[d] + (r > 0 ? tau[c] * Fc[c][d] / r : 0.0);
          double feq[Q];
          orc_feq(r, ueq, feq);
          for (int i = 0; i < Q; ++i) {
            double fi = F(L, c, i, s);
            L->ftmp[((int64_t)c * Q + i) * n + s] = fi - (fi - feq[i]) / tau[c]; /* Eq. (1) */
          }
        }
      }

  /* Streaming (push), periodic wrap, halfway bounce-back into solid sites. */
  memset(L->f, 0, sizeof(double) * (size_t)(2 * Q * n));
#pragma omp parallel for num_threads(n_threads) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t s = x + (int64_t)nx * (y + (int64_t)ny * z);
        if (L->cls[s] == 2) continue;
        for (int i = 0; i < Q; ++i) {
          int64_t xn = wrapi(x + CX[i], nx), yn = wrapi(y + CY[i], ny), zn = wrapi(z + CZ[i], nz);
          int64_t d = xn + (int64_t)nx * (yn + (int64_t)ny * zn);
          for (int c = 0; c < 2; ++c) {
            double v = L->ftmp[((int64_t)c * Q + i) * n + s];
            if (L->cls[d] == 2) F(L, c, OPP[i], s) = v;
            else F(L, c, i, d) = v;
          }
        }
      }

  double e = sink_reset(L);
  L->evaporated += e;
  L->flux_last = e;
  L->step += 1;
}

void orc_step(orc_lattice* L, int64_t nsteps) {
  for (int64_t t = 0; t < nsteps; ++t) one_step(L);
}

void orc_fields(const orc_lattice* L, double* rho_r, double* rho_b) {
  for (int64_t s = 0; s < L->n; ++s) {
    double rr = 0.0, rb = 0.0;
    for (int i = 0; i < Q; ++i) { rr += F(L, 0, i, s); rb += F(L, 1, i, s); }
    if (rho_r) rho_r[s] = rr;
    if (rho_b) rho_b[s] = rb;
  }
}

void orc_profile(const orc_lattice* L, double* phi) {
  const orc_params* p = &L->p;
  for (int z = 0; z < p->nz; ++z) {
    double acc = 0.0;
    int64_t cnt = 0;
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        int64_t s = x + (int64_t)p->nx * (y + (int64_t)p->ny * z);
        if (L->cls[s] == 2) continue;
        double rr = 0.0, rb = 0.0;
        for (int i = 0; i < Q; ++i) { rr += F(L, 0, i, s); rb += F(L, 1, i, s); }
        acc += rr - rb;
        ++cnt;
      }
    phi[z] = cnt ? acc / (double)cnt : NAN;
  }
}

void orc_diag_get(const orc_lattice* L, orc_diag* d) {
  const orc_params* p = &L->p;
  memset(d, 0, sizeof(*d));
  d->step = L->step;
  d->evaporated_mass = L->evaporated;
  d->flux_last = L->flux_last;
  int64_t cnt = 0;
  for (int64_t s = 0; s < L->n; ++s) {
    if (L->cls[s] == 2) continue;
    double rr = 0.0, rb = 0.0;
    for (int i = 0; i < Q; ++i) { rr += F(L, 0, i, s); rb += F(L, 1, i, s); }
    d->mass_r += rr;
    d->mass_b += rb;
    if (rr > rb) ++cnt;
  }
  d->droplet_sites = cnt;
  d->radius = cbrt(3.0 * (double)cnt / (4.0 * M_PI));
  /* Interface (Sec. III B: x_I where rho^c - rho^cbar = 0): first downward zero
     crossing of phi above the liquid base, linearly interpolated. */
  double* phi = (double*)malloc(sizeof(double) * (size_t)p->nz);
  orc_profile(L, phi);
  int z0 = p->wall_thickness > 0 ? p->wall_z0 + p->wall_thickness : 0;
  d->interface_z = -1.0;
  for (int z = z0; z + 1 < p->nz; ++z) {
    if (isnan(phi[z]) || isnan(phi[z + 1])) continue;
    if (phi[z] > 0.0 && phi[z + 1] <= 0.0) {
      d->interface_z = z + phi[z] / (phi[z] - phi[z + 1]);
      break;
    }
  }
  free(phi);
}

/* Eq. (flux) with Eq. (velw): j^r = rho^r (U^r - U); the paper writes them for
   tau = 1, which is the only case this helper supports. */
void orc_flux_field(const orc_lattice* L, double* j) {
  const orc_params* p = &L->p;
  const int64_t n = L->n;
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  orc_lattice* M = (orc_lattice*)L;
  densities(M);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t s = x + (int64_t)nx * (y + (int64_t)ny * z);
        if (L->cls[s] != 0) { j[s] = j[n + s] = j[2 * n + s] = 0.0; continue; }
        double Fc[2][3], m[2][3] = {{0, 0, 0}, {0, 0, 0}};
        force(L, x, y, z, Fc);
        for (int c = 0; c < 2; ++c) {
          for (int i = 0; i < Q; ++i) {
            double fi = F(L, c, i, s);
            m[c][0] += fi * CX[i]; m[c][1] += fi * CY[i]; m[c][2] += fi * CZ[i];
          }
        }
        double rr = L->rho[s], rb = L->rho[n + s], rt = rr + rb;
        for (int d = 0; d < 3; ++d) {
          double U = (m[0][d] + m[1][d] + 0.5 * (Fc[0][d] + Fc[1][d])) / rt;
          double Ur = (m[0][d] + Fc[0][d] + rr * (m[0][d] + m[1][d]) / rt) / (2.0 * rr);
          j[(int64_t)d * n + s] = rr * (Ur - U);
        }
      }
}

void orc_site_class(const orc_lattice* L, int8_t* cls) { memcpy(cls, L->cls, (size_t)L->n); }
