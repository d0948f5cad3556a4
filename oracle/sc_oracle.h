/*
 * FP64 reference ("oracle") for the two-component Shan-Chen D3Q19 BGK step with
 * the fixed-density evaporation boundary of Hessling, Xie & Harting,
 * "Diffusion dominated evaporation in multicomponent lattice Boltzmann
 * simulations" (arXiv:1701.03637), Sec. II.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library may include,
 * link or call this code; only the tests, the smoke check and the CPU
 * baseline leg of the benchmark use it. It shares no code, table or header
 * with the CUDA path.
 *
 * Layout of every population array passed in or out: f[c][i][s], c in {0=r
 * (the evaporating component c), 1=b (the other component c-bar)}, i in
 * 0..18, s = x + nx*(y + ny*z). Densities: rho[s].
 */
#ifndef SC_ORACLE_H
#define SC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
  int32_t nx, ny, nz;
  double tau_r, tau_b, G, rho_H;
  int32_t geometry;          /* 0 periodic, 1 planar z sink, 2 spherical-exterior sink */
  int32_t sink_z0, sink_layers;
  double sphere_cx, sphere_cy, sphere_cz, R_H;
  int32_t wall_z0, wall_thickness;   /* solid slab z in [wall_z0, wall_z0+thickness) */
  double G_rr, G_bb;         /* self couplings g^{rr}, g^{bb} of Eq. (3) (0 in all of the paper's runs) */
} orc_params;

typedef struct orc_init {
  int32_t shape;             /* 0 film (r-rich for z < film_z), 1 droplet (r-rich inside the sphere) */
  int32_t film_z;
  double cx, cy, cz, radius;
  double rho_hi, rho_lo, noise_amp;
  uint64_t seed;
} orc_init;

typedef struct orc_diag {
  int64_t step;
  double mass_r, mass_b, evaporated_mass, flux_last;
  double interface_z, radius;
  int64_t droplet_sites;
} orc_diag;

typedef struct orc_lattice orc_lattice;

int  orc_create(const orc_params* p, orc_lattice** out);
void orc_destroy(orc_lattice* L);
void orc_set_threads(int n);
int  orc_threads(void);

/* Seeded initial state (film or droplet, SplitMix64 noise), then the sink reset. */
int  orc_init_shape(orc_lattice* L, const orc_init* in);
/* Rest populations w_i*rho from density fields, then the sink reset. */
int  orc_init_fields(orc_lattice* L, const double* rho_r, const double* rho_b);
/* Canonical populations in; sink sites are reset (without counting evaporated mass). */
int  orc_set_populations(orc_lattice* L, const double* f);
void orc_get_populations(const orc_lattice* L, double* f);

void orc_step(orc_lattice* L, int64_t nsteps);
void orc_fields(const orc_lattice* L, double* rho_r, double* rho_b);
/* phi(z) = mean over non-solid (x,y) of rho_r - rho_b; NaN for all-solid planes */
void orc_profile(const orc_lattice* L, double* phi);
void orc_diag_get(const orc_lattice* L, orc_diag* d);
/* j^r = rho^r (U^r - U) per site (3 comps, [3][N]), the paper's Eq. (flux)/(velw)
   evaluated on the current canonical state. */
void orc_flux_field(const orc_lattice* L, double* j);
/* site class: 0 fluid, 1 sink, 2 solid */
void orc_site_class(const orc_lattice* L, int8_t* cls);

/* Tables and the equilibrium, exposed so the tests can pin them. */
void orc_lattice_tables(int32_t* c /* [19][3] */, double* w /* [19] */, int32_t* opp /* [19] */);
void orc_feq(double rho, const double* u, double* feq /* [19] */);
/* k-th SplitMix64 output for a seed (k >= 1) and its uniform in [0,1). */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k);
double   orc_uniform(uint64_t seed, uint64_t k);

#ifdef __cplusplus
}
#endif
#endif
