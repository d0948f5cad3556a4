/*
 * sc_lbm — GB300 (sm_103a) library for the two-component pseudopotential
 * (Shan-Chen) lattice Boltzmann time step with the fixed-density evaporation
 * boundary of Hessling, Xie & Harting, "Diffusion dominated evaporation in
 * multicomponent lattice Boltzmann simulations" (arXiv:1701.03637).
 *
 * The method (Sec. II):
 *   - D3Q19 BGK evolution per component, Eq. (1), toward the second-order
 *     equilibrium of Eq. (2) with c_s^2 = 1/3, weights 1/3, 1/18, 1/36;
 *   - densities rho^c = sum_i f_i^c, pseudopotential Psi = 1 - exp(-rho), Eq. (4);
 *   - inter-component force F^c = -Psi^c(x) g sum_i w_i Psi^cbar(x + e_i) e_i, Eq. (3),
 *     applied as the velocity shift tau F^c / rho^c on the common velocity (with
 *     optional self couplings g^{cc}: the same sum over cbar = c);
 *   - periodic boundaries, halfway bounce-back at solid sites (Sec. II A);
 *   - evaporation sink (Sec. II C): at sink sites the evaporating component r is
 *     reset to f_i = w_i rho_H and the other component b to
 *     f_i = w_i (rho^r + rho^b - rho_H), from the populations that arrived,
 *     so the total mass is conserved and the evaporated mass is
 *     sum (rho^r_arrived - rho_H).
 *
 * Component 0 ("r") is the paper's evaporating component c, component 1 ("b")
 * is c-bar, and G is g^{c cbar} = g^{cbar c}.
 *
 * Conventions for every call:
 *   - Return value 0 (SC_OK) on success, a negative SC_E* code otherwise; the
 *     message of the last failure on the calling thread is in sc_last_error().
 *   - Lattice site index s = x + nx*(y + ny*z) (x fastest).
 *   - Population arrays crossing the boundary are canonical: post-streaming,
 *     post-sink-reset populations f[c][i][s] (c in {0,1}, i in 0..18 in the
 *     direction order given by sc_lattice_directions).
 *   - Pointers named *_host are host memory owned by the caller; pointers
 *     named *_dev are device memory owned by the caller. Calls that touch host
 *     memory are synchronous with respect to the handle's stream; all other
 *     calls are asynchronous on that stream.
 *   - The library never calls exit() or abort(); invalid arguments return
 *     SC_EINVAL before any device work is queued.
 */
#ifndef SC_LBM_H
#define SC_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SC_OK 0
#define SC_EINVAL (-1)      /* invalid argument or parameter combination */
#define SC_ENOMEM (-2)      /* device or host allocation failed, or caller buffer too small */
#define SC_ECUDA (-3)       /* a CUDA runtime call failed (message has the CUDA error string) */
#define SC_ENONFINITE (-4)  /* diagnostics found a NaN/Inf density */
#define SC_ETIMEOUT (-5)    /* a bounded device-side wait gave up */
#define SC_ESINKNEG (-6)    /* a sink site had rho^r + rho^b < rho_H (negative complement) */

#define SC_GEOM_PERIODIC 0      /* no sink */
#define SC_GEOM_PLANAR_SINK 1   /* sink planes z in [sink_z0, sink_z0 + sink_layers) mod nz */
#define SC_GEOM_SPHERE_SINK 2   /* sink where |x - centre| >= R_H */

#define SC_STORAGE_F32 0        /* FP32 populations */
#define SC_STORAGE_F16 1        /* FP16 offsets f_i - w_i*rho0 (rho0 = 1), FP32 arithmetic */
#define SC_STORAGE_BF16 2       /* BF16 offsets f_i - w_i*rho0, FP32 arithmetic */
#define SC_STORAGE_F16_SCALED 3 /* FP16 of f_i / w_i (about rho: the same relative spacing in liquid
                                   and vapour; not in the paper), FP32 arithmetic */

#define SC_STAGING_AUTO 0       /* staged rows where nx allows, else per-thread pulls */
#define SC_STAGING_THREAD 1     /* each thread copies its site's 38 pulls (any nx) */
#define SC_STAGING_ROWS 2       /* the CTA copies the tile's source rows as 16-byte chunks
                                   (nx a multiple of 4 for FP32, of 8 for FP16/BF16) */
#define SC_STAGING_PERSISTENT 3 /* in place only (SC_LAYOUT_AA): one cooperative launch advances
                                   many steps, each CTA keeping one tile column and ordering its
                                   in-place writes against its neighbours' reads with bounded
                                   progress waits (see SC_LAYOUT_AA). SC_STAGING_AUTO picks it
                                   for in-place lattices when the device can keep one CTA per
                                   tile column resident; SC_STAGING_THREAD keeps the two-pass
                                   step. */

/* Population storage between steps (streaming, Sec. II A: each population moves to
   the neighbour x + e_i, or back to x in the opposite direction where x + e_i is
   solid). */
#define SC_LAYOUT_TWO_LATTICE 0 /* two population lattices: each step pulls from one and
                                   writes the other (one fused launch per step) */
#define SC_LAYOUT_AA 1          /* one lattice updated in place (the AA pattern): half the
                                   population memory. Steps alternate two forms: in the
                                   even form population i arriving at x is kept where the
                                   two-lattice pull reads it (at x - e_i, or at (opp(i), x)
                                   next to a wall), in the odd form at (opp(i), x); a step
                                   writes each post-collision population f*_j into the slot
                                   that population opp(j) was read from. Since the force of
                                   Eq. (3) needs Psi of the neighbours before any of them is
                                   overwritten, the step is either one persistent cooperative
                                   launch for many steps (SC_STAGING_PERSISTENT: each CTA owns a
                                   tile column, forms Psi of the next plane of its tile and halo,
                                   and waits, with a time limit, until its 8 neighbours have done
                                   the same before it overwrites a plane; 304 bytes of DRAM per
                                   FP32 site update) or two launches per step (SC_STAGING_THREAD:
                                   Psi of every site into an FP32 (Psi^r, Psi^b) array, 8 bytes
                                   per site, then stream + sink + force + collision in place;
                                   472 bytes). Results are bit-identical to
                                   SC_LAYOUT_TWO_LATTICE. Not for batch members. */

/* Physical and geometric parameters of one lattice (Sec. II; geometry of Sec. III). */
typedef struct sc_params {
  int32_t nx, ny, nz;             /* lattice extent, each >= 1 */
  double tau_r, tau_b;            /* BGK relaxation times (> 0.5); the paper uses 1 */
  double G;                       /* cross coupling g^{rb} = g^{br} of Eq. (3) */
  double rho_H;                   /* imposed density of component r at sink sites */
  int32_t geometry;               /* SC_GEOM_* */
  int32_t sink_z0, sink_layers;   /* planar sink: first plane and number of planes (1 or 2) */
  double sphere_cx, sphere_cy, sphere_cz, R_H;  /* spherical sink: centre and radius */
  int32_t wall_z0, wall_thickness;/* solid slab z in [wall_z0, wall_z0 + wall_thickness); 0 = none */
  int32_t storage;                /* SC_STORAGE_* */
  int32_t tile;                   /* kernel tile choice: 0 = automatic, k > 0 = entry k-1 of sc_tile_list */
  int32_t zchunk;                 /* planes per CTA along z: 0 = automatic */
  int32_t staging;                /* SC_STAGING_*: how the step kernel gathers its pulls */
  int32_t layout;                 /* SC_LAYOUT_*: two lattices or one updated in place */
  double G_rr, G_bb;              /* self couplings g^{rr}, g^{bb}: Eq. (3) sums the force over every
                                     component cbar, cbar = c included; the paper's runs have
                                     only g^{rb} = g^{br} = G (self couplings 0). g^{cc} < -4
                                     separates component c into liquid and vapour on its own
                                     (the multiphase pseudopotential model the paper names as an
                                     extension; with rho^b = 0 everywhere, the single-component
                                     model). Finite. */
} sc_params;

/* Seeded initial state: film or droplet with uniform noise. */
typedef struct sc_init {
  int32_t shape;                  /* 0 = film (r-rich for z < film_z), 1 = droplet (r-rich inside radius) */
  int32_t film_z;
  double cx, cy, cz, radius;      /* droplet centre and radius */
  double rho_hi, rho_lo;          /* majority / minority densities of the initial phases */
  double noise_amp;               /* each component's density gets U(-a, a) per site */
  uint64_t seed;                  /* SplitMix64 seed: the noise of (component c, site s) is
                                     a*(2u - 1), u = (out >> 11) * 2^-53, out = the
                                     (1 + c*N + s)-th output of SplitMix64(seed) */
} sc_init;

/* Diagnostics of the canonical state (Sec. III B/C observables). */
typedef struct sc_diag {
  int64_t step;                   /* completed time steps */
  double mass_r, mass_b;          /* FP64 sums of rho over non-solid sites */
  double evaporated_mass;         /* cumulative sum over steps and sink sites of (rho^r_arrived - rho_H) */
  double flux_last;               /* the same sum for the last step only */
  double interface_z;             /* first downward zero of phi(z) = <rho^r - rho^b>_xy above the
                                     liquid base, linearly interpolated; -1 if none */
  double radius;                  /* (3 V / 4 pi)^(1/3), V = number of sites with rho^r > rho^b */
  int64_t droplet_sites;          /* V */
  int32_t status;                 /* SC_OK, SC_ENONFINITE, SC_ESINKNEG, or SC_ETIMEOUT after a
                                     persistent in-place launch gave up a wait */
  int32_t reserved;
} sc_diag;

typedef struct sc_lbm sc_lbm;

/* D3Q19 direction order used by every population array (c: [19][3]) and the weights. */
int sc_lattice_directions(int32_t* c_host, double* w_host);

/* Device bytes one lattice with these parameters needs (the population lattices of
   its layout, the Psi array of the in-place layout, diagnostics scratch). */
int sc_lbm_required_bytes(const sc_params* p, size_t* bytes);

/* Create a lattice whose device memory the library allocates (cudaMalloc) and frees
   in sc_lbm_destroy. `stream` is a cudaStream_t (NULL = legacy default stream). */
int sc_lbm_create(const sc_params* p, void* stream, sc_lbm** out);

/* Same, on caller-owned device memory of at least sc_lbm_required_bytes() bytes,
   256-byte aligned; the buffer must outlive the handle and is not freed by it. */
int sc_lbm_create_ext(const sc_params* p, void* stream, void* buf_dev, size_t bytes, sc_lbm** out);

void sc_lbm_destroy(sc_lbm* h);
int sc_lbm_set_stream(sc_lbm* h, void* stream);
int sc_lbm_sync(sc_lbm* h);

/* Seeded film/droplet initial state computed on the device: rest populations
   w_i rho from the shape plus noise, then the sink reset. Resets the step count
   and the evaporated mass. */
int sc_lbm_init(sc_lbm* h, const sc_init* in);

/* Rest populations w_i rho from caller density fields (nx*ny*nz floats each),
   then the sink reset. Synchronous. */
int sc_lbm_init_fields(sc_lbm* h, const float* rho_r_host, const float* rho_b_host);

/* Advance nsteps time steps (asynchronous). Each step is one fused launch
   (stream + sink reset + densities + Psi + force + collision) with two lattices,
   two launches in place (Psi, then the rest; SC_LAYOUT_AA). */
int sc_lbm_step(sc_lbm* h, int64_t nsteps);

/* Canonical densities into caller buffers (nx*ny*nz floats each). */
int sc_lbm_read_fields(sc_lbm* h, float* rho_r_host, float* rho_b_host);
int sc_lbm_read_fields_device(sc_lbm* h, float* rho_r_dev, float* rho_b_dev);

/* Canonical populations (2*19*nx*ny*nz doubles, converted from the storage type). */
int sc_lbm_read_populations(sc_lbm* h, double* f_host);
/* Replace the state by canonical populations (checkpoint restore); sink sites are
   reset without counting evaporated mass, solid sites are ignored. Keeps the step
   count and evaporated mass. */
int sc_lbm_write_populations(sc_lbm* h, const double* f_host);
/* Restore the step count and evaporated mass saved from sc_diag (checkpoint). */
int sc_lbm_set_counters(sc_lbm* h, int64_t step, double evaporated_mass);

/* FP64 diagnostics of the canonical state (synchronous). */
int sc_lbm_diagnostics(sc_lbm* h, sc_diag* out);
/* phi(z) = mean over non-solid (x, y) of rho^r - rho^b, nz doubles (NaN for solid planes). */
int sc_lbm_profile(sc_lbm* h, double* phi_host);

/* Relative flux of component r of Sec. III A, j^r = rho^r (U^r - U) with the velocities
   of Eq. (velw): U = (m^r + m^b + (F^r + F^b) / 2) / rho and U^r = (m^r + F^r +
   rho^r u') / (2 rho^r), rho = rho^r + rho^b, u' = (m^r + m^b) / rho, F^c the force of
   Eq. (3); the paper states these for tau = 1, so the call requires tau_r = tau_b = 1
   (SC_EINVAL otherwise). Evaluated on the device in FP64 from the canonical populations
   (0 at sink and solid sites) and averaged over each plane's nx * ny sites:
   j_host[d * nz + z] (d = 0, 1, 2 for x, y, z; 3 * nz caller-owned doubles).
   Synchronous. */
int sc_lbm_flux_profile(sc_lbm* h, double* j_host);

/* Diagnostics for callers that cannot allocate device memory (for instance code
   running under an allocator they do not control, or inside a process whose
   memory budget is fixed up front). The paper has no counterpart: this is the
   same FP64 reduction as sc_lbm_diagnostics, but its per-plane partial sums go to
   a file-scope device array of 262144 doubles (2 MiB, held by every device that
   loads this library until the process exits) and are folded on the device, so
   the call allocates nothing (no cudaMalloc, no pinned host memory) and does not
   synchronize. It writes 8 doubles to out_dev (caller-owned device memory), in
   order: mass_r, mass_b, evaporated_mass, flux_last, interface_z, radius,
   droplet_sites, status; they are ready when the handle's stream reaches this
   point. Returns SC_EINVAL when nz * (plane splits) * 8 exceeds the array's 262144
   doubles; a lattice is split into max(1, min(ceil(608 / nz), ceil(nx * ny / 1024)))
   parts per plane, one for every nz >= 608, so this happens exactly when nz > 32768.
   The first call on a device (and the first after the device's context has been
   destroyed and recreated, e.g. by cudaDeviceReset) looks up the array's device
   address, so it should come before any stream capture on that device. All calls
   on a device share the array: calls whose work overlaps on the GPU race. Slabs
   (sc_slab_create) are rejected with SC_EINVAL. */
int sc_lbm_diagnostics_noalloc(sc_lbm* h, double* out_dev);

/* Kernel configuration in use: tile extents, planes per CTA, grid size and the
   staging (SC_STAGING_THREAD or SC_STAGING_ROWS). With SC_LAYOUT_AA: a row segment
   of tile_x sites per CTA, tile_y = zchunk = 1, SC_STAGING_THREAD. Any output
   pointer may be NULL. */
int sc_lbm_launch_info(sc_lbm* h, int32_t* tile_x, int32_t* tile_y, int32_t* zchunk, int64_t* ctas,
                       int32_t* staging);
/* Autotuner of the step kernel: times `trials` launches of every tile shape x
   z-chunk length (automatic, 16, 32, 64 planes) and keeps the fastest for the
   following steps; reports the tile (entry + 1 of sc_tile_list) and planes per
   CTA. Trial launches read the current state and write only the buffer the next
   step overwrites, booking their evaporated mass in scratch, so the state and
   the bookkeeping are unchanged. Synchronous. No counterpart in the paper. With
   SC_LAYOUT_AA there is no spare buffer and one configuration: it times nothing
   and reports tile 0 and the current planes per CTA. */
int sc_lbm_tune(sc_lbm* h, int32_t trials, int32_t* tile, int32_t* zchunk);
/* Kernel launches that sc_lbm_step(h, nsteps) issues with the current configuration
   (graph replays count each kernel they contain). */
int sc_lbm_launch_count(sc_lbm* h, int64_t nsteps, int64_t* launches);
/* Name of the kernel (or kernels) that carries the step in the current configuration,
   a static string ("" for a NULL handle). */
const char* sc_lbm_kernel_name(sc_lbm* h);
/* Time limit of each progress wait of the persistent in-place step (default 2 s), and a
   test hook: CTA withhold_cta (-1: none) never reports its progress, so its neighbours'
   waits run out after limit_ns. A wait that runs out ends the launch early; the state
   is then undefined, sc_lbm_sync returns SC_ETIMEOUT and diagnostics report status
   SC_ETIMEOUT until a state is loaded (sc_lbm_init, _init_fields, _write_populations).
   Nothing waits without a limit, so the device stays usable. No counterpart in the
   paper. */
int sc_lbm_set_wait(sc_lbm* h, int64_t limit_ns, int32_t withhold_cta);
/* Bands of the persistent in-place step. That step marches the lattice in `bands`
   bands of equal width along x, one after another within every step; each band is
   the paper's time step (Sec. II) restricted to its sites, its halo at a band edge
   being Psi saved by the band before it or the arrived populations of the band after
   it, so the result is the same for any band count, bit for bit. More bands keep a
   plane of a band in the L2 between its two reads, and make the step possible on
   planes whose tiles would not fit its shared-memory ring with one band. request: -1
   reports the current count only; 0 restores the automatic count (the fewest powers
   of two, dividing nx, for which a tile grid fits); k >= 1 uses k bands (k must
   divide nx into bands of at least 2 sites) and re-plans the tile grid for the
   following steps. *bands (may be NULL) receives the count in use, 0 for a lattice
   without the persistent step. SC_EINVAL for a request on such a lattice, for a k that
   does not divide nx, or when no tile grid fits k bands (the previous plan is kept).
   Tuning and test hook; no counterpart in the paper. */
int sc_lbm_persist_bands(sc_lbm* h, int32_t request, int32_t* bands);
/* Bytes one sc_lbm_diagnostics / sc_lbm_profile call copies device-to-host. */
int sc_lbm_diag_bytes(sc_lbm* h, size_t* bytes);
/* Number of compiled tile shapes and their extents. */
int sc_tile_list(int32_t* count, int32_t* tx_host, int32_t* ty_host, int32_t capacity);

/* ---------------------------------------------------------------- z slabs of one lattice
   One lattice split along z over several handles (one per GPU or rank). The step of
   Sec. II is local except for streaming and the force of Eq. (3), which reach one plane
   across a slab's faces (periodic boundaries with forces computed across them, Sec.
   II A). A slab holds planes [z0, z1) of the lattice described by the global
   parameters, plus 2 ghost planes on each side: before every step each slab sends its
   2 lowest and 2 highest planes (every population, as the current buffer holds them) to
   the ghost planes of its lower and upper neighbour (periodic in z), then steps as an
   ordinary two-lattice handle. Its geometry (sinks, walls, sphere) and its seeded
   initial state are the whole lattice's, so its own planes evolve exactly as the same
   planes of one lattice would, bit for bit. The paper has no counterpart: this
   distributes the one step it describes. Two-lattice layout only. */

/* A slab of planes [z0, z1) (z1 - z0 >= 2) of the lattice described by `global`; its
   handle's nz is z1 - z0 + 4 (local plane 2 is plane z0). Every sc_lbm_* call applies
   to it; populations and fields are its local planes, ghosts included. Its diagnostics
   count its own planes only (mass_r, mass_b, evaporated_mass, flux_last,
   droplet_sites); interface_z and radius need the whole lattice's sums. */
int sc_slab_create(const sc_params* global, int32_t z0, int32_t z1, void* stream, sc_lbm** out);
/* Planes [z0, z1), ghost planes per side, and the bytes of one face's exchange
   (2 * 19 populations of 2 planes). Any output may be NULL. */
int sc_slab_info(sc_lbm* h, int32_t* z0, int32_t* z1, int32_t* ghosts, size_t* face_bytes);
/* Copy the slab's 2 lowest (side 0) or 2 highest (side 1) own planes of the current
   buffer into out_dev (face_bytes of caller-owned device memory: population array k's
   2 planes at offset k * face_bytes / 38), asynchronously on the handle's stream. */
int sc_slab_pack(sc_lbm* h, int32_t side, void* out_dev);
/* Copy a neighbour's packed planes into the ghost planes below (side 0) or above
   (side 1) the slab's own planes: side 0 takes the lower neighbour's side-1 pack,
   side 1 the upper neighbour's side-0 pack. Asynchronous on the handle's stream. */
int sc_slab_unpack(sc_lbm* h, int32_t side, const void* in_dev);

/* ---------------------------------------------------------------- more than two components
   The paper names the extension of its two-component model to more components as
   straightforward (Sec. I); Eq. (3) already sums the force over the other components
   cbar. ncomp components (2 to SC_MAX_COMP) on a periodic lattice with an optional solid
   slab (halfway bounce-back, Psi = 0 at solid sites); the paper states its evaporation
   boundary for two components only, so there is no sink. Each component c has its
   relaxation time tau[c]; g[c][cbar] is the coupling g^{c cbar} of Eq. (3) (the diagonal
   the self couplings). The common velocity is u' = sum_c (m^c / tau_c) /
   sum_c (rho^c / tau_c) and the shift tau_c F^c / rho^c, as for two components. FP32
   populations, two lattices, one launch per step (tile columns of 32 x 8 sites marching
   chunks of planes, Psi of every component in a shared ring, then pull + force +
   collision). With two components and non-zero self couplings the populations are
   bit-identical to sc_lbm_step's. */
#define SC_MAX_COMP 4

typedef struct sc_nparams {
  int32_t nx, ny, nz;             /* lattice extent, each >= 1 */
  int32_t ncomp;                  /* components, 2 .. SC_MAX_COMP */
  double tau[SC_MAX_COMP];        /* relaxation times (> 0.5) of the first ncomp components */
  double g[SC_MAX_COMP][SC_MAX_COMP];  /* couplings g^{c cbar}; finite */
  int32_t wall_z0, wall_thickness;/* solid slab z in [wall_z0, wall_z0 + wall_thickness); 0 = none */
} sc_nparams;

typedef struct sc_ncomp sc_ncomp;

/* Create (cudaMalloc of two population lattices and the Psi array) on `stream`. */
int sc_ncomp_create(const sc_nparams* p, void* stream, sc_ncomp** out);
void sc_ncomp_destroy(sc_ncomp* h);
/* Canonical populations f[c][i][s] (ncomp * 19 * nx*ny*nz doubles, converted to FP32);
   solid sites are ignored. Synchronous. */
int sc_ncomp_write_populations(sc_ncomp* h, const double* f_host);
/* Rest populations w_i rho^c (Eq. 2 at u = 0) from caller density fields rho[c][s]
   (ncomp * nx*ny*nz floats, x fastest); solid sites are ignored. Resets the step
   count. Synchronous. */
int sc_ncomp_init_fields(sc_ncomp* h, const float* rho_host);
/* Canonical populations out (same layout; 0 at solid sites). Synchronous. */
int sc_ncomp_read_populations(sc_ncomp* h, double* f_host);
/* Advance nsteps steps (asynchronous, one launch per step). */
int sc_ncomp_step(sc_ncomp* h, int64_t nsteps);
int sc_ncomp_sync(sc_ncomp* h);

/* Thread-local message describing the last failure (never NULL). */
const char* sc_last_error(void);

/* ---------------------------------------------------------------- batched step
   Many lattices (extents, tau, g, rho_H, geometry may all differ; the storage type
   is the batch's) advanced together: one persistent launch per time step covers
   every member, each member computing exactly what sc_lbm_step computes for it
   (Sec. II), so a member's populations are bit-identical to the same lattice
   stepped alone. The paper has no counterpart: this serves ensembles of runs. */
typedef struct sc_batch sc_batch;

/* A batch whose members live in one device arena of arena_bytes (cudaMalloc'd
   here, freed by sc_batch_destroy). `stream` as for sc_lbm_create. */
int sc_batch_create(size_t arena_bytes, int32_t storage, void* stream, sc_batch** out);
/* Destroys every member and frees the arena. */
void sc_batch_destroy(sc_batch* b);

/* Admit a lattice: carve sc_lbm_required_bytes(p) from the arena (SC_ENOMEM when
   no free range is large enough: admission by free device memory) and create it
   there. *slot names it in this batch; *lattice (may be NULL) is a handle for
   every sc_lbm_* call except sc_lbm_destroy and sc_lbm_set_stream: the batch owns
   it (sc_lbm_destroy on it does nothing). The member starts with unlimited steps
   and must be initialised (sc_lbm_init / _init_fields / _write_populations).
   Members use SC_LAYOUT_TWO_LATTICE (SC_EINVAL otherwise). */
int sc_batch_add(sc_batch* b, const sc_params* p, int32_t* slot, sc_lbm** lattice);
int sc_batch_lattice(sc_batch* b, int32_t slot, sc_lbm** lattice);
/* Remove a member (synchronises the stream) and return its range to the arena. */
int sc_batch_remove(sc_batch* b, int32_t slot);

/* Steps the member still takes in sc_batch_step calls (< 0: unlimited); it stops
   exactly after that many. sc_batch_remaining reads the count left. */
int sc_batch_set_steps(sc_batch* b, int32_t slot, int64_t steps);
int sc_batch_remaining(sc_batch* b, int32_t slot, int64_t* steps);

/* Advance every member by min(nsteps, its remaining steps), asynchronously on the
   batch's stream: a CUDA graph of 32 persistent launches plus the bookkeeping
   kernel per 32 steps; CTAs claim (member, tile column, z chunk) items from a
   per-launch counter. */
int sc_batch_step(sc_batch* b, int64_t nsteps);

/* Kernel configuration: tile (0 = automatic, k > 0 = entry k-1 of sc_tile_list)
   and target planes per item (0 = 32). */
int sc_batch_configure(sc_batch* b, int32_t tile, int32_t zchunk);
/* Autotuner: time `trials` launches (<= 32) of every tile x {16, 32, 64}-plane
   configuration on the current members, keep the fastest and report it. Trial
   launches leave every member's state and bookkeeping unchanged (they write
   only the buffer the next real step overwrites). Synchronous. */
int sc_batch_tune(sc_batch* b, int32_t trials, int32_t* tile, int32_t* zchunk);
/* Members, work items per launch, free arena bytes, largest free range, and the
   configuration in use. Any output pointer may be NULL. */
int sc_batch_info(sc_batch* b, int32_t* members, int64_t* items, size_t* free_bytes, size_t* largest_free,
                  int32_t* tile, int32_t* zchunk);
int sc_batch_sync(sc_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* SC_LBM_H */
