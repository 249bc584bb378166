/*
 * memd.h -- C ABI of the GB300 (sm_103a) MEMD library: local Maxwell
 * Equations Molecular Dynamics for Coulomb interactions in an inhomogeneous
 * dielectric (Fahrenberger & Holm, "Computing Coulomb Interaction in
 * Inhomogeneous Dielectric Media via a Local Electrostatics Lattice
 * Algorithm").
 *
 * Model.  A periodic mesh of N[0] x N[1] x N[2] cubic cells of edge
 * a = box[d] / N[d] carries the displacement field D on its links, the
 * magnetic field B on its plaquettes and 1/eps on its links (Sec. II,
 * Fig. 2).  Point charges move through it; every step the plaquettes follow
 * dB/dt = -curl(D/eps) (Eq. 21), the links follow dD/dt = c^2 curl B - j
 * (Eq. 20), the current j is the exact charge transfer of each move, kept in
 * an int64 fixed-point ledger so that div D = rho holds exactly, and the
 * charges feel F = qE (Eq. 18 without v x B) with the self-energy (Sec. III)
 * and global-dipole (Sec. V) corrections.  Units: eps0 = 1, so the Coulomb
 * potential of a charge is q / (4 pi eps r).
 *
 * Layout.  Vertex v = (i, j, k) has flat index i + N0 (j + N1 k).  Link
 * (d, v) joins v to v + e_d; plaquette (d, v) has normal e_d and spans
 * e_{d+1}, e_{d+2} from v.  Field arrays crossing this ABI are FP64,
 * component major: element (d, v) at d * V + v, V = N0 N1 N2.  Particle
 * arrays are n x 3, row major.  Fixed point: S = 2^16 sub-cell steps per cell
 * edge; the ledger unit is e 2^-48.
 *
 * Conventions.  Every call returns a memd_status and never throws.  The
 * caller owns every pointer it passes; the library copies inputs before the
 * call returns and writes outputs into caller buffers, which are host memory
 * unless a name says "device".  One context is used by one host thread at a
 * time and issues all its GPU work on one CUDA stream.  memd_last_error()
 * gives a one-line reason for the last failure.
 */
#ifndef MEMD_H
#define MEMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct memd_ctx memd_ctx;

typedef enum memd_status {
  MEMD_OK = 0,
  MEMD_ERR_INVALID = 1,       /* bad argument or state for this call */
  MEMD_ERR_COURANT = 2,       /* c dt sqrt(3) >= a (Eq. 30) */
  MEMD_ERR_OOM = 3,           /* device allocation failed */
  MEMD_ERR_CUDA = 4,          /* a CUDA call failed */
  MEMD_ERR_CELL_JUMP = 5,     /* a charge moved by more than one cell in a step */
  MEMD_ERR_GAUSS = 6,         /* the ledger does not close (non-neutral scan) */
  MEMD_ERR_RELAX_NOCONV = 7,  /* the relaxation did not reach its tolerance */
  MEMD_ERR_DIPOLE_DRIFT = 8,  /* the dipole correction outgrew the field force (Sec. V) */
  MEMD_ERR_TIMEOUT = 9,       /* a bounded wait in a kernel gave up (step void) */
  MEMD_ERR_STATE = 10,        /* call out of order (e.g. step before init) */
  MEMD_ERR_OVERFLOW = 11      /* fixed-point range exceeded */
} memd_status;

enum { MEMD_FP64 = 0, MEMD_FP32 = 1 };                 /* link/plaquette fields */
enum { MEMD_SELF_NONE = 0, MEMD_SELF_GF = 1, MEMD_SELF_DIRECT = 2 };

/* Permittivity profiles (Sec. II, Fig. 2b).  A link takes the mean of its
 * end values; analytic profiles are sampled at the link midpoint.
 *
 * Interface links (Sec. II, Eq. dielectric-interpolation, read as the
 * harmonic average the text names): a link whose ends lie in different media
 * holds them in series, 1/eps_link = (d1/eps1 + d2/eps2) / a, d1 and d2 the
 * distances of its ends to the interface.  A link is an interface link when
 *   PLANES, SPHERE: its ends are on different sides of the interface (a
 *     vertex exactly on the interface takes the mean of the two media);
 *   CUT: the caller gives its cut position;
 *   VERTICES with params[0] = theta > 0: |eps2 - eps1| > theta min(eps1, eps2),
 *     the interface then at its midpoint (theta = 0: no interface links).
 * A slab or ball thinner than a link between two vertices is not seen. */
enum {
  MEMD_EPS_CONST = 0,     /* params[0] = eps */
  MEMD_EPS_LINKS = 1,     /* values[3 V]: eps per link, component major */
  MEMD_EPS_VERTICES = 2,  /* values[V]: eps per vertex; params[0] = theta >= 0 */
  MEMD_EPS_TANH = 3,      /* eps = p0 + p1 tanh((|s - p2| - p3) / p4), s = periodic
                             distance along `axis` */
  MEMD_EPS_SIN = 4,       /* eps = p0 + p1 sin(2 pi s / L_axis + p2) */
  MEMD_EPS_PLANES = 5,    /* p1 between the planes s = p2 and s = p3 normal to `axis`,
                             p0 elsewhere; 0 <= p2 <= p3 < L_axis */
  MEMD_EPS_SPHERE = 6,    /* p1 inside the ball of centre (p2, p3, p4) and radius p5
                             (nearest periodic image), p0 outside; p5 + a < L_d / 2 */
  MEMD_EPS_CUT = 7        /* values[4 V]: eps per vertex (V), then per link
                             (3 V, component major) where a surface cuts it, as a
                             fraction of a from its lower vertex in [0, 1]; any
                             other value (e.g. -1) marks an uncut link */
};

typedef struct memd_eps_profile {
  int32_t kind;
  int32_t axis;
  const double *values; /* caller owned, copied at create; may be NULL */
  double params[8];
} memd_eps_profile;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns a device pointer of at least `bytes` usable on `stream`, or NULL.
 * When alloc is NULL the library uses cudaMalloc / cudaFree. */
typedef void *(*memd_alloc_fn)(void *user, size_t bytes, void *stream);
typedef void (*memd_free_fn)(void *user, void *ptr, size_t bytes, void *stream);

typedef struct memd_options {
  int32_t precision;      /* MEMD_FP64 | MEMD_FP32 for D, B, 1/eps and the gather */
  int32_t self_mode;      /* MEMD_SELF_* (Sec. III) */
  int32_t dipole_corr;    /* 1: metallic k = 0 correction (Sec. V) */
  int32_t relax_max_iter; /* cap on relaxation iterations */
  double relax_tol;       /* stop when max|circulation of E| <= tol max|E| */
  uint64_t seed;          /* Langevin noise key */
  void *cuda_stream;      /* cudaStream_t to issue work on; NULL = own stream */
  int32_t device;         /* CUDA device ordinal; -1 = current */
  int32_t use_graphs;     /* 1: memd_step replays a captured CUDA graph */
  memd_alloc_fn alloc;
  memd_free_fn free;
  void *alloc_user;
  int32_t time_kernels;   /* 1: CUDA events around the field kernels, see
                             memd_get_kernel_stats */
  int32_t field_kernel;   /* MEMD_FIELD_AUTO: the ROWS kernel (its two CTA widths
                             timed) where the mesh fits it, else timed over the
                             kernels below;
                             MEMD_FIELD_LDG: plain-load kernel, halo loops per thread;
                             MEMD_FIELD_TMA: TMA-staged kernel (when x rows are
                             16-byte multiples, else the plain-load kernel);
                             MEMD_FIELD_SITE: plain loads, one thread per site of the
                             tile and its halo;
                             MEMD_FIELD_ROWS: whole rows of 16-byte vectors staged by
                             asynchronous copies on a persistent grid (x extent a
                             multiple of 4 sites for FP32, 2 for FP64; else the site
                             kernel).  All give the same results (TMA to rounding). */
  int32_t step_engine;    /* MEMD_STEP_AUTO: the single launch for small systems (at
                             most 2^17 sites and 16 particles per SM), else the graph;
                             MEMD_STEP_GRAPH: four kernels a step (field update beside
                             the deposition, transfers, gather); MEMD_STEP_SINGLE: the
                             whole step in one cooperative launch with one grid
                             barrier, its charge transfers applied lazily (every call
                             that reads or replaces the state applies them first);
                             when the device has no cooperative launches, the graph.
                             Both give identical results. */
  int32_t apply_mode;     /* how the graph step and batches apply a step's charge
                             transfers to D and the ledger: MEMD_APPLY_AUTO is the
                             sparse form (faster on the systems measured so far);
                             MEMD_APPLY_SPARSE: each charge's
                             quad takes its crossed links' transfers by atomic
                             exchange; MEMD_APPLY_DENSE: one pass over every link's
                             transfer word.  Both add each word once, so they give
                             identical results. */
  int32_t field_shape[4]; /* 0 everywhere: the field kernel's shape is autotuned.  Else
                             the shape is fixed: {ty, zchunk, planes_ahead, rows_nt}:
                             tile height 4, 8 or 16 (16 needs FP32) and z planes per
                             CTA >= 1 of the LDG, SITE and TMA kernels (SITE: planes
                             loaded ahead 1 or 2), threads a CTA 256 or 512 of the ROWS
                             kernel; a value the chosen field_kernel does not use must be
                             0, and field_kernel must not be AUTO.  Out of range:
                             INVALID at create.  A batch whose members all fix the same
                             ROWS width steps its field pass with that width, untuned. */
} memd_options;

enum { MEMD_FIELD_AUTO = 0, MEMD_FIELD_LDG = 1, MEMD_FIELD_TMA = 2, MEMD_FIELD_SITE = 3,
       MEMD_FIELD_ROWS = 4 };
enum { MEMD_STEP_AUTO = 0, MEMD_STEP_GRAPH = 1, MEMD_STEP_SINGLE = 2 };
enum { MEMD_APPLY_AUTO = 0, MEMD_APPLY_SPARSE = 1, MEMD_APPLY_DENSE = 2 };

typedef struct memd_thermostat {
  double gamma; /* friction rate; Langevin force -gamma m v + sqrt(2 gamma m kT / dt) xi */
  double kT;
} memd_thermostat;

typedef struct memd_energy_terms {
  double kinetic;        /* sum m v^2 / 2 */
  double electric;       /* a^3 sum D^2 / (2 eps) */
  double magnetic;       /* (c^2 a^3 / 2) sum B^{n+1/2} B^{n+3/2} */
  double self;           /* sum of the self energies the correction removes */
  double dipole;         /* P eps_eff^-1 P / (2 V) removed by the dipole correction */
  double total;          /* kinetic + electric + magnetic - self - dipole */
  double P[3];           /* dipole moment of the unfolded charges */
  double gauss_residual; /* max_v |a^2 div D - Q_v| in units of e */
  int32_t gauss_exact;   /* 1 when the ledger satisfies div Lg == Q exactly */
  int32_t pad;
  int64_t step;          /* steps taken since memd_init_field */
} memd_energy_terms;

typedef struct memd_kernel_stats {
  double field_ms;        /* summed CUDA-event time of the field (curl) kernels */
  int64_t field_launches; /* launches timed */
  double field_bytes;     /* algorithmic bytes per field launch */
  int64_t launches_per_step;
  int32_t field_tma;      /* field kernel chosen at create: 1 TMA-staged, 0 plain loads */
  int32_t field_ty;       /* its tile height (rows of field_tx sites) */
  int32_t field_zchunk;   /* its z planes per CTA */
  int32_t field_site;     /* k >= 1: the one-thread-per-site plain-load kernel, loads k
                             planes ahead */
  int32_t step_single;    /* 1: steps run as one cooperative launch; field_ms, field_bytes
                             and field_launches then time that whole kernel */
  int32_t field_tx;       /* tile width in sites (32, or 16 in batches of narrow meshes) */
  int32_t field_rows;     /* batches: nt > 0 when the row kernel runs (nt threads a CTA,
                             persistent grid), 0 for site tiles */
  int32_t pad;
  double phase_ms[3];     /* batches with timing on: summed CUDA-event time of the
                             deposition, the transfer application and the gather
                             (field_launches of each); 0 otherwise */
} memd_kernel_stats;

/* Fill *opt with defaults: FP64, GF self term, dipole correction on,
 * relax_tol 1e-12, 200000 iterations, seed 0, own stream, graphs on. */
void memd_default_options(memd_options *opt);

/* One-line text of a status code. */
const char *memd_status_string(memd_status s);

/* Reason for the last failure on ctx (empty string when none; a static
 * message when ctx is NULL). */
const char *memd_last_error(const memd_ctx *ctx);

/* Create a context (Sec. II, Sec. III, Sec. V).  mesh: N[d] >= 2; box: edge
 * lengths, cubic cells required (box[d] / N[d] equal); eps: profile mapped to
 * the links on the device; c_light, dt > 0 with c dt sqrt(3) < a (Eq. 30).
 * Computes 1/eps per link, the lattice Green's table and the effective
 * permittivity tensor.  Allocates all field memory.  On failure *out is NULL.
 * Errors: INVALID, COURANT, OOM, CUDA, RELAX_NOCONV. */
memd_status memd_create(const int32_t mesh[3], const double box[3],
                        const memd_eps_profile *eps, double c_light, double dt,
                        const memd_options *opt, memd_ctx **out);

/* Release every device resource of ctx (NULL is accepted). */
void memd_destroy(memd_ctx *ctx);

/* Initial field solution (Sec. II, Fig. 1, Eqs. 1-3).  n particles: pos (n x 3)
 * any real positions (folded into the box), q integer valences |q| < 2^15,
 * mass (n, positive and finite; NULL = 1), vel (n x 3, NULL = 0).  Deposits
 * the charges, solves Gauss's law exactly in the int64 ledger, sets the k = 0
 * mode of D to -P/V, relaxes to curl E = 0 in FP64, sets B = 0 and computes
 * the forces.  A
 * non-neutral system gets a uniform background, which must be an integer in
 * units of e 2^-48 per vertex.  Errors: INVALID, OOM, GAUSS, RELAX_NOCONV,
 * CUDA. */
memd_status memd_init_field(memd_ctx *ctx, int64_t n, const double *pos,
                            const int32_t *q, const double *mass,
                            const double *vel);

/* Advance nsteps time steps (Eqs. 18, 20, 21): half kick, plaquette update,
 * drift with charge transfer, link update, transfer application, force
 * gather with corrections and optional Langevin force, half kick.  th NULL
 * means constant energy.  Errors: STATE, CELL_JUMP (the offending charge did
 * not move), CUDA. */
memd_status memd_step(memd_ctx *ctx, int64_t nsteps, const memd_thermostat *th);

/* Copy the electrostatic forces of the current state (Eq. 18 with the
 * self-energy and dipole corrections of Secs. III and V; without the
 * Langevin part) into the caller's host array f_out of n x 3 doubles,
 * particle major.  Synchronises.  Errors: INVALID (NULL argument), STATE
 * before memd_init_field, CUDA. */
memd_status memd_forces(memd_ctx *ctx, double *f_out);

/* Device address of the n x 3 FP64 force array (the library's own memory:
 * read it on ctx's stream or after memd_synchronize; do not free it), valid
 * until the next memd_init_field or memd_destroy.  Errors: INVALID, STATE. */
memd_status memd_forces_device(memd_ctx *ctx, const double **f_dev);

/* Energy terms (kinetic, a^3 sum D^2 / 2 eps, the time-centred magnetic term,
 * the self energy and the dipole term of Secs. III and V), the dipole moment
 * P and the Gauss-law check (Sec. II: the largest |div D - rho| in FP64 and
 * the exact int64 identity div Lg == Q) into *out, all FP64 reductions on
 * the device; pending transfers are applied first.  Synchronises.  Errors:
 * INVALID, STATE before memd_init_field, CUDA. */
memd_status memd_energy(memd_ctx *ctx, memd_energy_terms *out);

/* Dipole drift (Sec. V).  The metallic correction removes P eps_eff^-1 / V
 * from the field every charge feels, P the dipole moment of the unfolded
 * charges.  A current driven through the system (an external field pulling
 * charges apart) makes P grow without bound until the correction outweighs
 * the field of the charges themselves and the method breaks down; the
 * remedy is a fresh initial solution (memd_init_field at the present
 * positions, or memd_set_eps with relax_field).  The lattice field's mean
 * tracks -eps_eff^-1 P / V (Sec. V), so the field the charges produce about
 * it is sqrt(sum_d mean over the d-links of (E_d - mean E_d)^2), E = D / eps.
 * This check compares the correction's field |eps_eff^-1 P| / V with that:
 * *ratio (may be NULL) receives their quotient, and a quotient above limit
 * (> 0; 1 is the paper's "outweighs") returns MEMD_ERR_DIPOLE_DRIFT.
 * Pending transfers are applied first.  Synchronises.  Errors: INVALID,
 * STATE before memd_init_field, CUDA, DIPOLE_DRIFT. */
memd_status memd_dipole_check(memd_ctx *ctx, double limit, double *ratio);

/* Failure injection for tests, on the host: no GPU fault, trap or hang.
 * MEMD_INJECT_BARRIER_SKEW adds one arrival to the grid-barrier count of a
 * context that steps as one cooperative launch (MEMD_STEP_SINGLE in effect,
 * decided at its first step), so the next step's barrier cannot complete:
 * its wait runs out after wait_s seconds (0: the default 0.2 s), the step is
 * void (fields and forces of that step are not to be used; reload a saved
 * state) and the next synchronising call reports MEMD_ERR_TIMEOUT and starts
 * the count afresh.  MEMD_INJECT_NONE only sets the wait bound (wait_s, 0:
 * the default).  Errors: INVALID (unknown kind, wait_s outside [0, 10]),
 * STATE (not initialised, or no grid barrier in this context's steps), CUDA. */
enum { MEMD_INJECT_NONE = 0, MEMD_INJECT_BARRIER_SKEW = 1 };
memd_status memd_inject(memd_ctx *ctx, int32_t kind, double wait_s);

/* Copy the folded positions (in [0, L)), velocities and image counters into
 * caller host arrays of n x 3, particle major (any may be NULL).
 * Synchronises.  Errors: INVALID, STATE before memd_init_field, CUDA. */
memd_status memd_get_particles(memd_ctx *ctx, double *pos, double *vel,
                               int32_t *img);

/* One call for a loop driven from the host: an optional state load (as
 * memd_set_particles: positions with image counters, velocities; any input
 * NULL is kept), nsteps steps (as memd_step), then copies of positions,
 * velocities, image counters and electrostatic forces (any output NULL is
 * skipped), with a single synchronisation at the end.  Host buffers in
 * page-locked memory make every copy asynchronous.  Errors as memd_step and
 * memd_set_particles. */
memd_status memd_step_host(memd_ctx *ctx, const double *pos_in, const double *vel_in,
                           const int32_t *img_in, int64_t nsteps, const memd_thermostat *th,
                           double *pos_out, double *vel_out, int32_t *img_out, double *f_out);

/* Library-owned page-locked I/O buffers for memd_step_io, n x 3 each,
 * particle major, valid until the next memd_init_field or memd_destroy (the
 * caller reads and writes them between calls, never frees them).  Errors:
 * INVALID, STATE before memd_init_field, OOM (page-locked allocation). */
typedef struct memd_io {
  double *pos;   /* positions (in and out) */
  double *vel;   /* velocities (in and out) */
  int32_t *img;  /* image counters (in and out) */
  double *f;     /* electrostatic forces (out) */
} memd_io;
memd_status memd_io_buffers(memd_ctx *ctx, memd_io *io);

/* memd_step_host over the buffers of memd_io_buffers, laid out as one block:
 * load != 0 takes positions, image counters and velocities from them (as
 * memd_set_particles), then nsteps steps, then the buffers receive the state
 * and the forces.  One host-to-device copy, one device-to-host copy, one
 * synchronisation; with load and one step the whole round trip is replayed
 * as one CUDA graph.  Errors as memd_step_host. */
memd_status memd_step_io(memd_ctx *ctx, int32_t load, int64_t nsteps,
                         const memd_thermostat *th);

/* Overwrite positions (folded, with img), velocities and image counters of
 * the n particles without depositing any current (state load); host arrays
 * of n x 3, copied.  img NULL keeps the counters, vel NULL keeps the
 * velocities.  The ledger is not rebuilt, so Gauss' law stays exact only if
 * the charges sit where the ledger has them (memd_move transfers charge).
 * Errors: INVALID (NULL pos; a position not finite or beyond 4 box lengths),
 * STATE before memd_init_field, OOM, CUDA. */
memd_status memd_set_particles(memd_ctx *ctx, const double *pos,
                               const double *vel, const int32_t *img);

/* Prescribed move (Eq. 20, current term only): move every particle to pos
 * (with img, NULL = the folding of pos) and apply the charge transfer of the
 * move to D and the ledger; no field propagation, no force update.
 * Errors: CELL_JUMP, STATE. */
memd_status memd_move(memd_ctx *ctx, const double *pos, const int32_t *img);

/* Copy D, B (FP64, 3V each) and the ledger Lg (int64 in units of e 2^-48,
 * 3V) into caller host arrays in the library's layout: component major, x
 * fastest (element (d, i, j, k) at d V + i + Nx (j + Ny k)); D on the links,
 * B on the plaquettes (Sec. II).  Any may be NULL.  Pending transfers are
 * applied first.  Errors: INVALID, OOM (conversion scratch), CUDA. */
memd_status memd_get_fields(memd_ctx *ctx, double *D, double *B, int64_t *Lg);

/* Overwrite D, B and Lg from caller host arrays in the layout of
 * memd_get_fields (any may be NULL; copied); FP32 contexts round D and B.
 * Nothing checks that the new D satisfies Gauss' law: memd_energy reports
 * it.  Errors: INVALID, OOM (conversion scratch), CUDA. */
memd_status memd_set_fields(memd_ctx *ctx, const double *D, const double *B,
                            const int64_t *Lg);

/* Recompute the forces from the current state (gather with corrections,
 * Eq. 18, Secs. III and V); the stored kick force becomes the electrostatic
 * force.  Errors: INVALID, STATE before memd_init_field, CUDA. */
memd_status memd_compute_forces(memd_ctx *ctx);

/* Replace the permittivity of a context (Sec. II; moving or re-shaped
 * dielectric backgrounds).  Valid before or after memd_init_field.  The
 * profile is mapped as at memd_create and the effective tensor recomputed.
 * Gauss' law constrains D alone, so D and B are kept unless relax_field != 0,
 * which rebuilds D from the exact charge ledger and relaxes it to the
 * electrostatic minimum of the new medium (B = 0), as memd_init_field does.
 * Forces are gathered again; the step counter (noise stream) continues.
 * Errors: MEMD_ERR_INVALID for a bad profile (nothing changed); a failure in
 * mapping or in the effective tensor restores the previous permittivity;
 * MEMD_ERR_RELAX_NOCONV from the relaxation leaves the new permittivity with
 * the previous D.  Batches holding the context rebuild their tables. */
memd_status memd_set_eps(memd_ctx *ctx, const memd_eps_profile *eps, int32_t relax_field);

/* Permittivity from the local salt density (Sec. I: the dielectric response
 * of water falls with its salt content, which the paper names as the
 * motivation of spatially varying eps; it gives no rule, so this one is
 * stated here).  The |q| of every charge is deposited on its cell's vertices
 * with the cloud-in-cell weights (the salt density rho(v), in e), smoothed by
 * the periodic Gaussian of sigma cells (weights exp(-j^2 / (2 sigma^2)) for
 * |j| <= ceil(3 sigma), normalised to sum 1) along x, then y, then z (sigma =
 * 0: no smoothing), and mapped to eps(v) = eps0 + slope (rho(v) / mean(rho) -
 * 1) clamped to [eps_lo, eps_hi] (eps0, clamped, when there are no charges).
 * The vertex values then replace the permittivity as memd_set_eps with
 * MEMD_EPS_VERTICES (theta 0: each link the mean of its ends) would, keeping D
 * or relaxing it (relax_field).  eps_out (host, V, may be NULL) receives the
 * vertex values.  Call it every few steps to let the medium follow the salt.
 * Errors: INVALID (a rule value not finite, eps_lo <= 0, eps_hi < eps_lo,
 * sigma outside [0, 64]), STATE before memd_init_field, OOM, CUDA, and those
 * of memd_set_eps. */
typedef struct memd_salt_rule {
  double eps0, slope, eps_lo, eps_hi, sigma;
} memd_salt_rule;
memd_status memd_eps_from_density(memd_ctx *ctx, const memd_salt_rule *rule, int32_t relax_field,
                                  double *eps_out);

/* Checkpoint and resume.  A saved state holds the whole dynamical state: D
 * and B in the field precision, the exact ledger, positions, velocities,
 * image counters, forces, valences, masses, the step counter (which keys the
 * Langevin noise) and the dipole of the last update; pending transfers are
 * applied first.  It is restored into a context created with the same mesh,
 * box and precision and initialised with the same particle count (the
 * permittivity, options and thermostat are the context's own); stepping on
 * from it gives bit for bit what the saved context would have given.
 * memd_state_bytes is the size of a saved state of ctx.  Errors: INVALID
 * (buffer too small, not a saved state, a mesh, precision or particle count
 * mismatch, or a particle array out of range: a position outside [0, L), a
 * valence beyond +-32767, a mass not positive and finite; nothing changed),
 * STATE before memd_init_field. */
int64_t memd_state_bytes(const memd_ctx *ctx);
memd_status memd_save_state(memd_ctx *ctx, void *buf, int64_t bytes);
memd_status memd_load_state(memd_ctx *ctx, const void *buf, int64_t bytes);

/* Create-time results: 1/eps per link (3V, may be NULL), the lattice Green's
 * table G(dx,dy,dz) at index dx + 2 dy + 4 dz (8, may be NULL) and the inverse
 * effective permittivity tensor (9, row major, may be NULL). */
/* Create-time quantities, into caller host arrays (any may be NULL):
 * inv_eps the FP64 1/eps of every link (3V, layout of memd_get_fields;
 * Eq. 24 on interface links), G8 the lattice Green's function at the 8
 * offsets {0,1}^3 (index rx + 2 ry + 4 rz; Eqs. 25-27, k = 0 removed),
 * eps_eff_inv the inverse effective permittivity tensor (9, row major) of
 * the dipole correction (Sec. V).  Synchronises.  Errors: INVALID, CUDA. */
memd_status memd_get_setup(memd_ctx *ctx, double *inv_eps, double *G8,
                           double *eps_eff_inv);

/* Event timing of the field kernels and launch counts into *out (the timing
 * needs time_kernels; the kernel choice and byte counts are always filled).
 * memd_reset_kernel_stats zeroes the accumulated time and launch count.
 * Errors: INVALID. */
memd_status memd_get_kernel_stats(memd_ctx *ctx, memd_kernel_stats *out);
memd_status memd_reset_kernel_stats(memd_ctx *ctx);

/* Block the host until all work issued by ctx has finished. */
memd_status memd_synchronize(memd_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Batched replicas.  A batch steps many independent, initialised contexts
 * (different meshes, charges and eps profiles) together: every time step is
 * one CUDA graph of four kernels over all members (deposition beside the
 * field update, then transfer application, then the gather), each kernel
 * covering every member through a per-replica descriptor table.  A member
 * gives the same result in the batch as stepped alone: the batched field
 * kernels (site tiles, or whole rows of 16-byte vectors on a persistent grid)
 * do the arithmetic of every field kernel, term for term.  Members must share
 * the device, the
 * precision and the CUDA stream; the batch does not own them, and they stay
 * usable one by one (memd_forces, memd_energy, ...) between batch steps.
 * Re-initialising a member is noticed at the next batch step. */
typedef struct memd_batch memd_batch;

/* Group count >= 1 initialised contexts.  The field kernel is chosen here by
 * timing each candidate on the members' own buffers, which leaves their
 * state unchanged: site tiles (width 16 or 32, height 4, 8 or 16 rows, 1 or
 * 2 planes loaded ahead, 4 to 32 planes per CTA) and the row kernel (256 or
 * 512 threads a CTA; it needs every member's x extent to be a multiple of 4
 * sites for FP32 fields, 2 for FP64).  Members created with field_kernel
 * MEMD_FIELD_ROWS and one width in field_shape[3] fix the row kernel and its
 * width instead (no timing).  Errors: INVALID (mixed device, precision or
 * stream, or a member not initialised), OOM, CUDA. */
memd_status memd_batch_create(int32_t count, memd_ctx *const *members, memd_batch **out);

/* As memd_batch_create, with the field kernel family fixed: MEMD_FIELD_AUTO
 * (both, as memd_batch_create), MEMD_FIELD_SITE (site tiles only) or
 * MEMD_FIELD_ROWS (the row kernel; site tiles when a member does not fit it).
 * Any other value: INVALID. */
memd_status memd_batch_create_kernel(int32_t count, memd_ctx *const *members,
                                     int32_t field_kernel, memd_batch **out);

/* Advance every member by nsteps steps (th NULL: constant energy).
 * Asynchronous like memd_step; errors of members are reported by their own
 * synchronising calls and by memd_batch_synchronize. */
memd_status memd_batch_step(memd_batch *b, int64_t nsteps, const memd_thermostat *th);

/* A host loop over a whole batch.  memd_batch_io_buffers gives the batch's
 * library-owned page-locked I/O block: positions, velocities, image counters
 * and electrostatic forces of every member, n_total x 3 each, particle major,
 * member r's particles at rows offsets[r] .. offsets[r + 1] - 1 (count + 1
 * offsets, in member order).  The block and the offsets stay valid until the
 * batch is destroyed or a member's particle count changes (the caller reads
 * and writes the arrays between calls and never frees them).
 * memd_batch_step_io is memd_step_io for all members at once: load != 0 takes
 * positions, image counters and velocities from the block (as
 * memd_set_particles on each member), then nsteps batch steps, then the
 * block receives every member's state and forces: one host-to-device copy,
 * the device-to-host copies and one synchronisation for the whole batch.
 * With load and one step the call is one CUDA graph in which the input copy
 * runs beside the field update and the positions and image counters are
 * copied back beside the transfer application and force gather; the result
 * is the same as with the copies around the step.
 * Errors: INVALID, STATE (a member not initialised), OOM (page-locked or
 * device block), CUDA; a member's own error (as memd_step_io reports it). */
typedef struct memd_batch_io {
  double *pos;
  double *vel;
  int32_t *img;
  double *f;
  const int64_t *offsets;
  int64_t n_total;
} memd_batch_io;
memd_status memd_batch_io_buffers(memd_batch *b, memd_batch_io *io);
memd_status memd_batch_step_io(memd_batch *b, int32_t load, int64_t nsteps,
                               const memd_thermostat *th);

/* How the batch steps.  MEMD_STEP_GRAPH: the graph of four kernels above.
 * MEMD_STEP_SINGLE: the whole step of every member in one cooperative launch
 * of persistent CTAs that claim work items from device queues: field
 * segments (row tiles over ranges of planes), deposition, transfer
 * application and gather chunks; a member's application chunks start as soon
 * as its own field segments and deposition chunks are done and its gather
 * chunks as soon as its application chunks are, so particle work of some
 * members overlaps the field update of others, with no grid-wide barrier.
 * Every member must fit the row tiles (x extent a multiple of 4 sites for
 * FP32, 2 for FP64), else INVALID.  MEMD_STEP_AUTO (the default): the graph,
 * the faster of the two on the batches measured (the single launch holds its
 * CTAs to the row tiles' shared memory and registers, 16 warps an SM, too few
 * to hide the latency of the particle work).  field_ctas: CTAs that start with
 * field segments (-1: half the grid; the others start with deposition);
 * item_planes: planes per field segment (0: about one segment per CTA).
 * Both engines give identical results.  A wait in the single launch is
 * bounded (0.5 s): when one runs out, memd_batch_synchronize reports
 * MEMD_ERR_TIMEOUT and the step is void.  Errors: INVALID, OOM, CUDA. */
memd_status memd_batch_set_engine(memd_batch *b, int32_t engine, int32_t field_ctas,
                                  int32_t item_planes);

/* Wait for the batch's work; returns the first member error, if any. */
memd_status memd_batch_synchronize(memd_batch *b);

/* Event timing of the batched field kernel (when member 0 has time_kernels)
 * and the algorithmic bytes of one launch over all members; reading the
 * timing resets it.  Errors: INVALID. */
memd_status memd_batch_kernel_stats(memd_batch *b, memd_kernel_stats *out);

/* Time the batched field update with CUDA events inside the step graph (on != 0)
 * or not; by default the batch times it when its first member was created with
 * time_kernels.  The step graphs are rebuilt at the next step.  Errors:
 * INVALID. */
memd_status memd_batch_set_timing(memd_batch *b, int32_t on);

/* Release the batch's own tables (members are untouched; destroy the batch
 * before any of its members). */
void memd_batch_destroy(memd_batch *b);

/* ---------------------------------------------------------------------------
 * Request server (continuous batching).  Requests -- a system plus a number
 * of steps -- queue in arrival order; each memd_server_pump call is one
 * scheduling round: finished requests are retired (results copied to host
 * memory, device memory released), queued requests are admitted first come
 * first served while the device-memory budget and the slot count allow,
 * and all resident systems advance together as one batch by one quantum of
 * steps (shortened so that no request overshoots).  A request that arrives
 * while others run joins at the next round and shares their kernel
 * launches.  Every request gets the same result as when run alone (all
 * field kernels and step engines share their arithmetic).  One server is
 * driven by one host thread. */
typedef struct memd_server memd_server;

enum { MEMD_REQ_QUEUED = 0, MEMD_REQ_RUNNING = 1, MEMD_REQ_DONE = 2, MEMD_REQ_FAILED = 3 };

typedef struct memd_server_options {
  int32_t precision;     /* MEMD_FP32 | MEMD_FP64 for every request */
  int32_t max_slots;     /* systems resident at once */
  int64_t budget_bytes;  /* device memory the resident systems may hold */
  int32_t quantum;       /* steps per scheduling round */
  int32_t device;        /* CUDA device, -1 = current */
  void *cuda_stream;     /* stream of all resident systems (NULL: the server's own) */
  memd_alloc_fn alloc;   /* device allocator of the systems (NULL: cudaMalloc) */
  memd_free_fn free;
  void *alloc_user;
  int32_t thermostat;    /* 1: Langevin (gamma, kT) for every request, 0: constant energy */
  int32_t pad;
  double gamma, kT;
  int32_t admission_workers;  /* threads (each with its own stream) that set requests
                                 up beside the stepping; 0: 3 */
  int32_t reserved[3];
} memd_server_options;

typedef struct memd_request {
  int32_t mesh[3];
  double box[3];
  memd_eps_profile eps;  /* values copied at submit */
  double c_light, dt;
  int64_t n;             /* charges; pos (n x 3), q (n) required, mass / vel may be NULL */
  const double *pos;
  const int32_t *q;
  const double *mass;
  const double *vel;
  uint64_t seed;
  int64_t nsteps;
} memd_request;

/* Defaults: FP32, 64 slots, 8 GiB budget, quantum 50, constant energy. */
void memd_server_default_options(memd_server_options *opt);
/* Create a server on opt->device (the device current at this call when -1;
 * its own stream unless opt->cuda_stream is given, and its admission
 * threads); opt NULL takes the defaults; *out is NULL on failure.
 * memd_server_destroy stops the threads, releases every request and all
 * device memory (NULL is accepted).  Errors: INVALID (bad options), CUDA. */
memd_status memd_server_create(const memd_server_options *opt, memd_server **out);
void memd_server_destroy(memd_server *s);

/* Queue a request (all inputs copied); *id identifies it.  Errors: INVALID. */
memd_status memd_server_submit(memd_server *s, const memd_request *req, int64_t *id);

/* One scheduling round (retire, admit, step one quantum); reports the
 * resident, queued and finished request counts (any may be NULL).  Admission
 * hands queued requests (in arrival order, while the memory budget and the
 * slots allow, their footprint reserved from then on) to three worker
 * threads, which create and initialise each system on their own streams
 * beside the stepping; a system joins the batch at the first round after its
 * setup finished.  A request counts as queued until it joins.  Blocks only
 * to collect the previous round's finished steps, or for at most 2 ms when
 * nothing is resident yet but setups are under way.  Errors: INVALID; the
 * status of a failed batch step (memd_server_last_error says why).  A
 * request whose own setup fails is marked failed and does not fail the
 * call. */
memd_status memd_server_pump(memd_server *s, int32_t *n_active, int32_t *n_queued,
                             int32_t *n_done);

/* MEMD_REQ_* state of a request into *state.  Errors: INVALID (unknown id). */
memd_status memd_server_status(memd_server *s, int64_t id, int32_t *state);

/* Results of a finished request (any pointer may be NULL): folded positions,
 * velocities, image counters, electrostatic forces (n x 3) and energy terms.
 * Errors: STATE (not finished, or failed: memd_server_last_error says why). */
memd_status memd_server_result(memd_server *s, int64_t id, double *pos, double *vel,
                               int32_t *img, double *forces, memd_energy_terms *e);

/* Forget a finished (or failed) request and its stored results.  Errors:
 * INVALID (unknown id), STATE (still queued or running). */
memd_status memd_server_release(memd_server *s, int64_t id);

/* Device bytes held by the resident systems (the admission ledger; 0 for a
 * NULL server). */
int64_t memd_server_used_bytes(const memd_server *s);

typedef struct memd_server_stats {
  double setup_s;          /* time creating and initialising admitted systems, summed over
                              the admission workers (setups run concurrently) */
  double budget_use_sum;   /* sum over rounds of resident footprint / budget */
  int64_t rounds;          /* memd_server_pump calls */
  int64_t steps_rounds;    /* rounds that stepped the batch */
  int64_t rebuilds;        /* batches created (one while requests keep it resident) */
  int64_t admitted;
  int64_t link_updates;    /* 3 V per system per step, summed */
  int64_t particle_steps;
  double step_gpu_s;       /* device time of the batch steps (CUDA events on the server's
                              stream) */
  int64_t table_updates;   /* batch tables rebuilt in place for a new membership */
} memd_server_stats;

/* Counters since create into *out (Errors: INVALID); the reason for the
 * last failure on s (empty when none). */
memd_status memd_server_get_stats(const memd_server *s, memd_server_stats *out);
const char *memd_server_last_error(const memd_server *s);

/* ---------------------------------------------------------------------------
 * Field energy without any device allocation.  The paper has no counterpart:
 * this is a service for callers that cannot allocate device memory -- code
 * that runs inside another framework's memory pool, a host that reserved all
 * device memory up front for its own arena, or a real-time loop where an
 * allocation could fail or stall the device.  It computes the same electric
 * and magnetic terms as memd_energy from device arrays the caller owns, and
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * mesh, a, c_light, dt: as at memd_create; precision: MEMD_FP32 or MEMD_FP64,
 * the element type of D, B and inv_eps, which are device arrays of 3 V values
 * in the library's layout (component major, x fastest).  out2: device pointer
 * to 2 doubles, set to a^3 sum D^2 / (2 eps) and (c^2 a^3 / 2) sum B^{n+1/2}
 * B^{n+3/2}.  cuda_stream: cudaStream_t the work is queued on (NULL = legacy
 * default stream); the call returns without synchronising.
 *
 * The per-block partial sums live in one fixed device array of
 * MEMD_STATIC_MAX_BLOCKS x 2 doubles (1 MiB) inside the library, held by
 * every GPU that loads the library until the process exits.  Meshes with
 * more than MEMD_STATIC_MAX_SITES vertices are rejected with
 * MEMD_ERR_INVALID.  The first call on each device (made with that device
 * current) looks up the array's device address; make that first call before
 * any CUDA stream capture.  That address is kept until the process exits, so
 * resetting the device (cudaDeviceReset) after the first call is not
 * supported.  All calls share the array and each overwrites it
 * completely, so nothing has to be cleared, but calls whose kernels overlap
 * on the GPU race: queue them on one stream or order them with events.
 * Errors: INVALID (bad argument, mesh too large, an edge or vertex count
 * that overflows), CUDA (also when an error of the caller's earlier work is
 * pending: the call then queues nothing and leaves that error in place). */
#define MEMD_STATIC_SITES_PER_BLOCK 2048
#define MEMD_STATIC_MAX_BLOCKS 65536
#define MEMD_STATIC_MAX_SITES ((int64_t)MEMD_STATIC_SITES_PER_BLOCK * MEMD_STATIC_MAX_BLOCKS)
memd_status memd_field_energy_static(const int32_t mesh[3], double a, double c_light,
                                     double dt, int32_t precision, const void *D,
                                     const void *B, const void *inv_eps, double *out2,
                                     void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
