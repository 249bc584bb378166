/*
 * memd_oracle.h -- declarations of the plain FP64 CPU oracle of local Maxwell
 * Equations Molecular Dynamics (MEMD) in an inhomogeneous dielectric
 * (Fahrenberger & Holm, "Computing Coulomb Interaction in Inhomogeneous
 * Dielectric Media via a Local Electrostatics Lattice Algorithm").
 *
 * TEST INFRASTRUCTURE ONLY.  This is the checker that the CUDA library is
 * compared against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no source, header,
 * table or constant with the CUDA library: every constant below is declared
 * here on its own.
 *
 * Conventions (all FP64 unless stated):
 *   mesh N[0] x N[1] x N[2], cubic cells of edge a = L[d] / N[d];
 *   vertex v = (i, j, k), flat index i + N0 * (j + N1 * k), periodic;
 *   link (d, v) joins v -> v + e_d, stored at d * V + v;
 *   plaquette (d, v) has normal e_d and spans e_{d+1}, e_{d+2} from v;
 *   fixed point: S = 2^16 sub-cell steps, charge unit e * 2^-48, flux
 *   ledger Lg in that unit with  sum_d Lg_d(v) - Lg_d(v - e_d) = Q_v.
 */
#ifndef MEMD_ORACLE_H
#define MEMD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_WBITS 16
#define ORC_S (1 << ORC_WBITS)

/* status codes */
#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_COURANT 2
#define ORC_ERR_OOM 3
#define ORC_ERR_CELL_JUMP 5
#define ORC_ERR_RELAX_NOCONV 7
#define ORC_ERR_OVERFLOW 11

/* permittivity profile kinds */
#define ORC_EPS_CONST 0    /* params[0] = eps */
#define ORC_EPS_LINKS 1    /* values[3 * V] = eps per link */
#define ORC_EPS_VERTICES 2 /* values[V] = eps per vertex, link = endpoint mean */
#define ORC_EPS_TANH 3     /* eps = p0 + p1 tanh((|s - p2| - p3) / p4), s along axis */
#define ORC_EPS_SIN 4      /* eps = p0 + p1 sin(2 pi s / L_axis + p2) */
/* Profiles with an explicit interface (Sec. II, Eq. dielectric-interpolation):
 * a link whose two end values differ crosses the interface and takes the
 * harmonic average weighted by the distances of its ends to the interface.
 * A vertex exactly on the interface of PLANES or SPHERE takes the mean of the
 * two media. */
#define ORC_EPS_PLANES 5   /* p1 between the planes s = p2 and s = p3 along
                              axis, p0 elsewhere; 0 <= p2 <= p3 < L_axis */
#define ORC_EPS_SPHERE 6   /* p1 inside the periodic ball of centre (p2, p3, p4)
                              and radius p5, p0 outside; p5 + a < L_d / 2 */
#define ORC_EPS_CUT 7      /* values[V] = eps per vertex, values[V + l] = where a
                              surface cuts link l, as a fraction of a from its
                              lower end (in [0, 1]; anything else: no cut) */
/* ORC_EPS_VERTICES reads params[0] = theta >= 0: a link with
 * |eps2 - eps1| > theta min(eps1, eps2) is an interface link with the
 * interface at its midpoint; theta = 0 marks none. */

/* self-energy corrections */
#define ORC_SELF_NONE 0
#define ORC_SELF_GF 1
#define ORC_SELF_DIRECT 2

typedef struct orc_eps {
  int32_t kind;
  int32_t axis;
  const double *values;
  double params[8];
} orc_eps;

typedef struct orc_sys orc_sys;

/* energy vector layout returned by orc_energy */
enum {
  ORC_E_KIN = 0, ORC_E_ELEC, ORC_E_MAG, ORC_E_SELF, ORC_E_DIP, ORC_E_TOTAL,
  ORC_E_P0, ORC_E_P1, ORC_E_P2, ORC_E_GAUSS_RES, ORC_E_GAUSS_EXACT, ORC_E_COUNT
};

/* array selectors for orc_ptr */
enum {
  ORC_A_IE = 0, ORC_A_D, ORC_A_B, ORC_A_LG, ORC_A_TB, ORC_A_X, ORC_A_V, ORC_A_IMG,
  ORC_A_Q, ORC_A_M, ORC_A_F, ORC_A_FT, ORC_A_G, ORC_A_MINV
};

orc_sys *orc_create(const int32_t N[3], const double L[3], const orc_eps *eps,
                    double c_light, double dt, int32_t self_mode,
                    int32_t dipole_corr, double relax_tol, int32_t relax_maxit,
                    double omega, uint64_t seed, const double *Minv_in,
                    int32_t *status);
void orc_destroy(orc_sys *s);

int64_t orc_nsites(const orc_sys *s);
int64_t orc_nparticles(const orc_sys *s);
int64_t orc_stepcount(const orc_sys *s);
void *orc_ptr(orc_sys *s, int32_t which);
double orc_scalar(const orc_sys *s, int32_t which); /* 0:a 1:c 2:dt 3:Vbox */

int32_t orc_set_particles(orc_sys *s, int64_t n, const double *x,
                          const int32_t *img, const double *v,
                          const int32_t *q, const double *m);
int32_t orc_init_field(orc_sys *s);
int32_t orc_step(orc_sys *s, int64_t nsteps, int32_t thermo, double gamma,
                 double kT);
int32_t orc_move(orc_sys *s, const double *x_new, const int32_t *img_new);
void orc_gather(orc_sys *s);
void orc_energy(orc_sys *s, double *out);
int32_t orc_relax(orc_sys *s, double tol, int32_t maxit, int32_t *iters);
/* replace the permittivity of a live system: map the profile onto the links,
 * recompute eps_eff; D keeps its value (Gauss' law does not involve eps)
 * unless relax != 0, which rebuilds the electrostatic minimum from the ledger
 * as orc_init_field does (B = 0).  Forces are gathered again. */
int32_t orc_set_eps(orc_sys *s, const orc_eps *eps, int32_t relax);

/* Permittivity from the local salt density (Sec. I: the dielectric
 * response of water falls with its salt content; the paper gives no rule,
 * this is the reading used here).  rho(v) = sum over charges of |q| times
 * their cloud-in-cell weight at vertex v (in e); smoothed by the periodic
 * Gaussian of sigma cells, truncated at R = ceil(3 sigma) cells, weights
 * exp(-j^2 / (2 sigma^2)) normalised to sum 1, along x, then y, then z
 * (sigma = 0: no smoothing); then eps(v) = eps0 + slope (rho(v) / mean(rho)
 * - 1), clamped to [eps_lo, eps_hi] (eps0 clamped when there are no
 * charges).  The vertex values are applied as ORC_EPS_VERTICES with theta
 * = 0 (links take the mean of their ends) by orc_set_eps(relax).  rule =
 * {eps0, slope, eps_lo, eps_hi, sigma}; eps_out (V, may be NULL) receives
 * the vertex values.  Returns orc_set_eps's status. */
int32_t orc_eps_from_density(orc_sys *s, const double rule[5], int32_t relax, double *eps_out);
/* the vertex values alone (V), nothing applied */
int32_t orc_salt_vertex_eps(const orc_sys *s, const double rule[5], double *eps_out);
/* the density and smoothing steps alone: rho (V) on input is smoothed in
 * place as above */
void orc_smooth_periodic(const int32_t N[3], double sigma, double *rho);

/* building blocks exposed for the tests */
void orc_cic_charges(const orc_sys *s, int64_t *Q);
int32_t orc_gauss_scan(const int32_t N[3], const int64_t *Q, int64_t *flux);
void orc_divergence(const int32_t N[3], const int64_t *flux, int64_t *div);
void orc_green_table(const int32_t N[3], double *G8);
void orc_self_force(const orc_sys *s, const int32_t f[3], const int32_t cell[3],
                    int32_t q, double *U, double *F3);
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);
void orc_curl_B(orc_sys *s);
void orc_curl_D(orc_sys *s);

#ifdef __cplusplus
}
#endif
#endif
