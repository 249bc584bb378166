/*
 * memd_oracle.c -- plain, slow, FP64 CPU oracle of local Maxwell Equations
 * Molecular Dynamics (MEMD) with a per-link permittivity (Fahrenberger &
 * Holm, "Computing Coulomb Interaction in Inhomogeneous Dielectric Media via
 * a Local Electrostatics Lattice Algorithm").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * it is loaded by the tests, by the smoke check and by the benchmark's CPU
 * baseline leg.  It shares no code with the CUDA library.  Every routine is
 * written as the definition or the algorithm step it follows, in the paper's
 * order, single-threaded, with no blocking or fusion.  Build it with
 * -ffp-contract=off so that a*b+c is two roundings, as in the CUDA path.
 *
 * Parity status of each part (what pins it is listed in the tests):
 *   Gauss scan, deposition, ledger      pinned (exact integer identities)
 *   curl updates, energy                pinned (Yee dispersion, conservation)
 *   relaxation                          pinned (FFT / layered exact solves)
 *   lattice Green's table, GF self term pinned (relaxed single-charge energy)
 *   DIRECT self term                    pinned by special cases and symmetry
 *                                       (Eq. 29 is garbled, so the reading
 *                                       itself has no printed values: GF at
 *                                       constant eps, uniform-medium values
 *                                       in layered media, mirror and axis
 *                                       rotation of a random medium)
 *   dipole correction, eps_eff          pinned (layered closed forms)
 *   interface links (planes, ball, cut) pinned (series closed form across
 *                                       off-lattice planes, chord lengths
 *                                       of a ball, image-charge force)
 */
#include "memd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct orc_sys {
  int32_t N[3];
  int64_t V;        /* number of vertices */
  double a, L[3], Vbox, c, dt;
  int32_t self_mode, dipole_corr;
  double relax_tol, omega;
  int32_t relax_maxit;
  double *ie;       /* [3V] 1/eps on links */
  double G[8];      /* lattice Green's function G(dx,dy,dz), index dx+2dy+4dz */
  double Minv[9];   /* inverse effective permittivity tensor, row major */
  double *D, *B;    /* [3V] link and plaquette fields */
  int64_t *Lg, *Tb; /* [3V] exact flux ledger and per-step transfer buffer */
  int64_t bg;       /* uniform neutralising background charge per vertex */
  int64_t n;
  double *x, *v, *m, *F, *Ft;
  int32_t *img, *q;
  int64_t step;
  uint64_t seed;
  int32_t thermo;
  double gamma, kT;
};

/* ---------------------------------------------------------------- indexing */

static int64_t vidx(const orc_sys *s, int64_t i, int64_t j, int64_t k) {
  i %= s->N[0]; if (i < 0) i += s->N[0];
  j %= s->N[1]; if (j < 0) j += s->N[1];
  k %= s->N[2]; if (k < 0) k += s->N[2];
  return i + (int64_t)s->N[0] * (j + (int64_t)s->N[1] * k);
}

/* vertex index of c + delta along the three axes */
static int64_t vshift(const orc_sys *s, const int64_t c[3], int d, int64_t by) {
  int64_t t[3] = {c[0], c[1], c[2]};
  t[d] += by;
  return vidx(s, t[0], t[1], t[2]);
}

static void vcoords(const orc_sys *s, int64_t v, int64_t c[3]) {
  c[0] = v % s->N[0];
  c[1] = (v / s->N[0]) % s->N[1];
  c[2] = v / ((int64_t)s->N[0] * s->N[1]);
}

static int64_t floordiv64(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
  return q;
}

/* ------------------------------------------------------------ Philox4x32-10
 * Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten
 * rounds of two 32x32->64 multiplications with the Weyl key schedule. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform noise of unit variance from one 32-bit word:
 * u = (r + 1/2) 2^-32 in (0,1),  xi = sqrt(3) (2u - 1). */
static double unit_noise(uint32_t r) {
  double u = ((double)r + 0.5) * ldexp(1.0, -32);
  return sqrt(3.0) * (2.0 * u - 1.0);
}

/* --------------------------------------------------- permittivity on links
 * Sec. II and Fig. 2: eps is a 1-form placed on the lattice links; a link
 * takes the mean of its two end values.  Analytic profiles are sampled at the
 * link midpoint. */
static double eps_profile_at(const orc_sys *s, const orc_eps *e, double pos) {
  const double *p = e->params;
  if (e->kind == ORC_EPS_TANH) {
    double Lax = s->L[e->axis];
    double dz = pos - p[2];
    dz = dz - Lax * round(dz / Lax);
    return p[0] + p[1] * tanh((fabs(dz) - p[3]) / p[4]);
  }
  /* ORC_EPS_SIN */
  return p[0] + p[1] * sin(2.0 * M_PI * pos / s->L[e->axis] + p[2]);
}

/* Eq. (dielectric-interpolation).  The text calls the interface-link value a
 * harmonic average; the printed expression eps1 d2/a + eps2 d1/a is its
 * denominator, the numerator eps1 eps2 being lost:
 *   eps_link = eps1 eps2 / (eps1 d2 / a + eps2 d1 / a),
 * where d1 (d2) is the distance from the first (second) end of the link to
 * the interface, d1 + d2 = a.  Equivalently 1/eps_link is the mean of 1/eps
 * along the link, i.e. the two media in series. */
static double interface_link_eps(double eps1, double eps2, double d1, double a) {
  double d2 = a - d1;
  return eps1 * eps2 / (eps1 * d2 / a + eps2 * d1 / a);
}

/* periodic representative of x (in cells) on a ring of n cells, in
 * [-n/2, n/2] */
static double min_image(double x, int32_t n) {
  return x - (double)n * round(x / (double)n);
}

static double clamp01(double t) { return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t); }

/* Two-medium profiles place each vertex inside (+1), outside (-1) or exactly
 * on the interface (0); a vertex on the interface takes the mean of the two
 * media, so that a link lying in the interface gets their average.
 *
 * Planar slab: eps_in (p1) between the planes s = p2 and s = p3 normal to
 * the axis, eps_out (p0) elsewhere, 0 <= p2 <= p3 < L; positions in cells. */
static int planes_side(const orc_sys *s, const orc_eps *e, int64_t k) {
  if (e->params[2] == e->params[3]) return -1;
  double u_lo = e->params[2] / s->a, u_hi = e->params[3] / s->a, u = (double)k;
  if (u == u_lo || u == u_hi) return 0;
  return (u > u_lo && u < u_hi) ? 1 : -1;
}

/* ball: eps_in (p1) closer than p5 to the centre (p2, p3, p4) in the
 * periodic metric, eps_out (p0) farther; offsets in cells */
static void sphere_offset(const orc_sys *s, const orc_eps *e, const int64_t c[3], double del[3]) {
  for (int d = 0; d < 3; ++d) del[d] = min_image((double)c[d] - e->params[2 + d] / s->a, s->N[d]);
}

static int sphere_side(const orc_sys *s, const orc_eps *e, const int64_t c[3]) {
  double del[3], r = e->params[5] / s->a;
  sphere_offset(s, e, c, del);
  double r2 = del[0] * del[0] + del[1] * del[1] + del[2] * del[2];
  double rr = r * r;
  return r2 < rr ? 1 : (r2 == rr ? 0 : -1);
}

static int vertex_side(const orc_sys *s, const orc_eps *e, const int64_t c[3]) {
  return e->kind == ORC_EPS_PLANES ? planes_side(s, e, c[e->axis]) : sphere_side(s, e, c);
}

static double side_eps(const orc_eps *e, int side) {
  return side > 0 ? e->params[1] : (side < 0 ? e->params[0] : 0.5 * (e->params[0] + e->params[1]));
}

/* value of the profile at vertex c for the kinds defined per vertex */
static double vertex_eps(const orc_sys *s, const orc_eps *e, const int64_t c[3]) {
  switch (e->kind) {
  case ORC_EPS_PLANES:
  case ORC_EPS_SPHERE: return side_eps(e, vertex_side(s, e, c));
  default: return e->values[vidx(s, c[0], c[1], c[2])]; /* VERTICES, CUT */
  }
}

/* where the interface cuts the link from vertex c (end 1) along d to its
 * neighbour c2 (end 2), as a fraction of a from end 1, for a link whose end
 * values differ; negative if the link is not an interface link */
static double interface_cut(const orc_sys *s, const orc_eps *e, const int64_t c[3],
                            const int64_t c2[3], int d, int64_t l, double eps1, double eps2) {
  switch (e->kind) {
  case ORC_EPS_VERTICES: {
    double lo = eps1 < eps2 ? eps1 : eps2;
    /* no position is known: the interface sits at the link midpoint */
    return (e->params[0] > 0.0 && fabs(eps2 - eps1) > e->params[0] * lo) ? 0.5 : -1.0;
  }
  case ORC_EPS_CUT: {
    double t = e->values[s->V + l];
    return (t >= 0.0 && t <= 1.0) ? t : -1.0;
  }
  case ORC_EPS_PLANES:
  case ORC_EPS_SPHERE: {
    int s1 = vertex_side(s, e, c), s2 = vertex_side(s, e, c2);
    if (s1 == 0) return 0.0; /* the interface passes through an end */
    if (s2 == 0) return 1.0;
    if (e->kind == ORC_EPS_PLANES) {
      /* entering the slab crosses the plane p2, leaving it the plane p3 */
      double face = (s1 < 0 ? e->params[2] : e->params[3]) / s->a;
      return clamp01(face - (double)c[d]);
    }
    /* the line c + t e_d meets the sphere where (del_d + t)^2 + rho^2 = r^2:
     * leaving at the larger root, entering at the smaller */
    double del[3], r = e->params[5] / s->a;
    sphere_offset(s, e, c, del);
    int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
    double rho2 = del[d1] * del[d1] + del[d2] * del[d2];
    double h2 = r * r - rho2;
    double h = h2 > 0.0 ? sqrt(h2) : 0.0;
    return clamp01(s1 > 0 ? -del[d] + h : -del[d] - h);
  }
  default: return -1.0;
  }
}

static int eps_profile_valid(const orc_sys *s, const orc_eps *e) {
  const double *p = e->params;
  switch (e->kind) {
  case ORC_EPS_CONST: return 1;
  case ORC_EPS_LINKS: return e->values != NULL;
  case ORC_EPS_VERTICES: return e->values != NULL && p[0] >= 0.0 && isfinite(p[0]);
  case ORC_EPS_CUT: return e->values != NULL;
  case ORC_EPS_TANH:
  case ORC_EPS_SIN: return e->axis >= 0 && e->axis <= 2;
  case ORC_EPS_PLANES:
    return e->axis >= 0 && e->axis <= 2 && p[0] > 0.0 && p[1] > 0.0 && isfinite(p[0]) &&
           isfinite(p[1]) && p[2] >= 0.0 && p[2] <= p[3] && p[3] < s->L[e->axis];
  case ORC_EPS_SPHERE: {
    if (!(p[0] > 0.0 && p[1] > 0.0 && isfinite(p[0]) && isfinite(p[1]) && p[5] > 0.0))
      return 0;
    for (int d = 0; d < 3; ++d)
      if (!isfinite(p[2 + d]) || !(p[5] + s->a < 0.5 * s->L[d])) return 0;
    return 1;
  }
  default: return 0;
  }
}

static int map_eps(orc_sys *s, const orc_eps *e) {
  if (!eps_profile_valid(s, e)) return ORC_ERR_INVALID;
  int64_t V = s->V;
  for (int d = 0; d < 3; ++d) {
    for (int64_t v = 0; v < V; ++v) {
      double eps;
      int64_t c[3];
      vcoords(s, v, c);
      switch (e->kind) {
      case ORC_EPS_CONST: eps = e->params[0]; break;
      case ORC_EPS_LINKS: eps = e->values[d * V + v]; break;
      case ORC_EPS_VERTICES:
      case ORC_EPS_CUT:
      case ORC_EPS_PLANES:
      case ORC_EPS_SPHERE: {
        /* end values; an interface link takes Eq. (dielectric-interpolation),
         * any other link the mean of its ends (Fig. 2b) */
        int64_t c2[3] = {c[0], c[1], c[2]};
        c2[d] = (c[d] + 1) % s->N[d];
        double eps1 = vertex_eps(s, e, c), eps2 = vertex_eps(s, e, c2);
        double t = eps1 != eps2 ? interface_cut(s, e, c, c2, d, d * V + v, eps1, eps2) : -1.0;
        if (t >= 0.0)
          eps = interface_link_eps(eps1, eps2, t * s->a, s->a);
        else
          eps = 0.5 * (eps1 + eps2);
        break;
      }
      case ORC_EPS_TANH:
      case ORC_EPS_SIN: {
        double pos = (double)c[e->axis] * s->a;
        if (d == e->axis) pos += 0.5 * s->a;
        eps = eps_profile_at(s, e, pos);
        break;
      }
      default: return ORC_ERR_INVALID;
      }
      if (!(eps > 0.0) || !isfinite(eps)) return ORC_ERR_INVALID;
      s->ie[d * V + v] = 1.0 / eps;
    }
  }
  return ORC_OK;
}

/* --------------------------------------------- lattice Green's function
 * Sec. III, Eqs. 25-27: G solves -Laplace G = delta on the periodic lattice
 * (unit spacing), with the k = 0 mode removed:
 *   G(r) = (1/V) sum_{k != 0} cos(k.r) / sum_d 4 sin^2(k_d / 2).
 * Only displacements with components in {0, 1} are needed for a linearly
 * interpolated charge. */
void orc_green_table(const int32_t N[3], double *G8) {
  int64_t V = (int64_t)N[0] * N[1] * N[2];
  for (int t = 0; t < 8; ++t) G8[t] = 0.0;
  for (int64_t mz = 0; mz < N[2]; ++mz)
    for (int64_t my = 0; my < N[1]; ++my)
      for (int64_t mx = 0; mx < N[0]; ++mx) {
        if (mx == 0 && my == 0 && mz == 0) continue;
        double kx = 2.0 * M_PI * (double)mx / N[0];
        double ky = 2.0 * M_PI * (double)my / N[1];
        double kz = 2.0 * M_PI * (double)mz / N[2];
        double sx = sin(0.5 * kx), sy = sin(0.5 * ky), sz = sin(0.5 * kz);
        double den = 4.0 * (sx * sx + sy * sy + sz * sz);
        for (int t = 0; t < 8; ++t) {
          double kr = kx * (t & 1) + ky * ((t >> 1) & 1) + kz * ((t >> 2) & 1);
          G8[t] += cos(kr) / den;
        }
      }
  for (int t = 0; t < 8; ++t) G8[t] /= (double)V;
}

/* ------------------------------------------------ particle fixed point
 * Sec. V: the periodic box is stitched locally, so a position leaving [0, L)
 * re-enters shifted by whole box lengths, counted in a per-axis image
 * counter (the unfolded coordinate is x + img L).  A sum that rounds up to L
 * is the start of the next image.  Callers bound |x| by a few L.  The
 * lattice coordinate u = x / a splits into a cell c and a sub-cell step
 * f = floor((u - c) S) in [0, S). */
static void fold(double L, double *x, int32_t *img) {
  double y = *x;
  int32_t k = 0;
  while (y >= L) { y -= L; k += 1; }
  while (y < 0.0) { y += L; k -= 1; }
  if (y >= L) { y = 0.0; k += 1; }
  *x = y;
  *img += k;
}

static void quantize(const orc_sys *s, int d, double x, int32_t *c, int32_t *f) {
  double u = x / s->a;
  double cu = floor(u);
  if (cu >= (double)s->N[d]) { *c = s->N[d] - 1; *f = ORC_S - 1; return; }
  if (cu < 0.0) { *c = 0; *f = 0; return; }
  *c = (int32_t)cu;
  *f = (int32_t)floor((u - cu) * (double)ORC_S);
}

/* linear (cloud-in-cell) weight of the corner at offset a in {0,1} */
static int64_t wgt(int32_t f, int a) { return a ? (int64_t)f : (int64_t)(ORC_S - f); }

/* ------------------------------------------------------ vertex charges
 * Sec. IV: charges are interpolated linearly onto the 8 vertices of their
 * cell, Q_v = q w_x w_y w_z in units of e 2^-48, minus a uniform background
 * when the system is not neutral. */
void orc_cic_charges(const orc_sys *s, int64_t *Q) {
  for (int64_t v = 0; v < s->V; ++v) Q[v] = -s->bg;
  for (int64_t p = 0; p < s->n; ++p) {
    int32_t c[3], f[3];
    for (int d = 0; d < 3; ++d) quantize(s, d, s->x[3 * p + d], &c[d], &f[d]);
    for (int az = 0; az < 2; ++az)
      for (int ay = 0; ay < 2; ++ay)
        for (int ax = 0; ax < 2; ++ax) {
          int64_t w = wgt(f[0], ax) * wgt(f[1], ay) * wgt(f[2], az);
          Q[vidx(s, c[0] + ax, c[1] + ay, c[2] + az)] += (int64_t)s->q[p] * w;
        }
  }
}

/* divergence of a link flux: div(v) = sum_d flux_d(v) - flux_d(v - e_d) */
void orc_divergence(const int32_t N[3], const int64_t *flux, int64_t *div) {
  int64_t V = (int64_t)N[0] * N[1] * N[2];
  for (int64_t k = 0; k < N[2]; ++k)
    for (int64_t j = 0; j < N[1]; ++j)
      for (int64_t i = 0; i < N[0]; ++i) {
        int64_t v = i + N[0] * (j + N[1] * k);
        int64_t im = (i + N[0] - 1) % N[0], jm = (j + N[1] - 1) % N[1],
                km = (k + N[2] - 1) % N[2];
        div[v] = flux[v] - flux[im + N[0] * (j + N[1] * k)] + flux[V + v] -
                 flux[V + i + N[0] * (jm + N[1] * k)] + flux[2 * V + v] -
                 flux[2 * V + i + N[0] * (j + N[1] * km)];
      }
}

/* share t (0 <= t < M) of the integer F split as evenly as possible over M
 * links: floor(F / M) each, plus one unit on the first (F mod M) links. */
static int64_t share(int64_t F, int64_t M, int64_t t) {
  int64_t base = floordiv64(F, M);
  int64_t rem = F - base * M;
  return base + (t < rem ? 1 : 0);
}

/* --------------------------------------------- initial Gauss solution
 * Sec. II, Fig. 1 and Eqs. 1-3: the average charge of each z-plane is carried
 * cumulatively on the z-links and removed from the plane; then the same for
 * the y-lines inside each plane; then the single vertices along x.  Done in
 * flux units (D a^2), where eps drops out, and in exact integers. */
int32_t orc_gauss_scan(const int32_t N[3], const int64_t *Q, int64_t *flux) {
  int64_t Nx = N[0], Ny = N[1], Nz = N[2];
  int64_t V = Nx * Ny * Nz;
  int64_t *r = (int64_t *)malloc(sizeof(int64_t) * V);
  if (!r) return ORC_ERR_OOM;
  memcpy(r, Q, sizeof(int64_t) * V);
  memset(flux, 0, sizeof(int64_t) * 3 * V);
  /* planes along z */
  int64_t Fz = 0;
  for (int64_t k = 0; k < Nz; ++k) {
    int64_t rho = 0;
    for (int64_t t = 0; t < Nx * Ny; ++t) rho += Q[t + Nx * Ny * k];
    int64_t Fprev = Fz;
    Fz += rho;
    for (int64_t t = 0; t < Nx * Ny; ++t) {
      int64_t vk = t + Nx * Ny * k;
      int64_t out = share(Fz, Nx * Ny, t);
      int64_t in = (k == 0) ? 0 : share(Fprev, Nx * Ny, t);
      flux[2 * V + vk] = out;
      r[vk] -= out - in;
    }
  }
  if (Fz != 0) { free(r); return ORC_ERR_INVALID; }
  /* lines along y inside each plane */
  for (int64_t k = 0; k < Nz; ++k) {
    int64_t Fy = 0;
    for (int64_t j = 0; j < Ny; ++j) {
      int64_t lam = 0;
      for (int64_t i = 0; i < Nx; ++i) lam += r[i + Nx * (j + Ny * k)];
      int64_t Fprev = Fy;
      Fy += lam;
      for (int64_t i = 0; i < Nx; ++i) {
        int64_t v = i + Nx * (j + Ny * k);
        int64_t out = share(Fy, Nx, i);
        int64_t in = (j == 0) ? 0 : share(Fprev, Nx, i);
        flux[V + v] = out;
        r[v] -= out - in;
      }
    }
    if (Fy != 0) { free(r); return ORC_ERR_INVALID; }
  }
  /* single vertices along x */
  for (int64_t k = 0; k < Nz; ++k)
    for (int64_t j = 0; j < Ny; ++j) {
      int64_t Fx = 0;
      for (int64_t i = 0; i < Nx; ++i) {
        int64_t v = i + Nx * (j + Ny * k);
        Fx += r[v];
        flux[v] = Fx;
      }
      if (Fx != 0) { free(r); return ORC_ERR_INVALID; }
    }
  free(r);
  return ORC_OK;
}

/* ---------------------------------------------------- plaquette geometry
 * Plaquette (d, v): normal e_d, edges e1 = e_{d+1}, e2 = e_{d+2}.  Its
 * circulation is  X_e1(v) + X_e2(v + e1) - X_e1(v + e2) - X_e2(v)
 * (Fig. 2a, finite-difference curl as in the original algorithm). */
static void plaquette_links(const orc_sys *s, int d, int64_t v, int64_t l[4]) {
  int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
  int64_t c[3];
  vcoords(s, v, c);
  l[0] = e1 * s->V + v;
  l[1] = e2 * s->V + vshift(s, c, e1, 1);
  l[2] = e1 * s->V + vshift(s, c, e2, 1);
  l[3] = e2 * s->V + v;
}

/* circulation of E = D / eps around plaquette (d, v) */
static double circulation(const orc_sys *s, int d, int64_t v) {
  int64_t l[4];
  plaquette_links(s, d, v, l);
  return s->D[l[0]] * s->ie[l[0]] + s->D[l[1]] * s->ie[l[1]] -
         s->D[l[2]] * s->ie[l[2]] - s->D[l[3]] * s->ie[l[3]];
}

/* ------------------------------------------------------ relaxation
 * Sec. II: iterative energy minimisation, equivalent to curl E = 0, applied
 * once to the Gauss solution.  Each plaquette rotation moves flux
 * delta = -omega Gamma / sum(1/eps) around the plaquette; it leaves div D
 * and the mean of every D component unchanged and lowers sum D^2 / 2 eps.
 * Sweeps are lexicographic, one orientation after the other; stop when
 * max |Gamma| <= tol * max |E|. */
static void residual(const orc_sys *s, double *maxG, double *maxE) {
  double g = 0.0, e = 0.0;
  for (int d = 0; d < 3; ++d)
    for (int64_t v = 0; v < s->V; ++v) {
      double c = fabs(circulation(s, d, v));
      if (c > g) g = c;
      double el = fabs(s->D[d * s->V + v] * s->ie[d * s->V + v]);
      if (el > e) e = el;
    }
  *maxG = g;
  *maxE = e;
}

int32_t orc_relax(orc_sys *s, double tol, int32_t maxit, int32_t *iters) {
  double g, e;
  residual(s, &g, &e);
  int32_t it = 0;
  while (!(g <= tol * e) && it < maxit) {
    for (int d = 0; d < 3; ++d)
      for (int64_t v = 0; v < s->V; ++v) {
        int64_t l[4];
        plaquette_links(s, d, v, l);
        double G = s->D[l[0]] * s->ie[l[0]] + s->D[l[1]] * s->ie[l[1]] -
                   s->D[l[2]] * s->ie[l[2]] - s->D[l[3]] * s->ie[l[3]];
        double den = s->ie[l[0]] + s->ie[l[1]] + s->ie[l[2]] + s->ie[l[3]];
        double delta = -s->omega * G / den;
        s->D[l[0]] += delta;
        s->D[l[1]] += delta;
        s->D[l[2]] -= delta;
        s->D[l[3]] -= delta;
      }
    ++it;
    residual(s, &g, &e);
  }
  if (iters) *iters = it;
  return (g <= tol * e) ? ORC_OK : ORC_ERR_RELAX_NOCONV;
}

/* ------------------------------------------- effective permittivity
 * Sec. V: the periodic lattice keeps the k = 0 mode of D equal to -P/V.
 * How that mode couples to a varying eps is not stated; this oracle uses the
 * homogenised tensor of the lattice medium: relax a charge-free field whose
 * mean D is e_d; the mean of E is then column d of eps_eff^-1.  The tensor
 * is symmetrised. */
static int32_t eps_effective(orc_sys *s) {
  double M[9];
  for (int d = 0; d < 3; ++d) {
    memset(s->D, 0, sizeof(double) * 3 * s->V);
    for (int64_t v = 0; v < s->V; ++v) s->D[d * s->V + v] = 1.0;
    int32_t st = orc_relax(s, s->relax_tol, s->relax_maxit, NULL);
    if (st != ORC_OK) return st;
    for (int e = 0; e < 3; ++e) {
      double sum = 0.0;
      for (int64_t v = 0; v < s->V; ++v) sum += s->D[e * s->V + v] * s->ie[e * s->V + v];
      M[3 * e + d] = sum / (double)s->V;
    }
  }
  for (int e = 0; e < 3; ++e)
    for (int d = 0; d < 3; ++d) s->Minv[3 * e + d] = 0.5 * (M[3 * e + d] + M[3 * d + e]);
  memset(s->D, 0, sizeof(double) * 3 * s->V);
  return ORC_OK;
}

/* ---------------------------------------------------------------- create */
orc_sys *orc_create(const int32_t N[3], const double L[3], const orc_eps *eps,
                    double c_light, double dt, int32_t self_mode,
                    int32_t dipole_corr, double relax_tol, int32_t relax_maxit,
                    double omega, uint64_t seed, const double *Minv_in,
                    int32_t *status) {
  *status = ORC_ERR_INVALID;
  for (int d = 0; d < 3; ++d)
    if (N[d] < 2 || !(L[d] > 0.0)) return NULL;
  double a = L[0] / N[0];
  for (int d = 1; d < 3; ++d)
    if (fabs(L[d] / N[d] - a) > 1e-12 * a) return NULL;
  if (!(c_light > 0.0) || !(dt > 0.0)) return NULL;
  /* Eq. 30: c << a / dt; the 3-d leapfrog is stable only for c dt sqrt(3) < a */
  if (!(c_light * dt * sqrt(3.0) < a)) { *status = ORC_ERR_COURANT; return NULL; }
  orc_sys *s = (orc_sys *)calloc(1, sizeof(orc_sys));
  if (!s) { *status = ORC_ERR_OOM; return NULL; }
  for (int d = 0; d < 3; ++d) { s->N[d] = N[d]; s->L[d] = L[d]; }
  s->V = (int64_t)N[0] * N[1] * N[2];
  s->a = a;
  s->Vbox = L[0] * L[1] * L[2];
  s->c = c_light;
  s->dt = dt;
  s->self_mode = self_mode;
  s->dipole_corr = dipole_corr;
  s->relax_tol = relax_tol;
  s->relax_maxit = relax_maxit;
  if (!(omega > 0.0)) {
    int32_t nm = N[0] > N[1] ? N[0] : N[1];
    nm = nm > N[2] ? nm : N[2];
    omega = 2.0 / (1.0 + sin(M_PI / nm));
  }
  s->omega = omega;
  s->seed = seed;
  s->ie = (double *)calloc(3 * s->V, sizeof(double));
  s->D = (double *)calloc(3 * s->V, sizeof(double));
  s->B = (double *)calloc(3 * s->V, sizeof(double));
  s->Lg = (int64_t *)calloc(3 * s->V, sizeof(int64_t));
  s->Tb = (int64_t *)calloc(3 * s->V, sizeof(int64_t));
  if (!s->ie || !s->D || !s->B || !s->Lg || !s->Tb) {
    orc_destroy(s); *status = ORC_ERR_OOM; return NULL;
  }
  int32_t st = map_eps(s, eps);
  if (st != ORC_OK) { orc_destroy(s); *status = st; return NULL; }
  orc_green_table(s->N, s->G);
  if (Minv_in) {
    /* a caller-supplied inverse effective permittivity (e.g. a closed form) */
    memcpy(s->Minv, Minv_in, sizeof(s->Minv));
  } else {
    st = eps_effective(s);
    if (st != ORC_OK) { orc_destroy(s); *status = st; return NULL; }
  }
  *status = ORC_OK;
  return s;
}

static void free_particles(orc_sys *s) {
  free(s->x); free(s->v); free(s->m); free(s->F); free(s->Ft);
  free(s->img); free(s->q);
  s->x = s->v = s->m = s->F = s->Ft = NULL;
  s->img = s->q = NULL;
  s->n = 0;
}

void orc_destroy(orc_sys *s) {
  if (!s) return;
  free(s->ie); free(s->D); free(s->B); free(s->Lg); free(s->Tb);
  free_particles(s);
  free(s);
}

int64_t orc_nsites(const orc_sys *s) { return s->V; }
int64_t orc_nparticles(const orc_sys *s) { return s->n; }
int64_t orc_stepcount(const orc_sys *s) { return s->step; }

double orc_scalar(const orc_sys *s, int32_t which) {
  switch (which) {
  case 0: return s->a;
  case 1: return s->c;
  case 2: return s->dt;
  case 3: return s->Vbox;
  default: return 0.0;
  }
}

void *orc_ptr(orc_sys *s, int32_t which) {
  switch (which) {
  case ORC_A_IE: return s->ie;
  case ORC_A_D: return s->D;
  case ORC_A_B: return s->B;
  case ORC_A_LG: return s->Lg;
  case ORC_A_TB: return s->Tb;
  case ORC_A_X: return s->x;
  case ORC_A_V: return s->v;
  case ORC_A_IMG: return s->img;
  case ORC_A_Q: return s->q;
  case ORC_A_M: return s->m;
  case ORC_A_F: return s->F;
  case ORC_A_FT: return s->Ft;
  case ORC_A_G: return s->G;
  case ORC_A_MINV: return s->Minv;
  default: return NULL;
  }
}

int32_t orc_set_particles(orc_sys *s, int64_t n, const double *x,
                          const int32_t *img, const double *v,
                          const int32_t *q, const double *m) {
  free_particles(s);
  if (n < 0) return ORC_ERR_INVALID;
  s->n = n;
  size_t n3 = (size_t)(3 * (n > 0 ? n : 1));
  s->x = (double *)calloc(n3, sizeof(double));
  s->v = (double *)calloc(n3, sizeof(double));
  s->F = (double *)calloc(n3, sizeof(double));
  s->Ft = (double *)calloc(n3, sizeof(double));
  s->img = (int32_t *)calloc(n3, sizeof(int32_t));
  s->m = (double *)calloc(n3 / 3, sizeof(double));
  s->q = (int32_t *)calloc(n3 / 3, sizeof(int32_t));
  if (!s->x || !s->v || !s->F || !s->Ft || !s->img || !s->m || !s->q) return ORC_ERR_OOM;
  int64_t qtot = 0;
  for (int64_t p = 0; p < n; ++p) {
    for (int d = 0; d < 3; ++d) {
      double xx = x[3 * p + d];
      int32_t k = img ? img[3 * p + d] : 0;
      if (!(fabs(xx) <= 4.0 * s->L[d])) return ORC_ERR_INVALID;
      fold(s->L[d], &xx, &k);
      s->x[3 * p + d] = xx;
      s->img[3 * p + d] = k;
      s->v[3 * p + d] = v ? v[3 * p + d] : 0.0;
    }
    s->q[p] = q[p];
    s->m[p] = m ? m[p] : 1.0;
    if (q[p] > 32767 || q[p] < -32767) return ORC_ERR_INVALID;
    qtot += q[p];
  }
  /* a non-neutral system carries a uniform compensating background on the
   * vertices; it must be an exact integer in units of e 2^-48 */
  __int128 tot = (__int128)qtot * ((__int128)1 << 48);
  if (tot % s->V != 0) return ORC_ERR_INVALID;
  s->bg = (int64_t)(tot / s->V);
  return ORC_OK;
}

/* --------------------------------------------------------- dipole moment
 * Sec. V: the total dipole moment of the unfolded coordinates,
 * P = sum_i q_i x_i, taken from the fixed-point position the lattice sees,
 * (img N + c) S + f sub-cell steps of a / S. */
static void dipole(const orc_sys *s, double P[3]) {
  for (int d = 0; d < 3; ++d) {
    int64_t sum = 0;
    for (int64_t p = 0; p < s->n; ++p) {
      int32_t c, f;
      quantize(s, d, s->x[3 * p + d], &c, &f);
      int64_t U = ((int64_t)s->img[3 * p + d] * s->N[d] + c) * ORC_S + f;
      sum += (int64_t)s->q[p] * U;
    }
    P[d] = (double)sum * (s->a / ORC_S);
  }
}

/* ----------------------------------------------------- self energy
 * Sec. III: the interpolated charge of one particle interacts with itself
 * through the lattice Green's function,
 *   U_self = q^2 / (2 a eps) sum_{corners u,w} W_u W_w G(u - w),
 * with normalised linear weights W.  G depends only on |u_d - w_d| per axis,
 * so the double sum folds into products of c0 = (1-f)^2 + f^2 and
 * c1 = 2 f (1 - f).  The correction force is +dU_self/dx. */
static void self_terms(const orc_sys *s, const int32_t f[3], double q,
                       double ie_energy, const double ie_dir[3], double *U,
                       double F3[3]) {
  double c[3][2], dc[3][2];
  for (int d = 0; d < 3; ++d) {
    double t = (double)f[d] / ORC_S;
    c[d][0] = 1.0 - 2.0 * t + 2.0 * t * t;
    c[d][1] = 2.0 * t - 2.0 * t * t;
    dc[d][0] = 4.0 * t - 2.0;
    dc[d][1] = 2.0 - 4.0 * t;
  }
  double u = 0.0, g[3] = {0.0, 0.0, 0.0};
  for (int t = 0; t < 8; ++t) {
    int dl[3] = {t & 1, (t >> 1) & 1, (t >> 2) & 1};
    u += s->G[t] * c[0][dl[0]] * c[1][dl[1]] * c[2][dl[2]];
    g[0] += s->G[t] * dc[0][dl[0]] * c[1][dl[1]] * c[2][dl[2]];
    g[1] += s->G[t] * c[0][dl[0]] * dc[1][dl[1]] * c[2][dl[2]];
    g[2] += s->G[t] * c[0][dl[0]] * c[1][dl[1]] * dc[2][dl[2]];
  }
  double pre = q * q / (2.0 * s->a);
  *U = pre * ie_energy * u;
  for (int d = 0; d < 3; ++d) F3[d] = pre * ie_dir[d] * g[d] / s->a;
}

/* links of the cell with lower corner c: the 4 d-links at the corners
 * (a1, a2) of the perpendicular axes, and their normalised weights */
static void cell_links(const orc_sys *s, const int32_t c[3], const int32_t f[3],
                       int d, int64_t l[4], double w[4]) {
  int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
  int t = 0;
  for (int a2 = 0; a2 < 2; ++a2)
    for (int a1 = 0; a1 < 2; ++a1) {
      int64_t cc[3] = {c[0], c[1], c[2]};
      cc[e1] += a1;
      cc[e2] += a2;
      l[t] = d * s->V + vidx(s, cc[0], cc[1], cc[2]);
      w[t] = ((double)wgt(f[e1], a1) / ORC_S) * ((double)wgt(f[e2], a2) / ORC_S);
      ++t;
    }
}

/* permittivities seen by the self-energy term of a particle in cell c:
 * GF uses the mean 1/eps of the 12 cell links for every direction; DIRECT
 * uses, per direction d, the weighted mean of 1/eps over the 4 d-links. */
static void self_ie(const orc_sys *s, const int32_t c[3], const int32_t f[3],
                    double *ie_cell, double ie_dir[3]) {
  double tot = 0.0;
  for (int d = 0; d < 3; ++d) {
    int64_t l[4];
    double w[4];
    cell_links(s, c, f, d, l, w);
    double wd = 0.0;
    for (int t = 0; t < 4; ++t) { tot += s->ie[l[t]]; wd += s->ie[l[t]] * w[t]; }
    ie_dir[d] = wd;
  }
  *ie_cell = tot / 12.0;
  if (s->self_mode != ORC_SELF_DIRECT)
    for (int d = 0; d < 3; ++d) ie_dir[d] = *ie_cell;
}

void orc_self_force(const orc_sys *s, const int32_t f[3], const int32_t cell[3],
                    int32_t q, double *U, double *F3) {
  double ie_cell, ie_dir[3];
  self_ie(s, cell, f, &ie_cell, ie_dir);
  self_terms(s, f, (double)q, ie_cell, ie_dir, U, F3);
}

/* ------------------------------------------------------------ force gather
 * Eq. 18 without the magnetic part (Sec. II): F = q E, with E_d at the
 * particle interpolated linearly from the 4 d-links of its cell (the same
 * weights that carry its current), plus the self-energy correction
 * (Sec. III) and the metallic dipole correction q eps_eff^-1 P / V
 * (Sec. V).  The sign is +qE: it is the one that conserves energy with
 * Eq. 20. */
void orc_gather(orc_sys *s) {
  double P[3];
  dipole(s, P);
  double MP[3];
  for (int e = 0; e < 3; ++e)
    MP[e] = s->Minv[3 * e] * P[0] + s->Minv[3 * e + 1] * P[1] + s->Minv[3 * e + 2] * P[2];
  for (int64_t p = 0; p < s->n; ++p) {
    int32_t c[3], f[3];
    for (int d = 0; d < 3; ++d) quantize(s, d, s->x[3 * p + d], &c[d], &f[d]);
    double q = (double)s->q[p];
    double F[3];
    for (int d = 0; d < 3; ++d) {
      int64_t l[4];
      double w[4];
      cell_links(s, c, f, d, l, w);
      double E = 0.0;
      for (int t = 0; t < 4; ++t) E += s->D[l[t]] * s->ie[l[t]] * w[t];
      F[d] = q * E;
    }
    if (s->self_mode != ORC_SELF_NONE) {
      double U, Fs[3], ie_cell, ie_dir[3];
      self_ie(s, c, f, &ie_cell, ie_dir);
      self_terms(s, f, q, ie_cell, ie_dir, &U, Fs);
      for (int d = 0; d < 3; ++d) F[d] += Fs[d];
    }
    if (s->dipole_corr)
      for (int d = 0; d < 3; ++d) F[d] += q * MP[d] / s->Vbox;
    for (int d = 0; d < 3; ++d) {
      s->F[3 * p + d] = F[d];
      s->Ft[3 * p + d] = F[d];
    }
  }
}

/* Langevin force added after the gather: -gamma m v + sqrt(2 gamma m kT/dt) xi
 * with xi from Philox4x32-10, key = seed, counter = (particle, step). */
static void langevin(orc_sys *s) {
  uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
  for (int64_t p = 0; p < s->n; ++p) {
    uint32_t ctr[4] = {(uint32_t)p, (uint32_t)((uint64_t)p >> 32), (uint32_t)s->step,
                       (uint32_t)((uint64_t)s->step >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    double m = s->m[p];
    double sig = sqrt(2.0 * s->gamma * m * s->kT / s->dt);
    for (int d = 0; d < 3; ++d) {
      double fr = -s->gamma * m * s->v[3 * p + d];
      double fn = sig * unit_noise(r[d]);
      s->Ft[3 * p + d] = s->F[3 * p + d] + (fr + fn);
    }
  }
}

/* ------------------------------------------------------------ curl updates
 * Eq. 21 (Faraday): dB/dt = -curl E with E = D / eps on the links; the
 * plaquette (d, v) loses (dt / a) times the circulation of E around it. */
void orc_curl_B(orc_sys *s) {
  double k = s->dt / s->a;
  for (int d = 0; d < 3; ++d)
    for (int64_t v = 0; v < s->V; ++v) s->B[d * s->V + v] -= k * circulation(s, d, v);
}

/* Eq. 20 (Ampere) without the current: dD/dt = c^2 curl B.  The link (d, v)
 * gains c^2 dt / a times the sum of B over the 4 plaquettes that contain it,
 *   B_{d+2}(v) - B_{d+2}(v - e_{d+1}) - B_{d+1}(v) + B_{d+1}(v - e_{d+2}),
 * which is the transpose of the circulation map above. */
void orc_curl_D(orc_sys *s) {
  double k = s->c * s->c * s->dt / s->a;
  for (int d = 0; d < 3; ++d) {
    int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    for (int64_t v = 0; v < s->V; ++v) {
      int64_t c[3];
      vcoords(s, v, c);
      double t = s->B[e2 * s->V + v] - s->B[e2 * s->V + vshift(s, c, e1, -1)] -
                 s->B[e1 * s->V + v] + s->B[e1 * s->V + vshift(s, c, e2, -1)];
      s->D[d * s->V + v] += k * t;
    }
  }
}

/* ------------------------------------------------------ charge transfer
 * Eq. 20, the current term: a charge that moves along axis d from (c0, f0)
 * to (c1, f1) changes the flux of the d-links of its cell by -q times the
 * distance moved times the perpendicular weight, so that div D = rho stays
 * exact.  A crossed cell boundary splits the move over the old and the new
 * link.  The axes move in the order x, y, z, each with the perpendicular
 * weights of the moves made so far. */
static int32_t deposit_axis(orc_sys *s, int d, int32_t q, int32_t c0, int32_t f0,
                            int32_t c1, int32_t f1, int32_t dimg,
                            const int32_t cur_c[3], const int32_t cur_f[3]) {
  int64_t dc = (int64_t)c1 + (int64_t)dimg * s->N[d] - c0;
  if (dc < -1 || dc > 1) return ORC_ERR_CELL_JUMP;
  int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
  for (int a2 = 0; a2 < 2; ++a2)
    for (int a1 = 0; a1 < 2; ++a1) {
      int64_t wp = wgt(cur_f[e1], a1) * wgt(cur_f[e2], a2);
      int64_t cc[3] = {cur_c[0], cur_c[1], cur_c[2]};
      cc[e1] += a1;
      cc[e2] += a2;
      cc[d] = c0;
      int64_t l0 = d * s->V + vidx(s, cc[0], cc[1], cc[2]);
      if (dc == 0) {
        s->Tb[l0] += -(int64_t)q * (int64_t)(f1 - f0) * wp;
      } else if (dc == 1) {
        cc[d] = (int64_t)c0 + 1;
        int64_t l1 = d * s->V + vidx(s, cc[0], cc[1], cc[2]);
        s->Tb[l0] += -(int64_t)q * (int64_t)(ORC_S - f0) * wp;
        s->Tb[l1] += -(int64_t)q * (int64_t)f1 * wp;
      } else {
        cc[d] = (int64_t)c0 - 1;
        int64_t l1 = d * s->V + vidx(s, cc[0], cc[1], cc[2]);
        s->Tb[l0] += (int64_t)q * (int64_t)f0 * wp;
        s->Tb[l1] += (int64_t)q * (int64_t)(ORC_S - f1) * wp;
      }
    }
  return ORC_OK;
}

/* move particle p to the folded position xn with image counters kn */
static int32_t move_particle(orc_sys *s, int64_t p, const double xn[3],
                             const int32_t kn[3]) {
  int32_t c0[3], f0[3], c1[3], f1[3];
  for (int d = 0; d < 3; ++d) {
    quantize(s, d, s->x[3 * p + d], &c0[d], &f0[d]);
    quantize(s, d, xn[d], &c1[d], &f1[d]);
  }
  int32_t cur_c[3] = {c0[0], c0[1], c0[2]}, cur_f[3] = {f0[0], f0[1], f0[2]};
  for (int d = 0; d < 3; ++d) {
    int32_t st = deposit_axis(s, d, s->q[p], c0[d], f0[d], c1[d], f1[d],
                              kn[d] - s->img[3 * p + d], cur_c, cur_f);
    if (st != ORC_OK) return st;
    cur_c[d] = c1[d];
    cur_f[d] = f1[d];
  }
  for (int d = 0; d < 3; ++d) {
    s->x[3 * p + d] = xn[d];
    s->img[3 * p + d] = kn[d];
  }
  return ORC_OK;
}

/* apply the step's transfers: the ledger takes them exactly, D takes them
 * scaled by 2^-48 / a^2 */
static void apply_transfer(orc_sys *s) {
  double scale = ldexp(1.0, -48) / (s->a * s->a);
  for (int64_t l = 0; l < 3 * s->V; ++l) {
    int64_t t = s->Tb[l];
    if (t != 0) {
      s->Lg[l] += t;
      s->D[l] += (double)t * scale;
      s->Tb[l] = 0;
    }
  }
}

static int32_t drift_deposit(orc_sys *s) {
  for (int64_t p = 0; p < s->n; ++p) {
    double xn[3];
    int32_t kn[3];
    for (int d = 0; d < 3; ++d) {
      double step = s->dt * s->v[3 * p + d];
      if (!(fabs(step) <= 2.0 * s->a)) return ORC_ERR_CELL_JUMP;
      xn[d] = s->x[3 * p + d] + step;
      kn[d] = s->img[3 * p + d];
      fold(s->L[d], &xn[d], &kn[d]);
    }
    int32_t st = move_particle(s, p, xn, kn);
    if (st != ORC_OK) return st;
  }
  return ORC_OK;
}

int32_t orc_move(orc_sys *s, const double *x_new, const int32_t *img_new) {
  for (int64_t p = 0; p < s->n; ++p) {
    double xn[3];
    int32_t kn[3];
    for (int d = 0; d < 3; ++d) {
      xn[d] = x_new[3 * p + d];
      kn[d] = img_new[3 * p + d];
      if (!(fabs(xn[d]) <= 4.0 * s->L[d])) return ORC_ERR_INVALID;
      fold(s->L[d], &xn[d], &kn[d]);
    }
    int32_t st = move_particle(s, p, xn, kn);
    if (st != ORC_OK) return st;
  }
  apply_transfer(s);
  return ORC_OK;
}

/* --------------------------------------------------- initial field solve
 * Sec. II: Gauss solution by the recursive scheme of Fig. 1 (exact, int64),
 * the k = 0 mode set to -P/V (Sec. V), relaxation to curl E = 0, B = 0 from
 * the initial condition dTheta/dt(0) = 0 (Eq. 13), then the forces. */
/* Sec. II and V: D from the exact flux ledger, its k = 0 mode set to -P/V,
 * then relaxed to curl E = 0; B = 0 and the forces gathered */
static int32_t field_from_ledger(orc_sys *s) {
  double scale = ldexp(1.0, -48) / (s->a * s->a);
  double P[3];
  dipole(s, P);
  for (int d = 0; d < 3; ++d) {
    int64_t sum = 0;
    for (int64_t v = 0; v < s->V; ++v) sum += s->Lg[d * s->V + v];
    double shift = -P[d] / s->Vbox - ((double)sum * scale) / (double)s->V;
    for (int64_t v = 0; v < s->V; ++v)
      s->D[d * s->V + v] = (double)s->Lg[d * s->V + v] * scale + shift;
  }
  int32_t st = orc_relax(s, s->relax_tol, s->relax_maxit, NULL);
  if (st != ORC_OK) return st;
  memset(s->B, 0, sizeof(double) * 3 * s->V);
  orc_gather(s);
  return ORC_OK;
}

int32_t orc_init_field(orc_sys *s) {
  int64_t *Q = (int64_t *)malloc(sizeof(int64_t) * s->V);
  if (!Q) return ORC_ERR_OOM;
  orc_cic_charges(s, Q);
  int32_t st = orc_gauss_scan(s->N, Q, s->Lg);
  free(Q);
  if (st != ORC_OK) return st;
  memset(s->Tb, 0, sizeof(int64_t) * 3 * s->V);
  s->step = 0;
  return field_from_ledger(s);
}

int32_t orc_set_eps(orc_sys *s, const orc_eps *eps, int32_t relax) {
  size_t bytes = sizeof(double) * 3 * s->V;
  double *ie0 = (double *)malloc(bytes), *D0 = (double *)malloc(bytes), M0[9];
  if (!ie0 || !D0) { free(ie0); free(D0); return ORC_ERR_OOM; }
  memcpy(ie0, s->ie, bytes);
  memcpy(D0, s->D, bytes);
  memcpy(M0, s->Minv, sizeof(M0));
  int32_t st = map_eps(s, eps);
  if (st == ORC_OK) st = eps_effective(s); /* uses D as scratch */
  memcpy(s->D, D0, bytes);
  if (st != ORC_OK) {
    memcpy(s->ie, ie0, bytes);
    memcpy(s->Minv, M0, sizeof(M0));
  }
  free(ie0);
  free(D0);
  if (st != ORC_OK) return st;
  if (relax) return field_from_ledger(s);
  orc_gather(s);
  return ORC_OK;
}

/* ----------------------------------------------- eps from salt density
 * Sec. I motivation, reading in memd_oracle.h: cloud-in-cell |q| density at
 * the vertices, periodic Gaussian smoothing axis by axis, a clamped linear
 * map to eps, applied as vertex values. */
void orc_smooth_periodic(const int32_t N[3], double sigma, double *rho) {
  if (!(sigma > 0.0)) return;
  int R = (int)ceil(3.0 * sigma);
  double *w = (double *)malloc(sizeof(double) * (2 * R + 1));
  double wsum = 0.0;
  for (int j = -R; j <= R; ++j) {
    w[j + R] = exp(-(double)(j * j) / (2.0 * sigma * sigma));
    wsum += w[j + R];
  }
  for (int j = 0; j <= 2 * R; ++j) w[j] /= wsum;
  int64_t V = (int64_t)N[0] * N[1] * N[2];
  double *tmp = (double *)malloc(sizeof(double) * V);
  for (int d = 0; d < 3; ++d) {
    for (int64_t k = 0; k < N[2]; ++k)
      for (int64_t jj = 0; jj < N[1]; ++jj)
        for (int64_t i = 0; i < N[0]; ++i) {
          int64_t c[3] = {i, jj, k};
          double acc = 0.0;
          for (int j = -R; j <= R; ++j) {
            int64_t e[3] = {c[0], c[1], c[2]};
            e[d] = ((e[d] + j) % N[d] + N[d]) % N[d];
            acc += w[j + R] * rho[e[0] + N[0] * (e[1] + N[1] * e[2])];
          }
          tmp[i + N[0] * (jj + N[1] * k)] = acc;
        }
    memcpy(rho, tmp, sizeof(double) * V);
  }
  free(tmp);
  free(w);
}

int32_t orc_salt_vertex_eps(const orc_sys *s, const double rule[5], double *ev) {
  double eps0 = rule[0], slope = rule[1], lo = rule[2], hi = rule[3], sigma = rule[4];
  double *rho = (double *)malloc(sizeof(double) * s->V);
  if (!rho) return ORC_ERR_OOM;
  /* |q| weights in fixed point (exact), then in units of e */
  for (int64_t v = 0; v < s->V; ++v) rho[v] = 0.0;
  int64_t *Qa = (int64_t *)calloc((size_t)s->V, sizeof(int64_t));
  for (int64_t p = 0; p < s->n; ++p) {
    int32_t c[3], f[3];
    for (int d = 0; d < 3; ++d) quantize(s, d, s->x[3 * p + d], &c[d], &f[d]);
    int64_t aq = s->q[p] < 0 ? -(int64_t)s->q[p] : (int64_t)s->q[p];
    for (int az = 0; az < 2; ++az)
      for (int ay = 0; ay < 2; ++ay)
        for (int ax = 0; ax < 2; ++ax)
          Qa[vidx(s, c[0] + ax, c[1] + ay, c[2] + az)] +=
              aq * (wgt(f[0], ax) * wgt(f[1], ay) * wgt(f[2], az));
  }
  for (int64_t v = 0; v < s->V; ++v) rho[v] = (double)Qa[v] * ldexp(1.0, -48);
  free(Qa);
  orc_smooth_periodic(s->N, sigma, rho);
  double mean = 0.0;
  for (int64_t v = 0; v < s->V; ++v) mean += rho[v];
  mean /= (double)s->V;
  for (int64_t v = 0; v < s->V; ++v) {
    double e = mean > 0.0 ? eps0 + slope * (rho[v] / mean - 1.0) : eps0;
    ev[v] = e < lo ? lo : (e > hi ? hi : e);
  }
  free(rho);
  return ORC_OK;
}

int32_t orc_eps_from_density(orc_sys *s, const double rule[5], int32_t relax, double *eps_out) {
  double *ev = (double *)malloc(sizeof(double) * s->V);
  if (!ev) return ORC_ERR_OOM;
  int32_t st = orc_salt_vertex_eps(s, rule, ev);
  if (st != ORC_OK) {
    free(ev);
    return st;
  }
  if (eps_out) memcpy(eps_out, ev, sizeof(double) * s->V);
  orc_eps e;
  memset(&e, 0, sizeof(e));
  e.kind = ORC_EPS_VERTICES;
  e.values = ev;
  st = orc_set_eps(s, &e, relax);
  free(ev);
  return st;
}

/* -------------------------------------------------------------- time step
 * One step of the coupled system, leapfrog in the fields and velocity
 * Verlet in the particles:
 *   v += dt/2m Ft;  B -= dt curl E (Eq. 21);  x += dt v and the charge
 *   transfer of the move;  D += c^2 dt curl B (Eq. 20) and D -= j dt from
 *   the transfers;  F = gather;  Ft = F + Langevin;  v += dt/2m Ft. */
int32_t orc_step(orc_sys *s, int64_t nsteps, int32_t thermo, double gamma,
                 double kT) {
  s->thermo = thermo;
  s->gamma = gamma;
  s->kT = kT;
  for (int64_t it = 0; it < nsteps; ++it) {
    for (int64_t p = 0; p < s->n; ++p) {
      double h = 0.5 * s->dt / s->m[p];
      for (int d = 0; d < 3; ++d) s->v[3 * p + d] += h * s->Ft[3 * p + d];
    }
    orc_curl_B(s);
    int32_t st = drift_deposit(s);
    if (st != ORC_OK) return st;
    orc_curl_D(s);
    apply_transfer(s);
    orc_gather(s);
    if (thermo) langevin(s);
    for (int64_t p = 0; p < s->n; ++p) {
      double h = 0.5 * s->dt / s->m[p];
      for (int d = 0; d < 3; ++d) s->v[3 * p + d] += h * s->Ft[3 * p + d];
    }
    s->step += 1;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ energy
 * Kinetic + electric a^3 sum D^2 / 2 eps + magnetic
 * (c^2 a^3 / 2) sum B^{n+1/2} B^{n+3/2} (the time-centred product that the
 * leapfrog conserves; B^{n+3/2} = B - dt/a circ E), minus the self energies
 * and the dipole energy P eps_eff^-1 P / 2V that the corrections remove.
 * Also the Gauss residual max |div D a^2 - Q| (in e) and whether the ledger
 * satisfies div Lg == Q exactly. */
void orc_energy(orc_sys *s, double *out) {
  double a3 = s->a * s->a * s->a;
  double ke = 0.0, el = 0.0, mag = 0.0, self = 0.0;
  for (int64_t p = 0; p < s->n; ++p)
    for (int d = 0; d < 3; ++d) ke += 0.5 * s->m[p] * s->v[3 * p + d] * s->v[3 * p + d];
  for (int64_t l = 0; l < 3 * s->V; ++l) el += 0.5 * s->D[l] * s->D[l] * s->ie[l];
  el *= a3;
  double k = s->dt / s->a;
  for (int d = 0; d < 3; ++d)
    for (int64_t v = 0; v < s->V; ++v) {
      double b = s->B[d * s->V + v];
      mag += b * (b - k * circulation(s, d, v));
    }
  mag *= 0.5 * s->c * s->c * a3;
  if (s->self_mode != ORC_SELF_NONE)
    for (int64_t p = 0; p < s->n; ++p) {
      int32_t c[3], f[3];
      for (int d = 0; d < 3; ++d) quantize(s, d, s->x[3 * p + d], &c[d], &f[d]);
      double U, F3[3], ie_cell, ie_dir[3];
      self_ie(s, c, f, &ie_cell, ie_dir);
      self_terms(s, f, (double)s->q[p], ie_cell, ie_dir, &U, F3);
      self += U;
    }
  double P[3];
  dipole(s, P);
  double dip = 0.0;
  if (s->dipole_corr)
    for (int e = 0; e < 3; ++e)
      for (int d = 0; d < 3; ++d) dip += 0.5 * P[e] * s->Minv[3 * e + d] * P[d] / s->Vbox;
  out[ORC_E_KIN] = ke;
  out[ORC_E_ELEC] = el;
  out[ORC_E_MAG] = mag;
  out[ORC_E_SELF] = self;
  out[ORC_E_DIP] = dip;
  out[ORC_E_TOTAL] = ke + el + mag - self - dip;
  out[ORC_E_P0] = P[0];
  out[ORC_E_P1] = P[1];
  out[ORC_E_P2] = P[2];
  /* Gauss law */
  int64_t *Q = (int64_t *)malloc(sizeof(int64_t) * s->V);
  int64_t *dv = (int64_t *)malloc(sizeof(int64_t) * s->V);
  double res = 0.0;
  int exact = 1;
  if (Q && dv) {
    orc_cic_charges(s, Q);
    orc_divergence(s->N, s->Lg, dv);
    double a2 = s->a * s->a;
    for (int64_t v = 0; v < s->V; ++v) {
      if (dv[v] != Q[v]) exact = 0;
      int64_t c[3];
      vcoords(s, v, c);
      double divD = 0.0;
      for (int d = 0; d < 3; ++d)
        divD += s->D[d * s->V + v] - s->D[d * s->V + vshift(s, c, d, -1)];
      double r = fabs(divD * a2 - (double)Q[v] * ldexp(1.0, -48));
      if (r > res) res = r;
    }
  } else {
    exact = 0;
    res = NAN;
  }
  free(Q);
  free(dv);
  out[ORC_E_GAUSS_RES] = res;
  out[ORC_E_GAUSS_EXACT] = exact ? 1.0 : 0.0;
}
