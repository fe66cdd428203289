/*
 * Plain FP64 CPU oracle of the TLBfind lattice Boltzmann step (arXiv 2109.12565).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the CUDA library.  Written for
 * readability against the paper, not for speed: every sub-step runs as its
 * own sweep over the lattice in the order the paper states the model
 * (moments -> pseudo-potentials -> forces -> velocities -> collision ->
 * streaming).  Compile with -ffp-contract=off; the OpenMP build only adds
 * "parallel for" over rows and computes the same numbers.
 *
 * Readings of the paper taken here (each is listed with its evidence in the
 * design notes of the repository):
 *   - F^x uses psi~ = rho/rho0 (Eq. FAB with the pseudo-potential stated
 *     right after it); F^a and F^r use psi = rho0 (1 - exp(-rho/rho0)).
 *   - G^r_ll > 0 as the text after Eq. (FintRepulsive) says; the negative
 *     signs printed in the input tables of Appendix A/B are not used.
 *   - u = total bare momentum / total density (Eq. velo); u_l = u + tau F_l / rho_l
 *     in f^eq (Eq. shift); u^(H) = u + F / (2 rho) (text after Eq. NS) in g^eq
 *     (Eq. Teq) and in the observables.
 *   - All forces use the moments of the same pre-collision state S_t.
 *   - Walls: half-way bounce-back for f (Sec. 2.2, u_w = 0); anti-bounce-back
 *     g_{-i}(x, t+1) = -g*_i(x, t) + 2 w_i T_w for g (thermal walls at fixed
 *     T, Sec. 3.2.3; the mechanism is not stated in the paper).  A solid node
 *     in the lower half of the lattice is at T_down, in the upper half at T_up.
 *   - Every solid or out-of-domain position reached by a force stencil takes
 *     the wall densities rho_w (Sec. 2.2.1): component 1 rho_w,max, component 2
 *     rho_w,min, and the pseudo-potentials of those densities.
 *   - Nu (Eq. NuTime): <.> averages over fluid nodes; u_y = u^(H)_y; dT/dy by
 *     central differences with the mirror value 2 T_w - T at a solid
 *     neighbour; "ny" of the formula is the wall-to-wall height H = ny - 2.
 */
#include "tlb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Fig. 1: lattice vectors.  0-8 are the D2Q9 links (NN), 9-24 the next-to-nearest belt (NNN). */
static const int CX[25] = {0, 1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0, 1, -1, -1, 1, 2, -2, -2, 2, 2, -2, -2, 2};
static const int CY[25] = {0, 0, 1, 0, -1, 1, 1, -1, -1, 0, 2, 0, -2, 2, 2, -2, -2, 1, 1, -1, -1, 2, 2, -2, -2};
/* Opposite D2Q9 link. */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* Fig. 1b: w_i = w(c_i) (D2Q9) and p_i = p(c_i) as functions of |c_i|^2. */
static double weight_w(int i) {
  int r2 = CX[i] * CX[i] + CY[i] * CY[i];
  if (r2 == 0) return 4.0 / 9.0;
  if (r2 == 1) return 1.0 / 9.0;
  if (r2 == 2) return 1.0 / 36.0;
  return 0.0;
}
static double weight_p(int i) {
  int r2 = CX[i] * CX[i] + CY[i] * CY[i];
  switch (r2) {
    case 0: return 247.0 / 420.0;
    case 1: return 4.0 / 63.0;
    case 2: return 4.0 / 135.0;
    case 4: return 1.0 / 180.0;
    case 5: return 2.0 / 945.0;
    case 8: return 1.0 / 15120.0;
  }
  return 0.0;
}

void orc_tables(int* c, double* w, double* p) {
  for (int i = 0; i < 25; ++i) {
    c[2 * i] = CX[i];
    c[2 * i + 1] = CY[i];
    p[i] = weight_p(i);
    if (i < 9) w[i] = weight_w(i);
  }
}

static int valid(const orc_params* prm) {
  if (!prm || prm->nx < 1 || prm->ny < 1) return 0;
  if (!prm->periodic_y && prm->ny < 3) return 0;
  return 1;
}

static int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

int orc_solid_map(const orc_params* prm, const uint8_t* mask, uint8_t* solid) {
  if (!valid(prm)) return -1;
  const int nx = prm->nx, ny = prm->ny;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int s = mask ? (mask[y * nx + x] != 0) : 0;
      if (!prm->periodic_y && (y == 0 || y == ny - 1)) s = 1;
      solid[y * nx + x] = (uint8_t)s;
    }
  return 0;
}

/* Wall temperature of a solid node (Sec. 3.2.3: hot bottom wall, cold top wall). */
static double wall_T(const orc_params* prm, int y) { return (2 * y < prm->ny) ? prm->T_down : prm->T_up; }

int orc_init(const orc_params* prm, const uint8_t* mask, const double* rho1, const double* rho2,
             const double* T, double* state) {
  if (!valid(prm)) return -1;
  const int nx = prm->nx, ny = prm->ny;
  const long N = (long)nx * ny;
  uint8_t* solid = (uint8_t*)malloc((size_t)N);
  orc_solid_map(prm, mask, solid);
  memset(state, 0, sizeof(double) * 27 * (size_t)N);
  for (long n = 0; n < N; ++n) {
    if (solid[n]) continue;
    for (int i = 0; i < 9; ++i) {
      state[(long)i * N + n] = weight_w(i) * rho1[n];
      state[(long)(9 + i) * N + n] = weight_w(i) * rho2[n];
      state[(long)(18 + i) * N + n] = weight_w(i) * T[n];
    }
  }
  free(solid);
  return 0;
}

/* Value of a per-node field at lattice position (x, y), any integers: x wraps; y wraps when
 * periodic; a solid or out-of-domain position returns the wall value (Sec. 2.2.1). */
static double field_at(const orc_params* prm, const uint8_t* solid, const double* field, double wall_value,
                       int x, int y) {
  const int nx = prm->nx, ny = prm->ny;
  x = wrap(x, nx);
  if (prm->periodic_y)
    y = wrap(y, ny);
  else if (y < 0 || y >= ny)
    return wall_value;
  if (solid[y * nx + x]) return wall_value;
  return field[y * nx + x];
}

/* Pseudo-potential of Eqs. (FintAttrattive)-(FintRepulsive): psi = rho0 (1 - exp(-rho/rho0)). */
static double psi_exp(double rho, double rho0) { return rho0 * (1.0 - exp(-rho / rho0)); }

/* Forces F_l = F^x_l + F^a_l + F^r_l + F^ext_l on every fluid node, Eqs. (FAB), (FintAttrattive),
 * (FintRepulsive), (alphaG), written out term by term. */
static void forces_from_fields(const orc_params* prm, const uint8_t* solid, const double* rho1,
                               const double* rho2, const double* T, double* F) {
  const int nx = prm->nx, ny = prm->ny;
  const long N = (long)nx * ny;
  const double rho0 = prm->rho0;
  const double* rho[2] = {rho1, rho2};
  double* psit[2]; /* psi~_l = rho_l / rho0, used by F^x */
  double* psie[2]; /* psi_l = rho0 (1 - exp(-rho_l/rho0)), used by F^a, F^r */
  double psit_w[2], psie_w[2];
  for (int l = 0; l < 2; ++l) {
    psit[l] = (double*)malloc(sizeof(double) * (size_t)N);
    psie[l] = (double*)malloc(sizeof(double) * (size_t)N);
    for (long n = 0; n < N; ++n) {
      if (solid[n]) {
        psit[l][n] = psie[l][n] = 0.0; /* never read: field_at returns the wall value */
      } else {
        psit[l][n] = rho[l][n] / rho0;
        psie[l][n] = psi_exp(rho[l][n], rho0);
      }
    }
    psit_w[l] = prm->rho_wall[l] / rho0;
    psie_w[l] = psi_exp(prm->rho_wall[l], rho0);
  }
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      const long n = (long)y * nx + x;
      for (int l = 0; l < 2; ++l) {
        double fx = 0.0, fy = 0.0;
        if (!solid[n]) {
          const int m = 1 - l;
          /* Eq. (FAB): F^x_l = -G12 psi~_l(x) sum_{i in NN} w_i psi~_m(x + c_i) c_i */
          double sx = 0.0, sy = 0.0;
          for (int i = 0; i < 9; ++i) {
            double v = field_at(prm, solid, psit[m], psit_w[m], x + CX[i], y + CY[i]);
            sx += weight_w(i) * v * CX[i];
            sy += weight_w(i) * v * CY[i];
          }
          fx += -prm->G12 * psit[l][n] * sx;
          fy += -prm->G12 * psit[l][n] * sy;
          /* Eq. (FintAttrattive): F^a_l = -G^a_ll psi_l(x) sum_{i in NN} w_i psi_l(x + c_i) c_i */
          sx = sy = 0.0;
          for (int i = 0; i < 9; ++i) {
            double v = field_at(prm, solid, psie[l], psie_w[l], x + CX[i], y + CY[i]);
            sx += weight_w(i) * v * CX[i];
            sy += weight_w(i) * v * CY[i];
          }
          fx += -prm->Ga[l] * psie[l][n] * sx;
          fy += -prm->Ga[l] * psie[l][n] * sy;
          /* Eq. (FintRepulsive): F^r_l = -G^r_ll psi_l(x) sum_{i in NN u NNN} p_i psi_l(x + c_i) c_i */
          sx = sy = 0.0;
          for (int i = 0; i < 25; ++i) {
            double v = field_at(prm, solid, psie[l], psie_w[l], x + CX[i], y + CY[i]);
            sx += weight_p(i) * v * CX[i];
            sy += weight_p(i) * v * CY[i];
          }
          fx += -prm->Gr[l] * psie[l][n] * sx;
          fy += -prm->Gr[l] * psie[l][n] * sy;
          /* Eq. (alphaG): F^ext_l = rho_l alpha g T e_y; plus the constant body acceleration along x */
          fy += rho[l][n] * prm->alpha_g * T[n];
          fx += rho[l][n] * prm->body_fx;
        }
        F[((long)l * 2 + 0) * N + n] = fx;
        F[((long)l * 2 + 1) * N + n] = fy;
      }
    }
  }
  for (int l = 0; l < 2; ++l) {
    free(psit[l]);
    free(psie[l]);
  }
}

int orc_forces(const orc_params* prm, const uint8_t* mask, const double* rho1, const double* rho2,
               const double* T, double* F) {
  if (!valid(prm)) return -1;
  const long N = (long)prm->nx * prm->ny;
  uint8_t* solid = (uint8_t*)malloc((size_t)N);
  orc_solid_map(prm, mask, solid);
  forces_from_fields(prm, solid, rho1, rho2, T, F);
  free(solid);
  return 0;
}

/* Moments of Sec. 2.1 and Sec. 2.3 at every fluid node: rho_l = sum_i f_{l,i}, j = sum_{l,i} c_i f_{l,i},
 * T = sum_i g_i.  Solid nodes get rho_w and the wall temperature (only used by the observables). */
static void moments(const orc_params* prm, const uint8_t* solid, const double* st, double* rho1, double* rho2,
                    double* jx, double* jy, double* T) {
  const int nx = prm->nx, ny = prm->ny;
  const long N = (long)nx * ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      const long n = (long)y * nx + x;
      if (solid[n]) {
        rho1[n] = prm->rho_wall[0];
        rho2[n] = prm->rho_wall[1];
        jx[n] = jy[n] = 0.0;
        T[n] = wall_T(prm, y);
        continue;
      }
      double r1 = 0.0, r2 = 0.0, mx = 0.0, my = 0.0, t = 0.0;
      for (int i = 0; i < 9; ++i) {
        const double a = st[(long)i * N + n], b = st[(long)(9 + i) * N + n];
        r1 += a;
        r2 += b;
        mx += CX[i] * a + CX[i] * b;
        my += CY[i] * a + CY[i] * b;
        t += st[(long)(18 + i) * N + n];
      }
      rho1[n] = r1;
      rho2[n] = r2;
      jx[n] = mx;
      jy[n] = my;
      T[n] = t;
    }
  }
}

/* Second-order equilibrium of Sec. 2.1 (and Eq. Teq with T in place of rho), c_s^2 = 1/3:
 * w_i a [1 + c.u / cs2 + (c.u)^2 / (2 cs4) - u.u / (2 cs2)]. */
static double equilibrium(int i, double a, double ux, double uy) {
  const double cs2 = 1.0 / 3.0;
  const double cu = CX[i] * ux + CY[i] * uy;
  const double uu = ux * ux + uy * uy;
  return weight_w(i) * a * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
}

/* x velocity of the wall that solid row yd belongs to: the flat bottom / top wall rows move with
 * u_wall (Couette, Sec. 2.2); obstacle posts and periodic lattices are at rest. */
static double wall_u(const orc_params* prm, int yd) {
  if (prm->periodic_y) return 0.0;
  if (yd == 0) return prm->u_wall[0];
  if (yd == prm->ny - 1) return prm->u_wall[1];
  return 0.0;
}

/* One step; with wall_fx != NULL also the x momentum handed to the bottom / top wall rows. */
static int step_impl(const orc_params* prm, const uint8_t* mask, const double* in, double* out, double* wall_fx) {
  if (!valid(prm)) return -1;
  const int nx = prm->nx, ny = prm->ny;
  const long N = (long)nx * ny;
  uint8_t* solid = (uint8_t*)malloc((size_t)N);
  double* buf = (double*)malloc(sizeof(double) * 9 * (size_t)N);
  double *rho1 = buf, *rho2 = buf + N, *jx = buf + 2 * N, *jy = buf + 3 * N, *T = buf + 4 * N;
  double* F = buf + 5 * N; /* [l][xy][N] */
  orc_solid_map(prm, mask, solid);

  /* 1. moments (Sec. 2.1, 2.3) */
  moments(prm, solid, in, rho1, rho2, jx, jy, T);
  /* 2-3. pseudo-potentials and forces (Eqs. FAB, FintAttrattive, FintRepulsive, alphaG) */
  forces_from_fields(prm, solid, rho1, rho2, T, F);

  memset(out, 0, sizeof(double) * 27 * (size_t)N);
  double* rowacc = (double*)calloc(2 * (size_t)ny, sizeof(double)); /* per row: bottom, top wall */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      const long n = (long)y * nx + x;
      if (solid[n]) continue;
      const double r[2] = {rho1[n], rho2[n]};
      const double rho = r[0] + r[1];
      /* 4. velocities: Eq. (velo), Eq. (shift), u^(H) = u + F/(2 rho) */
      const double ux = jx[n] / rho, uy = jy[n] / rho;
      const double Fx = F[0 * N + n] + F[2 * N + n], Fy = F[1 * N + n] + F[3 * N + n];
      const double uHx = ux + Fx / (2.0 * rho), uHy = uy + Fy / (2.0 * rho);
      double fpost[27];
      for (int l = 0; l < 2; ++l) {
        const double ulx = ux + prm->tau * F[((long)l * 2 + 0) * N + n] / r[l];
        const double uly = uy + prm->tau * F[((long)l * 2 + 1) * N + n] / r[l];
        /* 5. BGK collision, Eq. (BGK): f* = f - (f - f^eq(rho_l, u_l)) / tau */
        for (int i = 0; i < 9; ++i) {
          const double f = in[(long)(9 * l + i) * N + n];
          fpost[9 * l + i] = f - (f - equilibrium(i, r[l], ulx, uly)) / prm->tau;
        }
      }
      /* thermal BGK, Eq. (LBMg) with g^eq of Eq. (Teq) at u^(H) */
      for (int i = 0; i < 9; ++i) {
        const double g = in[(long)(18 + i) * N + n];
        fpost[18 + i] = g - (g - equilibrium(i, T[n], uHx, uHy)) / prm->tau_g;
      }
      /* 6. streaming, Eq. (LBM): f(x + c_i, t+1) = f*(x, t); a link into a solid node bounces back
       * (half-way), and the thermal population is anti-bounced with the wall temperature. */
      for (int i = 0; i < 9; ++i) {
        int xd = wrap(x + CX[i], nx), yd = y + CY[i];
        if (prm->periodic_y) yd = wrap(yd, ny);
        /* with walls, fluid rows are 1..ny-2, so yd is always inside the lattice */
        const long nd = (long)yd * nx + xd;
        if (!solid[nd]) {
          out[(long)i * N + nd] = fpost[i];
          out[(long)(9 + i) * N + nd] = fpost[9 + i];
          out[(long)(18 + i) * N + nd] = fpost[18 + i];
        } else {
          /* a moving flat wall gives the bounced population of component l the momentum
           * 2 w_i rho_l (c_i . u_w) / c_s^2 = 6 w_i rho_l c_ix u_w (mass-conserving: the links
           * that cross a flat wall have sum_i w_i c_ix = 0); posts and resting walls add nothing */
          const int o = OPP[i];
          const double uw = wall_u(prm, yd);
          const double b1 = fpost[i] - 6.0 * weight_w(i) * r[0] * CX[i] * uw;
          const double b2 = fpost[9 + i] - 6.0 * weight_w(i) * r[1] * CX[i] * uw;
          out[(long)o * N + n] = b1;
          out[(long)(9 + o) * N + n] = b2;
          out[(long)(18 + o) * N + n] = -fpost[18 + i] + 2.0 * weight_w(i) * wall_T(prm, yd);
          if (!prm->periodic_y && (yd == 0 || yd == ny - 1))
            rowacc[2 * y + (yd == 0 ? 0 : 1)] += CX[i] * ((fpost[i] + b1) + (fpost[9 + i] + b2));
        }
      }
    }
  }
  if (wall_fx) {
    wall_fx[0] = wall_fx[1] = 0.0;
    for (int y = 0; y < ny; ++y) {
      wall_fx[0] += rowacc[2 * y];
      wall_fx[1] += rowacc[2 * y + 1];
    }
  }
  free(rowacc);
  free(buf);
  free(solid);
  return 0;
}

int orc_step(const orc_params* prm, const uint8_t* mask, const double* in, double* out) {
  return step_impl(prm, mask, in, out, NULL);
}

int orc_wall_force(const orc_params* prm, const uint8_t* mask, const double* state, double* out) {
  if (!valid(prm) || !out) return -1;
  double* tmp = (double*)malloc(sizeof(double) * 27 * (size_t)prm->nx * prm->ny);
  if (!tmp) return -2;
  const int rc = step_impl(prm, mask, state, tmp, out);
  free(tmp);
  return rc;
}

int orc_run(const orc_params* prm, const uint8_t* mask, double* state, double* work, long nsteps) {
  if (!valid(prm) || nsteps < 0) return -1;
  const long N = (long)prm->nx * prm->ny;
  for (long s = 0; s < nsteps; ++s) {
    int rc = orc_step(prm, mask, state, work);
    if (rc) return rc;
    memcpy(state, work, sizeof(double) * 27 * (size_t)N);
  }
  return 0;
}

/* Fields of S_t including u^(H) = u + F / (2 rho). */
static void fields_full(const orc_params* prm, const uint8_t* solid, const double* st, double* rho1,
                        double* rho2, double* T, double* uHx, double* uHy) {
  const long N = (long)prm->nx * prm->ny;
  double* buf = (double*)malloc(sizeof(double) * 6 * (size_t)N);
  double *jx = buf, *jy = buf + N, *F = buf + 2 * N;
  moments(prm, solid, st, rho1, rho2, jx, jy, T);
  forces_from_fields(prm, solid, rho1, rho2, T, F);
  for (long n = 0; n < N; ++n) {
    if (solid[n]) {
      uHx[n] = uHy[n] = 0.0;
      continue;
    }
    const double rho = rho1[n] + rho2[n];
    const double Fx = F[0 * N + n] + F[2 * N + n], Fy = F[1 * N + n] + F[3 * N + n];
    uHx[n] = jx[n] / rho + Fx / (2.0 * rho);
    uHy[n] = jy[n] / rho + Fy / (2.0 * rho);
  }
  free(buf);
}

int orc_fields(const orc_params* prm, const uint8_t* mask, const double* state, double* rho1, double* rho2,
               double* T, double* ux, double* uy) {
  if (!valid(prm)) return -1;
  const long N = (long)prm->nx * prm->ny;
  uint8_t* solid = (uint8_t*)malloc((size_t)N);
  orc_solid_map(prm, mask, solid);
  fields_full(prm, solid, state, rho1, rho2, T, ux, uy);
  free(solid);
  return 0;
}

int orc_observables(const orc_params* prm, const uint8_t* mask, const double* state, double* out) {
  if (!valid(prm)) return -1;
  const int nx = prm->nx, ny = prm->ny;
  const long N = (long)nx * ny;
  uint8_t* solid = (uint8_t*)malloc((size_t)N);
  double* buf = (double*)malloc(sizeof(double) * 5 * (size_t)N);
  double *rho1 = buf, *rho2 = buf + N, *T = buf + 2 * N, *ux = buf + 3 * N, *uy = buf + 4 * N;
  orc_solid_map(prm, mask, solid);
  fields_full(prm, solid, state, rho1, rho2, T, ux, uy);
  double m1 = 0, m2 = 0, px = 0, py = 0, uyT = 0, dyT = 0, e = 0, bad = 0, nf = 0;
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      const long n = (long)y * nx + x;
      if (solid[n]) continue;
      nf += 1;
      if (!(rho1[n] > 0.0) || !(rho2[n] > 0.0) || !isfinite(rho1[n]) || !isfinite(rho2[n]) || !isfinite(T[n]))
        bad += 1;
      const double rho = rho1[n] + rho2[n];
      m1 += rho1[n];
      m2 += rho2[n];
      px += rho * ux[n];
      py += rho * uy[n];
      e += ux[n] * ux[n] + uy[n] * uy[n];
      uyT += uy[n] * T[n];
      /* central difference in y with the mirror value 2 T_w - T(x) at a solid neighbour */
      double Tn[2];
      for (int s = 0; s < 2; ++s) {
        int yy = y + (s ? 1 : -1);
        if (prm->periodic_y) yy = wrap(yy, ny);
        const long nn = (long)yy * nx + x;
        Tn[s] = solid[nn] ? 2.0 * wall_T(prm, yy) - T[n] : T[nn];
      }
      dyT += 0.5 * (Tn[1] - Tn[0]);
    }
  }
  const double kappa = (prm->tau_g - 0.5) / 3.0; /* Eq. (K) */
  const double dT = prm->T_down - prm->T_up;
  double Nu = 0.0;
  if (!prm->periodic_y && dT != 0.0 && nf > 0) {
    const double H = (double)(ny - 2);
    Nu = (uyT / nf - kappa * dyT / nf) / (kappa * dT / H); /* Eq. (NuTime) */
  }
  out[0] = m1;
  out[1] = m2;
  out[2] = px;
  out[3] = py;
  out[4] = Nu;
  out[5] = nf > 0 ? e / nf : 0.0;
  out[6] = bad;
  out[7] = nf;
  free(buf);
  free(solid);
  return 0;
}

/* ======================================================================================
 * Total shear stress of the rheology experiment (Sec. 2.1, text after Eq. NS; Sec. 3.2.1).
 *
 * The total stress is the bare viscous stress eta_0 (d_i u^(H)_j + d_j u^(H)_i), Eq. (VISCO):
 * eta_0 = rho c_s^2 (tau - 1/2), supplemented by the pressure tensor P_ij of the model.
 * The xy component at a fluid node x:
 *   sigma_xy(x) = eta_0(x) (d_x u^(H)_y + d_y u^(H)_x) - P^int_xy(x) - P^F_xy(x)
 * with central differences; a solid neighbour takes the mirror value 2 u_w - u(x) (u_w: the wall
 * velocity along x of a flat wall row, 0 for the y component and for obstacles).
 *   P^int: the virial form of the pair forces of Eqs. (FAB), (FintAttrattive), (FintRepulsive): a
 *          force -G psi(x) sum_i W_i psi(x + c_i) c_i contributes (G / 2) psi(x) sum_i W_i
 *          psi(x + c_i) c_ix c_iy, i.e. half of every pair term, so that the pair's two ends together
 *          carry it once.  Solid and out-of-domain positions carry the wall pseudo-potentials.
 *   P^F:   the momentum flux the forcing of Eq. (shift) adds: the equilibria carry
 *          sum_l rho_l u_l u_l with u_l = u + tau F_l / rho_l, which exceeds rho u^(H) u^(H) (plus the
 *          terms of the viscous stress) by tau^2 sum_l F_l F_l / rho_l - F F / (4 rho), F_l the total
 *          force on component l (interaction and external), F = F_1 + F_2.
 * ====================================================================================== */

/* x or y component (comp 0 / 1) of u^(H) at neighbour (xn, yn) of fluid node (x, y), with the mirror
 * rule at a solid neighbour. */
static double u_neighbour(const orc_params* prm, const uint8_t* solid, const double* u, int comp, int x, int y,
                          int xn, int yn) {
  const int nx = prm->nx, ny = prm->ny;
  xn = wrap(xn, nx);
  if (prm->periodic_y) yn = wrap(yn, ny);
  const double own = u[(long)y * nx + x];
  if (yn < 0 || yn >= ny || solid[(long)yn * nx + xn]) {
    const double uw = comp == 0 ? wall_u(prm, yn) : 0.0;
    return 2.0 * uw - own;
  }
  return u[(long)yn * nx + xn];
}

int orc_stress(const orc_params* prm, const uint8_t* mask, const double* state, double* sxy, double* pint, double* row,
               double* out4) {
  if (!valid(prm)) return -1;
  const int nx = prm->nx, ny = prm->ny;
  const long N = (long)nx * ny;
  uint8_t* solid = (uint8_t*)malloc((size_t)N);
  double* buf = (double*)malloc(sizeof(double) * 13 * (size_t)N);
  double *rho1 = buf, *rho2 = buf + N, *T = buf + 2 * N, *ux = buf + 3 * N, *uy = buf + 4 * N;
  double* psit[2] = {buf + 5 * N, buf + 6 * N};
  double* psie[2] = {buf + 7 * N, buf + 8 * N};
  double* F = buf + 9 * N; /* [l][xy][N], Eqs. (FAB), (FintAttrattive), (FintRepulsive), (alphaG) */
  orc_solid_map(prm, mask, solid);
  fields_full(prm, solid, state, rho1, rho2, T, ux, uy);
  forces_from_fields(prm, solid, rho1, rho2, T, F);
  const double* rho[2] = {rho1, rho2};
  double psit_w[2], psie_w[2];
  for (int l = 0; l < 2; ++l) {
    for (long n = 0; n < N; ++n) {
      psit[l][n] = rho[l][n] / prm->rho0;
      psie[l][n] = psi_exp(rho[l][n], prm->rho0);
    }
    psit_w[l] = prm->rho_wall[l] / prm->rho0;
    psie_w[l] = psi_exp(prm->rho_wall[l], prm->rho0);
  }
  double sum_s = 0.0, sum_v = 0.0, sum_p = 0.0, sum_f = 0.0, nf = 0.0;
  for (int y = 0; y < ny; ++y) {
    double rs = 0.0, rn = 0.0;
    for (int x = 0; x < nx; ++x) {
      const long n = (long)y * nx + x;
      if (solid[n]) {
        if (sxy) sxy[n] = 0.0;
        if (pint) pint[n] = 0.0;
        continue;
      }
      /* bare viscous stress, Eq. (VISCO) with c_s^2 = 1/3 */
      const double eta0 = (rho1[n] + rho2[n]) * (prm->tau - 0.5) / 3.0;
      const double dvdx = 0.5 * (u_neighbour(prm, solid, uy, 1, x, y, x + 1, y) -
                                 u_neighbour(prm, solid, uy, 1, x, y, x - 1, y));
      const double dudy = 0.5 * (u_neighbour(prm, solid, ux, 0, x, y, x, y + 1) -
                                 u_neighbour(prm, solid, ux, 0, x, y, x, y - 1));
      const double visc = eta0 * (dvdx + dudy);
      /* pressure tensor of the interaction forces, virial form */
      double p = 0.0;
      for (int l = 0; l < 2; ++l) {
        const int m = 1 - l;
        double sx = 0.0, sa = 0.0, sr = 0.0;
        for (int i = 0; i < 9; ++i) { /* Eq. (FAB) and Eq. (FintAttrattive): NN links, weights w_i */
          const double cc = (double)(CX[i] * CY[i]);
          sx += weight_w(i) * field_at(prm, solid, psit[m], psit_w[m], x + CX[i], y + CY[i]) * cc;
          sa += weight_w(i) * field_at(prm, solid, psie[l], psie_w[l], x + CX[i], y + CY[i]) * cc;
        }
        for (int i = 0; i < 25; ++i) { /* Eq. (FintRepulsive): NN and NNN links, weights p_i */
          const double cc = (double)(CX[i] * CY[i]);
          sr += weight_p(i) * field_at(prm, solid, psie[l], psie_w[l], x + CX[i], y + CY[i]) * cc;
        }
        p += 0.5 * prm->G12 * psit[l][n] * sx;
        p += 0.5 * prm->Ga[l] * psie[l][n] * sa;
        p += 0.5 * prm->Gr[l] * psie[l][n] * sr;
      }
      /* forcing part, Eq. (shift) */
      double pf = 0.0;
      for (int l = 0; l < 2; ++l)
        pf += prm->tau * prm->tau * F[((long)l * 2 + 0) * N + n] * F[((long)l * 2 + 1) * N + n] / rho[l][n];
      const double Fx = F[0 * N + n] + F[2 * N + n], Fy = F[1 * N + n] + F[3 * N + n];
      pf -= Fx * Fy / (4.0 * (rho1[n] + rho2[n]));
      const double s = visc - p - pf;
      if (sxy) sxy[n] = s;
      if (pint) pint[n] = p;
      rs += s;
      rn += 1.0;
      sum_s += s;
      sum_v += visc;
      sum_p += p;
      sum_f += pf;
      nf += 1.0;
    }
    if (row) row[y] = rn > 0.0 ? rs / rn : 0.0;
  }
  if (out4) {
    out4[0] = nf > 0.0 ? sum_s / nf : 0.0;
    out4[1] = nf > 0.0 ? sum_v / nf : 0.0;
    out4[2] = nf > 0.0 ? sum_p / nf : 0.0;
    out4[3] = nf > 0.0 ? sum_f / nf : 0.0;
  }
  free(buf);
  free(solid);
  return 0;
}

/* ======================================================================================
 * Discrete adjoint (reverse mode) of the step and of the time-averaged Nusselt number
 * J = (1/N) sum_{t=1..N} Nu(S_t)  (Eq. NuTime), w.r.t. the initial temperature field and T_down.
 *
 * One reverse step maps lam_out = dJ/dS_{t+1} to lam_in = (dS_{t+1}/dS_t)^T lam_out + cJ dNu/dS_t,
 * following the forward step of orc_step backwards, one sweep per forward sub-step:
 *   streaming (+ bounce-back, anti-bounce-back) -> BGK collisions -> velocities (Eq. shift,
 *   u^(H)) -> forces (Eqs. FAB, FintAttrattive, FintRepulsive, alphaG) -> pseudo-potentials ->
 *   moments.  Solid and out-of-domain positions carry constants and receive no adjoint.
 * ====================================================================================== */

typedef struct {
  uint8_t* solid;
  double *rho1, *rho2, *jx, *jy, *T;
  double *psit[2], *psie[2];
  double *Fx[2], *Fy[2];
} orc_fwd;

static void fwd_free(orc_fwd* w) {
  free(w->solid);
  free(w->rho1);
  free(w->rho2);
  free(w->jx);
  free(w->jy);
  free(w->T);
  for (int l = 0; l < 2; ++l) {
    free(w->psit[l]);
    free(w->psie[l]);
    free(w->Fx[l]);
    free(w->Fy[l]);
  }
}

/* Forward intermediates of state S (moments, pseudo-potentials, forces per component). */
static void fwd_recompute(const orc_params* prm, const uint8_t* mask, const double* S, orc_fwd* w) {
  const long N = (long)prm->nx * prm->ny;
  w->solid = (uint8_t*)malloc((size_t)N);
  orc_solid_map(prm, mask, w->solid);
  w->rho1 = (double*)malloc(sizeof(double) * N);
  w->rho2 = (double*)malloc(sizeof(double) * N);
  w->jx = (double*)malloc(sizeof(double) * N);
  w->jy = (double*)malloc(sizeof(double) * N);
  w->T = (double*)malloc(sizeof(double) * N);
  moments(prm, w->solid, S, w->rho1, w->rho2, w->jx, w->jy, w->T);
  double* F = (double*)malloc(sizeof(double) * 4 * N);
  forces_from_fields(prm, w->solid, w->rho1, w->rho2, w->T, F);
  const double* rho[2] = {w->rho1, w->rho2};
  for (int l = 0; l < 2; ++l) {
    w->psit[l] = (double*)malloc(sizeof(double) * N);
    w->psie[l] = (double*)malloc(sizeof(double) * N);
    w->Fx[l] = (double*)malloc(sizeof(double) * N);
    w->Fy[l] = (double*)malloc(sizeof(double) * N);
    for (long n = 0; n < N; ++n) {
      w->psit[l][n] = w->solid[n] ? 0.0 : rho[l][n] / prm->rho0;
      w->psie[l][n] = w->solid[n] ? 0.0 : psi_exp(rho[l][n], prm->rho0);
      w->Fx[l][n] = F[((long)l * 2 + 0) * N + n];
      w->Fy[l][n] = F[((long)l * 2 + 1) * N + n];
    }
  }
  free(F);
}

/* Position (x, y) + c_k as a fluid node index, or -1 when it is solid or outside the domain. */
static long fluid_at(const orc_params* prm, const uint8_t* solid, int x, int y) {
  const int nx = prm->nx, ny = prm->ny;
  x = wrap(x, nx);
  if (prm->periodic_y)
    y = wrap(y, ny);
  else if (y < 0 || y >= ny)
    return -1;
  const long n = (long)y * nx + x;
  return solid[n] ? -1 : n;
}

/* d(sum_z dT/dy(z))/dT_down for the mirror rule of the Nu discretisation (geometry only). */
static double dB_dTdown_sum(const orc_params* prm, const uint8_t* solid) {
  const int nx = prm->nx, ny = prm->ny;
  double s = 0.0;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      if (solid[(long)y * nx + x]) continue;
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        int yy = y + sgn;
        if (prm->periodic_y) yy = wrap(yy, ny);
        if (solid[(long)yy * nx + x] && 2 * yy < ny) s += (double)sgn; /* d(T_up - T_dn)/2 / dT_w */
      }
    }
  return s;
}

int orc_adjoint_step(const orc_params* prm, const uint8_t* mask, const double* S, const double* lam_out, double cJ,
                     double* lam_in, double* dJ_dTdown) {
  if (!valid(prm)) return -1;
  const int nx = prm->nx, ny = prm->ny;
  const long N = (long)nx * ny;
  orc_fwd w;
  fwd_recompute(prm, mask, S, &w);
  const double tau = prm->tau, om = 1.0 / prm->tau, omg = 1.0 / prm->tau_g, rho0 = prm->rho0;
  double dTd = 0.0;

  /* Nusselt-number normalisation (Eq. NuTime) */
  double nf = 0.0;
  for (long n = 0; n < N; ++n) nf += w.solid[n] ? 0.0 : 1.0;
  const double kappa = (prm->tau_g - 0.5) / 3.0, dT = prm->T_down - prm->T_up, H = (double)(ny - 2);
  const int nu_defined = !prm->periodic_y && dT != 0.0 && nf > 0;
  const double D = kappa * dT / H;

  /* 1. reverse streaming: lam_star = adjoint of the post-collision populations */
  double* lam_star = (double*)calloc(27 * (size_t)N, sizeof(double));
  if (lam_out) {
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long n = (long)y * nx + x;
        if (w.solid[n]) continue;
        for (int i = 0; i < 9; ++i) {
          int xd = wrap(x + CX[i], nx), yd = y + CY[i];
          if (prm->periodic_y) yd = wrap(yd, ny);
          const long nd = (long)yd * nx + xd;
          if (!w.solid[nd]) {
            for (int c = 0; c < 3; ++c) lam_star[(long)(9 * c + i) * N + n] = lam_out[(long)(9 * c + i) * N + nd];
          } else {
            const int o = OPP[i];
            lam_star[(long)i * N + n] = lam_out[(long)o * N + n];
            lam_star[(long)(9 + i) * N + n] = lam_out[(long)(9 + o) * N + n];
            lam_star[(long)(18 + i) * N + n] = -lam_out[(long)(18 + o) * N + n];
            if (2 * yd < ny) dTd += 2.0 * weight_w(i) * lam_out[(long)(18 + o) * N + n];
          }
        }
      }
  }

  /* 2. collision and velocity adjoints, local to each fluid node */
  double* lFx[2];
  double* lFy[2];
  double* lrho[2];
  for (int l = 0; l < 2; ++l) {
    lFx[l] = (double*)calloc((size_t)N, sizeof(double));
    lFy[l] = (double*)calloc((size_t)N, sizeof(double));
    lrho[l] = (double*)calloc((size_t)N, sizeof(double));
  }
  double* ljx = (double*)calloc((size_t)N, sizeof(double));
  double* ljy = (double*)calloc((size_t)N, sizeof(double));
  double* lT = (double*)calloc((size_t)N, sizeof(double));
  memset(lam_in, 0, sizeof(double) * 27 * (size_t)N);
  for (long n = 0; n < N; ++n) {
    if (w.solid[n]) continue;
    const double r[2] = {w.rho1[n], w.rho2[n]};
    const double rho = r[0] + r[1];
    const double ux = w.jx[n] / rho, uy = w.jy[n] / rho;
    const double Fx = w.Fx[0][n] + w.Fx[1][n], Fy = w.Fy[0][n] + w.Fy[1][n];
    const double uHx = ux + Fx / (2.0 * rho), uHy = uy + Fy / (2.0 * rho);
    double lux = 0.0, luy = 0.0;
    for (int l = 0; l < 2; ++l) {
      const double ulx = ux + tau * w.Fx[l][n] / r[l], uly = uy + tau * w.Fy[l][n] / r[l];
      const double uu = ulx * ulx + uly * uly;
      double lulx = 0.0, luly = 0.0;
      for (int i = 0; i < 9; ++i) {
        const double ls = lam_star[(long)(9 * l + i) * N + n];
        lam_in[(long)(9 * l + i) * N + n] = (1.0 - om) * ls; /* f* = f + om (feq - f) */
        const double lfeq = om * ls;
        const double cu = CX[i] * ulx + CY[i] * uly;
        /* feq = w rho_l (1 + 3 cu + 4.5 cu^2 - 1.5 u^2) */
        lrho[l][n] += lfeq * weight_w(i) * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        lulx += lfeq * weight_w(i) * r[l] * (3.0 * CX[i] + 9.0 * cu * CX[i] - 3.0 * ulx);
        luly += lfeq * weight_w(i) * r[l] * (3.0 * CY[i] + 9.0 * cu * CY[i] - 3.0 * uly);
      }
      /* u_l = u + tau F_l / rho_l (Eq. shift) */
      lux += lulx;
      luy += luly;
      lFx[l][n] += tau * lulx / r[l];
      lFy[l][n] += tau * luly / r[l];
      lrho[l][n] += -tau * (w.Fx[l][n] * lulx + w.Fy[l][n] * luly) / (r[l] * r[l]);
    }
    /* thermal collision, g^eq(T, u^(H)) (Eq. Teq) */
    double luHx = 0.0, luHy = 0.0;
    const double uuH = uHx * uHx + uHy * uHy;
    for (int i = 0; i < 9; ++i) {
      const double ls = lam_star[(long)(18 + i) * N + n];
      lam_in[(long)(18 + i) * N + n] = (1.0 - omg) * ls;
      const double lgeq = omg * ls;
      const double cu = CX[i] * uHx + CY[i] * uHy;
      lT[n] += lgeq * weight_w(i) * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uuH);
      luHx += lgeq * weight_w(i) * w.T[n] * (3.0 * CX[i] + 9.0 * cu * CX[i] - 3.0 * uHx);
      luHy += lgeq * weight_w(i) * w.T[n] * (3.0 * CY[i] + 9.0 * cu * CY[i] - 3.0 * uHy);
    }
    /* Nu seed: d/dS of cJ (<u^(H)_y T> - kappa <dT/dy>) / D; the dT/dy part is handled below */
    if (cJ != 0.0 && nu_defined) {
      luHy += cJ * w.T[n] / (nf * D);
      lT[n] += cJ * uHy / (nf * D);
    }
    /* u^(H) = u + F / (2 rho) */
    lux += luHx;
    luy += luHy;
    for (int l = 0; l < 2; ++l) {
      lFx[l][n] += luHx / (2.0 * rho);
      lFy[l][n] += luHy / (2.0 * rho);
      lrho[l][n] += -(Fx * luHx + Fy * luHy) / (2.0 * rho * rho);
    }
    /* u = j / rho (Eq. velo) */
    ljx[n] += lux / rho;
    ljy[n] += luy / rho;
    for (int l = 0; l < 2; ++l) lrho[l][n] += -(w.jx[n] * lux + w.jy[n] * luy) / (rho * rho);
    /* external force rho_l (body_fx, alpha_g T) (Eq. alphaG) */
    for (int l = 0; l < 2; ++l) {
      lrho[l][n] += lFx[l][n] * prm->body_fx + lFy[l][n] * prm->alpha_g * w.T[n];
      lT[n] += lFy[l][n] * prm->alpha_g * r[l];
    }
  }

  /* Nu seed, the dT/dy term: d(sum_z dT/dy(z))/dT(x) with the mirror rule */
  if (cJ != 0.0 && nu_defined) {
    const double c = cJ * (-kappa) / (nf * D);
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long n = (long)y * nx + x;
        if (w.solid[n]) continue;
        for (int s = 0; s < 2; ++s) {
          const int sgn = s ? 1 : -1; /* neighbour above (+1) enters with +1/2, below with -1/2 */
          int yy = y + sgn;
          if (prm->periodic_y) yy = wrap(yy, ny);
          const long nn = (long)yy * nx + x;
          if (w.solid[nn])
            lT[n] += c * 0.5 * sgn * (-1.0); /* mirror value 2 T_w - T(x) */
          else
            lT[nn] += c * 0.5 * sgn;
        }
      }
    dTd += cJ * (-kappa * dB_dTdown_sum(prm, w.solid) / (nf * D));
    /* Nu depends on T_down through D as well: dNu/dD = -Nu / D, dD/dT_down = kappa / H */
    double obs[8];
    orc_observables(prm, mask, S, obs);
    dTd += cJ * (-obs[4] / dT);
  }

  /* 3. force adjoint: scatter dF_l(x)/dpsi(y) back to psi~ and psi at every fluid y */
  double* lpt[2];
  double* lpe[2];
  for (int l = 0; l < 2; ++l) {
    lpt[l] = (double*)calloc((size_t)N, sizeof(double));
    lpe[l] = (double*)calloc((size_t)N, sizeof(double));
  }
  const double psit_w[2] = {prm->rho_wall[0] / rho0, prm->rho_wall[1] / rho0};
  const double psie_w[2] = {psi_exp(prm->rho_wall[0], rho0), psi_exp(prm->rho_wall[1], rho0)};
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const long n = (long)y * nx + x;
      if (w.solid[n]) continue;
      for (int l = 0; l < 2; ++l) {
        const int m = 1 - l;
        const double ax = lFx[l][n], ay = lFy[l][n];
        /* F^x_l = -G12 psi~_l(x) sum_NN w_i psi~_m(x + c_i) c_i */
        double sx = 0.0, sy = 0.0;
        for (int i = 0; i < 9; ++i) {
          const double v = field_at(prm, w.solid, w.psit[m], psit_w[m], x + CX[i], y + CY[i]);
          sx += weight_w(i) * v * CX[i];
          sy += weight_w(i) * v * CY[i];
          const long nb = fluid_at(prm, w.solid, x + CX[i], y + CY[i]);
          if (nb >= 0) lpt[m][nb] += -prm->G12 * w.psit[l][n] * weight_w(i) * (CX[i] * ax + CY[i] * ay);
        }
        lpt[l][n] += -prm->G12 * (sx * ax + sy * ay);
        /* F^a_l + F^r_l = -psi_l(x) sum_k (G^a w_k + G^r p_k) psi_l(x + c_k) c_k */
        sx = sy = 0.0;
        for (int k = 0; k < 25; ++k) {
          const double a = prm->Ga[l] * (k < 9 ? weight_w(k) : 0.0) + prm->Gr[l] * weight_p(k);
          const double v = field_at(prm, w.solid, w.psie[l], psie_w[l], x + CX[k], y + CY[k]);
          sx += a * v * CX[k];
          sy += a * v * CY[k];
          const long nb = fluid_at(prm, w.solid, x + CX[k], y + CY[k]);
          if (nb >= 0) lpe[l][nb] += -w.psie[l][n] * a * (CX[k] * ax + CY[k] * ay);
        }
        lpe[l][n] += -(sx * ax + sy * ay);
      }
    }

  /* 4. pseudo-potentials to densities: psi~ = rho / rho0, psi = rho0 (1 - exp(-rho / rho0)) */
  const double* rho[2] = {w.rho1, w.rho2};
  for (long n = 0; n < N; ++n) {
    if (w.solid[n]) continue;
    for (int l = 0; l < 2; ++l) lrho[l][n] += lpt[l][n] / rho0 + lpe[l][n] * exp(-rho[l][n] / rho0);
  }

  /* 5. moments: rho_l = sum_i f_{l,i}, j = sum c_i f, T = sum_i g_i */
  for (long n = 0; n < N; ++n) {
    if (w.solid[n]) continue;
    for (int i = 0; i < 9; ++i) {
      for (int l = 0; l < 2; ++l) lam_in[(long)(9 * l + i) * N + n] += lrho[l][n] + CX[i] * ljx[n] + CY[i] * ljy[n];
      lam_in[(long)(18 + i) * N + n] += lT[n];
    }
  }

  if (dJ_dTdown) *dJ_dTdown += dTd;
  for (int l = 0; l < 2; ++l) {
    free(lFx[l]);
    free(lFy[l]);
    free(lrho[l]);
    free(lpt[l]);
    free(lpe[l]);
  }
  free(ljx);
  free(ljy);
  free(lT);
  free(lam_star);
  fwd_free(&w);
  return 0;
}

int orc_adjoint_run(const orc_params* prm, const uint8_t* mask, const double* rho1, const double* rho2,
                    const double* T0, long nsteps, double* J, double* dJ_dT0, double* dJ_dTdown) {
  if (!valid(prm) || nsteps < 1) return -1;
  const long N = (long)prm->nx * prm->ny;
  const size_t SZ = 27 * (size_t)N;
  double* states = (double*)malloc(sizeof(double) * SZ * (size_t)(nsteps + 1));
  if (!states) return -2;
  orc_init(prm, mask, rho1, rho2, T0, states);
  double sumNu = 0.0, obs[8];
  for (long t = 0; t < nsteps; ++t) {
    orc_step(prm, mask, states + (size_t)t * SZ, states + (size_t)(t + 1) * SZ);
    orc_observables(prm, mask, states + (size_t)(t + 1) * SZ, obs);
    sumNu += obs[4];
  }
  *J = sumNu / (double)nsteps;
  double* lam = (double*)calloc(SZ, sizeof(double));
  double* lam2 = (double*)calloc(SZ, sizeof(double));
  double dTd = 0.0;
  /* lam_N = (1/N) dNu/dS_N; lam_t = Phi'(S_t)^T lam_{t+1} + (1/N) dNu/dS_t; lam_0 = Phi'(S_0)^T lam_1 */
  orc_adjoint_step(prm, mask, states + (size_t)nsteps * SZ, NULL, 1.0 / (double)nsteps, lam, &dTd);
  for (long t = nsteps - 1; t >= 0; --t) {
    orc_adjoint_step(prm, mask, states + (size_t)t * SZ, lam, t >= 1 ? 1.0 / (double)nsteps : 0.0, lam2, &dTd);
    double* tmp = lam;
    lam = lam2;
    lam2 = tmp;
  }
  /* S_0: g_i = w_i T0 at fluid nodes */
  uint8_t* solid = (uint8_t*)malloc((size_t)N);
  orc_solid_map(prm, mask, solid);
  for (long n = 0; n < N; ++n) {
    double s = 0.0;
    if (!solid[n])
      for (int i = 0; i < 9; ++i) s += weight_w(i) * lam[(long)(18 + i) * N + n];
    dJ_dT0[n] = s;
  }
  *dJ_dTdown = dTd;
  free(solid);
  free(lam);
  free(lam2);
  free(states);
  return 0;
}
