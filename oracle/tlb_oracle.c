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

int orc_step(const orc_params* prm, const uint8_t* mask, const double* in, double* out) {
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
          const int o = OPP[i];
          out[(long)o * N + n] = fpost[i];
          out[(long)(9 + o) * N + n] = fpost[9 + i];
          out[(long)(18 + o) * N + n] = -fpost[18 + i] + 2.0 * weight_w(i) * wall_T(prm, yd);
        }
      }
    }
  }
  free(buf);
  free(solid);
  return 0;
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
