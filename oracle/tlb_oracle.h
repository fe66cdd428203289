/*
 * Plain FP64 CPU oracle of the thermal two-component Shan-Chen lattice
 * Boltzmann step (TLBfind, arXiv 2109.12565, Sections 2.1-2.3 and 3.3.2).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously correct
 * statement of the method that the CUDA library is checked against.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or constant with the CUDA
 * library, and the library never calls it.
 *
 * Conventions (shared with the library only through the documented ABI
 * semantics, not through code):
 *   - lattice nx * ny, x fastest: node (x, y) has index y*nx + x;
 *   - x is periodic; y is periodic when periodic_y != 0, otherwise rows
 *     y = 0 and y = ny-1 are solid walls (bounce-back walls half-way between
 *     the wall row and the first fluid row);
 *   - an optional obstacle mask (nx*ny bytes, nonzero = solid) adds solid
 *     nodes (rough-wall posts);
 *   - the state holds the PRE-collision populations f(t) of Eq. (LBM):
 *     27 planes of nx*ny doubles, planes 0-8 = f_{1,i}, 9-17 = f_{2,i},
 *     18-26 = g_i (Eq. LBMg); solid nodes hold 0.
 *   - D2Q9 order: 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1),
 *     6 (-1,1), 7 (-1,-1), 8 (1,-1); links 9-24 are the 16 next-to-nearest
 *     neighbours of Fig. 1 (|c|^2 = 4, 5, 8).
 *
 * Parity pins: every function here is pinned by the CPU tests in
 * tests/test_oracle_*.py (closed forms, conservation laws, the Appendix B
 * phase-separation table, Poiseuille, conduction, Laplace, wave decay,
 * convective onset).
 */
#ifndef TLB_ORACLE_H
#define TLB_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
  int nx, ny;
  int periodic_y;
  int _pad;
  double tau;       /* fluid relaxation time, Eq. (BGK) */
  double tau_g;     /* thermal relaxation time, Eq. (LBMg) */
  double rho0;      /* reference density of both pseudo-potentials */
  double G12;       /* cross coupling, Eq. (FAB) */
  double Ga[2];     /* G^a_11, G^a_22, Eq. (FintAttrattive) */
  double Gr[2];     /* G^r_11, G^r_22, Eq. (FintRepulsive) */
  double rho_wall[2]; /* wall densities rho_w,max (component 1), rho_w,min (component 2), Sec. 2.2.1 */
  double T_down, T_up; /* bottom / top wall temperatures, Sec. 3.2.3 */
  double alpha_g;   /* buoyancy coefficient alpha*g, Eq. (alphaG) */
  double body_fx;   /* constant x-acceleration (Poiseuille pin only; 0 in the paper's runs) */
  double u_wall[2]; /* x velocity of the bottom / top flat wall (Couette, Sec. 2.2); posts rest */
} orc_params;

/* Velocity tables: c[25][2], w[9] (D2Q9 weights), p[25] (two-belt weights of Fig. 1b). */
void orc_tables(int* c, double* w, double* p);

/* Effective solid map: obstacle mask (may be NULL) united with the wall rows. */
int orc_solid_map(const orc_params* prm, const uint8_t* mask, uint8_t* solid);

/* Initial populations at rest: f_{l,i} = w_i rho_l, g_i = w_i T (fluid nodes). */
int orc_init(const orc_params* prm, const uint8_t* mask, const double* rho1, const double* rho2,
             const double* T, double* state);

/* Interaction + external forces F_l (Eqs. FAB, FintAttrattive, FintRepulsive, alphaG) from density
 * fields rho1, rho2 and temperature T (fluid nodes; solid nodes ignored).  F is [2 comps][2 xy][nx*ny]. */
int orc_forces(const orc_params* prm, const uint8_t* mask, const double* rho1, const double* rho2,
               const double* T, double* F);

/* One time step S_t -> S_{t+1}: moments, pseudo-potentials, forces, shifted velocities, BGK
 * collision, streaming with half-way bounce-back (fluid) and anti-bounce-back (thermal). */
int orc_step(const orc_params* prm, const uint8_t* mask, const double* in, double* out);

/* x momentum that the step from S_t hands to the bottom (out[0]) and top (out[1]) flat walls through
 * their bounce-back links, sum over both components of c_ix (f*_i + f_bounced); the force of the fluid
 * on each wall per time step.  0 when periodic in y. */
int orc_wall_force(const orc_params* prm, const uint8_t* mask, const double* state, double* out);

/* nsteps steps in place; work must hold 27*nx*ny doubles. */
int orc_run(const orc_params* prm, const uint8_t* mask, double* state, double* work, long nsteps);

/* Hydrodynamic fields of state S_t: rho1, rho2, T, u^(H)_x, u^(H)_y (each nx*ny).  Solid nodes
 * report rho_w, the wall temperature and zero velocity. */
int orc_fields(const orc_params* prm, const uint8_t* mask, const double* state, double* rho1,
               double* rho2, double* T, double* ux, double* uy);

/* Observables of S_t: out[0..1] mass per component, out[2..3] momentum sum rho u^(H),
 * out[4] Nusselt number Eq. (NuTime), out[5] kinetic energy <|u^(H)|^2>, out[6] number of fluid
 * nodes with a non-finite or non-positive density, out[7] number of fluid nodes. */
int orc_observables(const orc_params* prm, const uint8_t* mask, const double* state, double* out);

/* Total shear stress of S_t (Sec. 2.1 after Eq. NS, Sec. 3.2.1): at every fluid node
 * sigma_xy = eta_0 (d_x u^(H)_y + d_y u^(H)_x) - P^int_xy - P^F_xy, eta_0 = rho (tau - 1/2) / 3
 * (Eq. VISCO), central differences with the mirror 2 u_w - u at a solid neighbour, P^int_xy the virial
 * form of the interaction forces (half of every pair term of Eqs. FAB, FintAttrattive, FintRepulsive
 * times c_ix c_iy), P^F_xy = tau^2 sum_l F_lx F_ly / rho_l - F_x F_y / (4 rho) the momentum flux of the
 * forcing of Eq. shift.  sxy (sigma_xy), pint (P^int_xy) (nx*ny, 0 at solid nodes) and row (ny: mean
 * of sigma_xy over the row's fluid nodes, the x-wise average) may be NULL; out4 (may be NULL): means
 * over fluid nodes of sigma_xy, of the viscous part, of P^int_xy and of P^F_xy. */
int orc_stress(const orc_params* prm, const uint8_t* mask, const double* state, double* sxy, double* pint,
               double* row, double* out4);

/* Discrete adjoint of one step (reverse mode): lam_in = (dS_{t+1}/dS_t)^T lam_out + cJ dNu(S_t)/dS_t,
 * where S is the state S_t and lam_out (may be NULL = 0) the adjoint of S_{t+1}; all in the state
 * layout.  *dJ_dTdown (may be NULL) is incremented by lam_out . dS_{t+1}/dT_down + cJ dNu(S_t)/dT_down. */
int orc_adjoint_step(const orc_params* prm, const uint8_t* mask, const double* S, const double* lam_out, double cJ,
                     double* lam_in, double* dJ_dTdown);

/* J = (1/N) sum_{t=1..N} Nu(S_t) from the rest-equilibrium start of (rho1, rho2, T0), and its gradient
 * with respect to the initial temperature field (dJ_dT0, nx*ny, 0 at solid nodes) and to T_down,
 * by storing every state and running the reverse sweep. */
int orc_adjoint_run(const orc_params* prm, const uint8_t* mask, const double* rho1, const double* rho2,
                    const double* T0, long nsteps, double* J, double* dJ_dT0, double* dJ_dTdown);

/* ---- Droplet topology (Sec. 2.4; definitions D1-D6 in tlb_droplets.c). ---- */

/* label[n]: droplet id of node n (ids in the order of each droplet's smallest node index) or -1
 * (solid, or rho1 <= threshold); *n_drops: number of droplets. */
int orc_droplet_labels(const orc_params* prm, const uint8_t* mask, const double* rho1, double threshold, int* label,
                       int* n_drops);

/* Centre of every droplet (plain mean of its node coordinates, periodic unwrapping relative to its
 * smallest node) and its node count (size may be NULL). */
int orc_droplet_centres(const orc_params* prm, const int* label, int n_drops, double* cx, double* cy,
                        long long* size);

/* Digital Voronoi tessellation: color[n] = id of the nearest centre (ties: smaller id), -1 at solid
 * nodes. */
int orc_digital_voronoi(const orc_params* prm, const uint8_t* mask, const double* cx, const double* cy, int n_drops,
                        int* color);

/* Delaunay links read off the 2 x 2 windows where three or four Voronoi colours meet: sorted unique
 * pairs (a < b) into links[2 * max_links] (may be NULL to count only); returns -3 when more than
 * max_links exist (*n_links is still the full count). */
int orc_voronoi_links(const orc_params* prm, const int* color, int* links, long max_links, long* n_links);

#ifdef __cplusplus
}
#endif
#endif
