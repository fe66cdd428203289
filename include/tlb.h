/*
 * tlb.h - C ABI of the GB300 (sm_103a) thermal two-component lattice
 * Boltzmann library: the per-time-step update of a 2D emulsion model
 * (TLBfind, arXiv 2109.12565, Sec. 2.1-2.3) on one GPU.
 *
 * Model (Sec. 2.1-2.3): two D2Q9 fluid components f_{l,i} (l = 1, 2) and
 * one D2Q9 thermal population g_i.  Per step, at every fluid node:
 *   rho_l = sum_i f_{l,i},  u = sum_{l,i} c_i f_{l,i} / (rho_1 + rho_2),
 *   T = sum_i g_i                                   (Sec. 2.1 moments, Sec. 2.3)
 *   F_l = F^x_l + F^a_l + F^r_l + F^ext_l            (Eqs. FAB, FintAttrattive,
 *         F^ext_l = rho_l alpha_g T e_y               FintRepulsive, alphaG)
 *   u_l = u + tau F_l / rho_l                        (Eq. shift)
 *   u^(H) = u + F / (2 rho),  F = F_1 + F_2          (text after Eq. NS)
 *   f*_{l,i} = f - (f - f^eq(rho_l, u_l)) / tau      (Eq. BGK)
 *   g*_i = g - (g - g^eq(T, u^(H))) / tau_g          (Eq. LBMg, Eq. Teq)
 *   f(x + c_i, t + 1) = f*(x, t)                     (Eq. LBM, streaming)
 * with psi~ = rho/rho0 in F^x and psi = rho0 (1 - exp(-rho/rho0)) in F^a, F^r.
 * A link that ends on a solid node bounces back half-way (Sec. 2.2, zero wall
 * velocity); the thermal population is anti-bounced to hold the wall at its
 * temperature: g_{-i}(x, t + 1) = -g*_i(x, t) + 2 w_i T_w.  Every solid or
 * out-of-domain position reached by a force stencil carries the wall
 * densities rho_wall (Sec. 2.2.1).
 *
 * Grid: nx * ny nodes, x fastest, x periodic.  periodic_y = 0: rows y = 0 and
 * y = ny - 1 are solid walls (hot bottom at T_down, cold top at T_up);
 * periodic_y = 1: fully periodic, no walls, no obstacle mask allowed.
 * An optional obstacle mask (host, nx * ny bytes, nonzero = solid) adds
 * solid nodes (rough-wall posts); a solid node in the lower half of the
 * lattice is at T_down, in the upper half at T_up.
 *
 * Memory: the caller owns the device workspace (size from
 * lb_workspace_size, 256-byte aligned) and the CUDA stream; the library owns
 * only its host-side handle and its CUDA graph objects.  Host arrays passed
 * to the library are read or written before the call returns.  Every call
 * returns one of the LB_* codes below; lb_last_error gives the text.
 * Nothing throws across this interface.
 */
#ifndef TLB_H
#define TLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LB_OK 0
#define LB_EINVAL (-1)      /* invalid argument or parameter */
#define LB_ENOSPACE (-2)    /* workspace too small or misaligned */
#define LB_ECUDA (-3)       /* a CUDA runtime call failed */
#define LB_ETIMEOUT (-4)    /* a bounded device-side wait ran out */
#define LB_EUNSTABLE (-5)   /* non-finite or non-positive density detected */

/* Storage precision of the populations. */
#define LB_FP64 0           /* FP64 populations, FP64 arithmetic */
#define LB_FP32_SHIFTED 1   /* FP32 deviations f - w_i rho_bar_l, g - w_i T_bar; FP32 arithmetic;
                               FP64 shift constants and FP64 reductions */
#define LB_FP32_FP16T 2     /* as LB_FP32_SHIFTED, but the thermal deviations g - w_i T_bar are stored in
                               FP16 (round to nearest on every store): 180 bytes of population traffic
                               per lattice update instead of 216 (not in the paper).  Single lattices
                               only: lb_batch_* and lb_adjoint* return LB_EINVAL for it. */
#define LB_DF64 3           /* populations stored as double-float pairs (hi, lo) of FP32 numbers, 8 bytes each (the
                               FP64 footprint), every operation in double-float arithmetic on the FP32 pipe
                               (error-free two-sum and two-product; a 48-bit significand); results within the
                               FP64 form's tolerance of the FP64 oracle (not in the paper).  lb_get_state /
                               lb_set_state convert to and from FP64.  Single lattices only: lb_batch_* and
                               lb_adjoint* return LB_EINVAL for it. */

typedef struct lb_params {
  int nx, ny;          /* lattice size including wall rows */
  int periodic_y;      /* 0: solid rows y = 0, ny-1; 1: periodic in y */
  int precision;       /* LB_FP64, LB_FP32_SHIFTED, LB_FP32_FP16T or LB_DF64 */
  double tau;          /* fluid relaxation time (> 1/2), Eq. BGK */
  double tau_g;        /* thermal relaxation time (> 1/2), Eq. LBMg */
  double rho0;         /* reference density of psi~ and psi (> 0) */
  double G12;          /* inter-component coupling, Eq. FAB */
  double Ga[2];        /* G^a_11, G^a_22 (attraction, < 0 in the paper), Eq. FintAttrattive */
  double Gr[2];        /* G^r_11, G^r_22 (repulsion, > 0), Eq. FintRepulsive */
  double rho_wall[2];  /* wall densities: component 1 (rho_w,max), component 2 (rho_w,min) */
  double T_down, T_up; /* bottom / top wall temperature */
  double alpha_g;      /* buoyancy alpha * g, Eq. alphaG */
  double body_fx;      /* constant x acceleration on both components (0 in the paper's runs) */
  double shift_rho[2]; /* FP32 forms: rho_bar_l; NaN = mean initial density of the fluid nodes */
  double shift_T;      /* FP32 forms: T_bar; NaN = (T_down + T_up) / 2 */
  double u_wall[2];    /* x velocity of the flat bottom / top wall (Couette rheology, Sec. 2.2 and 3.2.1):
                          a population bounced off a moving wall row gains 6 w_i rho_l c_ix u_wall
                          (mass-conserving); obstacle posts stay at rest.  0 = resting walls.  The
                          adjoint needs resting walls. */
} lb_params;

/* Observables of the current state S_t (pre-collision populations at step t). */
typedef struct lb_obs {
  double mass[2];      /* sum over fluid nodes of rho_l */
  double mom[2];       /* sum over fluid nodes of rho u^(H) */
  double Nu;           /* Nusselt number, Eq. NuTime: (<u^(H)_y T> - kappa <dT/dy>) / (kappa dT / H),
                          <.> over fluid nodes, dT/dy central with mirror 2 T_w - T at solid
                          neighbours, H = ny - 2, dT = T_down - T_up; 0 if periodic_y or dT = 0 */
  double E;            /* <|u^(H)|^2> over fluid nodes */
  long long step;      /* number of steps taken since lb_init / lb_set_state */
  long long n_fluid;   /* number of fluid nodes */
  long long n_bad;     /* fluid nodes with a non-finite or non-positive density or non-finite T */
  int status;          /* LB_OK, or LB_EUNSTABLE when n_bad > 0 */
  int _pad;
  double wall_fx[2];   /* x momentum the next step hands to the bottom / top wall row through its
                          bounce-back links, sum over both components of c_ix (f*_i + f_bounced): the
                          force of the fluid on each flat wall per time step; in a steady Couette
                          flow -wall_fx[1] / nx is the shear stress.  0 when periodic_y. */
} lb_obs;

typedef struct lb_handle lb_handle;

/* Bytes of device workspace lb_init needs for these parameters; has_mask != 0 when an obstacle
 * mask will be passed.  Returns LB_EINVAL on invalid parameters, among them lattices beyond the size
 * limits: nx * ny < 2^31, 27 * pitch * ny < 2^31 population slots per buffer, ny <= 65535. */
int lb_workspace_size(const lb_params* p, int has_mask, size_t* bytes);

/* Create a lattice on the current CUDA device.  rho1, rho2, T0: host arrays of nx*ny doubles (x
 * fastest) with the initial densities and temperature; the initial populations are the rest
 * equilibria f_{l,i} = w_i rho_l, g_i = w_i T0 at fluid nodes.  mask: host nx*ny bytes or NULL.
 * d_workspace: device memory of ws_bytes >= lb_workspace_size, 256-byte aligned, owned by the
 * caller and not touched by anyone else while the handle lives.  stream: cudaStream_t or NULL for
 * the legacy default stream; every later call is ordered on it.  Blocks until the state is on the
 * device.  Errors: LB_EINVAL (bad parameters, tau <= 1/2, non-positive initial density, mask with
 * periodic_y), LB_ENOSPACE, LB_ECUDA. */
int lb_init(lb_handle** h, const lb_params* p, const uint8_t* mask, const double* rho1, const double* rho2,
            const double* T0, void* d_workspace, size_t ws_bytes, void* stream);

/* Advance n >= 0 time steps.  Asynchronous on the handle's stream (CUDA-graph replay of one fused
 * kernel per step). */
int lb_step(lb_handle* h, int n);

/* Observables of the current state.  Synchronises the stream; returns LB_EUNSTABLE (with *out
 * filled) when any fluid node has a non-finite or non-positive density. */
int lb_observables(lb_handle* h, lb_obs* out);

/* Hydrodynamic fields of the current state into host arrays of nx*ny doubles (any may be NULL):
 * rho1, rho2, T, u^(H)_x, u^(H)_y.  Solid nodes report rho_wall, the wall temperature and zero
 * velocity.  Synchronous. */
int lb_get_fields(lb_handle* h, double* rho1, double* rho2, double* T, double* ux, double* uy);

/* Copy the populations of S_t to / from host memory as 27 planes of nx*ny doubles (planes 0-8
 * f_{1,i}, 9-17 f_{2,i}, 18-26 g_i, D2Q9 order (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1)
 * (-1,-1) (1,-1)); solid nodes read as 0 and are ignored on write.  In the FP32 forms the
 * stored deviations are converted to full populations (lb_set_state rounds them to the storage
 * precision).  bytes must equal 27*nx*ny*8.
 * lb_set_state resets the step counter.  Synchronous. */
int lb_get_state(lb_handle* h, double* host, size_t bytes);
int lb_set_state(lb_handle* h, const double* host, size_t bytes);

/* Total shear stress of the current state: the stress of the rheology experiment (Sec. 2.1, text
 * after Eq. NS: the bare viscous stress supplemented by the pressure tensor; Sec. 3.2.1: its space and
 * time average is the stress Sigma of the flow curve, its x-wise average the Pxy_av profile).  At every
 * fluid node
 *   sigma_xy = eta_0 (d_x u^(H)_y + d_y u^(H)_x) - P^int_xy - P^F_xy,  eta_0 = rho (tau - 1/2) / 3 (Eq. VISCO),
 * with central differences (a solid neighbour takes the mirror value 2 u_w - u: u_w = u_wall along x for
 * a flat wall row, 0 otherwise), P^int_xy the virial form of the interaction forces of Eqs. FAB,
 * FintAttrattive, FintRepulsive (half of every pair term times c_ix c_iy) and
 * P^F_xy = tau^2 sum_l F_lx F_ly / rho_l - F_x F_y / (4 rho) the momentum flux of the forcing of Eq. shift
 * (F_l the total force on component l).  In a steady shear the space-time average of sigma_xy balances
 * the wall stress (wall_fx of lb_obs).  All arithmetic in FP64 from the fields of lb_get_fields.
 * out4 (host, 4 doubles or NULL): means over the fluid nodes of sigma_xy, of the viscous part, of
 * P^int_xy and of P^F_xy.  row (host, ny doubles or NULL): per row, the mean of sigma_xy over the row's
 * fluid nodes (0 for a row without any).  field (host, nx*ny doubles or NULL): sigma_xy, 0 at solid
 * nodes.  Uses the inactive buffer as staging; synchronous.  LB_EINVAL when all three are NULL. */
int lb_stress(lb_handle* h, double* out4, double* row, double* field);

/* Tile-shape autotuner of the fused step (not in the paper).  Times every step-kernel tile
 * candidate of the handle's precision over `launches` launches on the handle's stream and keeps the
 * fastest for later lb_step calls.  Each trial reads the current state and writes the inactive
 * buffer, so the state and the step counter do not change.  chosen (may be NULL) receives the
 * winning candidate; ms_per_candidate (may be NULL, n_slots entries) the mean milliseconds per
 * launch of each candidate.  Synchronous. */
int lb_autotune(lb_handle* h, int launches, int* chosen, double* ms_per_candidate, int n_slots);

/* The same autotuner for runs whose state does not stay in L2 between steps (not in the paper).
 * Before each timed launch it writes the first half of the caller's device buffer d_scratch and reads
 * the second half (give at least twice the L2 size, 16-byte aligned; its contents are overwritten),
 * so every trial starts with the populations evicted and L2 holding clean lines; only the launches
 * are timed.  Returns LB_EINVAL without a scratch buffer.  The state and the step counter do not
 * change.  Synchronous. */
int lb_autotune_cold(lb_handle* h, int launches, void* d_scratch, size_t scratch_bytes, int* chosen,
                     double* ms_per_candidate, int n_slots);

/* Use tile candidate `candidate` for later lb_step calls (LB_EINVAL if out of range). */
int lb_set_tile(lb_handle* h, int candidate);

/* Shape of tile candidate `candidate` (-1: the current one): tile width tx, height ty and threads
 * per CTA.  Returns the number of candidates (>= 1) or LB_EINVAL. */
int lb_tile_info(const lb_handle* h, int candidate, int* tx, int* ty, int* threads);

/* Observables of a state held in the caller's own device memory, for callers that cannot
 * allocate device memory (no cudaMalloc, no workspace): e.g. a plug-in whose host application owns
 * every device allocation, or a real-time loop that must not take the device-wide synchronisation
 * of cudaMalloc / cudaFree.  The paper has no counterpart; it is the lb_observables reduction with
 * its scratch moved into a fixed device array inside the library.
 * p: parameters (precision is ignored: the state is FP64).  d_state: device array of 27*nx*ny
 * doubles in the layout of lb_get_state (27 unpadded planes, x fastest).  d_mask: device nx*ny
 * bytes or NULL, as the mask given to lb_init.  out: host struct, filled before return (step = 0).
 * stream: cudaStream_t or NULL; the call synchronises it.
 * Scratch: a 2 MiB file-scope device array that every GPU loading the library holds until exit;
 * lattices needing more than 21,844 tiles of 32 x 16 nodes are rejected with LB_EINVAL before any
 * launch (4096 x 2720 fits, 4096 x 2736 does not).  With CUDA's lazy module loading the array is
 * created by the first call on a device, so make one warm-up call at initialisation, before any
 * stream capture; later calls allocate nothing.  Every call looks the array's device address up
 * afresh (cudaGetSymbolAddress), so a device reset between calls is harmless.  All calls on a device
 * share the array: calls that overlap on the GPU race and must be serialised by the caller.
 * Returns LB_OK, LB_EUNSTABLE (out filled), LB_EINVAL (bad parameters, d_state not 8-byte aligned,
 * lattice too large) or LB_ECUDA; lb_last_error is not updated. */
int lb_observables_static(const lb_params* p, const double* d_state, const uint8_t* d_mask, lb_obs* out,
                          void* stream);

/* ---- Adjoint (not in the paper): reverse-mode gradient of the time-averaged Nusselt number
 * J = (1/N) sum_{t=1..N} Nu(S_t) (Nu of Eq. NuTime) with respect to the initial temperature field T0
 * and the bottom-wall temperature T_down, by the discrete adjoint of the fused step. */

/* Storage layout of the handle's populations (also the layout of adjoint vectors): 27 planes of
 * pitch * ny elements of elem_bytes (8: LB_FP64, 4: LB_FP32_SHIFTED), x fastest.  LB_EINVAL for
 * LB_FP32_FP16T, whose planes do not share one element size. */
int lb_state_layout(const lb_handle* h, int* pitch, size_t* plane_elems, int* elem_bytes);

/* Device workspace bytes lb_adjoint needs for n_steps steps with a checkpoint every ckpt_every steps
 * (about (n_steps / ckpt_every + ckpt_every + 3) states; ckpt_every ~ sqrt(n_steps) minimises it).
 * lb_adjoint_step needs lb_adjoint_workspace_size(h, 1, 1). */
int lb_adjoint_workspace_size(const lb_handle* h, int n_steps, int ckpt_every, size_t* bytes);

/* One reverse step at the handle's current state S_t:
 *   d_lam = (dS_{t+1}/dS_t)^T d_lam_next + cJ dNu(S_t)/dS_t
 * d_lam_next (NULL = 0) and d_lam: device vectors in the lb_state_layout layout and precision.
 * *dJ_dTdown (host, may be NULL) receives d_lam_next . dS_{t+1}/dT_down + cJ dNu(S_t)/dT_down.
 * Synchronous. */
int lb_adjoint_step(lb_handle* h, const void* d_lam_next, void* d_lam, double cJ, void* d_adj_ws, size_t adj_bytes,
                    double* dJ_dTdown);

/* Treat the handle's current state as S_0 (the rest equilibrium of lb_init, g_i = w_i T0), run
 * n_steps steps computing Nu after each, then the reverse sweep with sqrt-N checkpointing: every
 * ckpt_every steps the state is stored; each segment is recomputed from its checkpoint and swept
 * backwards.  J (host) receives the time-averaged Nu; dJ_dT0 (host nx*ny doubles, 0 at solid
 * nodes) and dJ_dTdown (host) the gradient; with both NULL only J is computed.  The handle ends at
 * S_{n_steps}.  d_adj_ws: caller-owned device memory of lb_adjoint_workspace_size bytes.
 * Synchronous. */
int lb_adjoint(lb_handle* h, int n_steps, int ckpt_every, void* d_adj_ws, size_t adj_bytes, double* J, double* dJ_dT0,
               double* dJ_dTdown);

/* Phase times of the last full lb_adjoint call of this thread (CUDA events on the handle's stream):
 * out4[0] forward pass (steps + Nu) ms, out4[1] segment recomputation ms, out4[2] reverse sweep
 * (adjoint steps) ms, out4[3] number of adjoint steps. */
int lb_adjoint_timing(double* out4);

/* ---- Batched ensembles (not in the paper): n independent lattices, each with its own lb_params
 * (size, couplings, Rayleigh number, precision equal for all), obstacle mask and state, advanced
 * together by one launch per step or by one persistent launch per K steps.  Every replica runs the
 * same fused step as lb_step; results are bit-identical to n separate handles. */
typedef struct lb_batch lb_batch;

/* Device workspace bytes for n replicas; has_mask[r] != 0 when replica r has a mask (may be NULL). */
int lb_batch_workspace_size(const lb_params* reps, int n, const int* has_mask, size_t* bytes);

/* Create a batch.  masks[r] (host nx*ny bytes, or NULL; masks itself may be NULL), rho1[r],
 * rho2[r], T0[r] (host nx*ny doubles): as in lb_init for each replica.  d_workspace: caller-owned,
 * 256-byte aligned, >= lb_batch_workspace_size.  Starts with schedule 0 and tile candidate 0.
 * Synchronous. */
int lb_batch_init(lb_batch** b, const lb_params* reps, int n, const uint8_t* const* masks, const double* const* rho1,
                  const double* const* rho2, const double* const* T0, void* d_workspace, size_t ws_bytes, void* stream);

/* Advance every replica by n >= 0 steps, asynchronously.  Schedule 0: CUDA-graph replay of one
 * launch per step over all (replica, tile) items.  Schedule 1: cooperative persistent launches of
 * steps_per_launch steps each (graph-captured when the driver allows it); between steps every CTA
 * meets the others at a grid-wide barrier whose waits are bounded; a wait that runs out is reported
 * as LB_ETIMEOUT by the next lb_batch_sync / lb_batch_observables / lb_batch_get_*, and the state is
 * then invalid. */
int lb_batch_step(lb_batch* b, int n);

/* Choose the schedule (0 per-step, 1 persistent), the tile candidate and the steps per persistent
 * launch (even, >= 2). */
int lb_batch_configure(lb_batch* b, int schedule, int tile, int steps_per_launch);

/* Autotuner: runs every (schedule, tile) pair for 2 * trial_steps real steps (the state advances;
 * steps_taken receives the total), times the second half with CUDA events and keeps the fastest.
 * ms (may be NULL) receives the milliseconds per step of pair (schedule s, tile t) at s * ntiles + t
 * (n_slots >= 2 * ntiles). */
int lb_batch_autotune(lb_batch* b, int trial_steps, int* schedule, int* tile, long long* steps_taken, double* ms,
                      int n_slots);

/* Current work-list size, persistent grid, schedule, tile and whether graphs are in use; returns the
 * number of tile candidates. */
int lb_batch_info(const lb_batch* b, int* n_items, int* grid, int* schedule, int* tile, int* graphs);

/* Per-replica observables, fields and state, as lb_observables / lb_get_fields / lb_get_state. */
int lb_batch_observables(lb_batch* b, int replica, lb_obs* out);
int lb_batch_get_fields(lb_batch* b, int replica, double* rho1, double* rho2, double* T, double* ux, double* uy);
int lb_batch_get_state(lb_batch* b, int replica, double* host, size_t bytes);

/* Total shear stress of replica r, as lb_stress. */
int lb_batch_stress(lb_batch* b, int replica, double* out4, double* row, double* field);

/* Wait for the batch's stream; LB_ETIMEOUT if a persistent wait ran out. */
int lb_batch_sync(lb_batch* b);

/* Test hook for failure detection: sets the SM-clock budget of every persistent wait (default 4e9
 * cycles, about 2 s) and, when withhold_item >= 0, makes CTA number withhold_item (modulo the
 * persistent grid) leave before the first step barrier, so the other CTAs' bounded waits run out and
 * the launch ends with LB_ETIMEOUT instead of hanging. */
int lb_batch_set_wait_budget(lb_batch* b, long long cycles, int withhold_item);

void lb_batch_destroy(lb_batch* b);
const char* lb_batch_last_error(const lb_batch* b);

/* Wait for all work of the handle and report any asynchronous CUDA error. */
int lb_sync(lb_handle* h);

/* Release the handle and its graphs (not the caller's workspace or stream). */
void lb_destroy(lb_handle* h);

/* Text of the last error on this handle, or of the last failed lb_init / lb_workspace_size of
 * this thread when h is NULL.  Never NULL. */
const char* lb_last_error(const lb_handle* h);

/* Library version string. */
const char* lb_version(void);

/* ---- Droplet topology (Sec. 2.4, "Delaunay triangulation"; run between steps, not part of the
 * step).  Definitions:
 *   D1  a droplet node is a fluid node with rho_1 > threshold (the paper's bubble threshold B_th);
 *   D2  droplet nodes connect through the 4 nearest neighbours, x periodic, y periodic when
 *       periodic_y;
 *   D3  droplets are numbered 0, 1, ... in the order of their smallest node index y * nx + x;
 *   D4  the centre of a droplet is the plain mean of its node coordinates, unwrapped relative to
 *       its smallest node (offsets in (-nx/2, nx/2], likewise y when periodic), wrapped into the
 *       lattice;
 *   D5  the digital Voronoi colour of a fluid node is the id of the nearest centre (double
 *       precision, minimum image, ties to the smaller id); solid nodes are -1;
 *   D6  links: each 2 x 2 window of fluid nodes where three colours meet links the three pairs;
 *       where four meet, the four pairs of neighbouring corners (the sides, not the diagonals).
 * Results stay in a caller-owned device workspace; every result is independent of thread
 * scheduling. */

/* Device bytes of one droplet workspace for at most max_drops droplets (at most 16 * max_drops links,
 * 32 per droplet). */
int lb_droplets_workspace_size(const lb_handle* h, int max_drops, size_t* bytes);

/* Analyse the current state into d_ws (256-byte aligned, ws_bytes from lb_droplets_workspace_size
 * with the same max_drops): labels, centres, Voronoi colours, links.  *n_drops, *n_links (may be
 * NULL) receive the counts.  LB_ENOSPACE when there are more droplets than max_drops or a droplet
 * has more than 32 Voronoi neighbours.  Uses the handle's inactive buffer as staging; synchronous
 * (one read of the workspace header at the end).  The launches are captured into a CUDA graph the
 * first time a (d_ws, max_drops, threshold, current buffer) combination is seen and replayed after
 * that; the handle keeps four such graphs and frees them in lb_destroy.  Not to be called while the
 * handle's stream is being captured. */
int lb_droplets(lb_handle* h, double threshold, int max_drops, void* d_ws, size_t ws_bytes, int* n_drops,
                int* n_links);

/* Copy results of lb_droplets to host arrays (any may be NULL): centres cx, cy and node counts
 * size (n_drops each), links (2 * n_links ints: pairs a < b, ascending), label and color (nx * ny
 * ints, x fastest: droplet id / -1, Voronoi colour / -1).  Synchronous. */
int lb_droplets_get(lb_handle* h, const void* d_ws, size_t ws_bytes, double* cx, double* cy, long long* size,
                    int* links, int* label, int* color);

/* Droplet Nusselt number (Eq. NuDrops) of every droplet of an analysis of the CURRENT state (run
 * lb_droplets first, without stepping in between): (u_y T - kappa dT/dy) / (kappa Delta T / H) at the
 * node nearest to the centre (x rounded half up, periodic; y rounded half up), u_y = u^(H)_y, dT/dy
 * central with the mirror 2 T_w - T at a solid neighbour, kappa = (tau_g - 1/2) / 3, H = ny - 2.  nu:
 * host array of n_drops doubles; 0 when periodic_y or T_down = T_up, NaN when the nearest node is
 * solid.  Synchronous. */
int lb_droplets_nusselt(lb_handle* h, const void* d_ws, size_t ws_bytes, double* nu);

/* Plastic (T1) events between two analyses of this lattice (Sec. 2.4, diagonal flip of a
 * quadrilateral): a droplet of the later analysis matches one of the earlier when each is the
 * other's nearest centre within d_max.  Broken links: earlier links whose matched ends are no
 * longer linked; arising links: later links (in earlier ids) that were not links; a T1 event is
 * a broken link (a, b) with an arising link (c, d) such that c and d were linked to both a and b.
 * counts4 = {matched, broken, arising, t1}; broken and arising receive up to cap pairs (earlier
 * ids), t1 up to cap quadruples (a, b, c, d); all may be NULL.  d_scratch: device scratch; when
 * too small, LB_ENOSPACE with counts4[0] = KiB needed.  Synchronous. */
int lb_droplets_compare(lb_handle* h, const void* d_ws_prev, const void* d_ws_now, size_t ws_bytes, double d_max,
                        void* d_scratch, size_t scratch_bytes, int* counts4, int* broken, int* arising, int* t1,
                        int cap);

#ifdef __cplusplus
}
#endif
#endif
