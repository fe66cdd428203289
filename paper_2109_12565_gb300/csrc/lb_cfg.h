// Internal launch configuration of the CUDA library (host and device view).
// Every constant the fused step needs is precomputed on the host in FP64 and
// passed by value; the FP32 kernels round them once.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tlb {

// MODE_STEP_NU: a step that also sums u^(H)_y T over the fluid nodes of its input state, one partial
// per warp (the Nusselt number's advective part, Eq. NuTime), for the adjoint's forward pass.
enum Mode : int { MODE_STEP = 0, MODE_OBS = 1, MODE_FIELDS = 2, MODE_STEP_NU = 3, MODE_RHO1 = 4 };
__host__ __device__ constexpr bool mode_needs_T(int m) { return m == MODE_OBS || m == MODE_FIELDS; }
__host__ __device__ constexpr bool mode_steps(int m) { return m == MODE_STEP || m == MODE_STEP_NU; }

// Number of doubles each block writes to the partial-sum buffer in MODE_OBS.
constexpr int kObsSlots = 12;
// Final observable vector written by the reduction kernel.
constexpr int kObsOut = 16;

struct StepCfg {
  int nx, ny;           // lattice
  int pitch;            // elements per stored row (>= nx, rows 128-byte aligned)
  int periodic_y;
  long long plane;      // elements per population plane = pitch * ny
  const uint8_t* mask;  // device obstacle mask (nx * ny, unpadded) or nullptr
  double tau;           // tau (velocity shift, Eq. shift)
  double inv_tau, inv_tau_g;
  double rho0, inv_rho0;
  double gx;            // G12 / rho0^2: Eq. FAB written on rho instead of psi~ = rho / rho0
  // Self-interaction weights per shell, G^a w_i + G^r p_i (Eqs. FintAttrattive + FintRepulsive),
  // for |c|^2 = 1, 2 and twice the weight for |c|^2 = 4, 8 (those links have |c_x| or |c_y| = 2).
  double a1[2], a2[2], a4x2[2], a5[2], a8x2[2];
  double rho_w[2], psi_w[2];  // wall densities and their exp pseudo-potentials
  double T_down, T_up;
  double alpha_g, body_fx;
  double rho_bar[2], T_bar;   // storage shifts (0 in FP64)
  double kappa;               // (tau_g - 1/2) / 3, Eq. K
  double H;                   // wall-to-wall height ny - 2
  double u_wall[2];           // x velocity of the bottom / top flat wall rows (Couette)
};

// Tile shapes (nodes per CTA in x and y; threads per CTA = TX * BY).
template <class S> struct Tile;
template <> struct Tile<double> { static constexpr int TX = 32, TY = 16, BY = 8; };
template <> struct Tile<float> { static constexpr int TX = 64, TY = 16, BY = 4; };

inline dim3 grid_for(int nx, int ny, int tx, int ty) {
  return dim3((unsigned)((nx + tx - 1) / tx), (unsigned)((ny + ty - 1) / ty), 1u);
}

// ---- launchers (one translation unit per storage precision) ----
// mode MODE_STEP: fin -> fout;  MODE_OBS: aux = per-block partials (kObsSlots doubles each);
// MODE_FIELDS: aux = 5 planes of nx*ny doubles (rho1, rho2, T, ux, uy); MODE_RHO1: aux = the rho1
// plane alone, the same values (fout unused).
cudaError_t launch_f64(int mode, const StepCfg& c, const void* fin, void* fout, double* aux, cudaStream_t s);
cudaError_t launch_f32(int mode, const StepCfg& c, const void* fin, void* fout, double* aux, cudaStream_t s);
cudaError_t launch_f32h(int mode, const StepCfg& c, const void* fin, void* fout, double* aux, cudaStream_t s);
cudaError_t launch_df64(int mode, const StepCfg& c, const void* fin, void* fout, double* aux, cudaStream_t s);
// Initial rest equilibria from 3 planes (rho1, rho2, T) of nx*ny doubles.
cudaError_t init_f64(const StepCfg& c, const double* fields, void* buf, cudaStream_t s);
cudaError_t init_f32(const StepCfg& c, const double* fields, void* buf, cudaStream_t s);
cudaError_t init_f32h(const StepCfg& c, const double* fields, void* buf, cudaStream_t s);
cudaError_t init_df64(const StepCfg& c, const double* fields, void* buf, cudaStream_t s);
// One population plane k to / from nx*ny doubles (full populations; solid nodes 0 / ignored).
cudaError_t plane_get_f64(const StepCfg& c, int k, const void* buf, double* out, cudaStream_t s);
cudaError_t plane_get_f32(const StepCfg& c, int k, const void* buf, double* out, cudaStream_t s);
cudaError_t plane_get_f32h(const StepCfg& c, int k, const void* buf, double* out, cudaStream_t s);
cudaError_t plane_get_df64(const StepCfg& c, int k, const void* buf, double* out, cudaStream_t s);
cudaError_t plane_put_f64(const StepCfg& c, int k, const double* in, void* buf, cudaStream_t s);
cudaError_t plane_put_f32(const StepCfg& c, int k, const double* in, void* buf, cudaStream_t s);
cudaError_t plane_put_f32h(const StepCfg& c, int k, const double* in, void* buf, cudaStream_t s);
cudaError_t plane_put_df64(const StepCfg& c, int k, const double* in, void* buf, cudaStream_t s);
// Step-kernel tile candidates for the autotuner: tile TX x TY nodes, TX * BY threads, at least MINB
// resident CTAs per SM requested from the compiler.  Candidate 0 is the default.
struct TileChoice {
  int tx, ty, by, minb;
};
int tile_count_f64();
int tile_count_f32();
int tile_count_f32h();
int tile_count_df64();
TileChoice tile_info_f64(int k);
TileChoice tile_info_f32(int k);
TileChoice tile_info_f32h(int k);
TileChoice tile_info_df64(int k);
cudaError_t launch_step_tile_f64(int k, const StepCfg& c, const void* fin, void* fout, cudaStream_t s);
cudaError_t launch_step_tile_f32(int k, const StepCfg& c, const void* fin, void* fout, cudaStream_t s);
cudaError_t launch_step_tile_f32h(int k, const StepCfg& c, const void* fin, void* fout, cudaStream_t s);
cudaError_t launch_step_tile_df64(int k, const StepCfg& c, const void* fin, void* fout, cudaStream_t s);
// The observables / fields launch of a precision form (LB_FP64 0, LB_FP32_SHIFTED 1, LB_FP32_FP16T 2,
// LB_DF64 3).
inline cudaError_t launch_mode(int precision, int mode, const StepCfg& c, const void* fin, void* fout, double* aux,
                               cudaStream_t s) {
  switch (precision) {
    case 0: return launch_f64(mode, c, fin, fout, aux, s);
    case 1: return launch_f32(mode, c, fin, fout, aux, s);
    case 2: return launch_f32h(mode, c, fin, fout, aux, s);
    default: return launch_df64(mode, c, fin, fout, aux, s);
  }
}
// Double-float exp tables of the LB_DF64 form, written to the current device (lb_init, before capture).
cudaError_t df_exp_tables_init();
// Total shear stress (lb_stress.cu): the field mode writes rho_1, rho_2, T, u^(H) (5 planes of nx*ny
// doubles) to `stage`, then sigma_xy (1 plane), per-row partials, row sums and totals follow there;
// stress_staging_doubles is the staging it needs.  stress_fetch copies the means (out4), the per-row
// means (row, ny) and sigma_xy (field, nx*ny) to the host; each may be nullptr.  Synchronous.
constexpr int kStressTileX = 32, kStressRowVals = 5;
inline size_t stress_staging_doubles(int nx, int ny) {
  const size_t N = (size_t)nx * ny, ncol = (size_t)((nx + kStressTileX - 1) / kStressTileX);
  return 6 * N + (ncol * ny + ny + 1) * kStressRowVals;
}
cudaError_t stress_run(const StepCfg& cfg, int precision, const void* cur, double* stage, cudaStream_t s,
                       double** d_rows, double** d_tot);
cudaError_t stress_fetch(int nx, int ny, const double* stage, const double* d_rows, const double* d_tot, double* out4,
                         double* row, double* field, cudaStream_t s);
// A step (MODE_STEP_NU) from fin to fout that also writes, per warp, the sum of u^(H)_y T over the fluid
// nodes of fin in the arithmetic precision (step_nu_blocks partials, in CTA and warp order); one fixed
// tile shape per precision.
int step_nu_blocks(int precision, int nx, int ny);
cudaError_t launch_step_nu_f64(const StepCfg& c, const void* fin, void* fout, double* partials, cudaStream_t s);
cudaError_t launch_step_nu_f32(const StepCfg& c, const void* fin, void* fout, double* partials, cudaStream_t s);
// Deterministic final reduction of n_blocks partials into kObsOut doubles.
cudaError_t obs_finalize(const StepCfg& c, const double* partials, int n_blocks, double* out, cudaStream_t s);

}  // namespace tlb
