// Internal declarations shared by the kernels and the C-ABI host code.
// Not part of the public interface (include/dugks.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace dugks {

// Face-value weights of eq. flux_DS as printed, f-bar^+(x_b - xi h) =
// g + d.grad g + d^2 : grad^2 g with d = x_b - xi h - x_j = (a dx, b dy)
// (no factor 1/2 on the second-order term, reading Q2p), derivatives by
// second-order central differences on the 3x3 neighbourhood of cell j:
// T[(dy + 1) * 3 + dx + 1] for the cell at offset (dx, dy) from j.  The
// weights sum to one (the difference stencils sum to zero).
template <typename C>
__host__ __device__ __forceinline__ void flux_ds_weights(C a, C b, C (&T)[9]) {
  const C ab = C(0.5) * a * b;
  const C ha = C(0.5) * a, hb = C(0.5) * b;
  T[0] = ab;          T[1] = b * b - hb;                  T[2] = -ab;
  T[3] = a * a - ha;  T[4] = C(1) - C(2) * (a * a + b * b); T[5] = a * a + ha;
  T[6] = -ab;         T[7] = b * b + hb;                  T[8] = ab;
}

enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };
enum { BC_PERIODIC = 0, BC_BOUNCEBACK = 1, BC_DIFFUSE = 2 };

// Kernel ids for launch profiling (names in dugks_capi.cu).
enum KernelId {
  K_CELL_STAGE1 = 0,   // moments of f^, feq, g1 = f-bar^{+,dt/6}
  K_FACE_X_STAGE1,     // x-face interface values at t*
  K_FACE_Y_STAGE1,     // y-face interface values at t*
  K_UPDATE_STAGE1,     // L*, f~(t'), accumulator
  K_CELL_STAGE2,       // moments of f~(t'), feq', g2 = f-bar^{+,5dt/12}
  K_FACE_X_STAGE2,
  K_FACE_Y_STAGE2,
  K_UPDATE_STAGE2,     // L**, dt Omega', f^^{n+1}
  K_MOMENTS,
  K_SET_EQ,
  K_CHECK,
  K_D2Q9_PROLOGUE,     // fused D2Q9 path: g1 from f^ after a new state
  K_D2Q9_STAGE1,       // fused D2Q9 path: whole stage 1 (+ cell part of stage 2)
  K_D2Q9_STAGE2,       // fused D2Q9 path: whole stage 2 (+ cell part of next stage 1)
  K_D2Q9M_STAGE1,      // deviation-storage (FP32/BF16) D2Q9 path, stage 1
  K_D2Q9M_STAGE2,      // deviation-storage D2Q9 path, stage 2
  K_CONVERT,           // FP64 <-> deviation storage
  K_GDEV_CELL,         // deviation-storage generic path: cell pass (both stages)
  K_GDEV_FACE_X,       // interior x faces (both stages)
  K_GDEV_FACE_Y,       // y faces
  K_GDEV_WALLS,        // wall faces of both directions
  K_GDEV_UPDATE1,      // L*, f~(t'), accumulator
  K_GDEV_UPDATE2,      // L**, dt Omega', f^^{n+1}
  K_T2_CELL,           // T2 schemes: moments, g = f-bar^{+,dt/2}
  K_T2_FACE_X,
  K_T2_FACE_Y,
  K_T2_UPDATE,         // f~^{n+1} = f~^{+,n} + dt L
  K_D2Q9DW_STAGE1,     // fused D2Q9 path in double-word arithmetic, stage 1
  K_D2Q9DW_STAGE2,     // stage 2
  K_GNC_SUMS,          // class-moment generic path: class sums of a stage's source
  K_GNC_CELLFIN,       // cell moments, equilibrium parameters, stencil moments
  K_GNC_WALLS,         // wall faces' f-bar of a stage
  K_GNC_FACEFIN,       // face equilibrium parameters, wall densities
  K_GNC_UPDATE1,       // f~(t')
  K_GNC_UPDATE2,       // f^^{n+1}
  K_NUM
};

// Everything a kernel needs to know about the problem; passed by value.
struct DevParams {
  int nx, ny, nv, N;            // N = nx * ny cells
  int px, py;                   // periodic in x / y
  int has_ds;                   // any diffuse wall
  double dx, dy, inv_dx, inv_dy;
  double tau, dt, RT, inv_RT;
  const double* xi_x;           // [nv]
  const double* xi_y;           // [nv]
  const double* w;              // [nv]
  const int* opp;               // [nv], index of -xi_k or -1
  const double* feq_wall;       // [4][nv]  W_k P(xi_k; u_w) per side
  int bc_kind[4];
  double uw_x[4], uw_y[4];
  double ds_den[4];             // -sum_{xi.n<0} (xi.n) W_k P(xi_k; u_w) per side
  int recon;                    // face reconstruction: 0 eq. flux_DS as printed (T3S3, T2S3),
                                // 1 the original DUGKS interpolation (T2S2)
};

// Per-stage scalar coefficients (host-computed once at init).
struct StageCoef {
  double a, b;                  // g = a * src + b * feq
  double h;                     // interface time step of the stage
  double alpha, beta;           // f = alpha f-bar + beta feq at a face
};

// Fused D2Q9 path (dugks_d2q9.cu).  Velocities must be
// xi_k = c (ex_k, ey_k) with ex_k = k/3 - 1, ey_k = k%3 - 1 (the paper's
// listing order); the weights W_k are arbitrary.
//
// Per-stage interface tables.  x-face stencil columns q = 0..3 are the cells
// fi-2 .. fi+1 around face fi, rows r = 0..2 the cells j-1 .. j+1; y-faces
// swap the roles.  The one-sided tables (wall faces, tangential velocities)
// use only the fluid cell's 3x3 neighbourhood.
struct D2Q9Stage {
  double wx[9][3][4];        // x-face weights [k][row][col q]
  double wy[9][4][3];        // y-face weights [k][row q][col]
  double wxL[9][3][3];       // x-face from the left cell only (cols q = 0..2)
  double wxR[9][3][3];       // x-face from the right cell only (cols q = 1..3)
  double wyB[9][3][3];       // y-face from the cell below only (rows q = 0..2)
  double wyT[9][3][3];       // y-face from the cell above only (rows q = 1..3)
  double gamma;              // beta/alpha = h / (2 tau): f / alpha = f-bar + gamma feq
  double kx[9], ky[9];       // flux scale -(stage factor) alpha xi/dx, .../dy
};

struct D2Q9Params {
  int nx, ny, N, px, py, ty;  // ty = tile height (tile width is 32)
  double W[9];
  double c3;                  // c^2/RT (= 3 for the Gauss-Hermite set)
  double base_div;            // RT / c^2 / 2 ... |u|^2/(2RT) = (ut_x^2 + ut_y^2) * base_div
  double half_mb;             // 1/2 - base_div
  int wsym;                   // W_k depends only on |e_k|^2 (W[1] = W[3] = W[5] = W[7], corners equal)
  double c_over_RT;           // c / RT: ut = c u / RT
  double c;                   // lattice speed: xi = c (ex, ey)
  double a1, b1, a2, b2;      // g1 = a1 f^ + b1 feq, g2 = a2 f~' + b2 feq'
  double c_om34;              // 3/4 * (-6 dt / (6 tau + dt))
  double r37;                 // (3 dt/7) / (dt/3) = 9/7
  int bc_kind[4];
  double ds_den[4];
  double feq_wall[4][9];      // W_k P(xi_k; u_w)
  double bb[4][9];            // 2 W_k xi_k.u_w / RT
};

// Mixed-precision D2Q9 path (dugks_d2q9_mixed.cu): arrays hold deviations
// d = f - W_k rho0 in FP32 (store = 1) or BF16 (store = 2); reconstruction,
// fluxes and per-velocity equilibrium assembly in FP32, moment sums and the
// equilibrium parameters (rho, u, polynomial coefficients) in FP64.
struct D2Q9StageF {
  float wx[9][3][4];
  float wy[9][4][3];
  float wxL[9][3][3], wxR[9][3][3], wyB[9][3][3], wyT[9][3][3];
  float gamma;
  float kx[9], ky[9];
};
void d2q9_stage_to_float(const D2Q9Stage& s, D2Q9StageF& f);
cudaError_t launch_d2q9m_stage(const D2Q9Params& p, const D2Q9StageF& s, int store, int stage,
                               double rho0, const void* gin, const void* own,
                               const double* rho_in, void* out0, void* out1, double* rho_out,
                               cudaStream_t st);
// conversions between FP64 f^ and the deviation storage; moments; equilibrium
cudaError_t launch_dev_from_f64(const DevParams& p, int store, double rho0, const double* f,
                                void* d, cudaStream_t st);
cudaError_t launch_f64_from_dev(const DevParams& p, int store, double rho0, const void* d,
                                double* f, cudaStream_t st);
cudaError_t launch_dev_cell(const DevParams& p, int store, double rho0, const void* d,
                            void* g, double* mom, double a, double b, int write_g,
                            cudaStream_t st);
cudaError_t launch_dev_set_eq(const DevParams& p, int store, double rho0, const double* rho,
                              const double* ux, const double* uy, void* d, cudaStream_t st);
cudaError_t d2q9m_prepare();
int d2q9m_occupancy(int store, int ty);

// Optimised generic path (dugks_generic_mixed.cu), any velocity set, in
// three storage forms: store 0 = FP64 (rho0 = 0: the arrays hold f), 1 =
// FP32, 2 = BF16 deviations d = f - W rho0.  fhat/ftp/acc [nv][ny][nx] of
// the storage type; g padded; fbx/fby face values f-bar, eqp [5][N] the
// cell equilibrium parameters of the last cell pass, fpx/fpy [5][nf] the
// face ones, all in the compute type (FP64 for store 0, FP32 otherwise);
// mom FP64 (rho, ux, uy).
struct GDevRef {
  double rho0, W, Wx, Wy;       // rho0, rho0 sum W_k, rho0 sum W_k xi_x, rho0 sum W_k xi_y
};
struct GDevStep {
  DevParams p;
  GDevRef ref;
  int store;
  StageCoef s1, s2;
  double c_om;
  void *fhat, *ftp, *acc;       // [nv][ny][nx]
  void* g;                      // stage field, padded: [nv][ny + 4][pitch], cell (i, j) at (j+2, i+2)
  int pitch;                    // gdev_pitch(nx)
  size_t plane;                 // (ny + 4) * pitch
  void *fbx, *fby, *eqp;        // compute type
  void *fpx, *fpy;              // face assembly parameters [5][nf] of x / y faces
  const void* vq;               // compute-type 4-vectors [3][nv]: (xi_x hi, lo, xi_y hi, lo),
                                // (xi_x, xi_y, W, 0), stage flux factors (-(dt/3) alpha_1 xi/dx,
                                // y, -(4dt/7) alpha_2 xi/dx, y); lo = 0 in FP64
  double *mom, *part;           // part: [nch][3][nf] partial face moments, or [mch][3][N] cell ones
  int nchx, nchy;
  int mch;                      // velocity chunks of the cell moments (1: one thread per cell)
  double ds_out[4];             // rho0 sum over xi.n > 0 of (xi.n) W_k per wall side
  const double* tw;             // FP64 storage: Taylor weights [stage][dir][nv][lower 9, upper 9]
  int tgrid;                    // 1: xi_k = (X[k / n], Y[k % n]) with n a multiple of 16, so the
                                // 16 velocities an update / g-pass thread takes share xi_x
};
int gdev_pitch(int nx);
cudaError_t gdev_prepare(int store);
int gdev_chunks(const DevParams& p, int dir, int sms, int store);
cudaError_t launch_gdev_cell(const GDevStep& s, int stage, cudaStream_t st);
cudaError_t launch_gdev_faces(const GDevStep& s, int stage, int dir, cudaStream_t st);
cudaError_t launch_gdev_walls(const GDevStep& s, int stage, cudaStream_t st);
cudaError_t launch_gdev_update(const GDevStep& s, int stage, cudaStream_t st);

// Class-moment stage kernels for any velocity set (dugks_gnc.cu), FP32 and
// BF16 deviation storage.  Per stage: a streaming pass sums the moments of
// degree <= 3 of the stage's source per cell and sign class of xi; a cell
// pass forms rho, u, the equilibrium's parameters and the stencil moments
// of g; a face pass forms the face equilibria (and the wall densities) from
// them; a wall pass the wall faces' f-bar per velocity; and an update pass
// stages g tile by tile, forms the face values on chip and writes the
// stage's output.  Arrays per (cell, velocity) are [nv][ny][nx] of the
// storage type.
struct GncCombo {               // a sum over sign classes, weights lam, with the face's
  float lam[9];                 // offset (a0, b0) from the upwind cell's centre (cell units)
  float a0, b0;
};
struct GncStep {
  DevParams p;
  GDevRef ref;
  int store;                    // 1 FP32, 2 BF16
  StageCoef s1, s2;
  double c_om;
  void *fhat, *ftp;             // state f^ and f~(t')
  float *eqn, *eqp;             // cell equilibrium parameters [5][N] at t_n and t'
  double *mom_n, *mom_p;        // rho, ux, uy [3][N] at t_n and t'
  float *fpx, *fpy;             // face equilibrium parameters [5][nfx], [5][nfy]
  float* wf;                    // wall faces' f-bar [nv][nw]
  double* wrho;                 // wall density per wall face [nw]
  double* sums;                 // class sums [nsplit][ncls][10][N]
  float* nu;                    // stencil moments [ncombo][18][N]
  const void* vq;               // velocity table of GDevStep::vq (FP32)
  const float* fwt;             // face-value weights [2 stages][nv][48]
  const int* cls_off;           // [ncls + 1] first table entry of each class
  const int* cls_k;             // velocity of each entry
  const float* cls_mono;        // [entries][12]: the ten monomials of the velocity
  const float* zc;              // [ncombo][10][6] equilibrium quadrature per combination
  const float2* wbb;            // [nv][4] bounce-back (c_k, shift_k) per side
  const int* wsrc;              // [4][nv] velocity whose wall-face entry the update reads
  int ncls, ncombo, nsplit;      // classes, combinations, velocity splits of the sums
  int ties;                     // some velocity has xi_x = 0 or xi_y = 0
  GncCombo cmb[12];
  int c_lo[2], c_up[2];         // interior faces of x and y: xi.n > 0 / < 0 combinations
  int c_wf[4], c_win[4];        // per wall: fluid side (ties too), strictly incoming
  float tu[6][9];               // T(a, b) = sum_u tu[u] u(a, b), u = 1, a, b, a^2, ab, b^2
  int ntl;                      // the nonzero tu as a list: stencil cell, u, weight
  unsigned char tl_s[54], tl_u[54];
  float tl_w[54];
  double wB[4][3], wH[4][3];    // per wall, sums over the leaving velocities of (1, xi) x
  double wMo[4][3], wWo[4][3];  // bounce-back coefficient, shift, wall equilibrium, W rho0
  double ds_out[4];             // rho0 sum over xi.n > 0 of (xi.n) W_k per wall side
  int nw;                       // wall face slots: W rows, E rows, S columns, N columns
  int nch, kc;                  // velocity chunks and velocities per chunk
  int tiles_x, tiles_y;         // 32 x 16 cell tiles
};
struct GncTables {              // host tables of GncStep's device arrays
  std::vector<int> cls_off, cls_k, wsrc;
  std::vector<float> cls_mono, zc, fwt, wbb;
};
// Fill g's by-value tables and t from the velocity set (host arrays) and the
// wall data; false if the stencil weights are not quadratic in (a, b).
bool gnc_tables(GncStep& g, const double* xi_x, const double* xi_y, const double* w,
                const double* feq_wall, const int* opp, GncTables& t);
int gnc_chunks(const GncStep& g, int sms);
int gnc_splits(const GncStep& g, const GncTables& t, int sms);
cudaError_t gnc_prepare(int store);
cudaError_t launch_gnc_sums(const GncStep& s, int stage, cudaStream_t st);
cudaError_t launch_gnc_cellfin(const GncStep& s, int stage, cudaStream_t st);
cudaError_t launch_gnc_facefin(const GncStep& s, int stage, cudaStream_t st);
cudaError_t launch_gnc_walls(const GncStep& s, int stage, cudaStream_t st);
cudaError_t launch_gnc_update(const GncStep& s, int stage, cudaStream_t st);

// Many class-moment instances (one storage type and tie flag) stepped by
// one launch per kernel and stage: descriptors and per-kernel block
// prefixes in device memory.
struct GncBatch {
  GncStep* steps = nullptr;     // device [n]
  int* start = nullptr;         // device [5][n + 1]: blocks of sums, cellfin, facefin, walls, update
  float* coef = nullptr;        // device [n][2][5]: the update's coefficients per stage
  int n = 0, store = 1, ties = 0;
  int ncombo_max = 1;           // the instances' largest class-combination count
  int total[5] = {};
};
cudaError_t gnc_batch_init(const GncStep* const* steps, int n, GncBatch& b);
cudaError_t launch_gnc_batch_stage(const GncBatch& b, int stage, cudaStream_t st);
void gnc_batch_free(GncBatch& b);

// One instance of a batched D2Q9 FP64 launch (device memory).
struct D2Q9BatchItem {
  D2Q9Params P;
  D2Q9Stage S1, S2;
  double *fhat, *g1, *g2, *X, *mom;
  int tiles_x, pad;
};
cudaError_t launch_d2q9_batch(int stage, const D2Q9BatchItem* items, const int* tile_start,
                              int nitems, int max_ty, int* counter, int blocks, cudaStream_t st);
int d2q9_batch_blocks_per_sm(int max_ty);

cudaError_t launch_d2q9_stage(const D2Q9Params& p, const D2Q9Stage& s, int stage,
                              const double* gin, const double* own, const double* rho_in,
                              double* out0, double* out1, double* rho_out, cudaStream_t st);
size_t d2q9_smem_bytes(int ty);
cudaError_t d2q9_prepare(int ty);
// stage 1 of the fused FP64 path writing g2 and f~(t') (the adjoint's recomputation)
cudaError_t launch_d2q9_ftp(const D2Q9Params& p, const D2Q9Stage& s, const double* g1,
                            const double* fhat, const double* rho_fhat, double* g2, double* ftp,
                            double* rho_ftp, cudaStream_t st);
// moments of f^ into mom[3][N] (rho, ux, uy) and, with write_g, g1 (FP64 fused path)
cudaError_t launch_d2q9_cell(const D2Q9Params& p, bool write_g, const double* fhat, double* g1,
                             double* mom, cudaStream_t st);

// Double-word arithmetic form of the fused D2Q9 kernels: FP64 arrays, every
// operation in double-word (FP32 pair) arithmetic (dugks_dw.cuh).  The
// parameters are the FP64 ones split on the host into h + l pairs.
struct dw {
  float h, l;                   // value h + l, |l| <= ulp(h) / 2
};
struct D2Q9ParamsDW {
  int nx, ny, N, px, py, ty;
  dw W[9];
  dw c3, base_div, half_mb;
  int wsym;
  dw c;
  dw a1, b1, a2, b2;
  dw c_om34, r37;
  int bc_kind[4];
  dw c_ds[4];                   // c / ds_den: the diffuse wall density factor
  dw feq_wall[4][9];
  dw bb[4][9];
};
struct D2Q9StageDW {
  dw wx[9][3][4];
  dw wy[9][4][3];
  dw wxL[9][3][3], wxR[9][3][3], wyB[9][3][3], wyT[9][3][3];
  dw gamma;
  dw kx[9], ky[9];
};
// largest tile height of the FP64 / double-word stage kernels, and their
// resident blocks per SM at height ty (the smaller of the two stages; 0 if
// the occupancy query fails)
int d2q9_max_ty(bool dwa);
int d2q9_occupancy(bool dwa, bool wsym, int ty);
void d2q9_params_to_dw(const D2Q9Params& p, D2Q9ParamsDW& d);
void d2q9_stage_to_dw(const D2Q9Stage& s, D2Q9StageDW& d);
// the g1 prologue and moments of the double-word form (its stage-2 arithmetic)
cudaError_t launch_d2q9dw_cell(const D2Q9ParamsDW& p, const double* fhat, double* g1,
                               double* mom, cudaStream_t st);
cudaError_t launch_d2q9dw_stage(const D2Q9ParamsDW& p, const D2Q9StageDW& s, int stage,
                                const double* gin, const double* own, const double* rho_in,
                                double* out0, double* out1, double* rho_out, cudaStream_t st);

// Adjoint kernels (dugks_adjoint.cu); grads = [tau, uw_x(W), uw_y(W), uw_x(E), ...].
cudaError_t launch_flux_T(const DevParams& p, int dir, const double* A, double sa,
                          const double* B, double sb, double* phi, cudaStream_t s);
cudaError_t launch_face_T(const DevParams& p, int dir, const double* g, const double* mom,
                          double* phi, double* gbar, double* rhobar, double* grads,
                          const StageCoef& c, double dalpha, double* fbs, cudaStream_t s);
cudaError_t launch_cell_T(const DevParams& p, const double* x, const double* gbar,
                          const double* lam, const double* rhobar, double* xbar, double a,
                          double b, double c_extra, double da, double dc, double* grads,
                          cudaStream_t s);
cudaError_t launch_axpby(size_t n, const double* A, double sa, const double* B, double sb,
                         double* out, cudaStream_t s);
cudaError_t launch_eq_T(const DevParams& p, const double* rho, const double* ux,
                        const double* uy, const double* lam, double* drho, double* dux,
                        double* duy, cudaStream_t s);

// Sets the message returned by dugks_last_error() on the calling thread.
void set_last_error(const std::string& msg);

// Launchers (dugks_kernels.cu).  All asynchronous on `s`.
cudaError_t launch_cell(const DevParams& p, int groups, int stage, const double* src,
                        double* g, double* mom, double a, double b, cudaStream_t s);
// walls_only = 1: only the wall faces of direction dir (non-periodic sides)
cudaError_t launch_face(const DevParams& p, int groups, int dir, const double* g,
                        const double* mom, double* fb, const StageCoef& c, cudaStream_t s,
                        int walls_only = 0);
// Interior faces of large velocity sets (dugks_nc.cu): pass 1 (stencils,
// partial face moments per velocity chunk into part[nchunk][3][nf]) and
// pass 2 (f = alpha f-bar + beta feq).  Wall faces: launch_face(walls_only).
int nc_chunks(const DevParams& p, int dir, int sms);
cudaError_t launch_nc_faces(const DevParams& p, int dir, const double* g, double* fb,
                            double* part, int nchunk, const StageCoef& c, cudaStream_t s);
cudaError_t launch_update1(const DevParams& p, const double* fhat, const double* g1,
                           const double* fbx, const double* fby, double* ftp, double* acc,
                           cudaStream_t s);
cudaError_t launch_update2(const DevParams& p, const double* ftp, const double* acc,
                           const double* mom, const double* fbx, const double* fby,
                           double* fhat, double c_om, cudaStream_t s);
// T2 step update (Remark I): ft <- a ft + b feq(mom) + dt L
cudaError_t launch_update_t2(const DevParams& p, const double* mom, const double* fbx,
                            const double* fby, double* ft, double a, double b, cudaStream_t s);
cudaError_t launch_set_eq(const DevParams& p, const double* rho, const double* ux,
                          const double* uy, double* fhat, cudaStream_t s);
cudaError_t launch_check(const DevParams& p, const double* mom, int* flag, cudaStream_t s);

}  // namespace dugks
