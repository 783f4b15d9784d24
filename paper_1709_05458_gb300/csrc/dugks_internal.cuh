// Internal declarations shared by the kernels and the C-ABI host code.
// Not part of the public interface (include/dugks.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace dugks {

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
};

// Per-stage scalar coefficients (host-computed once at init).
struct StageCoef {
  double a, b;                  // g = a * src + b * feq
  double h;                     // interface time step of the stage
  double alpha, beta;           // f = alpha f-bar + beta feq at a face
};

// Sets the message returned by dugks_last_error() on the calling thread.
void set_last_error(const std::string& msg);

// Launchers (dugks_kernels.cu).  All asynchronous on `s`.
cudaError_t launch_cell(const DevParams& p, int groups, int stage, const double* src,
                        double* g, double* mom, double a, double b, cudaStream_t s);
cudaError_t launch_face(const DevParams& p, int groups, int dir, const double* g,
                        const double* mom, double* fb, const StageCoef& c, cudaStream_t s);
cudaError_t launch_update1(const DevParams& p, const double* fhat, const double* g1,
                           const double* fbx, const double* fby, double* ftp, double* acc,
                           cudaStream_t s);
cudaError_t launch_update2(const DevParams& p, const double* ftp, const double* acc,
                           const double* mom, const double* fbx, const double* fby,
                           double* fhat, double c_om, cudaStream_t s);
cudaError_t launch_set_eq(const DevParams& p, const double* rho, const double* ux,
                          const double* uy, double* fhat, cudaStream_t s);
cudaError_t launch_check(const DevParams& p, const double* mom, int* flag, cudaStream_t s);

}  // namespace dugks
