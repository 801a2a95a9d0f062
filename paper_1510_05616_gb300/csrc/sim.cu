// sim.cu -- channel response (extended linear system) and the semi-implicit vesicle step.
//
// Channel response (Sec. 2.2, 2.3, three-step procedure of Sec. 3.1):
//   u = D^near tau + sum_m c_m S(., y_m) (Eq. (urep)); the blocks A, B, C, Q of
//   [A B; C Q][tau; c] = [v; g] (Eq. (BIEU), (BIED), (BIEgu), (BIEgT)) are assembled densely in
//   FP64 by kernels; A is LU-factored (cuSOLVER), W = A^-1 B, S = Q - C W, and S's
//   pseudo-inverse comes from an SVD with singular values below 1e-13 sigma_max dropped; a
//   solve is c = S^+ (g - C A^-1 v), tau = A^-1 v - W c (the block elimination of Sec. 4.1,
//   with LU in place of the paper's fast direct solver).  Side points: K Gauss-Legendre nodes
//   across the inlet at x = 0, R = L + d, normal (1, 0); proxies: M points on a circle of
//   radius R_p about (d/2, 0).  The pressure drive p_drive (pressure drop per period) enters
//   as g_T = p_drive n.
// Vesicle step (Sec. 3.2, Eq. (tsteplinsys), Eq. (ALC), Algorithm 1 steps 2-9, App. B, C):
//   Fourier differentiation d/ds = (1/|x_alpha|) D_alpha per vesicle; forces, channel
//   response of the explicit forces, right-preconditioned GMRES on
//   [I + dt kB S d_ssss, -S d_s(x_s .); x_s . d_s, 0][u; sigma] = [S f_b + u_resp; rhs_ALC]
//   whose matvec calls the layer-potential sum (stokes_sum_eval) of all vesicles, with a
//   block-diagonal preconditioner made of each vesicle's self interaction (dense, batched
//   LU inverse); then x += dt u, area correction, reparameterization.
// The traction kernel of the double layer is Eq. (T) with d_x = (r . n_x) / r^2 (target) and
// d_y = (r . n_y) / r^2 (source), which makes it the traction of the (D, P) pair.
#include <cublas_v2.h>
#include <cusolverDn.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <vector>

#include "df.cuh"
#include "fds.cuh"
#include "stokes_internal.cuh"
#include "stokes_mlp_internal.cuh"

namespace stokes {
cudaError_t launch_kress_table(int n, double *T, cudaStream_t s);
}

using namespace stokes;

struct stokes_sim {
  int device = 0;
  std::string err;
  cudaStream_t s = nullptr;
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t sol = nullptr;
  double mu = 1.0, period = 0.0;
  // walls and the extended system
  bool have_walls = false;
  int Nt = 0, K = 0, M = 0, nA = 0;
  stokes_ctx *ctx_w = nullptr;         // walls only (double-layer sums at vesicle nodes)
  double2 *d_wx = nullptr;             // wall nodes (free targets of the vesicle sums)
  double2 *d_side = nullptr;           // [2K]: L points then R points
  double2 *d_proxy = nullptr;          // [M]
  double *d_LU = nullptr, *d_W = nullptr, *d_C = nullptr, *d_Spinv = nullptr;
  int *d_piv = nullptr, *d_info = nullptr;
  double *d_nrm_part = nullptr;        // [kNrmBlocks] partial sums of squares (dnrm)
  // wall solver: STOKES_WALLS_FDS (default) the fast direct solver of Sec. 4;
  // STOKES_WALLS_LU64 factors A in FP64; STOKES_WALLS_LU32_REFINE inverts an FP32 copy (LU, then
  // the inverse, d_Ainv32) and refines every solve with FP64 residuals of the FP64 A (d_A)
  int wall_solver = STOKES_WALLS_FDS;
  int walls_mode = STOKES_WALLS_FDS;  // the solver the current walls were factored for
  cusolverDnParams_t params = nullptr;
  double *d_A = nullptr;
  float *d_Ainv32 = nullptr;
  double *d_wb = nullptr, *d_wr = nullptr;  // refinement right-hand sides and residuals
  float *d_wr32 = nullptr, *d_wb32 = nullptr;  // FP32 residual and correction
  size_t wall_ws_len = 0;                   // capacity of d_wb / d_wr / d_wr32 (elements)
  int wall_refinements = 0;                 // last wall solve: refinement sweeps and
  double wall_residual = 0.0;               //   relative residual ||b - A x|| / ||b||
  // STOKES_WALLS_FDS: the fast direct solver of Sec. 4 (HBS A_0^-1, neighbour L R, SMW)
  stokes::fds_solver *fds = nullptr;
  stokes::fds_params fds_p;
  double walls_setup_ms = 0.0;              // last stokes_sim_set_walls, wall clock
  // vesicles
  bool have_ves = false;
  int V = 0, n = 0, Nv = 0;
  double kappa_b = 1.0;
  stokes_ctx *ctx_v = nullptr;         // vesicles only (single-layer sums, Kress self terms)
  double2 *d_x = nullptr, *d_nrm = nullptr, *d_xs = nullptr;
  double *d_w = nullptr, *d_spd = nullptr, *d_sigma = nullptr, *d_D = nullptr, *d_kress = nullptr;
  double *d_L0 = nullptr, *d_A0 = nullptr, *d_Lk = nullptr;
  double2 *d_f = nullptr, *d_fb = nullptr, *d_ures = nullptr, *d_tmp2 = nullptr, *d_tmp3 = nullptr;
  double *d_vrhs = nullptr, *d_c = nullptr;
  double *d_tau = nullptr;
  // refinement of the block solve on the whole extended system: B and Q kept, right-hand
  // side copies, residuals and corrections
  int block_refine = 3;
  double inner_tol = 1e-3;  // mixed-precision step: relative tolerance of each FP32-Kahan solve
  double *d_B = nullptr, *d_Q = nullptr;
  double *d_rv = nullptr, *d_rg = nullptr, *d_resv = nullptr, *d_resg = nullptr;
  double *d_side_part = nullptr;       // [K][kSideChunks][4] partial side-point sums
  double *d_dtau = nullptr, *d_dc = nullptr, *d_g2 = nullptr;
  // preconditioner (per vesicle 3n x 3n) and GMRES workspace
  double *d_G = nullptr, *d_Ds = nullptr, *d_D2 = nullptr, *d_D4 = nullptr, *d_T = nullptr;
  double *d_P = nullptr, *d_Pinv = nullptr;
  double **d_Pptr = nullptr, **d_Piptr = nullptr;
  // FP32 factorization of the same blocks (default): P32 = fl32(P), Pinv32 = its inverse,
  // applied with FP64 accumulation (a fixed FP64 linear operator)
  int precond_fp32 = 1;
  float *d_P32 = nullptr, *d_Pinv32 = nullptr;
  float **d_Pptr32 = nullptr, **d_Piptr32 = nullptr;
  // Newton-Schulz refresh of the FP32 inverse from the previous step's (opt-in): workspace, the
  // largest per-vesicle ||I - P X||_F (device), whether d_Pinv32 holds an inverse for the
  // current dt, the dt it was made for, and the last step's refresh count (0: LU)
  bool precond_refresh = false;
  // the FP32 assembly and refresh GEMMs by cuBLAS's BF16x9 FP32 emulation (opt-in)
  bool precond_tensor = false;
  float *d_T32 = nullptr, *d_X32 = nullptr;
  unsigned *d_enorm = nullptr;
  bool pinv_valid = false;
  double pinv_dt = 0.0;
  int last_refresh = 0;
  int *d_ppiv = nullptr, *d_pinfo = nullptr;
  int gm_m = 0;
  double *d_V = nullptr, *d_z = nullptr, *d_b = nullptr, *d_wk = nullptr, *d_h = nullptr;
  double *d_xsol = nullptr;            // last solution [u_x, u_y, sigma] per vesicle
  double *d_rr = nullptr, *d_dd = nullptr;  // refinement residual and correction
  // warm-start features / targets of the last step
  float *d_feat = nullptr, *d_targ = nullptr, *d_pred = nullptr;  // sized for the most modes
  int warm_modes = 16;                 // Fourier modes of the warm-start representation
  bool warm_history = false;           // features also carry z_prev and z_prev - z_prev2
  int warm_base = 0;                   // STOKES_WARM_BASE_*: what the network's change is added to
  int hist_count = 0;                  // solutions in the history: z_prev valid at 1, z_prev2 at 2
  double *d_zprev2 = nullptr;          // the solution two steps back
  double *d_frame = nullptr;           // per vesicle: cx, cy, theta, l, U, sigma scale
  double *d_bprev = nullptr, *d_zprev = nullptr;  // previous step's right-hand side and solution
  // mixed-precision step: the FP64-accurate vesicle sums (right-hand side S f_b and the
  // refinement residuals) by the FMM of order resid_fmm_order instead of double-float direct
  // sums (0 = off); the plan is rebuilt every step on a host thread beside the GPU's work
  int resid_fmm_order = 0, resid_fmm_leaf = 32;
  // mixed-precision step: the Krylov sweeps' vesicle sums by the same plan evaluated at order
  // sweep_fmm_order instead of the FP32-Kahan direct sum (0 = off); the plan is made at the
  // larger of the two orders
  int sweep_fmm_order = 0;
  stokes_fmm *fmm_v = nullptr;
  // with FMM residuals, the block refinement's wall double-layer sums (channel response) come
  // from an FMM plan of the fixed walls, made at the first such step after stokes_sim_set_walls
  stokes_fmm *fmm_w = nullptr;
  int fmm_w_order = 0;
  // ... and the channel response's two vesicle-wall sums from per-step plans with the other
  // kind's nodes as their only targets: vesicle sources at the wall nodes, wall sources at
  // the vesicle nodes
  stokes_fmm *fmm_vw = nullptr, *fmm_wv = nullptr;
  // close evaluation of the vesicle-vesicle single layer (stokes_sim_set_close_eval): every
  // vesicle sum of the step adds the correction of the close (node, vesicle image) pairs found
  // for the step's positions; factor 0 = off
  double close_factor = 0.0;
  int close_K = 16;
  stokes_close *close_v = nullptr;
};

namespace {

constexpr double kPiD = 3.14159265358979323846;
constexpr int kMaxN = 256;  // nodes per vesicle supported by the step kernels

int fail(stokes_sim *m, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (m) m->err = buf;
  return code;
}

#define SK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(m, e_ == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA, \
                  "%s: %s", #call, cudaGetErrorString(e_));                          \
  } while (0)
#define BK(call)                                                                   \
  do {                                                                             \
    cublasStatus_t e_ = (call);                                                    \
    if (e_ != CUBLAS_STATUS_SUCCESS) return fail(m, STOKES_ERR_CUDA, "%s: cublas %d", #call, int(e_)); \
  } while (0)
#define QK(call)                                                                   \
  do {                                                                             \
    cusolverStatus_t e_ = (call);                                                  \
    if (e_ != CUSOLVER_STATUS_SUCCESS) return fail(m, STOKES_ERR_CUDA, "%s: cusolver %d", #call, int(e_)); \
  } while (0)
#define ST(call)                  \
  do {                            \
    int st_ = (call);             \
    if (st_) return st_;          \
  } while (0)

template <class T>
void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <class T>
cudaError_t dalloc(T *&p, size_t count) {
  dfree(p);
  return cudaMalloc(reinterpret_cast<void **>(&p), std::max<size_t>(count, 1) * sizeof(T));
}

inline int nb(long n, int b) { return int((n + b - 1) / b); }

// ---------------------------------------------------------------------------
// 2x2 kernel tensors, FP64 (row-major a[0..3] = (11, 12, 21, 22))
// ---------------------------------------------------------------------------
__device__ __forceinline__ void k_stokeslet(double rx, double ry, double cmu, double *a) {
  const double rr = rx * rx + ry * ry;
  const double lg = -0.5 * log(rr);
  a[0] = cmu * (lg + rx * rx / rr);
  a[1] = a[2] = cmu * rx * ry / rr;
  a[3] = cmu * (lg + ry * ry / rr);
}

__device__ __forceinline__ void k_stresslet(double rx, double ry, double nx, double ny, double *a) {
  const double rr = rx * rx + ry * ry;
  const double c = (rx * nx + ry * ny) / (kPiD * rr * rr);
  a[0] = c * rx * rx;
  a[1] = a[2] = c * rx * ry;
  a[3] = c * ry * ry;
}

__device__ __forceinline__ void k_slp_traction(double rx, double ry, double nx, double ny, double *a) {
  const double rr = rx * rx + ry * ry;
  const double c = -(rx * nx + ry * ny) / (kPiD * rr * rr);
  a[0] = c * rx * rx;
  a[1] = a[2] = c * rx * ry;
  a[3] = c * ry * ry;
}

// Eq. (T): traction at x (normal nx) of the double layer at y (normal ny).
__device__ __forceinline__ void k_dlp_traction(double rx, double ry, double nxx, double nxy,
                                               double nyx, double nyy, double mu, double *a) {
  const double rr = rx * rx + ry * ry;
  const double dx = (rx * nxx + ry * nxy) / rr;
  const double dy = (rx * nyx + ry * nyy) / rr;
  const double nn = nxx * nyx + nxy * nyy;
  const double r[2] = {rx, ry}, nX[2] = {nxx, nxy}, nY[2] = {nyx, nyy};
  const double c1 = (nn / rr - 8.0 * dx * dy) / rr;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 2; ++k)
      a[2 * i + k] = (mu / kPiD) * (c1 * r[i] * r[k] + (i == k ? dx * dy : 0.0) + nX[i] * nY[k] / rr +
                                   dx * r[k] * nY[i] / rr + dy * r[i] * nX[k] / rr);
}

// ---------------------------------------------------------------------------
// assembly of the extended system (column-major)
// ---------------------------------------------------------------------------
__global__ void assemble_A_kernel(int Nt, const double2 *x, const double2 *nrm, const double *w,
                                  const double *kap, double d, double *A) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= Nt) return;
  const long lda = 2L * Nt;
  double s[4] = {0, 0, 0, 0}, t[4];
  for (int m = -1; m <= 1; ++m) {
    if (m == 0 && i == j) continue;
    k_stresslet(x[i].x - (x[j].x + m * d), x[i].y - x[j].y, nrm[j].x, nrm[j].y, t);
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += t[q];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) s[q] *= w[j];
  if (i == j) {
    const double tx = -nrm[j].y, ty = nrm[j].x, c = -kap[j] / (2.0 * kPiD) * w[j];
    s[0] += c * tx * tx - 0.5;
    s[1] += c * tx * ty;
    s[2] += c * tx * ty;
    s[3] += c * ty * ty - 0.5;
  }
  A[(2 * i) + (2L * j) * lda] = s[0];
  A[(2 * i) + (2L * j + 1) * lda] = s[1];
  A[(2 * i + 1) + (2L * j) * lda] = s[2];
  A[(2 * i + 1) + (2L * j + 1) * lda] = s[3];
}

__global__ void assemble_B_kernel(int Nt, int M, const double2 *x, const double2 *proxy, double cmu,
                                  double *B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (i >= Nt) return;
  const long ld = 2L * Nt;
  double a[4];
  k_stokeslet(x[i].x - proxy[m].x, x[i].y - proxy[m].y, cmu, a);
  B[2 * i + (2L * m) * ld] = a[0];
  B[2 * i + (2L * m + 1) * ld] = a[1];
  B[2 * i + 1 + (2L * m) * ld] = a[2];
  B[2 * i + 1 + (2L * m + 1) * ld] = a[3];
}

__global__ void assemble_C_kernel(int Nt, int K, const double2 *x, const double2 *nrm,
                                  const double *w, const double2 *side, double d, double mu,
                                  double *C) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (j >= Nt) return;
  const long ld = 4L * K;
  const double2 L = side[k], R = side[K + k];
  double a[4], b[4];
  // velocity discrepancy D(x_R, y - d) - D(x_L, y + d)
  k_stresslet(R.x - (x[j].x - d), R.y - x[j].y, nrm[j].x, nrm[j].y, a);
  k_stresslet(L.x - (x[j].x + d), L.y - x[j].y, nrm[j].x, nrm[j].y, b);
  C[2 * k + (2L * j) * ld] = w[j] * (a[0] - b[0]);
  C[2 * k + (2L * j + 1) * ld] = w[j] * (a[1] - b[1]);
  C[2 * k + 1 + (2L * j) * ld] = w[j] * (a[2] - b[2]);
  C[2 * k + 1 + (2L * j + 1) * ld] = w[j] * (a[3] - b[3]);
  // traction discrepancy with the side normal (1, 0)
  k_dlp_traction(R.x - (x[j].x - d), R.y - x[j].y, 1.0, 0.0, nrm[j].x, nrm[j].y, mu, a);
  k_dlp_traction(L.x - (x[j].x + d), L.y - x[j].y, 1.0, 0.0, nrm[j].x, nrm[j].y, mu, b);
  const int r0 = 2 * K + 2 * k;
  C[r0 + (2L * j) * ld] = w[j] * (a[0] - b[0]);
  C[r0 + (2L * j + 1) * ld] = w[j] * (a[1] - b[1]);
  C[r0 + 1 + (2L * j) * ld] = w[j] * (a[2] - b[2]);
  C[r0 + 1 + (2L * j + 1) * ld] = w[j] * (a[3] - b[3]);
}

__global__ void assemble_Q_kernel(int K, int M, const double2 *side, const double2 *proxy,
                                  double cmu, double *Q) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (k >= K) return;
  const long ld = 4L * K;
  const double2 L = side[k], R = side[K + k], y = proxy[m];
  double a[4], b[4];
  k_stokeslet(R.x - y.x, R.y - y.y, cmu, a);
  k_stokeslet(L.x - y.x, L.y - y.y, cmu, b);
  Q[2 * k + (2L * m) * ld] = a[0] - b[0];
  Q[2 * k + (2L * m + 1) * ld] = a[1] - b[1];
  Q[2 * k + 1 + (2L * m) * ld] = a[2] - b[2];
  Q[2 * k + 1 + (2L * m + 1) * ld] = a[3] - b[3];
  k_slp_traction(R.x - y.x, R.y - y.y, 1.0, 0.0, a);
  k_slp_traction(L.x - y.x, L.y - y.y, 1.0, 0.0, b);
  const int r0 = 2 * K + 2 * k;
  Q[r0 + (2L * m) * ld] = a[0] - b[0];
  Q[r0 + (2L * m + 1) * ld] = a[1] - b[1];
  Q[r0 + 1 + (2L * m) * ld] = a[2] - b[2];
  Q[r0 + 1 + (2L * m + 1) * ld] = a[3] - b[3];
}

// S^+ = U diag(1/sigma, truncated) V^T from the SVD S^T = U Sigma V^T:  scale U's columns.
__global__ void scale_columns_kernel(int rows, int cols, const double *sig, double cutoff,
                                     double *U) {
  const long t = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= long(rows) * cols) return;
  const int c = int(t / rows);
  const double s = sig[c];
  U[t] = (s > cutoff) ? U[t] / s : 0.0;
}

__global__ void transpose_kernel(int rows, int cols, const double *in, double *out) {
  const long t = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= long(rows) * cols) return;
  const int r = int(t % rows), c = int(t / rows);
  out[c + long(r) * cols] = in[t];
}

// Data g of the response to vesicle forces (Eq. (vesgu), (vesgT)) at the side points; one
// block per side point, fixed-order tree reduction over the vesicle nodes.
// Side-point data: CTA (k, c) sums the vesicle nodes j = c 256 + t, + kSideChunks 256, ...
// (thread t) for side pair k into part[k][c][4]; side_rhs_finish_kernel adds the chunks in
// order.  kSideChunks CTAs per side pair spread the 2K x N_v pairs over the SMs.
constexpr int kSideChunks = 32;
__global__ void side_rhs_kernel(int K, int Nv, const double2 *side, const double2 *xv,
                                const double *wv, const double2 *f, double d, double cmu,
                                double *part) {
  __shared__ double red[4][256];
  const int k = blockIdx.x, c = blockIdx.y;
  const double2 L = side[k], R = side[K + k];
  double acc[4] = {0, 0, 0, 0};
  for (int j = c * blockDim.x + threadIdx.x; j < Nv; j += kSideChunks * blockDim.x) {
    const double qx = wv[j] * f[j].x, qy = wv[j] * f[j].y;
    double a[4], b[4];
    k_stokeslet(R.x - (xv[j].x - d), R.y - xv[j].y, cmu, a);
    k_stokeslet(L.x - (xv[j].x + d), L.y - xv[j].y, cmu, b);
    acc[0] += -(a[0] * qx + a[1] * qy) + (b[0] * qx + b[1] * qy);
    acc[1] += -(a[2] * qx + a[3] * qy) + (b[2] * qx + b[3] * qy);
    k_slp_traction(R.x - (xv[j].x - d), R.y - xv[j].y, 1.0, 0.0, a);
    k_slp_traction(L.x - (xv[j].x + d), L.y - xv[j].y, 1.0, 0.0, b);
    acc[2] += -(a[0] * qx + a[1] * qy) + (b[0] * qx + b[1] * qy);
    acc[3] += -(a[2] * qx + a[3] * qy) + (b[2] * qx + b[3] * qy);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
#pragma unroll
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 4) part[(size_t(k) * kSideChunks + c) * 4 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void side_rhs_finish_kernel(int K, const double *part, double p_drive, double *g) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double a[4] = {0, 0, 0, 0};
  for (int c = 0; c < kSideChunks; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] += part[(size_t(k) * kSideChunks + c) * 4 + q];
  g[2 * k] = a[0];
  g[2 * k + 1] = a[1];
  g[2 * K + 2 * k] = a[2] + p_drive;  // + p_drive n, n = (1, 0)
  g[2 * K + 2 * k + 1] = a[3];
}

__global__ void empty_rhs_kernel(int K, double p_drive, double *g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * K) return;
  g[t] = (t >= 2 * K && ((t - 2 * K) & 1) == 0) ? p_drive : 0.0;
}

// u_i += sum_m S(x_i, y_m) c_m (proxy part of Eq. (urep)).
__global__ void proxy_eval_kernel(int n_t, const double2 *xt, int M, const double2 *proxy,
                                  const double *c, double cmu, double2 *u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_t) return;
  double ux = 0.0, uy = 0.0, a[4];
  for (int m = 0; m < M; ++m) {
    k_stokeslet(xt[i].x - proxy[m].x, xt[i].y - proxy[m].y, cmu, a);
    ux += a[0] * c[2 * m] + a[1] * c[2 * m + 1];
    uy += a[2] * c[2 * m] + a[3] * c[2 * m + 1];
  }
  u[i].x += ux;
  u[i].y += uy;
}

// p_i += sum_m c_m . Q(x_i, y_m), Q = r / (2 pi r^2) (Eq. (Q); pressure of the proxy part).
__global__ void proxy_pressure_kernel(int n_t, const double2 *xt, int M, const double2 *proxy,
                                      const double *c, double *p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_t) return;
  double acc = 0.0;
  for (int m = 0; m < M; ++m) {
    const double r1 = xt[i].x - proxy[m].x, r2 = xt[i].y - proxy[m].y;
    acc += (r1 * c[2 * m] + r2 * c[2 * m + 1]) / (r1 * r1 + r2 * r2);
  }
  p[i] += acc / (2.0 * kPiD);
}

__global__ void axpby_kernel(long n, double a, const double *x, double b, double *y) {
  const long t = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) y[t] = a * x[t] + b * y[t];
}

// ---------------------------------------------------------------------------
// per-vesicle spectral kernels (one block per vesicle, blockDim = n)
// ---------------------------------------------------------------------------
// Fourier differentiation on n equispaced points (n even) is circulant: D[a][k] = d[(a - k) mod
// n] with d[0] = 0, d[q] = (-1)^q cot(q pi / n) / 2; every entry is computed from q in [0, n).
__global__ void fourier_diff_kernel(int n, double *D) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int a = t / n, k = t % n, q = a >= k ? a - k : a - k + n;
  D[t] = (q == 0) ? 0.0 : 0.5 * ((q & 1) ? -1.0 : 1.0) / tan(q * kPiD / n);
}

// The per-vesicle kernels (blockDim = n, thread a) keep dd[j] = d[j mod n], j < 2n, in shared
// memory, taken from D's column 0, and read row a of D as dd[a + n - k]: broadcast-free,
// conflict-free shared loads instead of a strided walk through D's rows.  Needs a
// __syncthreads() before the first drow.
__device__ __forceinline__ void load_diff(const double *D, double *dd, int n, int a) {
  const double d = D[size_t(a) * n];
  dd[a] = d;
  dd[a + n] = d;
}

// out = D in over one vesicle's n values held in shared memory (D as dd above).
__device__ __forceinline__ double drow(const double *dd, const double *in, int n, int a) {
  double s = 0.0;
  const double *row = dd + a + n;
  for (int k = 0; k < n; ++k) s += row[-k] * in[k];
  return s;
}

// Geometry of the current positions: speed, unit tangent, outward normal, weights.
__global__ void ves_geom_kernel(int n, const double2 *x, const double *D, double *spd,
                                double2 *xs, double2 *nrm, double *w) {
  __shared__ double X[kMaxN], Y[kMaxN];
  const int v = blockIdx.x, a = threadIdx.x, i = v * n + a;
  __shared__ double dd[2 * kMaxN];
  load_diff(D, dd, n, a);
  X[a] = x[i].x;
  Y[a] = x[i].y;
  __syncthreads();
  const double xa = drow(dd, X, n, a), ya = drow(dd, Y, n, a);
  const double s = sqrt(xa * xa + ya * ya);
  spd[i] = s;
  xs[i] = make_double2(xa / s, ya / s);
  nrm[i] = make_double2(ya / s, -xa / s);
  w[i] = s * 2.0 * kPiD / n;
}

// Forces of Algorithm 1 step 2: f_b = -kB x_ssss, f = f_b + (sigma x_s)_s.
__global__ void ves_forces_kernel(int n, const double2 *x, const double *sigma, const double *D,
                                  const double *spd, const double2 *xs, double kb, double2 *fb,
                                  double2 *f) {
  __shared__ double X[kMaxN], Y[kMaxN], TX[kMaxN], TY[kMaxN];
  const int v = blockIdx.x, a = threadIdx.x, i = v * n + a;
  __shared__ double dd[2 * kMaxN];
  load_diff(D, dd, n, a);
  const double s = spd[i];
  X[a] = x[i].x;
  Y[a] = x[i].y;
  __syncthreads();
  for (int r = 0; r < 4; ++r) {  // d/ds four times
    const double dx = drow(dd, X, n, a) / s, dy = drow(dd, Y, n, a) / s;
    __syncthreads();
    X[a] = dx;
    Y[a] = dy;
    __syncthreads();
  }
  const double bx = -kb * X[a], by = -kb * Y[a];
  TX[a] = sigma[i] * xs[i].x;
  TY[a] = sigma[i] * xs[i].y;
  __syncthreads();
  const double sx = drow(dd, TX, n, a) / s, sy = drow(dd, TY, n, a) / s;
  fb[i] = make_double2(bx, by);
  f[i] = make_double2(bx + sx, by + sy);
}

// Matvec, first half: g = dt kB u_ssss - (sigma x_s)_s from z = [u_x, u_y, sigma] per vesicle.
__global__ void ves_mv_pre_kernel(int n, const double *z, const double *D, const double *spd,
                                  const double2 *xs, double dtkb, double2 *g) {
  __shared__ double X[kMaxN], Y[kMaxN], TX[kMaxN], TY[kMaxN];
  const int v = blockIdx.x, a = threadIdx.x, i = v * n + a;
  __shared__ double dd[2 * kMaxN];
  load_diff(D, dd, n, a);
  const double *zv = z + size_t(3) * n * v;
  const double s = spd[i];
  X[a] = zv[a];
  Y[a] = zv[n + a];
  TX[a] = zv[2 * n + a] * xs[i].x;
  TY[a] = zv[2 * n + a] * xs[i].y;
  __syncthreads();
  const double sx = drow(dd, TX, n, a) / s, sy = drow(dd, TY, n, a) / s;
  for (int r = 0; r < 4; ++r) {
    const double dx = drow(dd, X, n, a) / s, dy = drow(dd, Y, n, a) / s;
    __syncthreads();
    X[a] = dx;
    Y[a] = dy;
    __syncthreads();
  }
  g[i] = make_double2(dtkb * X[a] - sx, dtkb * Y[a] - sy);
}

// Matvec, second half: [u + S g; x_s . u_s].
__global__ void ves_mv_post_kernel(int n, const double *z, const double2 *Sg, const double *D,
                                   const double *spd, const double2 *xs, double *out) {
  __shared__ double X[kMaxN], Y[kMaxN];
  const int v = blockIdx.x, a = threadIdx.x, i = v * n + a;
  __shared__ double dd[2 * kMaxN];
  load_diff(D, dd, n, a);
  const double *zv = z + size_t(3) * n * v;
  double *ov = out + size_t(3) * n * v;
  X[a] = zv[a];
  Y[a] = zv[n + a];
  __syncthreads();
  const double s = spd[i];
  const double ux = drow(dd, X, n, a) / s, uy = drow(dd, Y, n, a) / s;
  ov[a] = X[a] + Sg[i].x;
  ov[n + a] = Y[a] + Sg[i].y;
  ov[2 * n + a] = xs[i].x * ux + xs[i].y * uy;
}

// Right-hand side: [S f_b + u_resp; (L0 - Lk) / (dt Lk)] (Eq. (ALC)).
__global__ void ves_rhs_kernel(int n, const double2 *Sfb, const double2 *ures, const double *w,
                               const double *L0, double dt, double *b, double *Lk_out) {
  __shared__ double red[kMaxN];
  const int v = blockIdx.x, a = threadIdx.x, i = v * n + a;
  red[a] = w[i];
  __syncthreads();
  if (a == 0) {
    double L = 0.0;
    for (int k = 0; k < n; ++k) L += red[k];
    red[0] = L;
    Lk_out[v] = L;
  }
  __syncthreads();
  const double Lk = red[0];
  double *bv = b + size_t(3) * n * v;
  bv[a] = Sfb[i].x + (ures ? ures[i].x : 0.0);
  bv[n + a] = Sfb[i].y + (ures ? ures[i].y : 0.0);
  bv[2 * n + a] = (L0[v] - Lk) / (dt * Lk);
}

// Perimeter L = sum w and area A = int x y_alpha of every vesicle (initial values).
__global__ void ves_LA_kernel(int n, const double2 *x, const double *D, const double *w, double *L,
                              double *A) {
  __shared__ double X[kMaxN], Y[kMaxN], P[kMaxN], W[kMaxN];
  const int v = blockIdx.x, a = threadIdx.x, i = v * n + a;
  __shared__ double dd[2 * kMaxN];
  load_diff(D, dd, n, a);
  X[a] = x[i].x;
  Y[a] = x[i].y;
  W[a] = w[i];
  __syncthreads();
  P[a] = X[a] * drow(dd, Y, n, a);
  __syncthreads();
  if (a == 0) {
    double l = 0.0, s = 0.0;
    for (int k = 0; k < n; ++k) {
      l += W[k];
      s += P[k];
    }
    L[v] = l;
    A[v] = s * 2.0 * kPiD / n;
  }
}

// x <- x + dt u, then the area correction of App. B (root of the quadratic closest to 0).
__global__ void ves_advance_kernel(int n, double2 *x, const double *z, const double *D,
                                   const double *A0, double dt) {
  __shared__ double X[kMaxN], Y[kMaxN], XA[kMaxN], YA[kMaxN], P[4][kMaxN];
  __shared__ double cc;
  const int v = blockIdx.x, a = threadIdx.x, i = v * n + a;
  __shared__ double dd[2 * kMaxN];
  load_diff(D, dd, n, a);
  const double *zv = z + size_t(3) * n * v;
  X[a] = x[i].x + dt * zv[a];
  Y[a] = x[i].y + dt * zv[n + a];
  __syncthreads();
  XA[a] = drow(dd, X, n, a);
  YA[a] = drow(dd, Y, n, a);
  __syncthreads();
  const double xaa = drow(dd, XA, n, a);
  P[0][a] = X[a] * YA[a];
  P[1][a] = X[a] * xaa;
  P[2][a] = YA[a] * YA[a];
  P[3][a] = YA[a] * xaa;
  __syncthreads();
  if (a == 0) {
    double I[4] = {0, 0, 0, 0};
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int q = 0; q < 4; ++q) I[q] += P[q][k];
    const double h = 2.0 * kPiD / n;
    const double a0 = I[0] * h - A0[v], a1 = (-I[1] + I[2]) * h, a2 = -I[3] * h;
    double c;
    if (fabs(a2) < 1e-300) {
      c = -a0 / a1;
    } else {
      const double disc = sqrt(fmax(a1 * a1 - 4.0 * a2 * a0, 0.0));
      const double r1 = (-a1 + disc) / (2.0 * a2), r2 = (-a1 - disc) / (2.0 * a2);
      c = fabs(r1) < fabs(r2) ? r1 : r2;
    }
    cc = c;
  }
  __syncthreads();
  x[i] = make_double2(X[a] + cc * YA[a], Y[a] - cc * XA[a]);
}

// App. C, Algorithm 2: nearly equal arc-length nodes (piecewise-linear inversion of s(alpha),
// Fourier interpolation of x at the new parameters).
__global__ void ves_reparam_kernel(int n, double2 *x, const double *D) {
  __shared__ double X[kMaxN], Y[kMaxN], S[kMaxN], Cr[kMaxN], Ci[kMaxN], SJ[kMaxN + 1];
  __shared__ double Xr[kMaxN], Xi[kMaxN], Yr[kMaxN], Yi[kMaxN], AS[kMaxN];
  const int v = blockIdx.x, a = threadIdx.x, i = v * n + a;
  __shared__ double dd[2 * kMaxN];
  load_diff(D, dd, n, a);
  const double h = 2.0 * kPiD / n;
  X[a] = x[i].x;
  Y[a] = x[i].y;
  __syncthreads();
  const double xa = drow(dd, X, n, a), ya = drow(dd, Y, n, a);
  S[a] = sqrt(xa * xa + ya * ya);
  __syncthreads();
  // Fourier coefficients (frequency index a; a > n/2 means a - n) of speed and position
  {
    double cr = 0, ci = 0, xr = 0, xi = 0, yr = 0, yi = 0;
    for (int k = 0; k < n; ++k) {
      double sn, cs;
      sincospi(-2.0 * double((long(a) * k) % n) / n, &sn, &cs);
      cr += S[k] * cs;
      ci += S[k] * sn;
      xr += X[k] * cs;
      xi += X[k] * sn;
      yr += Y[k] * cs;
      yi += Y[k] * sn;
    }
    Cr[a] = cr / n;
    Ci[a] = ci / n;
    Xr[a] = xr / n;
    Xi[a] = xi / n;
    Yr[a] = yr / n;
    Yi[a] = yi / n;
  }
  __syncthreads();
  // s at alpha_a = C0 alpha + sum_{k != 0, n/2} Re[C_k (e^{ik alpha} - 1) / (ik)]
  {
    const double al = h * a;
    double s = Cr[0] * al;
    for (int q = 1; q < n; ++q) {
      if (q == n / 2) continue;
      const int kf = q < n / 2 ? q : q - n;
      double sn, cs;
      sincos(kf * al, &sn, &cs);
      // (C (e - 1)) / (i k) = (Cr + i Ci)((cs - 1) + i sn) / (i k)
      const double re = Cr[q] * (cs - 1.0) - Ci[q] * sn, im = Cr[q] * sn + Ci[q] * (cs - 1.0);
      s += im / kf;  // Re[(re + i im) / (i k)] = im / k
      (void)re;
    }
    SJ[a] = s;
    if (a == 0) SJ[n] = Cr[0] * 2.0 * kPiD;
  }
  __syncthreads();
  if (a == 0) {
    const double total = SJ[n];
    AS[0] = 0.0;
    int j = 0;
    for (int q = 1; q < n; ++q) {
      const double tg = total / n * q;
      while (j < n - 1 && !(SJ[j] <= tg && tg < SJ[j + 1])) ++j;
      AS[q] = h * (j + (tg - SJ[j]) / (SJ[j + 1] - SJ[j]));
    }
  }
  __syncthreads();
  const double al = AS[a];
  double nx = 0.0, ny = 0.0;
  for (int q = 0; q < n; ++q) {
    if (q == n / 2) {
      const double c = cos(0.5 * n * al);
      nx += Xr[q] * c;
      ny += Yr[q] * c;
      continue;
    }
    const int kf = q < n / 2 ? q : q - n;
    double sn, cs;
    sincos(kf * al, &sn, &cs);
    nx += Xr[q] * cs - Xi[q] * sn;
    ny += Yr[q] * cs - Yi[q] * sn;
  }
  x[i] = make_double2(nx, ny);
}

// ---------------------------------------------------------------------------
// block-diagonal preconditioner: per vesicle the self-only operator (3n x 3n, column-major,
// unknown order [u_x, u_y, sigma])
// ---------------------------------------------------------------------------
// Kress self single-layer blocks G_ij (n x n column-major each) and D_s = diag(1/s) D.
template <typename T>
__global__ void pc_parts_kernel(int n, const double2 *x, const double2 *xs, const double *spd,
                                const double *kress, const double *D, double cmu, T *G, T *Ds) {
  const int v = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int a = t % n, k = t / n;  // row a, column k (column-major)
  const int ia = v * n + a, ik = v * n + k;
  const double h = 2.0 * kPiD / n;
  double coef, m11, m12, m22;
  if (a == k) {
    const double s = spd[ia];
    coef = kress[0] - (kPiD / n) * log(s * s);
    const double tx = xs[ia].x, ty = xs[ia].y;
    m11 = tx * tx;
    m12 = tx * ty;
    m22 = ty * ty;
  } else {
    const double rx = x[ia].x - x[ik].x, ry = x[ia].y - x[ik].y, rr = rx * rx + ry * ry;
    int dj = a - k;
    if (dj < 0) dj += n;
    coef = kress[dj] - (kPiD / n) * log(rr);
    m11 = rx * rx / rr;
    m12 = rx * ry / rr;
    m22 = ry * ry / rr;
  }
  const double sk = cmu * spd[ik];
  const size_t nn = size_t(n) * n, base = size_t(v) * 4 * nn + t;
  G[base + 0 * nn] = T((coef + h * m11) * sk);  // G_11
  G[base + 1 * nn] = T((h * m12) * sk);         // G_12
  G[base + 2 * nn] = T((h * m12) * sk);         // G_21
  G[base + 3 * nn] = T((coef + h * m22) * sk);  // G_22
  Ds[size_t(v) * nn + t] = T(D[size_t(a) * n + k] / spd[ia]);
}

// T_c = D_s diag(x_s,c)  (c = 0, 1), stored as two n x n blocks per vesicle.
template <typename F>
__global__ void pc_T_kernel(int n, const F *Ds, const double2 *xs, F *T) {
  const int v = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int k = t / n;
  const size_t nn = size_t(n) * n;
  const double d = Ds[size_t(v) * nn + t];
  T[size_t(v) * 2 * nn + t] = F(d * xs[v * n + k].x);
  T[size_t(v) * 2 * nn + nn + t] = F(d * xs[v * n + k].y);
}

// Fill the constraint rows [diag(x_s,1) D_s, diag(x_s,2) D_s, 0] and add the identity of the
// u block.
template <typename F>
__global__ void pc_fill_kernel(int n, const F *Ds, const double2 *xs, F *P) {
  const int v = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = 3 * n;
  if (t >= m * n) return;
  const int row = 2 * n + t % n, col = t / n;  // constraint rows, all 3n columns
  const size_t mm = size_t(m) * m;
  F *Pv = P + size_t(v) * mm;
  const int a = row - 2 * n;
  double val = 0.0;
  if (col < 2 * n) {
    const int c = col / n, k = col % n;
    const double xsc = c == 0 ? xs[v * n + a].x : xs[v * n + a].y;
    val = xsc * double(Ds[size_t(v) * n * n + size_t(k) * n + a]);
  }
  Pv[row + size_t(col) * m] = F(val);
  if (t < 2 * n) Pv[t + size_t(t) * m] += F(1.0);
}

// ---------------------------------------------------------------------------
// warm-start features, targets and guesses (per vesicle, principal-axes frame)
// ---------------------------------------------------------------------------
// Fourier modes of the warm-start representation: nm modes k = -nm/2 .. nm/2 - 1 of the shape
// and of the change of the explicit velocity (features: 4 nm reals), nm modes of the change of
// u and the modes k = 0 .. nm/2 - 1 of the change of sigma (targets: 3 nm reals).  nm is even,
// in [4, kMaxModes] and at most the nodes per vesicle (16 by default; 32 in the paper-scale
// workload definition).
constexpr int kDefaultModes = 16;
constexpr int kMaxModes = 64;
__host__ __device__ inline int targ_dim(int nm) { return 3 * nm; }
// features: shape and velocity-change modes (4 nm), with history also the previous solution and
// the previous step's change of it in the target representation (2 x 3 nm)
__host__ __device__ inline int feat_dim(int nm, bool hist = false) {
  return 4 * nm + (hist ? 2 * targ_dim(nm) : 0);
}

// Frame of one vesicle from its nodes in shared memory: centre, angle of the second moments'
// major axis, length l = sqrt(A0 / pi), velocity scale U = kB / (mu l^2), tension scale kB / l^2.
__device__ void vesicle_frame(int n, const double *X, const double *Y, double A0, double kb,
                              double mu, double *fr) {
  double cx = 0, cy = 0;
  for (int k = 0; k < n; ++k) {
    cx += X[k];
    cy += Y[k];
  }
  cx /= n;
  cy /= n;
  double sxx = 0, sxy = 0, syy = 0;
  for (int k = 0; k < n; ++k) {
    const double dx = X[k] - cx, dy = Y[k] - cy;
    sxx += dx * dx;
    sxy += dx * dy;
    syy += dy * dy;
  }
  const double th = 0.5 * atan2(2.0 * sxy, sxx - syy);
  const double l = sqrt(A0 / kPiD);
  fr[0] = cx;
  fr[1] = cy;
  fr[2] = th;
  fr[3] = l;
  fr[4] = kb / (mu * l * l);
  fr[5] = kb / (l * l);
}

// (1/n) sum_a (re_a + i im_a) e^{-i k alpha_a}
__device__ void dft_mode(int n, int k, const double *re, const double *im, double *out) {
  double sr = 0, si = 0;
  for (int a = 0; a < n; ++a) {
    double sn, cs;
    sincospi(-2.0 * double(((long(k) * a) % n + n) % n) / n, &sn, &cs);
    sr += re[a] * cs - im[a] * sn;
    si += re[a] * sn + im[a] * cs;
  }
  out[0] = sr / n;
  out[1] = si / n;
}

// Modes of a solution-like vector (u_x, u_y, sigma per node, staged as frame-rotated u / U in
// (UR, UI) and sigma / (kappa_B / l^2) in SG) in the target representation, written to out.
__device__ void solution_modes(int n, int nm, int a, const double *UR, const double *UI,
                               const double *SG, const double *ZERO, float *out) {
  for (int q = a; q < nm + nm / 2; q += n) {
    double o[2];
    if (q < nm) {
      dft_mode(n, q - nm / 2, UR, UI, o);
      out[2 * q] = float(o[0]);
      out[2 * q + 1] = float(o[1]);
    } else {
      dft_mode(n, q - nm, SG, ZERO, o);
      out[2 * nm + 2 * (q - nm)] = float(o[0]);
      out[2 * nm + 2 * (q - nm) + 1] = float(o[1]);
    }
  }
}

__global__ void ves_features_kernel(int n, int nm, const double2 *x, const double *b,
                                    const double *bprev, const double *zprev,
                                    const double *zprev2, int two_back, const double *A0,
                                    double kb, double mu, double *frame, float *feat) {
  __shared__ double X[kMaxN], Y[kMaxN], ZR[kMaxN], ZI[kMaxN], WR[kMaxN], WI[kMaxN];
  __shared__ double fr[6];
  const int v = blockIdx.x, a = threadIdx.x, i = v * n + a;
  X[a] = x[i].x;
  Y[a] = x[i].y;
  __syncthreads();
  if (a == 0) vesicle_frame(n, X, Y, A0[v], kb, mu, fr);
  __syncthreads();
  const double c = cos(fr[2]), s = sin(fr[2]);
  const double dx = X[a] - fr[0], dy = Y[a] - fr[1];
  ZR[a] = (c * dx + s * dy) / fr[3];
  ZI[a] = (-s * dx + c * dy) / fr[3];
  const double *bv = b + size_t(3) * n * v, *pv = bprev + size_t(3) * n * v;
  const double dbx = bv[a] - pv[a], dby = bv[n + a] - pv[n + a];
  WR[a] = (c * dbx + s * dby) / fr[4];
  WI[a] = (-s * dbx + c * dby) / fr[4];
  __syncthreads();
  const bool hist = zprev != nullptr;
  const int F = feat_dim(nm, hist);
  float *fv = feat + size_t(v) * F;
  for (int q = a; q < nm; q += n) {
    double o[2];
    dft_mode(n, q - nm / 2, ZR, ZI, o);
    fv[2 * q] = float(o[0]);
    fv[2 * q + 1] = float(o[1]);
    dft_mode(n, q - nm / 2, WR, WI, o);
    fv[2 * nm + 2 * q] = float(o[0]);
    fv[2 * nm + 2 * q + 1] = float(o[1]);
  }
  if (hist) {
    // the previous solution, then its change over the previous step, in this step's frame
    const double *z1 = zprev + size_t(3) * n * v, *z2 = zprev2 + size_t(3) * n * v;
    for (int pass = 0; pass < 2; ++pass) {
      __syncthreads();  // ZR..WI are reused as the staging arrays
      // the previous change needs two solutions in the history; with fewer it is zero
      const double g = pass ? double(two_back) : 0.0;
      const double ux = z1[a] - g * z2[a] - (pass && !two_back ? z1[a] : 0.0);
      const double uy = z1[n + a] - g * z2[n + a] - (pass && !two_back ? z1[n + a] : 0.0);
      ZR[a] = (c * ux + s * uy) / fr[4];
      ZI[a] = (-s * ux + c * uy) / fr[4];
      WR[a] = (z1[2 * n + a] - g * z2[2 * n + a] - (pass && !two_back ? z1[2 * n + a] : 0.0)) / fr[5];
      WI[a] = 0.0;
      __syncthreads();
      solution_modes(n, nm, a, ZR, ZI, WR, WI, fv + 4 * nm + pass * targ_dim(nm));
    }
  }
  if (a < 6) frame[v * 6 + a] = fr[a];
}

// Base guess of the learned warm start at node component j of vesicle v: z_prev, plus the
// previous change z_prev - z_prev2 when extrapolating (ext = 1).
__device__ __forceinline__ double base_guess(const double *zp, const double *zp2, int ext,
                                             size_t j) {
  return ext ? 2.0 * zp[j] - zp2[j] : zp[j];
}

// Targets: modes of z - (base guess) in the vesicle's frame.
__global__ void ves_targets_kernel(int n, int nm, const double *z, const double *zprev,
                                   const double *zprev2, int ext, const double *frame,
                                   float *targ) {
  __shared__ double UR[kMaxN], UI[kMaxN], SG[kMaxN], ZERO[kMaxN];
  const int v = blockIdx.x, a = threadIdx.x;
  const double *fr = frame + v * 6;
  const double c = cos(fr[2]), s = sin(fr[2]);
  const size_t o = size_t(3) * n * v;
  const double *zv = z + o;
  const double dux = zv[a] - base_guess(zprev, zprev2, ext, o + a);
  const double duy = zv[n + a] - base_guess(zprev, zprev2, ext, o + n + a);
  UR[a] = (c * dux + s * duy) / fr[4];
  UI[a] = (-s * dux + c * duy) / fr[4];
  SG[a] = (zv[2 * n + a] - base_guess(zprev, zprev2, ext, o + 2 * n + a)) / fr[5];
  ZERO[a] = 0.0;
  __syncthreads();
  solution_modes(n, nm, a, UR, UI, SG, ZERO, targ + size_t(v) * targ_dim(nm));
}

// Inverse of the targets' representation: z = z_prev + (predicted change at the nodes).
__global__ void ves_guess_kernel(int n, int nm, const float *pred, const double *frame,
                                 const double *zprev, const double *zprev2, int ext, double *z) {
  const int v = blockIdx.x, a = threadIdx.x;
  const double *fr = frame + v * 6;
  const float *p = pred + size_t(v) * targ_dim(nm);
  const double al = 2.0 * kPiD * a / n;
  double ur = 0, ui = 0, sg = 0;
  for (int q = 0; q < nm; ++q) {
    double sn, cs;
    sincos((q - nm / 2) * al, &sn, &cs);
    ur += p[2 * q] * cs - p[2 * q + 1] * sn;
    ui += p[2 * q] * sn + p[2 * q + 1] * cs;
  }
  const float *ps = p + 2 * nm;
  for (int q = 0; q < nm / 2; ++q) {
    double sn, cs;
    sincos(q * al, &sn, &cs);
    sg += (q == 0 ? 1.0 : 2.0) * (ps[2 * q] * cs - ps[2 * q + 1] * sn);
  }
  const double c = cos(fr[2]), s = sin(fr[2]);
  const size_t o = size_t(3) * n * v;
  double *zv = z + o;
  zv[a] = base_guess(zprev, zprev2, ext, o + a) + fr[4] * (c * ur - s * ui);
  zv[n + a] = base_guess(zprev, zprev2, ext, o + n + a) + fr[4] * (s * ur + c * ui);
  zv[2 * n + a] = base_guess(zprev, zprev2, ext, o + 2 * n + a) + fr[5] * sg;
}

// z = 2 z_prev - z_prev2 (linear extrapolation of the last two solutions).
__global__ void extrapolate_kernel(long len, const double *zprev, const double *zprev2, double *z) {
  for (long i = blockIdx.x * long(blockDim.x) + threadIdx.x; i < len; i += long(gridDim.x) * blockDim.x)
    z[i] = 2.0 * zprev[i] - zprev2[i];
}

__global__ void extract_sigma_kernel(int n, const double *z, double *sigma) {
  const int v = blockIdx.x, a = threadIdx.x;
  sigma[v * n + a] = z[size_t(3) * n * v + 2 * n + a];
}

__global__ void set_ptrs_kernel(int count, double *base, size_t stride, double **ptrs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) ptrs[t] = base + stride * t;
}

__global__ void set_ptrs32_kernel(int count, float *base, size_t stride, float **ptrs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) ptrs[t] = base + stride * t;
}

// zout_v = Pinv32_v zin_v for every vesicle v (one block each, k = 3n rows, column-major k x k
// blocks), products and sums in FP64: the FP32-stored inverse acts as a fixed FP64 operator.
// zout = Pinv zin per vesicle (k x k FP32 blocks, column-major; a CTA per vesicle).  Each
// product b z_j with the FP32 entry b and the FP64 z_j = z_h + z_l split into floats is formed
// as b z_h exactly (FMA) plus b z_l and added into a double-float accumulator, on the FP32
// pipes (~1e-14 relative, the FP64 operator to that accuracy); eight coalesced column loads
// are in flight per thread (the block is read once from HBM).
__global__ void precond32_apply_kernel(int k, const float *Pinv, const double *zin, double *zout) {
  extern __shared__ float2 zs2[];  // z split: (h, l)
  const size_t off = size_t(blockIdx.x) * k;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const df z = split_df(zin[off + j]);
    zs2[j] = make_float2(z.h, z.l);
  }
  __syncthreads();
  const float *B = Pinv + size_t(blockIdx.x) * k * k;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    df acc[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    int j = 0;
    for (; j + 7 < k; j += 8) {
      float b[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) b[u] = B[i + size_t(j + u) * k];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float2 z = zs2[j + u];
        df_mul_acc(acc[u & 1], {b[u], 0.0f}, {z.x, z.y});
      }
      df_renorm(acc[0]);
      df_renorm(acc[1]);
    }
    for (; j < k; ++j) {
      const float2 z = zs2[j];
      df_mul_acc(acc[0], {B[i + size_t(j) * k], 0.0f}, {z.x, z.y});
    }
    zout[off + i] = (double(acc[0].h) + double(acc[0].l)) + (double(acc[1].h) + double(acc[1].l));
  }
}

// Sum of squares of x (len), in fixed order: block b sums the elements b * 256 + t, + grid
// stride, reduced in shared memory; nrm_finish_kernel adds the kNrmBlocks partials in order.
constexpr int kNrmBlocks = 256;
__global__ void nrm_partial_kernel(long len, const double *x, double *part) {
  __shared__ double red[256];
  double a = 0.0;
  for (long i = long(blockIdx.x) * 256 + threadIdx.x; i < len; i += long(kNrmBlocks) * 256)
    a = fma(x[i], x[i], a);
  red[threadIdx.x] = a;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void nrm_finish_kernel(double *part) {
  __shared__ double red[kNrmBlocks];
  red[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int st = kNrmBlocks / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[0] = red[0];
}

// Newton-Schulz step of the preconditioner inverse: T = P X (per vesicle, k x k) is replaced in
// place by W = 2I - T = I + E with E = I - T, and the largest per-vesicle ||E||_F goes to *enorm
// (the bits of a non-negative float order as unsigned integers).  A CTA per vesicle.
__global__ void ns_prepare_kernel(int k, float *T, unsigned *enorm) {
  __shared__ float red[256];
  const size_t kk = size_t(k) * k;
  float *Tv = T + size_t(blockIdx.x) * kk;
  float acc = 0.0f;
  for (size_t i = threadIdx.x; i < kk; i += blockDim.x) {
    const float d = (i % size_t(k + 1)) == 0 ? 1.0f : 0.0f;
    const float e = d - Tv[i];
    acc = fmaf(e, e, acc);
    Tv[i] = d + e;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(enorm, __float_as_uint(sqrtf(red[0])));
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
// Gauss-Legendre nodes on [-1, 1] (Newton iteration on the Legendre recurrence).
std::vector<double> gauss_legendre(int K) {
  std::vector<double> x(K);
  for (int i = 0; i < K; ++i) {
    double z = cos(kPiD * (i + 0.75) / (K + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= K; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double dp = K * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[K - 1 - i] = z;
  }
  return x;
}

int set_stream_handles(stokes_sim *m) {
  BK(cublasSetStream(m->blas, m->s));
  QK(cusolverDnSetStream(m->sol, m->s));
  return STOKES_OK;
}

__global__ void d2f_kernel(size_t n, const double *a, float *b) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    b[i] = __double2float_rn(a[i]);
}

__global__ void add_f2d_kernel(size_t n, const float *a, double *b) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    b[i] += double(a[i]);
}

// Blocks of a 256-thread grid-stride launch over n elements: one per 256 elements, at most
// 32 per SM of the current device.
inline int grid_for(size_t n) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 1;
  return int(std::max<size_t>(1, std::min<size_t>((n + 255) / 256, size_t(sms) * 32)));
}

__global__ void identity_f32_kernel(int64_t n, float *a) {
  const size_t nn = size_t(n) * size_t(n);
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < nn; i += size_t(gridDim.x) * blockDim.x)
    a[i] = (i % size_t(n + 1) == 0) ? 1.0f : 0.0f;
}

// X (nA x nrhs, column-major) <- A^-1 X.  FP64 LU: one getrs.  FP32 inverse + refinement:
// starting from x = 0 and r = b, repeat  x += A32^-1 r (FP32 GEMV / GEMM of the FP32-rounded
// residual; A32^-1 is the inverse of the FP32-rounded A, formed once from its LU),
// r = b - A x (FP64 GEMV / GEMM with the FP64 A)  until ||r|| <= 1e-14 ||b||, the residual stops
// shrinking (its FP64 rounding floor), or 12 sweeps.  A = -I/2 + D is a second-kind operator
// with a small condition number, so each sweep gains about five digits; every sweep streams
// the two dense matrices once instead of running latency-bound triangular solves.
int wall_solve(stokes_sim *m, double *X, int nrhs, int max_sweeps = 12) {
  const int64_t nA = m->nA;
  if (m->walls_mode == STOKES_WALLS_FDS) {  // direct: HBS + SMW, no residual check
    const int st = stokes::fds_solve(m->fds, X, nrhs, m->s, m->blas, m->err);
    m->wall_refinements = 0;
    m->wall_residual = -1.0;
    return st;
  }
  if (m->walls_mode == STOKES_WALLS_LU64) {
    QK(cusolverDnDgetrs(m->sol, CUBLAS_OP_N, m->nA, nrhs, m->d_LU, m->nA, m->d_piv, X, m->nA,
                        m->d_info));
    m->wall_refinements = 0;
    m->wall_residual = 0.0;
    return STOKES_OK;
  }
  const size_t len = size_t(nA) * nrhs;
  if (len > m->wall_ws_len) {
    SK(dalloc(m->d_wb, len));
    SK(dalloc(m->d_wr, len));
    SK(dalloc(m->d_wr32, len));
    SK(dalloc(m->d_wb32, len));
    m->wall_ws_len = len;
  }
  SK(cudaMemcpyAsync(m->d_wb, X, sizeof(double) * len, cudaMemcpyDeviceToDevice, m->s));
  SK(cudaMemcpyAsync(m->d_wr, X, sizeof(double) * len, cudaMemcpyDeviceToDevice, m->s));
  SK(cudaMemsetAsync(X, 0, sizeof(double) * len, m->s));
  double bn = 0.0;
  BK(cublasDnrm2_64(m->blas, int64_t(len), m->d_wb, 1, &bn));
  m->wall_refinements = 0;
  m->wall_residual = 0.0;
  if (!(bn > 0.0)) return STOKES_OK;
  const double one = 1.0, mone = -1.0;
  double prev = 1e300;
  for (int it = 0; it < max_sweeps; ++it) {
    d2f_kernel<<<grid_for(len), 256, 0, m->s>>>(len, m->d_wr, m->d_wr32);
    const float fone = 1.0f, fzero = 0.0f;
    float *corr = reinterpret_cast<float *>(m->d_wb32);
    if (nrhs == 1)
      BK(cublasSgemv_64(m->blas, CUBLAS_OP_N, nA, nA, &fone, m->d_Ainv32, nA, m->d_wr32, 1, &fzero,
                        corr, 1));
    else
      BK(cublasSgemm_64(m->blas, CUBLAS_OP_N, CUBLAS_OP_N, nA, nrhs, nA, &fone, m->d_Ainv32, nA,
                        m->d_wr32, nA, &fzero, corr, nA));
    add_f2d_kernel<<<grid_for(len), 256, 0, m->s>>>(len, corr, X);
    SK(cudaGetLastError());
    if (it + 1 == max_sweeps && max_sweeps < 12) {  // an inner solve: no residual check
      m->wall_refinements = it + 1;
      m->wall_residual = -1.0;
      break;
    }
    SK(cudaMemcpyAsync(m->d_wr, m->d_wb, sizeof(double) * len, cudaMemcpyDeviceToDevice, m->s));
    if (nrhs == 1)
      BK(cublasDgemv_64(m->blas, CUBLAS_OP_N, nA, nA, &mone, m->d_A, nA, X, 1, &one, m->d_wr, 1));
    else
      BK(cublasDgemm_64(m->blas, CUBLAS_OP_N, CUBLAS_OP_N, nA, nrhs, nA, &mone, m->d_A, nA, X, nA,
                        &one, m->d_wr, nA));
    double rn = 0.0;
    BK(cublasDnrm2_64(m->blas, int64_t(len), m->d_wr, 1, &rn));
    m->wall_refinements = it + 1;
    m->wall_residual = rn / bn;
    if (!(rn == rn)) return fail(m, STOKES_ERR_NONFINITE, "wall solve: non-finite residual");
    if (rn <= 1e-14 * bn || rn > 0.5 * prev) break;
    prev = rn;
  }
  return STOKES_OK;
}

// Block elimination of Sec. 4.1 for data (v, g): y = A^-1 v, c = S^+ (g - C y), tau = y - W c.
// Under the block refinement the wall solve is a single FP32-inverse sweep (the outer
// residual corrections make up its ~1e-5 error along with the truncation of S^+).
int block_solve(stokes_sim *m, const double *v, const double *g, double *tau, double *c) {
  const double one = 1.0, mone = -1.0, zero = 0.0;
  SK(cudaMemcpyAsync(tau, v, sizeof(double) * m->nA, cudaMemcpyDeviceToDevice, m->s));
  ST(wall_solve(m, tau, 1, m->block_refine > 0 ? 1 : 12));
  SK(cudaMemcpyAsync(m->d_g2, g, sizeof(double) * 4 * m->K, cudaMemcpyDeviceToDevice, m->s));
  BK(cublasDgemv(m->blas, CUBLAS_OP_N, 4 * m->K, m->nA, &mone, m->d_C, 4 * m->K, tau, 1, &one,
                 m->d_g2, 1));
  BK(cublasDgemv(m->blas, CUBLAS_OP_N, 2 * m->M, 4 * m->K, &one, m->d_Spinv, 2 * m->M, m->d_g2, 1,
                 &zero, c, 1));
  BK(cublasDgemv(m->blas, CUBLAS_OP_N, m->nA, 2 * m->M, &mone, m->d_W, m->nA, c, 1, &one, tau, 1));
  return STOKES_OK;
}

// The block solve for (d_rv, d_rg) into (d_tau, d_c), then block_refine residual corrections
// on the whole extended system [A B; C Q]:  r = [v; g] - [A B; C Q][tau; c],
// [tau; c] += block solve of r.  The truncated pseudo-inverse S^+ leaves a residual in the
// side-point rows (~1e-6 of the data) and the single-sweep wall solves ~1e-5; each correction
// shrinks both by about five digits, so three reach round-off.  A tau is the walls'
// double-layer sum with the interior jump -1/2 (the same operator as the assembled A), in
// `prec` (FP64 or double-float).
// The walls' FMM plan at `order` (kept across steps: the walls do not move).
int wall_fmm(stokes_sim *m, int order) {
  if (m->fmm_w && m->fmm_w_order == order) return STOKES_OK;
  if (m->fmm_w) stokes_fmm_destroy(m->fmm_w);
  m->fmm_w = nullptr;
  m->fmm_w_order = 0;
  SK(cudaStreamSynchronize(m->s));
  const int st = stokes_fmm_create(m->ctx_w, order, m->resid_fmm_leaf, &m->fmm_w);
  if (st) return fail(m, st, "FMM plan of the walls failed (%s)", m->ctx_w->err.c_str());
  m->fmm_w_order = order;
  return STOKES_OK;
}

// Block solve of the extended system, then block_refine residual corrections on the whole
// system; the wall double-layer sums of the residuals in `prec`, or by the walls' FMM plan of
// order fmm_order (> 0).
int refined_block_solve(stokes_sim *m, int prec, int fmm_order = 0) {
  ST(block_solve(m, m->d_rv, m->d_rg, m->d_tau, m->d_c));
  const double one = 1.0, mone = -1.0;
  if (fmm_order > 0 && m->block_refine > 0) ST(wall_fmm(m, fmm_order));
  for (int k = 0; k < m->block_refine; ++k) {
    if (fmm_order > 0) {
      const int st = stokes_fmm_eval(m->fmm_w, nullptr, m->d_tau, -0.5, m->d_resv, m->s);
      if (st) {
        char buf[256];
        stokes_fmm_last_error(m->fmm_w, buf, sizeof(buf));
        return fail(m, st, "FMM wall sum: %s", buf);
      }
    } else {
      ST(stokes_sum_eval(m->ctx_w, prec, nullptr, m->d_tau, -0.5, m->d_resv, m->s));
    }
    axpby_kernel<<<nb(m->nA, 256), 256, 0, m->s>>>(m->nA, 1.0, m->d_rv, -1.0, m->d_resv);
    BK(cublasDgemv(m->blas, CUBLAS_OP_N, m->nA, 2 * m->M, &mone, m->d_B, m->nA, m->d_c, 1, &one,
                   m->d_resv, 1));
    SK(cudaMemcpyAsync(m->d_resg, m->d_rg, sizeof(double) * 4 * m->K, cudaMemcpyDeviceToDevice, m->s));
    BK(cublasDgemv(m->blas, CUBLAS_OP_N, 4 * m->K, m->nA, &mone, m->d_C, 4 * m->K, m->d_tau, 1, &one,
                   m->d_resg, 1));
    BK(cublasDgemv(m->blas, CUBLAS_OP_N, 4 * m->K, 2 * m->M, &mone, m->d_Q, 4 * m->K, m->d_c, 1, &one,
                   m->d_resg, 1));
    ST(block_solve(m, m->d_resv, m->d_resg, m->d_dtau, m->d_dc));
    axpby_kernel<<<nb(m->nA, 256), 256, 0, m->s>>>(m->nA, 1.0, m->d_dtau, 1.0, m->d_tau);
    axpby_kernel<<<nb(2 * m->M, 256), 256, 0, m->s>>>(2 * m->M, 1.0, m->d_dc, 1.0, m->d_c);
    SK(cudaGetLastError());
  }
  return STOKES_OK;
}

// Channel response to vesicle forces f (device, Nv x 2): u_resp at the vesicle nodes.  The
// pair sums run in `prec` (STOKES_FP64 or the equally accurate STOKES_DOUBLE_FLOAT).
// The free-target evaluation of a response plan (fmm_vw, fmm_wv), as fmm_sum.
int fmm_targets(stokes_sim *m, stokes_fmm *f, const double *slp, const double *dlp, double *out,
                const char *what) {
  const int st = stokes_fmm_eval_targets(f, slp, dlp, out, m->s);
  if (st) {
    char buf[256];
    stokes_fmm_last_error(f, buf, sizeof(buf));
    return fail(m, st, "%s: %s", what, buf);
  }
  return STOKES_OK;
}

int channel_response(stokes_sim *m, const double2 *f, double p_drive, double2 *u_out,
                     int prec = STOKES_FP64, int fmm_order = 0) {
  const double cmu = 1.0 / (4.0 * kPiD * m->mu);
  // v = -S^near f at the wall nodes (vesicle sums at free targets)
  if (fmm_order > 0 && m->fmm_vw)
    ST(fmm_targets(m, m->fmm_vw, reinterpret_cast<const double *>(f), nullptr, m->d_vrhs,
                   "FMM vesicle-to-wall sum"));
  else
    ST(stokes_sum_eval_targets(m->ctx_v, prec, reinterpret_cast<const double *>(f), nullptr,
                               m->Nt, reinterpret_cast<const double *>(m->d_wx), m->d_vrhs, m->s));
  side_rhs_kernel<<<dim3(m->K, kSideChunks), 256, 0, m->s>>>(m->K, m->Nv, m->d_side, m->d_x, m->d_w,
                                                            f, m->period, cmu, m->d_side_part);
  side_rhs_finish_kernel<<<nb(m->K, 128), 128, 0, m->s>>>(m->K, m->d_side_part, p_drive, m->d_rg);
  // v = -(S^near f) at the walls
  axpby_kernel<<<nb(m->nA, 256), 256, 0, m->s>>>(m->nA, -1.0, m->d_vrhs, 0.0, m->d_rv);
  SK(cudaGetLastError());
  ST(refined_block_solve(m, prec, fmm_order));
  // u_resp = D^near tau + sum_m c_m S(., y_m) at the vesicle nodes
  if (fmm_order > 0 && m->fmm_wv)
    ST(fmm_targets(m, m->fmm_wv, nullptr, m->d_tau, reinterpret_cast<double *>(u_out),
                   "FMM wall-to-vesicle sum"));
  else
    ST(stokes_sum_eval_targets(m->ctx_w, prec, nullptr, m->d_tau, m->Nv,
                               reinterpret_cast<const double *>(m->d_x),
                               reinterpret_cast<double *>(u_out), m->s));
  proxy_eval_kernel<<<nb(m->Nv, 128), 128, 0, m->s>>>(m->Nv, m->d_x, m->M, m->d_proxy, m->d_c,
                                                      cmu, u_out);
  SK(cudaGetLastError());
  return STOKES_OK;
}

// With close evaluation on: out (the vesicle node sum of density f) += the close correction.
int add_close(stokes_sim *m, const double2 *f, double2 *out) {
  if (!m->close_v) return STOKES_OK;
  const int st = stokes_close_eval(m->close_v, reinterpret_cast<const double *>(f),
                                   reinterpret_cast<double *>(out), m->s);
  if (st) {
    char buf[256];
    stokes_close_last_error(m->close_v, buf, sizeof(buf));
    return fail(m, st, "close evaluation: %s", buf);
  }
  return STOKES_OK;
}

// The vesicle sum of `dens` by the step's FMM plan at `order`, in FP64 or (for the low-order
// sweeps, whose truncation error is ~1e-7 and above) in FP32.
int fmm_sum(stokes_sim *m, int order, bool fp32, const double2 *dens, double2 *out,
            const char *what) {
  int st = stokes_fmm_set_eval_order(m->fmm_v, order);
  if (!st) st = stokes_fmm_set_precision(m->fmm_v, fp32 ? STOKES_FP32_KAHAN : STOKES_FP64);
  if (!st)
    st = stokes_fmm_eval(m->fmm_v, reinterpret_cast<const double *>(dens), nullptr, 0.0,
                         reinterpret_cast<double *>(out), m->s);
  if (st) {
    char buf[256];
    stokes_fmm_last_error(m->fmm_v, buf, sizeof(buf));
    return fail(m, st, "%s: %s", what, buf);
  }
  return STOKES_OK;
}

// Sweep evaluations up to this order (truncation error ~1e-7 and above) run in FP32.
constexpr int kSweepFp32MaxOrder = 16;

// z_out = A z_in (the operator of Eq. (tsteplinsys) at the current positions).  FP32-Kahan
// sums are the sweeps' operator: with sweep_fmm_order set they come from the step's FMM plan
// at that order instead.
int step_matvec(stokes_sim *m, double dt, int precision, const double *zin, double *zout) {
  ves_mv_pre_kernel<<<m->V, m->n, 0, m->s>>>(m->n, zin, m->d_D, m->d_spd, m->d_xs, dt * m->kappa_b,
                                             m->d_tmp2);
  SK(cudaGetLastError());
  if (precision == STOKES_FP32_KAHAN && m->sweep_fmm_order > 0 && m->fmm_v)
    ST(fmm_sum(m, m->sweep_fmm_order, m->sweep_fmm_order <= kSweepFp32MaxOrder, m->d_tmp2,
               m->d_tmp3, "FMM sweep"));
  else
    ST(stokes_sum_eval(m->ctx_v, precision, reinterpret_cast<const double *>(m->d_tmp2), nullptr,
                       0.0, reinterpret_cast<double *>(m->d_tmp3), m->s));
  ST(add_close(m, m->d_tmp2, m->d_tmp3));
  ves_mv_post_kernel<<<m->V, m->n, 0, m->s>>>(m->n, zin, m->d_tmp3, m->d_D, m->d_spd, m->d_xs,
                                              zout);
  SK(cudaGetLastError());
  return STOKES_OK;
}

// step_matvec with the vesicle sum by the step's FMM plan (FP64 expansions of order
// resid_fmm_order: FP64-accurate to the expansion error).
int step_matvec_fmm(stokes_sim *m, double dt, const double *zin, double *zout) {
  ves_mv_pre_kernel<<<m->V, m->n, 0, m->s>>>(m->n, zin, m->d_D, m->d_spd, m->d_xs, dt * m->kappa_b,
                                             m->d_tmp2);
  SK(cudaGetLastError());
  ST(fmm_sum(m, m->resid_fmm_order, false, m->d_tmp2, m->d_tmp3, "FMM residual"));
  ST(add_close(m, m->d_tmp2, m->d_tmp3));
  ves_mv_post_kernel<<<m->V, m->n, 0, m->s>>>(m->n, zin, m->d_tmp3, m->d_D, m->d_spd, m->d_xs,
                                              zout);
  SK(cudaGetLastError());
  return STOKES_OK;
}

// The FMM plan of the vesicles' current geometry, built by a host thread while the stream
// runs the step's other work (the plan reads the geometry with synchronous copies, so the
// geometry update must be complete when it starts).  The destructor joins the thread and
// destroys a plan nobody took.
struct FmmPlanJob {
  std::thread th;
  stokes_fmm *plan = nullptr;
  int status = STOKES_OK;
  double ms = 0.0;
  // A plan of ctx at `order`; when n_extra > 0, one whose only targets are n_extra free
  // points (device).
  void start(stokes_sim *m, stokes_ctx *ctx, int order, int n_extra = 0,
             const double *extra = nullptr) {
    th = std::thread([this, m, ctx, order, n_extra, extra] {
      const auto t0 = std::chrono::steady_clock::now();
      if (cudaSetDevice(m->device) != cudaSuccess) {
        status = STOKES_ERR_CUDA;
        return;
      }
      status = n_extra > 0
                   ? stokes_fmm_create_targets_only(ctx, order, m->resid_fmm_leaf, n_extra, extra, &plan)
                   : stokes_fmm_create(ctx, order, m->resid_fmm_leaf, &plan);
      ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    });
  }
  int join() {
    if (th.joinable()) th.join();
    return status;
  }
  stokes_fmm *take() {
    stokes_fmm *p = plan;
    plan = nullptr;
    return p;
  }
  ~FmmPlanJob() {
    join();
    if (plan) stokes_fmm_destroy(plan);
  }
};

int precond_apply(stokes_sim *m, const double *zin, double *zout) {
  const int k = 3 * m->n;
  if (m->precond_fp32) {
    precond32_apply_kernel<<<m->V, std::min(k, 1024), sizeof(float2) * k, m->s>>>(k, m->d_Pinv32,
                                                                                  zin, zout);
    SK(cudaGetLastError());
    return STOKES_OK;
  }
  const double one = 1.0, zero = 0.0;
  BK(cublasDgemvStridedBatched(m->blas, CUBLAS_OP_N, k, k, &one, m->d_Pinv, k, size_t(k) * k, zin, 1,
                               k, &zero, zout, 1, k, m->V));
  return STOKES_OK;
}

// The preconditioner's 3n x 3n blocks [I + dt kB G D4, -(G_1 T_1 + G_2 T_2); x_s . D_s, 0] per
// vesicle.  With an FP32 factorization (the default) they are assembled in FP32 as well
// (SGEMMs; the FP64 buffers hold the FP32 factors), since only the factors' inverse is used and
// it is a fixed operator either way; with FP64 factors, in FP64.
template <typename F>
int precond_assemble(stokes_sim *m, double dt, F *G, F *Ds, F *D2, F *D4, F *T, F *P) {
  const int n = m->n, V = m->V, k = 3 * n;
  const size_t nn = size_t(n) * n, kk = size_t(k) * k;
  const double cmu = 1.0 / (4.0 * kPiD * m->mu);
  dim3 g2(nb(n * n, 256), V);
  pc_parts_kernel<F><<<g2, 256, 0, m->s>>>(n, m->d_x, m->d_xs, m->d_spd, m->d_kress, m->d_D, cmu, G, Ds);
  SK(cudaGetLastError());
  const F one = F(1), zero = F(0), mone = F(-1), dtkb = F(dt * m->kappa_b);
  auto gemm = [&](const F *alpha, const F *A, int lda, long long sa, const F *B, int ldb,
                  long long sb, const F *beta, F *C, int ldc, long long sc) {
    if constexpr (sizeof(F) == 8)
      return cublasDgemmStridedBatched(m->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, alpha, A, lda, sa,
                                       B, ldb, sb, beta, C, ldc, sc, V);
    else
      return cublasSgemmStridedBatched(m->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, alpha, A, lda, sa,
                                       B, ldb, sb, beta, C, ldc, sc, V);
  };
  // D2 = Ds Ds, D4 = D2 D2
  BK(gemm(&one, Ds, n, nn, Ds, n, nn, &zero, D2, n, nn));
  BK(gemm(&one, D2, n, nn, D2, n, nn, &zero, D4, n, nn));
  pc_T_kernel<F><<<g2, 256, 0, m->s>>>(n, Ds, m->d_xs, T);
  SK(cudaGetLastError());
  // u block: dt kB G_ij D4 ; sigma column block: -(G_i1 T_1 + G_i2 T_2)
  for (int i = 0; i < 2; ++i) {
    for (int j = 0; j < 2; ++j) {
      BK(gemm(&dtkb, G + (2 * i + j) * nn, n, 4 * nn, D4, n, nn, &zero,
              P + i * n + size_t(j) * n * k, k, kk));
      BK(gemm(&mone, G + (2 * i + j) * nn, n, 4 * nn, T + j * nn, n, 2 * nn,
              j == 0 ? &zero : &one, P + i * n + size_t(2 * n) * k, k, kk));
    }
  }
  pc_fill_kernel<F><<<dim3(nb(3 * n * n, 256), V), 256, 0, m->s>>>(n, Ds, m->d_xs, P);
  SK(cudaGetLastError());
  return STOKES_OK;
}

// Newton-Schulz refresh of X = d_Pinv32 toward P^-1 (P = d_P32): X <- X (2I - P X), whose
// error E = I - P X squares at every update.  The previous step's inverse is kept as it stands
// when its ||E||_F (largest over the vesicles) is at most kNsDone, else updated at most three
// times while the error starts at most kNsLimit[0] and is seen to shrink like a square
// (kNsLimit[it] before update it), so the result is within kNsLimit[2]^2 ~ 1e-2 at worst: a fixed
// operator as close to P^-1 as the preconditioner needs.  Otherwise *done stays false and the
// caller factorises.  m->last_refresh counts the products P X evaluated.  (Measured at the paper
// channel: a start of 1 with four updates refreshes from a few steps earlier in a fresh run but
// costs one more update on every later step.)
constexpr float kNsDone = 1e-3f;
constexpr int kNsUpdates = 3;
constexpr float kNsLimit[kNsUpdates] = {0.5f, 0.3f, 0.1f};
int precond_refresh_ns(stokes_sim *m, bool *done) {
  const int V = m->V, k = 3 * m->n;
  const long long kk = (long long)k * k;
  const float one = 1.0f, zero = 0.0f;
  *done = false;
  for (int it = 0; it < kNsUpdates; ++it) {
    BK(cublasSgemmStridedBatched(m->blas, CUBLAS_OP_N, CUBLAS_OP_N, k, k, k, &one, m->d_P32, k, kk,
                                 m->d_Pinv32, k, kk, &zero, m->d_T32, k, kk, V));
    SK(cudaMemsetAsync(m->d_enorm, 0, sizeof(unsigned), m->s));
    ns_prepare_kernel<<<V, 256, 0, m->s>>>(k, m->d_T32, m->d_enorm);
    SK(cudaGetLastError());
    unsigned hb = 0;
    SK(cudaMemcpyAsync(&hb, m->d_enorm, sizeof(unsigned), cudaMemcpyDeviceToHost, m->s));
    SK(cudaStreamSynchronize(m->s));
    float en;
    memcpy(&en, &hb, sizeof(en));
    m->last_refresh = it + 1;
    if (en <= kNsDone) {  // accurate as it stands
      *done = true;
      return STOKES_OK;
    }
    if (!(en <= kNsLimit[it])) {  // too far, or not squaring
      *done = false;
      return STOKES_OK;
    }
    BK(cublasSgemmStridedBatched(m->blas, CUBLAS_OP_N, CUBLAS_OP_N, k, k, k, &one, m->d_Pinv32, k, kk,
                                 m->d_T32, k, kk, &zero, m->d_X32, k, kk, V));
    SK(cudaMemcpyAsync(m->d_Pinv32, m->d_X32, sizeof(float) * size_t(kk) * V, cudaMemcpyDeviceToDevice, m->s));
    *done = true;
  }
  return STOKES_OK;
}

// While alive, the handle's FP32 GEMMs run as cuBLAS's BF16x9 emulation on the tensor cores
// (each FP32 operand split into three BF16 parts, the products accumulated in FP32: FP32-class
// accuracy) wherever cuBLAS can emulate them; the default math mode is restored after.  The
// emulation is asked for no infinity/NaN handling (cuBLAS otherwise scans both operands and
// patches the product, which cost more than the GEMMs here): the blocks are finite when the
// geometry is, and a non-finite block would still show in the refresh's error norm and the
// step's FP64-accurate residuals.
struct Bf16x9Scope {
  cublasHandle_t h;
  bool on;
  cublasStatus_t st = CUBLAS_STATUS_SUCCESS;
  Bf16x9Scope(cublasHandle_t h_, bool on_) : h(h_), on(on_) {
    if (!on) return;
    st = cublasSetMathMode(h, CUBLAS_FP32_EMULATED_BF16X9_MATH);
    if (st == CUBLAS_STATUS_SUCCESS) st = cublasSetEmulationStrategy(h, CUBLAS_EMULATION_STRATEGY_EAGER);
    if (st == CUBLAS_STATUS_SUCCESS)
      st = cublasSetEmulationSpecialValuesSupport(h, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_NONE);
  }
  void restore() {
    if (!on) return;
    cublasSetEmulationSpecialValuesSupport(h, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_DEFAULT);
    cublasSetEmulationStrategy(h, CUBLAS_EMULATION_STRATEGY_DEFAULT);
    cublasSetMathMode(h, CUBLAS_DEFAULT_MATH);
    on = false;
  }
  ~Bf16x9Scope() { restore(); }
};

int precond_build(stokes_sim *m, double dt) {
  const int n = m->n, V = m->V, k = 3 * n;
  if (m->precond_fp32) {
    Bf16x9Scope emu(m->blas, m->precond_tensor);
    BK(emu.st);
    // FP32 views of the FP64 assembly buffers (each has room for twice its FP32 contents)
    ST(precond_assemble<float>(m, dt, reinterpret_cast<float *>(m->d_G), reinterpret_cast<float *>(m->d_Ds),
                               reinterpret_cast<float *>(m->d_D2), reinterpret_cast<float *>(m->d_D4),
                               reinterpret_cast<float *>(m->d_T), m->d_P32));
    m->last_refresh = 0;
    if (m->precond_refresh && m->pinv_valid && m->pinv_dt == dt) {
      if (!m->d_T32) {
        SK(dalloc(m->d_T32, size_t(k) * k * V));
        SK(dalloc(m->d_X32, size_t(k) * k * V));
        SK(dalloc(m->d_enorm, 1));
      }
      bool done = false;
      ST(precond_refresh_ns(m, &done));
      if (done) return STOKES_OK;
      m->last_refresh = 0;  // rejected: the blocks are factorised below
    }
    emu.restore();  // the factorisation in the default math mode
    BK(cublasSgetrfBatched(m->blas, k, m->d_Pptr32, k, m->d_ppiv, m->d_pinfo, V));
    BK(cublasSgetriBatched(m->blas, k, m->d_Pptr32, k, m->d_ppiv, m->d_Piptr32, k, m->d_pinfo, V));
    m->pinv_valid = true;
    m->pinv_dt = dt;
    return STOKES_OK;
  }
  ST(precond_assemble<double>(m, dt, m->d_G, m->d_Ds, m->d_D2, m->d_D4, m->d_T, m->d_P));
  BK(cublasDgetrfBatched(m->blas, k, m->d_Pptr, k, m->d_ppiv, m->d_pinfo, V));
  BK(cublasDgetriBatched(m->blas, k, m->d_Pptr, k, m->d_ppiv, m->d_Piptr, k, m->d_pinfo, V));
  return STOKES_OK;
}

// ||x||_2 (len doubles, device), synchronous: two fixed-order reduction kernels and one 8-byte
// read back.  (The sums of squares of the step's O(1) unknowns are far from FP64's range ends.)
double dnrm(stokes_sim *m, long len, const double *x, int *st) {
  double r = 0.0;
  nrm_partial_kernel<<<kNrmBlocks, 256, 0, m->s>>>(len, x, m->d_nrm_part);
  nrm_finish_kernel<<<1, kNrmBlocks, 0, m->s>>>(m->d_nrm_part);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&r, m->d_nrm_part, sizeof(double), cudaMemcpyDeviceToHost, m->s) != cudaSuccess ||
      cudaStreamSynchronize(m->s) != cudaSuccess)
    *st = STOKES_ERR_CUDA;
  return sqrt(r);
}

// Right-preconditioned restarted GMRES (classical Gram-Schmidt, twice) on z; FP64.
int gmres(stokes_sim *m, double dt, int precision, const double *b, double *x, double tol,
          int max_iter, int *iters, double *relres, bool x_zero = false) {
  const long len = 3L * m->Nv;
  const int mr = m->gm_m;
  int st = STOKES_OK;
  const double bn = dnrm(m, len, b, &st);
  if (st) return fail(m, st, "norm reduction failed");
  *iters = 0;
  *relres = 0.0;
  if (bn == 0.0) {
    SK(cudaMemsetAsync(x, 0, sizeof(double) * len, m->s));
    return STOKES_OK;
  }
  std::vector<double> H(size_t(mr + 1) * mr), cs(mr), sn(mr), gg(mr + 1), hcol(mr + 1),
      hcol2(mr + 1);
  const double one = 1.0, zero = 0.0, mone = -1.0;
  while (true) {
    // r = b - A x (r = b while x is the caller's zero iterate)
    SK(cudaMemcpyAsync(m->d_V, b, sizeof(double) * len, cudaMemcpyDeviceToDevice, m->s));
    if (!x_zero) {
      ST(step_matvec(m, dt, precision, x, m->d_wk));
      BK(cublasDaxpy(m->blas, int(len), &mone, m->d_wk, 1, m->d_V, 1));
    }
    x_zero = false;
    const double beta = dnrm(m, len, m->d_V, &st);
    if (st) return fail(m, st, "norm reduction failed");
    *relres = beta / bn;
    if (*relres <= tol) return STOKES_OK;
    if (*iters >= max_iter) return fail(m, STOKES_ERR_NOT_CONVERGED, "GMRES: %d iterations, relative residual %.3e", *iters, *relres);
    const double ib = 1.0 / beta;
    BK(cublasDscal(m->blas, int(len), &ib, m->d_V, 1));
    std::fill(gg.begin(), gg.end(), 0.0);
    gg[0] = beta;
    int j = 0;
    for (; j < mr && *iters < max_iter; ++j) {
      double *vj = m->d_V + size_t(j) * len, *vn = m->d_V + size_t(j + 1) * len;
      ST(precond_apply(m, vj, m->d_z));
      ST(step_matvec(m, dt, precision, m->d_z, vn));
      // CGS2
      BK(cublasDgemv(m->blas, CUBLAS_OP_T, int(len), j + 1, &one, m->d_V, int(len), vn, 1, &zero,
                     m->d_h, 1));
      BK(cublasDgemv(m->blas, CUBLAS_OP_N, int(len), j + 1, &mone, m->d_V, int(len), m->d_h, 1, &one,
                     vn, 1));
      SK(cudaMemcpyAsync(hcol.data(), m->d_h, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, m->s));
      BK(cublasDgemv(m->blas, CUBLAS_OP_T, int(len), j + 1, &one, m->d_V, int(len), vn, 1, &zero,
                     m->d_h, 1));
      BK(cublasDgemv(m->blas, CUBLAS_OP_N, int(len), j + 1, &mone, m->d_V, int(len), m->d_h, 1, &one,
                     vn, 1));
      SK(cudaMemcpyAsync(hcol2.data(), m->d_h, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, m->s));
      const double hn = dnrm(m, len, vn, &st);  // synchronises the stream
      if (st) return fail(m, st, "norm reduction failed");
      for (int q = 0; q <= j; ++q) hcol[q] += hcol2[q];
      hcol[j + 1] = hn;
      if (hn > 0.0) {
        const double ih = 1.0 / hn;
        BK(cublasDscal(m->blas, int(len), &ih, vn, 1));
      }
      // Givens rotations
      for (int q = 0; q < j; ++q) {
        const double t = cs[q] * hcol[q] + sn[q] * hcol[q + 1];
        hcol[q + 1] = -sn[q] * hcol[q] + cs[q] * hcol[q + 1];
        hcol[q] = t;
      }
      const double den = hypot(hcol[j], hcol[j + 1]);
      cs[j] = den > 0 ? hcol[j] / den : 1.0;
      sn[j] = den > 0 ? hcol[j + 1] / den : 0.0;
      hcol[j] = den;
      hcol[j + 1] = 0.0;
      gg[j + 1] = -sn[j] * gg[j];
      gg[j] = cs[j] * gg[j];
      for (int q = 0; q <= j; ++q) H[size_t(j) * (mr + 1) + q] = hcol[q];
      ++*iters;
      if (fabs(gg[j + 1]) / bn <= tol * 0.5 || hn == 0.0) {
        ++j;
        break;
      }
    }
    // y = H^-1 g (upper triangular), x += P^-1 (V y)
    std::vector<double> yv(j);
    for (int q = j - 1; q >= 0; --q) {
      double s = gg[q];
      for (int p = q + 1; p < j; ++p) s -= H[size_t(p) * (mr + 1) + q] * yv[p];
      yv[q] = s / H[size_t(q) * (mr + 1) + q];
    }
    SK(cudaMemcpyAsync(m->d_h, yv.data(), sizeof(double) * j, cudaMemcpyHostToDevice, m->s));
    BK(cublasDgemv(m->blas, CUBLAS_OP_N, int(len), j, &one, m->d_V, int(len), m->d_h, 1, &zero,
                   m->d_wk, 1));
    ST(precond_apply(m, m->d_wk, m->d_z));
    BK(cublasDaxpy(m->blas, int(len), &one, m->d_z, 1, x, 1));
    SK(cudaStreamSynchronize(m->s));
  }
}

void free_walls(stokes_sim *m) {
  for (stokes_fmm **pl : {&m->fmm_w, &m->fmm_vw, &m->fmm_wv})  // before their contexts
    if (*pl) {
      stokes_fmm_destroy(*pl);
      *pl = nullptr;
    }
  m->fmm_w_order = 0;
  if (m->ctx_w) stokes_destroy(m->ctx_w);
  m->ctx_w = nullptr;
  dfree(m->d_wx);
  dfree(m->d_side);
  dfree(m->d_proxy);
  dfree(m->d_LU);
  dfree(m->d_A);
  dfree(m->d_Ainv32);
  dfree(m->d_wb);
  dfree(m->d_wr);
  dfree(m->d_wr32);
  dfree(m->d_wb32);
  m->wall_ws_len = 0;
  stokes::fds_destroy(m->fds);
  m->fds = nullptr;
  dfree(m->d_W);
  dfree(m->d_C);
  dfree(m->d_Spinv);
  dfree(m->d_piv);
  dfree(m->d_vrhs);
  dfree(m->d_c);
  dfree(m->d_tau);
  for (double **p : {&m->d_B, &m->d_Q, &m->d_rv, &m->d_rg, &m->d_side_part, &m->d_resv, &m->d_resg, &m->d_dtau,
                     &m->d_dc, &m->d_g2})
    dfree(*p);
  m->have_walls = false;
}

void free_vesicles(stokes_sim *m) {
  for (stokes_fmm **pl : {&m->fmm_v, &m->fmm_vw, &m->fmm_wv})
    if (*pl) {
      stokes_fmm_destroy(*pl);
      *pl = nullptr;
    }
  if (m->close_v) stokes_close_destroy(m->close_v);
  m->close_v = nullptr;
  if (m->ctx_v) stokes_destroy(m->ctx_v);
  m->ctx_v = nullptr;
  double2 **p2[] = {&m->d_x, &m->d_nrm, &m->d_xs, &m->d_f, &m->d_fb, &m->d_ures, &m->d_tmp2, &m->d_tmp3};
  for (auto p : p2) dfree(*p);
  double **p1[] = {&m->d_w, &m->d_spd, &m->d_sigma, &m->d_D, &m->d_kress, &m->d_L0, &m->d_A0, &m->d_Lk,
                   &m->d_G, &m->d_Ds, &m->d_D2, &m->d_D4, &m->d_T, &m->d_P, &m->d_Pinv, &m->d_V,
                   &m->d_z, &m->d_b, &m->d_wk, &m->d_h, &m->d_xsol, &m->d_rr, &m->d_dd};
  for (auto p : p1) dfree(*p);
  dfree(m->d_feat);
  dfree(m->d_targ);
  dfree(m->d_pred);
  dfree(m->d_frame);
  dfree(m->d_bprev);
  dfree(m->d_zprev);
  dfree(m->d_zprev2);
  dfree(m->d_Pptr);
  dfree(m->d_Piptr);
  dfree(m->d_P32);
  dfree(m->d_Pinv32);
  dfree(m->d_Pptr32);
  dfree(m->d_Piptr32);
  dfree(m->d_T32);
  dfree(m->d_X32);
  dfree(m->d_enorm);
  m->pinv_valid = false;
  dfree(m->d_ppiv);
  dfree(m->d_pinfo);
  m->have_ves = false;
}

}  // namespace

extern "C" {

int stokes_sim_create(int device, stokes_sim **out) {
  if (!out) return STOKES_ERR_ARG;
  *out = nullptr;
  int nd = 0;
  if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) return STOKES_ERR_CUDA;
  stokes_sim *m = new stokes_sim();
  m->device = device;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&m->s, cudaStreamNonBlocking) != cudaSuccess ||
      cublasCreate(&m->blas) != CUBLAS_STATUS_SUCCESS ||
      cusolverDnCreate(&m->sol) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnCreateParams(&m->params) != CUSOLVER_STATUS_SUCCESS ||
      cudaMalloc(reinterpret_cast<void **>(&m->d_info), sizeof(int)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void **>(&m->d_nrm_part), sizeof(double) * kNrmBlocks) != cudaSuccess) {
    delete m;
    return STOKES_ERR_CUDA;
  }
  if (set_stream_handles(m) != STOKES_OK) {
    delete m;
    return STOKES_ERR_CUDA;
  }
  *out = m;
  return STOKES_OK;
}

int stokes_sim_destroy(stokes_sim *m) {
  if (!m) return STOKES_OK;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  free_walls(m);
  free_vesicles(m);
  dfree(m->d_info);
  dfree(m->d_nrm_part);
  if (m->blas) cublasDestroy(m->blas);
  if (m->params) cusolverDnDestroyParams(m->params);
  if (m->sol) cusolverDnDestroy(m->sol);
  if (m->s) cudaStreamDestroy(m->s);
  delete m;
  return STOKES_OK;
}

int stokes_sim_last_error(const stokes_sim *m, char *buf, size_t len) {
  if (!m || !buf || len == 0) return STOKES_ERR_ARG;
  snprintf(buf, len, "%s", m->err.c_str());
  return STOKES_OK;
}

int stokes_sim_set_walls(stokes_sim *m, int n_per_wall, const double *nodes, const double *weights,
                         const double *normals, const double *curvature, double period, double mu,
                         int K, int M, double proxy_radius) {
  if (!m) return STOKES_ERR_ARG;
  if (n_per_wall < 4 || !nodes || !weights || !normals || !curvature)
    return fail(m, STOKES_ERR_ARG, "need n_per_wall >= 4 and host wall arrays");
  if (!(period > 0.0) || !(mu > 0.0) || K < 2 || M < 2 || !(proxy_radius > 0.0))
    return fail(m, STOKES_ERR_ARG, "need period > 0, mu > 0, K >= 2, M >= 2, proxy radius > 0");
  if (m->have_ves && mu != m->mu) return fail(m, STOKES_ERR_ARG, "mu differs from the vesicles'");
  if (fabs(nodes[0]) > 1e-12 || fabs(nodes[2 * n_per_wall]) > 1e-12)
    return fail(m, STOKES_ERR_ARG, "each wall's first node must lie on x = 0 (the inlet)");
  SK(cudaSetDevice(m->device));
  free_walls(m);
  const auto t_setup = std::chrono::steady_clock::now();
  const int Nt = 2 * n_per_wall, nA = 2 * Nt;
  m->Nt = Nt;
  m->nA = nA;
  m->K = K;
  m->M = M;
  m->mu = mu;
  m->period = period;
  // walls-only context (double-layer sums at vesicle nodes)
  ST(stokes_create(m->device, &m->ctx_w));
  double *dx = nullptr, *dw = nullptr, *dn = nullptr, *dk = nullptr;
  SK(dalloc(dx, 2 * Nt));
  SK(dalloc(dw, Nt));
  SK(dalloc(dn, 2 * Nt));
  SK(dalloc(dk, Nt));
  SK(cudaMemcpy(dx, nodes, sizeof(double) * 2 * Nt, cudaMemcpyHostToDevice));
  SK(cudaMemcpy(dw, weights, sizeof(double) * Nt, cudaMemcpyHostToDevice));
  SK(cudaMemcpy(dn, normals, sizeof(double) * 2 * Nt, cudaMemcpyHostToDevice));
  SK(cudaMemcpy(dk, curvature, sizeof(double) * Nt, cudaMemcpyHostToDevice));
  const int32_t off[3] = {0, n_per_wall, Nt}, kind[2] = {STOKES_KIND_WALL, STOKES_KIND_WALL};
  int st = stokes_geom_set(m->ctx_w, 2, off, kind, dx, dw, dn, dk, period, mu, m->s);
  if (st) {
    char b[256];
    stokes_last_error(m->ctx_w, b, sizeof(b));
    cudaFree(dw);
    cudaFree(dn);
    cudaFree(dk);
    cudaFree(dx);
    return fail(m, st, "walls: %s", b);
  }
  m->d_wx = reinterpret_cast<double2 *>(dx);
  // side points and proxies (host setup)
  const double ylo = nodes[1], yhi = nodes[2 * n_per_wall + 1];
  std::vector<double> gl = gauss_legendre(K);
  std::vector<double2> side(2 * K), prox(M);
  for (int k = 0; k < K; ++k) {
    const double y = 0.5 * (ylo + yhi) + 0.5 * (yhi - ylo) * gl[k];
    side[k] = make_double2(0.0, y);
    side[K + k] = make_double2(period, y);
  }
  for (int q = 0; q < M; ++q)
    prox[q] = make_double2(0.5 * period + proxy_radius * cos(2.0 * kPiD * q / M),
                           proxy_radius * sin(2.0 * kPiD * q / M));
  SK(dalloc(m->d_side, 2 * K));
  SK(dalloc(m->d_proxy, M));
  SK(cudaMemcpy(m->d_side, side.data(), sizeof(double2) * 2 * K, cudaMemcpyHostToDevice));
  SK(cudaMemcpy(m->d_proxy, prox.data(), sizeof(double2) * M, cudaMemcpyHostToDevice));
  // assemble A, B, C, Q
  double *dQ = nullptr, *dS = nullptr, *dU = nullptr, *dVt = nullptr, *dsig = nullptr;
  m->walls_mode = m->wall_solver;  // later set_wall_solver calls wait for the next set_walls
  const bool lu32 = m->walls_mode == STOKES_WALLS_LU32_REFINE;
  const bool fds = m->walls_mode == STOKES_WALLS_FDS;
  double *dA = nullptr;
  if (!fds) {
    SK(dalloc(dA, size_t(nA) * nA));
    (lu32 ? m->d_A : m->d_LU) = dA;
  }
  SK(dalloc(m->d_W, size_t(nA) * 2 * M));
  SK(dalloc(m->d_C, size_t(4) * K * nA));
  SK(dalloc(dQ, size_t(4) * K * 2 * M));
  if (!lu32 && !fds) SK(dalloc(m->d_piv, nA));
  const double cmu = 1.0 / (4.0 * kPiD * mu);
  const double2 *wx = m->d_wx, *wn = reinterpret_cast<const double2 *>(dn);
  if (!fds) assemble_A_kernel<<<dim3(nb(Nt, 128), Nt), 128, 0, m->s>>>(Nt, wx, wn, dw, dk, period, dA);
  assemble_B_kernel<<<dim3(nb(Nt, 128), M), 128, 0, m->s>>>(Nt, M, wx, m->d_proxy, cmu, m->d_W);
  SK(dalloc(m->d_B, size_t(nA) * 2 * M));
  SK(cudaMemcpyAsync(m->d_B, m->d_W, sizeof(double) * nA * 2 * M, cudaMemcpyDeviceToDevice, m->s));
  assemble_C_kernel<<<dim3(nb(Nt, 128), K), 128, 0, m->s>>>(Nt, K, wx, wn, dw, m->d_side, period, mu,
                                                           m->d_C);
  assemble_Q_kernel<<<dim3(nb(K, 64), M), 64, 0, m->s>>>(K, M, m->d_side, m->d_proxy, cmu, dQ);
  SK(dalloc(m->d_Q, size_t(4) * K * 2 * M));
  SK(cudaMemcpyAsync(m->d_Q, dQ, sizeof(double) * 4 * K * 2 * M, cudaMemcpyDeviceToDevice, m->s));
  SK(cudaGetLastError());
  // LU of A (FP64, or FP32 with FP64 refinement) or the fast direct solver; W = A^-1 B
  double *work = nullptr;
  float *lu32f = nullptr;
  int64_t *piv64 = nullptr;
  if (fds) {
    SK(cudaStreamSynchronize(m->s));
    const int st = stokes::fds_build(&m->fds, n_per_wall, nodes, weights, normals, curvature,
                                     period, m->fds_p, m->s, m->blas, m->sol, m->err);
    if (st) {
      for (double *p : {dQ, dw, dn, dk}) cudaFree(p);
      return st;
    }
  } else if (lu32) {
    const size_t nn = size_t(nA) * nA;
    SK(dalloc(lu32f, nn));
    SK(dalloc(piv64, nA));
    d2f_kernel<<<grid_for(nn), 256, 0, m->s>>>(nn, dA, lu32f);
    SK(cudaGetLastError());
    size_t wd = 0, wh = 0;
    QK(cusolverDnXgetrf_bufferSize(m->sol, m->params, nA, nA, CUDA_R_32F, lu32f, nA, CUDA_R_32F,
                                   &wd, &wh));
    SK(dalloc(work, wd / sizeof(double) + 1));
    std::vector<char> hwork(std::max<size_t>(wh, 1));
    QK(cusolverDnXgetrf(m->sol, m->params, nA, nA, CUDA_R_32F, lu32f, nA, piv64, CUDA_R_32F,
                        work, wd, hwork.data(), wh, m->d_info));
  } else {
    int lwork = 0;
    QK(cusolverDnDgetrf_bufferSize(m->sol, nA, nA, m->d_LU, nA, &lwork));
    SK(dalloc(work, lwork));
    QK(cusolverDnDgetrf(m->sol, nA, nA, m->d_LU, nA, work, m->d_piv, m->d_info));
  }
  if (!fds) {
    int finfo = 0;
    SK(cudaMemcpyAsync(&finfo, m->d_info, sizeof(int), cudaMemcpyDeviceToHost, m->s));
    SK(cudaStreamSynchronize(m->s));
    if (finfo != 0) {
      cudaFree(lu32f);
      cudaFree(piv64);
      return fail(m, STOKES_ERR_CUDA, "LU of the wall operator failed (info %d)", finfo);
    }
  }
  if (lu32) {  // A32^-1 from the FP32 LU: solve A32 X = I, then drop the factors
    SK(dalloc(m->d_Ainv32, size_t(nA) * nA));
    identity_f32_kernel<<<grid_for(size_t(nA) * nA), 256, 0, m->s>>>(nA, m->d_Ainv32);
    SK(cudaGetLastError());
    QK(cusolverDnXgetrs(m->sol, m->params, CUBLAS_OP_N, nA, nA, CUDA_R_32F, lu32f, nA, piv64,
                        CUDA_R_32F, m->d_Ainv32, nA, m->d_info));
    SK(cudaStreamSynchronize(m->s));
    cudaFree(lu32f);
    cudaFree(piv64);
  }
  ST(wall_solve(m, m->d_W, 2 * M));
  // S = Q - C W  (4K x 2M); SVD of S^T (2M x 4K, needs rows >= cols)
  const double one = 1.0, mone = -1.0, zero = 0.0;
  BK(cublasDgemm(m->blas, CUBLAS_OP_N, CUBLAS_OP_N, 4 * K, 2 * M, nA, &mone, m->d_C, 4 * K, m->d_W,
                 nA, &one, dQ, 4 * K));
  const int rS = 2 * M, cS = 4 * K;
  if (rS < cS) return fail(m, STOKES_ERR_ARG, "need M >= 2K proxy points");
  SK(dalloc(dS, size_t(rS) * cS));
  transpose_kernel<<<nb(long(cS) * rS, 256), 256, 0, m->s>>>(cS, rS, dQ, dS);
  SK(dalloc(dU, size_t(rS) * cS));
  SK(dalloc(dVt, size_t(cS) * cS));
  SK(dalloc(dsig, cS));
  int lw2 = 0;
  QK(cusolverDnDgesvd_bufferSize(m->sol, rS, cS, &lw2));
  double *work2 = nullptr;
  SK(dalloc(work2, lw2));
  QK(cusolverDnDgesvd(m->sol, 'S', 'S', rS, cS, dS, rS, dsig, dU, rS, dVt, cS, work2, lw2, nullptr,
                      m->d_info));
  double smax = 0.0;
  SK(cudaMemcpyAsync(&smax, dsig, sizeof(double), cudaMemcpyDeviceToHost, m->s));
  SK(cudaStreamSynchronize(m->s));
  int info = 0;
  SK(cudaMemcpy(&info, m->d_info, sizeof(int), cudaMemcpyDeviceToHost));
  scale_columns_kernel<<<nb(long(rS) * cS, 256), 256, 0, m->s>>>(rS, cS, dsig, 1e-13 * smax, dU);
  // S^+ = U diag(1/sigma) V^T  (2M x 4K)
  SK(dalloc(m->d_Spinv, size_t(rS) * cS));
  BK(cublasDgemm(m->blas, CUBLAS_OP_N, CUBLAS_OP_N, rS, cS, cS, &one, dU, rS, dVt, cS, &zero,
                 m->d_Spinv, rS));
  SK(cudaStreamSynchronize(m->s));
  for (double *p : {dQ, dS, dU, dVt, dsig, work, work2, dw, dn, dk}) cudaFree(p);
  SK(dalloc(m->d_vrhs, nA));
  SK(dalloc(m->d_c, 2 * M));
  SK(dalloc(m->d_tau, nA));
  SK(dalloc(m->d_rv, nA));
  SK(dalloc(m->d_resv, nA));
  SK(dalloc(m->d_dtau, nA));
  SK(dalloc(m->d_rg, 4 * K));
  SK(dalloc(m->d_side_part, size_t(4) * kSideChunks * K));
  SK(dalloc(m->d_resg, 4 * K));
  SK(dalloc(m->d_g2, 4 * K));
  SK(dalloc(m->d_dc, 2 * M));
  if (info != 0) return fail(m, STOKES_ERR_CUDA, "SVD of the Schur complement did not converge (%d)", info);
  m->have_walls = true;
  SK(cudaStreamSynchronize(m->s));
  m->walls_setup_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_setup).count();
  return STOKES_OK;
}

int stokes_sim_set_vesicles(stokes_sim *m, int V, int n, const double *x, double kappa_b,
                            double mu, double period) {
  if (!m) return STOKES_ERR_ARG;
  if (V < 1 || n < 8 || (n & 1) || n > kMaxN || !x)
    return fail(m, STOKES_ERR_ARG, "need V >= 1 vesicles with an even n in [8, %d] nodes", kMaxN);
  if (!(mu > 0.0) || !(period >= 0.0)) return fail(m, STOKES_ERR_ARG, "need mu > 0, period >= 0");
  if (m->have_walls && (mu != m->mu || period != m->period))
    return fail(m, STOKES_ERR_ARG, "mu and period must match the walls'");
  SK(cudaSetDevice(m->device));
  free_vesicles(m);
  m->V = V;
  m->n = n;
  m->Nv = V * n;
  m->kappa_b = kappa_b;
  m->mu = mu;
  m->period = period;
  const int Nv = m->Nv;
  SK(dalloc(m->d_x, Nv));
  SK(dalloc(m->d_nrm, Nv));
  SK(dalloc(m->d_xs, Nv));
  SK(dalloc(m->d_w, Nv));
  SK(dalloc(m->d_spd, Nv));
  SK(dalloc(m->d_sigma, Nv));
  SK(dalloc(m->d_D, n * n));
  SK(dalloc(m->d_kress, n));
  SK(dalloc(m->d_L0, V));
  SK(dalloc(m->d_A0, V));
  SK(dalloc(m->d_Lk, V));
  for (double2 **p : {&m->d_f, &m->d_fb, &m->d_ures, &m->d_tmp2, &m->d_tmp3}) SK(dalloc(*p, Nv));
  SK(cudaMemcpy(m->d_x, x, sizeof(double2) * Nv, cudaMemcpyHostToDevice));
  SK(cudaMemsetAsync(m->d_sigma, 0, sizeof(double) * Nv, m->s));
  fourier_diff_kernel<<<nb(n * n, 256), 256, 0, m->s>>>(n, m->d_D);
  SK(launch_kress_table(n, m->d_kress, m->s));
  ves_geom_kernel<<<V, n, 0, m->s>>>(n, m->d_x, m->d_D, m->d_spd, m->d_xs, m->d_nrm, m->d_w);
  ves_LA_kernel<<<V, n, 0, m->s>>>(n, m->d_x, m->d_D, m->d_w, m->d_L0, m->d_A0);
  SK(cudaGetLastError());
  // vesicles-only context (single-layer sums with Kress self terms)
  ST(stokes_create(m->device, &m->ctx_v));
  std::vector<int32_t> off(V + 1), kind(V, STOKES_KIND_VESICLE);
  for (int v = 0; v <= V; ++v) off[v] = v * n;
  SK(cudaStreamSynchronize(m->s));
  int st = stokes_geom_set(m->ctx_v, V, off.data(), kind.data(), reinterpret_cast<double *>(m->d_x),
                           m->d_w, reinterpret_cast<double *>(m->d_nrm), nullptr, period, mu, m->s);
  if (st) {
    char b[256];
    stokes_last_error(m->ctx_v, b, sizeof(b));
    return fail(m, st, "vesicles: %s", b);
  }
  // preconditioner and GMRES workspace
  const int k = 3 * n;
  const size_t nn = size_t(n) * n, kk = size_t(k) * k;
  SK(dalloc(m->d_G, 4 * nn * V));
  SK(dalloc(m->d_Ds, nn * V));
  SK(dalloc(m->d_D2, nn * V));
  SK(dalloc(m->d_D4, nn * V));
  SK(dalloc(m->d_T, 2 * nn * V));
  SK(dalloc(m->d_P, kk * V));
  SK(dalloc(m->d_Pinv, kk * V));
  SK(dalloc(m->d_Pptr, V));
  SK(dalloc(m->d_Piptr, V));
  SK(dalloc(m->d_ppiv, size_t(k) * V));
  SK(dalloc(m->d_pinfo, V));
  set_ptrs_kernel<<<nb(V, 128), 128, 0, m->s>>>(V, m->d_P, kk, m->d_Pptr);
  set_ptrs_kernel<<<nb(V, 128), 128, 0, m->s>>>(V, m->d_Pinv, kk, m->d_Piptr);
  SK(dalloc(m->d_P32, kk * V));
  SK(dalloc(m->d_Pinv32, kk * V));
  SK(dalloc(m->d_Pptr32, V));
  SK(dalloc(m->d_Piptr32, V));
  set_ptrs32_kernel<<<nb(V, 128), 128, 0, m->s>>>(V, m->d_P32, kk, m->d_Pptr32);
  set_ptrs32_kernel<<<nb(V, 128), 128, 0, m->s>>>(V, m->d_Pinv32, kk, m->d_Piptr32);
  m->gm_m = 80;
  const long len = 3L * Nv;
  SK(dalloc(m->d_V, size_t(len) * (m->gm_m + 1)));
  SK(dalloc(m->d_z, len));
  SK(dalloc(m->d_b, len));
  SK(dalloc(m->d_wk, len));
  SK(dalloc(m->d_h, m->gm_m + 1));
  SK(dalloc(m->d_xsol, len));
  SK(dalloc(m->d_rr, len));
  SK(dalloc(m->d_dd, len));
  SK(cudaMemsetAsync(m->d_xsol, 0, sizeof(double) * len, m->s));
  SK(dalloc(m->d_feat, size_t(V) * feat_dim(kMaxModes, true)));
  SK(dalloc(m->d_targ, size_t(V) * targ_dim(kMaxModes)));
  SK(dalloc(m->d_pred, size_t(V) * targ_dim(kMaxModes)));
  SK(dalloc(m->d_frame, size_t(V) * 6));
  SK(dalloc(m->d_bprev, len));
  SK(dalloc(m->d_zprev, len));
  SK(dalloc(m->d_zprev2, len));
  SK(cudaMemsetAsync(m->d_bprev, 0, sizeof(double) * len, m->s));
  SK(cudaMemsetAsync(m->d_zprev, 0, sizeof(double) * len, m->s));
  SK(cudaMemsetAsync(m->d_zprev2, 0, sizeof(double) * len, m->s));
  SK(cudaStreamSynchronize(m->s));
  m->have_ves = true;
  m->hist_count = 0;
  return STOKES_OK;
}

int stokes_sim_channel_response(stokes_sim *m, const double *f, double p_drive, double *u_resp) {
  if (!m) return STOKES_ERR_ARG;
  if (!m->have_walls || !m->have_ves) return fail(m, STOKES_ERR_NO_GEOM, "walls and vesicles must be set");
  if (!f || !u_resp) return fail(m, STOKES_ERR_ARG, "NULL device pointer");
  SK(cudaSetDevice(m->device));
  ST(channel_response(m, reinterpret_cast<const double2 *>(f), p_drive,
                      reinterpret_cast<double2 *>(u_resp)));
  SK(cudaStreamSynchronize(m->s));
  return STOKES_OK;
}

int stokes_sim_set_wall_solver(stokes_sim *m, int mode) {
  if (!m) return STOKES_ERR_ARG;
  if (mode != STOKES_WALLS_LU64 && mode != STOKES_WALLS_LU32_REFINE && mode != STOKES_WALLS_FDS)
    return fail(m, STOKES_ERR_ARG, "unknown wall solver %d", mode);
  m->wall_solver = mode;
  return STOKES_OK;
}

int stokes_sim_wall_solve(stokes_sim *m, double *X, int nrhs) {
  if (!m) return STOKES_ERR_ARG;
  if (!X || nrhs < 1) return fail(m, STOKES_ERR_ARG, "need a device X and nrhs >= 1");
  if (!m->have_walls) return fail(m, STOKES_ERR_NO_GEOM, "no walls set");
  SK(cudaSetDevice(m->device));
  ST(wall_solve(m, X, nrhs));
  SK(cudaStreamSynchronize(m->s));
  return STOKES_OK;
}

int stokes_sim_set_fds_params(stokes_sim *m, double tol, int leaf_nodes, int n_proxy) {
  if (!m) return STOKES_ERR_ARG;
  if (!(tol >= 1e-15 && tol <= 1e-3) || leaf_nodes < 8 || leaf_nodes > 512 || n_proxy < 16 ||
      n_proxy > 512)
    return fail(m, STOKES_ERR_ARG,
                "need tol in [1e-15, 1e-3], leaf_nodes in [8, 512], n_proxy in [16, 512]");
  m->fds_p.tol = tol;
  m->fds_p.leaf = leaf_nodes;
  m->fds_p.n_proxy = n_proxy;
  return STOKES_OK;
}

int stokes_sim_set_fds_recompress(stokes_sim *m, int on) {
  if (!m) return STOKES_ERR_ARG;
  if (on != 0 && on != 1) return fail(m, STOKES_ERR_ARG, "recompress must be 0 or 1");
  m->fds_p.recompress = on == 1;
  return STOKES_OK;
}

int stokes_sim_fds_info(const stokes_sim *m, stokes_fds_info *out) {
  if (!m || !out) return STOKES_ERR_ARG;
  *out = stokes_fds_info{};
  out->walls_setup_ms = m->walls_setup_ms;
  if (!m->fds) return STOKES_OK;
  stokes::fds_info f;
  stokes::fds_get_info(m->fds, &f);
  out->levels = f.levels;
  out->max_rank = f.max_rank;
  out->root_size = f.root_size;
  out->neighbour_rank = f.neighbour_rank;
  out->sections = f.sections;
  out->host_ms = f.host_ms;
  out->device_ms = f.device_ms;
  out->device_bytes = double(f.device_bytes);
  out->solve_bytes = double(f.solve_bytes);
  out->neighbour_col_rank = f.neighbour_col_rank;
  return STOKES_OK;
}

int stokes_sim_set_precond_precision(stokes_sim *m, int precision) {
  if (!m) return STOKES_ERR_ARG;
  if (precision != STOKES_FP64 && precision != STOKES_FP32_KAHAN)
    return fail(m, STOKES_ERR_ARG, "preconditioner precision must be STOKES_FP64 or STOKES_FP32_KAHAN");
  m->precond_fp32 = precision == STOKES_FP32_KAHAN;
  m->pinv_valid = false;
  return STOKES_OK;
}

int stokes_sim_set_precond_refresh(stokes_sim *m, int on) {
  if (!m) return STOKES_ERR_ARG;
  if (on != 0 && on != 1) return fail(m, STOKES_ERR_ARG, "refresh must be 0 or 1");
  m->precond_refresh = on == 1;
  return STOKES_OK;
}

int stokes_sim_set_precond_tensor(stokes_sim *m, int on) {
  if (!m) return STOKES_ERR_ARG;
  if (on != 0 && on != 1) return fail(m, STOKES_ERR_ARG, "tensor must be 0 or 1");
  m->precond_tensor = on == 1;
  return STOKES_OK;
}

int stokes_sim_set_inner_tolerance(stokes_sim *m, double tol) {
  if (!m) return STOKES_ERR_ARG;
  if (!(tol >= 1e-8 && tol <= 0.5)) return fail(m, STOKES_ERR_ARG, "inner tolerance must be in [1e-8, 0.5]");
  m->inner_tol = tol;
  return STOKES_OK;
}

int stokes_sim_set_block_refinement(stokes_sim *m, int sweeps) {
  if (!m) return STOKES_ERR_ARG;
  if (sweeps < 0 || sweeps > 8) return fail(m, STOKES_ERR_ARG, "block refinement sweeps must be in [0, 8]");
  // with no outer corrections each wall solve is refined to FP64 accuracy itself
  m->block_refine = sweeps;
  return STOKES_OK;
}

int stokes_sim_wall_stats(const stokes_sim *m, int *refinements, double *residual) {
  if (!m || !refinements || !residual) return STOKES_ERR_ARG;
  *refinements = m->wall_refinements;
  *residual = m->wall_residual;
  return STOKES_OK;
}

}  // extern "C"

namespace {

// Density tau (d_tau) and proxy weights c (d_c) of the pressure-driven channel with wall
// velocity v_walls (device, NULL = no slip): the refined block solve of the empty-channel system.
int empty_solve(stokes_sim *m, double p_drive, const double *v_walls) {
  empty_rhs_kernel<<<nb(4 * m->K, 128), 128, 0, m->s>>>(m->K, p_drive, m->d_rg);
  if (v_walls)
    SK(cudaMemcpyAsync(m->d_rv, v_walls, sizeof(double) * m->nA, cudaMemcpyDeviceToDevice, m->s));
  else
    SK(cudaMemsetAsync(m->d_rv, 0, sizeof(double) * m->nA, m->s));
  return refined_block_solve(m, STOKES_FP64);
}

}  // namespace

extern "C" {

int stokes_sim_empty_channel(stokes_sim *m, double p_drive, const double *v_walls, int n_targets,
                             const double *targets, double *u_out) {
  if (!m) return STOKES_ERR_ARG;
  if (!m->have_walls) return fail(m, STOKES_ERR_NO_GEOM, "walls must be set");
  if (n_targets < 1 || !targets || !u_out) return fail(m, STOKES_ERR_ARG, "need targets and output");
  SK(cudaSetDevice(m->device));
  ST(empty_solve(m, p_drive, v_walls));
  ST(stokes_sum_eval_targets(m->ctx_w, STOKES_FP64, nullptr, m->d_tau, n_targets, targets, u_out, m->s));
  proxy_eval_kernel<<<nb(n_targets, 128), 128, 0, m->s>>>(n_targets, reinterpret_cast<const double2 *>(targets), m->M,
                                                         m->d_proxy, m->d_c, 1.0 / (4.0 * kPiD * m->mu),
                                                         reinterpret_cast<double2 *>(u_out));
  SK(cudaGetLastError());
  SK(cudaStreamSynchronize(m->s));
  return STOKES_OK;
}

int stokes_sim_empty_channel_pressure(stokes_sim *m, double p_drive, const double *v_walls,
                                      int n_targets, const double *targets, double *p_out) {
  if (!m) return STOKES_ERR_ARG;
  if (!m->have_walls) return fail(m, STOKES_ERR_NO_GEOM, "walls must be set");
  if (n_targets < 1 || !targets || !p_out) return fail(m, STOKES_ERR_ARG, "need targets and output");
  SK(cudaSetDevice(m->device));
  ST(empty_solve(m, p_drive, v_walls));
  const int st = stokes_sum_eval_pressure(m->ctx_w, nullptr, m->d_tau, n_targets, targets, p_out, m->s);
  if (st) {
    char b[256];
    stokes_last_error(m->ctx_w, b, sizeof(b));
    return fail(m, st, "walls: %s", b);
  }
  proxy_pressure_kernel<<<nb(n_targets, 128), 128, 0, m->s>>>(
      n_targets, reinterpret_cast<const double2 *>(targets), m->M, m->d_proxy, m->d_c, p_out);
  SK(cudaGetLastError());
  SK(cudaStreamSynchronize(m->s));
  return STOKES_OK;
}

int vesicle_step_warmstart(stokes_sim *m, double dt, double p_drive, int guess_mode,
                           stokes_mlp *model, const double *guess, double tol, int max_iter,
                           int precision, stokes_step_stats *out) {
  if (!m) return STOKES_ERR_ARG;
  if (!m->have_ves) return fail(m, STOKES_ERR_NO_GEOM, "vesicles must be set");
  if (guess_mode < STOKES_GUESS_ZERO || guess_mode > STOKES_GUESS_EXTRAPOLATE)
    return fail(m, STOKES_ERR_ARG, "unknown guess mode %d", guess_mode);
  if (guess_mode == STOKES_GUESS_USER && !guess) return fail(m, STOKES_ERR_ARG, "guess is NULL");
  if (guess_mode == STOKES_GUESS_MLP) {
    if (!model) return fail(m, STOKES_ERR_ARG, "model is NULL");
    int ni = 0, no = 0;
    mlp_dims(model, &ni, &no);
    const int nm = m->warm_modes;
    const int nf = feat_dim(nm, m->warm_history);
    if (ni != nf || no != targ_dim(nm) || m->n < nm)
      return fail(m, STOKES_ERR_ARG, "model must map %d features to %d targets (%d modes, n >= %d)",
                  nf, targ_dim(nm), nm, nm);
  }
  if (!(dt > 0.0) || !(tol > 0.0) || max_iter < 1)
    return fail(m, STOKES_ERR_ARG, "need dt > 0, tol > 0, max_iter >= 1");
  if (precision != STOKES_FP64 && precision != STOKES_FP32_KAHAN &&
      precision != STOKES_DOUBLE_FLOAT)
    return fail(m, STOKES_ERR_ARG, "unknown precision");
  // hp: the precision of every sum that must be FP64-accurate (right-hand side, channel
  // response, residuals): FP64 itself, or double-float for the two faster modes
  const int hp = precision == STOKES_FP64 ? STOKES_FP64 : STOKES_DOUBLE_FLOAT;
  // mixed precision with FMM residuals: the vesicle sums of the right-hand side and of the
  // refinement residuals go through this step's FMM plan
  const bool use_fmm = precision == STOKES_FP32_KAHAN && m->resid_fmm_order > 0;
  // a plan for this step: FMM residuals and/or FMM sweeps
  const bool use_plan = precision == STOKES_FP32_KAHAN && (use_fmm || m->sweep_fmm_order > 0);
  SK(cudaSetDevice(m->device));
  const auto t0 = std::chrono::steady_clock::now();
  const int V = m->V, n = m->n;
  const long len = 3L * m->Nv;
  for (stokes_fmm **pl : {&m->fmm_v, &m->fmm_vw, &m->fmm_wv})  // last step's plans: the
    if (*pl) {                                                  // geometry they hold is gone
      stokes_fmm_destroy(*pl);
      *pl = nullptr;
    }
  // with FMM residuals and walls, the channel response's vesicle-wall sums by FMM as well
  const bool resp_fmm = use_fmm && m->have_walls;
  // geometry at x^k (weights/normals feed the sums)
  ves_geom_kernel<<<V, n, 0, m->s>>>(n, m->d_x, m->d_D, m->d_spd, m->d_xs, m->d_nrm, m->d_w);
  SK(cudaGetLastError());
  ST(stokes_geom_update(m->ctx_v, reinterpret_cast<double *>(m->d_x), m->d_w,
                        reinterpret_cast<double *>(m->d_nrm), nullptr, m->s));
  if (m->close_v) {  // last step's pairs: its geometry is gone
    stokes_close_destroy(m->close_v);
    m->close_v = nullptr;
  }
  FmmPlanJob plan_job, plan_vw, plan_wv;
  if (use_plan || m->close_factor > 0.0)
    SK(cudaStreamSynchronize(m->s));  // the plans read the updated geometry
  if (use_plan)
    plan_job.start(m, m->ctx_v, std::max(m->resid_fmm_order, m->sweep_fmm_order));
  if (resp_fmm) {
    plan_vw.start(m, m->ctx_v, m->resid_fmm_order, m->Nt, reinterpret_cast<const double *>(m->d_wx));
    plan_wv.start(m, m->ctx_w, m->resid_fmm_order, m->Nv, reinterpret_cast<const double *>(m->d_x));
  }
  if (m->close_factor > 0.0) {
    const int cst = stokes_close_create(m->ctx_v, m->close_factor, m->close_K, &m->close_v);
    if (cst) return fail(m, cst, "close-evaluation pairs: %s", m->ctx_v->err.c_str());
  }
  // step 2: forces
  ves_forces_kernel<<<V, n, 0, m->s>>>(n, m->d_x, m->d_sigma, m->d_D, m->d_spd, m->d_xs, m->kappa_b,
                                       m->d_fb, m->d_f);
  SK(cudaGetLastError());
  // the block-diagonal self preconditioner of step 6 (geometry and dt only): built here, while
  // host threads build this step's FMM plans
  ST(precond_build(m, dt));
  // steps 3-5: channel response of the explicit forces
  double wait_ms = 0.0, resp_plan_ms = 0.0;
  auto join_timed = [&wait_ms](FmmPlanJob &job) {
    const auto tw = std::chrono::steady_clock::now();
    const int st = job.join();
    wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tw).count();
    return st;
  };
  if (resp_fmm) {
    int pst = join_timed(plan_vw);
    if (!pst) pst = join_timed(plan_wv);
    resp_plan_ms = std::max(plan_vw.ms, plan_wv.ms);
    if (pst) return fail(m, pst, "FMM plans of the channel response failed (%s / %s)",
                         m->ctx_v->err.c_str(), m->ctx_w->err.c_str());
    m->fmm_vw = plan_vw.take();
    m->fmm_wv = plan_wv.take();
  }
  if (m->have_walls)
    ST(channel_response(m, m->d_f, p_drive, m->d_ures, hp, use_fmm ? m->resid_fmm_order : 0));
  // right-hand side [S f_b + u_resp; ALC]
  double plan_ms = 0.0;
  if (use_plan) {
    const int pst = join_timed(plan_job);
    if (pst) return fail(m, pst, "FMM plan of the vesicles failed (%s)", m->ctx_v->err.c_str());
    m->fmm_v = plan_job.take();
    plan_ms = plan_job.ms;
  }
  if (use_fmm) {
    ST(fmm_sum(m, m->resid_fmm_order, false, m->d_fb, m->d_tmp3, "FMM right-hand side"));
  } else {
    ST(stokes_sum_eval(m->ctx_v, hp, reinterpret_cast<const double *>(m->d_fb), nullptr, 0.0,
                       reinterpret_cast<double *>(m->d_tmp3), m->s));
  }
  ST(add_close(m, m->d_fb, m->d_tmp3));
  ves_rhs_kernel<<<V, n, 0, m->s>>>(n, m->d_tmp3, m->have_walls ? m->d_ures : nullptr, m->d_w,
                                    m->d_L0, dt, m->d_b, m->d_Lk);
  SK(cudaGetLastError());
  // warm-start features of this step (principal-axes frame)
  if (n >= m->warm_modes) {
    ves_features_kernel<<<V, n, 0, m->s>>>(
        n, m->warm_modes, m->d_x, m->d_b, m->d_bprev, m->warm_history ? m->d_zprev : nullptr,
        m->d_zprev2, m->hist_count >= 2, m->d_A0, m->kappa_b, m->mu, m->d_frame, m->d_feat);
    SK(cudaGetLastError());
  }
  // step 6: GMRES with the block-diagonal self preconditioner, from the chosen initial iterate
  if (guess_mode == STOKES_GUESS_USER) {
    SK(cudaMemcpyAsync(m->d_xsol, guess, sizeof(double) * len, cudaMemcpyDeviceToDevice, m->s));
  } else if (guess_mode == STOKES_GUESS_MLP && m->warm_base == STOKES_WARM_BASE_EXTRAPOLATE &&
             m->hist_count < 2) {
    // a network trained on changes relative to the extrapolation has nothing to add to until
    // two solutions exist: the previous solution is the guess
    SK(cudaMemcpyAsync(m->d_xsol, m->d_zprev, sizeof(double) * len, cudaMemcpyDeviceToDevice, m->s));
  } else if (guess_mode == STOKES_GUESS_MLP) {
    int st = mlp_infer(model, V, m->d_feat, m->d_pred, m->s);
    if (st) return fail(m, st, "warm-start network inference failed");
    ves_guess_kernel<<<V, n, 0, m->s>>>(n, m->warm_modes, m->d_pred, m->d_frame, m->d_zprev,
                                        m->d_zprev2, m->warm_base == STOKES_WARM_BASE_EXTRAPOLATE,
                                        m->d_xsol);
    SK(cudaGetLastError());
  } else if (guess_mode == STOKES_GUESS_EXTRAPOLATE && m->hist_count >= 2) {
    extrapolate_kernel<<<grid_for(len), 256, 0, m->s>>>(len, m->d_zprev, m->d_zprev2, m->d_xsol);
    SK(cudaGetLastError());
  } else if (guess_mode == STOKES_GUESS_ZERO) {
    SK(cudaMemsetAsync(m->d_xsol, 0, sizeof(double) * len, m->s));
  } else {
    SK(cudaMemcpyAsync(m->d_xsol, m->d_zprev, sizeof(double) * len, cudaMemcpyDeviceToDevice, m->s));
  }
  SK(cudaStreamSynchronize(m->s));
  const auto t1 = std::chrono::steady_clock::now();
  int iters = 0, refinements = 0, accurate = 0;
  double rel = 0.0;
  int gst = STOKES_OK;
  if (precision != STOKES_FP32_KAHAN) {
    gst = gmres(m, dt, hp, m->d_b, m->d_xsol, tol, max_iter, &iters, &rel,
                guess_mode == STOKES_GUESS_ZERO);
  } else {
    // Mixed precision: corrections from GMRES with FP32-Kahan pair sums, residuals of the
    // FP64-accurate (double-float) operator (iterative refinement) while each refinement cuts
    // the residual at least 10x; the stiff operator S (dt kB u_ssss) makes FP32 sums of
    // high-mode densities cancel, so the refinement can stall -- GMRES on the FP64-accurate
    // operator then finishes from the refined iterate to tol.
    int st = STOKES_OK;
    const double bn = dnrm(m, len, m->d_b, &st);
    if (st) return fail(m, st, "norm reduction failed");
    const double one = 1.0, mone = -1.0;
    double prev = 1e300;
    bool finish64 = false;
    // A zero initial iterate needs no matvec (A 0 = 0).  A warm start's first residual only
    // feeds an inner solve to ~1e-3, so with double-float residuals (~8x an FP32-Kahan sum) it
    // is taken with the FP32-Kahan operator; with FMM residuals it is taken accurately like
    // every later one (a very good guess -- say an extrapolation -- leaves a residual below
    // what the FP32-Kahan operator resolves, and the refinement would stall on its noise).
    // Every convergence decision uses the FP64-accurate operator.
    bool zero_iterate = guess_mode == STOKES_GUESS_ZERO;
    bool rough = !zero_iterate && !use_fmm;
    for (;;) {
      SK(cudaMemcpyAsync(m->d_rr, m->d_b, sizeof(double) * len, cudaMemcpyDeviceToDevice, m->s));
      if (!zero_iterate) {
        if (!rough && use_fmm) {
          ST(step_matvec_fmm(m, dt, m->d_xsol, m->d_wk));
        } else {
          ST(step_matvec(m, dt, rough ? STOKES_FP32_KAHAN : hp, m->d_xsol, m->d_wk));
        }
        if (!rough) ++accurate;
        BK(cublasDaxpy(m->blas, int(len), &mone, m->d_wk, 1, m->d_rr, 1));
      }
      zero_iterate = false;
      const double rn = dnrm(m, len, m->d_rr, &st);
      if (st) return fail(m, st, "norm reduction failed");
      rel = bn > 0.0 ? rn / bn : 0.0;
      const bool was_rough = rough;
      rough = false;
      if (!was_rough && rel <= tol) break;
      if (rel > 0.1 * prev || refinements >= 8 || iters >= max_iter) {
        finish64 = true;
        break;
      }
      prev = rel;
      // inner solve to inner_tol (default 1e-3: about what the FP32-Kahan operator resolves on
      // stiff densities)
      const double tin = std::max(m->inner_tol, 0.5 * tol / rel);
      SK(cudaMemsetAsync(m->d_dd, 0, sizeof(double) * len, m->s));
      int it_in = 0;
      double rel_in = 0.0;
      const int gs = gmres(m, dt, STOKES_FP32_KAHAN, m->d_rr, m->d_dd, tin,
                           std::min(40, max_iter - iters), &it_in, &rel_in, true);
      iters += it_in;
      ++refinements;
      if (gs && gs != STOKES_ERR_NOT_CONVERGED) return gs;
      BK(cublasDaxpy(m->blas, int(len), &one, m->d_dd, 1, m->d_xsol, 1));
    }
    if (finish64) {
      int it64 = 0;
      gst = gmres(m, dt, hp, m->d_b, m->d_xsol, tol, std::max(max_iter - iters, 1), &it64, &rel);
      iters += it64;
    }
  }
  const auto t2 = std::chrono::steady_clock::now();
  if (out) {
    out->iterations = iters;
    out->residual = rel;
    out->setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    out->gmres_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
    out->refinements = refinements;
    out->accurate_residuals = accurate;
    out->fmm_plan_ms = plan_ms;
    out->precond_refresh = m->last_refresh;
    out->response_plan_ms = resp_plan_ms;
    out->plan_wait_ms = wait_ms;
  }
  if (gst) return gst;
  if (n >= m->warm_modes) {
    ves_targets_kernel<<<V, n, 0, m->s>>>(
        n, m->warm_modes, m->d_xsol, m->d_zprev, m->d_zprev2,
        m->warm_base == STOKES_WARM_BASE_EXTRAPOLATE && m->hist_count >= 2, m->d_frame, m->d_targ);
    SK(cudaGetLastError());
  }
  SK(cudaMemcpyAsync(m->d_bprev, m->d_b, sizeof(double) * len, cudaMemcpyDeviceToDevice, m->s));
  SK(cudaMemcpyAsync(m->d_zprev2, m->d_zprev, sizeof(double) * len, cudaMemcpyDeviceToDevice, m->s));
  SK(cudaMemcpyAsync(m->d_zprev, m->d_xsol, sizeof(double) * len, cudaMemcpyDeviceToDevice, m->s));
  m->hist_count = std::min(m->hist_count + 1, 2);
  // steps 7-9: x <- x + dt u, area correction, reparameterization; sigma <- sigma^{k+1}
  ves_advance_kernel<<<V, n, 0, m->s>>>(n, m->d_x, m->d_xsol, m->d_D, m->d_A0, dt);
  ves_reparam_kernel<<<V, n, 0, m->s>>>(n, m->d_x, m->d_D);
  extract_sigma_kernel<<<V, n, 0, m->s>>>(n, m->d_xsol, m->d_sigma);
  SK(cudaGetLastError());
  SK(cudaStreamSynchronize(m->s));
  if (out)
    out->total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return STOKES_OK;
}

int stokes_sim_last_features(stokes_sim *m, float *features, float *targets) {
  if (!m) return STOKES_ERR_ARG;
  if (!m->have_ves) return fail(m, STOKES_ERR_NO_GEOM, "vesicles must be set");
  const int nm = m->warm_modes;
  if (m->n < nm) return fail(m, STOKES_ERR_ARG, "features need n >= %d nodes per vesicle", nm);
  SK(cudaSetDevice(m->device));
  if (features)
    SK(cudaMemcpyAsync(features, m->d_feat, sizeof(float) * m->V * feat_dim(nm, m->warm_history),
                       cudaMemcpyDeviceToDevice, m->s));
  if (targets)
    SK(cudaMemcpyAsync(targets, m->d_targ, sizeof(float) * m->V * targ_dim(nm), cudaMemcpyDeviceToDevice, m->s));
  SK(cudaStreamSynchronize(m->s));
  return STOKES_OK;
}

int stokes_sim_get_state(stokes_sim *m, double *x_host, double *sigma_host, double *solution_host) {
  if (!m) return STOKES_ERR_ARG;
  if (!m->have_ves) return fail(m, STOKES_ERR_NO_GEOM, "vesicles must be set");
  SK(cudaSetDevice(m->device));
  SK(cudaStreamSynchronize(m->s));
  if (x_host) SK(cudaMemcpy(x_host, m->d_x, sizeof(double2) * m->Nv, cudaMemcpyDeviceToHost));
  if (sigma_host) SK(cudaMemcpy(sigma_host, m->d_sigma, sizeof(double) * m->Nv, cudaMemcpyDeviceToHost));
  if (solution_host)
    SK(cudaMemcpy(solution_host, m->d_xsol, sizeof(double) * 3 * m->Nv, cudaMemcpyDeviceToHost));
  return STOKES_OK;
}

int stokes_sim_set_state(stokes_sim *m, const double *x_host, const double *sigma_host) {
  if (!m) return STOKES_ERR_ARG;
  if (!m->have_ves) return fail(m, STOKES_ERR_NO_GEOM, "vesicles must be set");
  SK(cudaSetDevice(m->device));
  if (x_host) SK(cudaMemcpy(m->d_x, x_host, sizeof(double2) * m->Nv, cudaMemcpyHostToDevice));
  if (sigma_host) SK(cudaMemcpy(m->d_sigma, sigma_host, sizeof(double) * m->Nv, cudaMemcpyHostToDevice));
  // a new start: no previous step (nor its preconditioner)
  m->pinv_valid = false;
  SK(cudaMemset(m->d_bprev, 0, sizeof(double) * 3 * m->Nv));
  SK(cudaMemset(m->d_zprev, 0, sizeof(double) * 3 * m->Nv));
  SK(cudaMemset(m->d_zprev2, 0, sizeof(double) * 3 * m->Nv));
  m->hist_count = 0;
  return STOKES_OK;
}

int stokes_sim_get_history(stokes_sim *m, double *L0_host, double *A0_host, double *zprev_host,
                           double *bprev_host) {
  if (!m) return STOKES_ERR_ARG;
  if (!m->have_ves) return fail(m, STOKES_ERR_NO_GEOM, "vesicles must be set");
  SK(cudaSetDevice(m->device));
  SK(cudaStreamSynchronize(m->s));
  const size_t len = size_t(3) * m->Nv;
  if (L0_host) SK(cudaMemcpy(L0_host, m->d_L0, sizeof(double) * m->V, cudaMemcpyDeviceToHost));
  if (A0_host) SK(cudaMemcpy(A0_host, m->d_A0, sizeof(double) * m->V, cudaMemcpyDeviceToHost));
  if (zprev_host) SK(cudaMemcpy(zprev_host, m->d_zprev, sizeof(double) * len, cudaMemcpyDeviceToHost));
  if (bprev_host) SK(cudaMemcpy(bprev_host, m->d_bprev, sizeof(double) * len, cudaMemcpyDeviceToHost));
  return STOKES_OK;
}

int stokes_sim_set_history(stokes_sim *m, const double *L0_host, const double *A0_host,
                           const double *zprev_host, const double *bprev_host) {
  if (!m) return STOKES_ERR_ARG;
  if (!m->have_ves) return fail(m, STOKES_ERR_NO_GEOM, "vesicles must be set");
  SK(cudaSetDevice(m->device));
  SK(cudaStreamSynchronize(m->s));
  const size_t len = size_t(3) * m->Nv;
  if (L0_host) SK(cudaMemcpy(m->d_L0, L0_host, sizeof(double) * m->V, cudaMemcpyHostToDevice));
  if (A0_host) SK(cudaMemcpy(m->d_A0, A0_host, sizeof(double) * m->V, cudaMemcpyHostToDevice));
  if (zprev_host) {
    SK(cudaMemcpy(m->d_zprev, zprev_host, sizeof(double) * len, cudaMemcpyHostToDevice));
    SK(cudaMemcpy(m->d_xsol, zprev_host, sizeof(double) * len, cudaMemcpyHostToDevice));
    // the solution two steps back is not part of the history: the previous change restarts at 0
    SK(cudaMemcpy(m->d_zprev2, zprev_host, sizeof(double) * len, cudaMemcpyHostToDevice));
    m->hist_count = 1;
  }
  if (bprev_host) SK(cudaMemcpy(m->d_bprev, bprev_host, sizeof(double) * len, cudaMemcpyHostToDevice));
  return STOKES_OK;
}

int stokes_sim_set_warm_modes(stokes_sim *m, int modes) {
  if (!m) return STOKES_ERR_ARG;
  if (modes < 4 || modes > kMaxModes || (modes & 1))
    return fail(m, STOKES_ERR_ARG, "warm-start modes must be even and in [4, %d]", kMaxModes);
  if (m->have_ves && m->n < modes)
    return fail(m, STOKES_ERR_ARG, "%d modes need at least %d nodes per vesicle", modes, modes);
  m->warm_modes = modes;
  return STOKES_OK;
}

int stokes_sim_set_warm_base(stokes_sim *m, int base) {
  if (!m) return STOKES_ERR_ARG;
  if (base != STOKES_WARM_BASE_PREVIOUS && base != STOKES_WARM_BASE_EXTRAPOLATE)
    return fail(m, STOKES_ERR_ARG, "unknown warm-start base %d", base);
  m->warm_base = base;
  return STOKES_OK;
}

int stokes_sim_set_warm_history(stokes_sim *m, int on) {
  if (!m) return STOKES_ERR_ARG;
  m->warm_history = on != 0;
  return STOKES_OK;
}

int stokes_sim_get_warm_modes(const stokes_sim *m, int *modes) {
  if (!m || !modes) return STOKES_ERR_ARG;
  *modes = m->warm_modes;
  return STOKES_OK;
}

int stokes_sim_set_close_eval(stokes_sim *m, double factor, int upsample) {
  if (!m) return STOKES_ERR_ARG;
  if (!(factor == 0.0 || (factor > 0.0 && factor <= 50.0)) || upsample < 1 || upsample > 64)
    return fail(m, STOKES_ERR_ARG, "close evaluation: factor 0 (off) or in (0, 50], upsample in [1, 64]");
  m->close_factor = factor;
  m->close_K = upsample;
  return STOKES_OK;
}

int stokes_sim_set_residual_fmm(stokes_sim *m, int order, int leaf_size) {
  if (!m) return STOKES_ERR_ARG;
  if (order != 0 && (order < 4 || order > 40))
    return fail(m, STOKES_ERR_ARG, "FMM order must be 0 (off) or in [4, 40]");
  if (leaf_size < 4 || leaf_size > 4096) return fail(m, STOKES_ERR_ARG, "leaf size must be in [4, 4096]");
  m->resid_fmm_order = order;
  m->resid_fmm_leaf = leaf_size;
  return STOKES_OK;
}

int stokes_sim_set_sweep_fmm(stokes_sim *m, int order) {
  if (!m) return STOKES_ERR_ARG;
  if (order != 0 && (order < 4 || order > 40))
    return fail(m, STOKES_ERR_ARG, "FMM order must be 0 (off) or in [4, 40]");
  m->sweep_fmm_order = order;
  return STOKES_OK;
}

int stokes_sim_set_restart(stokes_sim *m, int restart) {
  if (!m) return STOKES_ERR_ARG;
  if (!m->have_ves) return fail(m, STOKES_ERR_NO_GEOM, "vesicles must be set");
  if (restart < 2 || restart > 2000) return fail(m, STOKES_ERR_ARG, "restart must be in [2, 2000]");
  SK(cudaSetDevice(m->device));
  SK(cudaStreamSynchronize(m->s));
  SK(dalloc(m->d_V, size_t(3) * m->Nv * (restart + 1)));
  SK(dalloc(m->d_h, restart + 1));
  m->gm_m = restart;
  return STOKES_OK;
}

int stokes_sim_sizes(const stokes_sim *m, int *n_vesicles, int *nodes_per_vesicle,
                     int *wall_nodes) {
  if (!m || !n_vesicles || !nodes_per_vesicle || !wall_nodes) return STOKES_ERR_ARG;
  *n_vesicles = m->have_ves ? m->V : 0;
  *nodes_per_vesicle = m->have_ves ? m->n : 0;
  *wall_nodes = m->have_walls ? m->Nt : 0;
  return STOKES_OK;
}

}  // extern "C"
