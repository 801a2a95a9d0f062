// fds.cuh -- fast direct solver for the fixed channel walls (Sec. 4), internal interface.
#pragma once
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <string>

namespace stokes {

struct fds_solver;

struct fds_params {
  double tol = 1e-12;  // relative truncation of every interpolative decomposition
  int leaf = 64;       // nodes per leaf box of the HBS tree
  int n_proxy = 64;    // proxy points per HBS box
  int n_proxy_nb = 80; // proxy points per neighbour section (Sec. 4.2)
  int sec_max = 45;    // nodes of the smallest (touching) neighbour section, n_max of Sec. 4.2
  bool recompress = true;  // also skeletonise A_m's columns: R = A_m(J, J_c) C (Sec. 4.2 remark)
};

struct fds_info {
  int levels = 0;          // HBS levels below the root
  int max_rank = 0;        // largest skeleton of any box
  int root_size = 0;       // order of the dense root block
  int neighbour_rank = 0;  // columns of L (both neighbours, both walls)
  int sections = 0;        // neighbour sections (both neighbours, both walls)
  int neighbour_col_rank = 0;  // rows of C (column skeletons; 0 without the recompression)
  double host_ms = 0.0;    // compression and per-box inverses (host threads)
  double device_ms = 0.0;  // uploads, the neighbour factors, K^-1 (device)
  size_t device_bytes = 0; // device memory held by the solver
  size_t solve_bytes = 0;  // matrices one single-right-hand-side solve reads
};

// Builds the solver for the walls of one cell: n_w nodes per wall, host arrays in the wall
// operator's node order (lower wall then upper): nodes (x, y), weights, unit normals,
// curvature; period d.  Runs the device part on stream s.  Returns a stokes.h status and
// sets err on failure.
int fds_build(fds_solver **out, int n_w, const double *nodes, const double *weights,
              const double *normals, const double *curvature, double period, const fds_params &p,
              cudaStream_t s, cublasHandle_t blas, cusolverDnHandle_t sol, std::string &err);

// X (4 n_w x nrhs, column-major, device) <- A^-1 X, asynchronous on stream s.
int fds_solve(fds_solver *f, double *X, int nrhs, cudaStream_t s, cublasHandle_t blas,
              std::string &err);

void fds_get_info(const fds_solver *f, fds_info *info);
void fds_destroy(fds_solver *f);

}  // namespace stokes
