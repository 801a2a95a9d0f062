// fds.cu -- fast direct solver for the fixed channel walls (Sec. 4).
//
// The wall operator A = -I/2 + D^near (Nystrom with the curvature diagonal; unknowns
// (tau_1, tau_2) interleaved per node, lower wall then upper) is split as in Eq. (formA) into
// the unit cell's self interaction A_0 and the neighbour interactions A_{-1}, A_{+1}:
//
//  * A_0 in HBS form (Sec. 4.3) by recursive skeletonisation: a binary tree of node ranges
//    (root; the two walls; halves down to leaves of <= `leaf` nodes).  At every box, an
//    interpolative decomposition of the box's unknowns against everything outside it gives
//    its skeleton J and interpolation matrix P (one skeleton for rows and columns, U = V = P):
//    the probe rows are the box's interactions, in both directions, with the active unknowns
//    of the other boxes of its level inside a proxy circle (1.5 x the box radius), the fields
//    of stokeslets and stresslets at the proxy points (any flow the far sources make inside the
//    circle) and the box's own field at the proxy points (what the far targets see).  The box
//    is then inverted by Eqs. (def_muhD)-(def_muG): D^ = (P^T D^-1 P)^-1, E = D^-1 P D^,
//    F^* = D^ P^T D^-1, G = D^-1 - D^-1 P D^ P^T D^-1, where D is the leaf's diagonal block of
//    A_0 or, for a parent, [D^_a, A_0(J_a, J_b); A_0(J_b, J_a), D^_b].  The root block is
//    inverted densely; A_0^-1 v is then one upward pass (v^ = F^* v), the root solve and one
//    downward pass (u = E u^ + G v).
//  * A_{+1} and A_{-1} factored as L R (Sec. 4.2): each wall is cut dyadically toward the
//    neighbour, down to a touching section of <= sec_max nodes.  A section away from the
//    neighbour is skeletonised against stokeslets and stresslets at n_proxy_nb points on a
//    circle 0.9 x its centre's distance to the shared cell boundary; the touching section
//    against points on a circle 1.75 x its radius together with the neighbour nodes inside
//    that circle.  L is block diagonal (the sections' P's) and R = A_m(J, :).
//  * Recompression (the remark closing Sec. 4.2, on by default): R = A_m(J, :) is itself low
//    rank block by block, so its columns are skeletonised the same way -- each wall cut
//    dyadically toward the end whose sources the shift m d carries next to the cell, a
//    section's columns interpolated from a column skeleton J_c against the velocity its
//    densities make on a proxy circle and, for the touching section, at the cell's own nodes
//    inside that circle -- giving A_m ~ L S C with S = A_m(J, J_c) (l x l_c) and C block
//    diagonal (the sections' interpolation matrices).
//  * A^-1 by Sherman-Morrison-Woodbury, Eq. (woodbury1): K^-1 = (I + R A_0^-1 L)^-1 is formed
//    once (A_0^-1 L by the tree passes on L's l columns, then discarded); a solve is
//    y = A_0^-1 v, x = A_0^-1 (v - L K^-1 R y) -- the same as y - A_0^-1 L K^-1 R y, with the
//    second tree pass in place of a stored dense A_0^-1 L.  With the recompression
//    K^-1 R y = (K^-1 S)(C y), K^-1 S stored (l x l_c), so a solve reads the HBS tables twice
//    and, once each, C's and L's section blocks and K^-1 S: nothing of size n x l.  Without it,
//    R (l x n) and K^-1 are read.
//
// The compression and the small per-box inverses run on the host in FP64 (threads over the
// boxes of one level); the neighbour factors, K^-1 and every solve run on the device.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <numeric>
#include <thread>
#include <vector>

#include "fds.cuh"
#include "bulk_pipe.cuh"
#include "stokes.h"

namespace stokes {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kHbsThreads = 256;
constexpr int kHbsCols = 8;       // right-hand sides per CTA of a level pass
constexpr int kRowTile = 32;      // output rows per CTA of a level pass
constexpr int kChunk = 256;       // right-hand sides per pass through the tree

// ---------------------------------------------------------------------------
// host dense matrices (column-major, FP64)
// ---------------------------------------------------------------------------
struct HMat {
  int r = 0, c = 0;
  std::vector<double> a;
  HMat() = default;
  HMat(int r_, int c_) : r(r_), c(c_), a(size_t(r_) * c_, 0.0) {}
  double &operator()(int i, int j) { return a[i + size_t(j) * r]; }
  double operator()(int i, int j) const { return a[i + size_t(j) * r]; }
  double *col(int j) { return a.data() + size_t(j) * r; }
  const double *col(int j) const { return a.data() + size_t(j) * r; }
};

HMat mul(const HMat &A, const HMat &B) {  // A B
  HMat C(A.r, B.c);
  for (int j = 0; j < B.c; ++j) {
    double *cj = C.col(j);
    for (int k = 0; k < A.c; ++k) {
      const double b = B(k, j);
      if (b == 0.0) continue;
      const double *ak = A.col(k);
      for (int i = 0; i < A.r; ++i) cj[i] += ak[i] * b;
    }
  }
  return C;
}

HMat mul_nt(const HMat &A, const HMat &B) {  // A B^T
  HMat C(A.r, B.r);
  for (int k = 0; k < A.c; ++k) {
    const double *ak = A.col(k);
    for (int j = 0; j < B.r; ++j) {
      const double b = B(j, k);
      if (b == 0.0) continue;
      double *cj = C.col(j);
      for (int i = 0; i < A.r; ++i) cj[i] += ak[i] * b;
    }
  }
  return C;
}

// In-place inverse by LU with partial pivoting (P A = L U, then L U X = P).
bool invert(HMat &A) {
  const int n = A.r;
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(A(k, k));
    for (int i = k + 1; i < n; ++i)
      if (fabs(A(i, k)) > best) {
        best = fabs(A(i, k));
        p = i;
      }
    if (!(best > 0.0)) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A(k, j), A(p, j));
    const double inv = 1.0 / A(k, k);
    double *ck = A.col(k);
    for (int i = k + 1; i < n; ++i) ck[i] *= inv;
    for (int j = k + 1; j < n; ++j) {
      double *cj = A.col(j);
      const double f = cj[k];
      if (f == 0.0) continue;
      for (int i = k + 1; i < n; ++i) cj[i] -= ck[i] * f;
    }
  }
  HMat X(n, n);
  for (int j = 0; j < n; ++j) X(j, j) = 1.0;
  for (int k = 0; k < n; ++k)
    if (piv[k] != k)
      for (int j = 0; j < n; ++j) std::swap(X(k, j), X(piv[k], j));
  for (int j = 0; j < n; ++j) {
    double *x = X.col(j);
    for (int k = 0; k < n; ++k) {  // unit lower triangle
      const double xk = x[k];
      if (xk == 0.0) continue;
      const double *l = A.col(k);
      for (int i = k + 1; i < n; ++i) x[i] -= l[i] * xk;
    }
    for (int k = n - 1; k >= 0; --k) {  // upper triangle
      x[k] /= A(k, k);
      const double xk = x[k];
      const double *u = A.col(k);
      for (int i = 0; i < k; ++i) x[i] -= u[i] * xk;
    }
  }
  A = std::move(X);
  return true;
}

// Column interpolative decomposition Z ~ Z(:, J) X (X is k x n with X(:, J) = I) by
// Householder QR with column pivoting, stopped once the next pivot's remaining norm is at most
// tol times the first's.  Z (m x n) is overwritten.
void column_id(HMat &Z, double tol, std::vector<int> &J, HMat &X) {
  const int m = Z.r, n = Z.c;
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::vector<double> nrm(n), ref(n);
  for (int q = 0; q < n; ++q) {
    const double *z = Z.col(q);
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += z[i] * z[i];
    nrm[q] = ref[q] = s;
  }
  const int kmax = std::min(m, n);
  int k = 0;
  double r00 = 0.0;
  std::vector<double> v(m);
  for (int j = 0; j < kmax; ++j) {
    int p = j;
    for (int q = j + 1; q < n; ++q)
      if (nrm[q] > nrm[p]) p = q;
    double s = 0.0;
    {
      const double *z = Z.col(p);
      for (int i = j; i < m; ++i) s += z[i] * z[i];
    }
    const double rjj = sqrt(s);
    if (j == 0) r00 = rjj;
    if (!(rjj > tol * r00) || rjj == 0.0) break;
    if (p != j) {
      std::swap_ranges(Z.col(j), Z.col(j) + m, Z.col(p));
      std::swap(perm[j], perm[p]);
      std::swap(nrm[j], nrm[p]);
      std::swap(ref[j], ref[p]);
    }
    double *zj = Z.col(j);
    const double x0 = zj[j];
    const double alpha = x0 >= 0.0 ? -rjj : rjj;
    v[j] = x0 - alpha;
    for (int i = j + 1; i < m; ++i) v[i] = zj[i];
    const double vtv = 2.0 * (s - x0 * alpha);
    const double beta = vtv > 0.0 ? 2.0 / vtv : 0.0;
    for (int q = j + 1; q < n; ++q) {
      double *zq = Z.col(q);
      double dot = 0.0;
      for (int i = j; i < m; ++i) dot += v[i] * zq[i];
      const double f = beta * dot;
      for (int i = j; i < m; ++i) zq[i] -= f * v[i];
      nrm[q] -= zq[j] * zq[j];
      if (nrm[q] <= 1e-8 * ref[q]) {  // cancellation: recompute the remaining norm
        double t = 0.0;
        for (int i = j + 1; i < m; ++i) t += zq[i] * zq[i];
        nrm[q] = ref[q] = t;
      }
    }
    zj[j] = alpha;
    k = j + 1;
  }
  if (k == 0) k = 1;  // a zero block keeps one unknown
  J.assign(perm.begin(), perm.begin() + k);
  X = HMat(k, n);
  for (int c = 0; c < k; ++c) X(c, perm[c]) = 1.0;
  std::vector<double> t(k);
  for (int q = k; q < n; ++q) {  // R11^-1 R12 by back substitution
    const double *zq = Z.col(q);
    for (int i = k - 1; i >= 0; --i) {
      double s = zq[i];
      for (int c = i + 1; c < k; ++c) s -= Z(i, c) * t[c];
      t[i] = Z(i, i) != 0.0 ? s / Z(i, i) : 0.0;
    }
    for (int c = 0; c < k; ++c) X(c, perm[q]) = t[c];
  }
}

template <class F>
void parallel_for(int n, F f) {
  const int nt = std::max(1, std::min<int>(n, int(std::thread::hardware_concurrency())));
  if (nt == 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&] {
      for (int i = next++; i < n; i = next++) f(i);
    });
  for (auto &x : th) x.join();
}

// ---------------------------------------------------------------------------
// the wall operator, entry by entry
// ---------------------------------------------------------------------------
struct WallGeom {
  int nw = 0, Nt = 0;
  double d = 0.0;
  std::vector<double> x, y, nx, ny, w, kap;
};

// A_m(u_i, u_j) for unknowns u = 2 node + component: the stresslet of Eq. (D) times w_j
// from node j shifted by m d; at m = 0 and i = j the curvature diagonal
// -kappa_j/(2 pi) w_j t t^T minus the jump 1/2.
__host__ __device__ inline double a_entry(int ui, int uj, int m, const double *x, const double *y,
                                          const double *nx, const double *ny, const double *w,
                                          const double *kap, double d) {
  const int i = ui >> 1, ci = ui & 1, j = uj >> 1, cj = uj & 1;
  if (m == 0 && i == j) {
    const double tx = -ny[j], ty = nx[j];
    const double c = -kap[j] / (2.0 * kPi) * w[j];
    return c * (ci ? ty : tx) * (cj ? ty : tx) - (ci == cj ? 0.5 : 0.0);
  }
  const double r1 = x[i] - (x[j] + m * d), r2 = y[i] - y[j];
  const double rr = r1 * r1 + r2 * r2;
  const double rn = r1 * nx[j] + r2 * ny[j];
  return (ci ? r2 : r1) * (cj ? r2 : r1) * rn / (kPi * rr * rr) * w[j];
}

inline double a_host(const WallGeom &g, int ui, int uj, int m) {
  return a_entry(ui, uj, m, g.x.data(), g.y.data(), g.nx.data(), g.ny.data(), g.w.data(),
                 g.kap.data(), g.d);
}

// Probe matrix of a group of unknowns `It` (one column each): rows A_m(It, near) (and, when
// two_sided, A_m(near, It)^T), then for every proxy point on the circle (cx, cy, rad) the
// stokeslet and the radial-normal stresslet it places on the unknown (two source components
// each), then (when targets) the velocity the unknown's density makes at the proxy point.
HMat probe_matrix(const WallGeom &g, const std::vector<int> &It, const std::vector<int> &near,
                  int m, bool two_sided, double cx, double cy, double rad, int npx,
                  bool targets) {
  const int nn = int(near.size());
  const int rows = nn * (two_sided ? 2 : 1) + 4 * npx + (targets ? 2 * npx : 0);
  HMat Z(rows, int(It.size()));
  for (int q = 0; q < int(It.size()); ++q) {
    const int u = It[q], node = u >> 1, comp = u & 1;
    double *z = Z.col(q);
    int r = 0;
    for (int p = 0; p < nn; ++p) z[r++] = a_host(g, u, near[p], m);
    if (two_sided)
      for (int p = 0; p < nn; ++p) z[r++] = a_host(g, near[p], u, m);
    for (int p = 0; p < npx; ++p) {
      const double c = cos(2.0 * kPi * p / npx), s = sin(2.0 * kPi * p / npx);
      const double px = cx + rad * c, py = cy + rad * s;
      const double r1 = g.x[node] - px, r2 = g.y[node] - py;
      const double rr = r1 * r1 + r2 * r2;
      const double rc = comp ? r2 : r1;
      const double lg = -0.5 * log(rr);
      z[r++] = ((comp == 0 ? lg : 0.0) + rc * r1 / rr) / (4.0 * kPi);
      z[r++] = ((comp == 1 ? lg : 0.0) + rc * r2 / rr) / (4.0 * kPi);
      const double rn = r1 * c + r2 * s;
      z[r++] = rc * r1 * rn / (kPi * rr * rr);
      z[r++] = rc * r2 * rn / (kPi * rr * rr);
      if (targets) {
        const double t1 = px - g.x[node], t2 = py - g.y[node];
        const double tt = t1 * t1 + t2 * t2;
        const double tn = t1 * g.nx[node] + t2 * g.ny[node];
        const double f = (comp ? t2 : t1) * tn / (kPi * tt * tt) * g.w[node];
        z[r++] = t1 * f;
        z[r++] = t2 * f;
      }
    }
  }
  return Z;
}

// Probe matrix of a group of source unknowns `It` of A_m (one column each), for its column
// skeleton: rows A_m(near, It) for the target unknowns `near`, then for every proxy point on
// the circle (cx, cy, rad) the velocity the unknown's density makes there.  The circle is
// drawn around the sources before the shift m d (the kernel depends on differences only), so
// the near targets are those within it once moved by -m d.
HMat probe_cols(const WallGeom &g, const std::vector<int> &It, const std::vector<int> &near,
                int m, double cx, double cy, double rad, int npx) {
  const int nn = int(near.size());
  HMat Z(nn + 2 * npx, int(It.size()));
  for (int q = 0; q < int(It.size()); ++q) {
    const int u = It[q], node = u >> 1, comp = u & 1;
    double *z = Z.col(q);
    int r = 0;
    for (int p = 0; p < nn; ++p) z[r++] = a_host(g, near[p], u, m);
    for (int p = 0; p < npx; ++p) {
      const double px = cx + rad * cos(2.0 * kPi * p / npx), py = cy + rad * sin(2.0 * kPi * p / npx);
      const double t1 = px - g.x[node], t2 = py - g.y[node];
      const double tt = t1 * t1 + t2 * t2;
      const double tn = t1 * g.nx[node] + t2 * g.ny[node];
      const double f = (comp ? t2 : t1) * tn / (kPi * tt * tt) * g.w[node];
      z[r++] = t1 * f;
      z[r++] = t2 * f;
    }
  }
  return Z;
}

struct Box {
  int a = 0, b = 0;                  // node range
  double x0 = 0, x1 = 0, y0 = 0, y1 = 0;  // bounding box of the nodes
  std::vector<int> act, skel;        // active unknowns, skeleton (a subset of act)
  HMat Dh, E, Ft, G;
};

// ---------------------------------------------------------------------------
// device passes
// ---------------------------------------------------------------------------
struct HbsBox {
  int n, k, in_off, out_off;  // active unknowns, skeleton, offsets in the level vectors
  long long ft, e, g;         // offsets of F^* (k x n), E (n x k), G (n x n)
};

// mode 0 (upward):   y[out_off + r] = sum_j F^*[r + j k] x1[in_off + j],   r < k
// mode 1 (downward): y[in_off + r]  = sum_j E[r + j n] x1[out_off + j]
//                                   + sum_j G[r + j n] x2[in_off + j],     r < n
// for the right-hand sides [blockIdx.z NC, ...) of column-major x1, x2, y.  E and G are stored
// back to back, so both modes are one column-major product y = M v with v the box's inputs,
// staged in shared memory.  A CTA takes the rows [blockIdx.y RT, ...) of its box: each row is
// split over kHbsThreads / RT threads that sum strided shares of the columns (two accumulators
// each, NC right-hand sides at once, so every matrix element is read once per CTA), reduced in
// shared memory.  A warp reads RT consecutive doubles of 32 / RT columns.  RT = kRowTile (32)
// for levels with many boxes; the small row tile (8 rows, 32 threads per row) serves the top
// levels, where a few boxes would leave most SMs idle and each thread would walk a long chain
// of columns: four times the CTAs and a quarter of the chain.
// Dynamic shared memory: (NC max_cols + kHbsThreads NC) doubles.
constexpr int kRowTileSmall = 8;
template <int NC, int RT = kRowTile>
__global__ void __launch_bounds__(kHbsThreads)
    hbs_level_kernel(const HbsBox *boxes, const double *mats, int mode, int ncol, const double *x1,
                     long long ld1, const double *x2, long long ld2, double *y, long long ldy) {
  extern __shared__ double sh[];
  const HbsBox b = boxes[blockIdx.x];
  const int R = mode == 0 ? b.k : b.n;
  const int r0 = blockIdx.y * RT;
  if (r0 >= R) return;  // uniform over the CTA
  const int c0 = blockIdx.z * NC;
  const int nc = min(NC, ncol - c0);
  const int C = mode == 0 ? b.n : b.k + b.n;
  const int C1 = mode == 0 ? b.n : b.k;
  const long long o1 = mode == 0 ? b.in_off : b.out_off;
  const long long oy = mode == 0 ? b.out_off : b.in_off;
  const double *M = mats + (mode == 0 ? b.ft : b.e);
  double *v = sh;            // [NC][C]
  double *part = sh + NC * C;  // [T][NC]
  for (int idx = threadIdx.x; idx < NC * C; idx += blockDim.x) {
    const int c = idx / C, j = idx - (idx / C) * C;
    double val = 0.0;
    if (c < nc)
      val = j < C1 ? x1[(c0 + c) * ld1 + o1 + j] : x2[(c0 + c) * ld2 + b.in_off + (j - C1)];
    v[idx] = val;
  }
  __syncthreads();
  constexpr int split = kHbsThreads / RT;
  const int Rt = min(RT, R - r0);
  const int r = threadIdx.x % RT, q = threadIdx.x / RT;
  double a0[NC], a1[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) a0[c] = a1[c] = 0.0;
  if (r < Rt) {
    const double *Mr = M + r0 + r;
    int j = q;
    for (; j + split < C; j += 2 * split) {
      const double m0 = Mr[size_t(j) * R], m1 = Mr[size_t(j + split) * R];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        a0[c] = fma(m0, v[c * C + j], a0[c]);
        a1[c] = fma(m1, v[c * C + j + split], a1[c]);
      }
    }
    if (j < C) {
      const double m0 = Mr[size_t(j) * R];
#pragma unroll
      for (int c = 0; c < NC; ++c) a0[c] = fma(m0, v[c * C + j], a0[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) part[threadIdx.x * NC + c] = a0[c] + a1[c];
  __syncthreads();
  if (q == 0 && r < Rt) {
#pragma unroll
    for (int c = 0; c < NC; ++c) a0[c] = part[r * NC + c];
    for (int p = 1; p < split; ++p)
#pragma unroll
      for (int c = 0; c < NC; ++c) a0[c] += part[(p * RT + r) * NC + c];
    for (int c = 0; c < nc; ++c) y[(c0 + c) * ldy + oy + r0 + r] = a0[c];
  }
}

// R (l x nA, column-major): R[r, u] = A_{m_r}(J_r, u).
__global__ void fill_rows_kernel(int l, int nA, const int *J, const int *mr, const double *x,
                                 const double *y, const double *nx, const double *ny,
                                 const double *w, const double *kap, double d, double *R) {
  const size_t total = size_t(l) * nA;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total;
       idx += size_t(gridDim.x) * blockDim.x) {
    const int r = int(idx % l), u = int(idx / l);
    R[idx] = a_entry(J[r], u, mr[r], x, y, nx, ny, w, kap, d);
  }
}

// L (nA x l) block diagonal: section s puts its rows x cols block at (row0, col0).
struct SecBlock {
  int row0, rows, col0, cols;
  long long off;
};

// S (l x lc, column-major): S[r, c] = A_m(J_r, J_c) where the row and column skeletons belong
// to the same neighbour m, else 0 (the two neighbours' factors are separate blocks).
__global__ void fill_core_kernel(int l, int lc, const int *J, const int *mr, const int *Jc,
                                 const int *mc, const double *x, const double *y,
                                 const double *nx, const double *ny, const double *w,
                                 const double *kap, double d, double *S) {
  const size_t total = size_t(l) * lc;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total;
       idx += size_t(gridDim.x) * blockDim.x) {
    const int r = int(idx % l), c = int(idx / l);
    S[idx] = mr[r] == mc[c] ? a_entry(J[r], Jc[c], mr[r], x, y, nx, ny, w, kap, d) : 0.0;
  }
}

__global__ void scatter_blocks_kernel(const SecBlock *sec, const double *vals, int nA, double *L) {
  const SecBlock s = sec[blockIdx.x];
  for (int idx = threadIdx.x; idx < s.rows * s.cols; idx += blockDim.x) {
    const int i = idx % s.rows, c = idx / s.rows;
    L[size_t(s.col0 + c) * nA + s.row0 + i] = vals[s.off + idx];
  }
}

__global__ void add_identity_kernel(int n, double *K) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) K[size_t(i) * n + i] += 1.0;
}

__global__ void set_identity_kernel(int n, double *K) {
  const size_t nn = size_t(n) * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < nn;
       i += size_t(gridDim.x) * blockDim.x)
    K[i] = (i % size_t(n + 1) == 0) ? 1.0 : 0.0;
}

// y = M x for a column-major M (rows x cols, leading dimension rows), one right-hand side,
// in two fixed-order passes: partial[ch][r] = sum over the columns of chunk ch of M[r, u] x[u]
// (a CTA per (tile of kGemvRows rows, column chunk), the chunk of x staged in shared memory;
// with an even leading dimension a thread takes two adjacent rows as one 16-byte load, else
// one row; eight columns in flight per thread), then y[r] = alpha sum_ch partial[ch][r]
// (+ y[r] when accumulate).  HBM-bound: M is read once.
constexpr int kGemvThreads = 128;
constexpr int kGemvRows = 2 * kGemvThreads;  // rows per CTA
constexpr int kGemvMaxChunk = 2048;          // columns per chunk (staged x: 16 KB)

template <bool PAIR>
__global__ void __launch_bounds__(kGemvThreads)
    gemv_cm_partial_kernel(int rows, int cols, int chunk, const double *__restrict__ M,
                           const double *__restrict__ x, double *__restrict__ partial) {
  __shared__ double xs[kGemvMaxChunk];
  const int u0 = blockIdx.y * chunk;
  const int nu = min(chunk, cols - u0);
  for (int j = threadIdx.x; j < nu; j += blockDim.x) xs[j] = x[u0 + j];
  __syncthreads();
  constexpr int RPT = PAIR ? 2 : 1;  // rows per thread
  for (int pass = 0; pass < 2 / RPT; ++pass) {
    const int r = blockIdx.x * kGemvRows + (PAIR ? 2 * threadIdx.x : pass * kGemvThreads + threadIdx.x);
    if (r >= rows) continue;
    double a[4][RPT];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int h = 0; h < RPT; ++h) a[q][h] = 0.0;
    const double *Mr = M + size_t(u0) * rows + r;
    int j = 0;
    for (; j + 7 < nu; j += 8) {
      double m[8][RPT];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if constexpr (PAIR) {
          const double2 v = __ldg(reinterpret_cast<const double2 *>(Mr + size_t(j + q) * rows));
          m[q][0] = v.x;
          m[q][RPT - 1] = v.y;
        } else {
          m[q][0] = __ldg(Mr + size_t(j + q) * rows);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int h = 0; h < RPT; ++h) a[q & 3][h] = fma(m[q][h], xs[j + q], a[q & 3][h]);
    }
    for (; j < nu; ++j) {
      if constexpr (PAIR) {
        const double2 v = __ldg(reinterpret_cast<const double2 *>(Mr + size_t(j) * rows));
        a[0][0] = fma(v.x, xs[j], a[0][0]);
        a[0][RPT - 1] = fma(v.y, xs[j], a[0][RPT - 1]);
      } else {
        a[0][0] = fma(__ldg(Mr + size_t(j) * rows), xs[j], a[0][0]);
      }
    }
    double *pr = partial + size_t(blockIdx.y) * rows + r;
#pragma unroll
    for (int h = 0; h < RPT; ++h)
      if (r + h < rows) pr[h] = (a[0][h] + a[1][h]) + (a[2][h] + a[3][h]);
  }
}

// The same partial products for an even leading dimension of at most kColsMaxRows rows, with
// every CTA streaming whole columns: CTA ch reads columns [ch chunk, ...) contiguously (all
// rows), a thread owning the row pairs t, t + kColsThreads, ... (P of them, 16-byte loads), U
// columns in flight.  Long contiguous runs keep the DRAM pages open; the tile kernel above reads
// 2 KB pieces of columns 8 l bytes apart instead.
constexpr int kColsThreads = 256;
constexpr int kColsMaxRows = 2 * kColsThreads * 8;  // 4096 (P = 8)
template <int P, int U>
__global__ void __launch_bounds__(kColsThreads)
    gemv_cols_partial_kernel(int rows, int cols, int chunk, const double *__restrict__ M,
                             const double *__restrict__ x, double *__restrict__ partial) {
  __shared__ double xs[kGemvMaxChunk];
  const int u0 = blockIdx.x * chunk;
  const int nu = min(chunk, cols - u0);
  for (int j = threadIdx.x; j < nu; j += blockDim.x) xs[j] = x[u0 + j];
  __syncthreads();
  const int pairs = rows / 2;
  double2 acc[P];
#pragma unroll
  for (int k = 0; k < P; ++k) acc[k] = make_double2(0.0, 0.0);
  const double2 *col = reinterpret_cast<const double2 *>(M + size_t(u0) * rows);
  const size_t ld2 = size_t(pairs);
  int j = 0;
  for (; j + U - 1 < nu; j += U) {
    double2 v[U][P];
#pragma unroll
    for (int q = 0; q < U; ++q)
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int rp = threadIdx.x + k * kColsThreads;
        v[q][k] = rp < pairs ? __ldg(col + size_t(j + q) * ld2 + rp) : make_double2(0.0, 0.0);
      }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const double xq = xs[j + q];
#pragma unroll
      for (int k = 0; k < P; ++k) {
        acc[k].x = fma(v[q][k].x, xq, acc[k].x);
        acc[k].y = fma(v[q][k].y, xq, acc[k].y);
      }
    }
  }
  for (; j < nu; ++j) {
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int rp = threadIdx.x + k * kColsThreads;
      if (rp < pairs) {
        const double2 v = __ldg(col + size_t(j) * ld2 + rp);
        acc[k].x = fma(v.x, xs[j], acc[k].x);
        acc[k].y = fma(v.y, xs[j], acc[k].y);
      }
    }
  }
  double *pr = partial + size_t(blockIdx.x) * rows;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int rp = threadIdx.x + k * kColsThreads;
    if (rp < pairs) {
      pr[2 * rp] = acc[k].x;
      pr[2 * rp + 1] = acc[k].y;
    }
  }
}

// The same partial products with every CTA's run of whole columns streamed into shared
// memory by 1-D bulk async copies (cp.async.bulk, completion on an mbarrier) through a ring of
// kBulkStages stages of `cpt` columns each, instead of per-thread global loads: the copy engine
// keeps the HBM stream going without the L1 request throttling the load-based kernels hit.
// A thread owns the row pairs t, t + kColsThreads, ... (P of them) and reads them from the
// staged columns as 16-byte shared loads.  Needs an even leading dimension (16-byte aligned
// column starts and copy sizes).  Dynamic shared memory: kBulkStages stages of cpt x rows
// doubles, the chunk of x, then the barriers.  A stage wait that runs out (~0.5 s) makes the
// CTA wait for its copies still in flight and write NaN partials, so the solve fails loudly.
constexpr int kBulkStages = 3;
constexpr int kBulkStageBytes = 32768;  // at most, per stage
template <int P>
__global__ void __launch_bounds__(kColsThreads)
    gemv_bulk_partial_kernel(int rows, int cols, int chunk, int cpt, const double *__restrict__ M,
                             const double *__restrict__ x, double *__restrict__ partial) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const size_t stage_elems = size_t(cpt) * rows;
  double *stage0 = reinterpret_cast<double *>(smem_raw);
  double *xs = stage0 + kBulkStages * stage_elems;
  uint64_t *bar = reinterpret_cast<uint64_t *>(xs + ((chunk + 1) & ~1));
  const int u0 = blockIdx.x * chunk;
  const int nu = min(chunk, cols - u0);
  const int ntile = (nu + cpt - 1) / cpt;
  const int pairs = rows / 2;
  if (threadIdx.x == 0) {
    for (int q = 0; q < kBulkStages; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  for (int j = threadIdx.x; j < nu; j += blockDim.x) xs[j] = x[u0 + j];
  __syncthreads();
  auto issue = [&](int t) {  // thread 0: columns [t cpt, ...) of the chunk into stage t mod S
    const int st = t % kBulkStages;
    const int nc = min(cpt, nu - t * cpt);
    const uint32_t bytes = uint32_t(nc) * uint32_t(rows) * 8u;
    mbar_arrive_expect_tx(&bar[st], bytes);
    bulk_g2s(stage0 + st * stage_elems, M + (size_t(u0) + size_t(t) * cpt) * rows, bytes, &bar[st]);
  };
  if (threadIdx.x == 0)
    for (int t = 0; t < kBulkStages && t < ntile; ++t) issue(t);
  double2 acc[P];
#pragma unroll
  for (int k = 0; k < P; ++k) acc[k] = make_double2(0.0, 0.0);
  bool failed = false;
  for (int t = 0; t < ntile; ++t) {
    const int st = t % kBulkStages;
    const bool ok = mbar_wait_bounded(&bar[st], (t / kBulkStages) & 1u);
    if (__syncthreads_or(!ok)) {  // uniform: record, drain the copies in flight, leave
      if (threadIdx.x == 0)
        for (int q = t; q < ntile && q < t + kBulkStages; ++q)
          mbar_wait_bounded(&bar[q % kBulkStages], (q / kBulkStages) & 1u);
      failed = true;
      break;
    }
    const double2 *S = reinterpret_cast<const double2 *>(stage0 + st * stage_elems);
    const int nc = min(cpt, nu - t * cpt);
    for (int q = 0; q < nc; ++q) {
      const double xq = xs[t * cpt + q];
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int rp = threadIdx.x + k * kColsThreads;
        if (rp < pairs) {
          const double2 v = S[size_t(q) * pairs + rp];
          acc[k].x = fma(v.x, xq, acc[k].x);
          acc[k].y = fma(v.y, xq, acc[k].y);
        }
      }
    }
    __syncthreads();  // stage st is consumed
    if (threadIdx.x == 0 && t + kBulkStages < ntile) issue(t + kBulkStages);
  }
  double *pr = partial + size_t(blockIdx.x) * rows;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int rp = threadIdx.x + k * kColsThreads;
    if (rp < pairs) {
      pr[2 * rp] = failed ? nan : acc[k].x;
      pr[2 * rp + 1] = failed ? nan : acc[k].y;
    }
  }
}

// Columns per stage of the bulk-copy product (stages of at most kBulkStageBytes) and its
// dynamic shared memory for a chunk of `chunk` columns.
int bulk_cols_per_stage(int rows) { return std::max(1, kBulkStageBytes / (rows * 8)); }
size_t bulk_smem_bytes(int rows, int chunk) {
  return sizeof(double) * (size_t(kBulkStages) * bulk_cols_per_stage(rows) * rows + ((chunk + 1) & ~1)) +
         sizeof(uint64_t) * kBulkStages;
}

// y[r] = alpha sum_ch partial[ch][r] (+ y[r]): a CTA per 32 rows, lane g of 8 summing the
// chunks g, g + 8, ..., then the 8 lane sums added in lane order (fixed order throughout).
constexpr int kRedRows = 32, kRedLanes = 8;
__global__ void __launch_bounds__(kRedRows * kRedLanes)
    gemv_reduce_kernel(int rows, int chunks, const double *partial, double alpha, int accumulate,
                       double *y) {
  __shared__ double part[kRedLanes][kRedRows];
  const int rl = threadIdx.x % kRedRows, g = threadIdx.x / kRedRows;
  const int r = blockIdx.x * kRedRows + rl;
  double acc = 0.0;
  if (r < rows)
    for (int ch = g; ch < chunks; ch += kRedLanes) acc += partial[size_t(ch) * rows + r];
  part[g][rl] = acc;
  __syncthreads();
  if (g == 0 && r < rows) {
    double t = part[0][rl];
    for (int q = 1; q < kRedLanes; ++q) t += part[q][rl];
    y[r] = accumulate ? fma(alpha, t, y[r]) : alpha * t;
  }
}

// X[:, c] -= L S[:, c] for the nc columns of X (nA x nc, ld nA) and S (l x nc, ld l) over the
// given section blocks (rows x cols at (row0, col0), values column-major); the blocks of one
// launch must cover disjoint rows.  CTA (section blockIdx.x, rows [blockIdx.y kSubRows, ...)):
// a thread per row, the section's coefficients s staged in shared memory; a warp reads 32
// consecutive rows of one column.
constexpr int kSubRows = 256;
constexpr int kSubMaxCols = 2048;
__global__ void __launch_bounds__(kSubRows)
    sub_blocks_kernel(const SecBlock *sec, const double *vals, int nA, int l, int nc,
                      const double *S, double *X) {
  __shared__ double ss[kSubMaxCols];
  const SecBlock b = sec[blockIdx.x];
  const int r0 = blockIdx.y * kSubRows;
  if (r0 >= b.rows) return;  // uniform over the CTA
  const int i = r0 + threadIdx.x;
  for (int c = 0; c < nc; ++c) {
    __syncthreads();
    for (int q = threadIdx.x; q < b.cols; q += blockDim.x) ss[q] = S[size_t(c) * l + b.col0 + q];
    __syncthreads();
    if (i < b.rows) {
      const double *v = vals + b.off + i;
      double a0 = 0.0, a1 = 0.0;
      int q = 0;
      for (; q + 1 < b.cols; q += 2) {
        a0 = fma(v[size_t(q) * b.rows], ss[q], a0);
        a1 = fma(v[size_t(q + 1) * b.rows], ss[q + 1], a1);
      }
      if (q < b.cols) a0 = fma(v[size_t(q) * b.rows], ss[q], a0);
      X[size_t(c) * nA + b.row0 + i] -= a0 + a1;
    }
  }
}

// c = C y, one right-hand side, for the column sections' blocks (rows x cols, column-major,
// block b covering c[col0, col0 + cols) and y[row0, row0 + rows)): c[r] = sum_q
// P_b[q, r - col0] y[row0 + q], with cmap[r] = b.  A CTA per output; column r - col0 of P_b
// is contiguous and read as 16-byte pairs (rows, row0 and every block offset are even), two
// accumulators a thread, then a fixed-order reduction (shuffles, then the warps in order).
constexpr int kDotThreads = 256;
__global__ void __launch_bounds__(kDotThreads)
    sec_dot_kernel(const SecBlock *sec, const int *cmap, const double *vals, const double *y,
                   double *c) {
  __shared__ double red[kDotThreads / 32];
  const int r = blockIdx.x;
  const SecBlock b = sec[cmap[r]];
  const double2 *pv = reinterpret_cast<const double2 *>(vals + b.off + size_t(r - b.col0) * b.rows);
  const double2 *yv = reinterpret_cast<const double2 *>(y + b.row0);
  double a0 = 0.0, a1 = 0.0;
  for (int q = threadIdx.x; q < b.rows / 2; q += kDotThreads) {
    const double2 p2 = pv[q], y2 = yv[q];
    a0 = fma(p2.x, y2.x, a0);
    a1 = fma(p2.y, y2.y, a1);
  }
  double a = a0 + a1;
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kDotThreads / 32; ++q) t += red[q];
    c[r] = t;
  }
}

// Blocks of a 256-thread grid-stride launch over n elements: one per 256 elements, at most
// 32 per SM of the current device.
int grid_for(size_t n) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 1;
  return int(std::max<size_t>(1, std::min<size_t>((n + 255) / 256, size_t(sms) * 32)));
}

}  // namespace

struct fds_solver {
  int nA = 0, L = 0, l = 0;
  // HBS: per level 1..L the box table and offsets, level vector lengths N[0..L]
  std::vector<int> nboxes;             // [L + 1], nboxes[0] = 1 (root)
  std::vector<HbsBox *> d_boxes;       // [L + 1]
  std::vector<long long> N;            // [L + 1]
  double *d_mats = nullptr;
  // neighbour factors: R = A_m(J, :) (l x nA), K^-1 = (I + R A_0^-1 L)^-1, L's section blocks;
  // recompressed: M = K^-1 S (l x lc) and C's blocks (host copy of their table for the
  // several-right-hand-side products) in place of R and K^-1
  double *d_R = nullptr, *d_Kinv = nullptr, *d_M = nullptr;
  SecBlock *d_sec = nullptr;
  double *d_svals = nullptr;
  int lc = 0;                          // rows of C (0: not recompressed)
  SecBlock *d_csec = nullptr;
  int *d_cmap = nullptr;               // [lc] block of every row of C
  double *d_cvals = nullptr;
  std::vector<SecBlock> h_csec;
  int n_sec = 0;
  int n_sec_left = 0;                  // sections of the m = -1 neighbour (they come first);
                                       //   each neighbour's sections partition both walls
  int sub_row_chunks = 1;              // row chunks of the largest section (grid.y)
  int sms = 1;                         // SMs of the device the solver was built on
  double *d_gpart = nullptr;           // partial sums of the one-right-hand-side products
  int gemv_chunks_R = 1, gemv_chunks_K = 1;
  int chunk_R = 1, chunk_K = 1;
  // workspace of one pass (kChunk right-hand sides)
  double *d_up = nullptr, *d_down = nullptr, *d_out = nullptr, *d_t = nullptr, *d_s = nullptr;
  size_t up_len = 0;                   // sum of N[0..L-1]
  int max_cols = 0;                    // widest level product (k + n, or n at the root)
  std::vector<int> max_k, max_n;       // [L + 1] largest skeleton / active set per level
  fds_info info;
};

namespace {

int cuda_fail(std::string &err, cudaError_t e, const char *what) {
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA;
}

#define FK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(err, e_, #call); \
  } while (0)
#define FB(call)                                                                 \
  do {                                                                           \
    cublasStatus_t e_ = (call);                                                  \
    if (e_ != CUBLAS_STATUS_SUCCESS) {                                           \
      err = std::string(#call) + ": cublas " + std::to_string(int(e_));          \
      return STOKES_ERR_CUDA;                                                    \
    }                                                                            \
  } while (0)
#define FQ(call)                                                                 \
  do {                                                                           \
    cusolverStatus_t e_ = (call);                                                \
    if (e_ != CUSOLVER_STATUS_SUCCESS) {                                         \
      err = std::string(#call) + ": cusolver " + std::to_string(int(e_));        \
      return STOKES_ERR_CUDA;                                                    \
    }                                                                            \
  } while (0)

template <class T>
cudaError_t dalloc(T *&p, size_t n, size_t &bytes) {
  bytes += sizeof(T) * n;
  return cudaMalloc(reinterpret_cast<void **>(&p), sizeof(T) * std::max<size_t>(n, 1));
}

void bounds(const WallGeom &g, Box &bx) {
  bx.x0 = bx.y0 = 1e300;
  bx.x1 = bx.y1 = -1e300;
  for (int i = bx.a; i < bx.b; ++i) {
    bx.x0 = std::min(bx.x0, g.x[i]);
    bx.x1 = std::max(bx.x1, g.x[i]);
    bx.y0 = std::min(bx.y0, g.y[i]);
    bx.y1 = std::max(bx.y1, g.y[i]);
  }
}

// One level pass: NC = 1 for a single right-hand side, else kHbsCols per CTA.
void level(const fds_solver *f, int lev, int mode, int nc, const double *x1, long long ld1,
           const double *x2, long long ld2, double *y, long long ldy, cudaStream_t s) {
  const int nb = f->nboxes[lev];
  const int rows = mode == 0 ? f->max_k[lev] : f->max_n[lev];
  const int tiles = (rows + kRowTile - 1) / kRowTile;
  if (nc == 1) {
    const size_t sm = sizeof(double) * (size_t(f->max_cols) + kHbsThreads);
    if (nb * tiles < f->sms) {  // a top level: small row tiles
      const int st = (rows + kRowTileSmall - 1) / kRowTileSmall;
      hbs_level_kernel<1, kRowTileSmall><<<dim3(nb, st, 1), kHbsThreads, sm, s>>>(
          f->d_boxes[lev], f->d_mats, mode, nc, x1, ld1, x2, ld2, y, ldy);
    } else {
      hbs_level_kernel<1><<<dim3(nb, tiles, 1), kHbsThreads, sm, s>>>(
          f->d_boxes[lev], f->d_mats, mode, nc, x1, ld1, x2, ld2, y, ldy);
    }
  } else {
    const size_t sm = sizeof(double) * kHbsCols * (size_t(f->max_cols) + kHbsThreads);
    hbs_level_kernel<kHbsCols><<<dim3(nb, tiles, (nc + kHbsCols - 1) / kHbsCols), kHbsThreads, sm,
                                 s>>>(f->d_boxes[lev], f->d_mats, mode, nc, x1, ld1, x2, ld2, y,
                                      ldy);
  }
}

// A_0^-1 X for up to kChunk columns (X column-major with leading dimension nA).
int hbs_pass(fds_solver *f, const double *X, double *out, int nc, cudaStream_t s,
             std::string &err) {
  const int L = f->L;
  std::vector<double *> up(L + 1), down(L + 1);
  {
    size_t o = 0;
    for (int lev = 0; lev < L; ++lev) {
      up[lev] = f->d_up + o * kChunk;
      down[lev] = f->d_down + o * kChunk;
      o += size_t(f->N[lev]);
    }
  }
  // upward: level L reads X, level l writes the level-(l-1) vector
  for (int lev = L; lev >= 1; --lev)
    level(f, lev, 0, nc, lev == L ? X : up[lev], f->N[lev], nullptr, 0, up[lev - 1], f->N[lev - 1], s);
  // root: u^ = G_root v^
  level(f, 0, 0, nc, up[0], f->N[0], nullptr, 0, down[0], f->N[0], s);
  // downward: u = E u^ + G v
  for (int lev = 1; lev <= L; ++lev)
    level(f, lev, 1, nc, down[lev - 1], f->N[lev - 1], lev == L ? X : up[lev], f->N[lev],
          lev == L ? out : down[lev], f->N[lev], s);
  FK(cudaGetLastError());
  return STOKES_OK;
}

// X <- A_0^-1 X, in passes of kChunk columns.
int hbs_apply(fds_solver *f, double *X, int nrhs, cudaStream_t s, std::string &err) {
  for (int c0 = 0; c0 < nrhs; c0 += kChunk) {
    const int nc = std::min(kChunk, nrhs - c0);
    double *Xc = X + size_t(c0) * f->nA;
    int st = hbs_pass(f, Xc, f->d_out, nc, s, err);
    if (st) return st;
    FK(cudaMemcpyAsync(Xc, f->d_out, sizeof(double) * f->nA * nc, cudaMemcpyDeviceToDevice, s));
  }
  return STOKES_OK;
}

struct HostFactors {
  int nA = 0, L = 0;
  std::vector<int> nboxes;
  std::vector<long long> N;
  std::vector<double> mats;               // F^*, E, G per box, then G_root
  std::vector<std::vector<HbsBox>> tabs;  // [L + 1], tabs[0] = the root
  std::vector<int> Jall, mall;            // neighbour skeleton unknowns and their image m
  std::vector<int> sec_m;                 // image m of every section block
  std::vector<SecBlock> sb;               // L's blocks
  std::vector<double> svals;
  std::vector<int> Jc, mc;                // column skeleton unknowns and their image m
  std::vector<SecBlock> csb;              // C's blocks (each stored transposed: rows x cols)
  std::vector<double> cvals;
  int max_cols = 0;                       // widest level product
  std::vector<int> max_k, max_n;          // [L + 1] per level
  fds_info info;
  WallGeom g;
};

// Host part of the build: the HBS tables and the neighbour sections, packed for the device.
int host_factor(int n_w, const double *nodes, const double *weights, const double *normals,
                const double *curvature, double period, const fds_params &p, HostFactors &hf,
                std::string &err) {
  if (n_w < 4 || !(period > 0.0) || p.leaf < 2 || p.n_proxy < 8 || p.n_proxy_nb < 8 ||
      p.sec_max < 2 || !(p.tol > 0.0)) {
    err = "fds: bad arguments";
    return STOKES_ERR_ARG;
  }
  const auto t0 = std::chrono::steady_clock::now();
  WallGeom g;
  g.nw = n_w;
  g.Nt = 2 * n_w;
  g.d = period;
  const int Nt = g.Nt, nA = 2 * Nt;
  g.x.resize(Nt);
  g.y.resize(Nt);
  g.nx.resize(Nt);
  g.ny.resize(Nt);
  g.w.assign(weights, weights + Nt);
  g.kap.assign(curvature, curvature + Nt);
  for (int i = 0; i < Nt; ++i) {
    g.x[i] = nodes[2 * i];
    g.y[i] = nodes[2 * i + 1];
    g.nx[i] = normals[2 * i];
    g.ny[i] = normals[2 * i + 1];
  }
  hf.nA = nA;
  // ---- HBS tree: level 0 the root, level 1 the walls, then halves ----
  std::vector<std::vector<Box>> lv(2);
  lv[0].resize(1);
  lv[0][0].a = 0;
  lv[0][0].b = Nt;
  lv[1].resize(2);
  lv[1][0].a = 0;
  lv[1][0].b = n_w;
  lv[1][1].a = n_w;
  lv[1][1].b = Nt;
  while (lv.back()[0].b - lv.back()[0].a > p.leaf) {
    std::vector<Box> nx;
    for (const Box &bx : lv.back()) {
      const int h = (bx.a + bx.b) / 2;
      Box c0, c1;
      c0.a = bx.a;
      c0.b = h;
      c1.a = h;
      c1.b = bx.b;
      nx.push_back(c0);
      nx.push_back(c1);
    }
    lv.push_back(nx);
  }
  const int L = int(lv.size()) - 1;
  hf.L = L;
  for (auto &level : lv)
    for (Box &bx : level) bounds(g, bx);
  for (Box &bx : lv[L]) {
    bx.act.resize(2 * (bx.b - bx.a));
    std::iota(bx.act.begin(), bx.act.end(), 2 * bx.a);
  }
  std::atomic<int> failed(0);
  for (int lev = L; lev >= 1; --lev) {
    std::vector<Box> &B = lv[lev];
    if (lev < L)
      for (int i = 0; i < int(B.size()); ++i) {
        const Box &c0 = lv[lev + 1][2 * i], &c1 = lv[lev + 1][2 * i + 1];
        B[i].act = c0.skel;
        B[i].act.insert(B[i].act.end(), c1.skel.begin(), c1.skel.end());
      }
    parallel_for(int(B.size()), [&](int i) {
      Box &bx = B[i];
      const double cx = 0.5 * (bx.x0 + bx.x1), cy = 0.5 * (bx.y0 + bx.y1);
      const double rad = 1.5 * 0.5 * hypot(bx.x1 - bx.x0, bx.y1 - bx.y0);
      std::vector<int> near;
      for (int j = 0; j < int(B.size()); ++j) {
        if (j == i) continue;
        const Box &o = B[j];
        const double dx = std::max({o.x0 - cx, 0.0, cx - o.x1});
        const double dy = std::max({o.y0 - cy, 0.0, cy - o.y1});
        if (dx * dx + dy * dy >= rad * rad) continue;
        for (int u : o.act) {
          const double ex = g.x[u >> 1] - cx, ey = g.y[u >> 1] - cy;
          if (ex * ex + ey * ey < rad * rad) near.push_back(u);
        }
      }
      HMat Z = probe_matrix(g, bx.act, near, 0, true, cx, cy, rad, p.n_proxy, true);
      std::vector<int> J;
      HMat X;
      column_id(Z, p.tol, J, X);
      bx.skel.resize(J.size());
      for (size_t c = 0; c < J.size(); ++c) bx.skel[c] = bx.act[J[c]];
      const int n = int(bx.act.size()), k = int(J.size());
      HMat D(n, n);
      if (lev == L) {
        for (int jj = 0; jj < n; ++jj)
          for (int ii = 0; ii < n; ++ii) D(ii, jj) = a_host(g, bx.act[ii], bx.act[jj], 0);
      } else {
        const Box &c0 = lv[lev + 1][2 * i], &c1 = lv[lev + 1][2 * i + 1];
        const int ka = int(c0.skel.size());
        for (int jj = 0; jj < n; ++jj)
          for (int ii = 0; ii < n; ++ii) {
            const bool ia = ii < ka, ja = jj < ka;
            if (ia && ja)
              D(ii, jj) = c0.Dh(ii, jj);
            else if (!ia && !ja)
              D(ii, jj) = c1.Dh(ii - ka, jj - ka);
            else
              D(ii, jj) = a_host(g, bx.act[ii], bx.act[jj], 0);
          }
      }
      if (!invert(D)) {
        failed = 1;
        return;
      }
      const HMat DiP = mul_nt(D, X);   // D^-1 P      (n x k)
      const HMat PtDi = mul(X, D);     // P^T D^-1    (k x n)
      HMat Dh = mul_nt(PtDi, X);       // P^T D^-1 P  (k x k)
      if (!invert(Dh)) {
        failed = 1;
        return;
      }
      bx.E = mul(DiP, Dh);
      bx.Ft = mul(Dh, PtDi);
      HMat EP = mul(bx.E, PtDi);
      for (size_t q = 0; q < D.a.size(); ++q) D.a[q] -= EP.a[q];
      bx.G = std::move(D);
      bx.Dh = std::move(Dh);
      (void)k;
    });
    if (failed) {
      err = "fds: singular diagonal block in the HBS factorization";
      return STOKES_ERR_CUDA;
    }
    // children's D^ are no longer needed
    if (lev < L)
      for (Box &c : lv[lev + 1]) c.Dh = HMat();
  }
  // root: [D^_a, A_0(J_a, J_b); A_0(J_b, J_a), D^_b]^-1
  HMat Groot;
  {
    const Box &c0 = lv[1][0], &c1 = lv[1][1];
    std::vector<int> act = c0.skel;
    act.insert(act.end(), c1.skel.begin(), c1.skel.end());
    const int n = int(act.size()), ka = int(c0.skel.size());
    Groot = HMat(n, n);
    for (int jj = 0; jj < n; ++jj)
      for (int ii = 0; ii < n; ++ii) {
        const bool ia = ii < ka, ja = jj < ka;
        Groot(ii, jj) = (ia && ja)     ? c0.Dh(ii, jj)
                        : (!ia && !ja) ? c1.Dh(ii - ka, jj - ka)
                                       : a_host(g, act[ii], act[jj], 0);
      }
    if (!invert(Groot)) {
      err = "fds: singular root block";
      return STOKES_ERR_CUDA;
    }
    lv[0][0].act = act;
  }
  // ---- neighbour sections (Sec. 4.2) ----
  struct Section {
    int a, b, m;
    std::vector<int> skel;
    HMat P;  // rows x k (interpolation matrix)
  };
  // Each wall of each neighbour m, cut dyadically toward the end that meets the shared cell
  // boundary: for A_m's rows the targets next to the neighbour (the right end for m = +1),
  // for its columns the sources that the shift m d carries next to the cell (the left end).
  auto cut = [&](bool cols) {
    std::vector<Section> out;
    for (int m : {-1, 1})
      for (int w0 : {0, n_w}) {
        const bool to_right = (m > 0) != cols;
        int a = 0, b = n_w;
        while (b - a > p.sec_max) {
          const int h = (a + b) / 2;
          if (to_right) {
            out.push_back({w0 + a, w0 + h, m, {}, HMat()});
            a = h;
          } else {
            out.push_back({w0 + h, w0 + b, m, {}, HMat()});
            b = h;
          }
        }
        out.push_back({w0 + a, w0 + b, m, {}, HMat()});
      }
    return out;
  };
  // The skeleton of a section: against a proxy circle 0.9 x its centre's distance to that
  // boundary or, for the touching section, 1.75 x its radius together with the nodes on the
  // other side within that circle (the neighbour's sources for rows, the cell's targets for
  // columns).
  auto skeletonise = [&](std::vector<Section> &secs, bool cols) {
    parallel_for(int(secs.size()), [&](int si) {
      Section &sc = secs[si];
      Box bx;
      bx.a = sc.a;
      bx.b = sc.b;
      bounds(g, bx);
      const double cx = 0.5 * (bx.x0 + bx.x1), cy = 0.5 * (bx.y0 + bx.y1);
      const int la = sc.a % n_w, lb = sc.b - (sc.a - la);
      const bool to_right = (sc.m > 0) != cols;
      const bool touch = to_right ? lb == n_w : la == 0;
      const double shift = (cols ? -sc.m : sc.m) * g.d;
      double rad;
      std::vector<int> near;
      if (!touch) {
        rad = 0.9 * fabs((to_right ? g.d : 0.0) - cx);
      } else {
        rad = 1.75 * 0.5 * hypot(bx.x1 - bx.x0, bx.y1 - bx.y0);
        for (int j = 0; j < Nt; ++j) {
          const double ex = g.x[j] + shift - cx, ey = g.y[j] - cy;
          if (ex * ex + ey * ey < rad * rad) {
            near.push_back(2 * j);
            near.push_back(2 * j + 1);
          }
        }
      }
      std::vector<int> It(2 * (sc.b - sc.a));
      std::iota(It.begin(), It.end(), 2 * sc.a);
      HMat Z = cols ? probe_cols(g, It, near, sc.m, cx, cy, rad, p.n_proxy_nb)
                    : probe_matrix(g, It, near, sc.m, false, cx, cy, rad, p.n_proxy_nb, false);
      std::vector<int> J;
      HMat X;
      column_id(Z, p.tol, J, X);
      sc.skel.resize(J.size());
      for (size_t c = 0; c < J.size(); ++c) sc.skel[c] = It[J[c]];
      // P = X^T
      sc.P = HMat(X.c, X.r);
      for (int c = 0; c < X.r; ++c)
        for (int r = 0; r < X.c; ++r) sc.P(r, c) = X(c, r);
    });
  };
  std::vector<Section> secs = cut(false), csecs;
  skeletonise(secs, false);
  if (p.recompress) {
    csecs = cut(true);
    skeletonise(csecs, true);
  }
  const auto t1 = std::chrono::steady_clock::now();
  hf.info.host_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  // ---- pack the HBS tables for the device ----
  hf.nboxes.assign(L + 1, 0);
  hf.N.assign(L + 1, 0);
  hf.N[L] = nA;
  
  hf.tabs.assign(L + 1, {});
  hf.max_k.assign(L + 1, 0);
  hf.max_n.assign(L + 1, 0);
  int max_rank = 0;
  for (int lev = L; lev >= 1; --lev) {
    int in_off = 0, out_off = 0;
    for (const Box &bx : lv[lev]) {
      HbsBox hb;
      hb.n = int(bx.act.size());
      hb.k = int(bx.skel.size());
      hb.in_off = in_off;
      hb.out_off = out_off;
      hb.ft = (long long)hf.mats.size();
      hf.mats.insert(hf.mats.end(), bx.Ft.a.begin(), bx.Ft.a.end());
      hb.e = (long long)hf.mats.size();
      hf.mats.insert(hf.mats.end(), bx.E.a.begin(), bx.E.a.end());
      hb.g = (long long)hf.mats.size();
      hf.mats.insert(hf.mats.end(), bx.G.a.begin(), bx.G.a.end());
      hf.tabs[lev].push_back(hb);
      in_off += hb.n;
      out_off += hb.k;
      max_rank = std::max(max_rank, hb.k);
      hf.max_k[lev] = std::max(hf.max_k[lev], hb.k);
      hf.max_n[lev] = std::max(hf.max_n[lev], hb.n);
      hf.max_cols = std::max(hf.max_cols, hb.k + hb.n);  // [E | G] is n x (k + n)
    }
    hf.nboxes[lev] = int(lv[lev].size());
    hf.N[lev - 1] = out_off;
  }
  {
    HbsBox hb;
    hb.n = hb.k = Groot.r;
    hb.in_off = hb.out_off = 0;
    hb.ft = (long long)hf.mats.size();
    hb.e = hb.g = 0;
    hf.max_cols = std::max(hf.max_cols, hb.n);
    hf.max_k[0] = hf.max_n[0] = hb.n;
    hf.mats.insert(hf.mats.end(), Groot.a.begin(), Groot.a.end());
    hf.tabs[0].push_back(hb);
    hf.nboxes[0] = 1;
  }
  hf.info.levels = L;
  hf.info.max_rank = max_rank;
  hf.info.root_size = Groot.r;
  // neighbour factor layout
  for (const Section &sc : secs) {
    SecBlock b;
    b.row0 = 2 * sc.a;
    b.rows = 2 * (sc.b - sc.a);
    b.col0 = int(hf.Jall.size());
    b.cols = int(sc.skel.size());
    b.off = (long long)hf.svals.size();
    hf.svals.insert(hf.svals.end(), sc.P.a.begin(), sc.P.a.end());
    hf.sb.push_back(b);
    hf.sec_m.push_back(sc.m);
    for (int u : sc.skel) {
      hf.Jall.push_back(u);
      hf.mall.push_back(sc.m);
    }
  }
  hf.info.neighbour_rank = int(hf.Jall.size());
  hf.info.sections = int(secs.size());
  for (const Section &sc : csecs) {
    SecBlock b;
    b.row0 = 2 * sc.a;
    b.rows = 2 * (sc.b - sc.a);
    b.col0 = int(hf.Jc.size());
    b.cols = int(sc.skel.size());
    b.off = (long long)hf.cvals.size();
    hf.cvals.insert(hf.cvals.end(), sc.P.a.begin(), sc.P.a.end());
    hf.csb.push_back(b);
    for (int u : sc.skel) {
      hf.Jc.push_back(u);
      hf.mc.push_back(sc.m);
    }
  }
  hf.info.neighbour_col_rank = int(hf.Jc.size());
  hf.g = std::move(g);
  return STOKES_OK;
}

}  // namespace

int fds_build(fds_solver **out, int n_w, const double *nodes, const double *weights,
              const double *normals, const double *curvature, double period, const fds_params &p,
              cudaStream_t s, cublasHandle_t blas, cusolverDnHandle_t sol, std::string &err) {
  *out = nullptr;
  HostFactors hf;
  {
    const int st = host_factor(n_w, nodes, weights, normals, curvature, period, p, hf, err);
    if (st) return st;
  }
  const WallGeom &g = hf.g;
  const int L = hf.L, nA = hf.nA, Nt = g.Nt, l = int(hf.Jall.size());
  fds_solver *f = new fds_solver();
  f->nA = nA;
  f->L = L;
  f->l = l;
  f->info = hf.info;
  f->nboxes = hf.nboxes;
  f->N = hf.N;
  f->max_cols = hf.max_cols;
  f->max_k = hf.max_k;
  f->max_n = hf.max_n;
  // ---- device side ----
  size_t &bytes = f->info.device_bytes;
  std::vector<void *> tmp;  // set-up scratch, freed on every exit
  auto bail = [&](int st) {
    for (void *q : tmp) cudaFree(q);
    fds_destroy(f);
    return st;
  };
#define FD(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return bail(cuda_fail(err, e_, #call)); \
  } while (0)
#define FDB(call)                                                      \
  do {                                                                 \
    cublasStatus_t e_ = (call);                                        \
    if (e_ != CUBLAS_STATUS_SUCCESS) {                                 \
      err = std::string(#call) + ": cublas " + std::to_string(int(e_)); \
      return bail(STOKES_ERR_CUDA);                                    \
    }                                                                  \
  } while (0)
#define FDQ(call)                                                        \
  do {                                                                   \
    cusolverStatus_t e_ = (call);                                        \
    if (e_ != CUSOLVER_STATUS_SUCCESS) {                                 \
      err = std::string(#call) + ": cusolver " + std::to_string(int(e_)); \
      return bail(STOKES_ERR_CUDA);                                      \
    }                                                                    \
  } while (0)
  const auto t2 = std::chrono::steady_clock::now();
  {
    const int sm1 = int(sizeof(double) * (size_t(f->max_cols) + kHbsThreads));
    const int sm8 = int(sizeof(double) * kHbsCols * (size_t(f->max_cols) + kHbsThreads));
    if (sm8 > 227 * 1024) {
      err = "fds: a level product is too wide for shared memory (lower leaf_nodes)";
      return bail(STOKES_ERR_ARG);
    }
    FD(cudaFuncSetAttribute(hbs_level_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm1));
    FD(cudaFuncSetAttribute(hbs_level_kernel<1, kRowTileSmall>,
                            cudaFuncAttributeMaxDynamicSharedMemorySize, sm1));
    int dev = 0;
    FD(cudaGetDevice(&dev));
    FD(cudaDeviceGetAttribute(&f->sms, cudaDevAttrMultiProcessorCount, dev));
    FD(cudaFuncSetAttribute(hbs_level_kernel<kHbsCols>,
                            cudaFuncAttributeMaxDynamicSharedMemorySize, sm8));
  }
  FD(dalloc(f->d_mats, hf.mats.size(), bytes));
  FD(cudaMemcpyAsync(f->d_mats, hf.mats.data(), sizeof(double) * hf.mats.size(), cudaMemcpyHostToDevice, s));
  f->d_boxes.assign(L + 1, nullptr);
  for (int lev = 0; lev <= L; ++lev) {
    FD(dalloc(f->d_boxes[lev], hf.tabs[lev].size(), bytes));
    FD(cudaMemcpyAsync(f->d_boxes[lev], hf.tabs[lev].data(), sizeof(HbsBox) * hf.tabs[lev].size(),
                       cudaMemcpyHostToDevice, s));
  }
  f->up_len = 0;
  for (int lev = 0; lev < L; ++lev) f->up_len += size_t(f->N[lev]);
  FD(dalloc(f->d_up, f->up_len * kChunk, bytes));
  FD(dalloc(f->d_down, f->up_len * kChunk, bytes));
  FD(dalloc(f->d_out, size_t(nA) * kChunk, bytes));
  const int lc = int(hf.Jc.size());
  f->lc = lc;
  FD(dalloc(f->d_t, size_t(std::max(l, lc)) * kChunk, bytes));
  FD(dalloc(f->d_s, size_t(l) * kChunk, bytes));
  // geometry and skeleton lists
  double *dg = nullptr;
  int *dJ = nullptr;
  size_t scratch = 0;
  FD(dalloc(dg, size_t(6) * Nt, scratch));
  tmp.push_back(dg);
  FD(dalloc(dJ, size_t(2) * (l + lc), scratch));
  tmp.push_back(dJ);
  const double *hs[6] = {g.x.data(), g.y.data(), g.nx.data(), g.ny.data(), g.w.data(), g.kap.data()};
  for (int q = 0; q < 6; ++q)
    FD(cudaMemcpyAsync(dg + size_t(q) * Nt, hs[q], sizeof(double) * Nt, cudaMemcpyHostToDevice, s));
  FD(cudaMemcpyAsync(dJ, hf.Jall.data(), sizeof(int) * l, cudaMemcpyHostToDevice, s));
  FD(cudaMemcpyAsync(dJ + l, hf.mall.data(), sizeof(int) * l, cudaMemcpyHostToDevice, s));
  if (lc > 0) {
    FD(cudaMemcpyAsync(dJ + 2 * l, hf.Jc.data(), sizeof(int) * lc, cudaMemcpyHostToDevice, s));
    FD(cudaMemcpyAsync(dJ + 2 * l + lc, hf.mc.data(), sizeof(int) * lc, cudaMemcpyHostToDevice, s));
  }
  // the row factor: R = A_m(J, :) (l x nA), or S = A_m(J, J_c) (l x lc) and C's blocks
  double *dRS = nullptr;  // R (kept) or S (set-up only)
  if (lc == 0) {
    FD(dalloc(f->d_R, size_t(l) * nA, bytes));
    dRS = f->d_R;
    fill_rows_kernel<<<grid_for(size_t(l) * nA), 256, 0, s>>>(
        l, nA, dJ, dJ + l, dg, dg + Nt, dg + 2 * Nt, dg + 3 * Nt, dg + 4 * Nt, dg + 5 * Nt, g.d, f->d_R);
  } else {
    FD(dalloc(dRS, size_t(l) * lc, scratch));
    tmp.push_back(dRS);
    fill_core_kernel<<<grid_for(size_t(l) * lc), 256, 0, s>>>(
        l, lc, dJ, dJ + l, dJ + 2 * l, dJ + 2 * l + lc, dg, dg + Nt, dg + 2 * Nt, dg + 3 * Nt,
        dg + 4 * Nt, dg + 5 * Nt, g.d, dRS);
    for (const SecBlock &b : hf.csb)
      if (b.rows % 2 || b.row0 % 2 || b.off % 2) {
        err = "fds: a column section is not made of whole nodes";
        return bail(STOKES_ERR_ARG);
      }
    std::vector<int> cmap(lc);
    for (int q = 0; q < int(hf.csb.size()); ++q)
      for (int c = 0; c < hf.csb[q].cols; ++c) cmap[hf.csb[q].col0 + c] = q;
    f->h_csec = hf.csb;
    FD(dalloc(f->d_csec, hf.csb.size(), bytes));
    FD(dalloc(f->d_cmap, size_t(lc), bytes));
    FD(dalloc(f->d_cvals, hf.cvals.size(), bytes));
    FD(cudaMemcpyAsync(f->d_csec, hf.csb.data(), sizeof(SecBlock) * hf.csb.size(), cudaMemcpyHostToDevice, s));
    FD(cudaMemcpyAsync(f->d_cmap, cmap.data(), sizeof(int) * lc, cudaMemcpyHostToDevice, s));
    FD(cudaMemcpyAsync(f->d_cvals, hf.cvals.data(), sizeof(double) * hf.cvals.size(), cudaMemcpyHostToDevice, s));
  }
  FD(cudaGetLastError());
  f->n_sec = int(hf.sb.size());
  f->n_sec_left = 0;
  while (f->n_sec_left < f->n_sec && hf.sec_m[f->n_sec_left] < 0) ++f->n_sec_left;
  for (const SecBlock &b : hf.sb) {
    f->sub_row_chunks = std::max(f->sub_row_chunks, (b.rows + kSubRows - 1) / kSubRows);
    if (b.cols > kSubMaxCols) {
      err = "fds: a neighbour section's rank exceeds the staging buffer";
      return bail(STOKES_ERR_ARG);
    }
  }
  for (int q = f->n_sec_left; q < f->n_sec; ++q)
    if (hf.sec_m[q] < 0) {
      err = "fds: neighbour sections are not grouped by image";
      return bail(STOKES_ERR_ARG);
    }
  FD(dalloc(f->d_sec, hf.sb.size(), bytes));
  FD(dalloc(f->d_svals, hf.svals.size(), bytes));
  FD(cudaMemcpyAsync(f->d_sec, hf.sb.data(), sizeof(SecBlock) * hf.sb.size(), cudaMemcpyHostToDevice, s));
  FD(cudaMemcpyAsync(f->d_svals, hf.svals.data(), sizeof(double) * hf.svals.size(), cudaMemcpyHostToDevice, s));
  // one-right-hand-side products: column chunks so that (row tiles x chunks) CTAs fill the
  // SMs about four times over, at most kGemvMaxChunk columns each
  {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the whole-column kernel runs one CTA per chunk, as many as are resident at once (one
    // wave); the tile kernel (odd or tall R) one per (row tile, chunk)
    const bool cols_kernel = l % 2 == 0 && l <= kColsMaxRows;
    int resident = 4;
    if (cols_kernel) {
      int nb = 0;
      const void *fn = l <= 2 * kColsThreads * 4
                           ? reinterpret_cast<const void *>(gemv_bulk_partial_kernel<4>)
                           : reinterpret_cast<const void *>(gemv_bulk_partial_kernel<8>);
      const size_t smem = bulk_smem_bytes(l, kGemvMaxChunk);
      FD(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kColsThreads, smem) == cudaSuccess && nb > 0)
        resident = nb;
    }
    const int row_tiles = cols_kernel ? 1 : std::max(1, (l + kGemvRows - 1) / kGemvRows);
    auto plan = [&](int cols, int &chunk, int &chunks) {
      const int want = std::max(1, resident * std::max(sms, 1) / row_tiles);
      chunk = std::min(kGemvMaxChunk, std::max(8, (cols + want - 1) / want));
      chunks = std::max(1, (cols + chunk - 1) / chunk);
    };
    plan(nA, f->chunk_R, f->gemv_chunks_R);
    plan(lc > 0 ? lc : l, f->chunk_K, f->gemv_chunks_K);
    FD(dalloc(f->d_gpart, size_t(std::max(1, l)) * std::max(f->gemv_chunks_R, f->gemv_chunks_K), bytes));
  }
  // Z = A_0^-1 L (set-up only: K = I + R Z)
  double *dZ = nullptr;
  FD(dalloc(dZ, size_t(nA) * l, scratch));
  tmp.push_back(dZ);
  FD(cudaMemsetAsync(dZ, 0, sizeof(double) * size_t(nA) * l, s));
  scatter_blocks_kernel<<<int(hf.sb.size()), 256, 0, s>>>(f->d_sec, f->d_svals, nA, dZ);
  FD(cudaGetLastError());
  {
    int st = hbs_apply(f, dZ, l, s, err);
    if (st) return bail(st);
  }
  // K = I + R Z (recompressed: R Z = S (C Z)), then K^-1 (or M = K^-1 S)
  double *dK = nullptr;
  FD(dalloc(dK, size_t(l) * l, scratch));
  tmp.push_back(dK);
  const double one = 1.0, zero = 0.0;
  cublasSetStream(blas, s);
  cusolverDnSetStream(sol, s);
  if (lc == 0) {
    FDB(cublasDgemm(blas, CUBLAS_OP_N, CUBLAS_OP_N, l, l, nA, &one, f->d_R, l, dZ, nA, &zero, dK, l));
  } else {
    double *dW = nullptr;  // C Z (lc x l)
    FD(dalloc(dW, size_t(lc) * l, scratch));
    tmp.push_back(dW);
    for (const SecBlock &b : hf.csb)
      FDB(cublasDgemm(blas, CUBLAS_OP_T, CUBLAS_OP_N, b.cols, l, b.rows, &one, f->d_cvals + b.off,
                      b.rows, dZ + b.row0, nA, &zero, dW + b.col0, lc));
    FDB(cublasDgemm(blas, CUBLAS_OP_N, CUBLAS_OP_N, l, l, lc, &one, dRS, l, dW, lc, &zero, dK, l));
  }
  add_identity_kernel<<<(l + 255) / 256, 256, 0, s>>>(l, dK);
  FD(cudaGetLastError());
  int lwork = 0;
  FDQ(cusolverDnDgetrf_bufferSize(sol, l, l, dK, l, &lwork));
  double *work = nullptr;
  int *piv = nullptr, *dinfo = nullptr;
  FD(dalloc(work, size_t(std::max(lwork, 1)), scratch));
  tmp.push_back(work);
  FD(dalloc(piv, size_t(l) + 1, scratch));
  tmp.push_back(piv);
  FD(dalloc(dinfo, 2, scratch));
  tmp.push_back(dinfo);
  FDQ(cusolverDnDgetrf(sol, l, l, dK, l, work, piv, dinfo));
  if (lc == 0) {
    FD(dalloc(f->d_Kinv, size_t(l) * l, bytes));
    set_identity_kernel<<<grid_for(size_t(l) * l), 256, 0, s>>>(l, f->d_Kinv);
    FDQ(cusolverDnDgetrs(sol, CUBLAS_OP_N, l, l, dK, l, piv, f->d_Kinv, l, dinfo + 1));
  } else {
    FD(dalloc(f->d_M, size_t(l) * lc, bytes));
    FD(cudaMemcpyAsync(f->d_M, dRS, sizeof(double) * size_t(l) * lc, cudaMemcpyDeviceToDevice, s));
    FDQ(cusolverDnDgetrs(sol, CUBLAS_OP_N, l, lc, dK, l, piv, f->d_M, l, dinfo + 1));
  }
  int hinfo[2] = {0, 0};
  FD(cudaMemcpyAsync(hinfo, dinfo, sizeof(hinfo), cudaMemcpyDeviceToHost, s));
  FD(cudaStreamSynchronize(s));
  if (hinfo[0] != 0 || hinfo[1] != 0) {
    err = "fds: I + R A_0^-1 L is singular";
    return bail(STOKES_ERR_CUDA);
  }
  for (void *q : tmp) cudaFree(q);
#undef FD
#undef FDB
#undef FDQ
  f->info.device_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t2).count();
  // a solve reads the HBS tables twice and L's blocks once, and either R and K^-1 or C's
  // blocks and M = K^-1 S once
  f->info.solve_bytes =
      sizeof(double) * (2 * hf.mats.size() + hf.svals.size() +
                        (lc == 0 ? size_t(l) * nA + size_t(l) * l : size_t(l) * lc + hf.cvals.size()));
  *out = f;
  return STOKES_OK;
}

// t (l) = alpha M x (+ t when accumulate) for the column-major l-row matrix M with `cols`
// columns, by the library's own two-pass product.
int gemv_rows(fds_solver *f, const double *M, int cols, int chunk, int chunks, const double *x,
              double *t, cudaStream_t s, std::string &err) {
  const int l = f->l;
  if (l % 2 == 0 && l <= kColsMaxRows) {  // whole columns per CTA, staged by bulk copies
    const int cpt = bulk_cols_per_stage(l);
    const size_t smem = bulk_smem_bytes(l, chunk);
    if (l <= 2 * kColsThreads * 4)
      gemv_bulk_partial_kernel<4><<<chunks, kColsThreads, smem, s>>>(l, cols, chunk, cpt, M, x, f->d_gpart);
    else
      gemv_bulk_partial_kernel<8><<<chunks, kColsThreads, smem, s>>>(l, cols, chunk, cpt, M, x, f->d_gpart);
  } else {
    dim3 grid((l + kGemvRows - 1) / kGemvRows, chunks);
    if (l % 2 == 0)  // column starts stay 16-byte aligned: two rows per load
      gemv_cm_partial_kernel<true><<<grid, kGemvThreads, 0, s>>>(l, cols, chunk, M, x, f->d_gpart);
    else
      gemv_cm_partial_kernel<false><<<grid, kGemvThreads, 0, s>>>(l, cols, chunk, M, x, f->d_gpart);
  }
  gemv_reduce_kernel<<<(l + kRedRows - 1) / kRedRows, kRedRows * kRedLanes, 0, s>>>(
      l, chunks, f->d_gpart, 1.0, 0, t);
  FK(cudaGetLastError());
  return STOKES_OK;
}

int fds_solve(fds_solver *f, double *X, int nrhs, cudaStream_t s, cublasHandle_t blas,
              std::string &err) {
  if (!f || !X || nrhs < 0) {
    err = "fds_solve: bad arguments";
    return STOKES_ERR_ARG;
  }
  const double one = 1.0, zero = 0.0;
  cublasSetStream(blas, s);
  for (int c0 = 0; c0 < nrhs; c0 += kChunk) {
    const int nc = std::min(kChunk, nrhs - c0);
    double *Xc = X + size_t(c0) * f->nA;
    int st = hbs_pass(f, Xc, f->d_out, nc, s, err);  // y = A_0^-1 v  (in d_out)
    if (st) return st;
    if (f->l > 0) {
      if (nc == 1 && f->lc > 0) {  // t = C y, s = M t: the library's own products
        sec_dot_kernel<<<f->lc, kDotThreads, 0, s>>>(f->d_csec, f->d_cmap, f->d_cvals, f->d_out, f->d_t);
        FK(cudaGetLastError());
        st = gemv_rows(f, f->d_M, f->lc, f->chunk_K, f->gemv_chunks_K, f->d_t, f->d_s, s, err);
        if (st) return st;
      } else if (nc == 1) {        // t = R y, s = K^-1 t
        st = gemv_rows(f, f->d_R, f->nA, f->chunk_R, f->gemv_chunks_R, f->d_out, f->d_t, s, err);
        if (!st) st = gemv_rows(f, f->d_Kinv, f->l, f->chunk_K, f->gemv_chunks_K, f->d_t, f->d_s, s, err);
        if (st) return st;
      } else if (f->lc > 0) {      // several right-hand sides: library GEMMs per C block, then M
        for (const SecBlock &b : f->h_csec)
          FB(cublasDgemm(blas, CUBLAS_OP_T, CUBLAS_OP_N, b.cols, nc, b.rows, &one, f->d_cvals + b.off,
                         b.rows, f->d_out + b.row0, f->nA, &zero, f->d_t + b.col0, f->lc));
        FB(cublasDgemm(blas, CUBLAS_OP_N, CUBLAS_OP_N, f->l, nc, f->lc, &one, f->d_M, f->l,
                       f->d_t, f->lc, &zero, f->d_s, f->l));
      } else {
        FB(cublasDgemm(blas, CUBLAS_OP_N, CUBLAS_OP_N, f->l, nc, f->nA, &one, f->d_R, f->l,
                       f->d_out, f->nA, &zero, f->d_t, f->l));
        FB(cublasDgemm(blas, CUBLAS_OP_N, CUBLAS_OP_N, f->l, nc, f->l, &one, f->d_Kinv, f->l,
                       f->d_t, f->l, &zero, f->d_s, f->l));
      }
      // v <- v - L s, then x = A_0^-1 v.  The two neighbours' sections each cover both walls,
      // so their row ranges overlap: one launch per neighbour (disjoint rows within each, and
      // a fixed order of the two updates)
      if (f->n_sec_left > 0)
        sub_blocks_kernel<<<dim3(f->n_sec_left, f->sub_row_chunks), kSubRows, 0, s>>>(
            f->d_sec, f->d_svals, f->nA, f->l, nc, f->d_s, Xc);
      if (f->n_sec > f->n_sec_left)
        sub_blocks_kernel<<<dim3(f->n_sec - f->n_sec_left, f->sub_row_chunks), kSubRows, 0, s>>>(
            f->d_sec + f->n_sec_left, f->d_svals, f->nA, f->l, nc, f->d_s, Xc);
      FK(cudaGetLastError());
      st = hbs_pass(f, Xc, f->d_out, nc, s, err);
      if (st) return st;
    }
    FK(cudaMemcpyAsync(Xc, f->d_out, sizeof(double) * f->nA * nc, cudaMemcpyDeviceToDevice, s));
  }
  return STOKES_OK;
}

void fds_get_info(const fds_solver *f, fds_info *info) {
  if (f && info) *info = f->info;
}

void fds_destroy(fds_solver *f) {
  if (!f) return;
  cudaFree(f->d_mats);
  for (HbsBox *b : f->d_boxes) cudaFree(b);
  cudaFree(f->d_R);
  cudaFree(f->d_Kinv);
  cudaFree(f->d_M);
  cudaFree(f->d_csec);
  cudaFree(f->d_cmap);
  cudaFree(f->d_cvals);
  cudaFree(f->d_sec);
  cudaFree(f->d_svals);
  cudaFree(f->d_gpart);
  cudaFree(f->d_up);
  cudaFree(f->d_down);
  cudaFree(f->d_out);
  cudaFree(f->d_t);
  cudaFree(f->d_s);
  delete f;
}

}  // namespace stokes
