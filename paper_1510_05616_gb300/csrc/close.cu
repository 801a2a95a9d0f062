// close.cu -- close evaluation of the vesicles' single layer at nearby nodes (FP64).
//
// The n-point trapezoid rule of the single layer (Eq. (S) summed over a vesicle's nodes) loses
// accuracy like exp(-2 pi delta / h) when a target comes within a few node spacings h of a
// vesicle.  For every (target node, vesicle, image m) pair closer than `factor` h -- the
// vesicle's own nodes at m = 0 excepted, which the Kress rule carries -- this pass adds
//     S_K[f](x) - S_1[f](x),
// S_1 the plain n-point sum the pair kernels take and S_K the same single layer of the curve's
// and the density's trigonometric interpolants by the trapezoid rule on K n resampled points
// (error ~ exp(-2 pi K delta / h)).  Added to stokes_sum_eval's result this gives the close
// interactions to the resampled rule's accuracy.
//
// Resampling: per vesicle, the real Fourier coefficients of x, y, f1, f2 (the Nyquist cosine
// halved, so the interpolant is real) by direct sums, then the interpolants and dx/dt, dy/dt
// at the K n fine parameters by direct synthesis, cosines and sines read from a table of the
// fine grid staged in shared memory.  Correction: one warp per listed target, lanes over the
// fine points and the nodes of each of its close vesicles, a fixed-order shuffle reduction.
// The pair list is built on the host from the context's geometry and kept until it changes.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <unordered_map>
#include <vector>

#include "stokes_internal.cuh"

namespace stokes {
unsigned long long geometry_generation(const stokes_ctx *c);  // fmm.cu

namespace {

constexpr double kPiC = 3.14159265358979323846;
constexpr int kMaxFine = 4096;   // K n per vesicle
constexpr int kResThreads = 256;
constexpr int kCloseWarps = 4;

// Per vesicle vc (curve ves[vc]): fine positions and fine weights
// q_l = f(t_l) |y'(t_l)| (2 pi / (K n)) / (4 pi mu), l < K n.
// Dynamic shared memory: 2 kMaxFine doubles of table + 8 (n/2 + 1) coefficients + 4 n samples.
__global__ void __launch_bounds__(kResThreads)
    resample_kernel(const int *ves, const CurveDev *curves, const double2 *x, const int *node_dens,
                    const double *slp, int K, double c_slp, int stride, double2 *fpos,
                    double2 *fq) {
  extern __shared__ double sm[];
  const CurveDev cv = curves[ves[blockIdx.x]];
  const int n = cv.n, nf = K * n, h = n / 2;
  double *tc = sm, *ts = sm + nf;                 // cos, sin of 2 pi j / nf
  double *co = ts + nf;                           // 8 series of h + 1 coefficients
  double *sv = co + 8 * (h + 1);                  // samples x, y, f1, f2 (n each)
  for (int j = threadIdx.x; j < nf; j += blockDim.x) sincospi(2.0 * j / nf, &ts[j], &tc[j]);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int i = cv.node_begin + j;
    const int row = node_dens[i];
    sv[j] = x[i].x;
    sv[n + j] = x[i].y;
    sv[2 * n + j] = slp[2 * row];
    sv[3 * n + j] = slp[2 * row + 1];
  }
  __syncthreads();
  // a_k = (2/n) sum_j v_j cos(k t_j), b_k = (2/n) sum_j v_j sin(k t_j); a_0, a_{n/2} with 1/n
  for (int idx = threadIdx.x; idx < 4 * (h + 1); idx += blockDim.x) {
    const int s = idx / (h + 1), k = idx - s * (h + 1);
    double a = 0.0, b = 0.0;
    for (int j = 0; j < n; ++j) {
      const int g = int((long long)k * j * K % nf);
      a = fma(sv[s * n + j], tc[g], a);
      b = fma(sv[s * n + j], ts[g], b);
    }
    const double sc = (k == 0 || k == h) ? 1.0 / n : 2.0 / n;
    co[(2 * s) * (h + 1) + k] = a * sc;
    co[(2 * s + 1) * (h + 1) + k] = (k == 0 || k == h) ? 0.0 : b * sc;
  }
  __syncthreads();
  const double dt = 2.0 * kPiC / nf;
  for (int l = threadIdx.x; l < nf; l += blockDim.x) {
    double v[4] = {0.0, 0.0, 0.0, 0.0}, dv[2] = {0.0, 0.0};
    for (int k = 0; k <= h; ++k) {
      const int g = int((long long)k * l % nf);
      const double c = tc[g], s = ts[g];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        v[q] = fma(co[(2 * q) * (h + 1) + k], c, fma(co[(2 * q + 1) * (h + 1) + k], s, v[q]));
#pragma unroll
      for (int q = 0; q < 2; ++q)
        dv[q] = fma(k * co[(2 * q + 1) * (h + 1) + k], c, fma(-k * co[(2 * q) * (h + 1) + k], s, dv[q]));
    }
    const double sp = sqrt(dv[0] * dv[0] + dv[1] * dv[1]) * dt * c_slp;
    fpos[size_t(blockIdx.x) * stride + l] = make_double2(v[0], v[1]);
    fq[size_t(blockIdx.x) * stride + l] = make_double2(v[2] * sp, v[3] * sp);
  }
}

__device__ __forceinline__ void stokeslet_add(double2 z, double px, double py, double q1, double q2,
                                              double &ux, double &uy) {
  const double r1 = z.x - px, r2 = z.y - py;
  const double rr = r1 * r1 + r2 * r2;
  const double lg = -0.5 * log(rr);
  const double c = (r1 * q1 + r2 * q2) / rr;
  ux += lg * q1 + c * r1;
  uy += lg * q2 + c * r2;
}

// One warp per listed target: out[node] += sum over its close (vesicle, image) pairs of
// (resampled sum - plain n-point sum).
__global__ void __launch_bounds__(32 * kCloseWarps)
    close_kernel(int n_tgt, const int *tgt, const int *off, const int2 *pair, const int *ves,
                 const CurveDev *curves, const double2 *x, const double *w, const int *node_dens,
                 const double *slp, double c_slp, double period, int K, int stride,
                 const double2 *fpos, const double2 *fq, double2 *out) {
  const int it = blockIdx.x * kCloseWarps + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (it >= n_tgt) return;
  const int node = tgt[it];
  const double2 z = x[node];
  double ux = 0.0, uy = 0.0;
  for (int e = off[it]; e < off[it + 1]; ++e) {
    const int2 pm = pair[e];  // (vesicle index, image m)
    const CurveDev cv = curves[ves[pm.x]];
    const double sh = pm.y * period;
    const int nf = K * cv.n;
    const double2 *P = fpos + size_t(pm.x) * stride, *Q = fq + size_t(pm.x) * stride;
    for (int l = lane; l < nf; l += 32) stokeslet_add(z, P[l].x + sh, P[l].y, Q[l].x, Q[l].y, ux, uy);
    double vx = 0.0, vy = 0.0;
    for (int j = lane; j < cv.n; j += 32) {
      const int i = cv.node_begin + j;
      const int row = node_dens[i];
      const double c = w[i] * c_slp;
      stokeslet_add(z, x[i].x + sh, x[i].y, c * slp[2 * row], c * slp[2 * row + 1], vx, vy);
    }
    ux -= vx;
    uy -= vy;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ux += __shfl_down_sync(0xffffffffu, ux, o);
    uy += __shfl_down_sync(0xffffffffu, uy, o);
  }
  if (lane == 0) out[node] = make_double2(out[node].x + ux, out[node].y + uy);
}

}  // namespace
}  // namespace stokes

// ---------------------------------------------------------------------------
// host plan and C API
// ---------------------------------------------------------------------------
struct stokes_close {
  stokes_ctx *ctx = nullptr;
  int K = 16, n_ves = 0, n_tgt = 0, stride = 0, smem = 0;
  double factor = 5.0;
  unsigned long long generation = 0;
  int *d_ves = nullptr, *d_tgt = nullptr, *d_off = nullptr;
  int2 *d_pair = nullptr;
  double2 *d_fpos = nullptr, *d_fq = nullptr;
  std::string err;
  stokes_close_info info{};
};

namespace stokes {
namespace {

template <class T>
cudaError_t put(T *&d, const std::vector<T> &h) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&d), sizeof(T) * std::max<size_t>(h.size(), 1));
  if (e != cudaSuccess || h.empty()) return e;
  return cudaMemcpy(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
}

void free_close(stokes_close *f) {
  void *ps[] = {f->d_ves, f->d_tgt, f->d_off, f->d_pair, f->d_fpos, f->d_fq};
  for (void *q : ps) cudaFree(q);
}

struct ClosePairs {
  std::vector<int> ves, tgt, off;
  std::vector<int2> pairs;
  int nmax = 0;
};

// Close (target, vesicle, image) pairs: a target within factor h of some node of the vesicle's
// image (h its largest node spacing), own vesicle at m = 0 excluded.  Vesicle images are binned
// by their bounding circles in a uniform grid; targets test their 3 x 3 cells.  Host data: node
// positions x, curve offsets off (n_curves + 1) and kinds.
void find_close_pairs(const std::vector<double2> &x, const std::vector<int> &coff,
                      const std::vector<int> &kind, double d, double factor, ClosePairs &cp) {
  const int N = int(x.size());
  std::vector<int> &ves = cp.ves;
  std::vector<int> node_ves(N, -1);
  int nmax = 0;
  for (int cv = 0; cv < int(kind.size()); ++cv)
    if (kind[cv] == STOKES_KIND_VESICLE) {
      for (int i = coff[cv]; i < coff[cv + 1]; ++i) node_ves[i] = int(ves.size());
      ves.push_back(cv);
      nmax = std::max(nmax, coff[cv + 1] - coff[cv]);
    }
  cp.nmax = nmax;
  const int V = int(ves.size());
  std::vector<double2> ctr(V);
  std::vector<double> rad(V), hsp(V);
  double G = 0.0;
  for (int v = 0; v < V; ++v) {
    const int b = coff[ves[v]], e = coff[ves[v] + 1], n = e - b;
    double cx = 0.0, cy = 0.0;
    for (int i = b; i < e; ++i) { cx += x[i].x; cy += x[i].y; }
    ctr[v] = make_double2(cx / n, cy / n);
    double R = 0.0, h = 0.0;
    for (int i = b; i < e; ++i) {
      R = std::max(R, std::hypot(x[i].x - ctr[v].x, x[i].y - ctr[v].y));
      const int j = (i + 1 < e) ? i + 1 : b;
      h = std::max(h, std::hypot(x[j].x - x[i].x, x[j].y - x[i].y));
    }
    rad[v] = R;
    hsp[v] = h;
    G = std::max(G, R + factor * h);
  }
  const int m0 = d != 0.0 ? -1 : 0, m1 = d != 0.0 ? 1 : 0;
  std::unordered_map<long long, std::vector<int2>> grid;
  // cell (gx, gy) -> one 64-bit key: gx in the high word, gy's low 32 bits in the low word
  // (shifted as unsigned: a left shift of a negative signed value is undefined)
  auto cell_key = [](long long gx, long long gy) {
    return (long long)((static_cast<unsigned long long>(gx) << 32) ^
                       (static_cast<unsigned long long>(gy) & 0xffffffffull));
  };
  auto key = [&](double px, double py) {
    return cell_key((long long)std::floor(px / G), (long long)std::floor(py / G));
  };
  if (V > 0)
    for (int v = 0; v < V; ++v)
      for (int m = m0; m <= m1; ++m) grid[key(ctr[v].x + m * d, ctr[v].y)].push_back(make_int2(v, m));
  std::vector<int> &tgt = cp.tgt, &off = cp.off;
  off.assign(1, 0);
  std::vector<int2> &pairs = cp.pairs;
  for (int i = 0; i < N && V > 0; ++i) {
    std::vector<int2> cand;
    const long long gx = (long long)std::floor(x[i].x / G), gy = (long long)std::floor(x[i].y / G);
    for (long long dy = -1; dy <= 1; ++dy)
      for (long long dx = -1; dx <= 1; ++dx) {
        const auto it = grid.find(cell_key(gx + dx, gy + dy));
        if (it != grid.end()) cand.insert(cand.end(), it->second.begin(), it->second.end());
      }
    std::sort(cand.begin(), cand.end(), [](int2 a, int2 b) { return a.x != b.x ? a.x < b.x : a.y < b.y; });
    for (const int2 &vm : cand) {
      const int v = vm.x, m = vm.y;
      if (m == 0 && node_ves[i] == v) continue;  // own vesicle: the Kress rule's
      const double reach = factor * hsp[v];
      if (std::hypot(x[i].x - (ctr[v].x + m * d), x[i].y - ctr[v].y) >= rad[v] + reach) continue;
      bool close = false;
      for (int j = coff[ves[v]]; j < coff[ves[v] + 1] && !close; ++j)
        close = std::hypot(x[i].x - (x[j].x + m * d), x[i].y - x[j].y) < reach;
      if (close) pairs.push_back(vm);
    }
    if (int(pairs.size()) > off.back()) {
      tgt.push_back(i);
      off.push_back(int(pairs.size()));
    }
  }
}

int build_close(stokes_close *f) {
  stokes_ctx *c = f->ctx;
  const int N = c->N;
  std::vector<double2> x(N);
  if (cudaMemcpy(x.data(), c->d_x, sizeof(double2) * N, cudaMemcpyDeviceToHost) != cudaSuccess) {
    f->err = "close: reading the geometry failed";
    return STOKES_ERR_CUDA;
  }
  ClosePairs cp;
  find_close_pairs(x, c->off, c->kind, c->period, f->factor, cp);
  const std::vector<int> &ves = cp.ves, &tgt = cp.tgt, &off = cp.off;
  const std::vector<int2> &pairs = cp.pairs;
  const int V = int(ves.size()), nmax = cp.nmax;
  f->n_ves = V;
  f->n_tgt = int(tgt.size());
  f->stride = std::max(1, f->K * nmax);
  f->smem = int(sizeof(double) * (2 * f->K * nmax + 8 * (nmax / 2 + 1) + 4 * nmax));
  cudaError_t e = cudaSuccess;
  auto up = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  up(put(f->d_ves, ves));
  up(put(f->d_tgt, tgt));
  up(put(f->d_off, off));
  up(put(f->d_pair, pairs));
  up(cudaMalloc(reinterpret_cast<void **>(&f->d_fpos), sizeof(double2) * size_t(std::max(V, 1)) * f->stride));
  up(cudaMalloc(reinterpret_cast<void **>(&f->d_fq), sizeof(double2) * size_t(std::max(V, 1)) * f->stride));
  if (f->smem > 48 * 1024)
    up(cudaFuncSetAttribute(resample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, f->smem));
  if (e != cudaSuccess) {
    f->err = std::string("close plan upload: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA;
  }
  f->info.pairs = int(pairs.size());
  f->info.targets = f->n_tgt;
  f->info.vesicles = V;
  return STOKES_OK;
}

}  // namespace
}  // namespace stokes

using namespace stokes;

extern "C" {

int stokes_close_create(stokes_ctx *c, double factor, int upsample, stokes_close **out) {
  if (!out) return STOKES_ERR_ARG;
  *out = nullptr;
  if (!c) return STOKES_ERR_ARG;
  if (!c->have_geom) return STOKES_ERR_NO_GEOM;
  if (c->n_inst != 1 || !(factor > 0.0 && factor <= 50.0) || upsample < 1 || upsample > 64 ||
      upsample * c->max_ves_n > kMaxFine)
    return STOKES_ERR_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return STOKES_ERR_CUDA;
  const auto t0 = std::chrono::steady_clock::now();
  stokes_close *f = new stokes_close();
  f->ctx = c;
  f->K = upsample;
  f->factor = factor;
  f->generation = geometry_generation(c);
  const int st = build_close(f);
  if (st) {
    c->err = f->err;
    free_close(f);
    delete f;
    return st;
  }
  f->info.upsample = upsample;
  f->info.factor = factor;
  f->info.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = f;
  return STOKES_OK;
}

int stokes_close_eval(stokes_close *f, const double *slp, double *out, void *stream) {
  if (!f) return STOKES_ERR_ARG;
  stokes_ctx *c = f->ctx;
  if (!c->have_geom || geometry_generation(c) != f->generation) {
    f->err = "the context's geometry changed since the plan was made";
    return STOKES_ERR_NO_GEOM;
  }
  if ((f->n_ves > 0 && !slp) || !out || (reinterpret_cast<uintptr_t>(out) & 15u)) {
    f->err = "need the vesicle density and a 16-byte aligned output";
    return STOKES_ERR_ARG;
  }
  if (f->n_ves == 0 || f->n_tgt == 0) return STOKES_OK;
  if (cudaSetDevice(c->device) != cudaSuccess) return STOKES_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const double c_slp = 1.0 / (4.0 * kPiC * c->mu);
  resample_kernel<<<f->n_ves, kResThreads, f->smem, s>>>(f->d_ves, c->d_curves, c->d_x,
                                                         c->d_node_dens, slp, f->K, c_slp,
                                                         f->stride, f->d_fpos, f->d_fq);
  close_kernel<<<(f->n_tgt + kCloseWarps - 1) / kCloseWarps, 32 * kCloseWarps, 0, s>>>(
      f->n_tgt, f->d_tgt, f->d_off, f->d_pair, f->d_ves, c->d_curves, c->d_x, c->d_w,
      c->d_node_dens, slp, c_slp, c->period, f->K, f->stride, f->d_fpos, f->d_fq,
      reinterpret_cast<double2 *>(out));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    f->err = cudaGetErrorString(e);
    return STOKES_ERR_CUDA;
  }
  return STOKES_OK;
}

int stokes_close_get_info(const stokes_close *f, stokes_close_info *info) {
  if (!f || !info) return STOKES_ERR_ARG;
  *info = f->info;
  return STOKES_OK;
}

int stokes_close_last_error(const stokes_close *f, char *buf, size_t len) {
  if (!f || !buf || len == 0) return STOKES_ERR_ARG;
  snprintf(buf, len, "%s", f->err.c_str());
  return STOKES_OK;
}

int stokes_close_destroy(stokes_close *f) {
  if (!f) return STOKES_OK;
  cudaSetDevice(f->ctx->device);
  cudaDeviceSynchronize();
  free_close(f);
  delete f;
  return STOKES_OK;
}

}  // extern "C"
