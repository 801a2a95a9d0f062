// k_prep.cu -- geometry preparation, per-call density packing and the FP64 finishing pass.
//
//  * geometry prep (once per stokes_geom_set): FP32 (hi, lo) source coordinates (each value
//    duplicated for the packed two-target arithmetic of the FP32 pair kernel), FP64
//    source coordinates, Kress product-rule tables, a finiteness check of the geometry;
//  * pack (every call): source density records q = w f / (4 pi mu) (stokeslet, Eq. (S))
//    and q = w tau / pi (stresslet, Eq. (D)), with a finiteness check of the densities;
//  * finish (every call): the FP64 cross-split reduction of the pair-kernel partials in
//    fixed order, plus the wall Nystrom diagonal -kappa/(2 pi) t t^T w tau and jump * tau
//    (Sec. 2.3, Eq. (JR)), plus the FP64 Kress self term of the single layer on each
//    vesicle (Sec. 3.2).
#include <algorithm>

#include "stokes_internal.cuh"
#include "bulk_pipe.cuh"

namespace stokes {

// ---------------------------------------------------------------------------
// geometry preparation
// ---------------------------------------------------------------------------
// FP32 source coordinates, every value duplicated into both halves of a packed pair:
// pos[2s] = (x_hi, x_hi, y_hi, y_hi), pos[2s+1] = (x_lo, x_lo, y_lo, y_lo).
__global__ void src_pos32_kernel(int slots, const int *slot_node, const double2 *x, float4 *pos) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= slots) return;
  const int i = slot_node[s];
  float4 hi = make_float4(0.f, 0.f, 0.f, 0.f), lo = hi;
  if (i >= 0) {
    const double2 p = x[i];
    const float xh = __double2float_rn(p.x), yh = __double2float_rn(p.y);
    const float xl = __double2float_rn(p.x - double(xh)), yl = __double2float_rn(p.y - double(yh));
    hi = make_float4(xh, xh, yh, yh);
    lo = make_float4(xl, xl, yl, yl);
  }
  pos[2 * s] = hi;
  pos[2 * s + 1] = lo;
}

__global__ void src_pos64_kernel(int slots, const int *slot_node, const double2 *x, double2 *pos) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= slots) return;
  const int i = slot_node[s];
  pos[s] = (i >= 0) ? x[i] : make_double2(0.0, 0.0);
}

// Kress table of a closed curve with n nodes (n even):
//   T_0 = -R_0 / 2,  T_j = -R_j / 2 + (pi / n) log(4 sin^2(pi j / n))  (j >= 1),
//   R_j = -(4 pi / n) sum_{p=1}^{n/2-1} cos(2 pi p j / n) / p - (4 pi / n^2) (-1)^j.
// The self term then reads  sum_k [T_{(i-k) mod n} - (pi/n) log |x_i - x_k|^2] g_k + ...
__global__ void kress_table_kernel(int n, double *T) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double acc = 0.0;
  for (int p = 1; p <= n / 2 - 1; ++p) {
    const long long k = (static_cast<long long>(p) * j) % n;  // cos(2 pi p j / n) exactly reduced
    acc += cospi(2.0 * double(k) / double(n)) / double(p);
  }
  const double R = -(4.0 * kPi / n) * acc - (4.0 * kPi / (double(n) * n)) * ((j & 1) ? -1.0 : 1.0);
  double t = -0.5 * R;
  if (j > 0) {
    const double sn = sinpi(double(j) / double(n));
    t += (kPi / n) * log(4.0 * sn * sn);
  }
  T[j] = t;
}

__global__ void geom_check_kernel(int n, const double2 *x, const double2 *nrm, const double *w,
                                  const double *kap, unsigned *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool ok = isfinite(x[i].x) && isfinite(x[i].y) && isfinite(nrm[i].x) && isfinite(nrm[i].y) &&
            isfinite(w[i]);
  if (kap) ok = ok && isfinite(kap[i]);
  if (!ok) atomicOr(status, kStatusNonfinite);
}

// ---------------------------------------------------------------------------
// per-call density packing
// ---------------------------------------------------------------------------
struct PackArgs {
  int slots, wall_slots;
  const int *slot_node;
  const int *node_dens;
  const double *w;
  const double2 *nrm;
  const double *slp, *dlp;
  double c_slp;  // 1 / (4 pi mu)
  unsigned *status;
  int N, n_slp_rows, n_dlp_rows;  // nodes and density rows (debug bounds checks)
};

// Node and density row of source slot s, bounds-checked in the debug build: false (and the
// slot packed as a zero-weight dummy) when either is out of range.
__device__ __forceinline__ bool slot_source(const PackArgs &a, int s, int &i, int &row) {
  i = a.slot_node[s];
  if (i < 0 || !dcheck(i < a.N, a.status)) return false;
  row = a.node_dens[i];
  const int rows = s < a.wall_slots ? a.n_dlp_rows : a.n_slp_rows;
  return dcheck(row >= 0 && row < rows, a.status);
}

// FP32 source records, duplicated like the coordinates: val[2s] = (q1, q1, q2, q2) and
// val[2s+1] = (p1, p1, p2, p2) for a stokeslet source, (n1, n1, n2, n2) for a stresslet source.
__global__ void pack_f32_kernel(PackArgs a, float4 *val) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.slots) return;
  int i = -1, row = 0;
  float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
  if (slot_source(a, s, i, row)) {
    const double w = a.w[i];
    if (s < a.wall_slots) {
      const double t1 = a.dlp[2 * row], t2 = a.dlp[2 * row + 1];
      if (!isfinite(t1) || !isfinite(t2)) atomicOr(a.status, kStatusNonfinite);
      const double2 n = a.nrm[i];
      const double c = w / kPi;
      v0 = __double2float_rn(c * t1);
      v1 = __double2float_rn(c * t2);
      v2 = __double2float_rn(n.x);
      v3 = __double2float_rn(n.y);
    } else {
      const double f1 = a.slp[2 * row], f2 = a.slp[2 * row + 1];
      if (!isfinite(f1) || !isfinite(f2)) atomicOr(a.status, kStatusNonfinite);
      const double c = w * a.c_slp;
      const double h = -0.5 * 0.69314718055994530942;  // -(ln 2)/2: log(1/r) = h log2(r^2)
      v0 = __double2float_rn(c * f1);
      v1 = __double2float_rn(c * f2);
      v2 = __double2float_rn(h * c * f1);
      v3 = __double2float_rn(h * c * f2);
    }
  }
  val[2 * s] = make_float4(v0, v0, v1, v1);
  val[2 * s + 1] = make_float4(v2, v2, v3, v3);
}

__global__ void pack_f64_kernel(PackArgs a, double4_32a *val) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.slots) return;
  int i = -1, row = 0;
  double4_32a r = make_double4_32a(0.0, 0.0, 0.0, 0.0);
  if (slot_source(a, s, i, row)) {
    const double w = a.w[i];
    if (s < a.wall_slots) {
      const double t1 = a.dlp[2 * row], t2 = a.dlp[2 * row + 1];
      if (!isfinite(t1) || !isfinite(t2)) atomicOr(a.status, kStatusNonfinite);
      const double2 n = a.nrm[i];
      const double c = w / kPi;
      r = make_double4_32a(c * t1, c * t2, n.x, n.y);
    } else {
      const double f1 = a.slp[2 * row], f2 = a.slp[2 * row + 1];
      if (!isfinite(f1) || !isfinite(f2)) atomicOr(a.status, kStatusNonfinite);
      const double c = w * a.c_slp;
      r = make_double4_32a(c * f1, c * f2, -0.5 * c * f1, -0.5 * c * f2);  // log(1/r) = -log(r^2)/2
    }
  }
  val[s] = r;
}

// ---------------------------------------------------------------------------
// finishing pass
// ---------------------------------------------------------------------------
// Where the split partials of a target live: one instance (partial[k * N + i], k < splits),
// or batched instances (each with its own split count, stride and offset).
struct PartLoc {
  const int *node_inst;   // NULL for a single instance
  const InstDev *inst;
  int f64;
  int N, splits;
  long long cap;          // elements of the partial buffer (debug bounds checks)
  unsigned *status;
};

__device__ __forceinline__ void part_sum(const PartLoc &L, const double2 *partial, int i,
                                         double &ux, double &uy) {
  long long base;
  int stride, cnt;
  if (L.node_inst) {
    const InstDev &I = L.inst[L.node_inst[i]];
    base = (L.f64 ? I.part_off64 : I.part_off32) + (i - I.node_begin);
    stride = I.N;
    cnt = L.f64 ? I.splits64 : I.splits32;
  } else {
    base = i;
    stride = L.N;
    cnt = L.splits;
  }
  ux = 0.0;
  uy = 0.0;
  for (int k = 0; k < cnt; ++k) {
    const long long idx = base + (long long)k * stride;
    if (!dcheck(idx >= 0 && idx < L.cap, L.status)) continue;
    const double2 p = partial[idx];
    ux += p.x;
    uy += p.y;
  }
}

__global__ void finish_walls_kernel(int n_wall, const int *wall_nodes, PartLoc L,
                                    const double2 *partial, const int *node_dens,
                                    const double2 *nrm, const double *w, const double *kap,
                                    const double *dlp, double jump, double2 *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_wall) return;
  const int i = wall_nodes[t];
  double ux, uy;
  part_sum(L, partial, i, ux, uy);
  const int row = node_dens[i];
  const double t1 = dlp[2 * row], t2 = dlp[2 * row + 1];
  const double2 n = nrm[i];
  const double tx = -n.y, ty = n.x;  // unit tangent
  const double c = -kap[i] / (2.0 * kPi) * w[i] * (tx * t1 + ty * t2);
  out[i] = make_double2(ux + c * tx + jump * t1, uy + c * ty + jump * t2);
}

// Kress self term of the single layer (Sec. 3.2), FP64, one block per vesicle; writes
// u_self to self[row] (row = the node's row in the vesicle density array).  Runs on a side
// stream, concurrently with the pair kernel (FP64 pipe vs FP32/MUFU pipes).
__global__ void self_kress_kernel(const int *ves_curves, const CurveDev *curves,
                                  const double *kress, const double2 *x, const double2 *nrm,
                                  const double *w, const double *slp, double c_slp,
                                  double2 *self, const LogTab *lt) {
  extern __shared__ double sh[];
  const CurveDev cv = curves[ves_curves[blockIdx.x]];
  const int n = cv.n;
  double *sx = sh, *sy = sh + n, *g1 = sh + 2 * n, *g2 = sh + 3 * n;
  const double h = 2.0 * kPi / n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int j = cv.node_begin + k;
    const double2 p = x[j];
    sx[k] = p.x;
    sy[k] = p.y;
    const double s = w[j] / h;  // speed |x'(t_k)|
    const int row = cv.dens_begin + k;
    g1[k] = c_slp * s * slp[2 * row];
    g2[k] = c_slp * s * slp[2 * row + 1];
  }
  __syncthreads();
  const double *T = kress + cv.kress_off;
  const double pin = kPi / n;
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    const int i = cv.node_begin + a;
    const double xa = sx[a], ya = sy[a];
    double vx = 0.0, vy = 0.0;
    for (int k = 0; k < n; ++k) {
      const double gx = g1[k], gy = g2[k];
      double coef, m11, m12, m22;
      if (k == a) {
        const double s = w[i] / h;
        const double2 nn = nrm[i];
        const double tx = -nn.y, ty = nn.x;
        coef = T[0] - pin * flog64(s * s, lt);
        m11 = tx * tx;
        m12 = tx * ty;
        m22 = ty * ty;
      } else {
        const double rx = xa - sx[k], ry = ya - sy[k];
        const double rr = rx * rx + ry * ry;
        const double inv = 1.0 / rr;
        int dj = a - k;
        if (dj < 0) dj += n;
        coef = T[dj] - pin * flog64(rr, lt);
        m11 = rx * rx * inv;
        m12 = rx * ry * inv;
        m22 = ry * ry * inv;
      }
      vx += coef * gx + h * (m11 * gx + m12 * gy);
      vy += coef * gy + h * (m12 * gx + m22 * gy);
    }
    self[cv.dens_begin + a] = make_double2(vx, vy);
  }
}

// The same Kress blocks stored (geometry only): thread p = k n + a of vesicle blockIdx.y writes
// G11, G12, G22 of the block c_slp s_k [coef I + h M] (coef and M as in self_kress_kernel) to
// G[off + p], G[off + n^2 + p], G[off + 2 n^2 + p].
__global__ void self_matrix_kernel(const int *ves_curves, const CurveDev *curves,
                                   const long long *g_off, const double *kress, const double2 *x,
                                   const double2 *nrm, const double *w, double c_slp,
                                   const LogTab *lt, double *G) {
  const CurveDev cv = curves[ves_curves[blockIdx.y]];
  const int n = cv.n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * n) return;
  const int k = p / n, a = p - k * n;
  const double h = 2.0 * kPi / n;
  const double pin = kPi / n;
  const double *T = kress + cv.kress_off;
  const int i = cv.node_begin + a, j = cv.node_begin + k;
  double coef, m11, m12, m22;
  if (k == a) {
    const double sp = w[i] / h;
    const double2 nn = nrm[i];
    const double tx = -nn.y, ty = nn.x;
    coef = T[0] - pin * flog64(sp * sp, lt);
    m11 = tx * tx;
    m12 = tx * ty;
    m22 = ty * ty;
  } else {
    const double2 xa = x[i], xk = x[j];
    const double rx = xa.x - xk.x, ry = xa.y - xk.y;
    const double rr = rx * rx + ry * ry;
    const double inv = 1.0 / rr;
    int dj = a - k;
    if (dj < 0) dj += n;
    coef = T[dj] - pin * flog64(rr, lt);
    m11 = rx * rx * inv;
    m12 = rx * ry * inv;
    m22 = ry * ry * inv;
  }
  const double sc = c_slp * (w[j] / h);  // density scale of source node k: c_slp s_k
  double *Gv = G + g_off[blockIdx.y];
  const size_t nn2 = size_t(n) * n;
  Gv[p] = sc * (coef + h * m11);
  Gv[nn2 + p] = sc * (h * m12);
  Gv[2 * nn2 + p] = sc * (coef + h * m22);
}

// u_self(a) = sum_k G_ak f_k from the stored blocks: one block per vesicle, the density staged
// in shared memory, a thread per target node reading column-contiguous G (coalesced).
__global__ void self_apply_kernel(const int *ves_curves, const CurveDev *curves,
                                  const long long *g_off, const double *G, const double *slp,
                                  double2 *self) {
  extern __shared__ double sh[];
  const CurveDev cv = curves[ves_curves[blockIdx.x]];
  const int n = cv.n;
  double *f1 = sh, *f2 = sh + n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int row = cv.dens_begin + k;
    f1[k] = slp[2 * row];
    f2[k] = slp[2 * row + 1];
  }
  __syncthreads();
  const double *G11 = G + g_off[blockIdx.x];
  const size_t nn2 = size_t(n) * n;
  const double *G12 = G11 + nn2, *G22 = G11 + 2 * nn2;
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    double vx = 0.0, vy = 0.0;
    for (int k = 0; k < n; ++k) {
      const size_t e = size_t(k) * n + a;
      const double g11 = G11[e], g12 = G12[e], g22 = G22[e];
      vx = fma(g11, f1[k], fma(g12, f2[k], vx));
      vy = fma(g12, f1[k], fma(g22, f2[k], vy));
    }
    self[cv.dens_begin + a] = make_double2(vx, vy);
  }
}

// Vesicle nodes: FP64 fixed-order reduction of the split partials plus the self term.
__global__ void finish_vesicle_nodes_kernel(int n_ves, const int *ves_nodes, PartLoc L,
                                            const double2 *partial, const int *node_dens,
                                            const double2 *self, double2 *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_ves) return;
  const int i = ves_nodes[t];
  double ux, uy;
  part_sum(L, partial, i, ux, uy);
  const double2 v = self[node_dens[i]];
  out[i] = make_double2(ux + v.x, uy + v.y);
}

__global__ void finish_free_kernel(int T, int splits, const double2 *partial, long long cap,
                                   unsigned *status, double2 *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  double ux = 0.0, uy = 0.0;
  for (int k = 0; k < splits; ++k) {
    const long long idx = (long long)k * T + t;
    if (!dcheck(idx < cap, status)) continue;
    const double2 p = partial[idx];
    ux += p.x;
    uy += p.y;
  }
  out[t] = make_double2(ux, uy);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int nblk(int n, int b) { return (n + b - 1) / b; }

cudaError_t launch_self_matrix(stokes_ctx *c, cudaStream_t s);

cudaError_t launch_geom_prep(stokes_ctx *c, cudaStream_t s) {
  const int s32 = c->wall_slots + c->ves_slots_f32;
  const int s64 = c->wall_slots_f64 + c->ves_slots_f64;
  geom_check_kernel<<<nblk(c->N, 256), 256, 0, s>>>(c->N, c->d_x, c->d_nrm, c->d_w,
                                                    c->n_wall_nodes ? c->d_kap : nullptr,
                                                    c->d_status);
  src_pos32_kernel<<<nblk(s32, 256), 256, 0, s>>>(s32, c->d_slot_node32, c->d_x, c->d_src_pos32);
  src_pos64_kernel<<<nblk(s64, 256), 256, 0, s>>>(s64, c->d_slot_node64, c->d_x, c->d_src_pos64);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_self_matrix(c, s);
  if (e != cudaSuccess) return e;
  return launch_geom_prep_df(c, s);
}

__global__ void logtab_init_kernel(LogTab *t) {
  const int k = threadIdx.x;
  if (k < kLogTab) {
    const double a = 1.0 + (k + 0.5) / kLogTab;
    t->a[k] = a;
    t->inv_a[k] = 1.0 / a;
    t->log_a[k] = log(a);
  }
  if (k == 0) {
    const double l2 = log(2.0);
    const double hi = __longlong_as_double(__double_as_longlong(l2) & ~0x1FFFFFLL);  // 32 bits
    t->ln2_hi = hi;
    t->ln2_lo = l2 - hi;
  }
}

cudaError_t launch_logtab_init(LogTab *t, cudaStream_t s) {
  logtab_init_kernel<<<1, kLogTab, 0, s>>>(t);
  return cudaGetLastError();
}

__global__ void check_log64_kernel(int n, const double *x, double *out, const LogTab *t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = flog64(x[i], t);
}

cudaError_t launch_check_log64(stokes_ctx *c, int n, const double *x, double *out,
                               cudaStream_t s) {
  check_log64_kernel<<<nblk(n, 256), 256, 0, s>>>(n, x, out, c->d_logtab);
  return cudaGetLastError();
}

cudaError_t launch_kress_table(int n, double *T, cudaStream_t s) {
  kress_table_kernel<<<nblk(n, 128), 128, 0, s>>>(n, T);
  return cudaGetLastError();
}

cudaError_t launch_pack(stokes_ctx *c, int precision, const double *slp, const double *dlp,
                        cudaStream_t s) {
  PackArgs a{};
  a.node_dens = c->d_node_dens;
  a.w = c->d_w;
  a.nrm = c->d_nrm;
  a.slp = slp;
  a.dlp = dlp;
  a.c_slp = 1.0 / (4.0 * kPi * c->mu);
  a.status = c->d_status;
  a.N = c->N;
  a.n_slp_rows = c->n_ves_nodes;
  a.n_dlp_rows = c->n_wall_nodes;
  if (precision == STOKES_DOUBLE_FLOAT) return launch_pack_df(c, slp, dlp, s);
  if (precision == STOKES_FP32_KAHAN) {
    a.slots = c->wall_slots + c->ves_slots_f32;
    a.wall_slots = c->wall_slots;
    a.slot_node = c->d_slot_node32;
    pack_f32_kernel<<<nblk(a.slots, 256), 256, 0, s>>>(a, c->d_src_val32);
  } else {
    a.slots = c->wall_slots_f64 + c->ves_slots_f64;
    a.wall_slots = c->wall_slots_f64;
    a.slot_node = c->d_slot_node64;
    pack_f64_kernel<<<nblk(a.slots, 256), 256, 0, s>>>(a, c->d_src_val64);
  }
  return cudaGetLastError();
}

cudaError_t launch_self_matrix(stokes_ctx *c, cudaStream_t s) {
  if (!c->self_matrix || c->n_ves_curves == 0) return cudaSuccess;
  const int nn = c->max_ves_n * c->max_ves_n;
  self_matrix_kernel<<<dim3(nblk(nn, 256), c->n_ves_curves), 256, 0, s>>>(
      c->d_ves_curve_ids, c->d_curves, c->d_selfG_off, c->d_kress, c->d_x, c->d_nrm, c->d_w,
      1.0 / (4.0 * kPi * c->mu), c->d_logtab, c->d_selfG);
  return cudaGetLastError();
}

cudaError_t launch_self(stokes_ctx *c, const double *slp, cudaStream_t s) {
  if (c->n_ves_curves > 0 && c->self_matrix) {
    self_apply_kernel<<<c->n_ves_curves, std::min(256, (c->max_ves_n + 31) / 32 * 32),
                        size_t(2) * c->max_ves_n * sizeof(double), s>>>(
        c->d_ves_curve_ids, c->d_curves, c->d_selfG_off, c->d_selfG, slp, c->d_self);
    return cudaGetLastError();
  }
  if (c->n_ves_curves > 0) {
    const size_t smem = size_t(4) * c->max_ves_n * sizeof(double);
    self_kress_kernel<<<c->n_ves_curves, 128, smem, s>>>(c->d_ves_curve_ids, c->d_curves,
                                                         c->d_kress, c->d_x, c->d_nrm, c->d_w,
                                                         slp, 1.0 / (4.0 * kPi * c->mu),
                                                         c->d_self, c->d_logtab);
  }
  return cudaGetLastError();
}

static cudaError_t finish_nodes(stokes_ctx *c, const PartLoc &L, const double *dlp, double jump,
                                double2 *out, cudaStream_t s) {
  if (c->n_wall_nodes > 0)
    finish_walls_kernel<<<nblk(c->n_wall_nodes, 256), 256, 0, s>>>(
        c->n_wall_nodes, c->d_wall_nodes, L, c->d_partial, c->d_node_dens, c->d_nrm, c->d_w,
        c->d_kap, dlp, jump, out);
  if (c->n_ves_nodes > 0)
    finish_vesicle_nodes_kernel<<<nblk(c->n_ves_nodes, 256), 256, 0, s>>>(
        c->n_ves_nodes, c->d_ves_nodes, L, c->d_partial, c->d_node_dens, c->d_self, out);
  return cudaGetLastError();
}

cudaError_t launch_finish_nodes(stokes_ctx *c, int splits, const double *slp, const double *dlp,
                                double jump, double2 *out, cudaStream_t s) {
  (void)slp;
  const PartLoc L{nullptr, nullptr, 0, c->N, splits,
                  partial_check_cap(c, (long long)c->partial_cap, (long long)splits * c->N),
                  c->d_status};
  return finish_nodes(c, L, dlp, jump, out, s);
}

cudaError_t launch_finish_batch(stokes_ctx *c, int precision, const double *dlp, double jump,
                                double2 *out, cudaStream_t s) {
  const PartLoc L{c->d_node_inst, c->d_inst, precision != STOKES_FP32_KAHAN ? 1 : 0, c->N, 0,
                  partial_check_cap(c, (long long)c->partial_cap,
                                    precision == STOKES_FP32_KAHAN ? c->batch_part32 : c->batch_part64),
                  c->d_status};
  return finish_nodes(c, L, dlp, jump, out, s);
}

cudaError_t launch_finish_free(stokes_ctx *c, int splits, int n_targets, double2 *out,
                               cudaStream_t s) {
  finish_free_kernel<<<nblk(n_targets, 256), 256, 0, s>>>(
      n_targets, splits, c->d_partial,
      partial_check_cap(c, (long long)c->partial_cap, (long long)splits * n_targets), c->d_status,
      out);
  return cudaGetLastError();
}

}  // namespace stokes

namespace stokes {

// Same as launch_finish_free, reading the partials from a caller-chosen buffer.
cudaError_t launch_finish_free_scratch(int splits, int n_targets, const double2 *partial,
                                       double2 *out, cudaStream_t s) {
  // the caller's buffer holds exactly the splits x targets partials (no status word here)
  finish_free_kernel<<<nblk(n_targets, 256), 256, 0, s>>>(
      n_targets, splits, partial, (long long)splits * n_targets, nullptr, out);
  return cudaGetLastError();
}

}  // namespace stokes

namespace stokes {

// Failure-handling check of the pipeline wait: one block waits on an mbarrier that nothing
// arrives at, gives up after the wait's bound (~0.5 s) and records the timeout in the status
// word, exactly as a pair kernel whose tile copy never lands would.
__global__ void wait_timeout_check_kernel(unsigned *status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait_bounded(&bar, 0u)) atomicOr(status, kStatusTimeout);
  }
}

cudaError_t launch_wait_timeout_check(stokes_ctx *c, cudaStream_t s) {
  wait_timeout_check_kernel<<<1, 32, 0, s>>>(c->d_status);
  return cudaGetLastError();
}

}  // namespace stokes
