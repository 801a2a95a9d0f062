// fmm.cu -- fast multipole evaluation of the near-image layer-potential sum at the nodes (FP64).
//
// The same discrete sum as stokes_sum_eval (stokeslet sources on the vesicles, stresslet sources
// on the walls, images m in {-1, 0, +1}, own curve skipped at m = 0, Kress self terms and the
// wall curvature diagonal), with the pair sum in O(N) by the classical 2-D FMM in complex
// variables.  With z = x1 + i x2, r = z - w, a stokeslet source of weight q = w f / (4 pi mu)
// and a stresslet source of weight T = w tau / pi with normal nu (complex numbers throughout):
//   stokeslet  -q log|r| + (r . q) r / |r|^2 = -q log|r| + q/2 + (1/2) r conj(q / r)
//   stresslet  (r . n)(r . T) r / |r|^4 = (1/4) [nu T / r + 2 (n . T) / conj(r)
//                                                + conj(nu T conj(r) / r^2)]
// so every target needs, over the sources, the log potentials Phi_c(z) = sum_j c_j log(z - w_j)
// of six charge sets -- q1, q2 (real parts of the values; q = q1 + i q2), conj(w) q, 2 n . T,
// nu T, nu T conj(w) -- and their first and second derivatives:
//   u = -(Re Phi_q1 + i Re Phi_q2) + Q/2 + (1/2) [z conj(Phi'_q1 + i Phi'_q2) - conj(Phi'_wq)]
//     + (1/4) [Phi'_nuT + conj(Phi'_2nT) + conj(Phi''_nuTw - conj(z) Phi''_nuT)],
// Q the sum of the stokeslet weights of the sources taken through the expansions.
// Expansions (scaled by the cell side h): multipole a_0 log(z - c) + sum_k a_k h^k / (z - c)^k,
// local sum_k b_k ((z - c)/h)^k, with the shift and conversion formulas of Greengard and
// Rokhlin for the 2-D log kernel.  The conj(w)-weighted sets are taken relative to each
// expansion's own centre c (conj(w - c) q, nu T conj(w - c)), re-centred exactly at every shift
// and conversion, and the assembly uses z - c of the target leaf: the terms z conj(Phi'_q) and
// conj(Phi'_wq) then no longer cancel from |z| |q| down to |q| (see recentred()).  Tree: a forest of square roots of side S covering the
// sources (the nodes and their +-d images) and the targets, uniform depth L, Morton keys;
// interaction lists are the children of the parent's neighbours that are not neighbours; the
// 3 x 3 neighbour leaves are summed directly (coincident pairs skipped).  Pairs of a vesicle
// with itself at m = 0 are then removed by a direct pass over each vesicle's own nodes.
//
// The plan (sorted sources, cells, lists) is built on the host from the context's geometry and
// reused by every evaluation until that geometry changes.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "df.cuh"
#include "stokes_internal.cuh"

namespace stokes {
namespace {

constexpr double kPiF = 3.14159265358979323846;
constexpr int kSets = 6;
constexpr int kMaxOrder = 40;               // expansion order p <= kMaxOrder
constexpr int kBin = 2 * kMaxOrder + 2;     // binomials C(n, k), n < kBin
constexpr int kLeafThreads = 128;

// Binomials in global memory (cached in L1): the threads of a warp read different entries, which
// the constant cache would serialize.
__device__ double c_binom[kBin][kBin];

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cinv(double2 a) {
  const double d = 1.0 / (a.x * a.x + a.y * a.y);
  return make_double2(a.x * d, -a.y * d);
}
// acc += a b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 cpow(double2 a, int n) {  // n >= 0, by squaring
  double2 r = make_double2(1.0, 0.0);
  while (n) {
    if (n & 1) r = cmul(r, a);
    a = cmul(a, a);
    n >>= 1;
  }
  return r;
}

// The same operations on FP32 complex numbers (the evaluations at low orders run their
// expansions in FP32), and the complex type of each real type.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
template <typename R> struct CxOf;
template <> struct CxOf<double> { using type = double2; };
template <> struct CxOf<float> { using type = float2; };
template <typename R> using cx = typename CxOf<R>::type;
template <typename R> __device__ __forceinline__ cx<R> mkc(double x, double y) {
  return cx<R>{R(x), R(y)};
}
template <typename R> __device__ __forceinline__ cx<R> tocx(double2 a) { return mkc<R>(a.x, a.y); }
__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }

// A complex number in double-float: (re.h, re.l, im.h, im.l).
__device__ __forceinline__ float4 split_c(double2 a) {
  const df r = split_df(a.x), i = split_df(a.y);
  return make_float4(r.h, r.l, i.h, i.l);
}
struct dfc {
  df re, im;
};
__device__ __forceinline__ dfc dfc_of(float4 a) { return {{a.x, a.y}, {a.z, a.w}}; }
__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
// acc += a b (complex, double-float)
__device__ __forceinline__ void dfc_mul_acc(dfc &acc, dfc a, dfc b) {
  df_mul_acc(acc.re, a.re, b.re);
  df_mul_acc(acc.re, df_neg(a.im), b.im);
  df_mul_acc(acc.im, a.re, b.im);
  df_mul_acc(acc.im, a.im, b.re);
}
// x + y (double-float): TwoSum of the high parts, the low parts added to its error.
__device__ __forceinline__ df df_sum(df x, df y) {
  const df s = two_sum(x.h, y.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ void dfc_renorm(dfc &a) {
  df_renorm(a.re);
  df_renorm(a.im);
}
__device__ __forceinline__ float4 dfc_pack(dfc a) { return make_float4(a.re.h, a.re.l, a.im.h, a.im.l); }

// Coefficient r of the expansion stored at E + base (kSets sets of p1 coefficients) with the
// sets 2 and 5 moved to a new centre.  Those two sets carry conj(w - c) q and nu T conj(w - c):
// each expansion keeps them relative to its own centre c, which spares the assembly the
// cancellation between z conj(Phi'_q) and conj(Phi'_wq) (terms of size |z| |q| whose
// difference is |q|-sized), and moving the centre by dc = c_old - c_new adds conj(dc) times the
// q (= q1 + i q2) or nu T expansion, coefficient by coefficient (the expansions are linear in
// the charges).
template <typename C>
__device__ __forceinline__ C recentred(const C *E, size_t base, int r, int p1, double2 dc) {
  const int si = r / p1, qi = r - si * p1;
  C a = E[base + r];
  if (si == 2 || si == 5) {
    const C cdc = C{decltype(a.x)(dc.x), decltype(a.x)(-dc.y)};
    C b;
    if (si == 2) {
      const C a0 = E[base + qi], a1 = E[base + p1 + qi];
      b = C{a0.x - a1.y, a0.y + a1.x};  // a0 + i a1
    } else {
      b = E[base + 4 * p1 + qi];
    }
    a = cfma(cdc, b, a);
  }
  return a;
}

// The six charges of one (image) source at w: vesicle value (q1, q2, ., .), wall value
// (T1, T2, n1, n2).
__device__ __forceinline__ void charges(bool wall, double2 w, double4_32a v, double2 (&c)[kSets]) {
  // w is taken relative to the expansion's centre (the source leaf's); see recentred()
  if (!wall) {
    const double2 q = make_double2(v.x, v.y);
    c[0] = make_double2(v.x, 0.0);
    c[1] = make_double2(v.y, 0.0);
    c[2] = cmul(cconj(w), q);
    c[3] = c[4] = c[5] = make_double2(0.0, 0.0);
  } else {
    const double2 T = make_double2(v.x, v.y), nu = make_double2(v.z, v.w);
    const double2 nT = cmul(nu, T);
    c[0] = c[1] = c[2] = make_double2(0.0, 0.0);
    c[3] = make_double2(2.0 * (v.z * v.x + v.w * v.y), 0.0);
    c[4] = nT;
    c[5] = cmul(nT, cconj(w));
  }
}

struct FmmDev {
  int p, n_src, N;            // p: the evaluation's expansion order; N: the context's nodes
  int want_nodes;             // 0: only the extra targets are wanted (node targets skipped)
  double2 *out_extra;         // [targets N ..] free-target velocities, or NULL (not wanted)
  int near32;                 // near-field pairs in FP32 arithmetic (accumulated in FP64)
  int tp1;                    // row length of tpow: the plan's order + 1
  int wall_slots;
  const int2 *src_slot;       // [n_src] (slot, m), sorted by leaf
  const double2 *src_pos;     // [n_src] image positions, sorted by leaf
  const double4_32a *val;     // FP64 slot values (packed per call)
  const double2 *scell_ctr;   // [source cells] centres
  const int2 *scell_rng;      // leaves: source range; others: child cell range
  const double2 *tcell_ctr;   // [target cells]
  const int *tcell_parent;    // [target cells] parent target cell or -1
  const int *il_off, *il_idx; // interaction lists (source cell indices)
  const int *nl_off, *nl_idx; // near lists of target leaves (source leaf indices)
  const int *tgt_node;        // [N] node of each sorted target
  const int2 *tleaf_rng;      // [target leaves] range of sorted targets
  const double2 *x;           // [N + extra] target positions: the nodes, then the free targets
  double2 *M;                 // [source cells][kSets][p + 1], FP64 or (FP32 evaluations) float2
  double2 *Lc;                // [target cells][kSets][p + 1], likewise
  double2 *out;               // [N] pair sums (node order)
  int n_roots_src, root_src0; // source cells of level 0: [root_src0, root_src0 + n_roots_src)
  const double2 *tpow;        // [49][tp1] t^-n of the integer offsets |t_x|, |t_y| <= 3
  const double2 *tlog;        // [49] log(-t) of the same offsets
  const int *src_own;         // [n_src] vesicle curve of an m = 0 source, else -1
  const int *node_curve;      // [N] vesicle curve of a node, else -1
  const float4 *m2m_df;       // M2M shift weights per child quadrant (double-float), plan order
  float4 *Mf;                 // FP64 evaluations: M split into float pairs (re.h, re.l, im.h,
                              // im.l), written beside M by P2M and M2M, read by m2l_df_kernel
  const float4 *tpow_df;      // [49][tp1] tpow split likewise
  int mp;                     // the plan's order (row stride of m2m_df: mp + 1, block: mp rows)
};

// P2M: one CTA per source leaf; thread (set, k).  Sources are staged 32 at a time with their
// charges and the powers u^k of their scaled offsets from the centre.
constexpr int kP2mChunk = 32;
template <typename R>
__global__ void p2m_kernel(FmmDev f, int cell0, double h) {
  using C = cx<R>;
  const int cell = cell0 + blockIdx.x;
  const int2 rg = f.scell_rng[cell];
  const double2 ctr = f.scell_ctr[cell];
  const int p = f.p, p1 = p + 1;
  const int t = threadIdx.x;
  const int set = t / p1, k = t - set * p1;
  // dynamic shared memory (p2m_smem): pw[kP2mChunk][p + 1], then sc[kP2mChunk][kSets]
  extern __shared__ double2 dyn_p2m[];
  C *pw = reinterpret_cast<C *>(dyn_p2m);
  C(*sc)[kSets] = reinterpret_cast<C(*)[kSets]>(pw + kP2mChunk * p1);
  C *M = reinterpret_cast<C *>(f.M);
  C acc = mkc<R>(0.0, 0.0);
  for (int j0 = rg.x; j0 < rg.y; j0 += kP2mChunk) {
    const int nj = min(kP2mChunk, rg.y - j0);
    __syncthreads();
    if (t < nj) {
      const int2 sm = f.src_slot[j0 + t];
      const double2 w = f.src_pos[j0 + t];
      const C u = mkc<R>((w.x - ctr.x) / h, (w.y - ctr.y) / h);
      double2 c[kSets];
      charges(sm.x < f.wall_slots, make_double2(w.x - ctr.x, w.y - ctr.y), f.val[sm.x], c);
#pragma unroll
      for (int s = 0; s < kSets; ++s) sc[t][s] = tocx<R>(c[s]);
      C uk = mkc<R>(1.0, 0.0);
      for (int n = 0; n <= p; ++n) {
        pw[t * p1 + n] = uk;
        uk = cmul(uk, u);
      }
    }
    __syncthreads();
    if (set < kSets)
      for (int j = 0; j < nj; ++j) acc = cfma(sc[j][set], pw[j * p1 + k], acc);
  }
  if (set < kSets) {
    const C v = k == 0 ? acc : cscale(acc, R(-1.0 / k));
    const size_t idx = (size_t(cell) * kSets + set) * p1 + k;
    M[idx] = v;
    if constexpr (sizeof(R) == 8)
      if (f.Mf) f.Mf[idx] = split_c(to_d2(v));
  }
}

// M2M: one CTA per source cell of a level above the leaves; thread (set, q).  The children's
// coefficients, the powers of their offsets and the binomials are staged in shared memory:
// a'_q += -a_0 s^q / q + sum_{k <= q} a_k 2^-k s^(q-k) C(q - 1, k - 1), s = (c_child - c) / h.
// DF (the FP64 evaluations): the shift sums sum_k a_k s^(q-k) C(q - 1, k - 1) 2^-k in
// double-float on the FP32 pipes, the weights from the plan's table of the four child
// quadrants, the children's coefficients split exactly into float pairs; the a_0 term stays
// FP64.  Without DF: the FP32 evaluations.
template <typename R, bool DF = false>
__global__ void m2m_kernel(FmmDev f, int cell0) {
  using C = cx<R>;
  const int cell = cell0 + blockIdx.x;
  const int2 ch = f.scell_rng[cell];
  const double2 ctr = f.scell_ctr[cell];
  const int p = f.p, p1 = p + 1, np = kSets * p1;
  const int t = threadIdx.x;
  const int set = t / p1, q = t - set * p1;
  const int nch = ch.y - ch.x;  // 1..4
  const R inv_q = q > 0 ? R(1.0 / q) : R(0);
  C *M = reinterpret_cast<C *>(f.M);
  // dynamic shared memory (m2m_smem): sa[4][np], sp[4][p + 1], then
  // bm[p * p] = C(q - 1, k - 1) 2^-k at (k - 1) p + q - 1, k = 1..p (consecutive q, consecutive
  // words)
  // (with DF: saf[4][np] the children's coefficients split (re.h, re.l, im.h, im.l) in place
  // of bm, and the quadrant of every child)
  extern __shared__ double2 dyn_m2m[];
  C *sa = reinterpret_cast<C *>(dyn_m2m), *sp = sa + 4 * np;
  R *bm = reinterpret_cast<R *>(sp + 4 * p1);
  float4 *saf = reinterpret_cast<float4 *>(sp + 4 * p1);
  __shared__ int quad[4];
  if constexpr (DF) {
    if (t < nch) {
      const double2 cc = f.scell_ctr[ch.x + t];
      quad[t] = (cc.x > ctr.x ? 1 : 0) + (cc.y > ctr.y ? 2 : 0);
    }
  } else {
    for (int i = t; i < p * p; i += blockDim.x) {
      const int k1 = i / p, qq = i - k1 * p;  // k1 = k - 1, qq = q - 1
      bm[i] = R(c_binom[qq][k1] * ldexp(1.0, -(k1 + 1)));
    }
  }
  for (int i = t; i < nch * np; i += blockDim.x) {
    const int c = i / np, r = i - c * np;
    const double2 cc = f.scell_ctr[ch.x + c];
    const C a = recentred(M, size_t(ch.x + c) * np, r, p1, make_double2(cc.x - ctr.x, cc.y - ctr.y));
    sa[c * np + r] = a;
    if constexpr (DF) {
      const df ar = split_df(double(a.x)), ai = split_df(double(a.y));
      saf[c * np + r] = make_float4(ar.h, ar.l, ai.h, ai.l);
    }
  }
  for (int i = t; i < nch * p1; i += blockDim.x) {
    const int c = i / p1, n = i - c * p1;
    const double2 cc = f.scell_ctr[ch.x + c];
    // the child centre sits a quarter of the parent side away along each axis
    const double2 d = make_double2(cc.x - ctr.x, cc.y - ctr.y);
    const double hp = 4.0 * fabs(d.x);
    sp[c * p1 + n] = tocx<R>(cpow(make_double2(d.x / hp, d.y / hp), n));
  }
  __syncthreads();
  if (set >= kSets) return;
  C acc = mkc<R>(0.0, 0.0);
  for (int c = 0; c < nch; ++c) {
    const C *a = sa + c * np + set * p1;
    const C *spc = sp + c * p1;
    if (q == 0) {
      acc = cadd(acc, a[0]);
    } else {
      C v = cscale(cmul(a[0], spc[q]), -inv_q);
      if constexpr (DF) {
        const float4 *af = saf + c * np + set * p1;
        const float4 *T = f.m2m_df + size_t(quad[c]) * f.mp * (f.mp + 1) + q;
        df vr = {0.0f, 0.0f}, vi = {0.0f, 0.0f};
        for (int k = 1; k <= q; ++k) {
          const float4 w = T[(k - 1) * (f.mp + 1)], ak = af[k];
          df_mul_acc(vr, {ak.x, ak.y}, {w.x, w.y});   // re: a.re w.re - a.im w.im
          df_mul_acc(vr, {-ak.z, -ak.w}, {w.z, w.w});
          df_mul_acc(vi, {ak.x, ak.y}, {w.z, w.w});   // im: a.re w.im + a.im w.re
          df_mul_acc(vi, {ak.z, ak.w}, {w.x, w.y});
          if ((k & 7) == 0) {
            df_renorm(vr);
            df_renorm(vi);
          }
        }
        v = cadd(v, C{R(double(vr.h) + double(vr.l)), R(double(vi.h) + double(vi.l))});
      } else {
        const R *B = bm + (q - 1);
        for (int k = 1; k <= q; ++k) v = cfma(a[k], cscale(spc[q - k], B[(k - 1) * p]), v);
      }
      acc = cadd(acc, v);
    }
  }
  const size_t idx = (size_t(cell) * kSets + set) * p1 + q;
  M[idx] = acc;
  if constexpr (sizeof(R) == 8)
    if (f.Mf) f.Mf[idx] = split_c(to_d2(acc));
}

// L2L from the parent and M2L from the interaction list: one CTA per target cell of one level;
// thread (set, q).  Per source cell the weights w_k = a_k (-1)^k t^-k (w_0 = a_0) are formed once
// in shared memory; then b_0 += a_0 log(-t h) + sum_k w_k and
// b_q += t^-q (sum_k C(q + k - 1, k - 1) w_k - a_0 / q).  Below the roots t is an integer
// offset with |t_x|, |t_y| <= 3, whose powers and log(-t) come from the plan's table.  Source
// cells are staged kM2lBatch at a time.  FP32 evaluations; the FP64 ones use m2l_df_kernel.
constexpr int kM2lBatch = 4;
template <typename R>
__global__ void m2l_kernel(FmmDev f, int cell0, double h, double log_h) {
  using C = cx<R>;
  const int cell = cell0 + blockIdx.x;
  const double2 ct = f.tcell_ctr[cell];
  const int p = f.p, p1 = p + 1, np = kSets * p1;
  const int t = threadIdx.x;
  const int set = t / p1, q = t - set * p1;
  const double inv_h = 1.0 / h;
  const R inv_q = q > 0 ? R(1.0 / q) : R(0);  // no divisions in the loops
  const C *M = reinterpret_cast<const C *>(f.M);
  C *Lc = reinterpret_cast<C *>(f.Lc);
  // dynamic shared memory (m2l_smem): sw[kM2lBatch][np], stq[kM2lBatch][p + 1],
  // slog[kM2lBatch], then bq[p * (p + 1)] = C(q + k - 1, k - 1) at (k - 1) (p + 1) + q, k = 1..p
  // (consecutive q -- the threads of one set -- read consecutive words: no bank conflicts)
  extern __shared__ double2 dyn_m2l[];
  C *sw = reinterpret_cast<C *>(dyn_m2l), *stq = sw + kM2lBatch * np, *slog = stq + kM2lBatch * p1;
  R *bq = reinterpret_cast<R *>(slog + kM2lBatch);
  for (int i = t; i < p1 * p; i += blockDim.x) {
    const int k1 = i / p1, qq = i - k1 * p1;  // k1 = k - 1
    bq[i] = R(c_binom[qq + k1][k1]);
  }
  C acc = mkc<R>(0.0, 0.0);
  const int par = f.tcell_parent[cell];
  if (par >= 0) {  // L2L: stage the parent's locals and the powers of the offset
    const double2 cp = f.tcell_ctr[par];
    const double2 s = make_double2((ct.x - cp.x) * (0.5 * inv_h), (ct.y - cp.y) * (0.5 * inv_h));  // parent side 2h
    for (int i = t; i < np; i += blockDim.x)
      sw[i] = recentred(Lc, size_t(par) * np, i, p1, make_double2(cp.x - ct.x, cp.y - ct.y));
    if (t <= p) stq[t] = tocx<R>(cpow(s, t));
    __syncthreads();
    if (set < kSets) {
      const C *b = sw + set * p1;
      C v = mkc<R>(0.0, 0.0);
      for (int k = q; k <= p; ++k) v = cfma(b[k], cscale(stq[k - q], R(c_binom[k][q])), v);
      acc = cscale(v, R(ldexp(1.0, -q)));
    }
  }
  const int il0 = f.il_off[cell], ne = f.il_off[cell + 1] - il0;
  for (int e0 = 0; e0 < ne; e0 += kM2lBatch) {
    const int nb = min(kM2lBatch, ne - e0);
    __syncthreads();
    for (int i = t; i < nb * np; i += blockDim.x) {
      const int el = i / np, r = i - el * np;
      const int si = r / p1, qi = r - si * p1;
      const int sc = f.il_idx[il0 + e0 + el];
      const double2 cs = f.scell_ctr[sc];
      const double ox = (cs.x - ct.x) * inv_h, oy = (cs.y - ct.y) * inv_h;
      const int dx = __double2int_rn(ox), dy = __double2int_rn(oy);
      const bool tab = abs(dx) <= 3 && abs(dy) <= 3;
      const int ti = (dy + 3) * 7 + (dx + 3);
      // off the table (roots only) the offset is an integer pair as well: use it exactly
      const C T = tocx<R>(tab ? f.tpow[ti * f.tp1 + qi] : cpow(cinv(make_double2(dx, dy)), qi));
      const C a = recentred(M, size_t(sc) * np, r, p1, make_double2(cs.x - ct.x, cs.y - ct.y));
      sw[el * np + r] = qi == 0 ? a : cscale(cmul(a, T), R((qi & 1) ? -1.0 : 1.0));
      if (si == 0) {
        stq[el * p1 + qi] = T;
        if (qi == 0)
          slog[el] = tocx<R>(tab ? f.tlog[ti]
                                 : make_double2(0.5 * log(double(dx) * dx + double(dy) * dy),
                                                atan2(-double(dy), -double(dx))));
      }
    }
    __syncthreads();
    if (set < kSets) {
      const R *B = bq + q;
      for (int el = 0; el < nb; ++el) {
        const C *w = sw + el * np + set * p1;
        R vx = R(0), vy = R(0);
        for (int k = 1; k <= p; ++k) {
          const R bk = B[(k - 1) * p1];
          vx = fma(bk, w[k].x, vx);
          vy = fma(bk, w[k].y, vy);
        }
        if (q == 0)
          acc = cadd(acc, cadd(cmul(w[0], mkc<R>(double(slog[el].x) + log_h, slog[el].y)),
                               C{vx, vy}));
        else
          acc = cfma(C{fma(-w[0].x, inv_q, vx), fma(-w[0].y, inv_q, vy)}, stq[el * p1 + q], acc);
      }
    }
  }
  if (set < kSets) Lc[(size_t(cell) * kSets + set) * p1 + q] = acc;
}

// M2L of FP64 evaluations with every per-interaction operation in double-float on the FP32
// pipes: the weights w_k = a_k (-1)^k t^-k from the double-float copy of the multipoles (Mf) and
// offset powers (tpow_df), the re-centring of sets 2 and 5, the binomial sums and the
// accumulation of b_q += t^-q (sum_k C(q + k - 1, k - 1) w_k - a_0 / q) (b_0: a_0 log(-t h) +
// sum_k w_k).  FP64 is left for the L2L from the parent (once per target cell), the per-source
// offsets (one thread each) and the final write.  Same thread layout and batching as m2l_kernel.
__global__ void m2l_df_kernel(FmmDev f, int cell0, double h, double log_h) {
  const int cell = cell0 + blockIdx.x;
  const double2 ct = f.tcell_ctr[cell];
  const int p = f.p, p1 = p + 1, np = kSets * p1;
  const int t = threadIdx.x;
  const int set = t / p1, q = t - set * p1;
  const double inv_h = 1.0 / h;
  const double2 *Lc64 = f.Lc;
  // dynamic shared memory: swf[kM2lBatch][np], stqf[kM2lBatch][p + 1], bqf[p][p + 1] (float2),
  // then the L2L staging sw[np], sp[p + 1] (double2)
  extern __shared__ double2 dyn_m2l_df[];
  float4 *swf = reinterpret_cast<float4 *>(dyn_m2l_df), *stqf = swf + kM2lBatch * np;
  float2 *bqf = reinterpret_cast<float2 *>(stqf + kM2lBatch * p1);
  double2 *sw = reinterpret_cast<double2 *>(bqf + p * p1 + (p * p1) % 2), *sp = sw + np;
  __shared__ float4 slogf[kM2lBatch], dcf[kM2lBatch];
  __shared__ int sidx[kM2lBatch], tidx[kM2lBatch];
  for (int i = t; i < p1 * p; i += blockDim.x) {
    const int k1 = i / p1, qq = i - k1 * p1;  // k1 = k - 1
    const df b = split_df(c_binom[qq + k1][k1]);
    bqf[i] = make_float2(b.h, b.l);
  }
  double2 acc64 = make_double2(0.0, 0.0);
  const int par = f.tcell_parent[cell];
  if (par >= 0) {  // L2L in FP64 (once per target cell)
    const double2 cp = f.tcell_ctr[par];
    const double2 s = make_double2((ct.x - cp.x) * (0.5 * inv_h), (ct.y - cp.y) * (0.5 * inv_h));
    for (int i = t; i < np; i += blockDim.x)
      sw[i] = recentred(Lc64, size_t(par) * np, i, p1, make_double2(cp.x - ct.x, cp.y - ct.y));
    if (t <= p) sp[t] = cpow(s, t);
    __syncthreads();
    if (set < kSets) {
      const double2 *b = sw + set * p1;
      double2 v = make_double2(0.0, 0.0);
      for (int k = q; k <= p; ++k) v = cfma(b[k], cscale(sp[k - q], c_binom[k][q]), v);
      acc64 = cscale(v, ldexp(1.0, -q));
    }
  }
  const df inv_q = split_df(q > 0 ? 1.0 / q : 0.0);
  dfc acc = {{0.0f, 0.0f}, {0.0f, 0.0f}};
  const int il0 = f.il_off[cell], ne = f.il_off[cell + 1] - il0;
  for (int e0 = 0; e0 < ne; e0 += kM2lBatch) {
    const int nb = min(kM2lBatch, ne - e0);
    __syncthreads();
    if (t < nb) {  // per source cell: the offset, its table row, conj(dc) and log(-t h)
      const int sc = f.il_idx[il0 + e0 + t];
      const double2 cs = f.scell_ctr[sc];
      const double ox = (cs.x - ct.x) * inv_h, oy = (cs.y - ct.y) * inv_h;
      const int dx = __double2int_rn(ox), dy = __double2int_rn(oy);
      const bool tab = abs(dx) <= 3 && abs(dy) <= 3;
      sidx[t] = sc;
      tidx[t] = tab ? (dy + 3) * 7 + (dx + 3) : -1 - ((dy + 64) * 256 + (dx + 64));
      dcf[t] = split_c(make_double2(cs.x - ct.x, -(cs.y - ct.y)));  // conj(c_s - c_t)
      const double2 lg = tab ? f.tlog[(dy + 3) * 7 + (dx + 3)]
                             : make_double2(0.5 * log(double(dx) * dx + double(dy) * dy),
                                            atan2(-double(dy), -double(dx)));
      slogf[t] = split_c(make_double2(lg.x + log_h, lg.y));
    }
    __syncthreads();
    for (int i = t; i < nb * np; i += blockDim.x) {
      const int el = i / np, r = i - el * np;
      const int si = r / p1, qi = r - si * p1;
      const size_t base = size_t(sidx[el]) * np;
      dfc a = dfc_of(f.Mf[base + r]);
      if (si == 2 || si == 5) {  // re-centre to c_t (see recentred())
        dfc b;
        if (si == 2) {
          const dfc a0 = dfc_of(f.Mf[base + qi]), a1 = dfc_of(f.Mf[base + p1 + qi]);
          b = {df_sum(a0.re, df_neg(a1.im)), df_sum(a0.im, a1.re)};  // a0 + i a1
        } else {
          b = dfc_of(f.Mf[base + 4 * p1 + qi]);
        }
        dfc_mul_acc(a, dfc_of(dcf[el]), b);
      }
      const int ti = tidx[el];
      dfc T;
      if (ti >= 0) {
        T = dfc_of(f.tpow_df[ti * f.tp1 + qi]);
      } else {  // off the table (roots only): the integer offset, powers in FP64
        const int code = -1 - ti, dy = code / 256 - 64, dx = code % 256 - 64;
        T = dfc_of(split_c(cpow(cinv(make_double2(dx, dy)), qi)));
      }
      dfc w = a;
      if (qi > 0) {
        w = {{0.0f, 0.0f}, {0.0f, 0.0f}};
        dfc_mul_acc(w, a, T);
        if (qi & 1) w = {df_neg(w.re), df_neg(w.im)};
      }
      swf[el * np + r] = dfc_pack(w);
      if (si == 0) stqf[el * p1 + qi] = dfc_pack(T);
    }
    __syncthreads();
    if (set < kSets) {
      const float2 *Bf = bqf + q;
      for (int el = 0; el < nb; ++el) {
        const float4 *wf = swf + el * np + set * p1;
        dfc v = {{0.0f, 0.0f}, {0.0f, 0.0f}};
        for (int k = 1; k <= p; ++k) {
          const float2 b = Bf[(k - 1) * p1];
          const float4 wk = wf[k];
          df_mul_acc(v.re, {b.x, b.y}, {wk.x, wk.y});
          df_mul_acc(v.im, {b.x, b.y}, {wk.z, wk.w});
          if ((k & 7) == 0) dfc_renorm(v);
        }
        const dfc w0 = dfc_of(wf[0]);
        if (q == 0) {  // b_0 += a_0 log(-t h) + sum_k w_k
          dfc_mul_acc(acc, w0, dfc_of(slogf[el]));
          acc = {df_sum(acc.re, v.re), df_sum(acc.im, v.im)};
        } else {       // b_q += t^-q (sum - a_0 / q)
          df_mul_acc(v.re, df_neg(w0.re), inv_q);
          df_mul_acc(v.im, df_neg(w0.im), inv_q);
          dfc_mul_acc(acc, v, dfc_of(stqf[el * p1 + q]));
        }
        dfc_renorm(acc);
      }
    }
  }
  if (set < kSets)
    f.Lc[(size_t(cell) * kSets + set) * p1 + q] =
        make_double2(acc64.x + (double(acc.re.h) + double(acc.re.l)),
                     acc64.y + (double(acc.im.h) + double(acc.im.l)));
}

// L2P and the near field: one CTA per target leaf, one thread per target (strided).
template <typename R>
__global__ void __launch_bounds__(kLeafThreads) leaf_kernel(FmmDev f, int tcell0, int leaf0,
                                                            double h) {
  using C = cx<R>;
  const int leaf = blockIdx.x;
  const int cell = tcell0 + leaf;
  const double2 ct = f.tcell_ctr[cell];
  const int p = f.p, p1 = p + 1;
  const C *M = reinterpret_cast<const C *>(f.M);
  const C *Lc = reinterpret_cast<const C *>(f.Lc);
  __shared__ C sb[kSets * (kMaxOrder + 1)];
  __shared__ double2 qtot;
  for (int i = threadIdx.x; i < kSets * p1; i += blockDim.x) sb[i] = Lc[size_t(cell) * kSets * p1 + i];
  if (threadIdx.x == 0) {  // stokeslet weight of all sources: the roots' a_0 of q1 and q2
    double2 s = make_double2(0.0, 0.0);
    for (int r = 0; r < f.n_roots_src; ++r) {
      const C *a = M + size_t(f.root_src0 + r) * kSets * p1;
      s.x += double(a[0].x);
      s.y += double(a[p1].x);
    }
    qtot = s;
  }
  __syncthreads();
  const double inv_h = 1.0 / h;
  const int2 trg = f.tleaf_rng[leaf];
  const int nb0 = f.nl_off[leaf0 + leaf], nb1 = f.nl_off[leaf0 + leaf + 1];
  for (int it = trg.x + threadIdx.x; it < trg.y; it += blockDim.x) {
    const int node = f.tgt_node[it];
    // targets past the nodes are the plan's free targets: no own curve (node_curve -1), and
    // their velocity is the pair sum itself (no self terms), written to out_extra
    if (node < f.N ? !f.want_nodes : !f.out_extra) continue;
    const double2 z = f.x[node];
    const int tcur = f.node_curve[node];
    const C u = mkc<R>((z.x - ct.x) * inv_h, (z.y - ct.y) * inv_h);
    // Horner: value, first and second derivative (in u) of every set
    double2 v[kSets], d1[kSets], d2[kSets];
#pragma unroll
    for (int s = 0; s < kSets; ++s) {
      const C *b = sb + s * p1;
      C a0 = b[p], a1 = mkc<R>(0.0, 0.0), a2 = mkc<R>(0.0, 0.0);
      for (int k = p - 1; k >= 0; --k) {
        a2 = cfma(a2, u, a1);
        a1 = cfma(a1, u, a0);
        a0 = cfma(a0, u, b[k]);
      }
      v[s] = to_d2(a0);
      d1[s] = cscale(to_d2(a1), inv_h);
      d2[s] = cscale(to_d2(a2), 2.0 * inv_h * inv_h);
    }
    // near field, directly (coincident pairs skipped); the near stokeslet weight is kept to
    // take it out of Q
    double ux = 0.0, uy = 0.0, qn1 = 0.0, qn2 = 0.0;
    if (f.near32) {  // the same pairs in FP32 arithmetic: differences rounded once from FP64
      for (int e = nb0; e < nb1; ++e) {
        const int2 rg = f.scell_rng[f.nl_idx[e]];
        for (int j = rg.x; j < rg.y; ++j) {
          const int2 sm = f.src_slot[j];
          const double2 w = f.src_pos[j];
          const double4_32a vv = f.val[sm.x];
          const bool wall = sm.x < f.wall_slots;
          if (!wall) {
            qn1 += vv.x;
            qn2 += vv.y;
          }
          const int own = f.src_own[j];
          if (own >= 0 && own == tcur) continue;
          const double d1 = z.x - w.x, d2 = z.y - w.y;
          if (d1 == 0.0 && d2 == 0.0) continue;
          const float r1 = float(d1), r2 = float(d2);
          const float rr = fmaf(r1, r1, r2 * r2);
          const float inv = __frcp_rn(rr);
          if (!wall) {
            const float q1 = float(vv.x), q2 = float(vv.y);
            const float lg = -0.5f * __logf(rr);
            const float c = fmaf(r1, q1, r2 * q2) * inv;
            ux += double(fmaf(lg, q1, c * r1));
            uy += double(fmaf(lg, q2, c * r2));
          } else {
            const float c = fmaf(r1, float(vv.z), r2 * float(vv.w)) *
                            fmaf(r1, float(vv.x), r2 * float(vv.y)) * inv * inv;
            ux += double(c * r1);
            uy += double(c * r2);
          }
        }
      }
    } else {
    for (int e = nb0; e < nb1; ++e) {
      const int2 rg = f.scell_rng[f.nl_idx[e]];
      for (int j = rg.x; j < rg.y; ++j) {
        const int2 sm = f.src_slot[j];
        const double2 w = f.src_pos[j];
        const double4_32a vv = f.val[sm.x];
        const bool wall = sm.x < f.wall_slots;
        if (!wall) {
          qn1 += vv.x;
          qn2 += vv.y;
        }
        // a vesicle's own nodes at m = 0 are the Kress rule's: skipped (own_curve_kernel takes
        // those that lie beyond the neighbour leaves out of the far field)
        const int own = f.src_own[j];
        if (own >= 0 && own == tcur) continue;
        const double r1 = z.x - w.x, r2 = z.y - w.y;
        const double rr = r1 * r1 + r2 * r2;
        if (rr == 0.0) continue;
        const double inv = __drcp_rn(rr);
        if (!wall) {
          const double lg = -0.5 * log(rr);
          const double c = (r1 * vv.x + r2 * vv.y) * inv;
          ux += lg * vv.x + c * r1;
          uy += lg * vv.y + c * r2;
        } else {
          const double c = (r1 * vv.z + r2 * vv.w) * (r1 * vv.x + r2 * vv.y) * inv * inv;
          ux += c * r1;
          uy += c * r2;
        }
      }
    }
    }
    // far field from the local expansion
    const double2 dq = make_double2(d1[0].x - d1[1].y, d1[0].y + d1[1].x);  // Phi'_q1 + i Phi'_q2
    const double2 zo = make_double2(z.x - ct.x, z.y - ct.y);  // sets 2 and 5 are centred at ct
    double2 s = make_double2(-v[0].x + 0.5 * (qtot.x - qn1), -v[1].x + 0.5 * (qtot.y - qn2));
    s = cadd(s, cscale(cadd(cmul(zo, cconj(dq)), cscale(cconj(d1[2]), -1.0)), 0.5));
    const double2 w5 = make_double2(d2[5].x, d2[5].y);
    const double2 zc_d2 = cmul(cconj(zo), d2[4]);
    double2 dl = cadd(d1[4], cconj(d1[3]));
    dl = cadd(dl, cconj(make_double2(w5.x - zc_d2.x, w5.y - zc_d2.y)));
    s = cadd(s, cscale(dl, 0.25));
    if (node < f.N)
      f.out[node] = make_double2(s.x + ux, s.y + uy);
    else
      f.out_extra[node - f.N] = make_double2(s.x + ux, s.y + uy);
  }
}

// Removes the pairs of every vesicle with itself at m = 0 that reached the far field (the Kress
// rule carries them; the near field skips them): pairs whose leaves are not neighbours, found
// with the plan's own binning.  One CTA per vesicle curve, one thread per target node.
struct Binning {
  double x0, y0, hmax;
  int gmaxx, gmaxy, shift;  // level-L leaf = (integer coordinate at depth kLmax) >> shift
};

__device__ __forceinline__ int2 leaf_of(const Binning &bn, double2 q) {
  const int gx = min(bn.gmaxx, max(0, int(floor((q.x - bn.x0) / bn.hmax))));
  const int gy = min(bn.gmaxy, max(0, int(floor((q.y - bn.y0) / bn.hmax))));
  return make_int2(gx >> bn.shift, gy >> bn.shift);
}

constexpr int kOwnMax = 256;  // nodes per vesicle (the step and Kress tables allow at most 256)
template <bool F32>
__global__ void own_curve_kernel(const int *ves_curve_ids, const CurveDev *curves,
                                 const double2 *x, const double *w, const int *node_dens,
                                 const double *slp, double c_slp, Binning bn, double2 *out) {
  const CurveDev cv = curves[ves_curve_ids[blockIdx.x]];
  __shared__ int2 sl[kOwnMax];
  const bool staged = cv.n <= kOwnMax;
  if (staged)
    for (int a = threadIdx.x; a < cv.n; a += blockDim.x) sl[a] = leaf_of(bn, x[cv.node_begin + a]);
  __syncthreads();
  for (int a = threadIdx.x; a < cv.n; a += blockDim.x) {
    const int i = cv.node_begin + a;
    const double2 z = x[i];
    const int2 li = staged ? sl[a] : leaf_of(bn, z);
    double ux = 0.0, uy = 0.0;
    for (int b = 0; b < cv.n; ++b) {
      if (b == a) continue;
      const int j = cv.node_begin + b;
      const int2 lj = staged ? sl[b] : leaf_of(bn, x[j]);
      if (abs(lj.x - li.x) <= 1 && abs(lj.y - li.y) <= 1) continue;  // near: never added
      const int row = node_dens[j];
      const double c = w[j] * c_slp;
      const double q1 = c * slp[2 * row], q2 = c * slp[2 * row + 1];
      const double r1 = z.x - x[j].x, r2 = z.y - x[j].y;
      if constexpr (F32) {  // as the FP32 near field
        if (r1 == 0.0 && r2 == 0.0) continue;
        const float f1 = float(r1), f2 = float(r2), g1 = float(q1), g2 = float(q2);
        const float rr = fmaf(f1, f1, f2 * f2);
        const float lg = -0.5f * __logf(rr);
        const float cc = fmaf(f1, g1, f2 * g2) * __frcp_rn(rr);
        ux += double(fmaf(lg, g1, cc * f1));
        uy += double(fmaf(lg, g2, cc * f2));
        continue;
      }
      const double rr = r1 * r1 + r2 * r2;
      if (rr == 0.0) continue;
      const double lg = -0.5 * log(rr);
      const double cc = (r1 * q1 + r2 * q2) * __drcp_rn(rr);
      ux += lg * q1 + cc * r1;
      uy += lg * q2 + cc * r2;
    }
    out[i] = make_double2(out[i].x - ux, out[i].y - uy);
  }
}

}  // namespace
}  // namespace stokes

// ---------------------------------------------------------------------------
// host plan
// ---------------------------------------------------------------------------
struct stokes_fmm {
  stokes_ctx *ctx = nullptr;
  int p = 20, L = 0, nx = 1, ny = 1, N = 0, n_src = 0;
  int eval_p = 0;  // order of the evaluations (0: p); expansions truncated below the plan's
  bool near32 = false;  // direct pairs (near field, own-curve removal) in FP32 arithmetic
  bool fp32 = false;    // expansions (P2M, M2M, M2L, L2L, L2P) in FP32 arithmetic
  double x0 = 0.0, y0 = 0.0, S = 1.0;
  std::vector<int> sc_off, tc_off;  // [L + 2] first source / target cell of each level
  int n_tleaf = 0;
  // device
  int2 *d_src_slot = nullptr;
  double2 *d_src_pos = nullptr, *d_sc_ctr = nullptr, *d_tc_ctr = nullptr;
  int2 *d_sc_rng = nullptr, *d_tleaf_rng = nullptr;
  int *d_tc_par = nullptr, *d_il_off = nullptr, *d_il_idx = nullptr, *d_nl_off = nullptr,
      *d_nl_idx = nullptr, *d_tgt_node = nullptr;
  double2 *d_M = nullptr, *d_Lc = nullptr;
  double2 *d_tpow = nullptr, *d_tlog = nullptr;  // offset table of the conversions below the roots
  float4 *d_m2m_df = nullptr;  // M2M shift weights per child quadrant, double-float (see m2m_kernel)
  float4 *d_tpow_df = nullptr, *d_Mf = nullptr;  // double-float copies for m2l_df_kernel
  int *d_src_own = nullptr, *d_node_curve = nullptr;
  int n_extra = 0;                // free targets after the nodes
  bool node_targets = true;       // the nodes are targets too (else only the free targets)
  double2 *d_tx = nullptr;        // [N + n_extra] target positions
  // the geometry the plan was made for
  unsigned long long generation = 0;
  std::string err;
  stokes_fmm_info info{};
};

namespace stokes {

// Geometry generation of every context: bumped whenever its geometry is freed (set again or
// destroyed), so a plan knows when it no longer applies.
namespace {
std::mutex g_gen_mu;
std::unordered_map<const stokes_ctx *, unsigned long long> g_gen;
unsigned long long generation_of(const stokes_ctx *c) {
  std::lock_guard<std::mutex> lk(g_gen_mu);
  const auto it = g_gen.find(c);
  return it == g_gen.end() ? 0ull : it->second;
}
}  // namespace

void fmm_geometry_changed(const stokes_ctx *c) {
  std::lock_guard<std::mutex> lk(g_gen_mu);
  ++g_gen[c];
}

// The generation of a context's geometry (plans built for an older one no longer apply).
unsigned long long geometry_generation(const stokes_ctx *c) { return generation_of(c); }

namespace {

constexpr int kLmax = 20;  // depth of the integer coordinates the keys are cut from

unsigned long long spread2(unsigned v) {  // bit b of v -> bit 2b
  unsigned long long x = v & 0xFFFFFu;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}
unsigned compact2(unsigned long long x) {  // inverse of spread2
  x &= 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
  x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
  x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
  return unsigned(x);
}

// Key of the level-l cell (gx, gy) (global integer coordinates at level l): root index above
// the 2l Morton bits of the coordinates within the root.
unsigned long long encode(int gx, int gy, int l, int nx) {
  const unsigned long long root = (unsigned long long)(gy >> l) * nx + (gx >> l);
  const unsigned mask = (1u << l) - 1u;
  return (root << (2 * l)) | spread2(unsigned(gx) & mask) | (spread2(unsigned(gy) & mask) << 1);
}
void decode(unsigned long long key, int l, int nx, int &gx, int &gy) {
  const unsigned long long root = key >> (2 * l);
  const unsigned long long m = key & ((1ull << (2 * l)) - 1ull);
  gx = int((root % nx) << l) | int(compact2(m));
  gy = int((root / nx) << l) | int(compact2(m >> 1));
}

int find_key(const std::vector<unsigned long long> &keys, int b, int e, unsigned long long k) {
  const auto it = std::lower_bound(keys.begin() + b, keys.begin() + e, k);
  return (it != keys.begin() + e && *it == k) ? int(it - keys.begin()) : -1;
}

template <class T>
cudaError_t upload(T *&d, const std::vector<T> &h, size_t &bytes) {
  bytes += sizeof(T) * std::max<size_t>(h.size(), 1);
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&d), sizeof(T) * std::max<size_t>(h.size(), 1));
  if (e != cudaSuccess || h.empty()) return e;
  return cudaMemcpy(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
}

void free_plan(stokes_fmm *f) {
  void *ps[] = {f->d_src_slot, f->d_src_pos, f->d_sc_ctr, f->d_tc_ctr, f->d_sc_rng,
                f->d_tleaf_rng, f->d_tc_par, f->d_il_off, f->d_il_idx, f->d_nl_off,
                f->d_nl_idx, f->d_tgt_node, f->d_M, f->d_Lc, f->d_tpow, f->d_tlog, f->d_src_own, f->d_node_curve,
                f->d_tx,
                f->d_m2m_df, f->d_tpow_df, f->d_Mf};
  for (void *q : ps) cudaFree(q);
}

// The plan on the host: node positions x, FP64 source slot positions and nodes (-1 = padding),
// period d.
struct PlanHost {
  int L = 0, nx = 1, ny = 1, N = 0, ns = 0, n_tleaf = 0;
  double x0 = 0.0, y0 = 0.0, S = 1.0;
  std::vector<int> sc_off, tc_off, tc_par, il_off, il_idx, nl_off, nl_idx, tord;
  std::vector<int2> src_sorted, sc_rng, tleaf_rng;
  std::vector<int> src_own;  // vesicle curve of an m = 0 source (sorted order), else -1
  std::vector<double2> pos_sorted, sc_ctr, tc_ctr;
  long long near_pairs = 0;
};

// Host threads of one plan build (the step builds up to three plans at once).
constexpr int kPlanThreads = 4;

// f(t, begin, end) over `threads` (1..kPlanThreads) contiguous chunks of [0, n), chunk t on
// its own thread (small n on the calling thread alone); every chunk writes only its own
// outputs.
template <class F>
void plan_for(int n, int threads, F f) {
  if (threads <= 1 || n < 4096) {
    f(0, 0, n);
    return;
  }
  std::thread th[kPlanThreads - 1];
  for (int t = 1; t < threads; ++t)
    th[t - 1] = std::thread(f, t, int((long long)n * t / threads), int((long long)n * (t + 1) / threads));
  f(0, 0, int((long long)n / threads));
  for (int t = 1; t < threads; ++t) th[t - 1].join();
}

// The indices 0..n-1 ordered by key[i], equal keys in index order (the order of a stable
// sort): least-significant-digit radix sort of (key, index) pairs, 11 bits per pass, over the
// bits the keys use.
std::vector<int> order_by_key(const std::vector<unsigned long long> &key) {
  const int n = int(key.size());
  constexpr int kBits = 11, kBuckets = 1 << kBits;
  std::vector<unsigned long long> ka(key), kb(n);
  std::vector<int> ia(n), ib(n);
  for (int i = 0; i < n; ++i) ia[i] = i;
  unsigned long long used = 0;
  for (unsigned long long k : key) used |= k;
  std::vector<int> cnt(kBuckets + 1);
  for (int shift = 0; shift < 64 && (used >> shift) != 0; shift += kBits) {
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int i = 0; i < n; ++i) ++cnt[((ka[i] >> shift) & (kBuckets - 1)) + 1];
    for (int b = 0; b < kBuckets; ++b) cnt[b + 1] += cnt[b];
    for (int i = 0; i < n; ++i) {
      const int at = cnt[(ka[i] >> shift) & (kBuckets - 1)]++;
      kb[at] = ka[i];
      ib[at] = ia[i];
    }
    ka.swap(kb);
    ia.swap(ib);
  }
  return ia;
}

void plan_host(const std::vector<double2> &x, const std::vector<double2> &spos,
               const std::vector<int> &snode, const std::vector<int> &node_curve, double d,
               int leaf_target, PlanHost &ph, int threads = kPlanThreads) {
  PlanHost *f = &ph;
  threads = std::max(1, std::min(threads, kPlanThreads));
  const int N = int(x.size());
  const int slots = int(spos.size());
  // image sources
  const int nimg = d != 0.0 ? 3 : 1;
  std::vector<int> live;  // the slots holding a node, in slot order
  live.reserve(slots);
  for (int s = 0; s < slots; ++s)
    if (snode[s] >= 0) live.push_back(s);
  const int nl = int(live.size()), ns = nl * nimg;
  std::vector<int2> src(ns);  // (slot, m): image m of every live slot, m = -1, 0, 1 in turn
  std::vector<double2> pos(ns);
  plan_for(ns, threads, [&](int, int b, int e) {
    for (int j = b; j < e; ++j) {
      const int m = (nimg == 3 ? j / nl - 1 : 0), sl = live[j % nl];
      src[j] = make_int2(sl, m);
      pos[j] = make_double2(spos[sl].x + m * d, spos[sl].y);
    }
  });
  // forest of square roots over sources and targets
  double xa = 1e300, xb = -1e300, ya = 1e300, yb = -1e300;
  for (const double2 &q : pos) {
    xa = std::min(xa, q.x); xb = std::max(xb, q.x); ya = std::min(ya, q.y); yb = std::max(yb, q.y);
  }
  for (const double2 &q : x) {
    xa = std::min(xa, q.x); xb = std::max(xb, q.x); ya = std::min(ya, q.y); yb = std::max(yb, q.y);
  }
  const double W = xb - xa, H = yb - ya;
  double S = std::max({H, W / 64.0, 1e-12 * (1.0 + fabs(xa) + fabs(ya))});
  S *= 1.0 + 1e-9;
  f->nx = std::max(1, int(ceil(W / S * (1.0 - 1e-12))));
  f->ny = std::max(1, int(ceil(H / S * (1.0 - 1e-12))));
  f->x0 = xa;
  f->y0 = ya;
  f->S = S;
  const int gmaxx = (f->nx << kLmax) - 1, gmaxy = (f->ny << kLmax) - 1;
  const double hmax = S / double(1 << kLmax);
  auto gcoord = [&](double2 q, int &gx, int &gy) {
    gx = std::min(gmaxx, std::max(0, int(floor((q.x - xa) / hmax))));
    gy = std::min(gmaxy, std::max(0, int(floor((q.y - ya) / hmax))));
  };
  std::vector<unsigned long long> skey(ns), tkey(N);
  plan_for(ns, threads, [&](int, int b, int e) {
    for (int j = b; j < e; ++j) {
      int gx, gy;
      gcoord(pos[j], gx, gy);
      skey[j] = encode(gx, gy, kLmax, f->nx);
    }
  });
  plan_for(N, threads, [&](int, int b, int e) {
    for (int i = b; i < e; ++i) {
      int gx, gy;
      gcoord(x[i], gx, gy);
      tkey[i] = encode(gx, gy, kLmax, f->nx);
    }
  });
  std::vector<int> sord, tord;  // the two orders, on two threads when threads > 1
  if (threads > 1) {
    std::thread tsort([&] { tord = order_by_key(tkey); });
    sord = order_by_key(skey);
    tsort.join();
  } else {
    sord = order_by_key(skey);
    tord = order_by_key(tkey);
  }
  // depth: the shallowest with at most leaf_target sources per occupied leaf
  int L = 0;
  for (; L < kLmax; ++L) {
    const int sh = 2 * (kLmax - L);
    int occ = 0;
    for (int j = 0; j < ns; ++j)
      if (j == 0 || (skey[sord[j]] >> sh) != (skey[sord[j - 1]] >> sh)) ++occ;
    if (ns <= (long long)leaf_target * occ) break;
  }
  f->L = L;
  const int sh = 2 * (kLmax - L);
  // source leaves and cells of every level (level 0 first)
  std::vector<std::vector<unsigned long long>> skeys(L + 1), tkeys(L + 1);
  std::vector<int> leaf_begin;
  for (int j = 0; j < ns; ++j) {
    const unsigned long long k = skey[sord[j]] >> sh;
    if (skeys[L].empty() || skeys[L].back() != k) {
      skeys[L].push_back(k);
      leaf_begin.push_back(j);
    }
  }
  leaf_begin.push_back(ns);
  for (int l = L - 1; l >= 0; --l)
    for (unsigned long long k : skeys[l + 1])
      if (skeys[l].empty() || skeys[l].back() != (k >> 2)) skeys[l].push_back(k >> 2);
  std::vector<int> tleaf_begin;
  for (int i = 0; i < N; ++i) {
    const unsigned long long k = tkey[tord[i]] >> sh;
    if (tkeys[L].empty() || tkeys[L].back() != k) {
      tkeys[L].push_back(k);
      tleaf_begin.push_back(i);
    }
  }
  tleaf_begin.push_back(N);
  for (int l = L - 1; l >= 0; --l)
    for (unsigned long long k : tkeys[l + 1])
      if (tkeys[l].empty() || tkeys[l].back() != (k >> 2)) tkeys[l].push_back(k >> 2);
  // flatten
  f->sc_off.assign(L + 2, 0);
  f->tc_off.assign(L + 2, 0);
  for (int l = 0; l <= L; ++l) {
    f->sc_off[l + 1] = f->sc_off[l] + int(skeys[l].size());
    f->tc_off[l + 1] = f->tc_off[l] + int(tkeys[l].size());
  }
  std::vector<unsigned long long> sk_all, tk_all;
  for (int l = 0; l <= L; ++l) {
    sk_all.insert(sk_all.end(), skeys[l].begin(), skeys[l].end());
    tk_all.insert(tk_all.end(), tkeys[l].begin(), tkeys[l].end());
  }
  const int nsc = f->sc_off[L + 1], ntc = f->tc_off[L + 1];
  auto centre = [&](unsigned long long k, int l) {
    int gx, gy;
    decode(k, l, f->nx, gx, gy);
    const double h = S / double(1 << l);
    return make_double2(xa + (gx + 0.5) * h, ya + (gy + 0.5) * h);
  };
  // the level of cell i of a flattened list with level offsets off[0..L+1]
  auto level_of = [L](const std::vector<int> &off, int i) {
    return int(std::upper_bound(off.begin(), off.begin() + L + 2, i) - off.begin()) - 1;
  };
  std::vector<double2> sc_ctr(nsc), tc_ctr(ntc);
  std::vector<int2> sc_rng(nsc);
  plan_for(nsc, threads, [&](int, int cb, int ce) {
    for (int i = cb; i < ce; ++i) {
      const int l = level_of(f->sc_off, i);
      sc_ctr[i] = centre(sk_all[i], l);
      if (l == L) {
        const int li = i - f->sc_off[L];
        sc_rng[i] = make_int2(leaf_begin[li], leaf_begin[li + 1]);
      } else {
        const auto b = std::lower_bound(sk_all.begin() + f->sc_off[l + 1], sk_all.begin() + f->sc_off[l + 2],
                                        sk_all[i] << 2);
        const auto e = std::upper_bound(sk_all.begin() + f->sc_off[l + 1], sk_all.begin() + f->sc_off[l + 2],
                                        (sk_all[i] << 2) | 3ull);
        sc_rng[i] = make_int2(int(b - sk_all.begin()), int(e - sk_all.begin()));
      }
    }
  });
  // interaction lists: each chunk of target cells lists into its own part, the parts joined in
  // cell order
  std::vector<int> tc_par(ntc, -1), il_off(ntc + 1, 0), il_idx, il_cnt(ntc, 0);
  std::vector<std::vector<int>> il_part(kPlanThreads);
  plan_for(ntc, threads, [&](int part_id, int cb, int ce) {
    std::vector<int> &part = il_part[part_id];
    for (int i = cb; i < ce; ++i) {
      const int l = level_of(f->tc_off, i);
      const int gnx = f->nx << l, gny = f->ny << l;
      const size_t before = part.size();
      tc_ctr[i] = centre(tk_all[i], l);
      if (l > 0) tc_par[i] = find_key(tk_all, f->tc_off[l - 1], f->tc_off[l], tk_all[i] >> 2);
      int gx, gy;
      decode(tk_all[i], l, f->nx, gx, gy);
      if (l == 0) {
        for (int sidx = f->sc_off[0]; sidx < f->sc_off[1]; ++sidx) {
          int sx, sy;
          decode(sk_all[sidx], 0, f->nx, sx, sy);
          if (std::max(abs(sx - gx), abs(sy - gy)) >= 2) part.push_back(sidx);
        }
      } else {
        const int px = gx >> 1, py = gy >> 1;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx)
            for (int ey = 0; ey < 2; ++ey)
              for (int ex = 0; ex < 2; ++ex) {
                const int cx = 2 * (px + dx) + ex, cy = 2 * (py + dy) + ey;
                if (cx < 0 || cy < 0 || cx >= gnx || cy >= gny) continue;
                if (std::max(abs(cx - gx), abs(cy - gy)) <= 1) continue;
                const int sidx = find_key(sk_all, f->sc_off[l], f->sc_off[l + 1], encode(cx, cy, l, f->nx));
                if (sidx >= 0) part.push_back(sidx);
              }
      }
      il_cnt[i] = int(part.size() - before);
    }
  });
  for (int i = 0; i < ntc; ++i) il_off[i + 1] = il_off[i] + il_cnt[i];
  il_idx.reserve(size_t(il_off[ntc]));
  for (const std::vector<int> &part : il_part) il_idx.insert(il_idx.end(), part.begin(), part.end());
  // near lists and target ranges of the target leaves
  const int ntl = int(tkeys[L].size());
  f->n_tleaf = ntl;
  std::vector<int> nl_off(ntl + 1, 0), nl_idx, nl_cnt(ntl, 0);
  std::vector<int2> tleaf_rng(ntl);
  const int gnx = f->nx << L, gny = f->ny << L;
  std::vector<std::vector<int>> nl_part(kPlanThreads);
  long long part_pairs[kPlanThreads] = {};
  plan_for(ntl, threads, [&](int part_id, int lb, int le) {
    std::vector<int> &part = nl_part[part_id];
    for (int t = lb; t < le; ++t) {
      const size_t before = part.size();
      tleaf_rng[t] = make_int2(tleaf_begin[t], tleaf_begin[t + 1]);
      int gx, gy;
      decode(tkeys[L][t], L, f->nx, gx, gy);
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int cx = gx + dx, cy = gy + dy;
          if (cx < 0 || cy < 0 || cx >= gnx || cy >= gny) continue;
          const int sidx = find_key(sk_all, f->sc_off[L], f->sc_off[L + 1], encode(cx, cy, L, f->nx));
          if (sidx >= 0) {
            part.push_back(sidx);
            part_pairs[part_id] +=
                (long long)(tleaf_begin[t + 1] - tleaf_begin[t]) * (sc_rng[sidx].y - sc_rng[sidx].x);
          }
        }
      nl_cnt[t] = int(part.size() - before);
    }
  });
  long long near_pairs = 0;
  for (long long q : part_pairs) near_pairs += q;
  for (int t = 0; t < ntl; ++t) nl_off[t + 1] = nl_off[t] + nl_cnt[t];
  nl_idx.reserve(size_t(nl_off[ntl]));
  for (const std::vector<int> &part : nl_part) nl_idx.insert(nl_idx.end(), part.begin(), part.end());
  std::vector<int2> src_sorted(ns);
  std::vector<double2> pos_sorted(ns);
  f->src_own.resize(ns);
  plan_for(ns, threads, [&](int, int b, int e) {
    for (int j = b; j < e; ++j) {
      src_sorted[j] = src[sord[j]];
      pos_sorted[j] = pos[sord[j]];
      const int2 sm = src_sorted[j];
      f->src_own[j] = sm.y == 0 ? node_curve[snode[sm.x]] : -1;
    }
  });
  f->N = N;
  f->ns = ns;
  f->tord = tord;
  f->near_pairs = near_pairs;
  ph.sc_rng = sc_rng;
  ph.sc_ctr = sc_ctr;
  ph.tc_ctr = tc_ctr;
  ph.tc_par = tc_par;
  ph.il_off = il_off;
  ph.il_idx = il_idx;
  ph.nl_off = nl_off;
  ph.nl_idx = nl_idx;
  ph.tleaf_rng = tleaf_rng;
  ph.src_sorted = src_sorted;
  ph.pos_sorted = pos_sorted;
}

int build_plan(stokes_fmm *f, int leaf_target, int n_extra, const double2 *extra, bool nodes) {
  stokes_ctx *c = f->ctx;
  const int N = c->N;
  const int slots = c->wall_slots_f64 + c->ves_slots_f64;
  std::vector<double2> x(size_t(N) + n_extra), spos(slots);
  std::vector<int> snode(slots);
  if ((n_extra > 0 && cudaMemcpy(x.data() + N, extra, sizeof(double2) * n_extra,
                                 cudaMemcpyDeviceToHost) != cudaSuccess) ||
      cudaMemcpy(x.data(), c->d_x, sizeof(double2) * N, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(spos.data(), c->d_src_pos64, sizeof(double2) * slots, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(snode.data(), c->d_slot_node64, sizeof(int) * slots, cudaMemcpyDeviceToHost) != cudaSuccess) {
    f->err = "fmm: reading the geometry failed";
    return STOKES_ERR_CUDA;
  }
  for (int i = 0; i < n_extra; ++i)
    if (!isfinite(x[N + i].x) || !isfinite(x[N + i].y)) {
      f->err = "fmm: a free target is not finite";
      return STOKES_ERR_NONFINITE;
    }
  std::vector<int> node_curve(size_t(N) + n_extra, -1);
  for (int cv = 0; cv < c->n_curves; ++cv)
    if (c->kind[cv] == STOKES_KIND_VESICLE)
      for (int i = c->off[cv]; i < c->off[cv + 1]; ++i) node_curve[i] = cv;
  PlanHost ph;
  if (nodes) {
    plan_host(x, spos, snode, node_curve, c->period, leaf_target, ph);
  } else {  // a forest over the sources and the free targets only; targets keep their index N + i
    const std::vector<double2> xt(x.begin() + N, x.end());
    plan_host(xt, spos, snode, node_curve, c->period, leaf_target, ph);
    for (int &t : ph.tord) t += N;
  }
  f->L = ph.L;
  f->nx = ph.nx;
  f->ny = ph.ny;
  f->x0 = ph.x0;
  f->y0 = ph.y0;
  f->S = ph.S;
  f->sc_off = ph.sc_off;
  f->tc_off = ph.tc_off;
  f->n_tleaf = ph.n_tleaf;
  f->N = N;
  f->n_src = ph.ns;
  const int L = ph.L, ns = ph.ns;
  const int nsc = ph.sc_off[L + 1], ntc = ph.tc_off[L + 1];
  const std::vector<int2> &src_sorted = ph.src_sorted, &sc_rng = ph.sc_rng, &tleaf_rng = ph.tleaf_rng;
  const std::vector<double2> &pos_sorted = ph.pos_sorted, &sc_ctr = ph.sc_ctr, &tc_ctr = ph.tc_ctr;
  const std::vector<int> &tc_par = ph.tc_par, &il_off = ph.il_off, &il_idx = ph.il_idx,
                         &nl_off = ph.nl_off, &nl_idx = ph.nl_idx, &tord = ph.tord;
  const long long near_pairs = ph.near_pairs;
  (void)ns;
  size_t bytes = 0;
  cudaError_t e = cudaSuccess;
  auto up = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  up(upload(f->d_src_slot, src_sorted, bytes));
  up(upload(f->d_src_pos, pos_sorted, bytes));
  up(upload(f->d_sc_ctr, sc_ctr, bytes));
  up(upload(f->d_sc_rng, sc_rng, bytes));
  up(upload(f->d_tc_ctr, tc_ctr, bytes));
  up(upload(f->d_tc_par, tc_par, bytes));
  up(upload(f->d_il_off, il_off, bytes));
  up(upload(f->d_il_idx, il_idx, bytes));
  up(upload(f->d_nl_off, nl_off, bytes));
  up(upload(f->d_nl_idx, nl_idx, bytes));
  up(upload(f->d_tgt_node, tord, bytes));
  up(upload(f->d_tleaf_rng, tleaf_rng, bytes));
  up(upload(f->d_src_own, ph.src_own, bytes));
  up(upload(f->d_node_curve, node_curve, bytes));
  up(upload(f->d_tx, x, bytes));
  f->n_extra = n_extra;
  f->node_targets = nodes;
  {  // t^-n and log(-t) of the integer offsets t = (dx, dy), |dx|, |dy| <= 3
    const int p1 = f->p + 1;
    std::vector<double2> tpow(49 * p1), tlog(49);
    for (int dy = -3; dy <= 3; ++dy)
      for (int dx = -3; dx <= 3; ++dx) {
        const int ti = (dy + 3) * 7 + (dx + 3);
        const double r2 = double(dx * dx + dy * dy);
        tlog[ti] = r2 > 0 ? make_double2(0.5 * log(r2), atan2(-double(dy), -double(dx))) : make_double2(0.0, 0.0);
        const double ix = r2 > 0 ? dx / r2 : 0.0, iy = r2 > 0 ? -dy / r2 : 0.0;  // 1 / t
        double px = 1.0, py = 0.0;
        for (int n = 0; n < p1; ++n) {
          tpow[ti * p1 + n] = make_double2(px, py);
          const double nx = px * ix - py * iy, ny = px * iy + py * ix;
          px = nx;
          py = ny;
        }
      }
    up(upload(f->d_tpow, tpow, bytes));
    up(upload(f->d_tlog, tlog, bytes));
    std::vector<float4> tpow_df(tpow.size());
    for (size_t i = 0; i < tpow.size(); ++i) {
      const float rh = float(tpow[i].x), ih = float(tpow[i].y);
      tpow_df[i] = make_float4(rh, float(tpow[i].x - double(rh)), ih, float(tpow[i].y - double(ih)));
    }
    up(upload(f->d_tpow_df, tpow_df, bytes));
  }
  {  // M2M weights s^(q-k) C(q - 1, k - 1) 2^-k for the child offsets s = (+-1 +- i)/4 (quadrant
     // c = [s_x > 0] + 2 [s_y > 0]), 1 <= k <= q <= p, at (c p + k - 1) (p + 1) + q, split into
     // float pairs (re.h, re.l, im.h, im.l)
    const int p = f->p, p1 = p + 1;
    std::vector<double> bn(size_t(p1) * p1, 0.0);  // C(n, k), Pascal's triangle (exact)
    for (int n = 0; n <= p; ++n)
      for (int k = 0; k <= n; ++k)
        bn[n * p1 + k] = (k == 0 || k == n) ? 1.0 : bn[(n - 1) * p1 + k - 1] + bn[(n - 1) * p1 + k];
    std::vector<float4> tab(size_t(4) * p * p1, make_float4(0.f, 0.f, 0.f, 0.f));
    auto split = [](double v, float &h, float &l) {
      h = float(v);
      l = float(v - double(h));
    };
    for (int c = 0; c < 4; ++c) {
      const double sx = (c & 1) ? 0.25 : -0.25, sy = (c & 2) ? 0.25 : -0.25;
      std::vector<double> pr(p1), pi(p1);  // s^n
      pr[0] = 1.0;
      pi[0] = 0.0;
      for (int n = 1; n <= p; ++n) {
        pr[n] = pr[n - 1] * sx - pi[n - 1] * sy;
        pi[n] = pr[n - 1] * sy + pi[n - 1] * sx;
      }
      for (int q = 1; q <= p; ++q)
        for (int k = 1; k <= q; ++k) {
          const double w = bn[(q - 1) * p1 + (k - 1)] * ldexp(1.0, -k);
          float4 &t = tab[(size_t(c) * p + (k - 1)) * p1 + q];
          split(pr[q - k] * w, t.x, t.y);
          split(pi[q - k] * w, t.z, t.w);
        }
    }
    up(upload(f->d_m2m_df, tab, bytes));
  }
  const size_t ne = size_t(kSets) * (f->p + 1);
  up(cudaMalloc(reinterpret_cast<void **>(&f->d_M), sizeof(double2) * ne * std::max(nsc, 1)));
  up(cudaMalloc(reinterpret_cast<void **>(&f->d_Mf), sizeof(float4) * ne * std::max(nsc, 1)));
  up(cudaMalloc(reinterpret_cast<void **>(&f->d_Lc), sizeof(double2) * ne * std::max(ntc, 1)));
  bytes += sizeof(double2) * ne * (nsc + ntc) + sizeof(float4) * ne * nsc;
  if (e != cudaSuccess) {
    f->err = std::string("fmm plan upload: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA;
  }
  f->info.levels = L;
  f->info.sources = ns;
  f->info.source_cells = nsc;
  f->info.target_cells = ntc;
  f->info.m2l_pairs = double(il_idx.size());
  f->info.near_pairs = double(near_pairs);
  f->info.device_bytes = double(bytes);
  return STOKES_OK;
}

}  // namespace
}  // namespace stokes

using namespace stokes;

namespace {

int fmm_fail(stokes_fmm *f, int code, const std::string &msg) {
  if (f) f->err = msg;
  return code;
}

#define FMK(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fmm_fail(f, e_ == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA,  \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

}  // namespace

extern "C" {

static int fmm_create(stokes_ctx *c, int order, int leaf_size, int n_extra, const double *extra,
                      bool nodes, stokes_fmm **out) {
  if (!out) return STOKES_ERR_ARG;
  *out = nullptr;
  if (!c) return STOKES_ERR_ARG;
  if (!c->have_geom) return STOKES_ERR_NO_GEOM;
  if (c->n_inst != 1 || order < 4 || order > kMaxOrder || leaf_size < 4 || leaf_size > 4096 ||
      n_extra < 0 || (n_extra > 0 && !extra) || n_extra > (1 << 26))
    return STOKES_ERR_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return STOKES_ERR_CUDA;
  const auto t0 = std::chrono::steady_clock::now();
  // binomial table (Pascal's triangle; the same on every call)
  std::vector<double> hb(size_t(kBin) * kBin, 0.0);
  for (int n = 0; n < kBin; ++n)
    for (int k = 0; k <= n; ++k)
      hb[n * kBin + k] = (k == 0 || k == n) ? 1.0 : hb[(n - 1) * kBin + k - 1] + hb[(n - 1) * kBin + k];
  if (cudaMemcpyToSymbol(c_binom, hb.data(), sizeof(double) * hb.size()) != cudaSuccess)
    return STOKES_ERR_CUDA;
  stokes_fmm *f = new stokes_fmm();
  f->ctx = c;
  f->p = order;
  const int st = build_plan(f, leaf_size, n_extra, reinterpret_cast<const double2 *>(extra), nodes);
  if (st) {
    c->err = f->err;
    free_plan(f);
    delete f;
    return st;
  }
  f->generation = generation_of(c);
  f->info.order = order;
  f->info.plan_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = f;
  return STOKES_OK;
}

int stokes_fmm_create(stokes_ctx *c, int order, int leaf_size, stokes_fmm **out) {
  return fmm_create(c, order, leaf_size, 0, nullptr, true, out);
}

int stokes_fmm_create_targets(stokes_ctx *c, int order, int leaf_size, int n_targets,
                              const double *targets, stokes_fmm **out) {
  if (n_targets < 1) {
    if (out) *out = nullptr;
    return STOKES_ERR_ARG;
  }
  return fmm_create(c, order, leaf_size, n_targets, targets, true, out);
}

int stokes_fmm_create_targets_only(stokes_ctx *c, int order, int leaf_size, int n_targets,
                                   const double *targets, stokes_fmm **out) {
  if (n_targets < 1) {
    if (out) *out = nullptr;
    return STOKES_ERR_ARG;
  }
  return fmm_create(c, order, leaf_size, n_targets, targets, false, out);
}

// An evaluation: the node sum into out (with the self terms, the curvature diagonal and the
// jump) when out is given, the free targets' velocities into out_targets when given.
static int fmm_eval(stokes_fmm *f, const double *slp, const double *dlp, double jump, double *out,
                    double *out_targets, void *stream) {
  if (!f) return STOKES_ERR_ARG;
  stokes_ctx *c = f->ctx;
  if (!c->have_geom || generation_of(c) != f->generation || c->N != f->N)
    return fmm_fail(f, STOKES_ERR_NO_GEOM, "the context's geometry changed since the plan was made");
  if ((c->n_ves_nodes > 0 && !slp) || (c->n_wall_nodes > 0 && !dlp) || (!out && !out_targets) ||
      (reinterpret_cast<uintptr_t>(out) & 15u) || (reinterpret_cast<uintptr_t>(out_targets) & 15u) ||
      !isfinite(jump))
    return fmm_fail(f, STOKES_ERR_ARG, "need the densities of every kind present, 16-byte aligned "
                                       "outputs and a finite jump");
  if (out_targets && f->n_extra == 0)
    return fmm_fail(f, STOKES_ERR_ARG, "the plan was made without free targets");
  if (out && !f->node_targets)
    return fmm_fail(f, STOKES_ERR_ARG, "the plan was made for its free targets only");
  FMK(cudaSetDevice(c->device));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int N = c->N;
  if (c->partial_cap < size_t(N)) {  // the finishing pass reads one split of partials
    FMK(cudaDeviceSynchronize());
    invalidate_node_graph(c);
    cudaFree(c->d_partial);
    c->d_partial = nullptr;
    c->partial_cap = 0;
    FMK(cudaMalloc(reinterpret_cast<void **>(&c->d_partial), sizeof(double2) * N));
    c->partial_cap = N;
  }
  const bool self = out && c->n_ves_curves > 0;  // the Kress self terms of the node sum
  if (self) {
    FMK(cudaEventRecord(c->ev_fork, s));
    FMK(cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
    FMK(launch_self(c, slp, c->side_stream));
    FMK(cudaEventRecord(c->ev_join, c->side_stream));
  }
  FMK(launch_pack(c, STOKES_FP64, slp, dlp, s));
  FmmDev d;
  const int pe = f->eval_p > 0 ? f->eval_p : f->p;  // every buffer is sized for f->p >= pe
  d.p = pe;
  d.tp1 = f->p + 1;
  d.near32 = f->near32 ? 1 : 0;
  d.m2m_df = f->d_m2m_df;
  d.mp = f->p;
  d.Mf = f->fp32 ? nullptr : f->d_Mf;
  d.tpow_df = f->d_tpow_df;
  d.n_src = f->n_src;
  d.N = N;
  d.want_nodes = out ? 1 : 0;
  d.out_extra = reinterpret_cast<double2 *>(out_targets);
  d.wall_slots = c->wall_slots_f64;
  d.src_slot = f->d_src_slot;
  d.src_pos = f->d_src_pos;
  d.val = c->d_src_val64;
  d.scell_ctr = f->d_sc_ctr;
  d.scell_rng = f->d_sc_rng;
  d.tcell_ctr = f->d_tc_ctr;
  d.tcell_parent = f->d_tc_par;
  d.il_off = f->d_il_off;
  d.il_idx = f->d_il_idx;
  d.nl_off = f->d_nl_off;
  d.nl_idx = f->d_nl_idx;
  d.tgt_node = f->d_tgt_node;
  d.tleaf_rng = f->d_tleaf_rng;
  d.x = f->d_tx;
  d.M = f->d_M;
  d.Lc = f->d_Lc;
  d.out = c->d_partial;
  d.root_src0 = f->sc_off[0];
  d.n_roots_src = f->sc_off[1] - f->sc_off[0];
  d.tpow = f->d_tpow;
  d.tlog = f->d_tlog;
  d.src_own = f->d_src_own;
  d.node_curve = f->d_node_curve;
  const int L = f->L;
  const int nthr = std::max(kLeafThreads, (kSets * (pe + 1) + 31) / 32 * 32);
  auto hl = [&](int l) { return f->S / double(1 << l); };
  const int nleaf_s = f->sc_off[L + 1] - f->sc_off[L];
  const int p1 = pe + 1, np = kSets * p1;
  const size_t cb = f->fp32 ? sizeof(float2) : sizeof(double2), rb = cb / 2;  // complex, real
  const size_t p2m_smem = cb * (kP2mChunk * p1 + kP2mChunk * kSets);
  const size_t m2m_smem = cb * (4 * np + 4 * p1) + rb * pe * pe;
  const size_t m2m_df_smem = sizeof(double2) * (4 * np + 4 * p1) + sizeof(float4) * 4 * np;
  const size_t m2l_smem = cb * (kM2lBatch * np + kM2lBatch * p1 + kM2lBatch) + rb * p1 * pe;
  const size_t m2l_df_smem = sizeof(float4) * (kM2lBatch * np + kM2lBatch * p1) +
                             sizeof(float2) * (size_t(p1) * pe + (size_t(p1) * pe) % 2) +
                             sizeof(double2) * (np + p1);
  auto passes = [&](auto real) {
    using R = decltype(real);
    if (nleaf_s > 0) p2m_kernel<R><<<nleaf_s, nthr, p2m_smem, s>>>(d, f->sc_off[L], hl(L));
    for (int l = L - 1; l >= 0; --l) {
      const int nc = f->sc_off[l + 1] - f->sc_off[l];
      if (nc == 0) continue;
      if constexpr (sizeof(R) == 8)  // FP64 evaluations: shift sums in double-float
        m2m_kernel<double, true><<<nc, nthr, m2m_df_smem, s>>>(d, f->sc_off[l]);
      else
        m2m_kernel<R><<<nc, nthr, m2m_smem, s>>>(d, f->sc_off[l]);
    }
    for (int l = 0; l <= L; ++l) {
      const int nc = f->tc_off[l + 1] - f->tc_off[l];
      if (nc == 0) continue;
      if constexpr (sizeof(R) == 8)  // FP64 evaluations: conversions in double-float
        m2l_df_kernel<<<nc, nthr, m2l_df_smem, s>>>(d, f->tc_off[l], hl(l), log(hl(l)));
      else
        m2l_kernel<R><<<nc, nthr, m2l_smem, s>>>(d, f->tc_off[l], hl(l), log(hl(l)));
    }
    if (f->n_tleaf > 0) leaf_kernel<R><<<f->n_tleaf, kLeafThreads, 0, s>>>(d, f->tc_off[L], 0, hl(L));
  };
  if (f->fp32)
    passes(0.0f);
  else
    passes(0.0);
  if (out && c->n_ves_curves > 0) {
    Binning bn;
    bn.x0 = f->x0;
    bn.y0 = f->y0;
    bn.hmax = f->S / double(1 << kLmax);  // the plan's binning, bit for bit
    bn.gmaxx = (f->nx << kLmax) - 1;
    bn.gmaxy = (f->ny << kLmax) - 1;
    bn.shift = kLmax - L;
    if (f->near32)
      own_curve_kernel<true><<<c->n_ves_curves, 128, 0, s>>>(c->d_ves_curve_ids, c->d_curves, c->d_x,
                                                             c->d_w, c->d_node_dens, slp,
                                                             1.0 / (4.0 * kPiF * c->mu), bn, c->d_partial);
    else
      own_curve_kernel<false><<<c->n_ves_curves, 128, 0, s>>>(c->d_ves_curve_ids, c->d_curves, c->d_x,
                                                              c->d_w, c->d_node_dens, slp,
                                                              1.0 / (4.0 * kPiF * c->mu), bn, c->d_partial);
  }
  FMK(cudaGetLastError());
  if (self) FMK(cudaStreamWaitEvent(s, c->ev_join, 0));
  if (out) FMK(launch_finish_nodes(c, 1, slp, dlp, jump, reinterpret_cast<double2 *>(out), s));
  return STOKES_OK;
}

int stokes_fmm_eval(stokes_fmm *f, const double *slp, const double *dlp, double jump, double *out,
                    void *stream) {
  if (!out) return fmm_fail(f, STOKES_ERR_ARG, "need an output");
  return fmm_eval(f, slp, dlp, jump, out, nullptr, stream);
}

int stokes_fmm_eval_targets(stokes_fmm *f, const double *slp, const double *dlp, double *out_targets,
                            void *stream) {
  if (!out_targets) return fmm_fail(f, STOKES_ERR_ARG, "need an output");
  return fmm_eval(f, slp, dlp, 0.0, nullptr, out_targets, stream);
}


int stokes_fmm_set_eval_order(stokes_fmm *f, int order) {
  if (!f) return STOKES_ERR_ARG;
  if (order != 0 && (order < 4 || order > f->p))
    return fmm_fail(f, STOKES_ERR_ARG, "the evaluation order must be 0 or in [4, the plan's order]");
  f->eval_p = order == f->p ? 0 : order;
  return STOKES_OK;
}

int stokes_fmm_set_precision(stokes_fmm *f, int precision) {
  if (!f) return STOKES_ERR_ARG;
  if (precision != STOKES_FP64 && precision != STOKES_FP32_KAHAN)
    return fmm_fail(f, STOKES_ERR_ARG, "evaluation precision must be STOKES_FP64 or STOKES_FP32_KAHAN");
  f->near32 = f->fp32 = precision == STOKES_FP32_KAHAN;
  return STOKES_OK;
}

int stokes_fmm_get_info(const stokes_fmm *f, stokes_fmm_info *info) {
  if (!f || !info) return STOKES_ERR_ARG;
  *info = f->info;
  return STOKES_OK;
}

int stokes_fmm_last_error(const stokes_fmm *f, char *buf, size_t len) {
  if (!f || !buf || len == 0) return STOKES_ERR_ARG;
  snprintf(buf, len, "%s", f->err.c_str());
  return STOKES_OK;
}

int stokes_fmm_destroy(stokes_fmm *f) {
  if (!f) return STOKES_OK;
  cudaSetDevice(f->ctx->device);
  cudaDeviceSynchronize();
  free_plan(f);
  delete f;
  return STOKES_OK;
}

}  // extern "C"
