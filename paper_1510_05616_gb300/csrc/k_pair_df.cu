// k_pair_df.cu -- the near-image layer-potential pair sum in double-float arithmetic.
//
// The sum is the one of k_pair.cu (stokeslet sources Eq. (S), stresslet sources Eq. (D),
// images m in {-1, 0, +1} of Eq. (Dnr) / Eq. (utotrep), own-curve m = 0 skip, coincident wall
// self pair contributing 0), evaluated on the FP32 pipes to the accuracy of FP64:
//
//  * a real number is an unevaluated pair of floats (h, l) with |l| at most a few ulp of h,
//    ~48 significant bits; sums use the error-free TwoSum / Fast2Sum transformations and
//    products the FMA-based exact product (Dekker / Knuth, as in double-double libraries);
//  * coordinates are split exactly into three floats v = h + m + l on power-of-two grids
//    g_h and g_m = g_h 2^-24 (h, m, l from the FP64 value by rounding to the grids; every
//    part is exactly representable), so that h_t - h_s and m_t - m_s are exact float
//    differences and r = x - y is known to ~2^-48 |r| even for adjacent wall nodes, where
//    r . n ~ kappa r^2 / 2 carries the stresslet;
//  * 1/r^2 from the MUFU approximation refined by one Newton step in double-float;
//  * the three images of one stokeslet source share a single logarithm:
//    sum_m log r_m^2 = log(r_-1^2 r_0^2 r_1^2); the logarithm is table-driven:
//    x = 2^e m, a_k = 1 + (k + 1/2)/128 from the top 7 fraction bits, u = (m - a_k)/a_k,
//    log x = e ln 2 + log a_k + log1p(u) with |u| <= 2^-8 and log1p by its series to u^6,
//    the (e ln 2) and (1/a_k, log a_k) tables in double-float (built in FP64 once);
//  * each source tile (64 sources, three images) is summed into a fresh double-float
//    accumulator per target (TwoSum of the high parts, the low parts and rounding errors
//    summed separately, renormalised after every source), and the tile sums are added into
//    FP64 accumulators: a double-float accumulator carried over ~10^6 additions would lose
//    ~sqrt(n) 2^-48 of its value, the FP64 one loses ~sqrt(tiles) 2^-53.  The FP64 partials
//    are reduced across splits in FP64 by the same finishing kernels as the other paths.
//
// Tiling and pipeline as the FP64 path: 64-source tiles in the FP64 slot layout, staged by
// cp.async.bulk into a 3-stage mbarrier ring with bounded waits; 64 threads x 2 targets, the
// two targets of a thread evaluated together by packed .f32x2 arithmetic (one instruction
// for both; the MUFU approximation and the logarithm's bit work and tables per target).
#include <algorithm>

#include "df.cuh"
#include "stokes_internal.cuh"
#include "bulk_pipe.cuh"

namespace stokes {

// ---------------------------------------------------------------------------
// double-float primitives beyond df.cuh's (the _rn intrinsics keep the compiler from
// contracting or reassociating the error-free transformations)
// ---------------------------------------------------------------------------
// (a.h + a.l)(b.h + b.l) without the l*l term; unnormalised result.
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return {p, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.h, b.h);
  return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}

// Sum of two non-negative values (squares): Fast2Sum after ordering.
__device__ __forceinline__ df df_add_pos(df a, df b) {
  const float big = fmaxf(a.h, b.h), sml = fminf(a.h, b.h);
  const df s = fast_two_sum(big, sml);
  return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ df df_sq(df a) {
  const float p = __fmul_rn(a.h, a.h);
  float e = __fmaf_rn(a.h, a.h, -p);
  e = __fmaf_rn(__fadd_rn(a.h, a.h), a.l, e);
  return {p, e};
}

// 1/a for a > 0: the MUFU estimate y0 and one Newton step, e = 1 - a y0 (error ~2^-23),
// 1/a = y0 (1 + e + e^2 + ...).  `floor` keeps y0 finite for a == 0 (coincident wall pair).
__device__ __forceinline__ df df_rcp(df a) {
  const float y0 = rcp_approx(fmaxf(a.h, 1e-30f));
  float e = __fmaf_rn(-a.h, y0, 1.0f);
  e = __fmaf_rn(-a.l, y0, e);
  return {y0, __fmul_rn(y0, __fmaf_rn(e, e, e))};
}

// v = h + m + l on the grids g_h, g_m (powers of two): h and m are exact floats while
// |v| <= 2^23 g_h; l is the (tiny) rest, rounded.
__device__ __forceinline__ float3 split3(double v, double g_h, double g_m) {
  const double h = rint(v / g_h) * g_h;
  const double r = v - h;
  const double m = rint(r / g_m) * g_m;
  return make_float3(__double2float_rn(h), __double2float_rn(m), __double2float_rn(r - m));
}

// r = t - s from three-part coordinates: h_t - h_s and m_t - m_s are exact, their sum is
// split exactly by Fast2Sum (|A| >= g_h >= |B| unless A == 0).
__device__ __forceinline__ df diff3(float th, float tm, float tl, float sh, float sm, float sl) {
  const float A = __fsub_rn(th, sh);
  const float B = __fsub_rn(tm, sm);
  const float C = __fsub_rn(tl, sl);
  const df s = fast_two_sum(A, B);
  return {s.h, __fadd_rn(s.l, C)};
}

// ---------------------------------------------------------------------------
// per-context constants
// ---------------------------------------------------------------------------
__global__ void df_init_kernel(DFConst *d) {
  const int k = threadIdx.x;
  if (k < 128) {
    const double a = 1.0 + (k + 0.5) / 128.0;
    const df ia = split_df(1.0 / a), la = split_df(log(a));
    d->kt[k] = make_float4(ia.h, ia.l, la.h, la.l);
  }
  if (k < 256) {
    // (e - 127) ln 2 with ln 2 in two parts, so the product is formed to ~2^-90
    const double ln2_hi = 0.693147180559945286226764;   // nearest double to ln 2
    const double ln2_lo = 2.319046813846299558e-17;     // ln 2 - ln2_hi
    const double e = double(k - 127);
    const double hi = e * ln2_hi;
    const double lo = fma(e, ln2_hi, -hi) + e * ln2_lo;
    const float h = __double2float_rn(hi + lo);
    d->et[k] = make_float2(h, __double2float_rn((hi - double(h)) + lo));
  }
  if (k == 0) d->maxabs_bits = 0u;
}

// maxabs_bits = float bits of an upper bound of max(|x|, |y|) + |period| over the nodes
// (positive floats order like their bit patterns).
__global__ void df_maxabs_kernel(int n, const double2 *x, double period, DFConst *d) {
  float m = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 p = x[i];
    m = fmaxf(m, __double2float_ru(fmax(fabs(p.x) + fabs(period), fabs(p.y))));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&d->maxabs_bits, __float_as_uint(m));
}

// g_h = 2^(ceil(log2(2 M)) - 24): h_t - h_s, |.| <= 2M, is an integer multiple of g_h below
// 2^24, hence an exact float; g_m = g_h 2^-24.
__global__ void df_grid_kernel(DFConst *d) {
  const double M = fmax(double(__uint_as_float(d->maxabs_bits)), 1e-30);
  int ex;
  frexp(2.0 * M, &ex);  // 2M <= 2^ex
  d->g_h = ldexp(1.0, ex - 24);
  d->g_m = ldexp(1.0, ex - 48);
}

// Source positions in the FP64 slot layout: pos[2s] = (x_h, x_m, x_l, y_h),
// pos[2s+1] = (y_m, y_l, 0, 0).
__global__ void src_pos_df_kernel(int slots, const int *slot_node, const double2 *x,
                                  const DFConst *d, float4 *pos) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= slots) return;
  const int i = slot_node[s];
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
  if (i >= 0) {
    const double2 p = x[i];
    const float3 X = split3(p.x, d->g_h, d->g_m), Y = split3(p.y, d->g_h, d->g_m);
    a = make_float4(X.x, X.y, X.z, Y.x);
    b = make_float4(Y.y, Y.z, 0.f, 0.f);
  }
  pos[2 * s] = a;
  pos[2 * s + 1] = b;
}

// Source values: stokeslet val[2s] = (q1 h, l, q2 h, l), val[2s+1] = (p1 h, l, p2 h, l) with
// q = w f / (4 pi mu), p = -q/2; stresslet val[2s] = q = w tau / pi, val[2s+1] = normal.
__global__ void pack_df_kernel(int slots, int wall_slots, const int *slot_node,
                               const int *node_dens, const double *w, const double2 *nrm,
                               const double *slp, const double *dlp, double c_slp,
                               unsigned *status, float4 *val, int N, int n_slp_rows,
                               int n_dlp_rows) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= slots) return;
  const int i = slot_node[s];
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
  // node and density row bounds-checked in the debug build (out of range: a dummy slot)
  const int row = (i >= 0 && dcheck(i < N, status)) ? node_dens[i] : -1;
  if (row >= 0 && dcheck(row < (s < wall_slots ? n_dlp_rows : n_slp_rows), status)) {
    if (s < wall_slots) {
      const double t1 = dlp[2 * row], t2 = dlp[2 * row + 1];
      if (!isfinite(t1) || !isfinite(t2)) atomicOr(status, kStatusNonfinite);
      const double c = w[i] / kPi;
      const df q1 = split_df(c * t1), q2 = split_df(c * t2);
      const double2 n = nrm[i];
      const df n1 = split_df(n.x), n2 = split_df(n.y);
      a = make_float4(q1.h, q1.l, q2.h, q2.l);
      b = make_float4(n1.h, n1.l, n2.h, n2.l);
    } else {
      const double f1 = slp[2 * row], f2 = slp[2 * row + 1];
      if (!isfinite(f1) || !isfinite(f2)) atomicOr(status, kStatusNonfinite);
      const double c = w[i] * c_slp;
      const df q1 = split_df(c * f1), q2 = split_df(c * f2);
      a = make_float4(q1.h, q1.l, q2.h, q2.l);
      b = make_float4(-0.5f * q1.h, -0.5f * q1.l, -0.5f * q2.h, -0.5f * q2.l);
    }
  }
  val[2 * s] = a;
  val[2 * s + 1] = b;
}

// ---------------------------------------------------------------------------
// double-float natural logarithm of P > 0 (normal float high part)
// ---------------------------------------------------------------------------
__device__ __forceinline__ df df_log(df P, const float4 *kt, const float2 *et) {
  const df Q = fast_two_sum(P.h, P.l);             // |Q.l| <= ulp(Q.h) / 2
  const unsigned bits = __float_as_uint(Q.h);
  const unsigned eb = bits >> 23;                  // biased exponent
  const float2 E = et[eb];                         // (eb - 127) ln 2
  const float4 T = kt[(bits >> 16) & 127u];        // 1/a_k, log a_k
  const float m = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
  const float a = __uint_as_float((bits & 0x007F0000u) | 0x3F808000u);  // a_k
  const float d = __fsub_rn(m, a);                 // exact
  const float corr = __fmul_rn(Q.l, __uint_as_float((254u - eb) << 23));  // Q.l 2^-e, exact
  // u = (d + corr) / a_k in double-float, |u| <= 2^-8
  const float uh = __fmul_rn(d, T.x);
  float ue = __fmaf_rn(d, T.x, -uh);
  ue = __fmaf_rn(d, T.y, ue);
  ue = __fmaf_rn(corr, T.x, ue);
  // log1p(u) = u - u^2/2 + u^3 (1/3 - u/4 + u^2/5 - u^3/6) + O(u^7)
  const float sq = __fmul_rn(uh, uh);
  float sqe = __fmaf_rn(uh, uh, -sq);
  sqe = __fmaf_rn(__fadd_rn(uh, uh), ue, sqe);
  float p = __fmaf_rn(uh, -1.0f / 6.0f, 0.2f);
  p = __fmaf_rn(p, uh, -0.25f);
  p = __fmaf_rn(p, uh, 1.0f / 3.0f);
  const float tail = __fmul_rn(__fmul_rn(sq, uh), p);
  const df s = fast_two_sum(E.x, T.z);             // |e ln 2| >= log a_k unless e == 0
  const df v = fast_two_sum(uh, -0.5f * sq);       // |u| >= u^2 / 2
  const df w = two_sum(s.h, v.h);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(s.l, v.l), w.l),
                             __fadd_rn(__fadd_rn(E.y, T.w), __fadd_rn(__fmaf_rn(-0.5f, sqe, ue), tail)));
  return {w.h, lo};
}

// ---------------------------------------------------------------------------
// pair evaluation
// ---------------------------------------------------------------------------
template <int NIMG>
struct TgtDF {
  float xh[NIMG], xm[NIMG], xl[NIMG];  // x - m d, three parts
  float yh, ym, yl;
  int2 skip;
};

template <int NIMG>
__device__ __forceinline__ void load_target_df(const PairArgs &a, double period, int i,
                                               TgtDF<NIMG> &t) {
  if (!dcheck(i >= 0 && i < a.n_targets, a.status)) i = 0;
  const double2 p = a.tgt[i];
  const double g_h = a.dfc->g_h, g_m = a.dfc->g_m;
#pragma unroll
  for (int k = 0; k < NIMG; ++k) {
    const double m = (NIMG == 3) ? double(k - 1) : 0.0;
    const float3 X = split3(p.x - m * period, g_h, g_m);
    t.xh[k] = X.x;
    t.xm[k] = X.y;
    t.xl[k] = X.z;
  }
  const float3 Y = split3(p.y, g_h, g_m);
  t.yh = Y.x;
  t.ym = Y.y;
  t.yl = Y.z;
  t.skip = a.tgt_skip ? a.tgt_skip[i] : make_int2(-1, -1);
}

// ---------------------------------------------------------------------------
// packed double-float arithmetic: the two targets of a thread in the two halves of .f32x2
// registers, one instruction for both (the MUFU approximation, the logarithm's bit work and
// table lookups stay per target)
// ---------------------------------------------------------------------------
typedef unsigned long long f2;  // two floats, the first target in the low word

__device__ __forceinline__ f2 pk(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ f2 bc(float a) { return pk(a, a); }
__device__ __forceinline__ void upk(f2 v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// -a (sign bits flipped on the integer pipe)
__device__ __forceinline__ f2 neg2(f2 a) { return a ^ 0x8000000080000000ull; }

struct df2 {
  f2 h, l;
};

__device__ __forceinline__ df2 two_sum2(f2 a, f2 b) {
  const f2 s = add2(a, b);
  const f2 bb = sub2(s, a);
  return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
// Exact when |a| >= |b| (or a == 0), per half.
__device__ __forceinline__ df2 fast_two_sum2(f2 a, f2 b) {
  const f2 s = add2(a, b);
  return {s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ df2 df_mul2(df2 a, df2 b) {
  const f2 p = mul2(a.h, b.h);
  f2 e = fma2(a.h, b.h, neg2(p));
  e = fma2(a.h, b.l, e);
  e = fma2(a.l, b.h, e);
  return {p, e};
}
__device__ __forceinline__ df2 df_add2(df2 a, df2 b) {
  const df2 s = two_sum2(a.h, b.h);
  return {s.h, add2(s.l, add2(a.l, b.l))};
}
__device__ __forceinline__ df2 df_sq2(df2 a) {
  const f2 p = mul2(a.h, a.h);
  f2 e = fma2(a.h, a.h, neg2(p));
  e = fma2(add2(a.h, a.h), a.l, e);
  return {p, e};
}
// 1/a for a > 0 per half, as df_rcp.
__device__ __forceinline__ df2 df_rcp2(df2 a) {
  float h0, h1;
  upk(a.h, h0, h1);
  const f2 y0 = pk(rcp_approx(fmaxf(h0, 1e-30f)), rcp_approx(fmaxf(h1, 1e-30f)));
  f2 e = fma2(neg2(a.h), y0, bc(1.0f));
  e = fma2(neg2(a.l), y0, e);
  return {y0, mul2(y0, fma2(e, e, e))};
}
__device__ __forceinline__ void df_mul_acc2(df2 &acc, df2 a, df2 b) {
  const f2 p = mul2(a.h, b.h);
  f2 e = fma2(a.h, b.h, neg2(p));
  e = fma2(a.h, b.l, e);
  e = fma2(a.l, b.h, e);
  const df2 s = two_sum2(acc.h, p);
  acc.h = s.h;
  acc.l = add2(acc.l, add2(s.l, e));
}
__device__ __forceinline__ void df_renorm2(df2 &a) { a = fast_two_sum2(a.h, a.l); }
// r = t - s from three-part coordinates (as diff3), targets packed, source broadcast.
__device__ __forceinline__ df2 diff3_2(f2 th, f2 tm, f2 tl, float sh, float sm, float sl) {
  const f2 A = sub2(th, bc(sh));
  const f2 B = sub2(tm, bc(sm));
  const f2 C = sub2(tl, bc(sl));
  const df2 s = fast_two_sum2(A, B);
  return {s.h, add2(s.l, C)};
}
__device__ __forceinline__ df2 df_log2(df2 P, const float4 *kt, const float2 *et) {
  float h0, h1, l0, l1;
  upk(P.h, h0, h1);
  upk(P.l, l0, l1);
  const df a = df_log(df{h0, l0}, kt, et), b = df_log(df{h1, l1}, kt, et);
  return {pk(a.h, b.h), pk(a.l, b.l)};
}
// per-half select: where the flag is set, take the replacement
__device__ __forceinline__ f2 sel2(f2 v, bool s0, bool s1, float r) {
  float a, b;
  upk(v, a, b);
  return pk(s0 ? r : a, s1 ? r : b);
}

// Two targets, packed: (x - m d) in three parts per image, y in three parts.
template <int NIMG>
struct TgtDF2 {
  f2 xh[NIMG], xm[NIMG], xl[NIMG];
  f2 yh, ym, yl;
};

template <int NIMG>
__device__ __forceinline__ TgtDF2<NIMG> pack_targets_df(const TgtDF<NIMG> &a, const TgtDF<NIMG> &b) {
  TgtDF2<NIMG> t;
#pragma unroll
  for (int k = 0; k < NIMG; ++k) {
    t.xh[k] = pk(a.xh[k], b.xh[k]);
    t.xm[k] = pk(a.xm[k], b.xm[k]);
    t.xl[k] = pk(a.xl[k], b.xl[k]);
  }
  t.yh = pk(a.yh, b.yh);
  t.ym = pk(a.ym, b.ym);
  t.yl = pk(a.yl, b.yl);
  return t;
}

// Stokeslet source (Eq. (S)) against two targets: adds, over the images, -(1/2) q log r^2 +
// r (r . q) / r^2 with q = w f / (4 pi mu); one logarithm of the product of the images' r^2
// per target.  pa, pb: position record; va = q, vb = p = -q/2.  MASK0 drops the m = 0 image
// of a target whose flag (s0, s1) is set (its r^2 enters the product as 1).
template <int NIMG, bool MASK0>
__device__ __forceinline__ void slp_source_df2(const TgtDF2<NIMG> &t, float4 pa, float4 pb,
                                               float4 va, float4 vb, bool s0, bool s1, df2 &ax,
                                               df2 &ay, const float4 *kt, const float2 *et) {
  const df2 dy = diff3_2(t.yh, t.ym, t.yl, pa.w, pb.x, pb.y);
  const df2 q1{bc(va.x), bc(va.y)}, q2{bc(va.z), bc(va.w)}, p1{bc(vb.x), bc(vb.y)},
      p2{bc(vb.z), bc(vb.w)};
  const df2 dyq = df_mul2(dy, q2);
  const df2 py = df_sq2(dy);
  df2 dx[NIMG], inv[NIMG], P;
#pragma unroll
  for (int k = 0; k < NIMG; ++k) {
    dx[k] = diff3_2(t.xh[k], t.xm[k], t.xl[k], pa.x, pa.y, pa.z);
    const df2 sq = df_sq2(dx[k]);
    const df2 sh = two_sum2(sq.h, py.h);
    df2 r2{sh.h, add2(sh.l, add2(sq.l, py.l))};
    if (MASK0 && k == NIMG / 2 && (s0 || s1)) r2 = {sel2(r2.h, s0, s1, 1.0f), sel2(r2.l, s0, s1, 0.0f)};
    inv[k] = df_rcp2(r2);
    P = (k == 0) ? r2 : df_mul2(P, r2);
  }
  const df2 L = df_log2(P, kt, et);
  df_mul_acc2(ax, L, p1);
  df_mul_acc2(ay, L, p2);
  df2 cs;
#pragma unroll
  for (int k = 0; k < NIMG; ++k) {
    df2 coef = df_mul2(df_add2(df_mul2(dx[k], q1), dyq), inv[k]);
    if (MASK0 && k == NIMG / 2 && (s0 || s1))
      coef = {sel2(coef.h, s0, s1, 0.0f), sel2(coef.l, s0, s1, 0.0f)};
    df_mul_acc2(ax, coef, dx[k]);
    cs = (k == 0) ? coef : df_add2(cs, coef);
  }
  df_mul_acc2(ay, cs, dy);
  df_renorm2(ax);
  df_renorm2(ay);
}

// Stresslet source (Eq. (D)) against two targets: adds, over the images,
// r (r . n)(r . q) / r^4, q = w tau / pi.  va = q, vb = n.  The coincident wall self pair has
// r = 0 exactly and adds 0.
template <int NIMG>
__device__ __forceinline__ void dlp_source_df2(const TgtDF2<NIMG> &t, float4 pa, float4 pb,
                                               float4 va, float4 vb, df2 &ax, df2 &ay) {
  const df2 dy = diff3_2(t.yh, t.ym, t.yl, pa.w, pb.x, pb.y);
  const df2 q1{bc(va.x), bc(va.y)}, q2{bc(va.z), bc(va.w)}, n1{bc(vb.x), bc(vb.y)},
      n2{bc(vb.z), bc(vb.w)};
  const df2 dyn = df_mul2(dy, n2), dyq = df_mul2(dy, q2);
  const df2 py = df_sq2(dy);
  df2 fs;
#pragma unroll
  for (int k = 0; k < NIMG; ++k) {
    const df2 dx = diff3_2(t.xh[k], t.xm[k], t.xl[k], pa.x, pa.y, pa.z);
    const df2 sq = df_sq2(dx);
    const df2 sh = two_sum2(sq.h, py.h);
    const df2 inv = df_rcp2({sh.h, add2(sh.l, add2(sq.l, py.l))});
    const df2 rn = df_add2(df_mul2(dx, n1), dyn);
    const df2 rq = df_add2(df_mul2(dx, q1), dyq);
    const df2 f = df_mul2(df_mul2(rn, inv), df_mul2(rq, inv));
    df_mul_acc2(ax, f, dx);
    fs = (k == 0) ? f : df_add2(fs, f);
  }
  df_mul_acc2(ay, fs, dy);
  df_renorm2(ax);
  df_renorm2(ay);
}

struct SmemDF {
  __align__(128) float4 pos[kStages][2 * kTileF64];
  __align__(128) float4 val[kStages][2 * kTileF64];
  float4 kt[128];
  float2 et[256];
  __align__(8) uint64_t bar[kStages];
};

__device__ __forceinline__ void load_tables_df(const DFConst *d, SmemDF &sm) {
  for (int k = threadIdx.x; k < 128; k += blockDim.x) sm.kt[k] = d->kt[k];
  for (int k = threadIdx.x; k < 256; k += blockDim.x) sm.et[k] = d->et[k];
}

// Source tile of a staged copy: the item's virtual tile vt, bounds-checked in the debug build
// (out of range: recorded in the status word and redirected to tile 0).
__device__ __forceinline__ int item_tile_df(const PairArgs &a, const ItemDesc &it, int vt) {
  const int tile = vt < it.nw ? it.wb + vt : it.vb + (vt - it.nw);
  return dcheck(tile >= 0 && tile < a.src_tiles, a.status) ? tile : 0;
}

// One work item (as run_item_f64): targets [tgt_begin, +tgt_count), two per thread, against
// virtual tiles [vt_begin, vt_end); `g` counts tiles consumed so far (stage and parity).
template <int NIMG>
__device__ __forceinline__ bool run_item_df(const PairArgs &a, const ItemDesc &it, SmemDF &sm,
                                            uint32_t &g) {
  const int ntl = it.vt_end - it.vt_begin;
  TgtDF<NIMG> tg[kTptDF];
  double ux[kTptDF], uy[kTptDF];  // FP64 sums of the per-tile double-float sums
#pragma unroll
  for (int q = 0; q < kTptDF; ++q) {
    const int loc = min(q * kThreadsDF + int(threadIdx.x), it.tgt_count - 1);
    load_target_df<NIMG>(a, it.period, it.tgt_begin + loc, tg[q]);
    ux[q] = uy[q] = 0.0;
  }
  const float4 *gpos = static_cast<const float4 *>(a.src_pos);
  const float4 *gval = static_cast<const float4 *>(a.src_val);
  constexpr uint32_t kBytes = 2 * kTileF64 * sizeof(float4);

  if (threadIdx.x == 0) {
    for (int r = 0; r < kStages && r < ntl; ++r) {
      const int st = (g + r) % kStages;
      const int tile = item_tile_df(a, it, it.vt_begin + r);
      mbar_arrive_expect_tx(&sm.bar[st], 2 * kBytes);
      bulk_g2s(sm.pos[st], gpos + size_t(tile) * 2 * kTileF64, kBytes, &sm.bar[st]);
      bulk_g2s(sm.val[st], gval + size_t(tile) * 2 * kTileF64, kBytes, &sm.bar[st]);
    }
  }
  for (int r = 0; r < ntl; ++r) {
    const uint32_t gr = g + r;
    const int st = gr % kStages;
    const bool ok = mbar_wait_bounded(&sm.bar[st], (gr / kStages) & 1u);
    if (ok) {
      const int vt = it.vt_begin + r;
      const int tile = item_tile_df(a, it, vt);
      const float4 *P = sm.pos[st];
      const float4 *V = sm.val[st];
      static_assert(kTptDF == 2, "the packed double-float kernel takes two targets per thread");
      const TgtDF2<NIMG> tp = pack_targets_df<NIMG>(tg[0], tg[1]);
      df2 ax2{0ull, 0ull}, ay2{0ull, 0ull};
      if (vt < it.nw) {
#pragma unroll 1
        for (int j = 0; j < kTileF64; ++j) {
          const float4 pa = P[2 * j], pb = P[2 * j + 1], va = V[2 * j], vb = V[2 * j + 1];
          dlp_source_df2<NIMG>(tp, pa, pb, va, vb, ax2, ay2);
        }
      } else {
        const int slot0 = tile * kTileF64;
        bool mine = false;
#pragma unroll
        for (int q = 0; q < kTptDF; ++q)
          mine |= (tg[q].skip.x < slot0 + kTileF64) && (tg[q].skip.y > slot0);
        if (__any_sync(0xffffffffu, mine)) {
#pragma unroll 1
          for (int j = 0; j < kTileF64; ++j) {
            const float4 pa = P[2 * j], pb = P[2 * j + 1], va = V[2 * j], vb = V[2 * j + 1];
            const bool s0 = (slot0 + j >= tg[0].skip.x) && (slot0 + j < tg[0].skip.y);
            const bool s1 = (slot0 + j >= tg[1].skip.x) && (slot0 + j < tg[1].skip.y);
            slp_source_df2<NIMG, true>(tp, pa, pb, va, vb, s0, s1, ax2, ay2, sm.kt, sm.et);
          }
        } else {
#pragma unroll 1
          for (int j = 0; j < kTileF64; ++j) {
            const float4 pa = P[2 * j], pb = P[2 * j + 1], va = V[2 * j], vb = V[2 * j + 1];
            slp_source_df2<NIMG, false>(tp, pa, pb, va, vb, false, false, ax2, ay2, sm.kt, sm.et);
          }
        }
      }
      df ax[kTptDF], ay[kTptDF];
      upk(ax2.h, ax[0].h, ax[1].h);
      upk(ax2.l, ax[0].l, ax[1].l);
      upk(ay2.h, ay[0].h, ay[1].h);
      upk(ay2.l, ay[0].l, ay[1].l);
#pragma unroll
      for (int q = 0; q < kTptDF; ++q) {
        ux[q] += double(ax[q].h) + double(ax[q].l);
        uy[q] += double(ay[q].h) + double(ay[q].l);
      }
    }
    if (__syncthreads_or(!ok)) {
      // A stage never arrived: record it, let the copies still in flight land, and leave.
      if (threadIdx.x == 0) {
        atomicOr(a.status, kStatusTimeout);
        for (int q = r; q < ntl && q < r + kStages; ++q)
          mbar_wait_bounded(&sm.bar[(g + q) % kStages], ((g + q) / kStages) & 1u);
      }
      __syncthreads();
      return false;
    }
    if (threadIdx.x == 0 && r + kStages < ntl) {
      const int tile = item_tile_df(a, it, it.vt_begin + r + kStages);
      mbar_arrive_expect_tx(&sm.bar[st], 2 * kBytes);
      bulk_g2s(sm.pos[st], gpos + size_t(tile) * 2 * kTileF64, kBytes, &sm.bar[st]);
      bulk_g2s(sm.val[st], gval + size_t(tile) * 2 * kTileF64, kBytes, &sm.bar[st]);
    }
  }
  g += ntl;
#pragma unroll
  for (int q = 0; q < kTptDF; ++q) {
    const int loc = q * kThreadsDF + int(threadIdx.x);
    const long long idx = it.part_off + it.tgt_begin + loc;
    if (loc < it.tgt_count && dcheck(idx >= 0 && idx < a.partial_cap, a.status))
      a.partial[idx] = make_double2(ux[q], uy[q]);
  }
  return true;
}

// Single instance: blockIdx.x = block of kThreadsDF x kTptDF targets, blockIdx.y = split.
template <int NIMG>
__global__ void __launch_bounds__(kThreadsDF) pair_df_kernel(PairArgs a) {
  __shared__ SmemDF sm;
  load_tables_df(a.dfc, sm);
  init_barriers(sm.bar);  // also orders the table loads before their use
  ItemDesc it;
  it.tgt_begin = blockIdx.x * (kThreadsDF * kTptDF);
  it.tgt_count = min(kThreadsDF * kTptDF, a.n_targets - it.tgt_begin);
  it.vt_begin = blockIdx.y * a.tiles_per_split;
  it.vt_end = min(a.n_tiles, it.vt_begin + a.tiles_per_split);
  it.wb = 0;
  it.nw = a.n_wall_tiles;
  it.vb = a.n_wall_tiles;
  it.part_off = (long long)blockIdx.y * a.n_targets;
  it.period = a.period;
  uint32_t g = 0;
  run_item_df<NIMG>(a, it, sm, g);
}

// Batched instances: persistent blocks take items of the FP64 item table (blocks of 128
// targets, 64-source tiles) through the work counter.
template <int NIMG>
__global__ void __launch_bounds__(kThreadsDF) pair_df_batch_kernel(PairArgs a) {
  __shared__ SmemDF sm;
  __shared__ int s_item;
  load_tables_df(a.dfc, sm);
  init_barriers(sm.bar);
  uint32_t g = 0;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int k = s_item;
    __syncthreads();
    if (k >= a.n_items) break;
    const ItemDesc it = a.items[k];
    if (!run_item_df<NIMG>(a, it, sm, g)) return;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int nblk_df(int n, int b) { return (n + b - 1) / b; }

cudaError_t launch_df_init(DFConst *d, cudaStream_t s) {
  df_init_kernel<<<1, 256, 0, s>>>(d);
  return cudaGetLastError();
}

// Grids from the geometry's coordinate bound, then the three-part source positions.
cudaError_t launch_geom_prep_df(stokes_ctx *c, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&c->d_dfc->maxabs_bits, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  double pmax = 0.0;
  for (const InstHost &in : c->inst) pmax = fmax(pmax, fabs(in.period));
  df_maxabs_kernel<<<std::min(nblk_df(c->N, 256), 1024), 256, 0, s>>>(c->N, c->d_x, pmax, c->d_dfc);
  df_grid_kernel<<<1, 1, 0, s>>>(c->d_dfc);
  const int s64 = c->wall_slots_f64 + c->ves_slots_f64;
  src_pos_df_kernel<<<nblk_df(s64, 256), 256, 0, s>>>(s64, c->d_slot_node64, c->d_x, c->d_dfc,
                                                       c->d_src_pos_df);
  return cudaGetLastError();
}

cudaError_t launch_pack_df(stokes_ctx *c, const double *slp, const double *dlp, cudaStream_t s) {
  const int slots = c->wall_slots_f64 + c->ves_slots_f64;
  pack_df_kernel<<<nblk_df(slots, 256), 256, 0, s>>>(
      slots, c->wall_slots_f64, c->d_slot_node64, c->d_node_dens, c->d_w, c->d_nrm, slp, dlp,
      1.0 / (4.0 * kPi * c->mu), c->d_status, c->d_src_val_df, c->N, c->n_ves_nodes,
      c->n_wall_nodes);
  return cudaGetLastError();
}

static PairArgs df_args(stokes_ctx *c) {
  PairArgs a{};
  a.partial = c->d_partial;
  a.partial_cap = partial_check_cap(c, (long long)c->partial_cap, c->batch_part64);
  a.src_tiles = (c->wall_slots_f64 + c->ves_slots_f64) / kTileF64;
  a.status = c->d_status;
  a.dfc = c->d_dfc;
  a.src_pos = c->d_src_pos_df;
  a.src_val = c->d_src_val_df;
  return a;
}

cudaError_t launch_pair_df(stokes_ctx *c, int n_targets, const double2 *tgt, const int2 *skip,
                           int splits, double2 *partial, cudaStream_t s) {
  PairArgs a = df_args(c);
  a.partial = partial;
  a.partial_cap = partial_check_cap(
      c, partial == c->d_partial ? (long long)c->partial_cap : (long long)splits * n_targets,
      (long long)splits * n_targets);
  a.n_targets = n_targets;
  a.tgt = tgt;
  a.tgt_skip = skip;
  a.period = c->period;
  a.n_wall_tiles = c->wall_slots_f64 / kTileF64;
  a.n_tiles = a.n_wall_tiles + c->ves_slots_f64 / kTileF64;
  a.tiles_per_split = (a.n_tiles + splits - 1) / splits;
  const int eff = (a.n_tiles + a.tiles_per_split - 1) / a.tiles_per_split;
  if (eff != splits) return cudaErrorInvalidValue;  // callers pass effective_splits() values
  dim3 grid((n_targets + kThreadsDF * kTptDF - 1) / (kThreadsDF * kTptDF), eff);
  if (c->period != 0.0)
    pair_df_kernel<3><<<grid, kThreadsDF, 0, s>>>(a);
  else
    pair_df_kernel<1><<<grid, kThreadsDF, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pair_batch_df(stokes_ctx *c, int blocks, cudaStream_t s) {
  PairArgs a = df_args(c);
  a.n_targets = c->N;
  a.tgt = c->d_x;
  a.tgt_skip = c->d_tgt_skip64;
  a.counter = c->d_counter;
  a.items = c->d_items64;
  a.n_items = c->n_items64;
  cudaError_t e = cudaMemsetAsync(c->d_counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (c->period != 0.0)
    pair_df_batch_kernel<3><<<blocks, kThreadsDF, 0, s>>>(a);
  else
    pair_df_batch_kernel<1><<<blocks, kThreadsDF, 0, s>>>(a);
  return cudaGetLastError();
}

static int occupancy_df(const void *f) {
  int nb = 0;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kThreadsDF, 0);
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

int pair_df_blocks_per_sm(stokes_ctx *c) {
  return c->period != 0.0 ? occupancy_df(reinterpret_cast<const void *>(pair_df_kernel<3>))
                          : occupancy_df(reinterpret_cast<const void *>(pair_df_kernel<1>));
}

int pair_df_batch_blocks_per_sm(stokes_ctx *c) {
  return c->period != 0.0 ? occupancy_df(reinterpret_cast<const void *>(pair_df_batch_kernel<3>))
                          : occupancy_df(reinterpret_cast<const void *>(pair_df_batch_kernel<1>));
}

}  // namespace stokes
