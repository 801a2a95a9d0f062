// k_pair.cu -- tiled N-body pair kernels of the near-image layer-potential sum.
//
// One block owns a block of targets and one split (contiguous range of source tiles).
// Source tiles are staged into shared memory by 1-D bulk async copies (cp.async.bulk,
// completion on an mbarrier) through a ring of kStages stages; every thread then reads
// each source record with two broadcast 16-byte shared loads and evaluates it against
// its targets for all images m in {-1, 0, +1} at once (the near-image sums of
// Eq. (Dnr) and Eq. (utotrep)).  Tiles hold one source kind only, so the stokeslet
// (Eq. (S)) / stresslet (Eq. (D)) branch is uniform over the block.
//
// FP32 path (STOKES_FP32_KAHAN):
//   * coordinates as (hi, lo) float pairs, targets pre-shifted by -m d in FP64 before the
//     split, so r = (x_hi - y_hi) + (x_lo - y_lo) is accurate to a few ulp of |r| even for
//     adjacent wall nodes (where r . n ~ kappa r^2 / 2 would otherwise be noise);
//   * 1/r^2 and log2(r^2) from the MUFU approximations (rcp.approx, lg2.approx);
//   * the image terms of KG consecutive sources are added in FP32, and that group sum
//     enters a per-target Kahan-compensated accumulator;
//   * each thread owns TPT targets and evaluates them two at a time with the packed
//     .f32x2 add/sub/mul/fma instructions (one instruction for both targets; the MUFU
//     approximations stay scalar), so source records are staged with every value
//     duplicated into both halves of a 64-bit pair;
//   * each (split, target) partial leaves the kernel as FP64 and is reduced across splits
//     in FP64, in fixed order, by the finishing kernel.
// FP64 path (STOKES_FP64): the same tiling in double precision, plain accumulation.
//
// Skips of the definition: a vesicle target skips the m = 0 image of its own curve's
// nodes (those are replaced by the Kress self rule); a wall target's own node at m = 0
// gives r = 0 exactly and contributes 0 (r2 carries a tiny floor so 1/r^2 stays finite
// while r . n = r . q = 0).
#include <algorithm>

#include "stokes_internal.cuh"
#include "bulk_pipe.cuh"

namespace stokes {

// Floor on r^2: keeps 1/r^2 and (1/r^2)^2 finite for the coincident wall self pair.
constexpr float kTiny32 = 1e-19f;
constexpr double kTiny64 = 1e-150;

// Knuth's error-free sum: s + e = a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (h + l) - o as one float, h, l the (hi, lo) split of a coordinate and o a float origin:
// the difference h - o is taken exactly, so only the final rounding remains.
__device__ __forceinline__ float local_coord(float h, float l, float o) {
  float b, e;
  two_sum(h, -o, b, e);
  return __fadd_rn(b, __fadd_rn(e, l));
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
  const float y = __fsub_rn(v, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// ---------------------------------------------------------------------------
// FP32 pair evaluation
// ---------------------------------------------------------------------------
template <int NIMG>
struct TgtF32 {
  float xh[NIMG], xl[NIMG];  // x - m d, split hi/lo
  float yh, yl;
  int2 skip;                 // own-curve source slots skipped at m = 0
};

// Target index of kernel target k (its node under the Morton order), bounds-checked in the
// debug build (an out-of-range index is recorded and redirected to target 0).
__device__ __forceinline__ int target_index(const PairArgs &a, int k) {
  const int i = a.tgt_perm ? a.tgt_perm[k] : k;
  return dcheck(i >= 0 && i < a.n_targets, a.status) ? i : 0;
}

// Source tile of a staged copy, bounds-checked in the debug build (out of range: recorded and
// redirected to tile 0, so the copy still arrives on its barrier).
__device__ __forceinline__ int checked_tile(const PairArgs &a, int tile) {
  return dcheck(tile >= 0 && tile < a.src_tiles, a.status) ? tile : 0;
}

// partial[idx] = v, bounds-checked in the debug build (out of range: recorded, not written).
__device__ __forceinline__ void store_partial(const PairArgs &a, long long idx, double2 v) {
  if (dcheck(idx >= 0 && idx < a.partial_cap, a.status)) a.partial[idx] = v;
}

template <int NIMG>
__device__ __forceinline__ void load_target_f32(const PairArgs &a, int k, TgtF32<NIMG> &t) {
  const int i = target_index(a, k);
  const double2 p = a.tgt[i];
#pragma unroll
  for (int k = 0; k < NIMG; ++k) {
    const double m = (NIMG == 3) ? double(k - 1) : 0.0;
    const double xm = p.x - m * a.period;
    const float h = __double2float_rn(xm);
    t.xh[k] = h;
    t.xl[k] = __double2float_rn(xm - double(h));
  }
  const float h = __double2float_rn(p.y);
  t.yh = h;
  t.yl = __double2float_rn(p.y - double(h));
  t.skip = a.tgt_skip ? a.tgt_skip[i] : make_int2(-1, -1);
}

// Stokeslet source (Eq. (S)); val = (q1, q2, p1, p2), q = w f / (4 pi mu), p = -(ln 2 / 2) q.
// Adds, for every image, log2(r^2) p + r (r . q) / r^2 to (ax, ay).
template <int NIMG, bool MASK0>
__device__ __forceinline__ void slp_source_f32(const TgtF32<NIMG> &t, const float4 pos,
                                               const float4 val, bool skip0, float &ax,
                                               float &ay) {
  const float dy = (t.yh - pos.y) + (t.yl - pos.w);
  const float dyq = dy * val.y;
  const float dy2 = fmaf(dy, dy, kTiny32);
  if constexpr (NIMG == 3) {
    // One rcp and one lg2 for the three images (see slp_source_x2).
    const float dx0 = (t.xh[0] - pos.x) + (t.xl[0] - pos.z);
    const float dx1 = (t.xh[1] - pos.x) + (t.xl[1] - pos.z);
    const float dx2 = (t.xh[2] - pos.x) + (t.xl[2] - pos.z);
    const float a = fmaf(dx0, dx0, dy2);
    const float b = (MASK0 && skip0) ? 1.0f : fmaf(dx1, dx1, dy2);
    const float c = fmaf(dx2, dx2, dy2);
    const float ab = a * b;
    const float abc = ab * c;
    const float inv = rcp_approx(abc);
    const float lg = lg2_approx(abc);
    const float s0 = fmaf(dx0, val.x, dyq) * ((b * c) * inv);
    const float s1 = (MASK0 && skip0) ? 0.0f : fmaf(dx1, val.x, dyq) * ((a * c) * inv);
    const float s2 = fmaf(dx2, val.x, dyq) * (ab * inv);
    ax = fmaf(lg, val.z, ax);
    ax = fmaf(s0, dx0, ax);
    ax = fmaf(s1, dx1, ax);
    ax = fmaf(s2, dx2, ax);
    ay = fmaf(lg, val.w, ay);
    ay = fmaf((s0 + s1) + s2, dy, ay);
  } else {
#pragma unroll
    for (int k = 0; k < NIMG; ++k) {
      if (MASK0 && k == NIMG / 2 && skip0) continue;
      const float dx = (t.xh[k] - pos.x) + (t.xl[k] - pos.z);
      const float r2 = fmaf(dx, dx, dy2);
      const float inv = rcp_approx(r2);
      const float lg = lg2_approx(r2);
      const float s = fmaf(dx, val.x, dyq) * inv;
      ax = fmaf(lg, val.z, ax);
      ax = fmaf(s, dx, ax);
      ay = fmaf(lg, val.w, ay);
      ay = fmaf(s, dy, ay);
    }
  }
}

// Stresslet source (Eq. (D)); val = (q1, q2, n1, n2), q = w tau / pi.
// Adds, for every image, r (r . n)(r . q) / r^4 to (ax, ay).
template <int NIMG>
__device__ __forceinline__ void dlp_source_f32(const TgtF32<NIMG> &t, const float4 pos,
                                               const float4 val, float &ax, float &ay) {
  const float dy = (t.yh - pos.y) + (t.yl - pos.w);
  const float dyn = dy * val.w;
  const float dyq = dy * val.y;
  const float dy2 = fmaf(dy, dy, kTiny32);
#pragma unroll
  for (int k = 0; k < NIMG; ++k) {
    const float dx = (t.xh[k] - pos.x) + (t.xl[k] - pos.z);
    const float r2 = fmaf(dx, dx, dy2);
    const float inv = rcp_approx(r2);
    const float rn = fmaf(dx, val.z, dyn);
    const float rq = fmaf(dx, val.x, dyq);
    const float f = (rn * rq) * (inv * inv);
    ax = fmaf(f, dx, ax);
    ay = fmaf(f, dy, ay);
  }
}

// ---------------------------------------------------------------------------
// Packed two-target FP32 evaluation (add/sub/mul/fma .f32x2): two targets share every
// instruction except the MUFU approximations, which stay scalar.
// ---------------------------------------------------------------------------
typedef unsigned long long f2;  // two floats; the first in the low word

__device__ __forceinline__ f2 f2_pack(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float &a, float &b) {
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
__device__ __forceinline__ f2 rcp2(f2 v) {
  float a, b;
  f2_unpack(v, a, b);
  return f2_pack(rcp_approx(a), rcp_approx(b));
}
__device__ __forceinline__ f2 lg22(f2 v) {
  float a, b;
  f2_unpack(v, a, b);
  return f2_pack(lg2_approx(a), lg2_approx(b));
}

__device__ __forceinline__ void kahan_add2(f2 &s, f2 &c, f2 v) {
  const f2 y = sub2(v, c);
  const f2 t = add2(s, y);
  c = sub2(sub2(t, s), y);
  s = t;
}

// Two targets, packed: (x - m d) hi/lo per image, y hi/lo.
template <int NIMG>
struct TgtF32x2 {
  f2 xh[NIMG], xl[NIMG];
  f2 yh, yl;
};

template <int NIMG>
__device__ __forceinline__ TgtF32x2<NIMG> pack_targets(const TgtF32<NIMG> &a, const TgtF32<NIMG> &b) {
  TgtF32x2<NIMG> t;
#pragma unroll
  for (int k = 0; k < NIMG; ++k) {
    t.xh[k] = f2_pack(a.xh[k], b.xh[k]);
    t.xl[k] = f2_pack(a.xl[k], b.xl[k]);
  }
  t.yh = f2_pack(a.yh, b.yh);
  t.yl = f2_pack(a.yl, b.yl);
  return t;
}

// A source record as packed duplicates: coordinates (x_hi, y_hi), (x_lo, y_lo) and
// values (q1, q2), (p1|n1, p2|n2), each half of a pair holding the same float.
struct SrcX2 {
  f2 xh, yh, xl, yl, v0, v1, v2, v3;
};

__device__ __forceinline__ SrcX2 load_src_x2(const float4 *P, const float4 *V, int j) {
  const ulonglong2 a = reinterpret_cast<const ulonglong2 *>(P)[2 * j];
  const ulonglong2 b = reinterpret_cast<const ulonglong2 *>(P)[2 * j + 1];
  const ulonglong2 c = reinterpret_cast<const ulonglong2 *>(V)[2 * j];
  const ulonglong2 d = reinterpret_cast<const ulonglong2 *>(V)[2 * j + 1];
  return SrcX2{a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y};
}

// Stokeslet terms of one source against two targets, from the packed differences dx[m] (one
// per image), dy, dyq = dy q2 and dy2 = dy^2 + tiny; v0..v3 = (q1, q2, p1, p2).  With MASK0,
// the m = 0 image is dropped (per target) where sa / sb is set.
template <int NIMG, bool MASK0>
__device__ __forceinline__ void slp_images_x2(const f2 (&dxm)[NIMG], f2 dy, f2 dyq, f2 dy2,
                                              f2 v0, f2 v2, f2 v3, bool sa, bool sb, f2 &ax,
                                              f2 &ay) {
  if constexpr (NIMG == 3) {
    // Three images share one MUFU pair: with a, b, c the squared distances to the images
    // m = -1, 0, +1, the log terms sum to p log2(abc) and 1/a = bc/(abc), 1/b = ac/(abc),
    // 1/c = ab/(abc).  A masked m = 0 image enters the product as b = 1 and its r r^T / r^2
    // term is dropped.  (abc stays a normal float while no two images of one source lie
    // within ~1e-10 of a target, i.e. for any period above the curves' node spacing.)
    const f2 dx0 = dxm[0], dx1 = dxm[1], dx2 = dxm[2];
    const f2 a = fma2(dx0, dx0, dy2);
    f2 b = fma2(dx1, dx1, dy2);
    const f2 c = fma2(dx2, dx2, dy2);
    if (MASK0 && (sa || sb)) {
      float b0, b1;
      f2_unpack(b, b0, b1);
      b = f2_pack(sa ? 1.0f : b0, sb ? 1.0f : b1);
    }
    const f2 ab = mul2(a, b);
    const f2 abc = mul2(ab, c);
    const f2 inv = rcp2(abc);
    const f2 lg = lg22(abc);
    const f2 ia = mul2(mul2(b, c), inv);
    f2 ib = mul2(mul2(a, c), inv);
    const f2 ic = mul2(ab, inv);
    if (MASK0 && (sa || sb)) {
      float i0, i1;
      f2_unpack(ib, i0, i1);
      ib = f2_pack(sa ? 0.0f : i0, sb ? 0.0f : i1);
    }
    const f2 s0 = mul2(fma2(dx0, v0, dyq), ia);
    const f2 s1 = mul2(fma2(dx1, v0, dyq), ib);
    const f2 s2 = mul2(fma2(dx2, v0, dyq), ic);
    ax = fma2(lg, v2, ax);
    ax = fma2(s0, dx0, ax);
    ax = fma2(s1, dx1, ax);
    ax = fma2(s2, dx2, ax);
    ay = fma2(lg, v3, ay);
    ay = fma2(add2(add2(s0, s1), s2), dy, ay);
  } else {
#pragma unroll
    for (int k = 0; k < NIMG; ++k) {
      const f2 ax0 = ax, ay0 = ay;
      const f2 dx = dxm[k];
      const f2 r2 = fma2(dx, dx, dy2);
      const f2 inv = rcp2(r2);
      const f2 lg = lg22(r2);
      const f2 s = mul2(fma2(dx, v0, dyq), inv);
      ax = fma2(lg, v2, ax);
      ax = fma2(s, dx, ax);
      ay = fma2(lg, v3, ay);
      ay = fma2(s, dy, ay);
      if (MASK0 && k == NIMG / 2 && (sa || sb)) {
        float n0, n1, o0, o1;
        f2_unpack(ax, n0, n1);
        f2_unpack(ax0, o0, o1);
        ax = f2_pack(sa ? o0 : n0, sb ? o1 : n1);
        f2_unpack(ay, n0, n1);
        f2_unpack(ay0, o0, o1);
        ay = f2_pack(sa ? o0 : n0, sb ? o1 : n1);
      }
    }
  }
}

// Stokeslet source against two targets from (hi, lo) coordinates: as slp_source_f32,
// v0..v3 = (q1, q2, p1, p2).
template <int NIMG, bool MASK0>
__device__ __forceinline__ void slp_source_x2(const TgtF32x2<NIMG> &t, const SrcX2 &src, bool sa,
                                              bool sb, f2 &ax, f2 &ay) {
  const f2 dy = add2(sub2(t.yh, src.yh), sub2(t.yl, src.yl));
  const f2 dyq = mul2(dy, src.v1);
  const f2 dy2 = fma2(dy, dy, f2_pack(kTiny32, kTiny32));
  f2 dxm[NIMG];
#pragma unroll
  for (int k = 0; k < NIMG; ++k) dxm[k] = add2(sub2(t.xh[k], src.xh), sub2(t.xl[k], src.xl));
  slp_images_x2<NIMG, MASK0>(dxm, dy, dyq, dy2, src.v0, src.v2, src.v3, sa, sb, ax, ay);
}

// Stokeslet source against two targets in a block-local frame: targets (tx, ty) and source
// images sx[m], sy are single floats relative to the block's origin, so each difference is
// one subtraction.
template <int NIMG, bool MASK0>
__device__ __forceinline__ void slp_local_x2(f2 tx, f2 ty, const f2 (&sx)[NIMG], f2 sy, f2 v0,
                                             f2 v1, f2 v2, f2 v3, bool sa, bool sb, f2 &ax,
                                             f2 &ay) {
  const f2 dy = sub2(ty, sy);
  const f2 dyq = mul2(dy, v1);
  const f2 dy2 = fma2(dy, dy, f2_pack(kTiny32, kTiny32));
  f2 dxm[NIMG];
#pragma unroll
  for (int k = 0; k < NIMG; ++k) dxm[k] = sub2(tx, sx[k]);
  slp_images_x2<NIMG, MASK0>(dxm, dy, dyq, dy2, v0, v2, v3, sa, sb, ax, ay);
}

// Stresslet terms of one source against two targets from the packed differences dx[m],
// dy, dyn = dy n2, dyq = dy q2 and dy2 = dy^2 + tiny; v0, v2 = q1, n1.
template <int NIMG>
__device__ __forceinline__ void dlp_images_x2(const f2 (&dxm)[NIMG], f2 dy, f2 dyn, f2 dyq, f2 dy2,
                                              f2 v0, f2 v2, f2 &ax, f2 &ay) {
#pragma unroll
  for (int k = 0; k < NIMG; ++k) {
    const f2 dx = dxm[k];
    const f2 r2 = fma2(dx, dx, dy2);
    const f2 inv = rcp2(r2);
    const f2 rn = fma2(dx, v2, dyn);
    const f2 rq = fma2(dx, v0, dyq);
    const f2 f = mul2(mul2(rn, rq), mul2(inv, inv));
    ax = fma2(f, dx, ax);
    ay = fma2(f, dy, ay);
  }
}

// Stresslet source against two targets from (hi, lo) coordinates: as dlp_source_f32,
// v0..v3 = (q1, q2, n1, n2).
template <int NIMG>
__device__ __forceinline__ void dlp_source_x2(const TgtF32x2<NIMG> &t, const SrcX2 &src, f2 &ax,
                                              f2 &ay) {
  const f2 dy = add2(sub2(t.yh, src.yh), sub2(t.yl, src.yl));
  const f2 dyn = mul2(dy, src.v3);
  const f2 dyq = mul2(dy, src.v1);
  const f2 dy2 = fma2(dy, dy, f2_pack(kTiny32, kTiny32));
  f2 dxm[NIMG];
#pragma unroll
  for (int k = 0; k < NIMG; ++k) dxm[k] = add2(sub2(t.xh[k], src.xh), sub2(t.xl[k], src.xl));
  dlp_images_x2<NIMG>(dxm, dy, dyn, dyq, dy2, src.v0, src.v2, ax, ay);
}

// Stresslet source against two targets in the block-local frame (see slp_local_x2).
template <int NIMG>
__device__ __forceinline__ void dlp_local_x2(f2 tx, f2 ty, const f2 (&sx)[NIMG], f2 sy, f2 v0,
                                             f2 v1, f2 v2, f2 v3, f2 &ax, f2 &ay) {
  const f2 dy = sub2(ty, sy);
  const f2 dyn = mul2(dy, v3);
  const f2 dyq = mul2(dy, v1);
  const f2 dy2 = fma2(dy, dy, f2_pack(kTiny32, kTiny32));
  f2 dxm[NIMG];
#pragma unroll
  for (int k = 0; k < NIMG; ++k) dxm[k] = sub2(tx, sx[k]);
  dlp_images_x2<NIMG>(dxm, dy, dyn, dyq, dy2, v0, v2, ax, ay);
}

// Sum over one tile: KG consecutive sources (all images) are added in FP32 into a group
// sum, and each group sum enters the Kahan-compensated per-target accumulator.  Targets
// are taken two at a time in packed arithmetic; an odd TPT leaves one scalar target.
// Accumulators: packed pairs (sx2, cx2, sy2, cy2)[TPT / 2]; the scalar one in (sx, cx, sy, cy).
// KIND: 0 stresslet, 1 stokeslet, 2 stokeslet with the own-curve m = 0 skip; in the
// block-local frame (even TPT only; source images from L, written by translate_source_f32,
// targets from (lx, ly)): 3 stokeslet, 4 stokeslet with the skip, 5 stresslet.
template <int NIMG, int TPT, int KG, int KIND>
__device__ __forceinline__ void tile_sum_f32(const TgtF32<NIMG> (&tg)[TPT], const float4 *P,
                                             const float4 *V, const float4 *L, int slot0,
                                             const f2 (&lx)[TPT / 2 + 1],
                                             const f2 (&ly)[TPT / 2 + 1],
                                             f2 (&acc)[TPT / 2 + 1][4], float (&acc1)[4]) {
  constexpr int NP = TPT / 2;
  static_assert(KIND < 3 || (TPT & 1) == 0, "the local frame needs an even TPT");
  TgtF32x2<NIMG> tp[NP > 0 ? NP : 1];
  if constexpr (KIND < 3) {
#pragma unroll
    for (int h = 0; h < NP; ++h) tp[h] = pack_targets<NIMG>(tg[2 * h], tg[2 * h + 1]);
  }
#pragma unroll((KIND == 2 || KIND == 4) ? 1 : 2)
  for (int j = 0; j < kTileF32; j += KG) {
    f2 gx[NP > 0 ? NP : 1], gy[NP > 0 ? NP : 1];
    float hx = -0.0f, hy = -0.0f;
#pragma unroll
    for (int h = 0; h < NP; ++h) gx[h] = gy[h] = f2_pack(-0.0f, -0.0f);
#pragma unroll
    for (int u = 0; u < KG; ++u) {
      const int slot = slot0 + j + u;
      if constexpr (KIND >= 3) {
        const ulonglong2 l0 = reinterpret_cast<const ulonglong2 *>(L)[2 * (j + u)];
        const ulonglong2 l1 = reinterpret_cast<const ulonglong2 *>(L)[2 * (j + u) + 1];
        const ulonglong2 w0 = reinterpret_cast<const ulonglong2 *>(V)[2 * (j + u)];
        const ulonglong2 w1 = reinterpret_cast<const ulonglong2 *>(V)[2 * (j + u) + 1];
        f2 sx[NIMG];
        if constexpr (NIMG == 3) {
          sx[0] = l0.x;
          sx[1] = l0.y;
          sx[2] = l1.x;
        } else {
          sx[0] = l0.y;
        }
#pragma unroll
        for (int h = 0; h < NP; ++h) {
          if (KIND == 5) {
            dlp_local_x2<NIMG>(lx[h], ly[h], sx, l1.y, w0.x, w0.y, w1.x, w1.y, gx[h], gy[h]);
            continue;
          }
          bool sa = false, sb = false;
          if (KIND == 4) {
            sa = slot >= tg[2 * h].skip.x && slot < tg[2 * h].skip.y;
            sb = slot >= tg[2 * h + 1].skip.x && slot < tg[2 * h + 1].skip.y;
          }
          slp_local_x2<NIMG, KIND == 4>(lx[h], ly[h], sx, l1.y, w0.x, w0.y, w1.x, w1.y, sa, sb,
                                         gx[h], gy[h]);
        }
        continue;
      }
      const SrcX2 src = load_src_x2(P, V, j + u);
#pragma unroll
      for (int h = 0; h < NP; ++h) {
        if (KIND == 0) {
          dlp_source_x2<NIMG>(tp[h], src, gx[h], gy[h]);
        } else if (KIND == 1) {
          slp_source_x2<NIMG, false>(tp[h], src, false, false, gx[h], gy[h]);
        } else {
          const TgtF32<NIMG> &ta = tg[2 * h], &tb = tg[2 * h + 1];
          const bool sa = slot >= ta.skip.x && slot < ta.skip.y;
          const bool sb = slot >= tb.skip.x && slot < tb.skip.y;
          slp_source_x2<NIMG, true>(tp[h], src, sa, sb, gx[h], gy[h]);
        }
      }
      if ((TPT & 1) && KIND < 3) {
        const TgtF32<NIMG> &t = tg[TPT - 1];
        const float4 a = P[2 * (j + u)], b = P[2 * (j + u) + 1];
        const float4 c = V[2 * (j + u)], d = V[2 * (j + u) + 1];
        const float4 p = make_float4(a.x, a.z, b.x, b.z), v = make_float4(c.x, c.z, d.x, d.z);
        if (KIND == 0) {
          dlp_source_f32<NIMG>(t, p, v, hx, hy);
        } else if (KIND == 1) {
          slp_source_f32<NIMG, false>(t, p, v, false, hx, hy);
        } else {
          const bool s0 = slot >= t.skip.x && slot < t.skip.y;
          slp_source_f32<NIMG, true>(t, p, v, s0, hx, hy);
        }
      }
    }
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      kahan_add2(acc[h][0], acc[h][1], gx[h]);
      kahan_add2(acc[h][2], acc[h][3], gy[h]);
    }
    if (TPT & 1) {
      kahan_add(acc1[0], acc1[1], hx);
      kahan_add(acc1[2], acc1[3], hy);
    }
  }
}

// Shared memory of the FP32 kernels: kStages source tiles and their mbarriers, and the
// current stokeslet tile's positions in the block-local frame.
struct SmemF32 {
  __align__(128) float4 pos[kStages][2 * kTileF32];
  __align__(128) float4 val[kStages][2 * kTileF32];
  __align__(16) float4 loc[2 * kTileF32];
  __align__(8) uint64_t bar[kStages];
};

// Source k of a staged tile in the block-local frame with origin (ox, oy): the images
// x + m d - ox for m = -1, 0, +1 (d = dh + dl) and y - oy, each rounded once, stored as
// loc[2k] = (x_-1, x_-1, x_0, x_0), loc[2k+1] = (x_+1, x_+1, y, y) (with images off, every x is
// x_0).  The origin is near the block's targets, so a source close to one of them gets small
// local coordinates and small rounding errors.
template <int NIMG>
__device__ __forceinline__ void translate_source_f32(const float4 *P, int k, float ox, float oy,
                                                     float dh, float dl, float4 *loc) {
  const float4 h = P[2 * k], l = P[2 * k + 1];  // (x_hi, ., y_hi, .), (x_lo, ., y_lo, .)
  float b, e;
  two_sum(h.x, -ox, b, e);
  const float el = __fadd_rn(e, l.x);
  const float x0 = __fadd_rn(b, el);
  float xm = x0, xp = x0;
  if constexpr (NIMG == 3) {
    float sm, em, sp, ep;
    two_sum(b, -dh, sm, em);
    two_sum(b, dh, sp, ep);
    xm = __fadd_rn(sm, __fadd_rn(em, __fsub_rn(el, dl)));
    xp = __fadd_rn(sp, __fadd_rn(ep, __fadd_rn(el, dl)));
  }
  const float y0 = local_coord(h.z, l.z, oy);
  loc[2 * k] = make_float4(xm, xm, x0, x0);
  loc[2 * k + 1] = make_float4(xp, xp, y0, y0);
}

__device__ __forceinline__ int item_tile(const ItemDesc &it, int vt) {
  return vt < it.nw ? it.wb + vt : it.vb + (vt - it.nw);
}

// One work item: targets [tgt_begin, +tgt_count) against virtual tiles [vt_begin, vt_end).
// `g` counts the tiles this block has consumed so far; stage = g mod kStages and the
// mbarrier parity = (g / kStages) mod 2, so the barriers carry over from item to item.
// Returns false when a stage wait timed out (the block must then leave; uniform).
template <int NIMG, int TPT, int KG>
__device__ __forceinline__ bool run_item_f32(const PairArgs &a, const ItemDesc &it, SmemF32 &sm,
                                             uint32_t &g) {
  const int ntl = it.vt_end - it.vt_begin;
  TgtF32<NIMG> tg[TPT];
  f2 acc[TPT / 2 + 1][4];  // packed (s_x, c_x, s_y, c_y) of target pairs
  float acc1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  {
    PairArgs b = a;
    b.period = it.period;
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int loc = min(q * kThreadsF32 + int(threadIdx.x), it.tgt_count - 1);
      load_target_f32<NIMG>(b, it.tgt_begin + loc, tg[q]);
    }
#pragma unroll
    for (int h = 0; h <= TPT / 2; ++h)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[h][c] = f2_pack(0.0f, 0.0f);
  }
  // Block-local frame for the stokeslet tiles: origin at the item's middle target; taken when
  // every target of the block lies within local_radius of it (max norm).
  f2 lx[TPT / 2 + 1], ly[TPT / 2 + 1];
  bool local = false, local_dlp = false;
  float ox = 0.f, oy = 0.f, dh = 0.f, dl = 0.f;
  if constexpr ((TPT & 1) == 0) {
    if (a.local_radius > 0.f) {
      const int k0 = it.tgt_begin + it.tgt_count / 2;
      const double2 o = a.tgt[target_index(a, k0)];
      ox = __double2float_rn(o.x);
      oy = __double2float_rn(o.y);
      float rmax = 0.f;
#pragma unroll
      for (int h = 0; h < TPT / 2; ++h) {
        const TgtF32<NIMG> &u = tg[2 * h], &v = tg[2 * h + 1];
        const float xa = local_coord(u.xh[NIMG / 2], u.xl[NIMG / 2], ox);
        const float xb = local_coord(v.xh[NIMG / 2], v.xl[NIMG / 2], ox);
        const float ya = local_coord(u.yh, u.yl, oy), yb = local_coord(v.yh, v.yl, oy);
        lx[h] = f2_pack(xa, xb);
        ly[h] = f2_pack(ya, yb);
        rmax = fmaxf(rmax, fmaxf(fmaxf(fabsf(xa), fabsf(xb)), fmaxf(fabsf(ya), fabsf(yb))));
      }
      local = !__syncthreads_or(!(rmax <= a.local_radius));
      // wall tiles too when every target is a vesicle node (they keep the gap from the walls)
      bool ves = true;
#pragma unroll
      for (int q = 0; q < TPT; ++q) ves = ves && tg[q].skip.x >= 0;
      local_dlp = __syncthreads_and(local && ves);
      dh = __double2float_rn(it.period);
      dl = __double2float_rn(it.period - double(dh));
    }
  }
  const float4 *gpos = static_cast<const float4 *>(a.src_pos);
  const float4 *gval = static_cast<const float4 *>(a.src_val);
  constexpr uint32_t kBytes = 2 * kTileF32 * sizeof(float4);

  if (threadIdx.x == 0) {
    for (int r = 0; r < kStages && r < ntl; ++r) {
      const int st = (g + r) % kStages;
      const int tile = checked_tile(a, item_tile(it, it.vt_begin + r));
      mbar_arrive_expect_tx(&sm.bar[st], 2 * kBytes);
      bulk_g2s(sm.pos[st], gpos + size_t(tile) * 2 * kTileF32, kBytes, &sm.bar[st]);
      bulk_g2s(sm.val[st], gval + size_t(tile) * 2 * kTileF32, kBytes, &sm.bar[st]);
    }
  }

  static_assert(kThreadsF32 == kTileF32, "one thread translates one source of a tile");
  for (int r = 0; r < ntl; ++r) {
    const uint32_t gr = g + r;
    const int st = gr % kStages;
    const bool ok = mbar_wait_bounded(&sm.bar[st], (gr / kStages) & 1u);
    const int vt = it.vt_begin + r;
    if (vt >= it.nw ? local : local_dlp) {  // uniform: tile in the block-local frame
      if (ok) translate_source_f32<NIMG>(sm.pos[st], threadIdx.x, ox, oy, dh, dl, sm.loc);
      __syncthreads();
    }
    if (ok) {
      const int tile = item_tile(it, vt);
      const int slot0 = tile * kTileF32;
      const float4 *P = sm.pos[st];
      const float4 *V = sm.val[st];
      if (vt < it.nw) {
        bool done = false;
        if constexpr ((TPT & 1) == 0) {
          if (local_dlp) {
            tile_sum_f32<NIMG, TPT, KG, 5>(tg, P, V, sm.loc, slot0, lx, ly, acc, acc1);
            done = true;
          }
        }
        if (!done) tile_sum_f32<NIMG, TPT, KG, 0>(tg, P, V, sm.loc, slot0, lx, ly, acc, acc1);
      } else {
        bool mine = false;
#pragma unroll
        for (int q = 0; q < TPT; ++q)
          mine |= (tg[q].skip.x < slot0 + kTileF32) && (tg[q].skip.y > slot0);
        const bool any_mine = __any_sync(0xffffffffu, mine);
        bool done = false;
        if constexpr ((TPT & 1) == 0) {
          if (local) {
            if (any_mine)
              tile_sum_f32<NIMG, TPT, KG, 4>(tg, P, V, sm.loc, slot0, lx, ly, acc, acc1);
            else
              tile_sum_f32<NIMG, TPT, KG, 3>(tg, P, V, sm.loc, slot0, lx, ly, acc, acc1);
            done = true;
          }
        }
        if (!done) {
          if (any_mine)
            tile_sum_f32<NIMG, TPT, KG, 2>(tg, P, V, sm.loc, slot0, lx, ly, acc, acc1);
          else
            tile_sum_f32<NIMG, TPT, KG, 1>(tg, P, V, sm.loc, slot0, lx, ly, acc, acc1);
        }
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
      const int tile = checked_tile(a, item_tile(it, it.vt_begin + r + kStages));
      mbar_arrive_expect_tx(&sm.bar[st], 2 * kBytes);
      bulk_g2s(sm.pos[st], gpos + size_t(tile) * 2 * kTileF32, kBytes, &sm.bar[st]);
      bulk_g2s(sm.val[st], gval + size_t(tile) * 2 * kTileF32, kBytes, &sm.bar[st]);
    }
  }
  g += ntl;

#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    float sx, cx, sy, cy;
    if ((TPT & 1) && q == TPT - 1) {
      sx = acc1[0];
      cx = acc1[1];
      sy = acc1[2];
      cy = acc1[3];
    } else {
      float o;
      const int h = q / 2;
      if (q & 1) {
        f2_unpack(acc[h][0], o, sx);
        f2_unpack(acc[h][1], o, cx);
        f2_unpack(acc[h][2], o, sy);
        f2_unpack(acc[h][3], o, cy);
      } else {
        f2_unpack(acc[h][0], sx, o);
        f2_unpack(acc[h][1], cx, o);
        f2_unpack(acc[h][2], sy, o);
        f2_unpack(acc[h][3], cy, o);
      }
    }
    const int loc = q * kThreadsF32 + int(threadIdx.x);
    if (loc < it.tgt_count) {
      const int k = it.tgt_begin + loc;
      store_partial(a, it.part_off + target_index(a, k),
                    make_double2(double(sx) - double(cx), double(sy) - double(cy)));
    }
  }
  return true;
}

// Single instance: blockIdx.x = target block, blockIdx.y = source split.
template <int NIMG, int TPT, int KG>
__global__ void __launch_bounds__(kThreadsF32, TPT == 4 ? 4 : TPT == 2 ? 6 : 8) pair_f32k_kernel(PairArgs a) {
  __shared__ SmemF32 sm;
  init_barriers(sm.bar);
  ItemDesc it;
  it.tgt_begin = blockIdx.x * (kThreadsF32 * TPT);
  it.tgt_count = min(kThreadsF32 * TPT, a.n_targets - it.tgt_begin);
  it.vt_begin = blockIdx.y * a.tiles_per_split;
  it.vt_end = min(a.n_tiles, it.vt_begin + a.tiles_per_split);
  it.wb = 0;
  it.nw = a.n_wall_tiles;
  it.vb = a.n_wall_tiles;
  it.part_off = (long long)blockIdx.y * a.n_targets;
  it.period = a.period;
  uint32_t g = 0;
  run_item_f32<NIMG, TPT, KG>(a, it, sm, g);
}

// Batched instances: a persistent grid takes items from the table through a work counter.
template <int NIMG, int TPT, int KG>
__global__ void __launch_bounds__(kThreadsF32, TPT == 4 ? 4 : TPT == 2 ? 6 : 8) pair_f32k_batch_kernel(PairArgs a) {
  __shared__ SmemF32 sm;
  __shared__ int s_item;
  init_barriers(sm.bar);
  uint32_t g = 0;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int k = s_item;
    __syncthreads();
    if (k >= a.n_items) break;
    const ItemDesc it = a.items[k];
    if (!run_item_f32<NIMG, TPT, KG>(a, it, sm, g)) return;
  }
}

// ---------------------------------------------------------------------------
// FP64 pair evaluation
// ---------------------------------------------------------------------------
template <int NIMG>
struct TgtF64 {
  double x[NIMG];
  double y;
  int2 skip;
};

// Stokeslet; val = (q1, q2, p1, p2) with q = w f / (4 pi mu), p = -q / 2.
template <int NIMG, bool MASK0>
__device__ __forceinline__ void slp_source_f64(const TgtF64<NIMG> &t, const double2 pos,
                                               const double4_32a val, bool skip0, double &ax,
                                               double &ay, const LogTab *lt) {
  const double dy = t.y - pos.y;
  const double dyq = dy * val.y;
  const double dy2 = fma(dy, dy, kTiny64);
#pragma unroll
  for (int k = 0; k < NIMG; ++k) {
    if (MASK0 && k == NIMG / 2 && skip0) continue;
    const double dx = t.x[k] - pos.x;
    const double r2 = fma(dx, dx, dy2);
    const double inv = __drcp_rn(r2);
    const double lg = flog64(r2, lt);
    const double s = fma(dx, val.x, dyq) * inv;
    ax = fma(lg, val.z, ax);
    ax = fma(s, dx, ax);
    ay = fma(lg, val.w, ay);
    ay = fma(s, dy, ay);
  }
}

// Stresslet; val = (q1, q2, n1, n2) with q = w tau / pi.
template <int NIMG>
__device__ __forceinline__ void dlp_source_f64(const TgtF64<NIMG> &t, const double2 pos,
                                               const double4_32a val, double &ax, double &ay) {
  const double dy = t.y - pos.y;
  const double dyn = dy * val.w;
  const double dyq = dy * val.y;
  const double dy2 = fma(dy, dy, kTiny64);
#pragma unroll
  for (int k = 0; k < NIMG; ++k) {
    const double dx = t.x[k] - pos.x;
    const double r2 = fma(dx, dx, dy2);
    const double inv = __drcp_rn(r2);
    const double rn = fma(dx, val.z, dyn);
    const double rq = fma(dx, val.x, dyq);
    const double f = (rn * rq) * (inv * inv);
    ax = fma(f, dx, ax);
    ay = fma(f, dy, ay);
  }
}

struct SmemF64 {
  __align__(128) double2 pos[kStages][kTileF64];
  __align__(128) double4_32a val[kStages][kTileF64];
  __align__(8) uint64_t bar[kStages];
};

template <int NIMG>
__device__ __forceinline__ bool run_item_f64(const PairArgs &a, const ItemDesc &it, SmemF64 &sm,
                                             uint32_t &g) {
  const int ntl = it.vt_end - it.vt_begin;
  const int loc = threadIdx.x;
  const int i = target_index(a, it.tgt_begin + min(loc, it.tgt_count - 1));
  TgtF64<NIMG> t;
  {
    const double2 p = a.tgt[i];
#pragma unroll
    for (int k = 0; k < NIMG; ++k) t.x[k] = p.x - ((NIMG == 3) ? double(k - 1) : 0.0) * it.period;
    t.y = p.y;
    t.skip = a.tgt_skip ? a.tgt_skip[i] : make_int2(-1, -1);
  }
  double ux = 0.0, uy = 0.0;
  const double2 *gpos = static_cast<const double2 *>(a.src_pos);
  const double4_32a *gval = static_cast<const double4_32a *>(a.src_val);
  constexpr uint32_t kBp = kTileF64 * sizeof(double2);
  constexpr uint32_t kBv = kTileF64 * sizeof(double4_32a);

  if (threadIdx.x == 0) {
    for (int r = 0; r < kStages && r < ntl; ++r) {
      const int st = (g + r) % kStages;
      const int tile = checked_tile(a, item_tile(it, it.vt_begin + r));
      mbar_arrive_expect_tx(&sm.bar[st], kBp + kBv);
      bulk_g2s(sm.pos[st], gpos + size_t(tile) * kTileF64, kBp, &sm.bar[st]);
      bulk_g2s(sm.val[st], gval + size_t(tile) * kTileF64, kBv, &sm.bar[st]);
    }
  }
  for (int r = 0; r < ntl; ++r) {
    const uint32_t gr = g + r;
    const int st = gr % kStages;
    const bool ok = mbar_wait_bounded(&sm.bar[st], (gr / kStages) & 1u);
    if (ok) {
      const int vt = it.vt_begin + r;
      const int tile = item_tile(it, vt);
      if (vt < it.nw) {
        for (int j = 0; j < kTileF64; ++j) dlp_source_f64<NIMG>(t, sm.pos[st][j], sm.val[st][j], ux, uy);
      } else {
        const int slot0 = tile * kTileF64;
        const bool mine = (t.skip.x < slot0 + kTileF64) && (t.skip.y > slot0);
        if (__any_sync(0xffffffffu, mine)) {
          for (int j = 0; j < kTileF64; ++j) {
            const bool s0 = (slot0 + j >= t.skip.x) && (slot0 + j < t.skip.y);
            slp_source_f64<NIMG, true>(t, sm.pos[st][j], sm.val[st][j], s0, ux, uy, a.logtab);
          }
        } else {
          for (int j = 0; j < kTileF64; ++j)
            slp_source_f64<NIMG, false>(t, sm.pos[st][j], sm.val[st][j], false, ux, uy, a.logtab);
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(a.status, kStatusTimeout);
        for (int q = r; q < ntl && q < r + kStages; ++q)
          mbar_wait_bounded(&sm.bar[(g + q) % kStages], ((g + q) / kStages) & 1u);
      }
      __syncthreads();
      return false;
    }
    if (threadIdx.x == 0 && r + kStages < ntl) {
      const int tile = checked_tile(a, item_tile(it, it.vt_begin + r + kStages));
      mbar_arrive_expect_tx(&sm.bar[st], kBp + kBv);
      bulk_g2s(sm.pos[st], gpos + size_t(tile) * kTileF64, kBp, &sm.bar[st]);
      bulk_g2s(sm.val[st], gval + size_t(tile) * kTileF64, kBv, &sm.bar[st]);
    }
  }
  g += ntl;
  if (loc < it.tgt_count) store_partial(a, it.part_off + it.tgt_begin + loc, make_double2(ux, uy));
  return true;
}

template <int NIMG>
__global__ void __launch_bounds__(kThreadsF64) pair_f64_kernel(PairArgs a) {
  __shared__ SmemF64 sm;
  init_barriers(sm.bar);
  ItemDesc it;
  it.tgt_begin = blockIdx.x * kThreadsF64;
  it.tgt_count = min(kThreadsF64, a.n_targets - it.tgt_begin);
  it.vt_begin = blockIdx.y * a.tiles_per_split;
  it.vt_end = min(a.n_tiles, it.vt_begin + a.tiles_per_split);
  it.wb = 0;
  it.nw = a.n_wall_tiles;
  it.vb = a.n_wall_tiles;
  it.part_off = (long long)blockIdx.y * a.n_targets;
  it.period = a.period;
  uint32_t g = 0;
  run_item_f64<NIMG>(a, it, sm, g);
}

template <int NIMG>
__global__ void __launch_bounds__(kThreadsF64) pair_f64_batch_kernel(PairArgs a) {
  __shared__ SmemF64 sm;
  __shared__ int s_item;
  init_barriers(sm.bar);
  uint32_t g = 0;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int k = s_item;
    __syncthreads();
    if (k >= a.n_items) break;
    const ItemDesc it = a.items[k];
    if (!run_item_f64<NIMG>(a, it, sm, g)) return;
  }
}

// ---------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------
typedef void (*PairKernel)(PairArgs);

template <bool BATCH, int NIMG, int TPT, int KG>
PairKernel f32_kernel() {
  if constexpr (BATCH)
    return pair_f32k_batch_kernel<NIMG, TPT, KG>;
  else
    return pair_f32k_kernel<NIMG, TPT, KG>;
}

template <bool BATCH, int NIMG, int TPT>
PairKernel f32_by_kg(int kg) {
  if constexpr (BATCH) {
    return f32_kernel<true, NIMG, TPT, 8>();  // the batched launch always groups by 8
  } else {
    return kg == 1   ? f32_kernel<false, NIMG, TPT, 1>()
           : kg == 2 ? f32_kernel<false, NIMG, TPT, 2>()
           : kg == 8 ? f32_kernel<false, NIMG, TPT, 8>()
           : kg == 16 ? f32_kernel<false, NIMG, TPT, 16>()
                     : f32_kernel<false, NIMG, TPT, 4>();
  }
}

template <bool BATCH, int NIMG>
PairKernel f32_by_tpt(int tpt, int kg) {
  return tpt == 1 ? f32_by_kg<BATCH, NIMG, 1>(kg)
                  : tpt == 2 ? f32_by_kg<BATCH, NIMG, 2>(kg) : f32_by_kg<BATCH, NIMG, 4>(kg);
}

// The FP32 kernel variant for (batched launch?, images?, targets per thread, Kahan group).
PairKernel pick_f32(bool batch, bool img, int tpt, int kg) {
  if (batch) return img ? f32_by_tpt<true, 3>(tpt, kg) : f32_by_tpt<true, 1>(tpt, kg);
  return img ? f32_by_tpt<false, 3>(tpt, kg) : f32_by_tpt<false, 1>(tpt, kg);
}

PairKernel pick_f64(bool batch, bool img) {
  if (batch) return img ? pair_f64_batch_kernel<3> : pair_f64_batch_kernel<1>;
  return img ? pair_f64_kernel<3> : pair_f64_kernel<1>;
}

cudaError_t launch_pair(stokes_ctx *c, int precision, int n_targets, const double2 *tgt,
                        const int2 *skip, int splits, double2 *partial, cudaStream_t s) {
  if (precision == STOKES_DOUBLE_FLOAT)
    return launch_pair_df(c, n_targets, tgt, skip, splits, partial, s);
  PairArgs a{};
  a.n_targets = n_targets;
  a.tgt = tgt;
  a.tgt_skip = skip;
  a.period = c->period;
  a.partial = partial;
  // the context's own buffer has its allocated size; a caller's buffer the splits x targets
  // this launch writes
  a.partial_cap = partial_check_cap(
      c, partial == c->d_partial ? (long long)c->partial_cap : (long long)splits * n_targets,
      (long long)splits * n_targets);
  a.status = c->d_status;
  a.logtab = c->d_logtab;
  const bool img = c->period != 0.0;
  if (precision == STOKES_FP32_KAHAN) {
    a.n_wall_tiles = c->wall_slots / kTileF32;
    a.n_tiles = a.n_wall_tiles + c->ves_slots_f32 / kTileF32;
    a.src_tiles = a.n_tiles;
    a.src_pos = c->d_src_pos32;
    a.src_val = c->d_src_val32;
    a.tiles_per_split = (a.n_tiles + splits - 1) / splits;
    const int eff = (a.n_tiles + a.tiles_per_split - 1) / a.tiles_per_split;
    if (eff != splits) return cudaErrorInvalidValue;  // callers pass effective_splits() values
    // node evaluations (they pass the skip table) take the Morton target order
    a.tgt_perm = skip ? c->d_tgt_perm : nullptr;
    a.local_radius = c->local_frame ? c->local_radius : 0.f;
    const int tpt = c->tpt_f32;
    dim3 grid((n_targets + kThreadsF32 * tpt - 1) / (kThreadsF32 * tpt), eff);
    pick_f32(false, img, tpt, c->kgroup_f32)<<<grid, kThreadsF32, 0, s>>>(a);
  } else {
    a.n_wall_tiles = c->wall_slots_f64 / kTileF64;
    a.n_tiles = a.n_wall_tiles + c->ves_slots_f64 / kTileF64;
    a.src_tiles = a.n_tiles;
    a.src_pos = c->d_src_pos64;
    a.src_val = c->d_src_val64;
    a.tiles_per_split = (a.n_tiles + splits - 1) / splits;
    const int eff = (a.n_tiles + a.tiles_per_split - 1) / a.tiles_per_split;
    if (eff != splits) return cudaErrorInvalidValue;
    dim3 grid((n_targets + kThreadsF64 - 1) / kThreadsF64, eff);
    pick_f64(false, img)<<<grid, kThreadsF64, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// Persistent launch over the context's item table (batched instances): `blocks` resident
// blocks take items in table order (largest first) through a zeroed work counter.
cudaError_t launch_pair_batch(stokes_ctx *c, int precision, int blocks, cudaStream_t s) {
  if (precision == STOKES_DOUBLE_FLOAT) return launch_pair_batch_df(c, blocks, s);
  PairArgs a{};
  a.n_targets = c->N;
  a.tgt = c->d_x;
  a.partial = c->d_partial;
  a.partial_cap = partial_check_cap(c, (long long)c->partial_cap,
                                    precision == STOKES_FP32_KAHAN ? c->batch_part32 : c->batch_part64);
  a.status = c->d_status;
  a.counter = c->d_counter;
  a.logtab = c->d_logtab;
  const bool img = c->period != 0.0;
  cudaError_t e = cudaMemsetAsync(c->d_counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (precision == STOKES_FP32_KAHAN) {
    a.tgt_skip = c->d_tgt_skip32;
    a.src_pos = c->d_src_pos32;
    a.src_val = c->d_src_val32;
    a.src_tiles = (c->wall_slots + c->ves_slots_f32) / kTileF32;
    a.items = c->d_items32;
    a.n_items = c->n_items32;
    a.tgt_perm = c->d_tgt_perm;
    a.local_radius = c->local_frame ? c->local_radius : 0.f;
    pick_f32(true, img, c->tpt_f32, 8)<<<blocks, kThreadsF32, 0, s>>>(a);
  } else {
    a.tgt_skip = c->d_tgt_skip64;
    a.src_pos = c->d_src_pos64;
    a.src_val = c->d_src_val64;
    a.src_tiles = (c->wall_slots_f64 + c->ves_slots_f64) / kTileF64;
    a.items = c->d_items64;
    a.n_items = c->n_items64;
    pick_f64(true, img)<<<blocks, kThreadsF64, 0, s>>>(a);
  }
  return cudaGetLastError();
}

static int occupancy(PairKernel f, int threads) {
  int nb = 0;
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, reinterpret_cast<const void *>(f), threads, 0);
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

// Resident blocks per SM of the pair-kernel variant the context would launch.
int pair_blocks_per_sm(stokes_ctx *c, int precision) {
  if (precision == STOKES_DOUBLE_FLOAT) return pair_df_blocks_per_sm(c);
  const bool img = c->period != 0.0;
  if (precision == STOKES_FP32_KAHAN)
    return occupancy(pick_f32(false, img, c->tpt_f32, c->kgroup_f32), kThreadsF32);
  return occupancy(pick_f64(false, img), kThreadsF64);
}

int pair_batch_blocks_per_sm(stokes_ctx *c, int precision) {
  if (precision == STOKES_DOUBLE_FLOAT) return pair_df_batch_blocks_per_sm(c);
  const bool img = c->period != 0.0;
  if (precision == STOKES_FP32_KAHAN)
    return occupancy(pick_f32(true, img, c->tpt_f32, 8), kThreadsF32);
  return occupancy(pick_f64(true, img), kThreadsF64);
}

// Effective number of splits actually launched for a requested count.
int effective_splits(stokes_ctx *c, int precision, int splits) {
  int n_tiles = (precision == STOKES_FP32_KAHAN)
                    ? (c->wall_slots + c->ves_slots_f32) / kTileF32
                    : (c->wall_slots_f64 + c->ves_slots_f64) / kTileF64;
  if (splits < 1) splits = 1;
  if (splits > n_tiles) splits = n_tiles;
  const int tps = (n_tiles + splits - 1) / splits;
  return (n_tiles + tps - 1) / tps;
}

}  // namespace stokes

