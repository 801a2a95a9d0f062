// k_field.cu -- pressure and traction of the near-image layer potentials at free points, FP64.
//
// At targets off the curves (plain trapezoid rule, nothing skipped), over the images
// m in {-1, 0, +1} and every source slot:
//   pressure  Eq. (Q) for stokeslet sources, Eq. (P) for stresslet sources;
//   traction  Eq. (K) for stokeslet sources, Eq. (T) for stresslet sources, with the target
//             normal n_x given per target and the dipole functions d_x = (r . n_x) / r^2,
//             d_y = (r . n_y) / r^2 (the reading under which Eq. (T) is the traction of the
//             (D, P) pair).
// The source records are the FP64 pair kernel's: q = w f / (4 pi mu) for a stokeslet source,
// q = w tau / pi with the source normal n for a stresslet source, so per source and image
//   stokeslet   p += 2 mu (r . q) / r^2           t += -4 mu r (r . q)(r . n_x) / r^4
//   stresslet   p += mu (-(n . q) / r^2 + 2 (r . n)(r . q) / r^4)
//               t += mu [ (n . n_x / r^2 - 8 d_x d_y) r (r . q) / r^2 + d_x d_y q
//                         + n_x (n . q) / r^2 + d_x (r . q) n / r^2 + d_y r (n_x . q) / r^2 ].
// One thread per target; the block stages 64-source tiles (one kind each) in shared memory;
// source splits over blockIdx.y write FP64 partials that are reduced in fixed order.
#include <algorithm>

#include "stokes_internal.cuh"

namespace stokes {

constexpr int kFieldThreads = 128;

template <int NIMG, bool TRACTION>
__global__ void __launch_bounds__(kFieldThreads)
    field_f64_kernel(int n_targets, const double2 *tgt, const double2 *tnrm, int n_tiles,
                     int n_wall_tiles, int tiles_per_split, const double2 *src_pos,
                     const double4_32a *src_val, double period, double mu, double2 *partial) {
  __shared__ double2 sp[kTileF64];
  __shared__ double4_32a sv[kTileF64];
  const int i = blockIdx.x * kFieldThreads + threadIdx.x;
  const int ic = min(i, n_targets - 1);
  const double2 x = tgt[ic];
  const double2 nx = TRACTION ? tnrm[ic] : make_double2(0.0, 0.0);
  double a1 = 0.0, a2 = 0.0;
  const int t0 = blockIdx.y * tiles_per_split;
  const int t1 = min(n_tiles, t0 + tiles_per_split);
  for (int tile = t0; tile < t1; ++tile) {
    __syncthreads();
    for (int k = threadIdx.x; k < kTileF64; k += kFieldThreads) {
      sp[k] = src_pos[size_t(tile) * kTileF64 + k];
      sv[k] = src_val[size_t(tile) * kTileF64 + k];
    }
    __syncthreads();
    const bool wall = tile < n_wall_tiles;  // uniform: tiles hold one kind
    for (int j = 0; j < kTileF64; ++j) {
      const double2 y = sp[j];
      const double4_32a v = sv[j];
#pragma unroll
      for (int k = 0; k < NIMG; ++k) {
        const double m = (NIMG == 3) ? double(k - 1) : 0.0;
        const double r1 = x.x - (y.x + m * period), r2 = x.y - y.y;
        // the floor keeps padding slots (q = 0 at the origin) finite at a target on the origin
        const double inv = 1.0 / fmax(r1 * r1 + r2 * r2, 1e-150);
        const double rq = r1 * v.x + r2 * v.y;
        if (!TRACTION) {
          if (wall) {
            const double rn = r1 * v.z + r2 * v.w;
            a1 += mu * (2.0 * rn * rq * inv - (v.z * v.x + v.w * v.y)) * inv;
          } else {
            a1 += 2.0 * mu * rq * inv;
          }
        } else {
          const double rnx = r1 * nx.x + r2 * nx.y;
          if (wall) {
            const double dx = rnx * inv, dy = (r1 * v.z + r2 * v.w) * inv;
            const double nn = v.z * nx.x + v.w * nx.y;
            const double nq = v.z * v.x + v.w * v.y;
            const double nxq = nx.x * v.x + nx.y * v.y;
            const double cr = ((nn * inv - 8.0 * dx * dy) * rq + dy * nxq) * inv;  // along r
            const double cd = dx * dy;                                              // along q
            const double cn = nq * inv;                                             // along n_x
            const double cy = dx * rq * inv;                                        // along n
            a1 += mu * (cr * r1 + cd * v.x + cn * nx.x + cy * v.z);
            a2 += mu * (cr * r2 + cd * v.y + cn * nx.y + cy * v.w);
          } else {
            const double c = -4.0 * mu * rq * rnx * inv * inv;
            a1 += c * r1;
            a2 += c * r2;
          }
        }
      }
    }
  }
  if (i < n_targets) partial[size_t(blockIdx.y) * n_targets + i] = make_double2(a1, a2);
}

// out[t] (pressure) or out[2t], out[2t + 1] (traction): fixed-order sum over the splits.
__global__ void field_finish_kernel(int n_targets, int splits, int comps, const double2 *partial,
                                    double *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_targets) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < splits; ++k) {
    const double2 p = partial[size_t(k) * n_targets + t];
    a += p.x;
    b += p.y;
  }
  if (comps == 1) {
    out[t] = a;
  } else {
    out[2 * t] = a;
    out[2 * t + 1] = b;
  }
}

// Source splits of a field launch: about eight blocks per SM in all.
int field_splits(const stokes_ctx *c, int n_targets) {
  const int n_tiles = (c->wall_slots_f64 + c->ves_slots_f64) / kTileF64;
  const int tb = (n_targets + kFieldThreads - 1) / kFieldThreads;
  const int want = (8 * std::max(c->num_sms, 1) + tb - 1) / tb;
  const int sp = std::max(1, std::min(want, n_tiles));
  const int tps = (n_tiles + sp - 1) / sp;
  return std::max(1, (n_tiles + tps - 1) / tps);
}

// Pressure (tnrm == NULL) or traction at n_targets free points; the FP64 source records must
// be packed and c->d_partial must hold splits x n_targets elements.
cudaError_t launch_field(stokes_ctx *c, int n_targets, const double2 *tgt, const double2 *tnrm,
                         int splits, double *out, cudaStream_t s) {
  const int n_wall_tiles = c->wall_slots_f64 / kTileF64;
  const int n_tiles = n_wall_tiles + c->ves_slots_f64 / kTileF64;
  const int tps = (n_tiles + splits - 1) / splits;
  const int eff = (n_tiles + tps - 1) / tps;
  if (eff != splits) return cudaErrorInvalidValue;  // callers pass field_splits() values
  const dim3 grid((n_targets + kFieldThreads - 1) / kFieldThreads, eff);
  const bool img = c->period != 0.0;
  auto k = tnrm ? (img ? field_f64_kernel<3, true> : field_f64_kernel<1, true>)
                : (img ? field_f64_kernel<3, false> : field_f64_kernel<1, false>);
  k<<<grid, kFieldThreads, 0, s>>>(n_targets, tgt, tnrm, n_tiles, n_wall_tiles, tps,
                                   c->d_src_pos64, c->d_src_val64, c->period, c->mu,
                                   c->d_partial);
  field_finish_kernel<<<(n_targets + 255) / 256, 256, 0, s>>>(n_targets, eff, tnrm ? 2 : 1,
                                                              c->d_partial, out);
  return cudaGetLastError();
}

}  // namespace stokes
