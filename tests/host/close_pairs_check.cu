// Host-logic check of close evaluation (tests/test_host_logic.py): finds the close pairs with
// csrc/close.cu's host search for nv vesicles of n nodes read from a file, emulates the
// resampling and correction kernels on the CPU (the same synthesis and sums) and writes the
// per-node correction for the test to compare with the close oracle.
// Usage: close_pairs_check <case.bin> <out.bin>
//   case.bin: int32 N, n, nv; float64 period, factor; int32 K; nodes (2 N), density (2 N),
//             weights (N); mu = 1.
#include "../../paper_1510_05616_gb300/csrc/close.cu"
#include <cstdio>
using namespace stokes;
namespace stokes { unsigned long long geometry_generation(const stokes_ctx *) { return 0; } }  // linker stub
int main(int argc, char **argv) {
  if (argc < 3) return 2;
  FILE *fp = fopen(argv[1], "rb");
  if (!fp) return 2;
  int hdr[3]; double dd[2]; int K;
  fread(hdr, 4, 3, fp); fread(dd, 8, 2, fp); fread(&K, 4, 1, fp);
  const int N = hdr[0], n = hdr[1], nv = hdr[2];
  std::vector<double2> x(N); std::vector<double> f(2 * N), w(N);
  fread(x.data(), 16, N, fp); fread(f.data(), 8, 2 * N, fp); fread(w.data(), 8, N, fp); fclose(fp);
  std::vector<int> coff(nv + 1), kind(nv, STOKES_KIND_VESICLE);
  for (int v = 0; v <= nv; ++v) coff[v] = v * n;
  ClosePairs cp;
  find_close_pairs(x, coff, kind, dd[0], dd[1], cp);
  printf("pairs %zu targets %zu\n", cp.pairs.size(), cp.tgt.size());
  const double c_slp = 1.0 / (4.0 * kPiC * 1.0);
  const int stride = K * cp.nmax;
  std::vector<double2> fpos(nv * stride), fq(nv * stride);
  for (int vc = 0; vc < int(cp.ves.size()); ++vc) {  // resample_kernel body
    const int nb = coff[cp.ves[vc]], nn = coff[cp.ves[vc] + 1] - nb, nf = K * nn, h = nn / 2;
    std::vector<double> tc(nf), ts(nf), co(8 * (h + 1)), sv(4 * nn);
    for (int j = 0; j < nf; ++j) { tc[j] = cos(kPiC * 2.0 * j / nf); ts[j] = sin(kPiC * 2.0 * j / nf); }
    for (int j = 0; j < nn; ++j) { sv[j] = x[nb + j].x; sv[nn + j] = x[nb + j].y; sv[2 * nn + j] = f[2 * (nb + j)]; sv[3 * nn + j] = f[2 * (nb + j) + 1]; }
    for (int idx = 0; idx < 4 * (h + 1); ++idx) {
      const int s = idx / (h + 1), k = idx - s * (h + 1);
      double a = 0, b = 0;
      for (int j = 0; j < nn; ++j) { const int g = int((long long)k * j * K % nf); a = fma(sv[s * nn + j], tc[g], a); b = fma(sv[s * nn + j], ts[g], b); }
      const double sc = (k == 0 || k == h) ? 1.0 / nn : 2.0 / nn;
      co[(2 * s) * (h + 1) + k] = a * sc; co[(2 * s + 1) * (h + 1) + k] = (k == 0 || k == h) ? 0.0 : b * sc;
    }
    const double dt = 2.0 * kPiC / nf;
    for (int l = 0; l < nf; ++l) {
      double v[4] = {0, 0, 0, 0}, dv[2] = {0, 0};
      for (int k = 0; k <= h; ++k) {
        const int g = int((long long)k * l % nf); const double c = tc[g], s = ts[g];
        for (int q = 0; q < 4; ++q) v[q] = fma(co[(2 * q) * (h + 1) + k], c, fma(co[(2 * q + 1) * (h + 1) + k], s, v[q]));
        for (int q = 0; q < 2; ++q) dv[q] = fma(k * co[(2 * q + 1) * (h + 1) + k], c, fma(-k * co[(2 * q) * (h + 1) + k], s, dv[q]));
      }
      const double sp = sqrt(dv[0] * dv[0] + dv[1] * dv[1]) * dt * c_slp;
      fpos[vc * stride + l] = make_double2(v[0], v[1]); fq[vc * stride + l] = make_double2(v[2] * sp, v[3] * sp);
    }
  }
  std::vector<double2> out(N, make_double2(0, 0));
  auto add = [](double2 z, double px, double py, double q1, double q2, double &ux, double &uy) {
    const double r1 = z.x - px, r2 = z.y - py, rr = r1 * r1 + r2 * r2, lg = -0.5 * log(rr), c = (r1 * q1 + r2 * q2) / rr;
    ux += lg * q1 + c * r1; uy += lg * q2 + c * r2; };
  for (int it = 0; it < int(cp.tgt.size()); ++it) {  // close_kernel body
    const int node = cp.tgt[it]; const double2 z = x[node]; double ux = 0, uy = 0;
    for (int e = cp.off[it]; e < cp.off[it + 1]; ++e) {
      const int2 pm = cp.pairs[e]; const int nb = coff[cp.ves[pm.x]], nn = coff[cp.ves[pm.x] + 1] - nb;
      const double sh = pm.y * dd[0];
      for (int l = 0; l < K * nn; ++l) add(z, fpos[pm.x * stride + l].x + sh, fpos[pm.x * stride + l].y, fq[pm.x * stride + l].x, fq[pm.x * stride + l].y, ux, uy);
      double vx = 0, vy = 0;
      for (int j = 0; j < nn; ++j) { const int i = nb + j; const double c = w[i] * c_slp; add(z, x[i].x + sh, x[i].y, c * f[2 * i], c * f[2 * i + 1], vx, vy); }
      ux -= vx; uy -= vy;
    }
    out[node] = make_double2(ux, uy);
  }
  FILE *fo = fopen(argv[2], "wb");
  if (!fo) return 2;
  fwrite(out.data(), 16, N, fo);
  fclose(fo);
  return 0;
}
