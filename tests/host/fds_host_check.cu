// Host-logic check of the fast direct wall solver (tests/test_host_logic.py): runs the host
// factorization of csrc/fds.cu (HBS tables, neighbour sections) on a wall geometry read from a
// file, emulates the device solve on the CPU with the packed tables (upward pass, root, downward
// pass; R = A_m(J, :) or, recompressed, R = A_m(J, J_c) C from the column sections;
// Z = A_0^-1 L, (I + R Z)^-1, Sherman-Morrison-Woodbury) and writes the solutions of the given
// right-hand sides for the test to check against the oracle's dense operator; prints the
// recompressed R's largest deviation from A_m(J, :) relative to its largest entry.
// Usage: fds_host_check <case.bin> <out.bin> [recompress 0|1, default 1]
//   case.bin: int32 n_w, int32 nrhs; float64 period; nodes (2 N), weights (N), normals (2 N),
//             curvature (N) with N = 2 n_w; right-hand sides (nrhs x 4 n_w).
#include <cstdio>

#include "../../paper_1510_05616_gb300/csrc/fds.cu"

using namespace stokes;

static void hbs_host(const HostFactors &hf, std::vector<double> &v) {  // v <- A_0^-1 v
  const int L = hf.L;
  std::vector<std::vector<double>> up(L + 1), down(L + 1);
  up[L] = v;
  for (int lev = 0; lev < L; ++lev) {
    up[lev].assign(hf.N[lev], 0.0);
    down[lev].assign(hf.N[lev], 0.0);
  }
  down[L].assign(hf.N[L], 0.0);
  for (int lev = L; lev >= 1; --lev)
    for (const HbsBox &b : hf.tabs[lev])
      for (int r = 0; r < b.k; ++r) {
        double s = 0;
        for (int j = 0; j < b.n; ++j) s += hf.mats[b.ft + r + size_t(j) * b.k] * up[lev][b.in_off + j];
        up[lev - 1][b.out_off + r] = s;
      }
  {
    const HbsBox &b = hf.tabs[0][0];
    for (int r = 0; r < b.k; ++r) {
      double s = 0;
      for (int j = 0; j < b.n; ++j) s += hf.mats[b.ft + r + size_t(j) * b.k] * up[0][j];
      down[0][r] = s;
    }
  }
  for (int lev = 1; lev <= L; ++lev)
    for (const HbsBox &b : hf.tabs[lev])
      for (int r = 0; r < b.n; ++r) {
        double s = 0;
        for (int j = 0; j < b.k; ++j) s += hf.mats[b.e + r + size_t(j) * b.n] * down[lev - 1][b.out_off + j];
        for (int j = 0; j < b.n; ++j) s += hf.mats[b.g + r + size_t(j) * b.n] * up[lev][b.in_off + j];
        down[lev][b.in_off + r] = s;
      }
  v = down[L];
}

int main(int argc, char **argv) {
  if (argc < 3) return 2;
  FILE *fp = fopen(argv[1], "rb");
  if (!fp) return 2;
  int hdr[2];
  double d;
  if (fread(hdr, 4, 2, fp) != 2 || fread(&d, 8, 1, fp) != 1) return 2;
  const int nw = hdr[0], nrhs = hdr[1], Nt = 2 * nw, nA = 2 * Nt;
  std::vector<double> nodes(2 * Nt), w(Nt), nrm(2 * Nt), kap(Nt), b(size_t(nrhs) * nA);
  if (fread(nodes.data(), 8, 2 * Nt, fp) != size_t(2 * Nt) || fread(w.data(), 8, Nt, fp) != size_t(Nt) ||
      fread(nrm.data(), 8, 2 * Nt, fp) != size_t(2 * Nt) || fread(kap.data(), 8, Nt, fp) != size_t(Nt) ||
      fread(b.data(), 8, b.size(), fp) != b.size())
    return 2;
  fclose(fp);
  fds_params p;
  p.recompress = argc < 4 || argv[3][0] != '0';
  HostFactors hf;
  std::string err;
  if (host_factor(nw, nodes.data(), w.data(), nrm.data(), kap.data(), d, p, hf, err) != STOKES_OK) {
    printf("host_factor failed: %s\n", err.c_str());
    return 1;
  }
  const WallGeom &g = hf.g;
  const int l = int(hf.Jall.size());
  HMat Lm(nA, l), R(l, nA);
  for (const SecBlock &sb : hf.sb)
    for (int c = 0; c < sb.cols; ++c)
      for (int i = 0; i < sb.rows; ++i) Lm(sb.row0 + i, sb.col0 + c) = hf.svals[sb.off + i + size_t(c) * sb.rows];
  for (int u = 0; u < nA; ++u)
    for (int r = 0; r < l; ++r) R(r, u) = a_host(g, hf.Jall[r], u, hf.mall[r]);
  const int lc = int(hf.Jc.size());
  double r_dev = 0.0;
  if (lc > 0) {  // R <- S C
    HMat S(l, lc), C(lc, nA);
    for (int c = 0; c < lc; ++c)
      for (int r = 0; r < l; ++r)
        S(r, c) = hf.mall[r] == hf.mc[c] ? a_host(g, hf.Jall[r], hf.Jc[c], hf.mall[r]) : 0.0;
    for (const SecBlock &sb : hf.csb)
      for (int c = 0; c < sb.cols; ++c)
        for (int i = 0; i < sb.rows; ++i) C(sb.col0 + c, sb.row0 + i) = hf.cvals[sb.off + i + size_t(c) * sb.rows];
    HMat SC = mul(S, C);
    double big = 0.0, dev = 0.0;
    for (size_t q = 0; q < R.a.size(); ++q) {
      big = std::max(big, fabs(R.a[q]));
      dev = std::max(dev, fabs(R.a[q] - SC.a[q]));
    }
    r_dev = dev / big;
    R = SC;
  }
  HMat Z = Lm;
  for (int c = 0; c < l; ++c) {
    std::vector<double> col(Z.col(c), Z.col(c) + nA);
    hbs_host(hf, col);
    std::copy(col.begin(), col.end(), Z.col(c));
  }
  HMat K = mul(R, Z);
  for (int i = 0; i < l; ++i) K(i, i) += 1.0;
  if (!invert(K)) return 1;
  FILE *fo = fopen(argv[2], "wb");
  if (!fo) return 2;
  for (int q = 0; q < nrhs; ++q) {
    std::vector<double> x(b.begin() + size_t(q) * nA, b.begin() + size_t(q + 1) * nA);
    hbs_host(hf, x);
    std::vector<double> t(l, 0.0), s(l, 0.0);
    for (int r = 0; r < l; ++r) {
      double acc = 0;
      for (int u = 0; u < nA; ++u) acc += R(r, u) * x[u];
      t[r] = acc;
    }
    for (int r = 0; r < l; ++r) {
      double acc = 0;
      for (int c = 0; c < l; ++c) acc += K(r, c) * t[c];
      s[r] = acc;
    }
    for (int u = 0; u < nA; ++u) {
      double acc = 0;
      for (int c = 0; c < l; ++c) acc += Z(u, c) * s[c];
      x[u] -= acc;
    }
    fwrite(x.data(), 8, nA, fo);
  }
  fclose(fo);
  printf("levels %d max_rank %d root %d neighbour_rank %d sections %d col_rank %d r_dev %.3e\n",
         hf.info.levels, hf.info.max_rank, hf.info.root_size, hf.info.neighbour_rank,
         hf.info.sections, hf.info.neighbour_col_rank, r_dev);
  return 0;
}
