// Host-logic check of the FMM (tests/test_host_logic.py): builds the plan of csrc/fmm.cu from a
// geometry file, checks its invariants, emulates every pass on the CPU with the plan's arrays
// (the same expansions and conversions, the conj(w)-weighted charge sets kept relative to each
// expansion's centre and re-centred at every shift and conversion) and writes the far + near
// sum for the test to compare with a direct sum.
// Usage: fmm_plan_check <case.bin> <order> <leaf> <out.bin>
#include "../../paper_1510_05616_gb300/csrc/fmm.cu"
#include <complex>
#include <cstdio>
#include <cstdlib>
using namespace stokes;
typedef std::complex<double> cd;
namespace stokes {  // unused on the CPU: stubs for the linker
cudaError_t launch_pack(stokes_ctx *, int, const double *, const double *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_finish_nodes(stokes_ctx *, int, const double *, const double *, double, double2 *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_self(stokes_ctx *, const double *, cudaStream_t) { return cudaErrorNotSupported; }
void invalidate_node_graph(stokes_ctx *) {}
}

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  double r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

int main(int argc, char **argv) {
  if (argc < 5) return 2;
  const int p = atoi(argv[2]), leaf = atoi(argv[3]);
  FILE *fp = fopen(argv[1], "rb");
  if (!fp) return 2;
  int hdr[3];
  double d;
  fread(hdr, 4, 3, fp);
  fread(&d, 8, 1, fp);
  const int N = hdr[0], slots = hdr[1], wall_slots = hdr[2];
  std::vector<double2> x(N);
  std::vector<int> order(slots);
  std::vector<double> vals(4 * N);
  fread(x.data(), 16, N, fp);
  fread(order.data(), 4, slots, fp);
  fread(vals.data(), 8, 4 * N, fp);
  fclose(fp);
  std::vector<double2> spos(slots);
  std::vector<int> snode(slots);
  std::vector<double> sval(4 * slots, 0.0);
  for (int s = 0; s < slots; ++s) {
    snode[s] = order[s];
    spos[s] = order[s] >= 0 ? x[order[s]] : make_double2(0.0, 0.0);
    if (order[s] >= 0)
      for (int k = 0; k < 4; ++k) sval[4 * s + k] = vals[4 * order[s] + k];
  }
  PlanHost ph;
  std::vector<int> ncur(N, -1);
  plan_host(x, spos, snode, ncur, d, leaf, ph);
  const int L = ph.L, ns = ph.ns;
  printf("L %d roots %d x %d sources %d source cells %d target cells %d tleaves %d il %zu near %lld\n",
         L, ph.nx, ph.ny, ns, ph.sc_off[L + 1], ph.tc_off[L + 1], ph.n_tleaf, ph.il_idx.size(), ph.near_pairs);
  // ---- invariants
  int bad = 0;
  const int nsc = ph.sc_off[L + 1], ntc = ph.tc_off[L + 1];
  {
    int cur = 0;
    for (int i = ph.sc_off[L]; i < nsc; ++i) {
      if (ph.sc_rng[i].x != cur || ph.sc_rng[i].y <= ph.sc_rng[i].x) ++bad;
      cur = ph.sc_rng[i].y;
    }
    if (cur != ns) ++bad;
    for (int l = 0; l < L; ++l)
      for (int i = ph.sc_off[l]; i < ph.sc_off[l + 1]; ++i) {
        const int2 r = ph.sc_rng[i];
        if (r.x < ph.sc_off[l + 1] || r.y > ph.sc_off[l + 2] || r.y <= r.x || r.y - r.x > 4) ++bad;
      }
    for (int i = 0; i < ntc; ++i) {
      const int l = int(std::upper_bound(ph.tc_off.begin(), ph.tc_off.end(), i) - ph.tc_off.begin()) - 1;
      if (l == 0 ? ph.tc_par[i] != -1 : (ph.tc_par[i] < ph.tc_off[l - 1] || ph.tc_par[i] >= ph.tc_off[l])) ++bad;
      for (int e = ph.il_off[i]; e < ph.il_off[i + 1]; ++e)
        if (ph.il_idx[e] < ph.sc_off[l] || ph.il_idx[e] >= ph.sc_off[l + 1]) ++bad;
    }
    int tc = 0;
    for (int t = 0; t < ph.n_tleaf; ++t) {
      if (ph.tleaf_rng[t].x != tc) ++bad;
      tc = ph.tleaf_rng[t].y;
      for (int e = ph.nl_off[t]; e < ph.nl_off[t + 1]; ++e)
        if (ph.nl_idx[e] < ph.sc_off[L] || ph.nl_idx[e] >= nsc) ++bad;
    }
    if (tc != N) ++bad;
    std::vector<int> seen(N, 0);
    for (int i : ph.tord) seen[i]++;
    for (int i = 0; i < N; ++i) if (seen[i] != 1) ++bad;
    if (ph.tc_off[L + 1] - ph.tc_off[L] != ph.n_tleaf) ++bad;
    for (int j = 0; j < ns; ++j) if (snode[ph.src_sorted[j].x] < 0) ++bad;
  }
  printf("invariant violations: %d\n", bad);
  // ---- emulated passes
  const int p1 = p + 1;
  // charges of source j with the conj(w)-weighted sets 2 and 5 relative to the centre ctr
  auto charges_h = [&](int j, cd ctr, cd (&c)[kSets]) {
    const int s = ph.src_sorted[j].x;
    const cd w = cd(ph.pos_sorted[j].x, ph.pos_sorted[j].y) - ctr;
    const double *v = &sval[4 * s];
    for (auto &q : c) q = 0;
    if (s >= wall_slots) {
      const cd q(v[0], v[1]);
      c[0] = v[0]; c[1] = v[1]; c[2] = std::conj(w) * q;
    } else {
      const cd T(v[0], v[1]), nu(v[2], v[3]);
      c[3] = 2.0 * (v[2] * v[0] + v[3] * v[1]); c[4] = nu * T; c[5] = nu * T * std::conj(w);
    }
  };
  auto hl = [&](int l) { return ph.S / double(1 << l); };
  // the kSets x p1 coefficients at e, sets 2 and 5 moved from their centre by dc = old - new:
  // they gain conj(dc) times the q = q1 + i q2 (set 2) or nu T (set 5) coefficients
  auto recentre = [&](const cd *e, cd dc, std::vector<cd> &out) {
    out.assign(e, e + kSets * p1);
    for (int k = 0; k <= p; ++k) {
      out[2 * p1 + k] += std::conj(dc) * (e[k] + cd(0, 1) * e[p1 + k]);
      out[5 * p1 + k] += std::conj(dc) * e[4 * p1 + k];
    }
  };
  std::vector<cd> rc;
  std::vector<cd> M(size_t(nsc) * kSets * p1, 0.0), Lc(size_t(ntc) * kSets * p1, 0.0);
  for (int i = ph.sc_off[L]; i < nsc; ++i) {
    const cd ctr(ph.sc_ctr[i].x, ph.sc_ctr[i].y);
    for (int j = ph.sc_rng[i].x; j < ph.sc_rng[i].y; ++j) {
      cd c[kSets];
      charges_h(j, ctr, c);
      const cd u = (cd(ph.pos_sorted[j].x, ph.pos_sorted[j].y) - ctr) / hl(L);
      for (int s = 0; s < kSets; ++s) {
        M[(size_t(i) * kSets + s) * p1] += c[s];
        cd uk = 1.0;
        for (int k = 1; k <= p; ++k) { uk *= u; M[(size_t(i) * kSets + s) * p1 + k] -= c[s] * uk / double(k); }
      }
    }
  }
  for (int l = L - 1; l >= 0; --l)
    for (int i = ph.sc_off[l]; i < ph.sc_off[l + 1]; ++i) {
      const cd c0(ph.sc_ctr[i].x, ph.sc_ctr[i].y);
      for (int ch = ph.sc_rng[i].x; ch < ph.sc_rng[i].y; ++ch) {
        const cd cc(ph.sc_ctr[ch].x, ph.sc_ctr[ch].y);
        const cd s = (cc - c0) / hl(l);
        recentre(&M[size_t(ch) * kSets * p1], cc - c0, rc);
        for (int st = 0; st < kSets; ++st) {
          const cd *a = &rc[size_t(st) * p1];
          cd *b = &M[(size_t(i) * kSets + st) * p1];
          b[0] += a[0];
          for (int q = 1; q <= p; ++q) {
            cd acc = -a[0] * std::pow(s, q) / double(q);
            for (int k = 1; k <= q; ++k) acc += a[k] * std::pow(0.5, k) * std::pow(s, q - k) * binom(q - 1, k - 1);
            b[q] += acc;
          }
        }
      }
    }
  for (int l = 0; l <= L; ++l)
    for (int i = ph.tc_off[l]; i < ph.tc_off[l + 1]; ++i) {
      const cd ct(ph.tc_ctr[i].x, ph.tc_ctr[i].y);
      const double h = hl(l);
      for (int st = 0; st < kSets; ++st) {
        cd *b = &Lc[(size_t(i) * kSets + st) * p1];
        if (ph.tc_par[i] >= 0) {
          const int pr = ph.tc_par[i];
          const cd cp(ph.tc_ctr[pr].x, ph.tc_ctr[pr].y);
          const cd s = (ct - cp) / (2 * h);
          recentre(&Lc[size_t(pr) * kSets * p1], cp - ct, rc);
          const cd *pb = &rc[size_t(st) * p1];
          for (int q = 0; q <= p; ++q) {
            cd acc = 0;
            for (int k = q; k <= p; ++k) acc += pb[k] * binom(k, q) * std::pow(s, k - q);
            b[q] += acc * std::pow(0.5, q);
          }
        }
        for (int e = ph.il_off[i]; e < ph.il_off[i + 1]; ++e) {
          const int sc = ph.il_idx[e];
          const cd cs(ph.sc_ctr[sc].x, ph.sc_ctr[sc].y);
          const cd t = (cs - ct) / h;
          recentre(&M[size_t(sc) * kSets * p1], cs - ct, rc);
          const cd *a = &rc[size_t(st) * p1];
          b[0] += a[0] * (std::log(-t) + std::log(h));
          for (int k = 1; k <= p; ++k) b[0] += a[k] * (k & 1 ? -1.0 : 1.0) / std::pow(t, k);
          for (int q = 1; q <= p; ++q) {
            cd acc = -a[0] / double(q);
            for (int k = 1; k <= p; ++k) acc += a[k] / std::pow(t, k) * binom(q + k - 1, k - 1) * (k & 1 ? -1.0 : 1.0);
            b[q] += acc / std::pow(t, q);
          }
        }
      }
    }
  // leaves: far field + near field, then the direct sum for comparison
  cd qtot = 0;
  for (int r = ph.sc_off[0]; r < ph.sc_off[1]; ++r)
    qtot += cd(M[(size_t(r) * kSets + 0) * p1].real(), M[(size_t(r) * kSets + 1) * p1].real());
  std::vector<cd> uf(N);
  for (int t = 0; t < ph.n_tleaf; ++t) {
    const int cell = ph.tc_off[L] + t;
    const cd ct(ph.tc_ctr[cell].x, ph.tc_ctr[cell].y);
    const double h = hl(L);
    for (int it = ph.tleaf_rng[t].x; it < ph.tleaf_rng[t].y; ++it) {
      const int node = ph.tord[it];
      const cd z(x[node].x, x[node].y), u = (z - ct) / h;
      cd v[kSets], d1[kSets], d2[kSets];
      for (int s = 0; s < kSets; ++s) {
        const cd *b = &Lc[(size_t(cell) * kSets + s) * p1];
        v[s] = d1[s] = d2[s] = 0;
        for (int k = 0; k <= p; ++k) {
          v[s] += b[k] * std::pow(u, k);
          if (k >= 1) d1[s] += double(k) * b[k] * std::pow(u, k - 1) / h;
          if (k >= 2) d2[s] += double(k * (k - 1)) * b[k] * std::pow(u, k - 2) / (h * h);
        }
      }
      cd near = 0, qn = 0;
      for (int e = ph.nl_off[t]; e < ph.nl_off[t + 1]; ++e)
        for (int j = ph.sc_rng[ph.nl_idx[e]].x; j < ph.sc_rng[ph.nl_idx[e]].y; ++j) {
          const int s = ph.src_sorted[j].x;
          const double *vv = &sval[4 * s];
          const bool wall = s < wall_slots;
          if (!wall) qn += cd(vv[0], vv[1]);
          const double r1 = z.real() - ph.pos_sorted[j].x, r2 = z.imag() - ph.pos_sorted[j].y, rr = r1 * r1 + r2 * r2;
          if (rr == 0) continue;
          if (!wall) {
            const double lg = -0.5 * log(rr), c = (r1 * vv[0] + r2 * vv[1]) / rr;
            near += cd(lg * vv[0] + c * r1, lg * vv[1] + c * r2);
          } else {
            const double c = (r1 * vv[2] + r2 * vv[3]) * (r1 * vv[0] + r2 * vv[1]) / (rr * rr);
            near += cd(c * r1, c * r2);
          }
        }
      const cd dq = d1[0] + cd(0, 1) * d1[1];
      const cd zo = z - ct;  // sets 2 and 5 are centred at the leaf's centre
      cd s = cd(-v[0].real(), -v[1].real()) + 0.5 * (qtot - qn) + 0.5 * (zo * std::conj(dq) - std::conj(d1[2]));
      s += 0.25 * (d1[4] + std::conj(d1[3]) + std::conj(d2[5] - std::conj(zo) * d2[4]));
      uf[node] = s + near;
    }
  }
  FILE *fo = fopen(argv[4], "wb");
  if (!fo) return 2;
  for (int i = 0; i < N; ++i) {
    const double v[2] = {uf[i].real(), uf[i].imag()};
    fwrite(v, sizeof(double), 2, fo);
  }
  fclose(fo);
  printf("levels %d sources %d m2l %zu near %lld invariant_violations %d\n", L, ns, ph.il_idx.size(),
         ph.near_pairs, bad);
  return bad != 0;
}
