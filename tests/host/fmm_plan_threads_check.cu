// Host check of the FMM plan build's threads (tests/test_host_logic.py): the key order of the
// plan (an LSD radix sort) equals std::stable_sort's on seeded keys -- many ties, keys up to 64
// bits, empty and single inputs; then builds the plan of csrc/fmm.cu for seeded random
// geometries -- small and large, periodic and not, with padding slots and free curve ids -- on
// one host thread and on 2, 3 and 4, and checks that every array of the plan is the same bit
// for bit.  Usage: fmm_plan_threads_check [cases, default 6]
#include "../../paper_1510_05616_gb300/csrc/fmm.cu"
#include <cstdio>
#include <cstring>
#include <random>
using namespace stokes;
namespace stokes {  // unused on the CPU: stubs for the linker
cudaError_t launch_pack(stokes_ctx *, int, const double *, const double *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_finish_nodes(stokes_ctx *, int, const double *, const double *, double, double2 *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_self(stokes_ctx *, const double *, cudaStream_t) { return cudaErrorNotSupported; }
void invalidate_node_graph(stokes_ctx *) {}
}

template <class T>
static bool same(const std::vector<T> &a, const std::vector<T> &b) {
  return a.size() == b.size() && (a.empty() || memcmp(a.data(), b.data(), sizeof(T) * a.size()) == 0);
}

static bool same_plan(const PlanHost &a, const PlanHost &b) {
  return a.L == b.L && a.nx == b.nx && a.ny == b.ny && a.N == b.N && a.ns == b.ns &&
         a.n_tleaf == b.n_tleaf && memcmp(&a.x0, &b.x0, 8) == 0 && memcmp(&a.y0, &b.y0, 8) == 0 &&
         memcmp(&a.S, &b.S, 8) == 0 && a.near_pairs == b.near_pairs && same(a.sc_off, b.sc_off) &&
         same(a.tc_off, b.tc_off) && same(a.tc_par, b.tc_par) && same(a.il_off, b.il_off) &&
         same(a.il_idx, b.il_idx) && same(a.nl_off, b.nl_off) && same(a.nl_idx, b.nl_idx) &&
         same(a.tord, b.tord) && same(a.src_sorted, b.src_sorted) && same(a.sc_rng, b.sc_rng) &&
         same(a.tleaf_rng, b.tleaf_rng) && same(a.src_own, b.src_own) &&
         same(a.pos_sorted, b.pos_sorted) && same(a.sc_ctr, b.sc_ctr) && same(a.tc_ctr, b.tc_ctr);
}

// order_by_key against the stable sort it stands for
static bool radix_matches_stable_sort() {
  std::mt19937_64 rng(11);
  const int sizes[] = {0, 1, 2, 7, 1000, 65537, 300000};
  const int bits[] = {1, 5, 12, 22, 38, 64};
  for (int n : sizes)
    for (int b : bits) {
      std::vector<unsigned long long> key(n);
      for (auto &k : key) k = b == 64 ? rng() : rng() & ((1ull << b) - 1);
      std::vector<int> ref(n);
      for (int i = 0; i < n; ++i) ref[i] = i;
      std::stable_sort(ref.begin(), ref.end(), [&](int a, int c) { return key[a] < key[c]; });
      if (order_by_key(key) != ref) {
        printf("MISMATCH order_by_key n %d bits %d\n", n, b);
        return false;
      }
    }
  printf("ok: order_by_key equals std::stable_sort (%zu sizes x %zu key widths)\n",
         sizeof(sizes) / sizeof(sizes[0]), sizeof(bits) / sizeof(bits[0]));
  return true;
}

int main(int argc, char **argv) {
  const int n_cases = argc > 1 ? std::max(1, std::min(6, atoi(argv[1]))) : 6;
  if (!radix_matches_stable_sort()) return 1;
  const double d = 2 * M_PI;
  std::mt19937 rng(7);
  std::uniform_real_distribution<double> U(0, 1);
  const int n_targets[] = {100, 3000, 5000, 40000, 130000, 70000};
  const int n_slots[] = {80, 2000, 9000, 33000, 100000, 200000};
  int checked = 0;
  for (int cs = 0; cs < n_cases; ++cs) {
    const int nt = n_targets[cs], nsl = n_slots[cs];
    std::vector<double2> x(nt), spos(nsl);
    std::vector<int> snode(nsl), curve(nt);
    for (int i = 0; i < nt; ++i) {  // odd cases: targets along a curve, even: in a box
      const double t = U(rng);
      x[i] = cs % 2 ? make_double2(d * t, 0.9 * sin(7 * t) + 0.05 * U(rng))
                    : make_double2(d * U(rng), 2 * U(rng) - 1);
      curve[i] = (i / 128) % 5 == 0 ? -1 : i / 128;
    }
    for (int s = 0; s < nsl; ++s) {
      spos[s] = make_double2(d * U(rng), 2 * U(rng) - 1);
      snode[s] = (s % 11 == 3) ? -1 : int(rng() % nt);  // every 11th slot padding
    }
    const double period = cs == 5 ? 0.0 : d;
    for (int leaf : {8, 32}) {
      PlanHost one;
      plan_host(x, spos, snode, curve, period, leaf, one, 1);
      for (int threads = 2; threads <= kPlanThreads; ++threads) {
        PlanHost many;
        plan_host(x, spos, snode, curve, period, leaf, many, threads);
        if (!same_plan(one, many)) {
          printf("MISMATCH case %d leaf %d threads %d\n", cs, leaf, threads);
          return 1;
        }
        ++checked;
      }
      printf("case %d leaf %d: %d sources, %d target cells, %zu conversions, %lld near pairs\n", cs,
             leaf, one.ns, one.tc_off[one.L + 1], one.il_idx.size(), one.near_pairs);
    }
  }
  printf("ok: %d threaded plans identical to the one-thread plan\n", checked);
  return 0;
}
