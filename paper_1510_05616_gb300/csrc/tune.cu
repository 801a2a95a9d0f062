// tune.cu -- launch-shape autotuner of the pair sum, and the process-wide table of tuned shapes
// by geometry size class.  Host code only: it drives the library's own entry points and times
// them with CUDA events on the caller's stream.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "stokes_internal.cuh"

namespace stokes {
int effective_splits(stokes_ctx *c, int precision, int splits);  // k_pair.cu
std::vector<int> ranked_splits(stokes_ctx *c, int precision, int k);  // stokes_abi.cu
}  // namespace stokes

namespace {

// Size class: SM count, precision, then half-octave buckets of the instance count and of the
// total, wall and vesicle node counts.
using Key = std::array<int, 6>;

struct Shape {
  int splits, tpt, kg, ips;
};

struct Entry {
  Shape shape;
  double ms;
};

std::mutex g_mu;
std::map<Key, Entry> g_table;

int bucket(long long x) { return x <= 0 ? -1 : int(ceil(2.0 * log2(double(x)) - 1e-9)); }

Key make_key(int sms, int prec, long long n_inst, long long n, long long nw, long long nv) {
  return Key{sms, prec, bucket(n_inst), bucket(n), bucket(nw), bucket(nv)};
}

Key ctx_key(const stokes_ctx *c, int prec) {
  return make_key(c->num_sms, prec, c->n_inst, c->N, c->n_wall_nodes, c->n_ves_nodes);
}

bool valid_prec(int p) {
  return p == STOKES_FP64 || p == STOKES_FP32_KAHAN || p == STOKES_DOUBLE_FLOAT;
}

bool valid_shape(int prec, const Shape &s) {
  const bool tpt_ok = prec == STOKES_FP32_KAHAN ? (s.tpt == 1 || s.tpt == 2 || s.tpt == 4)
                                                : s.tpt >= 1;
  const bool kg_ok = s.kg == 0 || s.kg == 1 || s.kg == 2 || s.kg == 4 || s.kg == 8 || s.kg == 16;
  return tpt_ok && kg_ok && s.splits >= 0 && s.ips >= 0 && s.ips <= 64;
}

int tfail(stokes_ctx *c, int code, const char *msg) {
  c->err = msg;
  return code;
}

int tcuda(stokes_ctx *c, cudaError_t e, const char *where) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  c->err = buf;
  return e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA;
}

Shape current_shape(stokes_ctx *c, int prec) {
  Shape s{0, 0, 0, 0};
  if (c->n_inst > 1) {
    int n_items = 0, blocks = 0;
    stokes_batch_info(c, prec, &n_items, &blocks, &s.tpt, &s.ips);
  } else {
    stokes_get_launch(c, prec, &s.splits, &s.tpt, &s.kg);
  }
  return s;
}

int apply_shape(stokes_ctx *c, int prec, const Shape &s) {
  const bool f32 = prec == STOKES_FP32_KAHAN;
  if (c->n_inst > 1) return stokes_batch_set_shape(c, prec, f32 ? s.tpt : 0, s.ips);
  return stokes_set_launch(c, prec, s.splits, f32 ? s.tpt : 0, f32 ? s.kg : 0);
}

bool same_shape(const Shape &a, const Shape &b) {
  return a.splits == b.splits && a.tpt == b.tpt && a.kg == b.kg && a.ips == b.ips;
}

// Split counts to time for one shape: the wave model's three cheapest, two and four times its
// cheapest (finer work units balance uneven tiles better than the model, which costs every tile
// the same, predicts), and the counts whose blocks fill exactly one or two waves of the resident
// slots (fewest, longest blocks for that many waves), as effective counts without repeats.
std::vector<int> split_candidates(stokes_ctx *c, int prec, int k) {
  std::vector<int> sp = stokes::ranked_splits(c, prec, k);
  auto add = [&](int want) {
    const int e = stokes::effective_splits(c, prec, want);
    if (std::find(sp.begin(), sp.end(), e) == sp.end()) sp.push_back(e);
  };
  if (!sp.empty()) {
    const int best = sp[0];
    for (int f : {2, 4}) add(best * f);
  }
  const bool f32 = prec == STOKES_FP32_KAHAN;
  const long per_block = f32 ? long(stokes::kThreadsF32) * c->tpt_f32
                             : prec == STOKES_DOUBLE_FLOAT ? long(stokes::kThreadsDF) * stokes::kTptDF
                                                           : long(stokes::kThreadsF64);
  const long tb = (c->N + per_block - 1) / per_block;
  const long slots = long(stokes::pair_blocks_per_sm(c, prec)) * std::max(c->num_sms, 1);
  for (int waves : {1, 2}) add(int(std::max(1L, (waves * slots) / std::max(tb, 1L))));
  return sp;
}

std::vector<Shape> candidates(stokes_ctx *c, int prec, const Shape &initial) {
  std::vector<Shape> out;
  const bool f32 = prec == STOKES_FP32_KAHAN;
  if (c->n_inst > 1) {
    const std::vector<int> tpts = f32 ? std::vector<int>{1, 2, 4} : std::vector<int>{initial.tpt};
    for (int t : tpts)
      for (int ips : {1, 2, 4, 8, 16}) out.push_back(Shape{0, t, 0, ips});
  } else if (f32) {
    const int saved = c->tpt_f32;
    for (int t : {1, 2, 4}) {
      c->tpt_f32 = t;  // the wave model sizes target blocks by targets per thread
      const std::vector<int> sp = split_candidates(c, prec, 3);
      for (int kg : {2, 4, 8, 16})
        for (int s : sp) out.push_back(Shape{s, t, kg, 0});
    }
    c->tpt_f32 = saved;
  } else {
    for (int s : split_candidates(c, prec, 3)) out.push_back(Shape{s, initial.tpt, 0, 0});
  }
  bool have = false;
  for (const auto &s : out) have = have || same_shape(s, initial);
  if (!have) out.insert(out.begin(), initial);
  return out;
}

// Device buffers of the timed calls (unit densities, one output), freed on scope exit.
struct Scratch {
  double *slp = nullptr, *dlp = nullptr, *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~Scratch() {
    if (slp) cudaFree(slp);
    if (dlp) cudaFree(dlp);
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

int eval_once(stokes_ctx *c, int prec, const Scratch &b, cudaStream_t s) {
  if (c->n_inst > 1) return stokes_batch_eval(c, prec, b.slp, b.dlp, 0.0, b.out, 0, s);
  return stokes_sum_eval(c, prec, b.slp, b.dlp, 0.0, b.out, s);
}

// Median time of `repeats` evaluations after one untimed call.
int time_shape(stokes_ctx *c, int prec, const Scratch &b, cudaStream_t s, int repeats,
               double *ms) {
  int st = eval_once(c, prec, b, s);
  if (st) return st;
  std::vector<float> t(repeats, 0.f);
  for (int r = 0; r < repeats; ++r) {
    cudaError_t e = cudaEventRecord(b.e0, s);
    if (e != cudaSuccess) return tcuda(c, e, "cudaEventRecord");
    st = eval_once(c, prec, b, s);
    if (st) return st;
    if ((e = cudaEventRecord(b.e1, s)) != cudaSuccess) return tcuda(c, e, "cudaEventRecord");
    if ((e = cudaEventSynchronize(b.e1)) != cudaSuccess) return tcuda(c, e, "cudaEventSynchronize");
    if ((e = cudaEventElapsedTime(&t[r], b.e0, b.e1)) != cudaSuccess)
      return tcuda(c, e, "cudaEventElapsedTime");
  }
  st = stokes_sync(c, s);
  if (st) return st;
  std::sort(t.begin(), t.end());
  *ms = (repeats & 1) ? double(t[repeats / 2])
                      : 0.5 * (double(t[repeats / 2 - 1]) + double(t[repeats / 2]));
  return STOKES_OK;
}

}  // namespace

namespace stokes {

void tune_apply_cached(stokes_ctx *c) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (int prec : {STOKES_FP32_KAHAN, STOKES_FP64, STOKES_DOUBLE_FLOAT}) {
    const auto it = g_table.find(ctx_key(c, prec));
    if (it == g_table.end()) continue;
    const Shape &s = it->second.shape;
    if (c->n_inst > 1) {
      if (prec == STOKES_FP32_KAHAN) {
        c->tpt_f32 = s.tpt;
        if (s.ips) c->batch_ips32 = s.ips;
      } else if (s.ips) {
        c->batch_ips64 = s.ips;
      }
      continue;
    }
    if (prec == STOKES_FP32_KAHAN) {
      c->tpt_f32 = s.tpt;
      if (s.kg) c->kgroup_f32 = s.kg;
    }
    if (s.splits > 0) {
      const int eff = effective_splits(c, prec, s.splits);
      (prec == STOKES_FP32_KAHAN ? c->splits_f32
       : prec == STOKES_FP64     ? c->splits_f64
                                 : c->splits_df) = eff;
    }
  }
}

}  // namespace stokes

extern "C" {

int stokes_autotune(stokes_ctx *c, int precision, int repeats, stokes_tune_result *out,
                    void *stream) {
  if (!c) return STOKES_ERR_ARG;
  if (!c->have_geom) return tfail(c, STOKES_ERR_NO_GEOM, "no geometry set");
  if (!valid_prec(precision)) return tfail(c, STOKES_ERR_ARG, "unknown precision");
  if (repeats < 0 || repeats > 50) return tfail(c, STOKES_ERR_ARG, "repeats must be in [0, 50]");
  if (repeats == 0) repeats = 5;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return tcuda(c, e, "cudaSetDevice");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  Scratch b;
  const size_t nv = size_t(2) * std::max(c->n_ves_nodes, 1);
  const size_t nw = size_t(2) * std::max(c->n_wall_nodes, 1);
  if ((e = cudaMalloc(reinterpret_cast<void **>(&b.slp), nv * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void **>(&b.dlp), nw * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void **>(&b.out), size_t(2) * c->N * sizeof(double))) !=
          cudaSuccess)
    return tcuda(c, e, "cudaMalloc (tuner scratch)");
  if ((e = cudaEventCreate(&b.e0)) != cudaSuccess || (e = cudaEventCreate(&b.e1)) != cudaSuccess)
    return tcuda(c, e, "cudaEventCreate");
  {
    const std::vector<double> ones(std::max(nv, nw), 1.0);
    if ((e = cudaMemcpyAsync(b.slp, ones.data(), nv * sizeof(double), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(b.dlp, ones.data(), nw * sizeof(double), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return tcuda(c, e, "density upload (tuner scratch)");
  }

  const Shape initial = current_shape(c, precision);
  const std::vector<Shape> cand = candidates(c, precision, initial);
  Shape best = initial;
  double best_ms = 1e300, initial_ms = 0.0;
  for (const Shape &sh : cand) {
    int st = apply_shape(c, precision, sh);
    double ms = 0.0;
    if (!st) st = time_shape(c, precision, b, s, repeats, &ms);
    if (st) {
      apply_shape(c, precision, initial);
      return st;
    }
    const Shape got = current_shape(c, precision);  // splits after effective_splits
    if (same_shape(sh, initial)) initial_ms = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = got;
    }
  }
  if (initial_ms == 0.0) initial_ms = best_ms;  // not reached: the initial shape is a candidate
  int st = apply_shape(c, precision, best);
  if (st) return st;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table[ctx_key(c, precision)] = Entry{best, best_ms};
  }
  if (out) {
    out->precision = precision;
    out->source_splits = best.splits;
    out->targets_per_thread = best.tpt;
    out->kahan_group = best.kg;
    out->items_per_slot = best.ips;
    out->candidates = int(cand.size());
    out->best_ms = best_ms;
    out->initial_ms = initial_ms;
  }
  return STOKES_OK;
}

int stokes_tune_lookup(int num_sms, int precision, int n_inst, int n_nodes, int n_wall_nodes,
                       int n_ves_nodes, stokes_tune_result *out) {
  if (num_sms < 1 || !valid_prec(precision) || n_inst < 1 || n_nodes < 1 || n_wall_nodes < 0 ||
      n_ves_nodes < 0 || !out)
    return STOKES_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  const auto it =
      g_table.find(make_key(num_sms, precision, n_inst, n_nodes, n_wall_nodes, n_ves_nodes));
  if (it == g_table.end()) return 0;
  const Shape &s = it->second.shape;
  *out = stokes_tune_result{precision, s.splits, s.tpt, s.kg, s.ips, 0, it->second.ms, 0.0};
  return 1;
}

int stokes_tune_save(const char *path) {
  if (!path) return STOKES_ERR_ARG;
  FILE *f = fopen(path, "w");
  if (!f) return STOKES_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  fprintf(f, "# libstokes tuned launch shapes v1: sms precision b_inst b_nodes b_wall b_ves "
             "splits targets_per_thread kahan_group items_per_slot ms\n");
  for (const auto &kv : g_table) {
    const Key &k = kv.first;
    const Shape &s = kv.second.shape;
    fprintf(f, "%d %d %d %d %d %d %d %d %d %d %.9g\n", k[0], k[1], k[2], k[3], k[4], k[5],
            s.splits, s.tpt, s.kg, s.ips, kv.second.ms);
  }
  const bool ok = ferror(f) == 0;
  return (fclose(f) == 0 && ok) ? STOKES_OK : STOKES_ERR_ARG;
}

int stokes_tune_load(const char *path) {
  if (!path) return STOKES_ERR_ARG;
  FILE *f = fopen(path, "r");
  if (!f) return STOKES_ERR_ARG;
  std::map<Key, Entry> got;
  char line[512];
  bool bad = false;
  while (fgets(line, sizeof(line), f)) {
    const char *p = line;
    while (*p == ' ' || *p == '\t') ++p;
    if (*p == '#' || *p == '\n' || *p == '\r' || *p == 0) continue;
    Key k;
    Shape s;
    double ms = 0.0;
    char tail = 0;
    const int n = sscanf(p, "%d %d %d %d %d %d %d %d %d %d %lf %c", &k[0], &k[1], &k[2], &k[3],
                         &k[4], &k[5], &s.splits, &s.tpt, &s.kg, &s.ips, &ms, &tail);
    if (n != 11 || k[0] < 1 || !valid_prec(k[1]) || !valid_shape(k[1], s) || !(ms >= 0.0)) {
      bad = true;
      break;
    }
    got[k] = Entry{s, ms};
  }
  bad = bad || ferror(f) != 0;
  fclose(f);
  if (bad) return STOKES_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  for (const auto &kv : got) g_table[kv.first] = kv.second;
  return STOKES_OK;
}

int stokes_tune_clear(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_table.clear();
  return STOKES_OK;
}

}  // extern "C"
