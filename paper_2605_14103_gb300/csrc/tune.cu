// Autotuner of the tensor-core contraction tiles.
//
// A table maps (precision, feeder-size bucket, batch-size bucket) to the
// compiled contraction variant (N-tile BN, pipeline stages) to use; buckets
// are the next powers of two of the largest feeder's unknowns and of the
// total scenario count.  zbus_autotune times every variant of a precision on
// the caller's own workload and records the fastest.  The table is read from
// and written to a JSON file: $ZBUS_TUNE_CACHE, else zbus_tune.json beside
// libzbus.so.  Missing entries fall back to the built-in choice.
#include <dlfcn.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "group.cuh"

namespace zbus {
namespace {

struct Choice {
  int BN = 0, stages = 0;
  double ms = 0.0;
};

std::mutex g_mu;
std::map<std::tuple<int, int, int>, Choice> g_table;
bool g_loaded = false;
uint64_t g_gen = 1;

int bucket(int64_t x) {
  int64_t b = 1;
  while (b < x) b <<= 1;
  return (int)std::min<int64_t>(b, 1 << 30);
}

std::string cache_path() {
  const char* e = std::getenv("ZBUS_TUNE_CACHE");
  if (e && e[0]) return e;
  Dl_info info;
  if (dladdr((void*)&cache_path, &info) && info.dli_fname) {
    std::string s(info.dli_fname);
    const size_t k = s.rfind('/');
    if (k != std::string::npos) return s.substr(0, k + 1) + "zbus_tune.json";
  }
  return "zbus_tune.json";
}

// One entry per line: {"precision": P, "n": N, "B": B, "BN": X, "stages": S, "ms": T}
void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  FILE* f = std::fopen(cache_path().c_str(), "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    int p, n, b, bn, st;
    double ms;
    if (std::sscanf(line, " {\"precision\": %d, \"n\": %d, \"B\": %d, \"BN\": %d, \"stages\": %d, "
                          "\"ms\": %lf",
                    &p, &n, &b, &bn, &st, &ms) == 6 &&
        tc_config_ok(p, bn, st))
      g_table[std::make_tuple(p, n, b)] = Choice{bn, st, ms};
  }
  std::fclose(f);
}

bool save_locked() {
  FILE* f = std::fopen(cache_path().c_str(), "w");
  if (!f) return false;
  std::fprintf(f, "{\"entries\": [\n");
  size_t i = 0;
  for (const auto& kv : g_table) {
    std::fprintf(f, " {\"precision\": %d, \"n\": %d, \"B\": %d, \"BN\": %d, \"stages\": %d, "
                    "\"ms\": %.6f}%s\n",
                 std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                 kv.second.BN, kv.second.stages, kv.second.ms,
                 ++i < g_table.size() ? "," : "");
  }
  std::fprintf(f, "]}\n");
  std::fclose(f);
  return true;
}

}  // namespace

uint64_t tune_generation() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_gen;
}

zbus_status tune_lookup(int32_t precision, int max_n, int64_t total_B, int* BN, int* stages) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  *BN = 0;
  *stages = 0;
  auto it = g_table.find(std::make_tuple((int)precision, bucket(max_n), bucket(total_B)));
  if (it != g_table.end()) {
    *BN = it->second.BN;
    *stages = it->second.stages;
  }
  return ZBUS_OK;
}

void tune_set(int32_t precision, int max_n, int64_t total_B, int BN, int stages, double ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  const auto key = std::make_tuple((int)precision, bucket(max_n), bucket(total_B));
  if (BN == 0)
    g_table.erase(key);
  else
    g_table[key] = Choice{BN, stages, ms};
  ++g_gen;
}

bool tune_save() {
  std::lock_guard<std::mutex> lk(g_mu);
  return save_locked();
}

}  // namespace zbus

using namespace zbus;

extern "C" zbus_status zbus_autotune(const zbus_batch_item* items, int32_t n_items,
                                     const zbus_solve_opts* opts, double tol, int32_t max_iter,
                                     int32_t reps, void* cuda_stream, int32_t* best_BN,
                                     int32_t* best_stages) {
  set_error("");
  if (n_items <= 0 || !items) return fail(ZBUS_ERR_ARG, "no items");
  if (!opts || opts->precision == ZBUS_FP64)
    return fail(ZBUS_ERR_ARG, "the autotuner needs a mixed precision in opts");
  if (opts->precision == ZBUS_TREE_SWEEP)
    return fail(ZBUS_ERR_UNSUPPORTED, "the tree sweep has no tensor-core tiles to tune");
  if (reps < 1) reps = 3;
  int max_n = 0;
  int64_t total_B = 0;
  for (int32_t k = 0; k < n_items; ++k) {
    if (!items[k].net) return fail(ZBUS_ERR_ARG, "network is NULL");
    if (items[k].net->phased)
      return fail(ZBUS_ERR_UNSUPPORTED, "the autotuner takes three-phase networks");
    max_n = std::max(max_n, items[k].net->n);
    total_B += items[k].B;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int BNs[16], Ss[16];
  const int nv = tc_variants(opts->precision, BNs, Ss, 16);
  double best = 1e300;
  int bbn = 0, bst = 0;
  zbus_solve_opts o = *opts;
  o.profile = 0;
  cudaEvent_t e0, e1;
  ZB_CUDA(cudaEventCreate(&e0));
  ZB_CUDA(cudaEventCreate(&e1));
  for (int v = 0; v < nv; ++v) {
    tune_set(opts->precision, max_n, total_B, BNs[v], Ss[v], 0.0);
    zbus_status s = zbus_solve_batched(items, n_items, tol, max_iter, &o, cuda_stream);  // warm-up
    if (s != ZBUS_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return s;
    }
    ZB_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) ZB_CHECK(zbus_solve_batched(items, n_items, tol, max_iter, &o, cuda_stream));
    ZB_CUDA(cudaEventRecord(e1, st));
    ZB_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    ZB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    const double per = ms / reps;
    if (per < best) {
      best = per;
      bbn = BNs[v];
      bst = Ss[v];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tune_set(opts->precision, max_n, total_B, bbn, bst, best);
  tune_save();
  if (best_BN) *best_BN = bbn;
  if (best_stages) *best_stages = bst;
  return ZBUS_OK;
}

extern "C" int32_t zbus_tune_variants(int32_t precision, int32_t* BN, int32_t* stages,
                                      int32_t max) {
  if (max < 0) return -1;
  int bn[16], st[16];
  const int nv = tc_variants(precision, bn, st, 16);
  for (int v = 0; v < nv && v < max; ++v) {
    if (BN) BN[v] = bn[v];
    if (stages) stages[v] = st[v];
  }
  return nv;
}

extern "C" zbus_status zbus_tune_set(int32_t precision, int32_t max_n, int64_t total_B,
                                     int32_t BN, int32_t stages) {
  set_error("");
  if (precision != ZBUS_MIXED_BF16X2 && precision != ZBUS_MIXED_FP16_SCALED)
    return fail(ZBUS_ERR_ARG, "only the tensor-core precisions have contraction variants");
  if (max_n < 1 || total_B < 1) return fail(ZBUS_ERR_ARG, "max_n and total_B must be >= 1");
  if (BN != 0 && !tc_config_ok(precision, BN, stages))
    return fail(ZBUS_ERR_ARG, "(BN, stages) is not a compiled variant of this precision");
  tune_set(precision, max_n, total_B, BN, stages, 0.0);
  return ZBUS_OK;
}
