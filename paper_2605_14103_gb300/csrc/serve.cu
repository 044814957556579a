// Serving loop (zbus_serve): continuous batching over a pool of feeders on
// the grouped mixed-precision engine.  One loop pass = admissions between
// sweeps, one sweep over every active slot, completion of finished requests.
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include "group.cuh"

namespace zbus {
namespace {

double clock_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Device bytes of a feeder's operands while it is resident in the serving
// cache: the tensor-core Z (mixed forms) and the FP64 3M copies (the
// correction sweeps).  The complex FP64 Z is released once those are formed.
size_t cache_bytes(zbus_network net, int32_t precision) {
  const size_t np = (size_t)net->n_pad;
  size_t b = 3 * np * np * sizeof(double);
  if (precision != ZBUS_TREE_SWEEP) {
    const size_t K = (size_t)round_up(2 * net->n, 64), N = (size_t)round_up(2 * net->n, 256);
    b += N * K * 2 * (precision == ZBUS_MIXED_BF16X2 ? 2 : 1) + N / 2 * sizeof(float);
  }
  return b;
}

// Bytes a formation needs on top of cache_bytes while it runs: the complex Z
// and the elimination's scratch.
size_t form_extra(zbus_network net) {
  const size_t n = (size_t)net->n;
  return n * n * sizeof(double2) + n * 24;
}

// Device bytes per scenario slot: the workspace of both methods plus the
// library result buffers.
size_t slot_bytes(zbus_network net) {
  const size_t n = (size_t)net->n;
  return 40 * n + 24 * (size_t)net->n_pad + 4 * (size_t)round_up(2 * net->n, 64) +
         64 * (size_t)(round_up(2 * net->n, 256) / 128 + 1) + 16 * n + 72;
}

// Forms a feeder's resident operands (the Gauss-Jordan inverse again if it
// was released), then drops the complex Z.
zbus_status cache_form(zbus_network net, int32_t precision, cudaStream_t st) {
  ZB_CHECK(ensure_3m(net, st));
  if (precision != ZBUS_TREE_SWEEP) ZB_CHECK(prepare_mixed(net, precision, st));
  ZB_CUDA(cudaStreamSynchronize(st));
  release_z(net);
  return ZBUS_OK;
}

// Frees every dense operand of a feeder (no work of it may be in flight).
void cache_evict(zbus_network net) {
  release_mixed_ops(net);
  release_3m(net);
  release_z(net);
}

struct Inflight {
  zbus_request req;
  int64_t s0;
  double t_admit;
  int32_t formed;   // its admission formed the feeder's operands (a cache miss)
};

struct Feeder {
  int64_t cap = 0;
  std::vector<char> used;
  std::vector<Inflight> live;
  double2* warm = nullptr;        // last converged voltage [n]
  bool warm_valid = false;
  double2* res_V = nullptr;       // library result buffers [cap][n], [cap], [cap]
  int32_t* res_it = nullptr;
  uint8_t* res_cv = nullptr;
  uint8_t* h_st = nullptr;        // pinned mirror of the slot states
};

int64_t first_fit(const std::vector<char>& used, int64_t B) {
  int64_t run = 0;
  for (int64_t s = 0; s < (int64_t)used.size(); ++s) {
    run = used[s] ? 0 : run + 1;
    if (run == B) return s - B + 1;
  }
  return -1;
}

}  // namespace
}  // namespace zbus

using namespace zbus;

extern "C" zbus_status zbus_serve_footprint(zbus_network net, int32_t precision,
                                            uint64_t* operand_bytes, uint64_t* formation_bytes,
                                            uint64_t* slot_bytes_out) {
  set_error("");
  if (!net) return fail(ZBUS_ERR_ARG, "network is NULL");
  if (precision != ZBUS_MIXED_FP16_SCALED && precision != ZBUS_MIXED_BF16X2 &&
      precision != ZBUS_TREE_SWEEP)
    return fail(ZBUS_ERR_ARG, "serving runs the mixed precisions");
  if (operand_bytes) *operand_bytes = cache_bytes(net, precision);
  if (formation_bytes) *formation_bytes = form_extra(net);
  if (slot_bytes_out) *slot_bytes_out = slot_bytes(net);
  return ZBUS_OK;
}

extern "C" zbus_status zbus_serve(const zbus_serve_config* cfg, zbus_network* pool,
                                  int32_t n_pool, zbus_request_source src,
                                  zbus_completion_sink sink, void* user, void* cuda_stream) {
  NvtxRange nvtx_range("zbus_serve");
  set_error("");
  if (!cfg || !pool || n_pool <= 0 || !src || !sink) return fail(ZBUS_ERR_ARG, "bad arguments");
  if (cfg->precision != ZBUS_MIXED_FP16_SCALED && cfg->precision != ZBUS_MIXED_BF16X2 &&
      cfg->precision != ZBUS_TREE_SWEEP)
    return fail(ZBUS_ERR_ARG, "serving runs the mixed precisions");
  if (cfg->max_iter < 1 || !(cfg->tol >= 0.0)) return fail(ZBUS_ERR_ARG, "bad tol / max_iter");
  if (cfg->conv_rule != ZBUS_CONV_MAXABS && cfg->conv_rule != ZBUS_CONV_SUMMAG)
    return fail(ZBUS_ERR_ARG, "unknown convergence rule");
  std::vector<zbus_network> nets(pool, pool + n_pool);
  for (int k = 0; k < n_pool; ++k) {
    if (!nets[k]) return fail(ZBUS_ERR_ARG, "pool network is NULL");
    if (nets[k]->phased)
      return fail(ZBUS_ERR_UNSUPPORTED, "the serving pool takes three-phase networks");
    for (int j = 0; j < k; ++j)
      if (nets[j] == nets[k]) return fail(ZBUS_ERR_ARG, "a network may appear once in the pool");
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double mtol = cfg->mismatch_tol > 0 ? cfg->mismatch_tol : 1e-6;

  // Budget: the scenario slots of every feeder (one capacity for all, the
  // largest multiple of 128 up to max_slots that leaves room for the largest
  // feeder's operands while they are formed) plus the operand cache.
  for (auto net : nets)
    if (cfg->precision == ZBUS_TREE_SWEEP) ZB_CHECK(prepare_tree(net, st));
  size_t per_slot = 0, peak_one = 0;
  for (auto net : nets) {
    per_slot += slot_bytes(net);
    peak_one = std::max(peak_one, cache_bytes(net, cfg->precision) + form_extra(net));
  }
  const uint64_t budget = cfg->hbm_budget_bytes;
  int64_t cap = (int64_t)std::max(128, cfg->max_slots) / 128 * 128;
  while (cap >= 128 && (double)per_slot * cap + peak_one > (double)budget) cap -= 128;
  if (cap < 128)
    return fail(ZBUS_ERR_OOM, "the HBM budget cannot hold 128 slots per feeder plus the "
                              "operands of the largest feeder (" +
                                  std::to_string(per_slot * 128 + peak_one) + " bytes)");
  const size_t ops_budget = budget - (size_t)per_slot * cap;
  // the operand cache starts with the feeders that hold their operands (or
  // the complex Z they are packed from) and fit, in pool order; the others
  // give their dense operands up now and are formed on demand
  std::vector<char> resident(nets.size(), 0);
  std::vector<int64_t> last_use(nets.size(), -1);
  size_t used = 0;
  const int pi = cfg->precision == ZBUS_MIXED_BF16X2 ? 1 : 0;
  for (size_t k = 0; k < nets.size(); ++k) {
    const zbus_network net = nets[k];
    const size_t cb = cache_bytes(net, cfg->precision);
    const bool holds = (net->Zr || net->Z) &&
                       (cfg->precision == ZBUS_TREE_SWEEP || net->mixed[pi].ready || net->Z);
    ZB_CUDA(cudaStreamSynchronize(st));
    if (holds && used + cb <= ops_budget) {
      ZB_CHECK(cache_form(nets[k], cfg->precision, st));
      resident[k] = 1;
      used += cb;
    } else {
      cache_evict(nets[k]);
    }
  }
  std::vector<int64_t> caps(nets.size(), cap);
  std::vector<Feeder> fd(nets.size());
  for (size_t k = 0; k < nets.size(); ++k) ZB_CHECK(ensure_workspace(nets[k], caps[k]));
  Group g;
  zbus_status s = group_build(&g, nets, caps, cfg->precision, st, true);
  if (s != ZBUS_OK) {
    group_free(&g);
    return s;
  }
  int32_t* h_err = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    cudaFreeHost(h_err);
    for (auto& f : fd) {
      cudaFree(f.warm);
      cudaFree(f.res_V);
      cudaFree(f.res_it);
      cudaFree(f.res_cv);
      cudaFreeHost(f.h_st);
    }
    group_free(&g);
  };
#define SV_CHECK(call)          \
  do {                          \
    zbus_status _s = (call);    \
    if (_s != ZBUS_OK) {        \
      cleanup();                \
      return _s;                \
    }                           \
  } while (0)
#define SV_CUDA(call)                                                         \
  do {                                                                        \
    cudaError_t _e = (call);                                                  \
    if (_e != cudaSuccess) {                                                  \
      zbus_status _s = cuda_fail(_e, #call, __FILE__, __LINE__);              \
      cleanup();                                                              \
      return _s;                                                              \
    }                                                                         \
  } while (0)
  for (size_t k = 0; k < nets.size(); ++k) {
    Feeder& f = fd[k];
    f.cap = caps[k];
    f.used.assign((size_t)f.cap, 0);
    const size_t n = (size_t)nets[k]->n;
    SV_CUDA(cudaMalloc((void**)&f.warm, n * sizeof(double2)));
    SV_CUDA(cudaMalloc((void**)&f.res_V, (size_t)f.cap * n * sizeof(double2)));
    SV_CUDA(cudaMalloc((void**)&f.res_it, (size_t)f.cap * sizeof(int32_t)));
    SV_CUDA(cudaMalloc((void**)&f.res_cv, (size_t)f.cap));
    SV_CUDA(cudaMallocHost((void**)&f.h_st, (size_t)f.cap));
  }
  SV_CUDA(cudaMallocHost((void**)&h_err, sizeof(int32_t)));
  *h_err = 0;
  SV_CHECK(group_reset(&g, st));
  SV_CHECK(group_start(&g, cfg->tol, cfg->max_iter, cfg->conv_rule, nullptr, 0, st));
  SV_CUDA(cudaStreamSynchronize(st));

  const auto t0 = std::chrono::steady_clock::now();
  std::deque<zbus_request> pending;
  bool ended = false;
  bool source_failed = false;
  int64_t live_total = 0;
  std::vector<int32_t> h_it;
  std::vector<uint8_t> h_cv;
  int64_t n_pass = 0;
  while (true) {
    ++n_pass;
    const double now = clock_s(t0);
    while (!ended) {
      zbus_request r;
      std::memset(&r, 0, sizeof(r));
      const int32_t got = src(user, now, &r);
      if (got == 1) {
        pending.push_back(r);
      } else if (got < 0) {
        ended = true;
        source_failed = got <= -2;
      } else {
        break;
      }
    }
    // admissions, in arrival order, first fit
    bool admitted = false;
    int n_adm = 0;
    for (auto it = pending.begin(); it != pending.end();) {
      if (cfg->max_admit_per_sweep > 0 && n_adm >= cfg->max_admit_per_sweep) break;
      zbus_request& r = *it;
      const bool bad_feeder = r.feeder < 0 || r.feeder >= n_pool;
      if (bad_feeder || r.B < 1 || r.B > (bad_feeder ? 0 : fd[r.feeder].cap) ||
          (r.S_delta && !nets[r.feeder]->bus_aligned)) {
        zbus_request_result res;
        std::memset(&res, 0, sizeof(res));
        res.status = ZBUS_ERR_ARG;
        res.t_admit = res.t_done = clock_s(t0);
        sink(user, &r, &res);
        it = pending.erase(it);
        continue;
      }
      Feeder& f = fd[r.feeder];
      const int64_t s0 = first_fit(f.used, r.B);
      if (s0 < 0) {
        ++it;
        continue;
      }
      int32_t formed = 0;
      if (!resident[r.feeder]) {
        // operand cache miss: evict idle feeders, least recently used first,
        // until this one can be formed; else it waits for one to go idle
        const size_t cb = cache_bytes(nets[r.feeder], cfg->precision);
        const size_t need = cb + form_extra(nets[r.feeder]);
        while (used + need > ops_budget) {
          int victim = -1;
          for (size_t j = 0; j < nets.size(); ++j)
            if (resident[j] && fd[j].live.empty() &&
                (victim < 0 || last_use[j] < last_use[victim]))
              victim = (int)j;
          if (victim < 0) break;
          SV_CUDA(cudaStreamSynchronize(st));
          cache_evict(nets[victim]);
          resident[victim] = 0;
          used -= cache_bytes(nets[victim], cfg->precision);
        }
        if (used + need > ops_budget) {
          ++it;
          continue;
        }
        SV_CHECK(cache_form(nets[r.feeder], cfg->precision, st));
        SV_CHECK(group_refresh_item(&g, r.feeder, st));
        resident[r.feeder] = 1;
        used += cb;
        formed = 1;
      }
      last_use[r.feeder] = n_pass;
      {
        // every pointer the sweep reads for this item is in place
        const ItemDesc& d = g.h_items[r.feeder];
        const bool ok = d.bsr_df && nets[r.feeder]->w_df && nets[r.feeder]->Zr &&
                        (cfg->precision == ZBUS_TREE_SWEEP || d.zinv);
        if (!ok) SV_CHECK(fail(ZBUS_ERR_DEVICE, "serving: a feeder's operands are missing"));
      }
      const bool warm = r.warm_start && f.warm_valid;
      SV_CHECK(group_admit(&g, r.feeder, s0, r.B, warm ? (const double*)f.warm : nullptr,
                           r.S_wye, r.S_delta, st, true, cfg->fp32_start != 0));
      std::fill(f.used.begin() + s0, f.used.begin() + s0 + r.B, 1);
      f.live.push_back(Inflight{r, s0, clock_s(t0), formed});
      live_total += 1;
      admitted = true;
      ++n_adm;
      it = pending.erase(it);
    }
    if (admitted) SV_CHECK(group_rebuild(&g, st));
    if (live_total == 0) {
      if (ended && pending.empty()) break;
      std::this_thread::sleep_for(std::chrono::microseconds(50));
      continue;
    }
    {
      NvtxRange sweep_range("zbus_serve sweep");
      SV_CHECK(group_sweep(&g, 0, false, st));
    }
    for (size_t k = 0; k < nets.size(); ++k)
      if (!fd[k].live.empty())
        SV_CUDA(cudaMemcpyAsync(fd[k].h_st, g.h_items[k].st, (size_t)fd[k].cap,
                                cudaMemcpyDeviceToHost, st));
    SV_CUDA(cudaMemcpyAsync(h_err, group_error_word(&g), sizeof(int32_t), cudaMemcpyDeviceToHost,
                            st));
    SV_CUDA(cudaStreamSynchronize(st));
    if (*h_err != 0) SV_CHECK(group_device_status(&g, st));   // a device wait gave up
    // completions
    struct Done {
      size_t k;
      Inflight fl;
      double* V;
      int32_t* it;
      uint8_t* cv;
    };
    std::vector<Done> done;
    for (size_t k = 0; k < nets.size(); ++k) {
      Feeder& f = fd[k];
      for (size_t q = 0; q < f.live.size();) {
        const Inflight& fl = f.live[q];
        bool finished = true;
        for (int64_t b = 0; b < fl.req.B && finished; ++b)
          finished = f.h_st[fl.s0 + b] != SLOT_ACTIVE;
        if (!finished) {
          ++q;
          continue;
        }
        const size_t n = (size_t)nets[k]->n;
        double* V = fl.req.V_out ? fl.req.V_out : (double*)(f.res_V + (size_t)fl.s0 * n);
        int32_t* itp = fl.req.V_out && fl.req.iters ? fl.req.iters : f.res_it + fl.s0;
        uint8_t* cvp = fl.req.V_out && fl.req.converged ? fl.req.converged : f.res_cv + fl.s0;
        SV_CHECK(group_collect(&g, (int)k, fl.s0, fl.req.B, V, itp, cvp, fl.req.S_wye,
                               fl.req.S_delta, mtol, nullptr, cfg->max_correction, st));
        done.push_back(Done{k, fl, V, itp, cvp});
        f.live.erase(f.live.begin() + q);
      }
    }
    if (done.empty()) continue;
    SV_CUDA(cudaStreamSynchronize(st));
    const double t_done = clock_s(t0);
    for (auto& d : done) {
      Feeder& f = fd[d.k];
      const int64_t B = d.fl.req.B;
      h_it.resize((size_t)B);
      h_cv.resize((size_t)B);
      SV_CUDA(cudaMemcpy(h_it.data(), d.it, (size_t)B * sizeof(int32_t), cudaMemcpyDeviceToHost));
      SV_CUDA(cudaMemcpy(h_cv.data(), d.cv, (size_t)B, cudaMemcpyDeviceToHost));
      zbus_request_result res;
      std::memset(&res, 0, sizeof(res));
      res.status = ZBUS_OK;
      res.t_admit = d.fl.t_admit;
      res.t_done = t_done;
      res.operands_formed = d.fl.formed;
      res.V = d.V;
      res.iters = d.it;
      res.converged = d.cv;
      int first_conv = -1;
      for (int64_t b = 0; b < B; ++b) {
        res.n_converged += h_cv[(size_t)b] ? 1 : 0;
        res.max_iters = std::max(res.max_iters, h_it[(size_t)b]);
        if (first_conv < 0 && h_cv[(size_t)b]) first_conv = (int)b;
      }
      if (first_conv >= 0) {
        const size_t n = (size_t)nets[d.k]->n;
        SV_CUDA(cudaMemcpy(f.warm, d.V + (size_t)first_conv * n * 2, n * sizeof(double2),
                           cudaMemcpyDeviceToDevice));
        f.warm_valid = true;
      }
      sink(user, &d.fl.req, &res);
      std::fill(f.used.begin() + d.fl.s0, f.used.begin() + d.fl.s0 + B, 0);
      live_total -= 1;
    }
  }
  cleanup();
  if (source_failed)
    return fail(ZBUS_ERR_SOURCE, "the request source reported a failure; the requests it had "
                                 "delivered were served");
  return ZBUS_OK;
#undef SV_CHECK
#undef SV_CUDA
}
