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

// Device bytes of the operands a network keeps resident for mixed solves.
size_t operand_bytes(zbus_network net) {
  const size_t n = (size_t)net->n, np = (size_t)net->n_pad;
  size_t b = n * n * 16 + 3 * np * np * 8 + n * 48;                  // Z, Zr/Zi/Zs, w, ys
  b += (size_t)net->nnz_ll * 20 + (size_t)net->nblk * (144 + 144);  // CSR, blocks (FP64, df)
  for (const auto& op : net->mixed)
    if (op.ready) b += (size_t)op.N_pad * op.K_pad * 2 * op.zparts;
  if (net->radial) b += (size_t)net->nbus * (16 + 4 + 72 + 4) + 4 * (size_t)(net->depth + 1);
  return b;
}

struct Inflight {
  zbus_request req;
  int64_t s0;
  double t_admit;
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

  // operands first, then the slot capacity the budget leaves
  size_t fixed = 0;
  for (auto net : nets) {
    ZB_CHECK(cfg->precision == ZBUS_TREE_SWEEP ? prepare_tree(net, st)
                                                : prepare_mixed(net, cfg->precision, st));
    fixed += operand_bytes(net);
  }
  if (fixed >= cfg->hbm_budget_bytes)
    return fail(ZBUS_ERR_OOM, "the pool's operands alone exceed the HBM budget (" +
                                  std::to_string(fixed) + " bytes)");
  const size_t share = (cfg->hbm_budget_bytes - fixed) / nets.size();
  std::vector<int64_t> caps(nets.size());
  std::vector<Feeder> fd(nets.size());
  for (size_t k = 0; k < nets.size(); ++k) {
    const size_t n = (size_t)nets[k]->n;
    // per slot: workspace of both methods plus the library result buffers
    const size_t per = 40 * n + 24 * (size_t)nets[k]->n_pad + 4 * (size_t)round_up(2 * nets[k]->n, 64) +
                       64 * (size_t)(round_up(2 * nets[k]->n, 256) / 128 + 1) + 16 * n + 64;
    int64_t cap = (int64_t)std::min<size_t>((size_t)std::max(128, cfg->max_slots), share / per);
    cap = cap / 128 * 128;
    if (cap < 128)
      return fail(ZBUS_ERR_OOM, "the HBM budget leaves fewer than 128 slots for feeder " +
                                    std::to_string(k));
    caps[k] = cap;
  }
  for (size_t k = 0; k < nets.size(); ++k) ZB_CHECK(ensure_workspace(nets[k], caps[k]));
  Group g;
  zbus_status s = group_build(&g, nets, caps, cfg->precision, st);
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
  while (true) {
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
      const bool warm = r.warm_start && f.warm_valid;
      SV_CHECK(group_admit(&g, r.feeder, s0, r.B, warm ? (const double*)f.warm : nullptr,
                           r.S_wye, r.S_delta, st, true));
      std::fill(f.used.begin() + s0, f.used.begin() + s0 + r.B, 1);
      f.live.push_back(Inflight{r, s0, clock_s(t0)});
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
