// C ABI of libzbus: argument checks, handle lifetime, scratch space, the
// device-resident iteration loop of the plain FP64 method (a CUDA graph whose
// WHILE node repeats one sweep until no scenario is active) and the entry
// points of the grouped mixed-precision engine (group.cu).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <set>

#include "group.cuh"
#include "zbus_internal.cuh"

namespace zbus {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

zbus_status fail(zbus_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

zbus_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                 std::to_string(line) + ")";
  cudaGetLastError();  // clear a sticky launch error where possible
  return e == cudaErrorMemoryAllocation ? ZBUS_ERR_OOM : ZBUS_ERR_CUDA;
}

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool known_precision(int32_t p) {
  return p == ZBUS_FP64 || p == ZBUS_MIXED_BF16X2 || p == ZBUS_MIXED_FP16_SCALED ||
         p == ZBUS_TREE_SWEEP;
}

}  // namespace

void drop_graphs(zbus_network net) {
  for (auto& g : net->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  net->graphs.clear();
  if (net->corr_exec) cudaGraphExecDestroy(net->corr_exec);
  if (net->corr_graph) cudaGraphDestroy(net->corr_graph);
  net->corr_exec = nullptr;
  net->corr_graph = nullptr;
}

namespace {

int max_ntn(const zbus_network net) {
  // the FP64 contraction tiles outputs by 48, the tensor-core one by >= 64 reals
  return std::max(net->n_pad / F64_BN, round_up(2 * net->n, 256) / 64);
}

int k_pad_tc(const zbus_network net) { return round_up(2 * net->n, 64); }

// Scratch of one solve: context, active list, per-tile partials, the FP64
// contraction operands and the low-precision residual rows.
struct WsLayout {
  size_t list, keep, part, iop, R, rinv, mm, vh, vl, swf, sdf, st, amax, mt, sit, sconv, total;
};

WsLayout workspace_layout(const zbus_network net, int64_t B) {
  // per-scenario arrays of the mixed sweeps are sized for B rounded up to the
  // 128-scenario tile of the tensor-core contraction
  const size_t Bp = (size_t)round_up((int)B, 128);
  WsLayout L;
  size_t o = align256(sizeof(SolveCtx));
  L.list = o;
  o += align256((size_t)B * sizeof(int32_t));
  L.keep = o;
  o += align256((size_t)B);
  L.part = o;
  o += align256(Bp * max_ntn(net) * 2 * sizeof(double));
  // FP64 contraction operands; the tree sweep's FP32 residual [n][Bp] shares
  // the region
  L.iop = o;
  o += align256(std::max((size_t)3 * B * net->n_pad * sizeof(double),
                         Bp * net->n * sizeof(float2)));
  L.R = o;
  o += align256(Bp * k_pad_tc(net) * 2);
  L.rinv = o;
  o += align256(Bp * sizeof(float));
  L.mm = o;
  o += align256((size_t)B * sizeof(double));
  const size_t f2 = align256(Bp * net->n * sizeof(float2));
  L.vh = o;
  o += f2;
  L.vl = o;
  o += f2;
  L.swf = o;
  o += f2;
  L.sdf = o;
  o += f2;
  L.st = o;
  o += align256(Bp);
  L.amax = o;
  o += align256(4 * Bp * sizeof(float));
  L.mt = o;
  o += align256(2 * (Bp / 128) * sizeof(int32_t));
  L.sit = o;
  o += align256(Bp * sizeof(int32_t));
  L.sconv = o;
  o += align256(Bp);
  L.total = o;
  return L;
}

}  // namespace

zbus_status ensure_workspace(zbus_network net, int64_t B) {
  Workspace& ws = net->ws;
  if (ws.base && ws.cap_B >= B) return ZBUS_OK;
  const WsLayout L = workspace_layout(net, B);
  const uint64_t gen = ws.gen + 1;
  if (ws.base) {
    ZB_CUDA(cudaDeviceSynchronize());
    drop_graphs(net);
    cudaFree(ws.base);
    ws = Workspace();
  }
  void* base = nullptr;
  ZB_CUDA(cudaMalloc(&base, L.total));
  char* p = (char*)base;
  ws.gen = gen;
  ws.base = base;
  ws.bytes = L.total;
  ws.cap_B = B;
  ws.cap_Bp = round_up((int)B, 128);
  ws.ctx = (SolveCtx*)p;
  ws.list = (int32_t*)(p + L.list);
  ws.keep = (uint8_t*)(p + L.keep);
  ws.part = (double*)(p + L.part);
  ws.Iop = (double*)(p + L.iop);
  ws.iop_bytes = L.R - L.iop;
  ws.R = (void*)(p + L.R);
  ws.rinv = (float*)(p + L.rinv);
  ws.mm = (double*)(p + L.mm);
  ws.Vh = (float2*)(p + L.vh);
  ws.Vl = (float2*)(p + L.vl);
  ws.Swf = (float2*)(p + L.swf);
  ws.Sdf = (float2*)(p + L.sdf);
  ws.st = (uint8_t*)(p + L.st);
  ws.amax = (float*)(p + L.amax);
  ws.mt = (int32_t*)(p + L.mt);
  ws.slot_it = (int32_t*)(p + L.sit);
  ws.slot_conv = (uint8_t*)(p + L.sconv);
  return ZBUS_OK;
}

bool use_graphs() {
  const char* e = std::getenv("ZBUS_NO_GRAPH");
  return !(e && e[0] == '1');
}

namespace {

// One sweep of the plain FP64 method on stream st (optionally bracketed by
// events for the profile mode).
zbus_status enqueue_sweep_f64(zbus_network net, int64_t B, int grid, cudaGraphConditionalHandle h,
                              bool use_handle, cudaStream_t st, cudaEvent_t* ev = nullptr) {
  if (ev) ZB_CUDA(cudaEventRecord(ev[0], st));
  launch_currents_f64(net->ws.ctx, net->n, net->n_pad, (int)B, st);
  if (ev) ZB_CUDA(cudaEventRecord(ev[1], st));
  launch_gemm_f64(net->ws.ctx, net->Zr, net->Zi, net->Zs, net->w, net->n, net->n_pad, grid, st);
  if (ev) ZB_CUDA(cudaEventRecord(ev[2], st));
  launch_converge(net->ws.ctx, (int)B, h, use_handle, st);
  if (ev) ZB_CUDA(cudaEventRecord(ev[3], st));
  return ZBUS_OK;
}

}  // namespace

// A graph whose WHILE node repeats one sweep (enqueued by `sweep`) until the
// sweep's last kernel clears the condition; cached per (B, key).
zbus_status get_while_graph(zbus_network net, int64_t B, int32_t key, int grid, SweepFn sweep,
                            GraphEntry** out) {
  for (auto& g : net->graphs)
    if (g.B == B && g.precision == key) {
      *out = &g;
      return ZBUS_OK;
    }
  GraphEntry e;
  e.B = B;
  e.precision = key;
  e.grid_gemm = grid;
  if (!net->cap_stream) ZB_CUDA(cudaStreamCreateWithFlags(&net->cap_stream, cudaStreamNonBlocking));
  ZB_CUDA(cudaGraphCreate(&e.graph, 0));
  cudaGraphConditionalHandle h;
  ZB_CUDA(cudaGraphConditionalHandleCreate(&h, e.graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  ZB_CUDA(cudaGraphAddNode(&node, e.graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  ZB_CUDA(cudaStreamBeginCaptureToGraph(net->cap_stream, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  zbus_status s = sweep(net, B, grid, h, true, net->cap_stream, nullptr);
  cudaGraph_t captured = nullptr;
  cudaError_t ce = cudaStreamEndCapture(net->cap_stream, &captured);
  if (s != ZBUS_OK || ce != cudaSuccess) {
    cudaGraphDestroy(e.graph);
    if (s != ZBUS_OK) return s;
    return cuda_fail(ce, "cudaStreamEndCapture(sweep)", __FILE__, __LINE__);
  }
  ce = cudaGraphInstantiate(&e.exec, e.graph, 0);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(e.graph);
    return cuda_fail(ce, "cudaGraphInstantiate(solve loop)", __FILE__, __LINE__);
  }
  net->graphs.push_back(e);
  *out = &net->graphs.back();
  return ZBUS_OK;
}

namespace {

// Profile buffers (events, per-sweep active counts) for up to max_iter sweeps.
zbus_status ensure_profile(zbus_network net, int32_t max_iter) {
  Profile& P = net->prof;
  if (P.cap >= max_iter) return ZBUS_OK;
  for (auto e : P.ev) cudaEventDestroy(e);
  P.ev.clear();
  cudaFree(P.d_hist);
  P.d_hist = nullptr;
  P.cap = 0;
  ZB_CUDA(cudaMalloc((void**)&P.d_hist, (size_t)max_iter * sizeof(int32_t)));
  P.ev.resize((size_t)4 * max_iter);
  for (auto& e : P.ev) ZB_CUDA(cudaEventCreate(&e));
  P.cap = max_iter;
  return ZBUS_OK;
}

// Groups of the batched entry point, keyed by their networks, sizes, precision.
std::vector<Group*> g_batch_groups;

void drop_groups_of(zbus_network net) {
  for (size_t i = 0; i < g_batch_groups.size();) {
    Group* g = g_batch_groups[i];
    if (std::find(g->nets.begin(), g->nets.end(), net) != g->nets.end()) {
      for (auto other : g->nets)
        if (other->last_group == g) other->last_group = nullptr;
      group_free(g);
      delete g;
      g_batch_groups.erase(g_batch_groups.begin() + i);
    } else {
      ++i;
    }
  }
}

bool group_current(const Group* g, const std::vector<zbus_network>& nets,
                   const std::vector<int64_t>& Bs, int32_t precision) {
  if (!g || g->precision != precision || g->nets != nets) return false;
  if (g->tune_gen != tune_generation()) return false;
  for (size_t k = 0; k < nets.size(); ++k)
    if (g->ws_gen[k] != nets[k]->ws.gen || g->op_gen[k] != nets[k]->op_gen ||
        g->h_items[k].Bp < Bs[k])
      return false;
  return true;
}

// Run a group of feeders from their admissions to their results on stream st.
zbus_status run_group(Group* g, const std::vector<zbus_network>& nets, const std::vector<int64_t>& Bs,
                      const std::vector<const double*>& Sw, const std::vector<const double*>& Sd,
                      const std::vector<const double*>& V0, const std::vector<double*>& Vout,
                      const std::vector<int32_t*>& iters, const std::vector<uint8_t*>& conv,
                      double tol, int32_t max_iter, const zbus_solve_opts& o, cudaStream_t st) {
  const double mtol = o.mismatch_tol > 0 ? o.mismatch_tol : 1e-6;
  for (auto net : nets) net->last_group = g;
  ZB_CHECK(group_reset(g, st));
  for (size_t k = 0; k < nets.size(); ++k)
    ZB_CHECK(group_admit(g, (int)k, 0, Bs[k], V0[k], Sw[k], Sd[k], st, false,
                         o.fp32_start != 0));
  zbus_network pn = nets[0];
  if (o.profile == 1) {
    ZB_CHECK(ensure_profile(pn, max_iter));
    ZB_CUDA(cudaMemsetAsync(pn->prof.d_hist, 0, (size_t)max_iter * sizeof(int32_t), st));
    ZB_CHECK(group_start(g, tol, max_iter, o.conv_rule, pn->prof.d_hist, max_iter, st));
    for (int k = 0; k < max_iter; ++k)
      ZB_CHECK(group_sweep(g, 0, false, st, &pn->prof.ev[(size_t)4 * k]));
    pn->prof.sweeps = max_iter;
  } else {
    ZB_CHECK(group_start(g, tol, max_iter, o.conv_rule, nullptr, 0, st));
    ZB_CHECK(group_run(g, st));
  }
  for (size_t k = 0; k < nets.size(); ++k)
    ZB_CHECK(group_collect(g, (int)k, 0, Bs[k], Vout[k], iters[k], conv[k], Sw[k], Sd[k], mtol,
                           nullptr, o.max_correction, st));
  return ZBUS_OK;
}

zbus_status check_device(zbus_network net) {
  int dev = -1;
  ZB_CUDA(cudaGetDevice(&dev));
  if (dev != net->device)
    return fail(ZBUS_ERR_ARG, "current CUDA device " + std::to_string(dev) +
                                  " differs from the network's device " +
                                  std::to_string(net->device));
  return ZBUS_OK;
}

}  // namespace

// Where a caller buffer lives: 1 device (or managed) memory, 0 host memory
// (pinned or pageable), -1 null.
int buffer_kind(const void* p) {
  if (!p) return -1;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? 1 : 0;
}

}  // namespace zbus

using namespace zbus;

extern "C" {

void zbus_solve_opts_default(zbus_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = ZBUS_FP64;
  o->conv_rule = ZBUS_CONV_MAXABS;
  o->mismatch_tol = 1e-6;
  o->max_correction = 8;
  o->fp32_start = 1;
}

zbus_status zbus_last_device_status(zbus_network net, void* cuda_stream) {
  g_last_error.clear();
  if (!net) return fail(ZBUS_ERR_ARG, "network is NULL");
  ZB_CHECK(check_device(net));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!net->last_group) {
    ZB_CUDA(cudaStreamSynchronize(st));
    return ZBUS_OK;
  }
  return group_device_status(net->last_group, st);
}

const char* zbus_status_string(zbus_status s) {
  switch (s) {
    case ZBUS_OK: return "ZBUS_OK";
    case ZBUS_ERR_ARG: return "ZBUS_ERR_ARG";
    case ZBUS_ERR_SINGULAR: return "ZBUS_ERR_SINGULAR";
    case ZBUS_ERR_OOM: return "ZBUS_ERR_OOM";
    case ZBUS_ERR_CUDA: return "ZBUS_ERR_CUDA";
    case ZBUS_ERR_TIMEOUT: return "ZBUS_ERR_TIMEOUT";
    case ZBUS_ERR_DEVICE: return "ZBUS_ERR_DEVICE";
    case ZBUS_ERR_UNSUPPORTED: return "ZBUS_ERR_UNSUPPORTED";
    case ZBUS_ERR_SOURCE: return "ZBUS_ERR_SOURCE";
  }
  return "ZBUS_UNKNOWN_STATUS";
}

const char* zbus_last_error(void) { return g_last_error.c_str(); }

int32_t zbus_checked_status(uint32_t* word) {
  cudaDeviceSynchronize();
  uint32_t (*const words[])(bool) = {check_word_f64, check_word_group, check_word_adjoint,
                                     check_word_nr, check_word_phased};
  uint32_t first = 0;
  for (auto fn : words) {
    const uint32_t w = fn(true);
    if (!first) first = w;
  }
  if (word) *word = first;
#ifdef ZBUS_CHECKED
  return 1;
#else
  return 0;
#endif
}

zbus_status zbus_network_create(int32_t n_total, int64_t nnz, const int32_t* row,
                                const int32_t* col, const double* val_reim,
                                const int32_t* slack_idx, const double* v_slack_reim,
                                void* cuda_stream, zbus_network* out) {
  NvtxRange nvtx_range("zbus_network_create");
  g_last_error.clear();
  if (!out) return fail(ZBUS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_total < 4) return fail(ZBUS_ERR_ARG, "n_total must be >= 4 (three slack phases + 1)");
  if (nnz < 1) return fail(ZBUS_ERR_ARG, "nnz must be >= 1");
  if (!row || !col || !val_reim || !slack_idx || !v_slack_reim)
    return fail(ZBUS_ERR_ARG, "a required host array is NULL");
  std::set<int32_t> sl;
  for (int p = 0; p < 3; ++p) {
    if (slack_idx[p] < 0 || slack_idx[p] >= n_total)
      return fail(ZBUS_ERR_ARG, "slack index out of range");
    sl.insert(slack_idx[p]);
  }
  if (sl.size() != 3) return fail(ZBUS_ERR_ARG, "slack indices must be distinct");
  for (int p = 0; p < 6; ++p)
    if (!std::isfinite(v_slack_reim[p])) return fail(ZBUS_ERR_ARG, "slack voltage not finite");
  for (int64_t t = 0; t < nnz; ++t) {
    if (row[t] < 0 || row[t] >= n_total || col[t] < 0 || col[t] >= n_total)
      return fail(ZBUS_ERR_ARG, "COO index out of range at entry " + std::to_string(t));
    if (!std::isfinite(val_reim[2 * t]) || !std::isfinite(val_reim[2 * t + 1]))
      return fail(ZBUS_ERR_ARG, "COO value not finite at entry " + std::to_string(t));
  }
  auto* net = new zbus_network_s();
  cudaError_t ce = cudaGetDevice(&net->device);
  if (ce != cudaSuccess) {
    delete net;
    return cuda_fail(ce, "cudaGetDevice", __FILE__, __LINE__);
  }
  zbus_status s = build_network(net, n_total, nnz, row, col, val_reim, slack_idx, v_slack_reim,
                                (cudaStream_t)cuda_stream);
  // the allocation-free solve's static array is loaded now, while the caller
  // still allocates, not at its first zbus_solve_noalloc call
  if (s == ZBUS_OK) s = noalloc_prepare(net->device);
  if (s != ZBUS_OK) {
    std::string msg = g_last_error;
    cudaStreamSynchronize((cudaStream_t)cuda_stream);
    zbus_network_destroy(net);
    g_last_error = msg;
    return s;
  }
  *out = net;
  return ZBUS_OK;
}

zbus_status zbus_network_create_phased(int32_t n_total, int64_t nnz, const int32_t* row,
                                       const int32_t* col, const double* val_reim,
                                       const int32_t* slack_idx, const double* v_slack_reim,
                                       const int32_t* bus_phase, void* cuda_stream,
                                       zbus_network* out) {
  g_last_error.clear();
  if (!out) return fail(ZBUS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_total < 4) return fail(ZBUS_ERR_ARG, "n_total must be >= 4 (three slack phases + 1)");
  if (nnz < 1) return fail(ZBUS_ERR_ARG, "nnz must be >= 1");
  if (!row || !col || !val_reim || !slack_idx || !v_slack_reim)
    return fail(ZBUS_ERR_ARG, "a required host array is NULL");
  for (int p = 0; p < 3; ++p)
    if (slack_idx[p] < 0 || slack_idx[p] >= n_total)
      return fail(ZBUS_ERR_ARG, "slack index out of range");
  for (int64_t t = 0; t < nnz; ++t)
    if (row[t] < 0 || row[t] >= n_total || col[t] < 0 || col[t] >= n_total)
      return fail(ZBUS_ERR_ARG, "COO index out of range at entry " + std::to_string(t));
  int32_t n_bus = 0;
  ZB_CHECK(phased_validate(n_total, slack_idx, bus_phase, &n_bus));
  std::vector<int32_t> r2, c2;
  std::vector<double> v2;
  phased_pad_coo(n_total, nnz, row, col, val_reim, bus_phase, n_bus, r2, c2, v2);
  const int32_t slack3[3] = {0, 1, 2};
  zbus_network net = nullptr;
  ZB_CHECK(zbus_network_create(3 * n_bus, (int64_t)r2.size(), r2.data(), c2.data(), v2.data(),
                               slack3, v_slack_reim, cuda_stream, &net));
  zbus_status s = phased_attach(net, n_total, slack_idx, bus_phase, (cudaStream_t)cuda_stream);
  if (s != ZBUS_OK) {
    std::string msg = g_last_error;
    zbus_network_destroy(net);
    g_last_error = msg;
    return s;
  }
  *out = net;
  return ZBUS_OK;
}

void zbus_network_destroy(zbus_network net) {
  if (!net) return;
  drop_graphs(net);
  drop_groups_of(net);
  if (net->group1) {
    group_free(net->group1);
    delete net->group1;
  }
  if (net->cap_stream) cudaStreamDestroy(net->cap_stream);
  for (auto e : net->prof.ev) cudaEventDestroy(e);
  {
    HostStage& h = net->stage;
    if (h.h2d) cudaStreamSynchronize(h.h2d);
    if (h.d2h) cudaStreamSynchronize(h.d2h);
    for (int s = 0; s < 2; ++s) cudaFree(h.buf[s]);
    if (h.h2d) cudaStreamDestroy(h.h2d);
    if (h.d2h) cudaStreamDestroy(h.d2h);
    cudaEvent_t evs[] = {h.start, h.end, h.in[0], h.in[1], h.done[0], h.done[1], h.out[0], h.out[1]};
    for (auto e : evs)
      if (e) cudaEventDestroy(e);
  }
  cudaFree(net->prof.d_hist);
  cudaFree(net->ws.base);
  free_mixed(net);
  phased_free(net);
  free_adjoint(net);
  cudaFree(net->Z);
  cudaFree(net->w);
  cudaFree(net->ys);
  cudaFree(net->Zr);
  cudaFree(net->Zi);
  cudaFree(net->Zs);
  cudaFree(net->csr_ptr);
  cudaFree(net->csr_col);
  cudaFree(net->csr_val);
  cudaFree(net->bsr_ptr);
  cudaFree(net->bsr_col);
  cudaFree(net->bsr_val);
  cudaFree(net->br_tab);
  cudaFree(net->bsr_br);
  cudaFree(net->t_node);
  cudaFree(net->t_lvl);
  cudaFree(net->t_mask);
  cudaFree(net->t_z);
  cudaFree(net->t_zs);
  cudaFree(net->t_z64);
  cudaFree(net->t_pblk);
  delete net;
}

int32_t zbus_network_size(zbus_network net) {
  return net ? (net->phased ? net->n_user : net->n) : -1;
}

zbus_status zbus_network_get_z(zbus_network net, double* Z_out, double* w_out, void* cuda_stream) {
  g_last_error.clear();
  if (!net) return fail(ZBUS_ERR_ARG, "network is NULL");
  ZB_CHECK(check_device(net));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  ZB_CHECK(ensure_z(net, st));
  if (net->phased) {   // the caller's unknowns only
    if (Z_out) ZB_CHECK(phased_z(net, Z_out, st));
    if (w_out) ZB_CHECK(phased_out(net, 1, (const double*)net->w, w_out, st));
    return ZBUS_OK;
  }
  if (Z_out)
    ZB_CUDA(cudaMemcpyAsync(Z_out, net->Z, (size_t)net->n * net->n * sizeof(double2),
                            cudaMemcpyDeviceToDevice, st));
  if (w_out)
    ZB_CUDA(cudaMemcpyAsync(w_out, net->w, (size_t)net->n * sizeof(double2),
                            cudaMemcpyDeviceToDevice, st));
  return ZBUS_OK;
}

zbus_status zbus_probe_fp64_rate(double* tflops, float* ms, void* cuda_stream) {
  g_last_error.clear();
  if (!tflops && !ms) return fail(ZBUS_ERR_ARG, "both outputs are NULL");
  return probe_fp64_rate(tflops, ms, (cudaStream_t)cuda_stream);
}

zbus_status zbus_network_reserve(zbus_network net, int64_t B, int32_t precision) {
  g_last_error.clear();
  if (!net) return fail(ZBUS_ERR_ARG, "network is NULL");
  if (B < 0 || B > INT32_MAX / 4) return fail(ZBUS_ERR_ARG, "B out of range");
  if (!known_precision(precision)) return fail(ZBUS_ERR_ARG, "unknown precision");
  ZB_CHECK(check_device(net));
  ZB_CHECK(ensure_workspace(net, B));
  ZB_CHECK(ensure_3m(net, nullptr));
  if (precision == ZBUS_TREE_SWEEP) ZB_CHECK(prepare_tree(net, nullptr));
  else if (precision != ZBUS_FP64) ZB_CHECK(prepare_mixed(net, precision, nullptr));
  return ZBUS_OK;
}

}  // extern "C"

namespace zbus {
namespace {

// The solve on device buffers (the arguments checked by zbus_solve).
zbus_status solve_device(zbus_network net, int64_t B, const double* S_wye, const double* S_delta,
                         const double* V_init, double tol, int32_t max_iter,
                         const zbus_solve_opts& o, double* V_out, int32_t* iters,
                         uint8_t* converged, cudaStream_t st) {
  ZB_CHECK(ensure_workspace(net, B));
  // the FP64 operands (the plain method's contraction, the mixed forms'
  // correction sweeps), formed again if a serving cache released them
  ZB_CHECK(ensure_3m(net, st));
  if (o.precision != ZBUS_FP64) {
    // mixed precision: a group of one feeder
    if (!net->group1) net->group1 = new Group();
    if (!group_current(net->group1, {net}, {B}, o.precision))
      ZB_CHECK(group_build(net->group1, {net}, {B}, o.precision, st));
    return run_group(net->group1, {net}, {B}, {S_wye}, {S_delta}, {V_init}, {V_out}, {iters},
                     {converged}, tol, max_iter, o, st);
  }

  net->last_group = nullptr;   // the plain method has no device-side waits
  if (o.profile != 1 && B <= F64_BM && net->n_pad <= FUSED_MAX_NPAD) {
    // a small feeder and at most one tile of scenarios: the whole solve in
    // one launch (bitwise the results of the sweep-per-launch path below)
    launch_solve_fused_f64(net->Zr, net->Zi, net->Zs, net->w, (const double2*)V_init,
                           (const double2*)S_wye, (const double2*)S_delta, net->n, net->n_pad,
                           (int)B, tol, max_iter, o.conv_rule, (double2*)V_out, iters, converged,
                           st);
    ZB_CUDA(cudaGetLastError());
    return ZBUS_OK;
  }
  SolveCtx h;
  std::memset(&h, 0, sizeof(h));
  h.S_wye = (const double2*)S_wye;
  h.S_del = (const double2*)S_delta;
  h.V_init = (const double2*)V_init;
  h.V = (double2*)V_out;
  h.iters = iters;
  h.conv = converged;
  h.list = net->ws.list;
  h.keep = net->ws.keep;
  h.part = net->ws.part;
  h.Iop = net->ws.Iop;
  h.tol = tol;
  h.mismatch_tol = o.mismatch_tol > 0 ? o.mismatch_tol : 1e-6;
  h.B = (int32_t)B;
  h.max_iter = max_iter;
  h.rule = o.conv_rule;
  h.ntn = net->n_pad / F64_BN;
  const int grid = gemm_f64_grid((int)B, net->n_pad);
  if (o.profile == 1) {
    ZB_CHECK(ensure_profile(net, max_iter));
    Profile& P = net->prof;
    ZB_CUDA(cudaMemsetAsync(P.d_hist, 0, (size_t)max_iter * sizeof(int32_t), st));
    h.hist = P.d_hist;
    h.hist_n = max_iter;
    launch_init(net->ws.ctx, h, net->w, net->n, (int)B, st);
    for (int k = 0; k < max_iter; ++k)
      ZB_CHECK(enqueue_sweep_f64(net, B, grid, 0, false, st, &P.ev[(size_t)4 * k]));
    P.sweeps = max_iter;
  } else {
    launch_init(net->ws.ctx, h, net->w, net->n, (int)B, st);
    ZB_CUDA(cudaGetLastError());
    if (use_graphs()) {
      GraphEntry* g = nullptr;
      ZB_CHECK(get_while_graph(net, B, ZBUS_FP64, grid, enqueue_sweep_f64, &g));
      ZB_CUDA(cudaGraphLaunch(g->exec, st));
    } else {
      for (int k = 0; k < max_iter; ++k) ZB_CHECK(enqueue_sweep_f64(net, B, grid, 0, false, st));
    }
  }
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}


// The solve on device buffers in the caller's layout: for a partial-phase
// network the arrays move into the padded layout and the voltages back.
zbus_status solve_device_user(zbus_network net, int64_t B, const double* S_wye,
                              const double* S_delta, const double* V_init, double tol,
                              int32_t max_iter, const zbus_solve_opts& o, double* V_out,
                              int32_t* iters, uint8_t* converged, cudaStream_t st) {
  if (!net->phased)
    return solve_device(net, B, S_wye, S_delta, V_init, tol, max_iter, o, V_out, iters,
                        converged, st);
  double* buf[4];
  ZB_CHECK(phased_stage(net, B, buf));
  if (S_wye) ZB_CHECK(phased_in(net, B, S_wye, buf[0], false, st));
  if (S_delta) ZB_CHECK(phased_in(net, B, S_delta, buf[1], true, st));
  if (V_init) ZB_CHECK(phased_in(net, B, V_init, buf[2], false, st));
  ZB_CHECK(solve_device(net, B, S_wye ? buf[0] : nullptr, S_delta ? buf[1] : nullptr,
                        V_init ? buf[2] : nullptr, tol, max_iter, o, buf[3], iters, converged,
                        st));
  return phased_out(net, B, buf[3], V_out, st);
}

// Staging of host-buffer solves: two sets of device buffers (loads, warm
// start, outputs) of `cap` scenarios, copy streams and events.
zbus_status ensure_stage(zbus_network net, int64_t cap) {
  HostStage& h = net->stage;
  if (!h.h2d) {
    ZB_CUDA(cudaStreamCreateWithFlags(&h.h2d, cudaStreamNonBlocking));
    ZB_CUDA(cudaStreamCreateWithFlags(&h.d2h, cudaStreamNonBlocking));
    cudaEvent_t* evs[] = {&h.start, &h.end, &h.in[0], &h.in[1], &h.done[0], &h.done[1],
                          &h.out[0], &h.out[1]};
    for (auto e : evs) ZB_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  if (h.cap >= cap) return ZBUS_OK;
  ZB_CUDA(cudaDeviceSynchronize());
  for (int s = 0; s < 2; ++s) {
    cudaFree(h.buf[s]);
    h.buf[s] = nullptr;
  }
  h.cap = 0;
  const size_t vec = (size_t)cap * net->n * 2;   // doubles of one [cap][n] complex array
  for (int s = 0; s < 2; ++s)
    ZB_CUDA(cudaMalloc((void**)&h.buf[s], 4 * vec * sizeof(double) + (size_t)cap * 8));
  h.cap = cap;
  return ZBUS_OK;
}

// The solve on host buffers: chunks of the batch staged through two sets of
// device buffers, so that the copies of one chunk (host to device on one
// stream, device to host on another) overlap the sweeps of the next on the
// caller's stream.  The caller's stream waits for the last copy.
zbus_status solve_host(zbus_network net, int64_t B, const double* S_wye, const double* S_delta,
                       const double* V_init, double tol, int32_t max_iter,
                       const zbus_solve_opts& o, double* V_out, int32_t* iters,
                       uint8_t* converged, cudaStream_t st) {
  // four chunks for the defect forms (whose sweeps take about as long as the
  // copies), 1/8, 3/8, 3/8 and 1/8 of the batch in multiples of 128: the
  // small first chunk shortens the copy nothing overlaps at the start, the
  // small last one the copy back at the end, and each middle chunk's copy
  // fits under the solve of the chunk before it.  One chunk for the plain
  // method, whose FP64 sweeps take some fifty times longer than its copies
  // and run less efficiently on smaller batches, and for inputs under 256
  // MB (about a millisecond of copies), which a chunk's fixed cost outweighs
  const size_t n2u = (size_t)(net->phased ? net->n_user : net->n) * 2;
  const size_t in_bytes = (size_t)B * n2u * sizeof(double) *
                          ((S_wye ? 1 : 0) + (S_delta ? 1 : 0) + (V_init ? 1 : 0));
  std::vector<int64_t> lo{0};
  if (B <= 2048 || o.precision == ZBUS_FP64 || in_bytes < ((size_t)256 << 20)) {
    lo.push_back(B);
  } else {
    const int64_t c0 = round_up((int)((B + 7) / 8), 128);
    const int64_t c1 = round_up((int)((3 * B + 7) / 8), 128);
    for (int64_t b : {c0, c0 + c1, c0 + 2 * c1})
      if (b < B) lo.push_back(b);
    lo.push_back(B);
  }
  int64_t C = 0;
  for (size_t k = 0; k + 1 < lo.size(); ++k) C = std::max(C, lo[k + 1] - lo[k]);
  ZB_CHECK(ensure_stage(net, C));
  ZB_CHECK(ensure_workspace(net, C));
  HostStage& h = net->stage;
  const size_t n2 = (size_t)(net->phased ? net->n_user : net->n) * 2;   // doubles per scenario
  const size_t vec = (size_t)h.cap * n2;
  ZB_CUDA(cudaEventRecord(h.start, st));
  ZB_CUDA(cudaStreamWaitEvent(h.h2d, h.start, 0));
  ZB_CUDA(cudaStreamWaitEvent(h.d2h, h.start, 0));
  for (size_t k = 0; k + 1 < lo.size(); ++k) {
    const int64_t b0 = lo[k], Bk = lo[k + 1] - lo[k];
    const int s = (int)(k & 1);
    double* sw = h.buf[s];
    double* sd = sw + vec;
    double* v0 = sd + vec;
    double* vo = v0 + vec;
    int32_t* it = reinterpret_cast<int32_t*>(vo + vec);
    uint8_t* cv = reinterpret_cast<uint8_t*>(it + h.cap);
    if (k >= 2) {   // the set's previous chunk: inputs consumed, outputs copied out
      ZB_CUDA(cudaStreamWaitEvent(h.h2d, h.done[s], 0));
      ZB_CUDA(cudaStreamWaitEvent(h.h2d, h.out[s], 0));
    }
    const size_t bytes = (size_t)Bk * n2 * sizeof(double);
    if (S_wye)
      ZB_CUDA(cudaMemcpyAsync(sw, S_wye + b0 * n2, bytes, cudaMemcpyHostToDevice, h.h2d));
    if (S_delta)
      ZB_CUDA(cudaMemcpyAsync(sd, S_delta + b0 * n2, bytes, cudaMemcpyHostToDevice, h.h2d));
    if (V_init)
      ZB_CUDA(cudaMemcpyAsync(v0, V_init + b0 * n2, bytes, cudaMemcpyHostToDevice, h.h2d));
    ZB_CUDA(cudaEventRecord(h.in[s], h.h2d));
    ZB_CUDA(cudaStreamWaitEvent(st, h.in[s], 0));
    ZB_CHECK(solve_device_user(net, Bk, S_wye ? sw : nullptr, S_delta ? sd : nullptr,
                               V_init ? v0 : nullptr, tol, max_iter, o, vo, it, cv, st));
    ZB_CUDA(cudaEventRecord(h.done[s], st));
    ZB_CUDA(cudaStreamWaitEvent(h.d2h, h.done[s], 0));
    ZB_CUDA(cudaMemcpyAsync(V_out + b0 * n2, vo, bytes, cudaMemcpyDeviceToHost, h.d2h));
    ZB_CUDA(cudaMemcpyAsync(iters + b0, it, (size_t)Bk * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            h.d2h));
    ZB_CUDA(cudaMemcpyAsync(converged + b0, cv, (size_t)Bk, cudaMemcpyDeviceToHost, h.d2h));
    ZB_CUDA(cudaEventRecord(h.out[s], h.d2h));
  }
  ZB_CUDA(cudaEventRecord(h.end, h.d2h));
  ZB_CUDA(cudaStreamWaitEvent(st, h.end, 0));
  return ZBUS_OK;
}

}  // namespace
}  // namespace zbus

extern "C" {

zbus_status zbus_solve(zbus_network net, int64_t B, const double* S_wye, const double* S_delta,
                       const double* V_init, double tol, int32_t max_iter,
                       const zbus_solve_opts* opts, double* V_out, int32_t* iters,
                       uint8_t* converged, void* cuda_stream) {
  NvtxRange nvtx_range("zbus_solve");
  g_last_error.clear();
  if (!net) return fail(ZBUS_ERR_ARG, "network is NULL");
  if (B < 0 || B > INT32_MAX / 4) return fail(ZBUS_ERR_ARG, "B out of range");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(ZBUS_ERR_ARG, "tol must be finite, >= 0");
  if (max_iter < 1) return fail(ZBUS_ERR_ARG, "max_iter must be >= 1");
  zbus_solve_opts o;
  zbus_solve_opts_default(&o);
  if (opts) o = *opts;
  if (o.conv_rule != ZBUS_CONV_MAXABS && o.conv_rule != ZBUS_CONV_SUMMAG)
    return fail(ZBUS_ERR_ARG, "unknown convergence rule");
  if (!known_precision(o.precision)) return fail(ZBUS_ERR_ARG, "unknown precision");
  if (B == 0) return ZBUS_OK;
  if (!V_out || !iters || !converged) return fail(ZBUS_ERR_ARG, "an output pointer is NULL");
  if (S_delta && !net->bus_aligned)
    return fail(ZBUS_ERR_ARG, "delta loads need three unknowns per bus (n % 3 == 0)");
  ZB_CHECK(check_device(net));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // every buffer on the device, or every buffer in host memory
  const int kinds[] = {buffer_kind(S_wye), buffer_kind(S_delta), buffer_kind(V_init),
                       buffer_kind(V_out), buffer_kind(iters), buffer_kind(converged)};
  int host = 0, dev = 0;
  for (int x : kinds) {
    host += x == 0;
    dev += x == 1;
  }
  if (host && dev) return fail(ZBUS_ERR_ARG, "buffers must all be on the device or all in host memory");
  if (host) {
    if (o.profile == 1) return fail(ZBUS_ERR_ARG, "profiling needs device buffers");
    return solve_host(net, B, S_wye, S_delta, V_init, tol, max_iter, o, V_out, iters, converged,
                      st);
  }
  return solve_device_user(net, B, S_wye, S_delta, V_init, tol, max_iter, o, V_out, iters,
                           converged, st);
}

zbus_status zbus_solve_batched(const zbus_batch_item* items, int32_t n_items, double tol,
                               int32_t max_iter, const zbus_solve_opts* opts, void* cuda_stream) {
  NvtxRange nvtx_range("zbus_solve_batched");
  g_last_error.clear();
  if (n_items < 0 || (n_items > 0 && !items)) return fail(ZBUS_ERR_ARG, "items is NULL");
  if (n_items == 0) return ZBUS_OK;
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(ZBUS_ERR_ARG, "tol must be finite, >= 0");
  if (max_iter < 1) return fail(ZBUS_ERR_ARG, "max_iter must be >= 1");
  zbus_solve_opts o;
  zbus_solve_opts_default(&o);
  if (opts) o = *opts;
  if (o.conv_rule != ZBUS_CONV_MAXABS && o.conv_rule != ZBUS_CONV_SUMMAG)
    return fail(ZBUS_ERR_ARG, "unknown convergence rule");
  if (!known_precision(o.precision)) return fail(ZBUS_ERR_ARG, "unknown precision");
  std::vector<zbus_network> nets;
  std::vector<int64_t> Bs;
  std::vector<const double*> Sw, Sd, V0;
  std::vector<double*> Vo;
  std::vector<int32_t*> it;
  std::vector<uint8_t*> cv;
  std::set<zbus_network> seen;
  for (int32_t k = 0; k < n_items; ++k) {
    const zbus_batch_item& x = items[k];
    if (!x.net) return fail(ZBUS_ERR_ARG, "item " + std::to_string(k) + ": network is NULL");
    if (!seen.insert(x.net).second)
      return fail(ZBUS_ERR_ARG, "item " + std::to_string(k) + ": a network may appear once");
    if (x.B < 0 || x.B > INT32_MAX / 4) return fail(ZBUS_ERR_ARG, "item B out of range");
    if (x.B > 0 && (!x.V_out || !x.iters || !x.converged))
      return fail(ZBUS_ERR_ARG, "item " + std::to_string(k) + ": an output pointer is NULL");
    if (x.S_delta && !x.net->bus_aligned)
      return fail(ZBUS_ERR_ARG, "delta loads need three unknowns per bus (n % 3 == 0)");
    if (x.net->phased)
      return fail(ZBUS_ERR_UNSUPPORTED, "batched solves take three-phase networks; solve a "
                                        "partial-phase network with zbus_solve");
    ZB_CHECK(check_device(x.net));
    if (x.B == 0) continue;
    nets.push_back(x.net);
    Bs.push_back(x.B);
    Sw.push_back(x.S_wye);
    Sd.push_back(x.S_delta);
    V0.push_back(x.V_init);
    Vo.push_back(x.V_out);
    it.push_back(x.iters);
    cv.push_back(x.converged);
  }
  if (nets.empty()) return ZBUS_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (o.precision == ZBUS_FP64) {
    // the plain method runs feeder after feeder
    for (size_t k = 0; k < nets.size(); ++k)
      ZB_CHECK(zbus_solve(nets[k], Bs[k], Sw[k], Sd[k], V0[k], tol, max_iter, &o, Vo[k], it[k],
                          cv[k], cuda_stream));
    return ZBUS_OK;
  }
  for (size_t k = 0; k < nets.size(); ++k) ZB_CHECK(ensure_workspace(nets[k], Bs[k]));
  Group* g = nullptr;
  for (Group* c : g_batch_groups)
    if (group_current(c, nets, Bs, o.precision)) g = c;
  if (!g) {
    g = new Group();
    zbus_status s = group_build(g, nets, Bs, o.precision, st);
    if (s != ZBUS_OK) {
      group_free(g);
      delete g;
      return s;
    }
    g_batch_groups.push_back(g);
  }
  return run_group(g, nets, Bs, Sw, Sd, V0, Vo, it, cv, tol, max_iter, o, st);
}

zbus_status zbus_last_profile(zbus_network net, int32_t max_n, float* ms, int32_t* active,
                              int32_t* sweeps) {
  g_last_error.clear();
  if (!net) return fail(ZBUS_ERR_ARG, "network is NULL");
  Profile& P = net->prof;
  if (sweeps) *sweeps = P.sweeps;
  const int m = std::min(max_n, P.sweeps);
  if (m <= 0) return ZBUS_OK;
  if (ms) {
    for (int k = 0; k < m; ++k)
      for (int q = 0; q < 3; ++q)
        ZB_CUDA(cudaEventElapsedTime(&ms[3 * k + q], P.ev[(size_t)4 * k + q],
                                     P.ev[(size_t)4 * k + q + 1]));
  }
  if (active) ZB_CUDA(cudaMemcpy(active, P.d_hist, (size_t)m * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost));
  return ZBUS_OK;
}

zbus_status zbus_power_mismatch(zbus_network net, int64_t B, const double* V,
                                const double* S_wye, const double* S_delta, double* out,
                                void* cuda_stream) {
  NvtxRange nvtx_range("zbus_power_mismatch");
  g_last_error.clear();
  if (!net) return fail(ZBUS_ERR_ARG, "network is NULL");
  if (B < 0 || B > INT32_MAX) return fail(ZBUS_ERR_ARG, "B out of range");
  if (B == 0) return ZBUS_OK;
  if (!V || !out) return fail(ZBUS_ERR_ARG, "V or out is NULL");
  if (S_delta && !net->bus_aligned)
    return fail(ZBUS_ERR_ARG, "delta loads need three unknowns per bus (n % 3 == 0)");
  ZB_CHECK(check_device(net));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (net->phased) {   // into the padded layout first
    double* buf[4];
    ZB_CHECK(phased_stage(net, B, buf));
    ZB_CHECK(phased_in(net, B, V, buf[3], false, st));
    if (S_wye) ZB_CHECK(phased_in(net, B, S_wye, buf[0], false, st));
    if (S_delta) ZB_CHECK(phased_in(net, B, S_delta, buf[1], true, st));
    V = buf[3];
    S_wye = S_wye ? buf[0] : nullptr;
    S_delta = S_delta ? buf[1] : nullptr;
  }
  launch_mismatch((const double2*)V, (const double2*)S_wye, (const double2*)S_delta,
                  net->csr_ptr, net->csr_col, net->csr_val, net->ys, net->n, (int)B, out, st);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

}  // extern "C"
