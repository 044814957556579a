// zbus_solve_noalloc: the plain FP64 solve with its scratch in a fixed,
// file-scope device array instead of memory obtained from cudaMalloc.
//
// It exists for callers that cannot allocate device memory when they solve:
// processes whose device memory is entirely owned by another allocator (a
// framework's caching pool that has reserved the free memory), real-time
// control loops that forbid allocation after start-up, and plug-in hosts that
// do not let their plug-ins allocate.  Such a caller creates the network once
// at start-up (zbus_network_create allocates) and then calls this entry point,
// which calls no cudaMalloc, cudaFree or allocating library routine.
//
// The scratch array is STATIC_SCRATCH_BYTES (16 MiB).  The CUDA runtime loads
// it on a device lazily, when its address is first asked for; so that this
// never happens inside a call that must not allocate, zbus_network_create
// asks for it (noalloc_prepare), and every device on which a network was
// created holds the array from then until the process exits.  All calls share
// it and it keeps the last call's contents, so calls that overlap on the GPU
// (on different streams, or from several host threads) race on it.  Every
// array argument must be device memory: the sweeps read and write the
// caller's arrays directly, with no staging.
#include <cmath>
#include <cstring>
#include <mutex>

#include "zbus_internal.cuh"

namespace zbus {
namespace {

constexpr size_t STATIC_SCRATCH_BYTES = size_t(16) << 20;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

std::mutex g_addr_mu;
void* g_addr[MAX_DEVICES] = {};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array on the current device.  The name
// g_static_scratch in host code is only a host-side stand-in, so the address
// is looked up once per device (with that device current) and cached.
zbus_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= MAX_DEVICES) return fail(ZBUS_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)", __FILE__, __LINE__);
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return ZBUS_OK;
}

}  // namespace

zbus_status noalloc_prepare(int dev) {
  void* p = nullptr;
  return scratch_address(dev, &p);
}

}  // namespace zbus

using namespace zbus;

extern "C" zbus_status zbus_solve_noalloc(zbus_network net, int64_t B, const double* S_wye,
                                          const double* S_delta, const double* V_init,
                                          double tol, int32_t max_iter, int32_t conv_rule,
                                          double* V_out, int32_t* iters, uint8_t* converged,
                                          void* cuda_stream) {
  set_error("");
  if (!net) return fail(ZBUS_ERR_ARG, "network is NULL");
  if (B < 0 || B > INT32_MAX / 4) return fail(ZBUS_ERR_ARG, "B out of range");
  if (!(tol >= 0.0) || !(tol < INFINITY)) return fail(ZBUS_ERR_ARG, "tol must be finite, >= 0");
  if (max_iter < 1) return fail(ZBUS_ERR_ARG, "max_iter must be >= 1");
  if (conv_rule != ZBUS_CONV_MAXABS && conv_rule != ZBUS_CONV_SUMMAG)
    return fail(ZBUS_ERR_ARG, "unknown convergence rule");
  if (net->phased)
    return fail(ZBUS_ERR_UNSUPPORTED, "the allocation-free solve takes three-phase networks");
  if (!net->Zr)   // released by a serving loop: forming it again would allocate
    return fail(ZBUS_ERR_UNSUPPORTED,
                "the network's FP64 operands were released; zbus_network_reserve forms them");
  if (B == 0) return ZBUS_OK;
  if (!V_out || !iters || !converged) return fail(ZBUS_ERR_ARG, "an output pointer is NULL");
  if (S_delta && !net->bus_aligned)
    return fail(ZBUS_ERR_ARG, "delta loads need three unknowns per bus (n % 3 == 0)");

  // scratch layout: context | active list | keep marks | per-tile partials | 3M operands
  const int ntn = net->n_pad / F64_BN;
  const size_t o_list = a256(sizeof(SolveCtx));
  const size_t o_keep = o_list + a256((size_t)B * sizeof(int32_t));
  const size_t o_part = o_keep + a256((size_t)B);
  const size_t o_iop = o_part + a256((size_t)B * ntn * 2 * sizeof(double));
  const size_t need = o_iop + (size_t)3 * B * net->n_pad * sizeof(double);
  if (need > STATIC_SCRATCH_BYTES) {
    const size_t per = sizeof(int32_t) + 1 + (size_t)ntn * 2 * sizeof(double) +
                       (size_t)3 * net->n_pad * sizeof(double);
    return fail(ZBUS_ERR_ARG, "batch too large for the static scratch: needs " +
                                  std::to_string(need) + " bytes, the maximum is " +
                                  std::to_string(STATIC_SCRATCH_BYTES) + " (about " +
                                  std::to_string((STATIC_SCRATCH_BYTES - 4096) / per) +
                                  " scenarios for this network)");
  }
  int dev = -1;
  ZB_CUDA(cudaGetDevice(&dev));
  if (dev != net->device) return fail(ZBUS_ERR_ARG, "current device differs from the network's");
  // no staging here: host arrays are refused (cudaPointerGetAttributes
  // allocates nothing)
  const void* arrays[] = {S_wye, S_delta, V_init, V_out, iters, converged};
  for (const void* a : arrays)
    if (buffer_kind(a) == 0)
      return fail(ZBUS_ERR_ARG, "the allocation-free solve takes device memory only");
  void* base = nullptr;
  ZB_CHECK(scratch_address(dev, &base));
  char* p = (char*)base;

  SolveCtx h;
  memset(&h, 0, sizeof(h));
  h.S_wye = (const double2*)S_wye;
  h.S_del = (const double2*)S_delta;
  h.V_init = (const double2*)V_init;
  h.V = (double2*)V_out;
  h.iters = iters;
  h.conv = converged;
  h.list = (int32_t*)(p + o_list);
  h.keep = (uint8_t*)(p + o_keep);
  h.part = (double*)(p + o_part);
  h.Iop = (double*)(p + o_iop);
  h.tol = tol;
  h.mismatch_tol = 1e-6;
  h.B = (int32_t)B;
  h.max_iter = max_iter;
  h.rule = conv_rule;
  h.ntn = ntn;
  SolveCtx* ctx = (SolveCtx*)p;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the FP64 sweeps have no device-side waits: zbus_last_device_status must
  // not report the error word of an earlier mixed-precision solve
  net->last_group = nullptr;
  // The run start writes the whole context, the active list, iters and flags,
  // so nothing left in the array by an earlier call is read: every partial,
  // keep mark and operand element (padding included) is written in a sweep
  // before the kernels of that sweep read it.
  launch_init(ctx, h, net->w, net->n, (int)B, st);
  const int grid = gemm_f64_grid((int)B, net->n_pad);
  for (int k = 0; k < max_iter; ++k) {
    launch_currents_f64(ctx, net->n, net->n_pad, (int)B, st);
    launch_gemm_f64(ctx, net->Zr, net->Zi, net->Zs, net->w, net->n, net->n_pad, grid, st);
    launch_converge(ctx, (int)B, 0, false, st);
  }
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}
