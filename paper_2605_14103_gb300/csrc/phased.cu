// Partial-phase networks: the caller describes a feeder whose buses carry any
// subset of the phases (single- and two-phase laterals); the device solves
// the network padded to three phase slots per bus, an absent phase being an
// isolated node with a unit self-admittance and no load (its voltage stays 0
// in every form; Sec. II-B's map restricted to the present phases).  The
// kernels here move the caller's [B][n_user] arrays (present phases in
// ascending global index) into and out of the padded [B][n] layout.
#include <algorithm>
#include <cstring>
#include <map>
#include <set>
#include <vector>

#include "zbus_internal.cuh"

namespace zbus {
namespace {

// dst[b][map[j]] = src[b][j] (dst zeroed beforehand); with keep, entries
// whose keep[j] is 0 stay zero.
__global__ void k_ph_scatter(const double2* __restrict__ src, double2* __restrict__ dst, int B,
                             int n_user, int n, const int32_t* __restrict__ map,
                             const uint8_t* __restrict__ keep) {
  const int64_t total = (int64_t)B * n_user;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / n_user;
    const int j = (int)(t - b * n_user);
    if (keep && !keep[j]) continue;
    if (!ZB_IN(map[j], n, 0x501u)) continue;
    dst[b * n + map[j]] = src[t];
  }
}

// dst[b][j] = src[b][map[j]]; with keep, zero where keep[j] is 0.
__global__ void k_ph_gather(const double2* __restrict__ src, double2* __restrict__ dst, int B,
                            int n_user, int n, const int32_t* __restrict__ map,
                            const uint8_t* __restrict__ keep) {
  const int64_t total = (int64_t)B * n_user;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / n_user;
    const int j = (int)(t - b * n_user);
    dst[t] = (keep && !keep[j]) || !ZB_IN(map[j], n, 0x502u) ? make_double2(0.0, 0.0)
                                                              : src[b * n + map[j]];
  }
}

// Z_user[i][j] = Z[map[i]][map[j]].
__global__ void k_ph_gather_z(const double2* __restrict__ Z, double2* __restrict__ Zu, int n_user,
                              int n, const int32_t* __restrict__ map) {
  const int64_t total = (int64_t)n_user * n_user;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n_user), j = (int)(t - (int64_t)i * n_user);
    Zu[t] = ZB_IN(map[i], n, 0x503u) && ZB_IN(map[j], n, 0x504u) ? Z[(int64_t)map[i] * n + map[j]]
                                                                 : make_double2(0.0, 0.0);
  }
}

int grid_for(int64_t total) { return (int)std::min<int64_t>(4096, (total + 255) / 256); }

}  // namespace

zbus_status phased_validate(int32_t n_total, const int32_t* slack_idx, const int32_t* bus_phase,
                            int32_t* n_bus) {
  if (!bus_phase) return fail(ZBUS_ERR_ARG, "bus_phase is NULL");
  std::set<int32_t> seen;
  int32_t top = 0;
  for (int32_t g = 0; g < n_total; ++g) {
    const int32_t v = bus_phase[g];
    if (v < 0 || v > (1 << 27)) return fail(ZBUS_ERR_ARG, "bus_phase out of range at " + std::to_string(g));
    if (!seen.insert(v).second)
      return fail(ZBUS_ERR_ARG, "two global indices share bus_phase " + std::to_string(v));
    top = std::max(top, v);
  }
  for (int p = 0; p < 3; ++p)
    if (bus_phase[slack_idx[p]] != p)
      return fail(ZBUS_ERR_ARG, "the slack phases must map to bus 0, phases 0, 1, 2 in order");
  for (int32_t g = 0; g < n_total; ++g) {
    bool slack = g == slack_idx[0] || g == slack_idx[1] || g == slack_idx[2];
    if (!slack && bus_phase[g] < 3)
      return fail(ZBUS_ERR_ARG, "a non-slack index maps to the slack bus");
  }
  *n_bus = top / 3 + 1;
  std::vector<uint8_t> has((size_t)*n_bus, 0);
  for (int32_t v : seen) has[v / 3] = 1;
  for (int32_t k = 0; k < *n_bus; ++k)
    if (!has[k]) return fail(ZBUS_ERR_ARG, "bus " + std::to_string(k) + " has no phase (buses must be numbered 0 .. n_bus - 1)");
  return ZBUS_OK;
}

void phased_pad_coo(int32_t n_total, int64_t nnz, const int32_t* row, const int32_t* col,
                    const double* val, const int32_t* bus_phase, int32_t n_bus,
                    std::vector<int32_t>& r2, std::vector<int32_t>& c2, std::vector<double>& v2) {
  const int32_t n3 = 3 * n_bus;
  std::vector<uint8_t> used(n3, 0);
  for (int32_t g = 0; g < n_total; ++g) used[bus_phase[g]] = 1;
  r2.clear();
  c2.clear();
  v2.clear();
  r2.reserve(nnz + n3);
  c2.reserve(nnz + n3);
  v2.reserve(2 * (nnz + n3));
  for (int64_t t = 0; t < nnz; ++t) {
    r2.push_back(bus_phase[row[t]]);
    c2.push_back(bus_phase[col[t]]);
    v2.push_back(val[2 * t]);
    v2.push_back(val[2 * t + 1]);
  }
  for (int32_t g = 3; g < n3; ++g)
    if (!used[g]) {   // an absent phase: isolated, unit self-admittance
      r2.push_back(g);
      c2.push_back(g);
      v2.push_back(1.0);
      v2.push_back(0.0);
    }
}

zbus_status phased_attach(zbus_network net, int32_t n_total, const int32_t* slack_idx,
                          const int32_t* bus_phase, cudaStream_t st) {
  std::vector<int32_t> map;
  std::vector<uint8_t> dvalid;
  std::set<int32_t> present(bus_phase, bus_phase + n_total);
  for (int32_t g = 0; g < n_total; ++g) {
    if (g == slack_idx[0] || g == slack_idx[1] || g == slack_idx[2]) continue;
    const int32_t v = bus_phase[g];
    map.push_back(v - 3);
    const int32_t k = v / 3, x = v % 3;
    dvalid.push_back(present.count(3 * k + (x + 1) % 3) ? 1 : 0);
  }
  net->n_user = (int)map.size();
  ZB_CUDA(cudaMalloc((void**)&net->ph_map, std::max<size_t>(1, map.size()) * sizeof(int32_t)));
  ZB_CUDA(cudaMalloc((void**)&net->ph_dvalid, std::max<size_t>(1, dvalid.size())));
  ZB_CUDA(cudaMemcpyAsync(net->ph_map, map.data(), map.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice, st));
  ZB_CUDA(cudaMemcpyAsync(net->ph_dvalid, dvalid.data(), dvalid.size(), cudaMemcpyHostToDevice,
                          st));
  ZB_CUDA(cudaStreamSynchronize(st));
  net->phased = true;
  return ZBUS_OK;
}

zbus_status phased_stage(zbus_network net, int64_t B, double** bufs) {
  const size_t one = (size_t)B * net->n * 2;   // doubles of a padded [B][n] complex array
  if (net->ph_cap < B) {
    ZB_CUDA(cudaDeviceSynchronize());
    cudaFree(net->ph_buf);
    net->ph_buf = nullptr;
    net->ph_cap = 0;
    ZB_CUDA(cudaMalloc((void**)&net->ph_buf, 4 * one * sizeof(double)));
    net->ph_cap = B;
  }
  const size_t cap = (size_t)net->ph_cap * net->n * 2;
  for (int a = 0; a < 4; ++a) bufs[a] = net->ph_buf + a * cap;
  return ZBUS_OK;
}

zbus_status phased_in(zbus_network net, int64_t B, const double* src, double* dst, bool delta,
                      cudaStream_t st) {
  ZB_CUDA(cudaMemsetAsync(dst, 0, (size_t)B * net->n * sizeof(double2), st));
  if (B == 0 || net->n_user == 0) return ZBUS_OK;
  const int64_t total = B * (int64_t)net->n_user;
  k_ph_scatter<<<grid_for(total), 256, 0, st>>>((const double2*)src, (double2*)dst, (int)B,
                                                 net->n_user, net->n, net->ph_map,
                                                 delta ? net->ph_dvalid : nullptr);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

zbus_status phased_out(zbus_network net, int64_t B, const double* src, double* dst,
                       cudaStream_t st) {
  if (B == 0 || net->n_user == 0) return ZBUS_OK;
  const int64_t total = B * (int64_t)net->n_user;
  k_ph_gather<<<grid_for(total), 256, 0, st>>>((const double2*)src, (double2*)dst, (int)B,
                                                net->n_user, net->n, net->ph_map, nullptr);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

zbus_status phased_out_delta(zbus_network net, int64_t B, const double* src, double* dst,
                             cudaStream_t st) {
  if (B == 0 || net->n_user == 0) return ZBUS_OK;
  const int64_t total = B * (int64_t)net->n_user;
  k_ph_gather<<<grid_for(total), 256, 0, st>>>((const double2*)src, (double2*)dst, (int)B,
                                                net->n_user, net->n, net->ph_map,
                                                net->ph_dvalid);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

zbus_status phased_z(zbus_network net, double* Z_out, cudaStream_t st) {
  const int64_t total = (int64_t)net->n_user * net->n_user;
  if (total == 0) return ZBUS_OK;
  k_ph_gather_z<<<grid_for(total), 256, 0, st>>>(net->Z, (double2*)Z_out, net->n_user, net->n,
                                                  net->ph_map);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

void phased_free(zbus_network net) {
  cudaFree(net->ph_map);
  cudaFree(net->ph_dvalid);
  cudaFree(net->ph_buf);
  net->ph_map = nullptr;
  net->ph_dvalid = nullptr;
  net->ph_buf = nullptr;
  net->ph_cap = 0;
}

}  // namespace zbus

namespace zbus {
ZB_CHECK_WORD_ACCESSOR(check_word_phased)
}  // namespace zbus
