// Constant-power load currents (Sec. II-B), shared by the FP64 and the mixed
// sweeps and by the mismatch checks.
#pragma once

#include <cuda_runtime.h>

namespace zbus {

// conj(S / v) = conj(S) v / |v|^2; zero when the slot has no load.
__device__ __forceinline__ double2 load_draw(double2 S, double2 v) {
  if (S.x == 0.0 && S.y == 0.0) return make_double2(0.0, 0.0);
  const double inv = 1.0 / (v.x * v.x + v.y * v.y);
  return make_double2((S.x * v.x + S.y * v.y) * inv, (S.x * v.y - S.y * v.x) * inv);
}

// Current injection of one bus (three consecutive unknowns).  Wye slot p draws
// conj(S_wye_p / v_p); delta branch xy in order (ab, bc, ca) draws
// conj(S_xy / (v_x - v_y)) from phase x and returns it into phase y.
// Injection = -(drawn).  `m` = number of valid slots (3 unless the network
// ends inside a bus, which only wye loads allow).
__device__ __forceinline__ void bus_injection(const double2* v, const double2* sw,
                                              const double2* sd, int m, double2* inj) {
  double2 d[3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
    d[p] = (p < m && sw) ? load_draw(sw[p], v[p]) : make_double2(0.0, 0.0);
  if (sd && m == 3) {
    const double2 vab = make_double2(v[0].x - v[1].x, v[0].y - v[1].y);
    const double2 vbc = make_double2(v[1].x - v[2].x, v[1].y - v[2].y);
    const double2 vca = make_double2(v[2].x - v[0].x, v[2].y - v[0].y);
    const double2 iab = load_draw(sd[0], vab);
    const double2 ibc = load_draw(sd[1], vbc);
    const double2 ica = load_draw(sd[2], vca);
    d[0].x += iab.x - ica.x; d[0].y += iab.y - ica.y;
    d[1].x += ibc.x - iab.x; d[1].y += ibc.y - iab.y;
    d[2].x += ica.x - ibc.x; d[2].y += ica.y - ibc.y;
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) inj[p] = make_double2(-d[p].x, -d[p].y);
}

// FP32 versions for the mixed sweeps: conj(S / v) with a rounded reciprocal.
__device__ __forceinline__ float2 load_draw_f(float2 S, float2 v) {
  if (S.x == 0.f && S.y == 0.f) return make_float2(0.f, 0.f);
  const float inv = __frcp_rn(__fmaf_rn(v.x, v.x, v.y * v.y));
  return make_float2((S.x * v.x + S.y * v.y) * inv, (S.x * v.y - S.y * v.x) * inv);
}

__device__ __forceinline__ void bus_injection_f(const float2* v, const float2* sw,
                                                const float2* sd, int m, float2* inj) {
  float2 d[3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
    d[p] = (p < m && sw) ? load_draw_f(sw[p], v[p]) : make_float2(0.f, 0.f);
  if (sd && m == 3) {
    const float2 iab = load_draw_f(sd[0], make_float2(v[0].x - v[1].x, v[0].y - v[1].y));
    const float2 ibc = load_draw_f(sd[1], make_float2(v[1].x - v[2].x, v[1].y - v[2].y));
    const float2 ica = load_draw_f(sd[2], make_float2(v[2].x - v[0].x, v[2].y - v[0].y));
    d[0].x += iab.x - ica.x; d[0].y += iab.y - ica.y;
    d[1].x += ibc.x - iab.x; d[1].y += ibc.y - iab.y;
    d[2].x += ica.x - ibc.x; d[2].y += ica.y - ibc.y;
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) inj[p] = make_float2(-d[p].x, -d[p].y);
}

}  // namespace zbus
