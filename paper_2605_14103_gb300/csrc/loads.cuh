// Constant-power load currents (Sec. II-B): FP64 for the FP64 sweeps and the
// mismatch checks, double-float for the residual of the mixed defect forms.
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

// Double-float versions for the defect residual.  The current drawn by a
// load, conj(S / v), is formed at the double-float voltage v = vh + vl: the
// FP32 quotient at vh, then one correction step on the remainder
// e = conj(S) - d conj(v), whose leading terms are formed error-free (FMA
// products, two-sums), so the result (dh + dl) is accurate to the
// double-float level and continuous in v.  A current formed from vh alone
// would jump whenever the rounding of vh changes, and the iteration could
// settle into a small cycle instead of its fixed point.
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float4 load_draw_df(float2 S, float2 vh, float2 vl) {
  if (S.x == 0.f && S.y == 0.f) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float inv = __frcp_rn(__fmaf_rn(vh.x, vh.x, vh.y * vh.y));
  const float2 d = make_float2((S.x * vh.x + S.y * vh.y) * inv, (S.x * vh.y - S.y * vh.x) * inv);
  // real part: S.x - d.x vh.x - d.y vh.y - (d.x vl.x + d.y vl.y)
  const float p1 = d.x * vh.x, e1 = __fmaf_rn(d.x, vh.x, -p1);
  const float p2 = d.y * vh.y, e2 = __fmaf_rn(d.y, vh.y, -p2);
  float s1, t1, s2, t2;
  df_two_sum(S.x, -p1, s1, t1);
  df_two_sum(s1, -p2, s2, t2);
  const float er = s2 + (((t1 + t2) - (e1 + e2)) - (d.x * vl.x + d.y * vl.y));
  // imaginary part: -S.y - d.y vh.x + d.x vh.y - (d.y vl.x - d.x vl.y)
  const float q1 = d.y * vh.x, f1 = __fmaf_rn(d.y, vh.x, -q1);
  const float q2 = d.x * vh.y, f2 = __fmaf_rn(d.x, vh.y, -q2);
  df_two_sum(-S.y, -q1, s1, t1);
  df_two_sum(s1, q2, s2, t2);
  const float ei = s2 + (((t1 + t2) - f1 + f2) - (d.y * vl.x - d.x * vl.y));
  // d + e / conj(vh) = d + e vh / |vh|^2
  return make_float4(d.x, (er * vh.x - ei * vh.y) * inv, d.y, (er * vh.y + ei * vh.x) * inv);
}

// Injection of one bus with every current in double-float: inj[p] and
// injl[p] the hi and lo parts (rules of bus_injection, m == 3 for delta).
__device__ __forceinline__ void bus_injection_df(const float2* vh, const float2* vl,
                                                 const float2* sw, const float2* sd, int m,
                                                 float2* inj, float2* injl) {
  float4 dw[3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
    dw[p] = (p < m && sw) ? load_draw_df(sw[p], vh[p], vl[p]) : make_float4(0.f, 0.f, 0.f, 0.f);
  if (sd && m == 3) {
    float4 ib[3];   // branches ab, bc, ca on the double-float line-to-line voltages
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const int y = x == 2 ? 0 : x + 1;
      float uhx, ulx, uhy, uly;
      df_two_sum(vh[x].x, -vh[y].x, uhx, ulx);
      df_two_sum(vh[x].y, -vh[y].y, uhy, uly);
      ulx += vl[x].x - vl[y].x;
      uly += vl[x].y - vl[y].y;
      ib[x] = load_draw_df(sd[x], make_float2(uhx, uhy), make_float2(ulx, uly));
    }
    // phase x draws branch x and returns branch x - 1
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const int w = x == 0 ? 2 : x - 1;
      float h, l;
      df_two_sum(dw[x].x, ib[x].x, h, l);
      float h2, l2;
      df_two_sum(h, -ib[w].x, h2, l2);
      dw[x].x = h2;
      dw[x].y += l + l2 + ib[x].y - ib[w].y;
      df_two_sum(dw[x].z, ib[x].z, h, l);
      df_two_sum(h, -ib[w].z, h2, l2);
      dw[x].z = h2;
      dw[x].w += l + l2 + ib[x].w - ib[w].w;
    }
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    inj[p] = make_float2(-dw[p].x, -dw[p].z);
    injl[p] = make_float2(-dw[p].y, -dw[p].w);
  }
}

// FP32 injection at v = vh + vl rounded to FP32 (rules of bus_injection),
// for the first sweeps of a cold start, where the residual is still far
// above the FP32 rounding of the line currents.
__device__ __forceinline__ float2 load_draw_f32(float2 S, float2 v) {
  if (S.x == 0.f && S.y == 0.f) return make_float2(0.f, 0.f);
  const float inv = __frcp_rn(__fmaf_rn(v.x, v.x, v.y * v.y));
  return make_float2(__fmaf_rn(S.x, v.x, S.y * v.y) * inv, __fmaf_rn(S.x, v.y, -S.y * v.x) * inv);
}

__device__ __forceinline__ void bus_injection_f32(const float2* vh, const float2* vl,
                                                  const float2* sw, const float2* sd, int m,
                                                  float2* inj) {
  float2 d[3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
    d[p] = (p < m && sw) ? load_draw_f32(sw[p], make_float2(vh[p].x + vl[p].x, vh[p].y + vl[p].y))
                         : make_float2(0.f, 0.f);
  if (sd && m == 3) {
    float2 ib[3];   // branches ab, bc, ca
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const int y = x == 2 ? 0 : x + 1;
      const float2 u = make_float2((vh[x].x - vh[y].x) + (vl[x].x - vl[y].x),
                                   (vh[x].y - vh[y].y) + (vl[x].y - vl[y].y));
      ib[x] = load_draw_f32(sd[x], u);
    }
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const int w = x == 0 ? 2 : x - 1;
      d[x].x += ib[x].x - ib[w].x;
      d[x].y += ib[x].y - ib[w].y;
    }
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) inj[p] = make_float2(-d[p].x, -d[p].y);
}

}  // namespace zbus
