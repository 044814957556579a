// Grouped mixed-precision defect sweep (Sec. II-B fixed point in the form
// v <- v + Z_lp r(v)), for one or many feeders at once.
//
// Per sweep, four kernels cover every item of the group:
//   k_residual_group   r(v) over 3x3 bus blocks, one slot per lane, in FP32
//                      for a cold start's first sweeps and in double-float
//                      after them, written as scaled FP16 / BF16 rows of R
//   k_contract_group   persistent tcgen05 contraction D = R Z_emb^T over the
//                      list of (item, 128-slot tile, N-tile) with an active
//                      slot; double-float epilogue v += D and step partials
//   k_decide_group     per-slot stop test (own sweep counter per slot)
//   k_finish_group     list of tiles for the next sweep, loop condition
// (the tree form replaces the last three by k_tree_group).  Slots are
// admitted (k_slot_init) and collected (k_slot_merge + k_branch_f64 +
// k_check, the FP64 power-mismatch test, then the FP64 correction sweeps)
// outside the loop.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "df.cuh"
#include "group.cuh"
#include "loads.cuh"
#include "tc_ptx.cuh"

namespace zbus {
namespace {

using namespace tc;

constexpr int RES_WARPS = 4;
constexpr int CHUNK_BUS = 4;
constexpr int CHUNK_ROWS = 3 * CHUNK_BUS;
constexpr int DEC_THREADS = 256;
constexpr int64_t FUSE_DECIDE = 1024;   // slots up to which the stop test joins the sweep end
// output of the residual: scaled FP16 / BF16 rows of R (tensor-core
// contraction) or FP32 values, scenario-minor (tree sweep)
constexpr int RES_FP16 = 0, RES_BF16 = 1, RES_F32 = 2;
// a cold start's sweeps stay on the FP32 residual while its max |r| exceeds
// this fraction of the largest line or load current (decide_slot).  The FP32
// rounding of the block products, a few 2^-24 of those currents, then stays
// below about 2^-3 of the residual, so an FP32 sweep still removes most of
// it; the double-float sweeps that follow remove the rest.  Measured: at
// 2^-20 the fifth of the eight sweeps of the 1024-bus workload runs on FP32
// with the iteration counts unchanged; at 2^-22 the rounding stalls the
// FP32 sweeps and scenarios need up to two more double-float sweeps.
constexpr float F32_SWITCH = 0x1p-20f;
constexpr int TREE_BATCH = 4;   // buses whose state a tree-sweep warp loads at once
constexpr size_t TREE_ONCHIP_MAX = 200 * 1024;   // shared memory of an on-chip tree block


// Item owning global index x, for a non-decreasing begin field.
__device__ __forceinline__ int find_item(const ItemDesc* items, int n_items, int x, int which) {
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int v = which == 0   ? items[mid].res_begin
                  : which == 1 ? items[mid].dec_begin
                  : which == 2 ? items[mid].mt_begin
                               : items[mid].tree_begin;
    if (v <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Admission: slots [s0, s0 + B) of item k take v^0 (V0 with row stride
// v0_stride, 0 broadcasting one row; else w) and the loads (FP64, [B][n]),
// transposed to the scenario-minor state through 32 x 32 shared-memory tiles.
// Admitted slots become active.  WARM: a start V0 is given (a cold start
// needs no tile for it, which leaves room for more blocks per SM).
// ---------------------------------------------------------------------------
template <bool WARM>
__global__ void k_slot_init(GroupState* __restrict__ gs, const ItemDesc* __restrict__ items, int k,
                            int s0, int B, const double2* __restrict__ V0, int v0_stride,
                            const float4* __restrict__ w_df, const double2* __restrict__ Sw,
                            const double2* __restrict__ Sd, int fp32_start) {
  __shared__ double2 tv[WARM ? 32 : 1][33];
  __shared__ double2 tw[32][33];
  __shared__ double2 td[32][33];
  const ItemDesc it = items[k];
  const int n = it.n, Bp = it.Bp;
  const int j0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    const int b = b0 + r, j = j0 + tx;
    double2 v = make_double2(0.0, 0.0), a = v, d = v;
    if (b < B && j < n) {
      const int64_t g = (int64_t)b * n + j;
      if (WARM) v = V0[(int64_t)b * v0_stride + j];
      if (Sw) a = Sw[g];
      if (Sd) d = Sd[g];
    }
    if (WARM) tv[r][tx] = v;
    tw[r][tx] = a;
    td[r][tx] = d;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, b = b0 + tx;
    if (j < n && b < B) {
      const int64_t g = (int64_t)j * Bp + s0 + b;
      if (WARM) {
        const double2 v = tv[tx][r];
        const float2 xr = df_split(v.x), xi = df_split(v.y);
        it.Vh[g] = make_float2(xr.x, xi.x);
        it.Vl[g] = make_float2(xr.y, xi.y);
      } else {
        // no-load start: the double-float copy of w made at setup
        const float4 wd = w_df[j];
        it.Vh[g] = make_float2(wd.x, wd.z);
        it.Vl[g] = make_float2(wd.y, wd.w);
      }
      it.Swf[g] = make_float2(d2f_rn(tw[tx][r].x), d2f_rn(tw[tx][r].y));
      it.Sdf[g] = make_float2(d2f_rn(td[tx][r].x), d2f_rn(td[tx][r].y));
    }
  }
  if (blockIdx.x == 0 && ty == 0) {
    const int b = b0 + tx;
    const bool adm = b < B;
    if (adm) {
      const int slot = s0 + b;
      it.st[slot] = SLOT_ACTIVE;
      it.it[slot] = 0;
      it.conv[slot] = 0;
      it.amax[slot] = 1.0f;
      it.amax[Bp + slot] = 0.0f;
      it.amax[2 * Bp + slot] = 0.0f;
      it.amax[3 * Bp + slot] = (fp32_start && !WARM) ? 1.0f : 0.0f;
    }
  }
}

// Every slot of every item free, tile flags cleared, loop state zeroed.
__global__ void k_group_reset(GroupState* __restrict__ gs, const ItemDesc* __restrict__ items,
                              int n_items) {
  for (int k = blockIdx.y; k < n_items; k += gridDim.y) {
    const ItemDesc it = items[k];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < it.Bp; b += gridDim.x * blockDim.x) {
      it.st[b] = SLOT_FREE;
    }
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    gs->active = 0;
    gs->sweep = 0;
    gs->err = 0;
    gs->n_tiles = 0;
    gs->tree_done = 0;
    gs->tree_active = 0;
  }
}

__global__ void k_group_params(GroupState* gs, double tol, int max_iter, int rule, int32_t* hist,
                               int hist_n) {
  gs->tol = tol;
  gs->max_iter = max_iter;
  gs->rule = rule;
  gs->hist = hist;
  gs->hist_n = hist_n;
  gs->sweep = 0;
  gs->err = 0;
}

// One block of the FP32 residual: J = Y_ab d (d = v_b - v_a, the slack's
// voltage minus v_a, or v_a itself for the shunt term) with the hi part of
// Y, added to acc, the largest |Re J|, |Im J| kept in mag.
__device__ __forceinline__ void block_f32(const float2* d, const float4* __restrict__ yb,
                                          float2* acc, float& mag) {
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    float jr = 0.f, ji = 0.f;
#pragma unroll
    for (int q2 = 0; q2 < 3; ++q2) {
      const float4 y = yb[p * 3 + q2];
      jr = __fmaf_rn(y.x, d[q2].x, jr);
      jr = __fmaf_rn(-y.z, d[q2].y, jr);
      ji = __fmaf_rn(y.x, d[q2].y, ji);
      ji = __fmaf_rn(y.z, d[q2].x, ji);
    }
    acc[p].x += jr;
    acc[p].y += ji;
    mag = fmaxf(mag, fmaxf(fabsf(jr), fabsf(ji)));
  }
}

// ---------------------------------------------------------------------------
// Defect residual, one slot per lane, double-float, branch form per bus a
// (rows 3a..3a+2):
//   r_a = i_a(v) - [sum_b Y_ab (v_b - v_a) + Y_as (v_s - v_a) + Sh_a v_a]
// The admittance sum (currents up to ~10 pu cancelling to ~1e-10 near the
// solution) runs in double-float with the blocks loaded once per warp for 32
// slots; the load currents in double-float at hi + lo (bus_injection_df), so
// the residual is continuous in v.  R[b][2j],
// R[b][2j+1] = round(c_b Re r_j), round(c_b Im r_j) with c_b = 2^(12 -
// floor(log2 amax_prev_b)) from the previous sweep's max |r| (the residual
// shrinks from sweep to sweep; values beyond the FP16 range saturate, which
// only shortens that step: the next residual is exact again).  Each warp
// covers 4 buses (12 rows) per chunk and writes them through a shared-memory
// transpose; rows n .. K_pad/2 - 1 are written as zeros.
// ---------------------------------------------------------------------------
template <int OUT, int MINB>
__global__ void __launch_bounds__(RES_WARPS * 32, MINB)
k_residual_group(GroupState* __restrict__ gs, const ItemDesc* __restrict__ items) {
  constexpr bool BF = OUT == RES_BF16;
  __shared__ uint32_t stage[RES_WARPS][CHUNK_ROWS][32];
  __shared__ float sred[RES_WARPS][32];
  __shared__ float smag[RES_WARPS][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = find_item(items, gs->n_items, blockIdx.x, 0);
  const ItemDesc& it = items[k];
  const int local = blockIdx.x - it.res_begin;
  const int split = it.res_split;
  const int grp = local / split, ys = local % split;
  const int Bp = it.Bp;
  const int b = grp * 32 + lane;
  const bool act = it.st[b] == SLOT_ACTIVE;
  if (!__syncthreads_or(act)) return;   // all 32 slots of this group are idle
  // FP32 sweep for this slot (its flag, set at a cold start and kept by the
  // stop test while the residual stays above F32_SWITCH of the largest line
  // current); lanes of a warp may differ and then take both paths
  const bool lp = act && it.amax[3 * it.Bp + b] != 0.f;
  float c = 1.f;
  if (OUT != RES_F32) {
    const float ap = it.amax[b];
    int e = (ap > 0.f && ap <= 3.0e38f) ? 12 - ilogbf(ap) : 12;
    e = max(-126, min(126, e));
    c = ldexpf(1.f, e);
    if (ys == 0 && warp == 0) it.rinv[b] = ldexpf(1.f, -e);
  }
  const float2* __restrict__ Vh = it.Vh;
  const float2* __restrict__ Vl = it.Vl;
  const float2* __restrict__ Sw = it.Swf;
  const float2* __restrict__ Sd = it.Sdf;
  const int32_t* __restrict__ bptr = it.bsr_ptr;
  const int32_t* __restrict__ bcol = it.bsr_col;
  const float4* __restrict__ bval = it.bsr_df;
  const int nb = it.nbus;
  const int rows_pad = OUT == RES_F32 ? it.n : it.K_pad >> 1;
  const int nchunks = (rows_pad + CHUNK_ROWS - 1) / CHUNK_ROWS;
  float amax = 0.f, mag = 0.f;
  for (int ch = ys * RES_WARPS + warp; ch < nchunks; ch += split * RES_WARPS) {
    for (int q = 0; q < CHUNK_BUS; ++q) {
      const int a = ch * CHUNK_BUS + q;
      float2 r[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      if (a < nb && act) {
        float2 ah3[3], al3[3], sw[3], sd[3], inj[3], injl[3];   // own state, loads
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const int64_t g = (int64_t)(3 * a + p) * Bp + b;
          ah3[p] = Vh[g];
          al3[p] = Vl[g];
          sw[p] = Sw[g];
          sd[p] = Sd[g];
        }
        if (lp) {
          // FP32: d = v_b - v_a from the hi and lo parts, block products with
          // the hi part of Y, each line's term J = Y_ab d kept for the bound
          bus_injection_f32(ah3, al3, sw, sd, 3, inj);
          // the accumulator starts at -i(v) (ends at -r), so the currents
          // hold no registers in the block loop; the next block's neighbour
          // state is requested before the current block is multiplied
          float2 acc[3];
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            mag = fmaxf(mag, fmaxf(fabsf(inj[p].x), fabsf(inj[p].y)));
            acc[p] = make_float2(-inj[p].x, -inj[p].y);
          }
          const int t1 = bptr[a + 1];
          int t = bptr[a];
          int cb = t < t1 ? bcol[t] : -3;
          float2 xh[3], xl[3];
#pragma unroll
          for (int q2 = 0; q2 < 3; ++q2) xh[q2] = xl[q2] = make_float2(0.f, 0.f);
          if (cb >= 0 && ZB_IN(cb, nb, 0x202u)) {
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) {
              const int64_t g = (int64_t)(3 * cb + q2) * Bp + b;
              xh[q2] = Vh[g];
              xl[q2] = Vl[g];
            }
          }
          for (; t < t1; ++t) {
            const int cn = t + 1 < t1 ? bcol[t + 1] : -3;
            float2 nh[3], nl[3];
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) nh[q2] = nl[q2] = make_float2(0.f, 0.f);
            if (cn >= 0 && ZB_IN(cn, nb, 0x203u)) {
#pragma unroll
              for (int q2 = 0; q2 < 3; ++q2) {
                const int64_t g = (int64_t)(3 * cn + q2) * Bp + b;
                nh[q2] = Vh[g];
                nl[q2] = Vl[g];
              }
            }
            if (cb >= 0 && !ZB_IN(cb, nb, 0x204u)) cb = -3;
            if (cb != -3) {
              float2 d[3];
#pragma unroll
              for (int q2 = 0; q2 < 3; ++q2) {
                if (cb >= 0) {
                  d[q2] = make_float2((xh[q2].x - ah3[q2].x) + (xl[q2].x - al3[q2].x),
                                      (xh[q2].y - ah3[q2].y) + (xl[q2].y - al3[q2].y));
                } else if (cb == -1) {
                  const float4 s4 = it.vs_df[q2];
                  d[q2] = make_float2((s4.x - ah3[q2].x) + (s4.y - al3[q2].x),
                                      (s4.z - ah3[q2].y) + (s4.w - al3[q2].y));
                } else {
                  d[q2] = make_float2(ah3[q2].x + al3[q2].x, ah3[q2].y + al3[q2].y);
                }
              }
              block_f32(d, bval + (int64_t)t * 9, acc, mag);
            }
            cb = cn;
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) {
              xh[q2] = nh[q2];
              xl[q2] = nl[q2];
            }
          }
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            r[p] = make_float2(-acc[p].x, -acc[p].y);
            const float m = fmaxf(fabsf(r[p].x), fabsf(r[p].y));
            amax = (m == m) ? fmaxf(amax, m) : __int_as_float(0x7f800000);
          }
        } else {
        bus_injection_df(ah3, al3, sw, sd, 3, inj, injl);
        // accumulators (re, im) per phase, hi / lo, started at -i(v): the
        // block products are added to them error-free, so they end at -r
        // and the currents need no registers during the block loop
        float ah[3][2], al[3][2];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          ah[p][0] = -inj[p].x;
          al[p][0] = -injl[p].x;
          ah[p][1] = -inj[p].y;
          al[p][1] = -injl[p].y;
        }
        for (int t = bptr[a]; t < bptr[a + 1]; ++t) {
          const int cb = bcol[t];   // the same for the whole warp
          if (cb >= 0 && !ZB_IN(cb, nb, 0x201u)) continue;
          float dh[3][2], dl[3][2];   // vector multiplied by the block, double-float
          if (cb >= 0) {
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) {
              const int64_t g = (int64_t)(3 * cb + q2) * Bp + b;
              const float2 xh = Vh[g], xl = Vl[g];
              df_sub(xh.x, xl.x, ah3[q2].x, al3[q2].x, dh[q2][0], dl[q2][0]);
              df_sub(xh.y, xl.y, ah3[q2].y, al3[q2].y, dh[q2][1], dl[q2][1]);
            }
          } else if (cb == -1) {
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) {
              const float4 s4 = it.vs_df[q2];
              df_sub(s4.x, s4.y, ah3[q2].x, al3[q2].x, dh[q2][0], dl[q2][0]);
              df_sub(s4.z, s4.w, ah3[q2].y, al3[q2].y, dh[q2][1], dl[q2][1]);
            }
          } else {
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) {
              dh[q2][0] = ah3[q2].x; dl[q2][0] = al3[q2].x;
              dh[q2][1] = ah3[q2].y; dl[q2][1] = al3[q2].y;
            }
          }
          const float4* yb = bval + (int64_t)t * 9;
#pragma unroll
          for (int p = 0; p < 3; ++p) {
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) {
              const float4 y = yb[p * 3 + q2];
              df_mac(ah[p][0], al[p][0], y.x, y.y, dh[q2][0], dl[q2][0]);     // + yr dr
              df_mac(ah[p][0], al[p][0], -y.z, -y.w, dh[q2][1], dl[q2][1]);   // - yi di
              df_mac(ah[p][1], al[p][1], y.x, y.y, dh[q2][1], dl[q2][1]);     // + yr di
              df_mac(ah[p][1], al[p][1], y.z, y.w, dh[q2][0], dl[q2][0]);     // + yi dr
            }
          }
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          // r = -(ah + al), one rounding
          r[p] = make_float2(-__fadd_rn(ah[p][0], al[p][0]), -__fadd_rn(ah[p][1], al[p][1]));
          const float m = fmaxf(fabsf(r[p].x), fabsf(r[p].y));
          amax = (m == m) ? fmaxf(amax, m) : __int_as_float(0x7f800000);
        }
        }
      }
      if constexpr (OUT == RES_F32) {
        if (a < nb && act) {
#pragma unroll
          for (int p = 0; p < 3; ++p) it.Rt[(int64_t)(3 * a + p) * Bp + b] = r[p];
        }
      } else {
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          float x = r[p].x * c, y = r[p].y * c;
          uint32_t u;
          if (BF) {
            __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
            u = *reinterpret_cast<uint32_t*>(&h);
          } else {
            x = fminf(fmaxf(x, -65504.f), 65504.f);
            y = fminf(fmaxf(y, -65504.f), 65504.f);
            __half2 h = __floats2half2_rn(x, y);
            u = *reinterpret_cast<uint32_t*>(&h);
          }
          stage[warp][3 * q + p][lane] = u;
        }
      }
    }
    if constexpr (OUT == RES_F32) continue;
    __syncwarp();
    if (act) {
      // CHUNK_ROWS rows = CHUNK_ROWS / 4 16-byte stores into this slot's R row
      uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<uint32_t*>(it.R) +
                                            (int64_t)b * rows_pad + (int64_t)ch * CHUNK_ROWS);
#pragma unroll
      for (int v = 0; v < CHUNK_ROWS / 4; ++v) {
        if (ch * CHUNK_ROWS + 4 * v < rows_pad)
          dst[v] = make_uint4(stage[warp][4 * v][lane], stage[warp][4 * v + 1][lane],
                              stage[warp][4 * v + 2][lane], stage[warp][4 * v + 3][lane]);
      }
    }
    __syncwarp();
  }
  // the tree sweep needs no residual scale, only the FP32-sweep bounds
  if constexpr (OUT == RES_F32) {
    if (!__syncthreads_or(lp)) return;
  }
  sred[warp][lane] = amax;
  smag[warp][lane] = mag == mag ? mag : __int_as_float(0x7f800000);
  __syncthreads();
  if (warp == 0 && act) {
    float m = sred[0][lane], g = smag[0][lane];
    for (int w = 1; w < RES_WARPS; ++w) {
      m = fmaxf(m, sred[w][lane]);
      g = fmaxf(g, smag[w][lane]);
    }
    atomicMax(reinterpret_cast<int*>(&it.amax[Bp + b]), __float_as_int(m));
    if (lp) atomicMax(reinterpret_cast<int*>(&it.amax[2 * Bp + b]), __float_as_int(g));
  }
}

// ---------------------------------------------------------------------------
// tcgen05 contraction, persistent: one CTA per SM walks the tile list (one
// feeder with 8 or more N-tiles: groups of 128-slot tiles, N-tile by N-tile
// within a group, so CTAs running together share a Z panel and the group's
// R rows stay in L2 across the group; otherwise the tiles of one 128-slot
// group are consecutive, N fastest, and CTAs running together share the R
// tile).  Each tile is a 128 x BN block of D = R Z_emb^T
// over K_pad of its item in steps of 64 (128-byte swizzled rows staged by
// TMA).  Two tensor-memory accumulators (2 x BN columns) let the epilogue of
// one tile overlap the MMAs of the next.  Warp roles: 0 = TMA producer,
// 1 = TMEM owner and MMA issuer, 2..5 = epilogue (warp w reads TMEM lanes
// 32 (w % 4) .. + 31).  Barriers: full / empty per stage (TMA -> MMA -> TMA),
// tfull / tempty per accumulator (MMA -> epilogue -> MMA).
//
// L2: every CTA re-reads Z_emb (75 MB at 3069 unknowns) during the launch,
// while the epilogue streams the double-float state (16 B per unknown and
// slot each way); Z's tiles are loaded with an evict-last policy and, where
// the state is larger than L2 keeps between kernels (gs->stream_state), the
// state with an evict-first policy, which favours Z over the state.  A state
// that fits is left to the normal policy: the next residual re-reads it.
//
// Giving up: every pipeline wait is bounded (tc_wait_ns()).  A role whose
// wait runs out records its code in gs->err and stops issuing; then, before
// the CTA frees its tensor memory and exits, the MMA issuer waits for all
// of its committed MMAs (a final tcgen05.commit on the drain barrier) and
// the producer for every TMA load it issued (the last fill of each stage),
// each with its own fixed limit (DRAIN_NS), so nothing lands in tensor or
// shared memory after the CTA is gone.
// ---------------------------------------------------------------------------
constexpr unsigned long long DRAIN_NS = 2000000000ull;

#ifdef ZBUS_CHECKED
// checked build: the pipeline waits' limit can be lowered by
// zbus_checked_set_wait (0: a wait not complete at its first test gives up)
__device__ unsigned long long g_tc_wait_ns = WAIT_NS;
__device__ __forceinline__ unsigned long long tc_wait_ns() { return g_tc_wait_ns; }
#else
__device__ __forceinline__ unsigned long long tc_wait_ns() { return WAIT_NS; }
#endif

template <int BN, int ZP, int STAGES, bool BF>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_contract_group(GroupState* __restrict__ gs, const ItemDesc* __restrict__ items,
                 const CUtensorMap* __restrict__ tmR, const CUtensorMap* __restrict__ tmZ0,
                 const CUtensorMap* __restrict__ tmZ1) {
  constexpr int A_BYTES = BM * BK * 2;
  constexpr int B_BYTES = BN * BK * 2;
  constexpr int STAGE_BYTES = A_BYTES + ZP * B_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_holder = (uint32_t*)(drain + 1);

  const int total = gs->n_tiles;
  if ((int)blockIdx.x >= total) return;   // whole block, before any barrier
  const uint64_t* __restrict__ tiles = gs->tiles;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long wait_ns = tc_wait_ns();

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int u = 0; u < 2; ++u) {
      mbar_init(&tfull[u], 1);
      mbar_init(&tempty[u], 4);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_holder)),
                 "r"((uint32_t)(2 * BN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      const uint64_t zpol = policy_evict_last();
      uint32_t kc = 0;   // stage fills issued
      bool ok = true;
      for (int g = blockIdx.x; g < total && ok; g += gridDim.x) {
        const uint64_t e = tiles[g];
        const int k = (int)(e >> 32), mt = (int)((e >> 16) & 0xFFFF), nt = (int)(e & 0xFFFF);
        const int num_kb = items[k].K_pad / BK;
        const CUtensorMap* mR = tmR + k;
        const CUtensorMap* mZ0 = tmZ0 + k;
        const CUtensorMap* mZ1 = tmZ1 + k;
        for (int kb = 0; kb < num_kb; ++kb) {
          const int s = kc % STAGES;
          const uint32_t round = kc / STAGES;
          if (!mbar_wait(&empty[s], (round & 1) ^ 1, wait_ns)) {
            atomicCAS(&gs->err, 0, 101);
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          tma_load_2d(st, mR, &full[s], kb * BK, mt * BM);
          tma_load_2d_hint(st + A_BYTES, mZ0, &full[s], kb * BK, nt * BN, zpol);
          if (ZP == 2)
            tma_load_2d_hint(st + A_BYTES + B_BYTES, mZ1, &full[s], kb * BK, nt * BN, zpol);
          ++kc;
        }
      }
      // drain: the last fill of every stage has landed (fills complete in
      // order per stage; nothing refills a stage after this point)
      const uint32_t first = kc > (uint32_t)STAGES ? kc - STAGES : 0u;
      for (uint32_t j = first; j < kc; ++j)
        if (!mbar_wait(&full[j % STAGES], (j / STAGES) & 1, DRAIN_NS)) {
          atomicCAS(&gs->err, 0, 105);
          break;
        }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // kind::f16 instruction descriptor: D f32, A/B f16 or bf16, both K-major
      const uint32_t idesc = (1u << 4) | ((BF ? 1u : 0u) << 7) | ((BF ? 1u : 0u) << 10) |
                             ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
      uint32_t kc = 0;
      bool ok = true, issued = false;
      int i = 0;
      for (int g = blockIdx.x; g < total && ok; g += gridDim.x, ++i) {
        const int k = (int)(tiles[g] >> 32);
        const int num_kb = items[k].K_pad / BK;
        const int buf = i & 1;
        const uint32_t use = (uint32_t)(i >> 1);
        if (!mbar_wait(&tempty[buf], (use & 1) ^ 1, wait_ns)) {
          atomicCAS(&gs->err, 0, 104);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * BN);
        for (int kb = 0; kb < num_kb; ++kb, ++kc) {
          const int s = kc % STAGES;
          const uint32_t round = kc / STAGES;
          if (!mbar_wait(&full[s], round & 1, wait_ns)) {
            atomicCAS(&gs->err, 0, 102);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = su32(smem + s * STAGE_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
            for (int p = 0; p < ZP; ++p) {
              const uint32_t b0 = a0 + A_BYTES + p * B_BYTES;
              umma_f16(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                       (kb | kk | p) != 0 ? 1u : 0u);
            }
          }
          issued = true;
          umma_commit(&empty[s]);
        }
        if (ok) umma_commit(&tfull[buf]);
      }
      // drain: every MMA this thread issued has completed before the
      // tensor memory is freed
      if (issued) {
        umma_commit(drain);
        if (!mbar_wait(drain, 0, DRAIN_NS)) atomicCAS(&gs->err, 0, 106);
      }
    }
  } else {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const bool summag = gs->rule == ZBUS_CONV_SUMMAG;
    // evict-first for a state larger than L2 keeps, else the default
    const uint64_t spol = gs->stream_state != 0 ? policy_evict_first() : policy_evict_normal();
    int i = 0;
    for (int g = blockIdx.x; g < total; g += gridDim.x, ++i) {
      const uint64_t e = tiles[g];
      const int k = (int)(e >> 32), mt = (int)((e >> 16) & 0xFFFF), nt = (int)(e & 0xFFFF);
      const ItemDesc& it = items[k];
      const int buf = i & 1;
      const uint32_t use = (uint32_t)(i >> 1);
      const bool ok = mbar_wait(&tfull[buf], use & 1, wait_ns);
      tc_fence_after();
      if (!ok) {
        if (lane == 0) atomicCAS(&gs->err, 0, 103);
        break;
      }
      const int n = it.n, Bp = it.Bp, ntn = it.ntn;
      const int b = mt * BM + row;
      const bool valid = it.st[b] == SLOT_ACTIVE;
      const float rs = valid ? it.rinv[b] : 0.f;
      const float* __restrict__ zinv = it.zinv;
      float2* __restrict__ Vh = it.Vh + b;
      float2* __restrict__ Vl = it.Vl + b;
      float dmax = 0.f, dsum = 0.f;
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        const int i0 = (nt * BN + c * 32) >> 1;
        // the chunk's 16 state entries are requested before any of them is
        // used, so their memory latencies overlap
        float2 h[16], l[16];
        float zs[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int oi = i0 + t;
          const bool in = valid && oi < n;
          const int64_t gi = (int64_t)(in ? oi : 0) * Bp;
          h[t] = in ? ld_f2_hint(Vh + gi, spol) : make_float2(0.f, 0.f);
          l[t] = in ? ld_f2_hint(Vl + gi, spol) : make_float2(0.f, 0.f);
          zs[t] = in ? zinv[oi] : 0.f;
        }
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + c * 32), v);
        if (c == BN / 32 - 1) {
          // the accumulator is in registers now: hand the buffer back
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        if (valid) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int oi = i0 + t;
            if (oi < n) {
              const float sc = rs * zs[t];
              const float dr = v[2 * t] * sc, di = v[2 * t + 1] * sc;
              float sr, er, si, ei;
              two_sum(h[t].x, dr, sr, er);
              two_sum(h[t].y, di, si, ei);
              float2 nh, nl;
              fast_two_sum(sr, __fadd_rn(er, l[t].x), nh.x, nl.x);
              fast_two_sum(si, __fadd_rn(ei, l[t].y), nh.y, nl.y);
              const int64_t gi = (int64_t)oi * Bp;
              st_f2_hint(Vh + gi, nh, spol);
              st_f2_hint(Vl + gi, nl, spol);
              float step = sqrtf(__fmaf_rn(dr, dr, di * di));
              if (step != step) step = __int_as_float(0x7f800000);
              dmax = fmaxf(dmax, step);
              if (summag) {
                // |v + d| - |v| = (2 Re(conj(v) d) + |d|^2) / (|v + d| + |v|)
                const float o2 = __fmaf_rn(h[t].x, h[t].x, h[t].y * h[t].y);
                const float n2 = __fmaf_rn(nh.x, nh.x, nh.y * nh.y);
                dsum += (2.f * (h[t].x * dr + h[t].y * di) + dr * dr + di * di) /
                        (sqrtf(n2) + sqrtf(o2));
              }
            }
          }
        }
      }
      if (valid) {
        it.part[((int64_t)b * ntn + nt) * 2 + 0] = (double)dmax;
        it.part[((int64_t)b * ntn + nt) * 2 + 1] = (double)dsum;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * BN)));
  }
}

// ---------------------------------------------------------------------------
// Stop test, one thread per slot of every item: partials reduced in a fixed
// order; a slot stops when its step meets tol (converged), is not finite or
// reaches max_iter sweeps since its admission.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void decide_slot(const GroupState* __restrict__ gs, const ItemDesc& it,
                                            int b) {
  int keep = 0;
  if (b < it.Bp && it.st[b] == SLOT_ACTIVE) {
    const int sw = it.it[b] + 1;
    it.it[b] = sw;
    const int ntn = it.ntn;
    const double* part = it.part + (int64_t)b * ntn * 2;
    double dmax = 0.0, dsum = 0.0;
    for (int t = 0; t < ntn; ++t) {
      dmax = fmax(dmax, part[2 * t]);
      dsum += part[2 * t + 1];
    }
    const double delta = gs->rule == ZBUS_CONV_SUMMAG ? fabs(dsum) : dmax;
    // a sweep on the FP32 residual never stops a slot
    const bool lp = it.amax[3 * it.Bp + b] != 0.f;
    if (!isfinite(delta)) {
      it.conv[b] = 0;
    } else if (delta <= gs->tol && !lp) {
      it.conv[b] = 1;
    } else if (sw < gs->max_iter) {
      keep = 1;
    }
    if (!keep) it.st[b] = SLOT_DONE;
    const float am = it.amax[it.Bp + b], prev = it.amax[b];
    it.amax[b] = am;
    it.amax[it.Bp + b] = 0.f;
    if (lp) {
      // the next sweep stays on FP32 while max |r| exceeds F32_SWITCH of
      // the largest line current or load current of this one, still falls,
      // and the step is above the stop tolerance; once off, the slot runs
      // double-float to its stop
      const float g = it.amax[2 * it.Bp + b];
      const bool more = keep && am > F32_SWITCH * g && am < prev && delta > gs->tol;
      it.amax[3 * it.Bp + b] = more ? 1.f : 0.f;
      it.amax[2 * it.Bp + b] = 0.f;
    }
  }
}

__global__ void __launch_bounds__(DEC_THREADS)
k_decide_group(GroupState* __restrict__ gs, const ItemDesc* __restrict__ items) {
  const int k = find_item(items, gs->n_items, blockIdx.x, 1);
  const ItemDesc& it = items[k];
  decide_slot(gs, it, (blockIdx.x - it.dec_begin) * DEC_THREADS + threadIdx.x);
}

// ---------------------------------------------------------------------------
// Tree sweep (radial feeders): the step X = T r of a defect sweep, with T the
// inverse of the series admittance of the tree, applied without forming it:
//   backward, deepest level first: S_c = r_c + the sum of the children's S
//     (the current into the subtree of c);
//   forward, from the slack: X_c = X_parent + z_c S_c (z_c the impedance of
//     c's parent branch, X = 0 at the slack);
// in place in the FP32 residual rows (scenario-minor, one slot per lane, so
// every access is a coalesced row segment).  A block's warps split each
// level's buses, TREE_BATCH at a time with all their loads issued before any
// store, and a barrier separates the levels; the position tables (bus,
// parent, children; FP16 z blocks scaled per bus, which set only the
// convergence rate of the defect form, not its fixed point) sit in shared
// memory.  Then v += X in double-float, the step partials per slot reduced
// over the warps, and the stop test of each slot (the rule of
// k_decide_group), so the sweep needs neither a contraction nor a separate
// stop-test launch.
// ---------------------------------------------------------------------------
// End of a tree-sweep block: add its slots still active to the sweep's sum;
// the block that arrives last closes the sweep (the work of k_finish_group
// without a tile list): profile record, active count, sweep counter, the
// graph's loop condition, and the counters reset for the next sweep.
__device__ void tree_block_done(GroupState* gs, int still_active, cudaGraphConditionalHandle h,
                                int use_handle) {
  if (still_active) atomicAdd(&gs->tree_active, still_active);
  __threadfence();
  if (atomicAdd(&gs->tree_done, 1) != (int)gridDim.x - 1) return;
  __threadfence();
  const int total = atomicAdd(&gs->tree_active, 0);
  if (gs->hist && gs->sweep < gs->hist_n) gs->hist[gs->sweep] = gs->active;
  gs->active = total;
  gs->sweep = gs->sweep + 1;
  gs->tree_active = 0;
  gs->tree_done = 0;
  if (use_handle) cudaGraphSetConditional(h, (total > 0 && gs->err == 0) ? 1u : 0u);
}

template <int TREE_WARPS, int MINB, bool ONCHIP>
__global__ void __launch_bounds__(32 * TREE_WARPS, MINB)
k_tree_group(GroupState* __restrict__ gs, const ItemDesc* __restrict__ items,
             cudaGraphConditionalHandle h, int use_handle) {
  extern __shared__ __align__(16) uint8_t tsm[];
  __shared__ float sdmax[TREE_WARPS][32];
  __shared__ float sdsum[TREE_WARPS][32];
  const int k = find_item(items, gs->n_items, blockIdx.x, 3);
  const ItemDesc& it = items[k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = (blockIdx.x - it.tree_begin) * 32 + lane;
  const bool act = it.st[b] == SLOT_ACTIVE;
  if (!__syncthreads_or(act)) {   // the block's 32 slots are idle
    if (threadIdx.x == 0) tree_block_done(gs, 0, h, use_handle);
    return;
  }
  const int Bp = it.Bp, D = it.tlevels, nb = it.nbus;
  int4* node = reinterpret_cast<int4*>(tsm);                 // bus, parent, children
  __half2* zt = reinterpret_cast<__half2*>(node + nb);       // [nb][9]
  float* zst = reinterpret_cast<float*>(zt + 9 * nb);        // [nb]
  uint8_t* pmask = reinterpret_cast<uint8_t*>(zst + nb);     // [nb] phases of the parent line
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    int4 nd = it.t_node[i];
    // checked build: a node out of range becomes a leaf hanging off the slack
    if (!ZB_IN(nd.x, nb, 0x202u) || !ZB_IN(nd.y + 1, nb + 1, 0x203u) ||
        !ZB_IN(nd.z, nb + 1, 0x204u) || !ZB_IN(nd.w, nb + 1, 0x205u) ||
        !ZB_IN(nd.w - nd.z, nb + 1, 0x206u))
      nd = make_int4(0, -1, 0, 0);
    node[i] = nd;
    zst[i] = it.t_zs[i];
    pmask[i] = it.t_mask[i];
  }
  for (int i = threadIdx.x; i < 9 * nb; i += blockDim.x) {
    const float2 z = it.t_z[i];
    zt[i] = __floats2half2_rn(z.x, z.y);
  }
  __syncthreads();
  const int32_t* __restrict__ lvl = it.t_lvl;
  // row j of this slot at R[j * rs]: the residual rows in place in global
  // memory, or (ONCHIP, small feeders) a shared-memory copy of the block's
  // 32 slots, so that the level sweeps never leave the SM
  float2* R;
  int64_t rs;
  if (ONCHIP) {
    float2* rsm = reinterpret_cast<float2*>(tsm + tree_table_bytes(nb));
    const int n = 3 * nb;
    for (int j0 = warp; j0 < n; j0 += TREE_WARPS * TREE_BATCH) {
      float2 v[TREE_BATCH];
#pragma unroll
      for (int u = 0; u < TREE_BATCH; ++u) {
        const int j = j0 + u * TREE_WARPS;
        v[u] = (act && j < n) ? it.Rt[(int64_t)j * Bp + b] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < TREE_BATCH; ++u) {
        const int j = j0 + u * TREE_WARPS;
        if (j < n) rsm[j * 32 + lane] = v[u];
      }
    }
    __syncthreads();
    R = rsm + lane;
    rs = 32;
  } else {
    R = it.Rt + b;
    rs = Bp;
  }
  const int64_t r3 = 3 * rs;
  const int first = warp;   // the warp's first bus of a level
  constexpr int STRIDE = TREE_WARPS;
  for (int L = D - 2; L >= 0; --L) {
    const int l0 = lvl[L], l1 = lvl[L + 1];
    for (int i0 = l0 + first; i0 < l1; i0 += STRIDE * TREE_BATCH) {
      float2 acc[TREE_BATCH][3];
#pragma unroll
      for (int u = 0; u < TREE_BATCH; ++u) {
        const int i = i0 + u * STRIDE;
        if (i < l1 && act) {
          const int4 nd = node[i];
          if (nd.z != nd.w) {
            const float2* own = R + nd.x * r3;
#pragma unroll
            for (int p = 0; p < 3; ++p) acc[u][p] = own[p * rs];
            for (int c = nd.z; c < nd.w; ++c) {
              const float2* ch = R + node[c].x * r3;
              const int cm = pmask[c];   // a phase the child's line lacks stays below
#pragma unroll
              for (int p = 0; p < 3; ++p) {
                const float2 x = ch[p * rs];
                if ((cm >> p) & 1) {
                  acc[u][p].x += x.x;
                  acc[u][p].y += x.y;
                }
              }
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < TREE_BATCH; ++u) {
        const int i = i0 + u * STRIDE;
        if (i < l1 && act) {
          const int4 nd = node[i];
          if (nd.z != nd.w) {
            float2* own = R + nd.x * r3;
#pragma unroll
            for (int p = 0; p < 3; ++p) own[p * rs] = acc[u][p];
          }
        }
      }
    }
    __syncthreads();
  }
  for (int L = 0; L < D; ++L) {
    const int l0 = lvl[L], l1 = lvl[L + 1];
    for (int i0 = l0 + first; i0 < l1; i0 += STRIDE * TREE_BATCH) {
      float2 sv[TREE_BATCH][3], xp[TREE_BATCH][3];
#pragma unroll
      for (int u = 0; u < TREE_BATCH; ++u) {
        const int i = i0 + u * STRIDE;
#pragma unroll
        for (int p = 0; p < 3; ++p) sv[u][p] = xp[u][p] = make_float2(0.f, 0.f);
        if (i < l1 && act) {
          const int4 nd = node[i];
          const float2* own = R + nd.x * r3;
#pragma unroll
          for (int p = 0; p < 3; ++p) sv[u][p] = own[p * rs];
          if (nd.y >= 0) {
            const float2* pa = R + node[nd.y].x * r3;
            const int cm = pmask[i];   // the parent's drop reaches the phases the line carries
#pragma unroll
            for (int p = 0; p < 3; ++p)
              if ((cm >> p) & 1) xp[u][p] = pa[p * rs];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < TREE_BATCH; ++u) {
        const int i = i0 + u * STRIDE;
        if (i < l1 && act) {
          float2* own = R + node[i].x * r3;
          const float sc = zst[i];
          const __half2* z = zt + 9 * i;
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            float ar = 0.f, ai = 0.f;
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) {
              const float2 zz = __half22float2(z[3 * p + q2]);
              ar = __fmaf_rn(zz.x, sv[u][q2].x, __fmaf_rn(-zz.y, sv[u][q2].y, ar));
              ai = __fmaf_rn(zz.x, sv[u][q2].y, __fmaf_rn(zz.y, sv[u][q2].x, ai));
            }
            own[p * rs] = make_float2(__fmaf_rn(ar, sc, xp[u][p].x), __fmaf_rn(ai, sc, xp[u][p].y));
          }
        }
      }
    }
    __syncthreads();
  }
  // v += X (double-float) and the step partials, TREE_BATCH buses per warp
  // requested before any of them is written back
  const bool summag = gs->rule == ZBUS_CONV_SUMMAG;
  float dmax = 0.f, dsum = 0.f;
  if (act) {
    for (int a0 = first; a0 < nb; a0 += STRIDE * TREE_BATCH) {
      float2 xb[TREE_BATCH][3], hb[TREE_BATCH][3], lb[TREE_BATCH][3];
#pragma unroll
      for (int u = 0; u < TREE_BATCH; ++u) {
        const int a = a0 + u * STRIDE;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const int j = 3 * (a < nb ? a : 0) + p;
          const int64_t g = (int64_t)j * Bp + b;
          xb[u][p] = R[j * rs];
          hb[u][p] = it.Vh[g];
          lb[u][p] = it.Vl[g];
        }
      }
#pragma unroll
      for (int u = 0; u < TREE_BATCH; ++u) {
        const int a = a0 + u * STRIDE;
        if (a >= nb) break;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const float2 d = xb[u][p], h = hb[u][p], l = lb[u][p];
          float sr, er, si, ei;
          two_sum(h.x, d.x, sr, er);
          two_sum(h.y, d.y, si, ei);
          float2 nh, nl;
          fast_two_sum(sr, __fadd_rn(er, l.x), nh.x, nl.x);
          fast_two_sum(si, __fadd_rn(ei, l.y), nh.y, nl.y);
          const int64_t g = (int64_t)(3 * a + p) * Bp + b;
          it.Vh[g] = nh;
          it.Vl[g] = nl;
          float step = sqrtf(__fmaf_rn(d.x, d.x, d.y * d.y));
          if (step != step) step = __int_as_float(0x7f800000);
          dmax = fmaxf(dmax, step);
          if (summag) {
            const float o2 = __fmaf_rn(h.x, h.x, h.y * h.y);
            const float n2 = __fmaf_rn(nh.x, nh.x, nh.y * nh.y);
            dsum += (2.f * (h.x * d.x + h.y * d.y) + d.x * d.x + d.y * d.y) /
                    (sqrtf(n2) + sqrtf(o2));
          }
        }
      }
    }
  }
  // per slot, over the warps in order
  sdmax[warp][lane] = dmax;
  sdsum[warp][lane] = dsum;
  __syncthreads();
  if (warp == 0) {
    int keep = 0;
    if (act) {
      float m = 0.f, u = 0.f;
      for (int w = 0; w < TREE_WARPS; ++w) {
        m = fmaxf(m, sdmax[w][lane]);
        u += sdsum[w][lane];
      }
      const int sw = it.it[b] + 1;
      it.it[b] = sw;
      const double delta = summag ? fabs((double)u) : (double)m;
      const bool lp = it.amax[3 * it.Bp + b] != 0.f;   // FP32 residual (rules of decide_slot)
      if (!isfinite(delta)) {
        it.conv[b] = 0;
      } else if (delta <= gs->tol && !lp) {
        it.conv[b] = 1;
      } else if (sw < gs->max_iter) {
        keep = 1;
      }
      if (!keep) it.st[b] = SLOT_DONE;
      if (lp) {
        const float am = it.amax[it.Bp + b], prev = it.amax[b], g = it.amax[2 * it.Bp + b];
        const bool more = keep && am > F32_SWITCH * g && am < prev && delta > gs->tol;
        it.amax[3 * it.Bp + b] = more ? 1.f : 0.f;
        it.amax[b] = am;
        it.amax[it.Bp + b] = 0.f;
        it.amax[2 * it.Bp + b] = 0.f;
      }
    }
    const int still = __popc(__ballot_sync(0xffffffffu, keep));
    if (lane == 0) tree_block_done(gs, still, h, use_handle);
  }
}

// ---------------------------------------------------------------------------
// Sweep end (one block of 1024): the tile list of the next sweep (every
// 128-slot tile holding an active slot, times its item's N-tiles, in a stable
// order), the active count, the sweep counter and the graph's loop
// condition.  initial = 1 only rebuilds the list and the count (after
// admissions), without counting a sweep.  decide = 1 first runs the stop test
// of every slot (k_decide_group's work, for groups of at most FUSE_DECIDE
// slots, where the extra launch costs more than the test).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_finish_group(GroupState* __restrict__ gs, const ItemDesc* __restrict__ items, int initial,
               cudaGraphConditionalHandle h, int use_handle, int decide) {
  __shared__ int swarp[32], sact[32];
  __shared__ int sbase, stotal, sactive;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int mt_total = gs->mt_total, n_items = gs->n_items;
  const int raster = n_items == 1 ? gs->raster : 0;
  uint64_t* tiles = gs->tiles;
  if (decide) {
    // small groups: the stop test of every slot here, saving a launch per sweep
    for (int k = 0; k < n_items; ++k) {
      const ItemDesc& it = items[k];
      for (int b = tid; b < it.Bp; b += blockDim.x) decide_slot(gs, it, b);
    }
    __syncthreads();
  }
  if (tid == 0) {
    sbase = 0;
    sactive = 0;
  }
  __syncthreads();
  for (int base = 0; base < mt_total; base += 1024) {
    const int m = base + tid;
    int cnt = 0, k = 0, lm = 0, na = 0;
    if (m < mt_total) {
      k = find_item(items, n_items, m, 2);
      lm = m - items[k].mt_begin;
      const uint32_t* st4 = reinterpret_cast<const uint32_t*>(items[k].st + lm * 128);
      for (int q = 0; q < 32; ++q) {
        const uint32_t x = st4[q];   // four slot states, SLOT_ACTIVE == 0
#pragma unroll
        for (int y = 0; y < 4; ++y) na += ((x >> (8 * y)) & 0xFFu) == SLOT_ACTIVE;
      }
      if (na) cnt = items[k].ntn;
    }
    int incl = cnt, acc = na;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
      acc += __shfl_xor_sync(0xffffffffu, acc, o);
    }
    if (lane == 31) swarp[wid] = incl;
    if (lane == 0) sact[wid] = acc;
    __syncthreads();
    if (wid == 0) {
      const int x = swarp[lane];
      int inc2 = x;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc2, o);
        if (lane >= o) inc2 += y;
      }
      swarp[lane] = inc2 - x;
      int a2 = sact[lane];
      for (int o = 16; o > 0; o >>= 1) a2 += __shfl_xor_sync(0xffffffffu, a2, o);
      if (lane == 31) stotal = inc2;
      if (lane == 0) sactive += a2;
    }
    __syncthreads();
    const int pos = sbase + swarp[wid] + incl - cnt;
    if (raster == 0)
      for (int t = 0; t < cnt; ++t)
        tiles[pos + t] = ((uint64_t)k << 32) | ((uint64_t)lm << 16) | (uint64_t)t;
    __syncthreads();
    if (tid == 0) sbase += stotal;
    __syncthreads();
  }
  if (raster > 0) {
    // one item: the active 128-slot tiles (rank r among them, in order) in
    // groups of `raster`; within a group, N-tile by N-tile: tile (r, t) of
    // group g = r / raster (size sz) at g raster ntn + t sz + r % raster.
    // Concurrent CTAs then share a group's R rows and a few Z panels in L2.
    const int ntn = items[0].ntn;
    const int n_act = sbase / ntn;
    int rbase = 0;
    for (int base = 0; base < mt_total; base += 1024) {
      const int m = base + tid;
      int act = 0;
      if (m < mt_total) {
        const uint32_t* st4 = reinterpret_cast<const uint32_t*>(items[0].st + m * 128);
        for (int q = 0; q < 32 && !act; ++q) {
          const uint32_t x = st4[q];
#pragma unroll
          for (int y = 0; y < 4; ++y) act |= ((x >> (8 * y)) & 0xFFu) == SLOT_ACTIVE;
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, act);
      if (lane == 0) swarp[wid] = __popc(bal);
      __syncthreads();
      if (wid == 0) {
        const int x = swarp[lane];
        int inc2 = x;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, inc2, o);
          if (lane >= o) inc2 += y;
        }
        swarp[lane] = inc2 - x;
        if (lane == 31) stotal = inc2;
      }
      __syncthreads();
      if (act) {
        const int r = rbase + swarp[wid] + __popc(bal & ((1u << lane) - 1u));
        const int g = r / raster, i = r % raster;
        const int sz = min(raster, n_act - g * raster);
        for (int t = 0; t < ntn; ++t)
          tiles[g * raster * ntn + t * sz + i] = ((uint64_t)m << 16) | (uint64_t)t;
      }
      __syncthreads();
      rbase += stotal;
      __syncthreads();
    }
  }
  if (tid == 0) {
    gs->n_tiles = sbase;
    if (!initial && gs->hist && gs->sweep < gs->hist_n) gs->hist[gs->sweep] = gs->active;
    gs->active = sactive;
    if (!initial) gs->sweep = gs->sweep + 1;
    // a pipeline wait that gave up ends the loop (zbus_last_device_status
    // reports it); the slots still active keep their flags cleared
    if (use_handle) cudaGraphSetConditional(h, (sactive > 0 && gs->err == 0) ? 1u : 0u);
  }
}

// ---------------------------------------------------------------------------
// Collection: slots [s0, s0 + B) of item k merged into the FP64 output
// [B][n], with their sweep counts and flags; the slots become free.  Tiles of
// MERGE_T unknowns x MERGE_T slots: every thread issues its 32 loads (hi and
// lo of 8 unknowns x 2 slots, 256-byte row pieces) before converting any, and
// every output row goes out as 1 KB of consecutive unknowns.
// ---------------------------------------------------------------------------
constexpr int MERGE_T = 64;
constexpr size_t MERGE_SMEM = (size_t)MERGE_T * (MERGE_T + 1) * sizeof(double2);

__global__ void __launch_bounds__(256)
k_slot_merge(const ItemDesc* __restrict__ items, int k, int s0, int B,
             double2* __restrict__ V, int32_t* __restrict__ iters,
             uint8_t* __restrict__ conv, unsigned long long* __restrict__ mmax) {
  extern __shared__ double2 tm[];   // [MERGE_T slots][MERGE_T + 1 unknowns]
  const ItemDesc it = items[k];
  const int n = it.n, Bp = it.Bp;
  const int j0 = blockIdx.x * MERGE_T, b0 = blockIdx.y * MERGE_T;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const float2* __restrict__ Vh = it.Vh;
  const float2* __restrict__ Vl = it.Vl;
  float2 h[8][2], l[8][2];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int j = j0 + ty + 8 * i;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int b = b0 + tx + 32 * c;
      h[i][c] = l[i][c] = make_float2(0.f, 0.f);
      if (j < n && b < B) {
        const int64_t g = (int64_t)j * Bp + s0 + b;
        h[i][c] = Vh[g];
        l[i][c] = Vl[g];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 2; ++c)
      tm[(tx + 32 * c) * (MERGE_T + 1) + ty + 8 * i] =
          make_double2(f2d_exact(h[i][c].x) + f2d_exact(l[i][c].x),
                       f2d_exact(h[i][c].y) + f2d_exact(l[i][c].y));
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = ty + 8 * i, b = b0 + r;
    if (b >= B) continue;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int j = j0 + tx + 32 * c;
      if (j < n) V[(int64_t)b * n + j] = tm[r * (MERGE_T + 1) + tx + 32 * c];
    }
  }
  if (blockIdx.x == 0 && ty < 2) {
    const int b = b0 + tx + 32 * ty;
    if (b < B) {
      iters[b] = it.it[s0 + b];
      conv[b] = it.conv[s0 + b];
      mmax[b] = 0ull;
      it.st[s0 + b] = SLOT_FREE;
    }
  }
}

// 1 / d: a single-precision reciprocal refined by two Newton-Raphson steps
// r <- r (2 - d r) (quadratic convergence, 24 -> 48 -> beyond 53 bits);
// plain division outside [2^-99, 2^100), well inside the single-precision
// range (zero, infinities and NaNs included).  The range test reads the
// exponent field and the conversions to and from float are the integer
// ones, so the FP64 units only do the FMAs.
__device__ __forceinline__ double recip64(double d) {
  const unsigned ex = (unsigned)((unsigned long long)__double_as_longlong(d) >> 52) & 0x7FFu;
  if (ex < 1023u - 99u || ex >= 1023u + 100u) return 1.0 / d;
  double r = f2d_exact(__frcp_rn(d2f_rn(d)));
  r = r * fma(-d, r, 2.0);
  r = r * fma(-d, r, 2.0);
  return r;
}

// conj(S / v), zero for an absent load (both parts +-0, tested on the
// integer units).
__device__ __forceinline__ double2 draw64(double2 S, double2 v) {
  if (((unsigned long long)(__double_as_longlong(S.x) | __double_as_longlong(S.y)) << 1) == 0ull)
    return make_double2(0.0, 0.0);
  const double inv = recip64(fma(v.x, v.x, v.y * v.y));
  return make_double2(fma(S.x, v.x, S.y * v.y) * inv, fma(S.x, v.y, -S.y * v.x) * inv);
}

// FP64 admittance sum of bus a of one scenario (row vg of the [B][n] voltages):
//   acc_p = (Y_LL v + Y_Ls v_s)_{3a+p}
//         = sum_b Y_ab (v_b - v_a) + Y_as (v_s - v_a) + Sh_a v_a   (branch form)
// va = the bus's own voltages.  The 3x3 blocks are the same for every lane of
// a warp working on bus a (broadcast loads).
//
// With branch terms (jg: the scenario's J_k = Y_ab (v_b - v_a) of phase p at
// jg[(3 k + p) js], k_branch_f64) and the block-to-branch map br, a neighbour
// block adds +J_k (block (a, b)) or -J_k (its mirror) instead of forming the
// product.
__device__ __forceinline__ void admittance_sum_f64(const double2* __restrict__ vg, int a, int nb,
                                                   const int32_t* __restrict__ bptr,
                                                   const int32_t* __restrict__ bcol,
                                                   const double2* __restrict__ bval,
                                                   const double2 (&vs)[3], const double2 (&va)[3],
                                                   double (&ar)[3], double (&ai)[3],
                                                   const double2* __restrict__ jg = nullptr,
                                                   const int32_t* __restrict__ br = nullptr,
                                                   int nbr = 0, int64_t js = 0) {
#pragma unroll
  for (int p = 0; p < 3; ++p) ar[p] = ai[p] = 0.0;
  const int t1 = bptr[a + 1];
  for (int t = bptr[a]; t < t1; ++t) {
    const int cb = bcol[t];
    if (cb >= 0 && !ZB_IN(cb, nb, 0x207u)) continue;
    if (jg && cb >= 0) {
      const int k = br[t];
      const int kk = k >= 0 ? k : -k - 1;
      if (!ZB_IN(kk, nbr, 0x20au)) continue;
      const double sg = k >= 0 ? 1.0 : -1.0;
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const double2 x = jg[(3 * kk + p) * js];
        ar[p] = fma(sg, x.x, ar[p]);
        ai[p] = fma(sg, x.y, ai[p]);
      }
      continue;
    }
    double dr[3], di[3];
    if (cb >= 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double2 x = vg[3 * cb + q];
        dr[q] = x.x - va[q].x;
        di[q] = x.y - va[q].y;
      }
    } else if (cb == -1) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        dr[q] = vs[q].x - va[q].x;
        di[q] = vs[q].y - va[q].y;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        dr[q] = va[q].x;
        di[q] = va[q].y;
      }
    }
    const double2* y = bval + (int64_t)t * 9;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double2 yy = y[p * 3 + q];
        ar[p] = fma(yy.x, dr[q], fma(-yy.y, di[q], ar[p]));
        ai[p] = fma(yy.x, di[q], fma(yy.y, dr[q], ai[p]));
      }
  }
}

// FP64 check of one bus of one scenario, in power form: for its unknowns j,
//   dS_j = v_j conj((Y_LL v + Y_Ls v_s)_j) - v_j conj(i_j(v)),  |dS_j| = |v_j| |r_j|
// with the wye term exactly S_j (v conj(conj(S / v)) = S, no division) and the
// delta term v_j conj(drawn) from FP64 branch currents.  Returns the bit
// pattern of the largest |dS_j|^2 of the bus (+inf for a NaN), which orders
// like the value.  sw, sd: the scenario's load rows or null.
__device__ __forceinline__ unsigned long long check_bus_f64(const double2* __restrict__ vg,
                                                const double2* __restrict__ sw,
                                                const double2* __restrict__ sd, int a, int nb,
                                                const int32_t* __restrict__ bptr,
                                                const int32_t* __restrict__ bcol,
                                                const double2* __restrict__ bval,
                                                const double2 (&vs)[3],
                                                const double2* __restrict__ jg = nullptr,
                                                const int32_t* __restrict__ br = nullptr,
                                                int nbr = 0, int64_t js = 0) {
  double2 va[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) va[p] = vg[3 * a + p];
  double ar[3], ai[3];
  admittance_sum_f64(vg, a, nb, bptr, bcol, bval, vs, va, ar, ai, jg, br, nbr, js);
  // dS_p = v_p conj(acc_p) + S_wye_p + v_p conj(drawn_delta_p)
  double sr[3], si[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    sr[p] = fma(va[p].x, ar[p], va[p].y * ai[p]);
    si[p] = fma(va[p].y, ar[p], -va[p].x * ai[p]);
  }
  if (sw) {
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const double2 x = sw[3 * a + p];
      sr[p] += x.x;
      si[p] += x.y;
    }
  }
  if (sd) {
    const double2 s0 = sd[3 * a], s1 = sd[3 * a + 1], s2 = sd[3 * a + 2];
    const bool any = (__double_as_longlong(s0.x) | __double_as_longlong(s0.y) |
                      __double_as_longlong(s1.x) | __double_as_longlong(s1.y) |
                      __double_as_longlong(s2.x) | __double_as_longlong(s2.y)) != 0;
    if (any) {
      double2 ib[3];
      const double2 ss[3] = {s0, s1, s2};
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const int q = (p + 1) % 3;
        ib[p] = draw64(ss[p], make_double2(va[p].x - va[q].x, va[p].y - va[q].y));
      }
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const int m = (p + 2) % 3;   // branch p leaves phase p, branch m returns into it
        const double gx = ib[p].x - ib[m].x, gy = ib[p].y - ib[m].y;
        sr[p] += fma(va[p].x, gx, va[p].y * gy);
        si[p] += fma(va[p].y, gx, -va[p].x * gy);
      }
    }
  }
  // the largest |dS_j|^2 by its bit pattern (non-negative doubles order like
  // their bits; a NaN, whatever its sign bit, counts as +inf), compared on
  // the integer units
  unsigned long long worst = 0ull;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const double e = fma(sr[p], sr[p], si[p] * si[p]);
    unsigned long long eb = (unsigned long long)__double_as_longlong(e) & 0x7FFFFFFFFFFFFFFFull;
    eb = eb > 0x7FF0000000000000ull ? 0x7FF0000000000000ull : eb;
    worst = eb > worst ? eb : worst;
  }
  return worst;
}

// FP64 check of converged scenarios (every bus, check_bus_f64).
//
// Lanes are scenarios and every lane of a warp works on the same bus, so the
// loop over a bus's blocks is uniform and the 3x3 blocks are broadcast loads;
// the FP64 pipe (2 operations per clock per SM) only sees useful work.  Grid
// ceil(B / 32) x ny blocks of (32, CHECK_WARPS), the ny blocks of one group
// of 32 scenarios consecutive, so they run together and share that group's
// rows (its neighbour voltages) in L2; their warps interleave over the
// buses.  Each block folds its max |dS|^2 per scenario into mmax[b]
// (non-negative doubles order like their bit patterns; NaN counts as +inf);
// mmax is zeroed by k_slot_merge.
//
// With branch terms J ([nbr][3][B], k_branch_f64 of the same grid), each
// line's block product is formed once, by k_branch_f64, and both of its
// buses add it (identical mirror blocks, build_branches): about a third
// fewer FP64 operations.
constexpr int CHECK_WARPS = 4;

// Branch terms J_k = Y_ab (v_b - v_a) of every live scenario, FP64, in the
// check's layout (lanes = 32 scenarios, warps over the branches), stored
// scenario-minor, J[(3 k + p) B + b], so both kernels move whole rows.
__global__ void __launch_bounds__(32 * CHECK_WARPS)
k_branch_f64(const double2* __restrict__ V, const uint8_t* __restrict__ conv, int B, int n,
             const int4* __restrict__ tab, int nbr, const double2* __restrict__ bval,
             double2* __restrict__ J, int ny) {
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int bx = blockIdx.x / ny, by = blockIdx.x % ny;
  const int b = bx * 32 + lane;
  const bool live = b < B && conv[b] != 0;
  if (__ballot_sync(0xffffffffu, live) == 0u) return;
  if (!live) return;
  const double2* vg = V + (int64_t)b * n;
  double2* jg = J + b;
  const int nb = n / 3;
  for (int k = by * CHECK_WARPS + ty; k < nbr; k += ny * CHECK_WARPS) {
    const int4 e = tab[k];
    if (!ZB_IN(e.x, nb, 0x20bu) || !ZB_IN(e.y, nb, 0x20cu)) continue;
    double dr[3], di[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double2 xb = vg[3 * e.y + q], xa = vg[3 * e.x + q];
      dr[q] = xb.x - xa.x;
      di[q] = xb.y - xa.y;
    }
    const double2* y = bval + (int64_t)e.z * 9;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      double ar = 0.0, ai = 0.0;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double2 yy = y[p * 3 + q];
        ar = fma(yy.x, dr[q], fma(-yy.y, di[q], ar));
        ai = fma(yy.x, di[q], fma(yy.y, dr[q], ai));
      }
      jg[(int64_t)(3 * k + p) * B] = make_double2(ar, ai);
    }
  }
}

__global__ void __launch_bounds__(32 * CHECK_WARPS)
k_check(const double2* __restrict__ V, const double2* __restrict__ Sw,
        const double2* __restrict__ Sd, const uint8_t* __restrict__ conv, int B, int n,
        const int32_t* __restrict__ bptr, const int32_t* __restrict__ bcol,
        const double2* __restrict__ bval, double2 vs0, double2 vs1, double2 vs2,
        unsigned long long* __restrict__ mmax, int ny, const double2* __restrict__ J,
        const int32_t* __restrict__ br, int nbr) {
  __shared__ unsigned long long red[CHECK_WARPS][32];
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int bx = blockIdx.x / ny, by = blockIdx.x % ny;   // scenario group, bus stride
  const int b = bx * 32 + lane;
  const bool live = b < B && conv[b] != 0;
  if (__ballot_sync(0xffffffffu, live) == 0u) return;   // same for every warp of the block
  const int64_t row = (int64_t)(b < B ? b : B - 1) * n;
  const double2 vs[3] = {vs0, vs1, vs2};
  unsigned long long worst = 0ull;   // max |dS|^2, as its bit pattern
  const int nb = n / 3;
  const double2* jg = J ? J + (b < B ? b : B - 1) : nullptr;
  for (int a = by * CHECK_WARPS + ty; a < nb; a += ny * CHECK_WARPS) {
    const unsigned long long w =
        check_bus_f64(V + row, Sw ? Sw + row : nullptr, Sd ? Sd + row : nullptr, a, nb, bptr,
                      bcol, bval, vs, jg, br, nbr, (int64_t)B);
    worst = w > worst ? w : worst;
  }
  red[ty][lane] = worst;
  __syncthreads();
  if (ty == 0 && live) {
    unsigned long long x = red[0][lane];
#pragma unroll
    for (int w = 1; w < CHECK_WARPS; ++w) x = red[w][lane] > x ? red[w][lane] : x;
    if (x > 0ull) atomicMax(&mmax[b], x);
  }
}

// Outcome per scenario: mm = sqrt(max |dS|^2); a converged flag with mm above
// mtol is cleared; mm_out[b] = mm, or -1 for a scenario that was not checked.
__global__ void k_check_finish(const unsigned long long* mmax, uint8_t* __restrict__ conv, int B,
                               double mtol, double* mm_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  if (conv[b] == 0) {
    if (mm_out) mm_out[b] = -1.0;
    return;
  }
  const double mm = sqrt(__longlong_as_double((long long)mmax[b]));
  if (mm_out) mm_out[b] = mm;
  if (!(mm <= mtol)) conv[b] = 0;
}

// ---------------------------------------------------------------------------
// FP64 correction of the mixed forms: a converged scenario whose FP64
// mismatch exceeds mtol gets up to max_correction FP64 defect sweeps
//   r = i(v) - Y_LL v - Y_Ls v_s   (FP64, branch-form blocks)
//   v <- v + Z r                   (the FP64 3M contraction, exact Z)
// each followed by the FP64 check; it keeps its flag once the check passes,
// and loses it if none of the sweeps brings it below mtol.  Each sweep counts
// as an iteration.  The per-call arguments arrive in the solve context
// (k_corr_setup); the select kernel, a WHILE node over the sweep (residual,
// contraction, check, update) and the end kernel form one graph per network
// and workspace.  With nothing to correct the graph runs two small kernels.
// ---------------------------------------------------------------------------
__global__ void k_corr_setup(SolveCtx* ctx, SolveCtx h) { *ctx = h; }

// One block of 1024 threads: stable compaction of the index range [0, n) by a
// predicate into list; returns the count (valid in every thread).
template <typename Pred>
__device__ int block_compact(int n, int32_t* __restrict__ list, Pred pred, const int32_t* src) {
  __shared__ int swarp[32];
  __shared__ int sbase, stotal;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) sbase = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    const int i = base + tid;
    int keep = 0, v = -1;
    if (i < n) {
      v = src ? src[i] : i;
      keep = pred(v) ? 1 : 0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int wpre = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) swarp[wid] = __popc(bal);
    __syncthreads();
    if (wid == 0) {
      const int x = swarp[lane];
      int incl = x;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      swarp[lane] = incl - x;
      if (lane == 31) stotal = incl;
    }
    __syncthreads();
    // in place (src == list) is safe: every read of this chunk happened
    // before the barriers, every write lands at or before its own index
    if (keep) list[sbase + swarp[wid] + wpre] = v;
    __syncthreads();
    if (tid == 0) sbase += stotal;
    __syncthreads();
  }
  return sbase;
}

// Scenarios to correct: converged by the stop rule, FP64 mismatch above mtol.
// The others get their outcome (mm_out); the selected ones start from a zero
// mismatch record.
__global__ void __launch_bounds__(1024)
k_corr_select(SolveCtx* __restrict__ ctx, cudaGraphConditionalHandle h) {
  const int B = ctx->B;
  const double mtol = ctx->mismatch_tol;
  uint8_t* conv = ctx->conv;
  unsigned long long* mmax = ctx->mmax;
  double* mm_out = ctx->mm_out;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    if (conv[b] == 0) {
      if (mm_out) mm_out[b] = -1.0;
    } else {
      const double mm = sqrt(__longlong_as_double((long long)mmax[b]));
      if (mm_out) mm_out[b] = mm;
    }
  }
  __syncthreads();
  const int cnt = block_compact(B, ctx->list, [&](int b) {
    return conv[b] != 0 && !(sqrt(__longlong_as_double((long long)mmax[b])) <= mtol);
  }, nullptr);
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) mmax[ctx->list[i]] = 0ull;
  if (threadIdx.x == 0) {
    ctx->count = cnt;
    ctx->iter = 0;
    cudaGraphSetConditional(h, (cnt > 0 && ctx->max_iter > 0) ? 1u : 0u);
  }
}

// FP64 residual of every listed scenario, per (slot, bus), into the 3M
// operands [slot][n_pad] (Re, Im, Re + Im; zero in the padding).
__global__ void __launch_bounds__(256)
k_corr_resid(const SolveCtx* __restrict__ ctx, int n, int n_pad, const int32_t* __restrict__ bptr,
             const int32_t* __restrict__ bcol, const double2* __restrict__ bval, double2 vs0,
             double2 vs1, double2 vs2) {
  const int count = ctx->count;
  const int nbp = n_pad / 3, nb = n / 3;
  const int64_t tot = (int64_t)count * nbp;
  const int64_t plane = (int64_t)ctx->B * n_pad;
  double* Ir = ctx->Iop;
  double* Ii = Ir + plane;
  double* Is = Ii + plane;
  const double2 vs[3] = {vs0, vs1, vs2};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int slot = (int)(t / nbp);
    const int a = (int)(t % nbp);
    const int64_t o = (int64_t)slot * n_pad + 3 * a;
    double rr[3] = {0.0, 0.0, 0.0}, ri[3] = {0.0, 0.0, 0.0};
    if (a < nb && ZB_IN(ctx->list[slot], ctx->B, 0x209u)) {
      const int b = ctx->list[slot];
      const int64_t row = (int64_t)b * n;
      const double2* vg = ctx->V + row;
      double2 va[3], sw[3], sd[3], inj[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        va[p] = vg[3 * a + p];
        sw[p] = ctx->S_wye ? ctx->S_wye[row + 3 * a + p] : make_double2(0.0, 0.0);
        sd[p] = ctx->S_del ? ctx->S_del[row + 3 * a + p] : make_double2(0.0, 0.0);
      }
      bus_injection(va, ctx->S_wye ? sw : nullptr, ctx->S_del ? sd : nullptr, 3, inj);
      double ar[3], ai[3];
      admittance_sum_f64(vg, a, nb, bptr, bcol, bval, vs, va, ar, ai);
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        rr[p] = inj[p].x - ar[p];
        ri[p] = inj[p].y - ai[p];
      }
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      Ir[o + p] = rr[p];
      Ii[o + p] = ri[p];
      Is[o + p] = rr[p] + ri[p];
    }
  }
}

// End of a correction sweep (one block of 1024): every listed scenario took
// one more iteration; those whose check passed keep their flag and leave the
// list (stable compaction); the others start the next check from zero.
__global__ void __launch_bounds__(1024)
k_corr_update(SolveCtx* __restrict__ ctx, cudaGraphConditionalHandle h) {
  const int cnt0 = ctx->count;
  const double mtol = ctx->mismatch_tol;
  int32_t* list = ctx->list;
  unsigned long long* mmax = ctx->mmax;
  double* mm_out = ctx->mm_out;
  for (int i = threadIdx.x; i < cnt0; i += blockDim.x) {
    const int b = list[i];
    ctx->iters[b] += 1;
    if (mm_out) mm_out[b] = sqrt(__longlong_as_double((long long)mmax[b]));
  }
  __syncthreads();
  const int cnt = block_compact(cnt0, list, [&](int b) {
    return !(sqrt(__longlong_as_double((long long)mmax[b])) <= mtol);
  }, list);
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) mmax[list[i]] = 0ull;
  if (threadIdx.x == 0) {
    const int it = ctx->iter + 1;
    ctx->iter = it;
    ctx->count = cnt;
    cudaGraphSetConditional(h, (cnt > 0 && it < ctx->max_iter) ? 1u : 0u);
  }
}

// The FP64 check (k_check's layout) of the listed scenarios: lane slot i of
// the grid checks scenario list[i] for i < count.
__global__ void __launch_bounds__(32 * CHECK_WARPS)
k_corr_check(const SolveCtx* __restrict__ ctx, int n, const int32_t* __restrict__ bptr,
             const int32_t* __restrict__ bcol, const double2* __restrict__ bval, double2 vs0,
             double2 vs1, double2 vs2, int ny) {
  __shared__ unsigned long long red[CHECK_WARPS][32];
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int bx = blockIdx.x / ny, by = blockIdx.x % ny;
  const int i = bx * 32 + lane;
  const int B = ctx->B;
  const bool live = i < ctx->count && ZB_IN(ctx->list[i], B, 0x208u);
  if (__ballot_sync(0xffffffffu, live) == 0u) return;
  const int b = live ? ctx->list[i] : 0;
  const int64_t row = (int64_t)b * n;
  const double2 vs[3] = {vs0, vs1, vs2};
  const double2* Sw = ctx->S_wye;
  const double2* Sd = ctx->S_del;
  unsigned long long worst = 0ull;
  const int nb = n / 3;
  for (int a = by * CHECK_WARPS + ty; a < nb; a += ny * CHECK_WARPS) {
    const unsigned long long w = check_bus_f64(ctx->V + row, Sw ? Sw + row : nullptr,
                                               Sd ? Sd + row : nullptr, a, nb, bptr, bcol,
                                               bval, vs);
    worst = w > worst ? w : worst;
  }
  red[ty][lane] = worst;
  __syncthreads();
  if (ty == 0 && live) {
    unsigned long long x = red[0][lane];
#pragma unroll
    for (int w = 1; w < CHECK_WARPS; ++w) x = red[w][lane] > x ? red[w][lane] : x;
    if (x > 0ull) atomicMax(&ctx->mmax[b], x);
  }
}

// Scenarios still above mtol after the correction sweeps lose their flag.
__global__ void k_corr_end(const SolveCtx* __restrict__ ctx) {
  const int cnt = ctx->count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    ctx->conv[ctx->list[i]] = 0;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int BN, int ZP, int STAGES, bool BF>
constexpr size_t tc_smem() {
  return 1024 + (size_t)STAGES * (BM * BK * 2 + ZP * BN * BK * 2) + 256;
}

template <int BN, int ZP, int STAGES, bool BF>
cudaError_t tc_attr() {
  return cudaFuncSetAttribute(k_contract_group<BN, ZP, STAGES, BF>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem<BN, ZP, STAGES, BF>());
}

template <int BN, int ZP, int STAGES, bool BF>
cudaError_t tc_launch(Group* g, int grid, cudaStream_t st) {
  k_contract_group<BN, ZP, STAGES, BF><<<grid, TC_THREADS, tc_smem<BN, ZP, STAGES, BF>(), st>>>(
      g->d_state, g->d_items, g->d_tmR, g->d_tmZ0, g->d_tmZ1);
  return cudaGetLastError();
}

// (precision, BN, stages) variants compiled: FP16 x1 and BF16 x2.
struct TcVariant {
  int32_t precision;
  int BN, stages;
  cudaError_t (*attr)();
  cudaError_t (*launch)(Group*, int, cudaStream_t);
};

const TcVariant kVariants[] = {
    {ZBUS_MIXED_FP16_SCALED, 64, 8, tc_attr<64, 1, 8, false>, tc_launch<64, 1, 8, false>},
    {ZBUS_MIXED_FP16_SCALED, 128, 4, tc_attr<128, 1, 4, false>, tc_launch<128, 1, 4, false>},
    {ZBUS_MIXED_FP16_SCALED, 128, 6, tc_attr<128, 1, 6, false>, tc_launch<128, 1, 6, false>},
    {ZBUS_MIXED_FP16_SCALED, 256, 3, tc_attr<256, 1, 3, false>, tc_launch<256, 1, 3, false>},
    {ZBUS_MIXED_FP16_SCALED, 256, 4, tc_attr<256, 1, 4, false>, tc_launch<256, 1, 4, false>},
    {ZBUS_MIXED_BF16X2, 64, 6, tc_attr<64, 2, 6, true>, tc_launch<64, 2, 6, true>},
    {ZBUS_MIXED_BF16X2, 128, 3, tc_attr<128, 2, 3, true>, tc_launch<128, 2, 3, true>},
    {ZBUS_MIXED_BF16X2, 128, 4, tc_attr<128, 2, 4, true>, tc_launch<128, 2, 4, true>},
    {ZBUS_MIXED_BF16X2, 256, 2, tc_attr<256, 2, 2, true>, tc_launch<256, 2, 2, true>},
};

const TcVariant* find_variant(int32_t precision, int BN, int stages) {
  for (const auto& v : kVariants)
    if (v.precision == precision && v.BN == BN && v.stages == stages) return &v;
  return nullptr;
}

// Built-in choice where the tuning table has no entry, from timed solves of
// every variant: FP16 256 x 4 above 1024 reals per row (128 x 4 below, 64 x 8
// within 1.5 % at 381 unknowns); BF16 128 x 4 at every size measured (3 %
// ahead of 256 x 2 at 3069 unknowns and on the 64-feeder set).
const TcVariant* default_variant(int32_t precision, int max_n) {
  const bool big = 2 * max_n > 1024;
  if (precision == ZBUS_MIXED_BF16X2) return find_variant(precision, 128, 4);
  return find_variant(precision, big ? 256 : 128, 4);
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

bool tc_config_ok(int32_t precision, int BN, int stages) {
  return find_variant(precision, BN, stages) != nullptr;
}

int tc_variants(int32_t precision, int* BN, int* stages, int max) {
  int m = 0;
  for (const auto& v : kVariants)
    if (v.precision == precision && m < max) {
      BN[m] = v.BN;
      stages[m] = v.stages;
      ++m;
    }
  return m;
}

void group_free(Group* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  for (auto e : g->ev) cudaEventDestroy(e);
  cudaFree(g->d_hist);
  cudaFree(g->dmem);
  *g = Group();
}

zbus_status group_build(Group* g, const std::vector<zbus_network>& nets,
                        const std::vector<int64_t>& Bs, int32_t precision, cudaStream_t st,
                        bool lazy_ops) {
  group_free(g);
  g->nets = nets;
  g->Bs = Bs;
  g->precision = precision;
  g->n_items = (int)nets.size();
  const bool tree = precision == ZBUS_TREE_SWEEP;
  int max_n = 0;
  int64_t total_B = 0;
  const int pi = precision == ZBUS_MIXED_BF16X2 ? 1 : 0;
  for (size_t k = 0; k < nets.size(); ++k) {
    // the double-float branch blocks, slack and no-load voltages every item's
    // residual and admission read (also for an item whose Z comes later)
    ZB_CHECK(prepare_df(nets[k], st));
    if (tree) ZB_CHECK(prepare_tree(nets[k], st));
    else if (!lazy_ops || nets[k]->mixed[pi].ready) ZB_CHECK(prepare_mixed(nets[k], precision, st));
    // the FP64 correction sweeps use the FP64 Z (formed again if released)
    if (!lazy_ops) ZB_CHECK(ensure_3m(nets[k], st));
    ZB_CHECK(ensure_workspace(nets[k], Bs[k]));
    max_n = std::max(max_n, nets[k]->n);
    total_B += Bs[k];
  }
  g->tune_gen = tune_generation();
  g->max_n = max_n;
  if (!tree) {
    int BN = 0, stages = 0;
    ZB_CHECK(tune_lookup(precision, max_n, total_B, &BN, &stages));
    const TcVariant* var = find_variant(precision, BN, stages);
    if (!var) var = default_variant(precision, max_n);
    g->BN = var->BN;
    g->stages = var->stages;
    ZB_CUDA(var->attr());
  }
  int dev = 0;
  ZB_CUDA(cudaGetDevice(&dev));
  ZB_CUDA(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, dev));

  g->h_items.resize(nets.size());
  g->ws_gen.resize(nets.size());
  g->op_gen.resize(nets.size());
  int res = 0, dec = 0, mt = 0, tiles = 0, tb = 0;
  g->tree_smem = 0;
  // tree-sweep blocks of 32 slots: 16 warps per block while the blocks are
  // fewer than the SMs can hold, else 8 warps and two blocks per SM
  int64_t tree_slots = 0;
  for (size_t k = 0; k < nets.size(); ++k) tree_slots += nets[k]->ws.cap_Bp;
  g->tree_wide = tree_slots / 32 <= 2 * g->num_sms;
  for (size_t k = 0; k < nets.size(); ++k) {
    zbus_network net = nets[k];
    const MixedOperands& op = net->mixed[precision == ZBUS_MIXED_BF16X2 ? 1 : 0];
    Workspace& ws = net->ws;
    ItemDesc& d = g->h_items[k];
    std::memset(&d, 0, sizeof(d));
    d.bsr_ptr = net->bsr_ptr;
    d.bsr_col = net->bsr_col;
    d.bsr_df = net->bsr_df;
    for (int q = 0; q < 3; ++q) {
      const double2 v = net->v_slack[q];
      const float rh = (float)v.x, ih = (float)v.y;
      d.vs_df[q] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
    }
    d.n = net->n;
    d.nbus = net->nbus;
    d.Bp = (int32_t)ws.cap_Bp;
    if (tree) {
      d.K_pad = round_up(2 * net->n, 64);
      d.N_pad = 0;
      d.ntn = 1;
      d.t_node = net->t_node;
      d.t_z = net->t_z;
      d.t_zs = net->t_zs;
      d.Rt = reinterpret_cast<float2*>(ws.Iop);
      d.t_lvl = net->t_lvl;
      d.t_mask = net->t_mask;
      d.tlevels = net->depth;
      d.tree_begin = tb;
      tb += d.Bp / 32;
      g->tree_smem = std::max(g->tree_smem, tree_table_bytes(net->nbus));
    } else {
      // the operand layout (K_pad, N_pad) also for an item formed later
      d.zinv = op.zinv;
      d.K_pad = round_up(2 * net->n, 64);
      d.N_pad = round_up(2 * net->n, 256);
      d.ntn = d.N_pad / g->BN;
    }
    d.Vh = ws.Vh;
    d.Vl = ws.Vl;
    d.Swf = ws.Swf;
    d.Sdf = ws.Sdf;
    d.st = ws.st;
    d.it = ws.slot_it;
    d.conv = ws.slot_conv;
    d.amax = ws.amax;
    d.R = ws.R;
    d.rinv = ws.rinv;
    d.part = ws.part;
    const int rows_pad = tree ? d.n : d.K_pad / 2;
    const int nchunks = (rows_pad + CHUNK_ROWS - 1) / CHUNK_ROWS;
    d.res_split = (nchunks + RES_WARPS - 1) / RES_WARPS;
    d.res_begin = res;
    res += (d.Bp / 32) * d.res_split;
    d.dec_begin = dec;
    dec += (d.Bp + DEC_THREADS - 1) / DEC_THREADS;
    d.mt_begin = mt;
    mt += d.Bp / 128;
    tiles += (d.Bp / 128) * d.ntn;
    g->ws_gen[k] = ws.gen;
    g->op_gen[k] = net->op_gen;
  }
  g->res_blocks = res;
  g->dec_blocks = dec;
  g->tree_groups = tb;
  if (tree) {
    // the residual rows of a block's 32 slots on chip where they fit
    int max_nb = 0;
    for (size_t k = 0; k < nets.size(); ++k) max_nb = std::max(max_nb, nets[k]->nbus);
    const size_t onchip = tree_table_bytes(max_nb) + (size_t)3 * max_nb * 32 * sizeof(float2);
    g->tree_onchip = onchip <= TREE_ONCHIP_MAX;
    if (g->tree_onchip) g->tree_smem = onchip;
    const int smem = (int)g->tree_smem;
    ZB_CUDA(cudaFuncSetAttribute(k_tree_group<16, 1, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ZB_CUDA(cudaFuncSetAttribute(k_tree_group<16, 1, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ZB_CUDA(cudaFuncSetAttribute(k_tree_group<8, 2, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  }
  ZB_CUDA(cudaFuncSetAttribute(k_slot_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)MERGE_SMEM));
  g->mt_total = mt;
  g->max_tiles = tiles;

  g->total_Bp = 0;
  for (size_t k = 0; k < nets.size(); ++k) g->total_Bp += g->h_items[k].Bp;

  const size_t o_items = 0;
  const size_t o_state = a256(o_items + nets.size() * sizeof(ItemDesc));
  const size_t o_tiles = a256(o_state + sizeof(GroupState));
  const size_t o_maps = a256(o_tiles + (size_t)tiles * sizeof(uint64_t));
  const size_t total = o_maps + 3 * nets.size() * sizeof(CUtensorMap);
  ZB_CUDA(cudaMalloc(&g->dmem, total));
  char* p = (char*)g->dmem;
  g->d_items = (ItemDesc*)(p + o_items);
  g->d_state = (GroupState*)(p + o_state);
  g->d_tiles = (uint64_t*)(p + o_tiles);
  g->d_tmR = (CUtensorMap*)(p + o_maps);
  g->d_tmZ0 = g->d_tmR + nets.size();
  g->d_tmZ1 = g->d_tmZ0 + nets.size();

  std::vector<CUtensorMap> maps(3 * nets.size());
  std::memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
  const bool bf = precision == ZBUS_MIXED_BF16X2;
  for (size_t k = 0; k < nets.size() && !tree; ++k) {
    const MixedOperands& op = nets[k]->mixed[bf ? 1 : 0];
    const ItemDesc& d = g->h_items[k];
    ZB_CHECK(make_tmap_2d(&maps[k], d.R, bf, (uint64_t)d.K_pad, (uint64_t)d.Bp, BK, BM));
    if (!op.ready) continue;   // lazy: encoded by group_refresh_item
    ZB_CHECK(make_tmap_2d(&maps[nets.size() + k], op.Z0, bf, (uint64_t)op.K_pad,
                          (uint64_t)op.N_pad, BK, g->BN));
    ZB_CHECK(make_tmap_2d(&maps[2 * nets.size() + k], bf ? op.Z1 : op.Z0, bf, (uint64_t)op.K_pad,
                          (uint64_t)op.N_pad, BK, g->BN));
  }
  GroupState s;
  std::memset(&s, 0, sizeof(s));
  s.n_items = g->n_items;
  s.mt_total = mt;
  s.res_blocks = res;
  s.dec_blocks = dec;
  s.tree_groups = tb;
  s.tiles = g->d_tiles;
  if (!tree && nets.size() == 1) {
    // tile groups whose R rows (128 x K_pad 16-bit values per 128-slot tile)
    // take about a quarter of L2 (all tiles in one group below twice that),
    // when the feeder has enough N-tiles for the grouping to matter.  At
    // 3069 unknowns (K_pad = 6144, 24 N-tiles of 256) the contraction went
    // from 1394-1431 to 1469-1480 TFLOP/s at 16384 scenarios (groups of 20)
    // and from 1147 to 1219 at 4096 (one group of 32); groups sized to L2/2
    // or L2/8, R loaded evict-last instead of Z, or Z loaded with the
    // normal or evict-first policy, were slower.
    int l2 = 0;
    ZB_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    const ItemDesc& d = g->h_items[0];
    const size_t rtile = (size_t)BM * d.K_pad * 2;
    const int gm = (int)std::max<size_t>(1, (size_t)l2 / 4 / rtile);
    if (d.ntn >= 8) s.raster = mt >= 2 * gm ? gm : mt;
  }
  {
    // double-float state of every slot (hi and lo, 16 B per unknown): streamed
    // when it is more than a third of L2
    size_t state = 0;
    for (size_t k = 0; k < nets.size(); ++k)
      state += (size_t)g->h_items[k].Bp * (size_t)g->h_items[k].n * 16;
    int l2 = 0;
    ZB_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    s.stream_state = state > (size_t)l2 / 3 ? 1 : 0;
  }
  ZB_CUDA(cudaMemcpyAsync(g->d_items, g->h_items.data(), nets.size() * sizeof(ItemDesc),
                          cudaMemcpyHostToDevice, st));
  ZB_CUDA(cudaMemcpyAsync(g->d_state, &s, sizeof(s), cudaMemcpyHostToDevice, st));
  ZB_CUDA(cudaMemcpyAsync(g->d_tmR, maps.data(), maps.size() * sizeof(CUtensorMap),
                          cudaMemcpyHostToDevice, st));
  ZB_CUDA(cudaStreamSynchronize(st));
  return ZBUS_OK;
}

zbus_status group_refresh_item(Group* g, int k, cudaStream_t st) {
  zbus_network net = g->nets[k];
  ItemDesc& d = g->h_items[k];
  g->op_gen[k] = net->op_gen;
  if (!net->bsr_df || d.bsr_df != net->bsr_df || !net->w_df)
    return fail(ZBUS_ERR_DEVICE, "group item without its double-float blocks");
  if (g->precision == ZBUS_TREE_SWEEP) return ZBUS_OK;
  const bool bf = g->precision == ZBUS_MIXED_BF16X2;
  const MixedOperands& op = net->mixed[bf ? 1 : 0];
  if (!op.ready || !op.zinv || !op.Z0 || (bf && !op.Z1))
    return fail(ZBUS_ERR_DEVICE, "group item refreshed without its operands");
  if (op.K_pad != d.K_pad || op.N_pad != d.N_pad)
    return fail(ZBUS_ERR_DEVICE, "group item operand layout differs");
  d.zinv = op.zinv;
  CUtensorMap m[2];
  ZB_CHECK(make_tmap_2d(&m[0], op.Z0, bf, (uint64_t)op.K_pad, (uint64_t)op.N_pad, BK, g->BN));
  ZB_CHECK(make_tmap_2d(&m[1], bf ? op.Z1 : op.Z0, bf, (uint64_t)op.K_pad, (uint64_t)op.N_pad, BK,
                        g->BN));
  ZB_CUDA(cudaMemcpyAsync(g->d_items + k, &d, sizeof(ItemDesc), cudaMemcpyHostToDevice, st));
  ZB_CUDA(cudaMemcpyAsync(g->d_tmZ0 + k, &m[0], sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
  ZB_CUDA(cudaMemcpyAsync(g->d_tmZ1 + k, &m[1], sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
  ZB_CUDA(cudaStreamSynchronize(st));
  return ZBUS_OK;
}

zbus_status group_reset(Group* g, cudaStream_t st) {
  k_group_reset<<<dim3(16, std::min(g->n_items, 64)), 256, 0, st>>>(g->d_state, g->d_items,
                                                                  g->n_items);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

zbus_status group_admit(Group* g, int k, int64_t s0, int64_t B, const double* V0,
                        const double* S_wye, const double* S_delta, cudaStream_t st,
                        bool v0_broadcast, bool fp32_start) {
  if (B <= 0) return ZBUS_OK;
  const ItemDesc& d = g->h_items[k];
  const dim3 grid((d.n + 31) / 32, (unsigned)((B + 31) / 32)), block(32, 8);
  if (V0)
    k_slot_init<true><<<grid, block, 0, st>>>(
        g->d_state, g->d_items, k, (int)s0, (int)B, (const double2*)V0, v0_broadcast ? 0 : d.n,
        g->nets[k]->w_df, (const double2*)S_wye, (const double2*)S_delta, fp32_start ? 1 : 0);
  else
    k_slot_init<false><<<grid, block, 0, st>>>(
        g->d_state, g->d_items, k, (int)s0, (int)B, nullptr, 0, g->nets[k]->w_df,
        (const double2*)S_wye, (const double2*)S_delta, fp32_start ? 1 : 0);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

zbus_status group_start(Group* g, double tol, int32_t max_iter, int32_t rule, int32_t* hist,
                        int32_t hist_n, cudaStream_t st) {
  k_group_params<<<1, 1, 0, st>>>(g->d_state, tol, max_iter, rule, hist, hist_n);
  return group_rebuild(g, st);
}

zbus_status group_rebuild(Group* g, cudaStream_t st) {
  k_finish_group<<<1, 1024, 0, st>>>(g->d_state, g->d_items, 1, 0, 0, 0);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

namespace {

// Residual of every slot on stream st.  Register budget: 4 blocks per SM at
// small n (latency), 6 or 8 at large n (FP32 issue), measured on both
// workloads.
void launch_residual(Group* g, cudaStream_t st) {
  const bool bf = g->precision == ZBUS_MIXED_BF16X2;
  const bool tree = g->precision == ZBUS_TREE_SWEEP;
#define ZB_RES(OUT, M)                                                                     \
  k_residual_group<OUT, M><<<g->res_blocks, RES_WARPS * 32, 0, st>>>(g->d_state, g->d_items)
  const int out = tree ? RES_F32 : (bf ? RES_BF16 : RES_FP16);
  if (g->max_n > 1024) {
    // the tree sweep's FP32 rows: 8 blocks (64 registers) beat 6 and 7
    // (17.50 / 17.90 / 17.54 ms per 1024-bus x 16384 step); the FP16 rows,
    // with six of the eight sweeps on the FP32 path: 7 blocks (17.14 ms)
    // against 6 (17.25) and 8 (17.42); the BF16 rows: 7 (24.09) against 6
    // (24.22)
    if (out == RES_F32) ZB_RES(RES_F32, 8);
    else if (out == RES_BF16) ZB_RES(RES_BF16, 7);
    else ZB_RES(RES_FP16, 7);
  } else {
    if (out == RES_F32) ZB_RES(RES_F32, 4);
    else if (out == RES_BF16) ZB_RES(RES_BF16, 4);
    else ZB_RES(RES_FP16, 4);
  }
#undef ZB_RES
}

}  // namespace

zbus_status group_sweep(Group* g, cudaGraphConditionalHandle h, bool use_handle, cudaStream_t st,
                        cudaEvent_t* ev) {
  const bool tree = g->precision == ZBUS_TREE_SWEEP;
  if (ev) ZB_CUDA(cudaEventRecord(ev[0], st));
  launch_residual(g, st);
  if (ev) ZB_CUDA(cudaEventRecord(ev[1], st));
  if (tree) {
    // step, update, stop test and the end of the sweep in one launch
    const int uh = use_handle ? 1 : 0;
    if (g->tree_onchip)
      k_tree_group<16, 1, true><<<g->tree_groups, 512, g->tree_smem, st>>>(g->d_state,
                                                                             g->d_items, h, uh);
    else if (g->tree_wide)
      k_tree_group<16, 1, false><<<g->tree_groups, 512, g->tree_smem, st>>>(g->d_state,
                                                                              g->d_items, h, uh);
    else
      k_tree_group<8, 2, false><<<g->tree_groups, 256, g->tree_smem, st>>>(g->d_state,
                                                                             g->d_items, h, uh);
    if (ev) ZB_CUDA(cudaEventRecord(ev[2], st));
  } else {
    const TcVariant* var = find_variant(g->precision, g->BN, g->stages);
    ZB_CUDA(var->launch(g, std::min(g->num_sms, g->max_tiles), st));
    if (ev) ZB_CUDA(cudaEventRecord(ev[2], st));
    const bool fuse = g->total_Bp <= FUSE_DECIDE;
    if (!fuse) k_decide_group<<<g->dec_blocks, DEC_THREADS, 0, st>>>(g->d_state, g->d_items);
    k_finish_group<<<1, 1024, 0, st>>>(g->d_state, g->d_items, 0, h, use_handle ? 1 : 0,
                                       fuse ? 1 : 0);
  }
  if (ev) ZB_CUDA(cudaEventRecord(ev[3], st));
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

zbus_status group_run(Group* g, cudaStream_t st) {
  if (!g->exec) {
    if (!g->cap_stream) ZB_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    ZB_CUDA(cudaGraphCreate(&g->graph, 0));
    cudaGraphConditionalHandle h;
    ZB_CUDA(cudaGraphConditionalHandleCreate(&h, g->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    ZB_CUDA(cudaGraphAddNode(&node, g->graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ZB_CUDA(cudaStreamBeginCaptureToGraph(g->cap_stream, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    zbus_status s = group_sweep(g, h, true, g->cap_stream);
    cudaGraph_t captured = nullptr;
    cudaError_t ce = cudaStreamEndCapture(g->cap_stream, &captured);
    if (s != ZBUS_OK) return s;
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture(group sweep)", __FILE__, __LINE__);
    ce = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate(group loop)", __FILE__, __LINE__);
  }
  ZB_CUDA(cudaGraphLaunch(g->exec, st));
  return ZBUS_OK;
}

const int32_t* group_error_word(const Group* g) { return &g->d_state->err; }

zbus_status group_device_status(Group* g, cudaStream_t st) {
  if (!g || !g->d_state) return ZBUS_OK;
  int32_t err = 0;
  ZB_CUDA(cudaMemcpyAsync(&err, group_error_word(g), sizeof(err), cudaMemcpyDeviceToHost, st));
  ZB_CUDA(cudaStreamSynchronize(st));
  if (err == 0) return ZBUS_OK;
  if (err >= 101 && err <= 106)
    return fail(ZBUS_ERR_TIMEOUT, "a bounded wait of the tensor-core pipeline gave up (code " +
                                      std::to_string(err) + ")");
  return fail(ZBUS_ERR_DEVICE, "device error word " + std::to_string(err));
}

namespace {

// Grid of k_check over B scenarios (32 per group, ny blocks per group).
void check_grid(int64_t B, int n, int num_sms, int* gx, int* ny) {
  *gx = (int)((B + 31) / 32);
  const int nb = n / 3;
  *ny = std::max(1, std::min((nb + CHECK_WARPS - 1) / CHECK_WARPS, (8 * num_sms + *gx - 1) / *gx));
}

// The correction graph of a network for its current workspace: select, then
// WHILE (residual, contraction, check, update), then end.  Every per-call
// argument is read from the workspace's solve context.
zbus_status corr_graph(zbus_network net, int num_sms) {
  if (net->corr_exec && net->corr_gen == net->ws.gen) return ZBUS_OK;
  if (net->corr_exec) cudaGraphExecDestroy(net->corr_exec);
  if (net->corr_graph) cudaGraphDestroy(net->corr_graph);
  net->corr_exec = nullptr;
  net->corr_graph = nullptr;
  if (!net->cap_stream) ZB_CUDA(cudaStreamCreateWithFlags(&net->cap_stream, cudaStreamNonBlocking));
  cudaStream_t cs = net->cap_stream;
  SolveCtx* ctx = net->ws.ctx;
  const int64_t cap = net->ws.cap_B;
  const int n = net->n, n_pad = net->n_pad;
  cudaGraph_t graph = nullptr;
  ZB_CUDA(cudaGraphCreate(&graph, 0));
  net->corr_graph = graph;
  cudaGraphConditionalHandle h;
  ZB_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault));
  cudaGraph_t out = nullptr;
  ZB_CUDA(cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  k_corr_select<<<1, 1024, 0, cs>>>(ctx, h);
  cudaError_t ce = cudaStreamEndCapture(cs, &out);
  if (ce != cudaSuccess) return cuda_fail(ce, "capture (correction select)", __FILE__, __LINE__);
  cudaGraphNode_t sel = nullptr;
  size_t num = 1;
  ZB_CUDA(cudaGraphGetNodes(graph, &sel, &num));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cond = nullptr;
  ZB_CUDA(cudaGraphAddNode(&cond, graph, &sel, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  ZB_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  {
    const int64_t tot = cap * (n_pad / 3);
    const int grid = (int)std::min<int64_t>(152 * 16, std::max<int64_t>(1, (tot + 255) / 256));
    k_corr_resid<<<grid, 256, 0, cs>>>(ctx, n, n_pad, net->bsr_ptr, net->bsr_col, net->bsr_val,
                                       net->v_slack[0], net->v_slack[1], net->v_slack[2]);
    launch_gemm_f64(ctx, net->Zr, net->Zi, net->Zs, nullptr, n, n_pad,
                    gemm_f64_grid((int)cap, n_pad), cs);
    int gx = 0, ny = 0;
    check_grid(cap, n, num_sms, &gx, &ny);
    k_corr_check<<<(unsigned)((int64_t)gx * ny), dim3(32, CHECK_WARPS), 0, cs>>>(
        ctx, n, net->bsr_ptr, net->bsr_col, net->bsr_val, net->v_slack[0], net->v_slack[1],
        net->v_slack[2], ny);
    k_corr_update<<<1, 1024, 0, cs>>>(ctx, h);
  }
  ce = cudaStreamEndCapture(cs, &out);
  if (ce != cudaSuccess) return cuda_fail(ce, "capture (correction sweep)", __FILE__, __LINE__);
  ZB_CUDA(cudaStreamBeginCaptureToGraph(cs, graph, &cond, nullptr, 1,
                                        cudaStreamCaptureModeThreadLocal));
  k_corr_end<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (cap + 255) / 256)), 256, 0,
               cs>>>(ctx);
  ce = cudaStreamEndCapture(cs, &out);
  if (ce != cudaSuccess) return cuda_fail(ce, "capture (correction end)", __FILE__, __LINE__);
  ce = cudaGraphInstantiate(&net->corr_exec, graph, 0);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate(correction)", __FILE__, __LINE__);
  net->corr_gen = net->ws.gen;
  return ZBUS_OK;
}

}  // namespace

zbus_status group_collect(Group* g, int k, int64_t s0, int64_t B, double* V_out, int32_t* iters,
                          uint8_t* converged, const double* S_wye, const double* S_delta,
                          double mtol, double* mm_out, int32_t max_corr, cudaStream_t st) {
  if (B <= 0) return ZBUS_OK;
  zbus_network net = g->nets[k];
  if (!net->ws.mm || B > net->ws.cap_B) return fail(ZBUS_ERR_ARG, "collect: batch above workspace");
  unsigned long long* mmax = reinterpret_cast<unsigned long long*>(net->ws.mm);
  k_slot_merge<<<dim3((net->n + MERGE_T - 1) / MERGE_T, (unsigned)((B + MERGE_T - 1) / MERGE_T)),
                 dim3(32, 8), MERGE_SMEM, st>>>(
      g->d_items, k, (int)s0, (int)B, (double2*)V_out, iters, converged, mmax);
  int gx = 0, ny = 0;
  check_grid(B, net->n, g->num_sms, &gx, &ny);
  // branch terms once per line, in the FP64 scratch (free between sweeps)
  double2* J = nullptr;
  if (net->nbr > 0 && (size_t)B * net->nbr * 3 * sizeof(double2) <= net->ws.iop_bytes) {
    J = reinterpret_cast<double2*>(net->ws.Iop);
    k_branch_f64<<<(unsigned)((int64_t)gx * ny), dim3(32, CHECK_WARPS), 0, st>>>(
        (const double2*)V_out, converged, (int)B, net->n, net->br_tab, net->nbr, net->bsr_val, J,
        ny);
  }
  k_check<<<(unsigned)((int64_t)gx * ny), dim3(32, CHECK_WARPS), 0, st>>>(
      (const double2*)V_out, (const double2*)S_wye, (const double2*)S_delta, converged, (int)B,
      net->n, net->bsr_ptr, net->bsr_col, net->bsr_val, net->v_slack[0], net->v_slack[1],
      net->v_slack[2], mmax, ny, J, net->bsr_br, net->nbr);
  if (max_corr <= 0) {
    k_check_finish<<<(unsigned)((B + 255) / 256), 256, 0, st>>>(mmax, converged, (int)B, mtol,
                                                                 mm_out);
    ZB_CUDA(cudaGetLastError());
    return ZBUS_OK;
  }
  SolveCtx h;
  std::memset(&h, 0, sizeof(h));
  h.S_wye = (const double2*)S_wye;
  h.S_del = (const double2*)S_delta;
  h.V = (double2*)V_out;
  h.iters = iters;
  h.conv = converged;
  h.list = net->ws.list;
  h.keep = net->ws.keep;
  h.part = net->ws.part;
  h.Iop = net->ws.Iop;
  h.mismatch_tol = mtol;
  h.B = (int32_t)B;
  h.max_iter = max_corr;
  h.ntn = net->n_pad / F64_BN;
  h.mmax = mmax;
  h.mm_out = mm_out;
  ZB_CHECK(corr_graph(net, g->num_sms));
  k_corr_setup<<<1, 1, 0, st>>>(net->ws.ctx, h);
  ZB_CUDA(cudaGetLastError());
  ZB_CUDA(cudaGraphLaunch(net->corr_exec, st));
  return ZBUS_OK;
}

}  // namespace zbus

namespace zbus {
ZB_CHECK_WORD_ACCESSOR(check_word_group)
}  // namespace zbus

extern "C" zbus_status zbus_checked_set_wait(uint64_t wait_ns) {
#ifdef ZBUS_CHECKED
  zbus::set_error("");
  cudaError_t e = cudaMemcpyToSymbol(zbus::g_tc_wait_ns, &wait_ns, sizeof(wait_ns));
  if (e != cudaSuccess)
    return zbus::cuda_fail(e, "cudaMemcpyToSymbol(wait limit)", __FILE__, __LINE__);
  return ZBUS_OK;
#else
  (void)wait_ns;
  return zbus::fail(ZBUS_ERR_UNSUPPORTED, "the wait limit is settable in the checked build only");
#endif
}
