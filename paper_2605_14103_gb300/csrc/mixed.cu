// Mixed-precision defect sweep of the Z-bus fixed point (Sec. II-B).
//
// With Z Y_LL = I, the map v <- Z i(v) + w equals v <- v + Z r(v) with the
// residual r(v) = i(v) - Y_LL v - Y_Ls v_s.  The residual is formed from the
// sparse admittance matrix in double-float arithmetic (FP32 hi + lo pairs,
// ~48 bits; the FP32 pipes are ~64x faster than FP64 here), so the fixed
// point is that of the full-precision map; the dense product Z r runs on the
// tcgen05 tensor cores with Z in FP16 (rows scaled by powers of two) or BF16
// hi+lo, r rounded per scenario with a power-of-two scale, FP32 accumulation
// in tensor memory, and a double-float epilogue v <- v + D.  A low-precision
// Z only changes the rate of convergence.  v lives as a double-float pair
// during the sweeps and is merged into the FP64 output at the end, where an
// FP64 power-mismatch test confirms every converged scenario.
//
//   k_pack_tc         Z (complex FP64) -> real 2x2 embedding operand(s)
//   k_init_df         v^0 and the loads -> scenario-minor double-float state
//   k_residual_df     r(v), one scenario per lane -> low-precision R rows
//   k_contract_tc     D = R Z_emb^T on tcgen05, epilogue v += D, step partials
//   k_merge_df        double-float state -> FP64 output
//   k_final_check     FP64 power mismatch of converged scenarios
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "df.cuh"
#include "loads.cuh"
#include "mixed.cuh"

namespace zbus {
namespace {

// ---------------------------------------------------------------------------
// Operand packing.  Row 2i of the embedding gives Re D_i, row 2i+1 Im D_i;
// column 2j multiplies Re r_j, column 2j+1 Im r_j:
//   row 2i   : [ Zr_ij, -Zi_ij ]      row 2i+1 : [ Zi_ij, Zr_ij ]
// Both rows of output i share the scale s_i = 2^(12 - floor(log2 max|Z_i.|)),
// which maps the row's largest entry into [4096, 8192).  zinv[i] = 1 / s_i.
// One block per complex output i.
// ---------------------------------------------------------------------------
template <bool BF>
__global__ void k_pack_tc(const double2* __restrict__ Z, int n, int K_pad, int N_pad,
                          void* out0, void* out1, float* zinv) {
  __shared__ double sm[32];
  const int i = blockIdx.x;
  if (i >= N_pad / 2) return;
  double mx = 0.0;
  if (i < n)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double2 z = Z[(int64_t)i * n + j];
      mx = fmax(mx, fmax(fabs(z.x), fabs(z.y)));
    }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (threadIdx.x == 0) sm[0] = x;
  }
  __syncthreads();
  mx = sm[0];
  const int e = (mx > 0.0) ? 12 - ilogb(mx) : 0;
  const double s = ldexp(1.0, e);
  if (threadIdx.x == 0 && i < n) zinv[i] = (float)ldexp(1.0, -e);
  for (int k = threadIdx.x; k < K_pad; k += blockDim.x) {
    const int j = k >> 1;
    double a = 0.0, b = 0.0;   // row 2i, row 2i+1 entries at column k
    if (i < n && j < n) {
      const double2 z = Z[(int64_t)i * n + j];
      if ((k & 1) == 0) { a = z.x; b = z.y; } else { a = -z.y; b = z.x; }
      a *= s;
      b *= s;
    }
    const int64_t o0 = (int64_t)(2 * i) * K_pad + k, o1 = o0 + K_pad;
    if (BF) {
      __nv_bfloat16* h = (__nv_bfloat16*)out0;
      __nv_bfloat16* l = (__nv_bfloat16*)out1;
      const __nv_bfloat16 ha = __double2bfloat16(a), hb = __double2bfloat16(b);
      h[o0] = ha;
      h[o1] = hb;
      l[o0] = __double2bfloat16(a - (double)__bfloat162float(ha));
      l[o1] = __double2bfloat16(b - (double)__bfloat162float(hb));
    } else {
      __half* h = (__half*)out0;
      h[o0] = __double2half(a);
      h[o1] = __double2half(b);
    }
  }
}

// ---------------------------------------------------------------------------
// Run start of the mixed sweeps: v^0 (already written to the FP64 output by
// the common run start) and the loads, scenario-major [B][n] FP64, become the
// scenario-minor [n][B_pad] double-float state and FP32 loads (32 x 32 tiles
// through shared memory).  Padding scenarios (b >= B) are zero and stopped.
// ---------------------------------------------------------------------------
__global__ void k_init_df(SolveCtx* __restrict__ ctx, int n, int B, int Bp) {
  __shared__ double2 tv[32][33];
  __shared__ double2 tw[32][33];
  __shared__ double2 td[32][33];
  const int j0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const bool hw = ctx->Swf != nullptr, hd = ctx->Sdf != nullptr;
  for (int r = ty; r < 32; r += 8) {
    const int b = b0 + r, j = j0 + tx;
    double2 v = make_double2(0.0, 0.0), w = v, d = v;
    if (b < B && j < n) {
      const int64_t g = (int64_t)b * n + j;
      v = ctx->V[g];
      if (hw) w = ctx->S_wye[g];
      if (hd) d = ctx->S_del[g];
    }
    tv[r][tx] = v;
    tw[r][tx] = w;
    td[r][tx] = d;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, b = b0 + tx;
    if (j < n && b < Bp) {
      const int64_t g = (int64_t)j * Bp + b;
      const double2 v = tv[tx][r];
      const float2 xr = df_split(v.x), xi = df_split(v.y);
      ctx->Vh[g] = make_float2(xr.x, xi.x);
      ctx->Vl[g] = make_float2(xr.y, xi.y);
      if (hw) ctx->Swf[g] = make_float2(__double2float_rn(tw[tx][r].x), __double2float_rn(tw[tx][r].y));
      if (hd) ctx->Sdf[g] = make_float2(__double2float_rn(td[tx][r].x), __double2float_rn(td[tx][r].y));
    }
  }
  if (blockIdx.x == 0) {
    for (int t = ty * 32 + tx; t < 32; t += 256) {
      const int b = b0 + t;
      if (b < Bp) {
        ctx->st[b] = b < B ? 0 : 1;
        ctx->amax_prev[b] = 1.0f;
        ctx->amax_cur[b] = 0.0f;
      }
    }
  }
  if (blockIdx.x == 0 && tx == 0 && ty == 0 && (b0 % 128) == 0) {
    ctx->mt_list[b0 / 128] = b0 / 128;
    ctx->mt_flag[b0 / 128] = 0;
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && tx == 0 && ty == 0) {
    ctx->count_next = 0;
    ctx->mt_count = Bp / 128;
  }
}

// The double-float state merged back into the FP64 output [B][n].
__global__ void k_merge_df(SolveCtx* __restrict__ ctx, int n, int B, int Bp) {
  __shared__ double2 t[32][33];
  const int j0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, b = b0 + tx;
    double2 v = make_double2(0.0, 0.0);
    if (j < n && b < Bp) {
      const int64_t g = (int64_t)j * Bp + b;
      const float2 h = ctx->Vh[g], l = ctx->Vl[g];
      v = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
    }
    t[tx][r] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int b = b0 + r, j = j0 + tx;
    if (b < B && j < n) ctx->V[(int64_t)b * n + j] = t[r][tx];
  }
}

// Double-float copies of complex FP64 values (admittance blocks, Y_Ls v_s).
__global__ void k_split_c(const double2* __restrict__ val, int64_t m, float4* out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double2 y = val[t];
    const float2 a = df_split(y.x), b = df_split(y.y);
    out[t] = make_float4(a.x, a.y, b.x, b.y);
  }
}

// ---------------------------------------------------------------------------
// Defect residual, one scenario per lane, double-float:
//   r_j = i_j(v) - sum_b Y_LL[a][b] v_b - ys_j        (bus a holds rows 3a..3a+2)
// The admittance sum (terms ~1e3 cancelling to ~1e-10 near the solution) runs
// in double-float over the 3x3 bus blocks, loaded once per warp for 32
// scenarios; the load current (~1e-2, no cancellation) in FP32 from the hi
// part.  R[b][2j], R[b][2j+1] = round(c_b Re r_j), round(c_b Im r_j), with
// c_b = 2^(12 - floor(log2 amax_prev_b)) from the previous sweep's max |r|
// (the residual shrinks from sweep to sweep; values beyond the FP16 range
// saturate, which only shortens that step: the next residual is exact again).
// Each warp covers 4 buses (12 rows) per chunk and writes them through a
// shared-memory transpose; rows n .. K_pad/2 - 1 are written as zeros.
// ---------------------------------------------------------------------------
constexpr int RES_WARPS = 4;
constexpr int CHUNK_BUS = 4;
constexpr int CHUNK_ROWS = 3 * CHUNK_BUS;

template <bool BF>
__global__ void __launch_bounds__(RES_WARPS * 32)
k_residual_df(SolveCtx* __restrict__ ctx, const int32_t* __restrict__ bptr,
              const int32_t* __restrict__ bcol, const float4* __restrict__ bval,
              const float4* __restrict__ ys4, int nb, int K_pad, void* Rout,
              float* __restrict__ rinv) {
  __shared__ uint32_t stage[RES_WARPS][CHUNK_ROWS][32];
  __shared__ float sred[RES_WARPS][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Bp = ctx->B_pad;
  const int b = blockIdx.x * 32 + lane;
  const bool act = ctx->st[b] == 0;
  if (!__syncthreads_or(act)) return;   // the whole group of 32 has stopped
  const float ap = ctx->amax_prev[b];
  int e = (ap > 0.f && ap <= 3.0e38f) ? 12 - ilogbf(ap) : 12;
  e = max(-126, min(126, e));
  const float c = ldexpf(1.f, e);
  if (blockIdx.y == 0 && warp == 0) rinv[b] = ldexpf(1.f, -e);
  const float2* __restrict__ Vh = ctx->Vh;
  const float2* __restrict__ Vl = ctx->Vl;
  const float2* __restrict__ Sw = ctx->Swf;
  const float2* __restrict__ Sd = ctx->Sdf;
  const int rows_pad = K_pad >> 1;
  const int nchunks = (rows_pad + CHUNK_ROWS - 1) / CHUNK_ROWS;
  float amax = 0.f;
  for (int ch = blockIdx.y * RES_WARPS + warp; ch < nchunks; ch += gridDim.y * RES_WARPS) {
    for (int q = 0; q < CHUNK_BUS; ++q) {
      const int a = ch * CHUNK_BUS + q;
      float2 r[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      if (a < nb && act) {
        float2 vv[3], sw[3], sd[3], inj[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const int64_t g = (int64_t)(3 * a + p) * Bp + b;
          vv[p] = Vh[g];
          sw[p] = Sw ? Sw[g] : make_float2(0.f, 0.f);
          sd[p] = Sd ? Sd[g] : make_float2(0.f, 0.f);
        }
        bus_injection_f(vv, Sw ? sw : nullptr, Sd ? sd : nullptr, 3, inj);
        float ah[3][2], al[3][2];   // accumulators (re, im) per phase, hi / lo
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const float4 y0 = ys4[3 * a + p];
          ah[p][0] = y0.x; al[p][0] = y0.y; ah[p][1] = y0.z; al[p][1] = y0.w;
        }
        for (int t = bptr[a]; t < bptr[a + 1]; ++t) {
          const int cb = bcol[t];
          float2 xh[3], xl[3];
#pragma unroll
          for (int q2 = 0; q2 < 3; ++q2) {
            const int64_t g = (int64_t)(3 * cb + q2) * Bp + b;
            xh[q2] = Vh[g];
            xl[q2] = Vl[g];
          }
          const float4* yb = bval + (int64_t)t * 9;
#pragma unroll
          for (int p = 0; p < 3; ++p) {
#pragma unroll
            for (int q2 = 0; q2 < 3; ++q2) {
              const float4 y = yb[p * 3 + q2];
              df_mac(ah[p][0], al[p][0], y.x, y.y, xh[q2].x, xl[q2].x);     // + yr vr
              df_mac(ah[p][0], al[p][0], -y.z, -y.w, xh[q2].y, xl[q2].y);   // - yi vi
              df_mac(ah[p][1], al[p][1], y.x, y.y, xh[q2].y, xl[q2].y);     // + yr vi
              df_mac(ah[p][1], al[p][1], y.z, y.w, xh[q2].x, xl[q2].x);     // + yi vr
            }
          }
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          r[p] = make_float2(__fsub_rn(__fsub_rn(inj[p].x, ah[p][0]), al[p][0]),
                             __fsub_rn(__fsub_rn(inj[p].y, ah[p][1]), al[p][1]));
          const float m = fmaxf(fabsf(r[p].x), fabsf(r[p].y));
          amax = (m == m) ? fmaxf(amax, m) : __int_as_float(0x7f800000);
        }
      }
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
    __syncwarp();
    if (act) {
      // CHUNK_ROWS rows = CHUNK_ROWS / 4 16-byte stores into this scenario's R row
      uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<uint32_t*>(Rout) +
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
  sred[warp][lane] = amax;
  __syncthreads();
  if (warp == 0 && act) {
    float m = sred[0][lane];
    for (int w = 1; w < RES_WARPS; ++w) m = fmaxf(m, sred[w][lane]);
    atomicMax(reinterpret_cast<int*>(&ctx->amax_cur[b]), __float_as_int(m));
  }
}

// ---------------------------------------------------------------------------
// Stop test of the mixed sweeps, one thread per scenario (stopped ones are
// skipped): partials reduced in a fixed order, iters / flags recorded, the
// residual scale carried to the next sweep, active scenarios counted.
// ---------------------------------------------------------------------------
__global__ void k_decide_mixed(SolveCtx* __restrict__ ctx, int B) {
  __shared__ int scount;
  if (threadIdx.x == 0) scount = 0;
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  int keep = 0;
  if (b < B && ctx->st[b] == 0) {
    const int it = ctx->iter + 1;
    const int ntn = ctx->ntn;
    const double* part = ctx->part + (int64_t)b * ntn * 2;
    double dmax = 0.0, dsum = 0.0;
    for (int t = 0; t < ntn; ++t) {
      dmax = fmax(dmax, part[2 * t]);
      dsum += part[2 * t + 1];
    }
    const double delta = ctx->rule == ZBUS_CONV_SUMMAG ? fabs(dsum) : dmax;
    ctx->iters[b] = it;
    if (!isfinite(delta)) {
      ctx->conv[b] = 0;
    } else if (delta <= ctx->tol) {
      ctx->conv[b] = 1;
    } else if (it < ctx->max_iter) {
      keep = 1;
    }
    if (!keep) ctx->st[b] = 1;
    else atomicOr(&ctx->mt_flag[b / 128], 1u);
    ctx->amax_prev[b] = ctx->amax_cur[b];
    ctx->amax_cur[b] = 0.f;
  }
  const unsigned bal = __ballot_sync(0xffffffffu, keep);
  if ((threadIdx.x & 31) == 0 && bal) atomicAdd(&scount, __popc(bal));
  __syncthreads();
  if (threadIdx.x == 0 && scount) atomicAdd(&ctx->count_next, scount);
}

// Sweep end (one block of 1024): publish the active count, rebuild the list
// of 128-scenario tiles that still hold an active scenario (stable order),
// advance the sweep counter, set the loop condition of the graph.
__global__ void __launch_bounds__(1024) k_finish_mixed(SolveCtx* ctx, int mtiles,
                                                       cudaGraphConditionalHandle h,
                                                       int use_handle) {
  __shared__ int swarp[32];
  __shared__ int sbase, stotal;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) sbase = 0;
  __syncthreads();
  for (int base = 0; base < mtiles; base += 1024) {
    const int m = base + tid;
    int keep = 0;
    if (m < mtiles) {
      keep = ctx->mt_flag[m] != 0;
      ctx->mt_flag[m] = 0;
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
    if (keep) ctx->mt_list[sbase + swarp[wid] + wpre] = m;
    __syncthreads();
    if (tid == 0) sbase += stotal;
    __syncthreads();
  }
  if (tid == 0) {
    const int it = ctx->iter + 1;
    if (ctx->hist && it - 1 < ctx->hist_n) ctx->hist[it - 1] = ctx->count;
    const int c = ctx->count_next;
    ctx->count = c;
    ctx->count_next = 0;
    ctx->mt_count = sbase;
    ctx->iter = it;
    if (use_handle) cudaGraphSetConditional(h, c > 0 ? 1u : 0u);
  }
}

// ---------------------------------------------------------------------------
// tcgen05 contraction.  One CTA computes a BM x BN tile of D = R Z_emb^T
// (rows: active scenario slots, columns: real outputs) over K_pad in steps
// of BK = 64 (128-byte swizzled rows), then adds the scaled accumulator to v.
// Warp roles: 0 = TMA producer, 1 = TMEM owner and MMA issuer, 2..5 = epilogue
// (warp w reads TMEM lanes 32 (w % 4) .. + 31).
// ---------------------------------------------------------------------------
constexpr int BM = 128;
constexpr int BK = 64;
constexpr int TC_THREADS = 192;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // any single wait gives up after 2 s

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on a barrier phase: false after WAIT_NS without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_try(bar, parity))
    if (gtimer() - t0 > WAIT_NS) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}
// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused with swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Persistent form: one CTA per SM walks the list of active 128-scenario tiles
// times the N-tiles (N fastest, so CTAs running together share the R tile in
// L2).  Two tensor-memory accumulators (2 x BN columns) let the epilogue of
// one tile overlap the MMAs of the next.  Barriers: full / empty per smem
// stage (TMA -> MMA -> TMA), tfull / tempty per accumulator (MMA -> epilogue
// -> MMA).
template <int BN, int ZP, int STAGES, bool BF>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_contract_tc(SolveCtx* __restrict__ ctx, const __grid_constant__ CUtensorMap tmR,
              const __grid_constant__ CUtensorMap tmZ0, const __grid_constant__ CUtensorMap tmZ1,
              const float* __restrict__ zinv, const float* __restrict__ rinv, int n, int K_pad,
              int N_pad) {
  constexpr int A_BYTES = BM * BK * 2;
  constexpr int B_BYTES = BN * BK * 2;
  constexpr int STAGE_BYTES = A_BYTES + ZP * B_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_holder = (uint32_t*)(tempty + 2);

  const int Bp = ctx->B_pad;
  const int ntn = N_pad / BN;
  const int total = ctx->mt_count * ntn;
  if ((int)blockIdx.x >= total) return;   // whole block, before any barrier
  const int* __restrict__ mt_list = ctx->mt_list;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_kb = K_pad / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int u = 0; u < 2; ++u) {
      mbar_init(&tfull[u], 1);
      mbar_init(&tempty[u], 4);
    }
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
      uint32_t kc = 0;
      bool ok = true;
      for (int g = blockIdx.x; g < total && ok; g += gridDim.x) {
        const int mt = mt_list[g / ntn], nt = g % ntn;
        for (int kb = 0; kb < num_kb; ++kb, ++kc) {
          const int s = kc % STAGES;
          const uint32_t round = kc / STAGES;
          if (!mbar_wait(&empty[s], (round & 1) ^ 1)) {
            atomicCAS(&ctx->err, 0, 101);
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          tma_load_2d(st, &tmR, &full[s], kb * BK, mt * BM);
          tma_load_2d(st + A_BYTES, &tmZ0, &full[s], kb * BK, nt * BN);
          if (ZP == 2) tma_load_2d(st + A_BYTES + B_BYTES, &tmZ1, &full[s], kb * BK, nt * BN);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // kind::f16 instruction descriptor: D f32, A/B f16 or bf16, both K-major
      const uint32_t idesc = (1u << 4) | ((BF ? 1u : 0u) << 7) | ((BF ? 1u : 0u) << 10) |
                             ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
      uint32_t kc = 0;
      bool ok = true;
      int i = 0;
      for (int g = blockIdx.x; g < total && ok; g += gridDim.x, ++i) {
        const int buf = i & 1;
        const uint32_t use = (uint32_t)(i >> 1);
        if (!mbar_wait(&tempty[buf], (use & 1) ^ 1)) {
          atomicCAS(&ctx->err, 0, 104);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * BN);
        for (int kb = 0; kb < num_kb; ++kb, ++kc) {
          const int s = kc % STAGES;
          const uint32_t round = kc / STAGES;
          if (!mbar_wait(&full[s], round & 1)) {
            atomicCAS(&ctx->err, 0, 102);
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
          umma_commit(&empty[s]);
        }
        if (ok) umma_commit(&tfull[buf]);
      }
    }
  } else {
    // epilogue warps 2..5; warp w reads TMEM lanes 32 (w % 4) .. + 31
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const bool summag = ctx->rule == ZBUS_CONV_SUMMAG;
    int i = 0;
    for (int g = blockIdx.x; g < total; g += gridDim.x, ++i) {
      const int mt = mt_list[g / ntn], nt = g % ntn;
      const int buf = i & 1;
      const uint32_t use = (uint32_t)(i >> 1);
      const bool ok = mbar_wait(&tfull[buf], use & 1);
      tc_fence_after();
      if (!ok) {
        if (lane == 0) atomicCAS(&ctx->err, 0, 103);
        break;
      }
      const int b = mt * BM + row;
      const bool valid = b < Bp && ctx->st[b] == 0;
      const float rs = valid ? rinv[b] : 0.f;
      float2* Vh = ctx->Vh + b;
      float2* Vl = ctx->Vl + b;
      float dmax = 0.f, dsum = 0.f;
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + c * 32), v);
        if (c == BN / 32 - 1) {
          // the accumulator is in registers now: hand the buffer back
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        if (valid) {
          const int i0 = (nt * BN + c * 32) >> 1;
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int oi = i0 + t;
            if (oi < n) {
              const float sc = rs * zinv[oi];
              const float dr = v[2 * t] * sc, di = v[2 * t + 1] * sc;
              const int64_t gi = (int64_t)oi * Bp;
              const float2 h = Vh[gi], l = Vl[gi];
              float sr, er, si, ei;
              two_sum(h.x, dr, sr, er);
              two_sum(h.y, di, si, ei);
              float2 nh, nl;
              fast_two_sum(sr, __fadd_rn(er, l.x), nh.x, nl.x);
              fast_two_sum(si, __fadd_rn(ei, l.y), nh.y, nl.y);
              Vh[gi] = nh;
              Vl[gi] = nl;
              float step = sqrtf(__fmaf_rn(dr, dr, di * di));
              if (step != step) step = __int_as_float(0x7f800000);
              dmax = fmaxf(dmax, step);
              if (summag) {
                // |v + d| - |v| = (2 Re(conj(v) d) + |d|^2) / (|v + d| + |v|)
                const float o2 = __fmaf_rn(h.x, h.x, h.y * h.y);
                const float n2 = __fmaf_rn(nh.x, nh.x, nh.y * nh.y);
                dsum += (2.f * (h.x * dr + h.y * di) + dr * dr + di * di) /
                        (sqrtf(n2) + sqrtf(o2));
              }
            }
          }
        }
      }
      if (valid) {
        ctx->part[((int64_t)b * ntn + nt) * 2 + 0] = (double)dmax;
        ctx->part[((int64_t)b * ntn + nt) * 2 + 1] = (double)dsum;
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
// FP64 check of converged scenarios: the power mismatch
//   max_j |v_j| |(Y_LL v + ys)_j - i_j(v)|
// with the sparse admittance matrix; a converged scenario above mtol loses
// its flag.  One block per scenario, v staged in shared memory (16 n bytes).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_final_check(SolveCtx* __restrict__ ctx, const int32_t* __restrict__ ptr,
              const int32_t* __restrict__ col, const double2* __restrict__ val,
              const double2* __restrict__ ys, int n, double* mm_out) {
  extern __shared__ double2 vsm[];
  __shared__ double red[32];
  const int b = blockIdx.x;
  if (b >= ctx->B) return;
  if (ctx->conv[b] == 0) {
    if (threadIdx.x == 0 && mm_out) mm_out[b] = -1.0;
    return;
  }
  const double2* vg = ctx->V + (int64_t)b * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) vsm[j] = vg[j];
  __syncthreads();
  const double2* Sw = ctx->S_wye ? ctx->S_wye + (int64_t)b * n : nullptr;
  const double2* Sd = ctx->S_del ? ctx->S_del + (int64_t)b * n : nullptr;
  double worst = 0.0;   // max |v|^2 |r|^2
  const int nb = (n + 2) / 3;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    const int j0 = 3 * k;
    const int m = min(3, n - j0);
    double2 vv[3], sw[3], sd[3], inj[3];
    for (int p = 0; p < 3; ++p) {
      vv[p] = p < m ? vsm[j0 + p] : make_double2(1.0, 0.0);
      sw[p] = (Sw && p < m) ? Sw[j0 + p] : make_double2(0.0, 0.0);
      sd[p] = (Sd && p < m) ? Sd[j0 + p] : make_double2(0.0, 0.0);
    }
    bus_injection(vv, Sw ? sw : nullptr, Sd ? sd : nullptr, m, inj);
    for (int p = 0; p < m; ++p) {
      const int j = j0 + p;
      double2 acc = ys[j];
      for (int t = ptr[j]; t < ptr[j + 1]; ++t) {
        const double2 y = val[t], x = vsm[col[t]];
        acc.x = fma(y.x, x.x, fma(-y.y, x.y, acc.x));
        acc.y = fma(y.x, x.y, fma(y.y, x.x, acc.y));
      }
      const double rx = acc.x - inj[p].x, ry = acc.y - inj[p].y;
      double e = (vv[p].x * vv[p].x + vv[p].y * vv[p].y) * (rx * rx + ry * ry);
      if (e != e) e = INFINITY;
      worst = fmax(worst, e);
    }
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x = fmax(x, red[w]);
    const double mm = sqrt(x);
    if (mm_out) mm_out[b] = mm;
    if (!(mm <= ctx->mismatch_tol)) ctx->conv[b] = 0;
  }
}

template <int BN, int ZP, int STAGES, bool BF>
constexpr size_t tc_smem_bytes() {
  return 1024 + (size_t)STAGES * (BM * BK * 2 + ZP * BN * BK * 2) + 256;   // + barriers
}

template <int BN, int ZP, int STAGES, bool BF>
cudaError_t launch_tc_impl(SolveCtx* ctx, const MixedOperands& op, const CUtensorMap& tmR,
                           const float* rinv, int n, int grid, cudaStream_t st) {
  constexpr size_t smem = tc_smem_bytes<BN, ZP, STAGES, BF>();
  auto kern = k_contract_tc<BN, ZP, STAGES, BF>;
  kern<<<grid, TC_THREADS, smem, st>>>(ctx, tmR, op.tmZ0, op.tmZ1, op.zinv, rinv, n, op.K_pad,
                                       op.N_pad);
  return cudaGetLastError();
}

template <int BN, int ZP, int STAGES, bool BF>
cudaError_t set_tc_attr() {
  return cudaFuncSetAttribute(k_contract_tc<BN, ZP, STAGES, BF>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes<BN, ZP, STAGES, BF>());
}

// Opt the kernels of this file into large dynamic shared memory on the
// current device (outside any stream capture).
cudaError_t set_attributes() {
  cudaError_t e;
  if ((e = set_tc_attr<256, 2, 2, true>()) != cudaSuccess) return e;
  if ((e = set_tc_attr<128, 2, 3, true>()) != cudaSuccess) return e;
  if ((e = set_tc_attr<256, 1, 4, false>()) != cudaSuccess) return e;
  if ((e = set_tc_attr<128, 1, 4, false>()) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_final_check, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              220 * 1024);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

}  // namespace

zbus_status make_tmap_2d(CUtensorMap* map, const void* base, bool bf16, uint64_t cols,
                         uint64_t rows, uint32_t box_cols, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return fail(ZBUS_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                  const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(ZBUS_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return ZBUS_OK;
}

zbus_status prepare_mixed(zbus_network net, int32_t precision, cudaStream_t st) {
  MixedOperands& op = net->mixed[precision == ZBUS_MIXED_BF16X2 ? 1 : 0];
  if (op.ready) return ZBUS_OK;
  if (!net->bus_aligned)
    return fail(ZBUS_ERR_UNSUPPORTED, "mixed modes need three unknowns per bus (n % 3 == 0)");
  if ((size_t)16 * net->n > 220 * 1024)
    return fail(ZBUS_ERR_UNSUPPORTED, "mixed modes support n <= 14080 unknowns");
  ZB_CUDA(set_attributes());
  if (!net->bsr_df) {
    const int64_t m = std::max<int64_t>(1, net->nblk * 9);
    ZB_CUDA(cudaMalloc((void**)&net->bsr_df, m * sizeof(float4)));
    ZB_CUDA(cudaMalloc((void**)&net->ys_df, (size_t)net->n * sizeof(float4)));
    if (net->nblk > 0)
      k_split_c<<<(int)std::min<int64_t>(2048, (net->nblk * 9 + 255) / 256), 256, 0, st>>>(
          net->bsr_val, net->nblk * 9, net->bsr_df);
    k_split_c<<<(net->n + 255) / 256, 256, 0, st>>>(net->ys, net->n, net->ys_df);
    ZB_CUDA(cudaGetLastError());
  }
  const bool bf = precision == ZBUS_MIXED_BF16X2;
  op.bf16 = bf;
  op.zparts = bf ? 2 : 1;
  op.K_pad = round_up(2 * net->n, BK);
  op.N_pad = round_up(2 * net->n, 256);
  op.BN = (2 * net->n > 1024) ? 256 : 128;
  {
    int dev = 0;
    ZB_CUDA(cudaGetDevice(&dev));
    ZB_CUDA(cudaDeviceGetAttribute(&op.num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const size_t bytes = (size_t)op.N_pad * op.K_pad * 2;
  ZB_CUDA(cudaMalloc(&op.Z0, bytes));
  if (bf) ZB_CUDA(cudaMalloc(&op.Z1, bytes));
  ZB_CUDA(cudaMalloc((void**)&op.zinv, (size_t)op.N_pad / 2 * sizeof(float)));
  if (bf)
    k_pack_tc<true><<<op.N_pad / 2, 256, 0, st>>>(net->Z, net->n, op.K_pad, op.N_pad, op.Z0, op.Z1,
                                                  op.zinv);
  else
    k_pack_tc<false><<<op.N_pad / 2, 256, 0, st>>>(net->Z, net->n, op.K_pad, op.N_pad, op.Z0,
                                                   nullptr, op.zinv);
  ZB_CUDA(cudaGetLastError());
  ZB_CHECK(make_tmap_2d(&op.tmZ0, op.Z0, bf, op.K_pad, op.N_pad, BK, op.BN));
  ZB_CHECK(make_tmap_2d(&op.tmZ1, bf ? op.Z1 : op.Z0, bf, op.K_pad, op.N_pad, BK, op.BN));
  ZB_CUDA(cudaStreamSynchronize(st));
  op.ready = true;
  return ZBUS_OK;
}

void free_mixed(zbus_network net) {
  cudaFree(net->bsr_df);
  cudaFree(net->ys_df);
  net->bsr_df = nullptr;
  net->ys_df = nullptr;
  for (auto& op : net->mixed) {
    cudaFree(op.Z0);
    cudaFree(op.Z1);
    cudaFree(op.zinv);
    op = MixedOperands();
  }
}

int tc_grid(const MixedOperands& op, int B) {
  // persistent: one CTA per SM, at most one per tile
  return std::min(op.num_sms, ((B + BM - 1) / BM) * (op.N_pad / op.BN));
}

zbus_status launch_residual_mixed(zbus_network net, const MixedOperands& op, int B, void* R,
                                  float* rinv, cudaStream_t st) {
  const int Bp = round_up(B, 128);
  const int nchunks = ((op.K_pad >> 1) + CHUNK_ROWS - 1) / CHUNK_ROWS;
  const dim3 grid(Bp / 32, (nchunks + RES_WARPS - 1) / RES_WARPS);
  if (op.bf16)
    k_residual_df<true><<<grid, RES_WARPS * 32, 0, st>>>(net->ws.ctx, net->bsr_ptr, net->bsr_col,
                                                         net->bsr_df, net->ys_df, net->nbus,
                                                         op.K_pad, R, rinv);
  else
    k_residual_df<false><<<grid, RES_WARPS * 32, 0, st>>>(net->ws.ctx, net->bsr_ptr, net->bsr_col,
                                                          net->bsr_df, net->ys_df, net->nbus,
                                                          op.K_pad, R, rinv);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

zbus_status launch_contract_tc(zbus_network net, const MixedOperands& op, const CUtensorMap& tmR,
                               const float* rinv, int grid, cudaStream_t st) {
  cudaError_t e;
  if (op.bf16) {
    if (op.BN == 256) e = launch_tc_impl<256, 2, 2, true>(net->ws.ctx, op, tmR, rinv, net->n, grid, st);
    else e = launch_tc_impl<128, 2, 3, true>(net->ws.ctx, op, tmR, rinv, net->n, grid, st);
  } else {
    if (op.BN == 256) e = launch_tc_impl<256, 1, 4, false>(net->ws.ctx, op, tmR, rinv, net->n, grid, st);
    else e = launch_tc_impl<128, 1, 4, false>(net->ws.ctx, op, tmR, rinv, net->n, grid, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "tcgen05 contraction launch", __FILE__, __LINE__);
  return ZBUS_OK;
}

zbus_status launch_final_check(zbus_network net, int B, double* mm_out, cudaStream_t st) {
  k_final_check<<<B, 256, (size_t)16 * net->n, st>>>(net->ws.ctx, net->csr_ptr, net->csr_col,
                                                     net->csr_val, net->ys, net->n, mm_out);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

void launch_init_df(SolveCtx* ctx, int n, int B, int Bp, cudaStream_t st) {
  k_init_df<<<dim3((n + 31) / 32, Bp / 32), dim3(32, 8), 0, st>>>(ctx, n, B, Bp);
}

void launch_merge_df(SolveCtx* ctx, int n, int B, int Bp, cudaStream_t st) {
  k_merge_df<<<dim3((n + 31) / 32, Bp / 32), dim3(32, 8), 0, st>>>(ctx, n, B, Bp);
}

void launch_converge_mixed(SolveCtx* ctx, int B, cudaGraphConditionalHandle h, bool use_handle,
                           cudaStream_t st) {
  k_decide_mixed<<<(B + 255) / 256, 256, 0, st>>>(ctx, B);
  k_finish_mixed<<<1, 1024, 0, st>>>(ctx, round_up(B, 128) / 128, h, use_handle ? 1 : 0);
}

}  // namespace zbus
