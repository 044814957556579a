// Mixed-precision defect sweep of the Z-bus fixed point (Sec. II-B).
//
// With Z Y_LL = I, the map v <- Z i(v) + w equals v <- v + Z r(v) with the
// residual r(v) = i(v) - Y_LL v - Y_Ls v_s.  The residual is formed in FP64
// from the sparse admittance matrix, so the fixed point is the FP64 one; the
// dense product Z r runs on the tcgen05 tensor cores with Z in FP16 (rows
// scaled by powers of two) or BF16 hi+lo, r rounded per scenario with a power
// of two scale, FP32 accumulation in tensor memory, and an FP64 epilogue
// v <- v + D.  A low-precision Z only changes the rate of convergence.
//
//   k_pack_tc         Z (complex FP64) -> real 2x2 embedding operand(s)
//   k_residual_mixed  r(v) in FP64 per active scenario -> low-precision R rows
//   k_contract_tc     D = R Z_emb^T on tcgen05, epilogue v += D, step partials
//   k_final_check     FP64 power mismatch of converged scenarios
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "loads.cuh"
#include "mixed.cuh"

namespace zbus {
namespace {

size_t residual_smem(int n) { return (size_t)32 * n; }

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
// Defect residual of one active scenario per block, in FP64:
//   r_j = i_j(v) - sum_c Y_LL[j][c] v_c - ys_j
// then R[slot][2j], R[slot][2j+1] = round(c_b Re r_j), round(c_b Im r_j) with
// c_b = 2^(12 - floor(log2 max|r|)); rinv[slot] = 1 / c_b.  v and r are staged
// in shared memory (32 n bytes).
// ---------------------------------------------------------------------------
template <bool BF>
__global__ void __launch_bounds__(256)
k_residual_mixed(const SolveCtx* __restrict__ ctx, const int32_t* __restrict__ ptr,
                 const int32_t* __restrict__ col, const double2* __restrict__ val,
                 const double2* __restrict__ ys, int n, int K_pad, void* Rout,
                 float* __restrict__ rinv) {
  extern __shared__ double2 dsm[];
  __shared__ double red[32];
  const int slot = blockIdx.x;
  if (slot >= ctx->count) return;
  const int b = ctx->list[slot];
  double2* sV = dsm;
  double2* sR = dsm + n;
  const double2* V = ctx->V + (int64_t)b * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) sV[j] = V[j];
  __syncthreads();
  const double2* Sw = ctx->S_wye ? ctx->S_wye + (int64_t)b * n : nullptr;
  const double2* Sd = ctx->S_del ? ctx->S_del + (int64_t)b * n : nullptr;
  double amax = 0.0;
  const int nb = (n + 2) / 3;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    const int j0 = 3 * k;
    const int m = min(3, n - j0);
    double2 vv[3], sw[3], sd[3], inj[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      vv[p] = p < m ? sV[j0 + p] : make_double2(1.0, 0.0);
      sw[p] = (Sw && p < m) ? Sw[j0 + p] : make_double2(0.0, 0.0);
      sd[p] = (Sd && p < m) ? Sd[j0 + p] : make_double2(0.0, 0.0);
    }
    bus_injection(vv, Sw ? sw : nullptr, Sd ? sd : nullptr, m, inj);
    for (int p = 0; p < m; ++p) {
      const int j = j0 + p;
      double2 acc = ys[j];
      for (int t = ptr[j]; t < ptr[j + 1]; ++t) {
        const double2 y = val[t], x = sV[col[t]];
        acc.x = fma(y.x, x.x, fma(-y.y, x.y, acc.x));
        acc.y = fma(y.x, x.y, fma(y.y, x.x, acc.y));
      }
      const double2 r = make_double2(inj[p].x - acc.x, inj[p].y - acc.y);
      sR[j] = r;
      amax = fmax(amax, fmax(fabs(r.x), fabs(r.y)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (threadIdx.x == 0) red[0] = x;
  }
  __syncthreads();
  amax = red[0];
  // a non-finite residual propagates as NaN into the step (the scenario then
  // stops as diverged); zero residual gives zero rows
  const int e = (amax > 0.0 && isfinite(amax)) ? 12 - ilogb(amax) : 0;
  const double c = ldexp(1.0, e);
  if (threadIdx.x == 0) rinv[slot] = isfinite(amax) ? (float)ldexp(1.0, -e) : __int_as_float(0x7fc00000);
  const int64_t row = (int64_t)slot * K_pad;
  for (int k = threadIdx.x; k < K_pad / 2; k += blockDim.x) {
    double2 r = k < n ? sR[k] : make_double2(0.0, 0.0);
    const double x = r.x * c, y = r.y * c;
    if (BF) {
      __nv_bfloat162 h = __halves2bfloat162(__double2bfloat16(x), __double2bfloat16(y));
      ((__nv_bfloat162*)Rout)[(row >> 1) + k] = h;
    } else {
      __half2 h = __halves2half2(__double2half(x), __double2half(y));
      ((__half2*)Rout)[(row >> 1) + k] = h;
    }
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
  uint64_t* accf = empty + STAGES;
  uint32_t* tmem_holder = (uint32_t*)(accf + 1);

  const int count = ctx->count;
  const int ntn = N_pad / BN;
  const int mtiles = (count + BM - 1) / BM;
  if ((int)blockIdx.x >= mtiles * ntn) return;   // whole block, before any barrier
  const int mt = blockIdx.x / ntn;
  const int nt = blockIdx.x % ntn;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_kb = K_pad / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_holder)),
                 "r"((uint32_t)BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      for (int kb = 0; kb < num_kb; ++kb) {
        const int s = kb % STAGES;
        const uint32_t round = kb / STAGES;
        if (!mbar_wait(&empty[s], (round & 1) ^ 1)) {
          atomicCAS(&ctx->err, 0, 101);
          break;
        }
        uint8_t* st = smem + s * STAGE_BYTES;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        tma_load_2d(st, &tmR, &full[s], kb * BK, mt * BM);
        tma_load_2d(st + A_BYTES, &tmZ0, &full[s], kb * BK, nt * BN);
        if (ZP == 2) tma_load_2d(st + A_BYTES + B_BYTES, &tmZ1, &full[s], kb * BK, nt * BN);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // kind::f16 instruction descriptor: D f32, A/B f16 or bf16, both K-major
      const uint32_t idesc = (1u << 4) | ((BF ? 1u : 0u) << 7) | ((BF ? 1u : 0u) << 10) |
                             ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
      bool ok = true;
      for (int kb = 0; kb < num_kb; ++kb) {
        const int s = kb % STAGES;
        const uint32_t round = kb / STAGES;
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
            umma_f16(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                     (kb | kk | p) != 0 ? 1u : 0u);
          }
        }
        umma_commit(&empty[s]);
      }
      if (ok) umma_commit(accf);
    }
  } else {
    // epilogue warps 2..5
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int slot = mt * BM + row;
    const bool ok = mbar_wait(accf, 0);
    tc_fence_after();
    if (!ok) {
      if (lane == 0) atomicCAS(&ctx->err, 0, 103);
    } else {
      const bool valid = slot < count;
      const int b = valid ? ctx->list[slot] : 0;
      const float rs = valid ? rinv[slot] : 0.f;
      double2* V = ctx->V + (int64_t)b * n;
      double dmax = 0.0, dsum = 0.0;
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 32), v);
        if (valid) {
          const int i0 = (nt * BN + c * 32) >> 1;
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int i = i0 + t;
            if (i < n) {
              const double sc = (double)rs * (double)zinv[i];
              const double dr = (double)v[2 * t] * sc, di = (double)v[2 * t + 1] * sc;
              const double2 vo = V[i];
              const double2 vn = make_double2(vo.x + dr, vo.y + di);
              V[i] = vn;
              double step = hypot(dr, di);
              if (step != step) step = INFINITY;
              dmax = fmax(dmax, step);
              dsum += hypot(vn.x, vn.y) - hypot(vo.x, vo.y);
            }
          }
        }
      }
      if (valid) {
        ctx->part[((int64_t)slot * ntn + nt) * 2 + 0] = dmax;
        ctx->part[((int64_t)slot * ntn + nt) * 2 + 1] = dsum;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)BN));
  }
}

// ---------------------------------------------------------------------------
// FP64 check of converged scenarios: the power mismatch
//   max_j |v_j| |(Y_LL v + ys)_j - i_j(v)|
// with the sparse admittance matrix; a converged scenario above mtol loses
// its flag.  One block per scenario.
// ---------------------------------------------------------------------------
__global__ void k_final_check(SolveCtx* __restrict__ ctx, const int32_t* __restrict__ ptr,
                              const int32_t* __restrict__ col, const double2* __restrict__ val,
                              const double2* __restrict__ ys, int n, double* mm_out) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  if (b >= ctx->B) return;
  if (ctx->conv[b] == 0) {
    if (threadIdx.x == 0 && mm_out) mm_out[b] = -1.0;
    return;
  }
  const double2* v = ctx->V + (int64_t)b * n;
  const double2* Sw = ctx->S_wye ? ctx->S_wye + (int64_t)b * n : nullptr;
  const double2* Sd = ctx->S_del ? ctx->S_del + (int64_t)b * n : nullptr;
  double worst = 0.0;
  const int nb = (n + 2) / 3;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    const int j0 = 3 * k;
    const int m = min(3, n - j0);
    double2 vv[3], sw[3], sd[3], inj[3];
    for (int p = 0; p < 3; ++p) {
      vv[p] = p < m ? v[j0 + p] : make_double2(1.0, 0.0);
      sw[p] = (Sw && p < m) ? Sw[j0 + p] : make_double2(0.0, 0.0);
      sd[p] = (Sd && p < m) ? Sd[j0 + p] : make_double2(0.0, 0.0);
    }
    bus_injection(vv, Sw ? sw : nullptr, Sd ? sd : nullptr, m, inj);
    for (int p = 0; p < m; ++p) {
      const int j = j0 + p;
      double2 acc = ys[j];
      for (int t = ptr[j]; t < ptr[j + 1]; ++t) {
        const double2 y = val[t], x = v[col[t]];
        acc.x += y.x * x.x - y.y * x.y;
        acc.y += y.x * x.y + y.y * x.x;
      }
      double e = hypot(vv[p].x, vv[p].y) * hypot(acc.x - inj[p].x, acc.y - inj[p].y);
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
    if (mm_out) mm_out[b] = x;
    if (!(x <= ctx->mismatch_tol)) ctx->conv[b] = 0;
  }
}

template <int BN, int ZP, int STAGES, bool BF>
constexpr size_t tc_smem_bytes() {
  return 1024 + (size_t)STAGES * (BM * BK * 2 + ZP * BN * BK * 2) + 256;
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
  if ((e = cudaFuncSetAttribute(k_residual_mixed<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                220 * 1024)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_residual_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
  if (residual_smem(net->n) > 220 * 1024)
    return fail(ZBUS_ERR_UNSUPPORTED, "mixed modes support n <= 7040 unknowns");
  ZB_CUDA(set_attributes());
  const bool bf = precision == ZBUS_MIXED_BF16X2;
  op.bf16 = bf;
  op.zparts = bf ? 2 : 1;
  op.K_pad = round_up(2 * net->n, BK);
  op.N_pad = round_up(2 * net->n, 256);
  op.BN = (2 * net->n > 1024) ? 256 : 128;
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
  for (auto& op : net->mixed) {
    cudaFree(op.Z0);
    cudaFree(op.Z1);
    cudaFree(op.zinv);
    op = MixedOperands();
  }
}

int tc_grid(const MixedOperands& op, int B) {
  return ((B + BM - 1) / BM) * (op.N_pad / op.BN);
}

zbus_status launch_residual_mixed(zbus_network net, const MixedOperands& op, int B, void* R,
                                  float* rinv, cudaStream_t st) {
  const size_t smem = residual_smem(net->n);
  if (smem > 220 * 1024)
    return fail(ZBUS_ERR_UNSUPPORTED, "mixed modes support n <= 7040 unknowns");
  if (op.bf16) {
    k_residual_mixed<true><<<B, 256, smem, st>>>(net->ws.ctx, net->csr_ptr, net->csr_col,
                                                 net->csr_val, net->ys, net->n, op.K_pad, R, rinv);
  } else {
    k_residual_mixed<false><<<B, 256, smem, st>>>(net->ws.ctx, net->csr_ptr, net->csr_col,
                                                  net->csr_val, net->ys, net->n, op.K_pad, R, rinv);
  }
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
  k_final_check<<<B, 256, 0, st>>>(net->ws.ctx, net->csr_ptr, net->csr_col, net->csr_val, net->ys,
                                   net->n, mm_out);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

}  // namespace zbus
