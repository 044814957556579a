// Low-precision operands of the reduced impedance for the tensor-core
// contraction of the mixed-precision defect sweep (Sec. II-B fixed point as
// v <- v + Z_lp r(v)): the real 2x2 embedding of Z as row-scaled FP16 or as
// BF16 hi + lo, the double-float copies of the admittance blocks used by the
// residual, and the TMA tensor maps.  The sweep kernels are in group.cu.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "df.cuh"
#include "group.cuh"
#include "zbus_internal.cuh"

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

// Double-float copies of complex FP64 values (admittance blocks, Y_Ls v_s).
__global__ void k_split_c(const double2* __restrict__ val, int64_t m, float4* out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double2 y = val[t];
    const float2 a = df_split(y.x), b = df_split(y.y);
    out[t] = make_float4(a.x, a.y, b.x, b.y);
  }
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

// Double-float copies of the branch-form blocks, Y_Ls v_s and w, shared by
// the defect forms (independent of Z: kept when the dense operands are
// released).
zbus_status prepare_df(zbus_network net, cudaStream_t st) {
  if (!net->bsr_df) {
    const int64_t m = std::max<int64_t>(1, net->nblk * 9);
    ZB_CUDA(cudaMalloc((void**)&net->bsr_df, m * sizeof(float4)));
    ZB_CUDA(cudaMalloc((void**)&net->ys_df, (size_t)net->n * sizeof(float4)));
    if (net->nblk > 0)
      k_split_c<<<(int)std::min<int64_t>(2048, (net->nblk * 9 + 255) / 256), 256, 0, st>>>(
          net->bsr_val, net->nblk * 9, net->bsr_df);
    k_split_c<<<(net->n + 255) / 256, 256, 0, st>>>(net->ys, net->n, net->ys_df);
    ZB_CUDA(cudaMalloc((void**)&net->w_df, (size_t)net->n * sizeof(float4)));
    k_split_c<<<(net->n + 255) / 256, 256, 0, st>>>(net->w, net->n, net->w_df);
    ZB_CUDA(cudaGetLastError());
  }
  return ZBUS_OK;
}

zbus_status prepare_tree(zbus_network net, cudaStream_t st) {
  if (!net->bus_aligned)
    return fail(ZBUS_ERR_UNSUPPORTED, "the tree sweep needs three unknowns per bus (n % 3 == 0)");
  if (!net->radial)
    return fail(ZBUS_ERR_UNSUPPORTED,
                "the tree sweep needs a radial feeder (buses form a tree hanging off the slack, "
                "reciprocal invertible branch blocks)");
  if (tree_table_bytes(net->nbus) > (size_t)200 * 1024)
    return fail(ZBUS_ERR_UNSUPPORTED, "the tree sweep supports up to 3592 buses");
  ZB_CHECK(prepare_df(net, st));
  ZB_CUDA(cudaStreamSynchronize(st));
  return ZBUS_OK;
}

zbus_status prepare_mixed(zbus_network net, int32_t precision, cudaStream_t st) {
  MixedOperands& op = net->mixed[precision == ZBUS_MIXED_BF16X2 ? 1 : 0];
  if (op.ready) return ZBUS_OK;
  if (!net->bus_aligned)
    return fail(ZBUS_ERR_UNSUPPORTED, "mixed modes need three unknowns per bus (n % 3 == 0)");
  if (net->n > 16383)
    return fail(ZBUS_ERR_UNSUPPORTED, "mixed modes support n <= 16383 unknowns");
  ZB_CHECK(prepare_df(net, st));
  ZB_CHECK(ensure_z(net, st));
  const bool bf = precision == ZBUS_MIXED_BF16X2;
  op.bf16 = bf;
  op.zparts = bf ? 2 : 1;
  op.K_pad = round_up(2 * net->n, 64);
  op.N_pad = round_up(2 * net->n, 256);
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
  ZB_CUDA(cudaStreamSynchronize(st));
  op.ready = true;
  return ZBUS_OK;
}

void release_mixed_ops(zbus_network net) {
  for (auto& op : net->mixed) {
    cudaFree(op.Z0);
    cudaFree(op.Z1);
    cudaFree(op.zinv);
    op = MixedOperands();
  }
  net->op_gen += 1;
}

void free_mixed(zbus_network net) {
  cudaFree(net->bsr_df);
  cudaFree(net->ys_df);
  cudaFree(net->w_df);
  net->bsr_df = nullptr;
  net->ys_df = nullptr;
  net->w_df = nullptr;
  for (auto& op : net->mixed) {
    cudaFree(op.Z0);
    cudaFree(op.Z1);
    cudaFree(op.zinv);
    op = MixedOperands();
  }
}

}  // namespace zbus
