// Batched Newton-Raphson power flow for transmission grids (Sec. II-A).
//
// State x_b = [theta_Theta; |V|_Q] (angles of the PV and PQ buses, magnitudes
// of the PQ buses), mismatch F_b = [P_calc - P on Theta; Q_calc - Q on Q]
// with S_calc = V o conj(Y V) (eqs. 1-2), Newton step J dx = -F (eq. 3)
// solved by restarted GMRES on the left-preconditioned system
// M^-1 J dx = -M^-1 F.  J is never formed: GMRES uses the Jacobian-vector
// product dS = dV o conj(Y V) + V o conj(Y dV), dV = V o (j dtheta + d|V| / |V|).
// The preconditioner is the paper's block lower-triangular surrogate
// (eqs. 7-9):
//     z_Theta = (B' + eps I)^-1 diag(|V|_Theta)^-1 r_Theta
//     z_Q     = (B'' + eps I)^-1 diag(|V|_Q)^-1 (r_Q - G_Q,Theta z_Theta)
// with B' = -Im(Y)[Theta, Theta], B'' = -Im(Y)[Q, Q], G_Q,Theta = -Re(Y)[Q, Theta].
// The paper stores dense inverses of B' + eps I and B'' + eps I (its JAX
// stack lacks batched sparse direct solvers); here each is applied through
// its sparse LU factors (minimum-degree order, no pivoting: both matrices are
// diagonally dominant), whose triangular solves run level by level.  The
// operator is the same; a 2224-bus grid needs ~15 k factor entries and 35
// levels instead of a 40 MB dense inverse.
//
// GPU layout: one CTA solves one scenario at a time, from the flat start to
// the stop test, with every Newton and GMRES step inside the CTA (block-wide
// barriers only, no grid synchronisation, no host round trip); CTAs stride
// over the scenarios.  Per-CTA vectors and the Krylov basis live in a global
// scratch slice of the CTA (L1/L2 resident); the network (Y in CSR, the
// factors, their level lists) is shared read-only by all CTAs.  Arnoldi uses
// classical Gram-Schmidt applied twice (all dot products of one pass in one
// block reduction), the Hessenberg matrix is reduced by Givens rotations.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <vector>

#include "zbus_internal.cuh"

namespace zbus {
namespace nr {

constexpr int NR_THREADS = 128;
constexpr int NR_MIN_CTAS = 8;   // CTAs per SM the register budget is sized for
constexpr int NR_WARPS = NR_THREADS / 32;
constexpr int NR_MAX_RESTART_LEN = 60;

// One factor P A P^T = L U of the preconditioner on the device.
struct Factor {
  int n = 0;
  int32_t* perm = nullptr;    // [n] factor index -> position in the block
  // Rows of both triangles are stored in the order of their solve's levels:
  // slot k of the forward solve is row fl_row[k], its strictly lower entries
  // l_col / l_val[l_ptr[k] .. l_ptr[k+1]); slot k of the backward solve is
  // row bl_row[k] with strictly upper entries u_* and 1 / U_kk in dinv[k].
  int32_t* l_ptr = nullptr;
  int32_t* l_col = nullptr;
  double* l_val = nullptr;
  int32_t* u_ptr = nullptr;
  int32_t* u_col = nullptr;
  double* u_val = nullptr;
  double* dinv = nullptr;
  float* l_val_f = nullptr;   // FP32 copies of the values (mixed form)
  float* u_val_f = nullptr;
  float* dinv_f = nullptr;
  int32_t* fl_ptr = nullptr;  // forward levels: slots fl_ptr[l] .. fl_ptr[l+1]
  int32_t* fl_row = nullptr;
  int32_t* bl_ptr = nullptr;  // backward levels
  int32_t* bl_row = nullptr;
  int n_fl = 0, n_bl = 0;
  int64_t nnz = 0;
};

// Everything the solve kernel reads, by value.
struct NrDev {
  int N, nt, nq, dim, m;
  const int32_t* y_ptr;
  const int32_t* y_col;
  const double2* y_val;
  const int32_t* bus_type;
  const double* v_set;
  const int32_t* pos_t;   // [N] position in the angle block, -1 at the slack
  const int32_t* pos_q;   // [N] position in the magnitude block, -1 unless PQ
  const int32_t* t_bus;   // [nt]
  const int32_t* q_bus;   // [nq]
  const int32_t* g_ptr;   // G_Q,Theta CSR: rows = Q positions, cols = Theta positions
  const int32_t* g_col;
  const double* g_val;
  const float2* y_val_f;  // FP32 copies (mixed form)
  const float* g_val_f;
  Factor Bp, Bpp;
  double* scratch;
  int64_t stride;         // doubles of scratch per CTA
};

}  // namespace nr
}  // namespace zbus

struct zbus_nr_network_s {
  int device = 0;
  int N = 0, nt = 0, nq = 0;
  int slack = 0;
  zbus::nr::NrDev dev{};
  std::vector<void*> allocs;      // every device buffer of the network
  double* scratch = nullptr;
  int64_t scratch_ctas = 0;
  int64_t scratch_stride = 0;
  size_t smem_set[2] = {0, 0};
  int sms = 1;
};

namespace zbus {
namespace nr {
namespace {

// ---------------------------------------------------------------------------
// Device helpers (block-wide; every thread of the CTA calls them).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(0xffffffffu, v, o);
    v = (y > v || y != y) ? y : v;
  }
  return v;
}

// Sum (or max) over the CTA of one value per thread; every thread gets it.
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NR_WARPS; ++k) s += red[k];
  return s;
}
__device__ double block_max(double v, double* red) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NR_WARPS; ++k) s = (red[k] > s || red[k] != red[k]) ? red[k] : s;
  return s;
}

// Values in the Krylov precision T: FP64 (the paper's solver) or FP32 (the
// mixed form, whose Newton direction is found in FP32 while the mismatch,
// the state and the stop test stay FP64).
template <class T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };

template <class T> __device__ __forceinline__ const T* lval(const Factor& f);
template <> __device__ __forceinline__ const double* lval<double>(const Factor& f) { return f.l_val; }
template <> __device__ __forceinline__ const float* lval<float>(const Factor& f) { return f.l_val_f; }
template <class T> __device__ __forceinline__ const T* uval(const Factor& f);
template <> __device__ __forceinline__ const double* uval<double>(const Factor& f) { return f.u_val; }
template <> __device__ __forceinline__ const float* uval<float>(const Factor& f) { return f.u_val_f; }
template <class T> __device__ __forceinline__ const T* dval(const Factor& f);
template <> __device__ __forceinline__ const double* dval<double>(const Factor& f) { return f.dinv; }
template <> __device__ __forceinline__ const float* dval<float>(const Factor& f) { return f.dinv_f; }
template <class T> __device__ __forceinline__ const T* gval(const NrDev& d);
template <> __device__ __forceinline__ const double* gval<double>(const NrDev& d) { return d.g_val; }
template <> __device__ __forceinline__ const float* gval<float>(const NrDev& d) { return d.g_val_f; }
template <class T> __device__ __forceinline__ const typename Cx<T>::type* yval(const NrDev& d);
template <> __device__ __forceinline__ const double2* yval<double>(const NrDev& d) { return d.y_val; }
template <> __device__ __forceinline__ const float2* yval<float>(const NrDev& d) { return d.y_val_f; }

// Solve (P A P^T) with its LU factors: out[perm[i]] = (U^-1 L^-1 (in o perm))_i.
// in / out indexed by block position; y is factor-order work space.
template <class T>
__device__ void factor_solve(const Factor& f, const T* in, T* y, T* out) {
  const int t = threadIdx.x;
  const T* lv = lval<T>(f);
  const T* uv = uval<T>(f);
  const T* dv = dval<T>(f);
  for (int i = t; i < f.n; i += NR_THREADS)
    y[i] = ZB_IN(f.perm[i], f.n, 0x401u) ? in[f.perm[i]] : T(0);
  __syncthreads();
  for (int l = 0; l < f.n_fl; ++l) {
    for (int k = f.fl_ptr[l] + t; k < f.fl_ptr[l + 1]; k += NR_THREADS) {
      const int i = __ldg(f.fl_row + k);
      const int e0 = __ldg(f.l_ptr + k), e1 = __ldg(f.l_ptr + k + 1);
      if (!ZB_IN(i, f.n, 0x402u)) continue;
      T s = y[i];
      for (int e = e0; e < e1; ++e)
        if (ZB_IN(__ldg(f.l_col + e), f.n, 0x403u)) s -= __ldg(lv + e) * y[__ldg(f.l_col + e)];
      y[i] = s;
    }
    __syncthreads();
  }
  for (int l = 0; l < f.n_bl; ++l) {
    for (int k = f.bl_ptr[l] + t; k < f.bl_ptr[l + 1]; k += NR_THREADS) {
      const int i = __ldg(f.bl_row + k);
      const int e0 = __ldg(f.u_ptr + k), e1 = __ldg(f.u_ptr + k + 1);
      const T di = __ldg(dv + k);
      if (!ZB_IN(i, f.n, 0x404u)) continue;
      T s = y[i];
      for (int e = e0; e < e1; ++e)
        if (ZB_IN(__ldg(f.u_col + e), f.n, 0x405u)) s -= __ldg(uv + e) * y[__ldg(f.u_col + e)];
      y[i] = s * di;
    }
    __syncthreads();
  }
  for (int i = t; i < f.n; i += NR_THREADS)
    if (ZB_IN(f.perm[i], f.n, 0x406u)) out[f.perm[i]] = y[i];
  __syncthreads();
}

// z = M^-1 r (eqs. 8-9).  ivm = 1 / |V|; tmp: dim values, y: max(nt, nq) values.
template <class T>
__device__ void precondition(const NrDev& d, const T* ivm, const T* r, T* z, T* tmp, T* y) {
  const int t = threadIdx.x;
  for (int p = t; p < d.nt; p += NR_THREADS)
    tmp[p] = ZB_IN(d.t_bus[p], d.N, 0x407u) ? r[p] * ivm[d.t_bus[p]] : T(0);
  __syncthreads();
  factor_solve<T>(d.Bp, tmp, y, z);
  if (d.nq > 0) {
    const T* gv = gval<T>(d);
    for (int p = t; p < d.nq; p += NR_THREADS) {
      T s = r[d.nt + p];
      for (int e = __ldg(d.g_ptr + p); e < __ldg(d.g_ptr + p + 1); ++e)
        if (ZB_IN(__ldg(d.g_col + e), d.nt, 0x408u)) s -= __ldg(gv + e) * z[__ldg(d.g_col + e)];
      tmp[d.nt + p] = ZB_IN(d.q_bus[p], d.N, 0x409u) ? s * ivm[d.q_bus[p]] : T(0);
    }
    __syncthreads();
    factor_solve<T>(d.Bpp, tmp + d.nt, y, z + d.nt);
  }
}

// out = J u, the Jacobian of F at V (I = Y V) applied to u (dim); ivm = 1 / |V|.
template <class T>
__device__ void jvp(const NrDev& d, const T* Vr, const T* Vi, const T* Ir, const T* Ii,
                    const T* ivm, const T* u, T* dVr, T* dVi, T* out) {
  const int t = threadIdx.x;
  const typename Cx<T>::type* yv = yval<T>(d);
  for (int i = t; i < d.N; i += NR_THREADS) {
    const int pt = d.pos_t[i], pq = d.pos_q[i];
    const T dth = pt >= 0 ? u[pt] : T(0);
    const T a = pq >= 0 ? u[d.nt + pq] * ivm[i] : T(0);
    dVr[i] = Vr[i] * a - Vi[i] * dth;
    dVi[i] = Vi[i] * a + Vr[i] * dth;
  }
  __syncthreads();
  for (int i = t; i < d.N; i += NR_THREADS) {
    const int pt = d.pos_t[i], pq = d.pos_q[i];
    if (pt < 0 && pq < 0) continue;
    T yr = 0, yi = 0;
    for (int e = d.y_ptr[i]; e < d.y_ptr[i + 1]; ++e) {
      const auto y = __ldg(yv + e);
      const int j = __ldg(d.y_col + e);
      if (!ZB_IN(j, d.N, 0x40au)) continue;
      yr += y.x * dVr[j] - y.y * dVi[j];
      yi += y.x * dVi[j] + y.y * dVr[j];
    }
    // dS = dV conj(I) + V conj(Y dV)
    const T sr = dVr[i] * Ir[i] + dVi[i] * Ii[i] + Vr[i] * yr + Vi[i] * yi;
    const T si = dVi[i] * Ir[i] - dVr[i] * Ii[i] + Vi[i] * yr - Vr[i] * yi;
    if (pt >= 0) out[pt] = sr;
    if (pq >= 0) out[d.nt + pq] = si;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The solve: one CTA per scenario at a time.
// ---------------------------------------------------------------------------
struct SolveArgs {
  int B;
  const double* P;        // [B][N]
  const double* Q;        // [B][N]
  double tol;
  int max_iter;
  double eta;             // GMRES relative tolerance on the preconditioned residual
  int max_restart;
  double2* V;             // [B][N]
  int32_t* iters;
  uint8_t* conv;
  int32_t* gmres;
};

// Per-CTA scratch: the FP64 state (7 N + dim doubles), then the Krylov-
// precision arrays (FP32 copies of V, I, 1/|V| for the mixed form; dV;
// right-hand side, solution, work vectors; the basis).
__host__ __device__ constexpr int64_t state_doubles(int64_t N, int64_t dim) {
  return 7 * N + dim;
}
template <class T>
__host__ __device__ constexpr int64_t krylov_values(int64_t N, int64_t dim, int m) {
  return (sizeof(T) == 4 ? 5 * N : 0) + 2 * N + 5 * dim + (int64_t)(m + 1) * dim;
}

template <class T>
__global__ void __launch_bounds__(NR_THREADS, NR_MIN_CTAS) k_nr_solve(NrDev d, SolveArgs a) {
  constexpr bool MIXED = sizeof(T) == 4;
  extern __shared__ double sm[];
  const int m = d.m;
  double* H = sm;                          // [(m + 1) * m], column j at H[j * (m + 1)]
  double* cs = H + (m + 1) * m;            // [m]
  double* sn = cs + m;                     // [m]
  double* gv = sn + m;                     // [m + 1]
  double* hh = gv + m + 1;                 // [m + 1] this step's Gram-Schmidt coefficients
  double* red = hh + m + 1;                // [(m + 1) * NR_WARPS]
  T* hT = reinterpret_cast<T*>(red + (m + 1) * NR_WARPS);  // [m + 1] hh in T, converted once
  T* y = hT + m + 2;                       // [N] factor work space
  __shared__ int s_flag;
  __shared__ int s_jd;

  const int t = threadIdx.x, w = t >> 5, l = t & 31;
  const int N = d.N, nt = d.nt, dim = d.dim;
  double* base = d.scratch + (int64_t)blockIdx.x * d.stride;
  double* Vr = base;
  double* Vi = Vr + N;
  double* Ir = Vi + N;
  double* Ii = Ir + N;
  double* vm = Ii + N;
  double* va = vm + N;
  double* ivm = va + N;                    // N, 1 / |V| of the current iterate
  double* F = ivm + N;                     // dim
  T* kb = reinterpret_cast<T*>(F + dim);
  const T *VrT, *ViT, *IrT, *IiT, *ivmT;   // the state in the Krylov precision
  T *VrW = nullptr, *ViW = nullptr, *IrW = nullptr, *IiW = nullptr, *ivmW = nullptr;
  if constexpr (MIXED) {
    VrW = kb;
    ViW = VrW + N;
    IrW = ViW + N;
    IiW = IrW + N;
    ivmW = IiW + N;
    kb = ivmW + N;
    VrT = VrW, ViT = ViW, IrT = IrW, IiT = IiW, ivmT = ivmW;
  } else {
    VrT = reinterpret_cast<const T*>(Vr), ViT = reinterpret_cast<const T*>(Vi);
    IrT = reinterpret_cast<const T*>(Ir), IiT = reinterpret_cast<const T*>(Ii);
    ivmT = reinterpret_cast<const T*>(ivm);
  }
  T* dVr = kb;
  T* dVi = dVr + N;
  T* bv = dVi + N;
  T* x = bv + dim;
  T* wv = x + dim;
  T* tmp = wv + dim;
  T* work = tmp + dim;
  T* Vk = work + dim;                      // basis, (m + 1) * dim

  for (int b = blockIdx.x; b < a.B; b += gridDim.x) {
    const double* P = a.P + (int64_t)b * N;
    const double* Q = a.Q + (int64_t)b * N;
    for (int i = t; i < N; i += NR_THREADS) {
      vm[i] = d.bus_type[i] == 0 ? 1.0 : d.v_set[i];
      va[i] = 0.0;
    }
    int gm_total = 0, it = 0, ok = 0;
    __syncthreads();
    for (int k = 0;; ++k) {
      // V, I = Y V, mismatch F and its max (FP64)
      for (int i = t; i < N; i += NR_THREADS) {
        double s, c;
        sincos(va[i], &s, &c);
        Vr[i] = vm[i] * c;
        Vi[i] = vm[i] * s;
        ivm[i] = 1.0 / vm[i];
        if constexpr (MIXED) {
          VrW[i] = (T)Vr[i];
          ViW[i] = (T)Vi[i];
          ivmW[i] = (T)ivm[i];
        }
      }
      __syncthreads();
      double fmax = 0.0;
      for (int i = t; i < N; i += NR_THREADS) {
        double ir = 0.0, ii = 0.0;
        for (int e = d.y_ptr[i]; e < d.y_ptr[i + 1]; ++e) {
          const double2 yv = d.y_val[e];
          const int j = d.y_col[e];
          if (!ZB_IN(j, N, 0x40bu)) continue;
          ir += yv.x * Vr[j] - yv.y * Vi[j];
          ii += yv.x * Vi[j] + yv.y * Vr[j];
        }
        Ir[i] = ir;
        Ii[i] = ii;
        if constexpr (MIXED) {
          IrW[i] = (T)ir;
          IiW[i] = (T)ii;
        }
        const double sr = Vr[i] * ir + Vi[i] * ii;   // V conj(I)
        const double si = Vi[i] * ir - Vr[i] * ii;
        const int pt = d.pos_t[i], pq = d.pos_q[i];
        if (pt >= 0) {
          const double f = sr - P[i];
          F[pt] = f;
          fmax = (fabs(f) > fmax || f != f) ? fabs(f) : fmax;
        }
        if (pq >= 0) {
          const double f = si - Q[i];
          F[nt + pq] = f;
          fmax = (fabs(f) > fmax || f != f) ? fabs(f) : fmax;
        }
      }
      fmax = block_max(fmax, red);
      it = k;
      if (!(fmax <= a.tol)) {
        if (fmax != fmax || isinf(fmax) || k == a.max_iter) break;
      } else {
        ok = 1;
        break;
      }
      // GMRES on M^-1 J dx = M^-1 (-F), x0 = 0
      for (int e = t; e < dim; e += NR_THREADS) {
        wv[e] = (T)(-F[e]);
        x[e] = T(0);
      }
      __syncthreads();
      precondition<T>(d, ivmT, wv, bv, tmp, y);
      T nb = 0;
      for (int e = t; e < dim; e += NR_THREADS) nb += bv[e] * bv[e];
      const double beta0 = sqrt(block_sum((double)nb, red));
      bool done = !(beta0 > 0.0);
      for (int rs = 0; rs < a.max_restart && !done; ++rs) {
        // r = b - A x (x = 0 on the first pass)
        if (rs > 0) {
          jvp<T>(d, VrT, ViT, IrT, IiT, ivmT, x, dVr, dVi, tmp);
          precondition<T>(d, ivmT, tmp, wv, work, y);
          for (int e = t; e < dim; e += NR_THREADS) Vk[e] = bv[e] - wv[e];
        } else {
          for (int e = t; e < dim; e += NR_THREADS) Vk[e] = bv[e];
        }
        T nr = 0;
        for (int e = t; e < dim; e += NR_THREADS) nr += Vk[e] * Vk[e];
        const double beta = sqrt(block_sum((double)nr, red));
        if (!(beta > a.eta * beta0)) break;
        const T ib = (T)(1.0 / beta);
        for (int e = t; e < dim; e += NR_THREADS) Vk[e] *= ib;
        if (t == 0) {
          gv[0] = beta;
          s_jd = 0;
          s_flag = 0;
        }
        __syncthreads();
        for (int j = 0; j < m; ++j) {
          T* vj = Vk + (int64_t)j * dim;
          jvp<T>(d, VrT, ViT, IrT, IiT, ivmT, vj, dVr, dVi, tmp);
          precondition<T>(d, ivmT, tmp, wv, work, y);
          // classical Gram-Schmidt, twice; products in T, sums across the
          // warp and the CTA in FP64
          for (int i = t; i <= j; i += NR_THREADS) H[j * (m + 1) + i] = 0.0;
          __syncthreads();
          for (int pass = 0; pass < 2; ++pass) {
            for (int i = 0; i <= j; ++i) {
              const T* vi = Vk + (int64_t)i * dim;
              T s = 0;
              for (int e = t; e < dim; e += NR_THREADS) s += vi[e] * wv[e];
              const double sw = warp_sum((double)s);
              if (l == 0) red[i * NR_WARPS + w] = sw;
            }
            __syncthreads();
            for (int i = t; i <= j; i += NR_THREADS) {
              double s = 0.0;
              for (int q = 0; q < NR_WARPS; ++q) s += red[i * NR_WARPS + q];
              hh[i] = s;
              hT[i] = (T)s;
              H[j * (m + 1) + i] += s;
            }
            __syncthreads();
            for (int e = t; e < dim; e += NR_THREADS) {
              T s = wv[e];
              for (int i = 0; i <= j; ++i) s -= hT[i] * Vk[(int64_t)i * dim + e];
              wv[e] = s;
            }
            __syncthreads();
          }
          T nw = 0;
          for (int e = t; e < dim; e += NR_THREADS) nw += wv[e] * wv[e];
          const double hn = sqrt(block_sum((double)nw, red));
          T* vn = Vk + (int64_t)(j + 1) * dim;
          const T inv = hn > 0.0 ? (T)(1.0 / hn) : T(0);
          for (int e = t; e < dim; e += NR_THREADS) vn[e] = wv[e] * inv;
          if (t == 0) {
            double* h = H + j * (m + 1);
            h[j + 1] = hn;
            for (int i = 0; i < j; ++i) {   // earlier rotations
              const double r0 = cs[i] * h[i] + sn[i] * h[i + 1];
              h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
              h[i] = r0;
            }
            const double den = hypot(h[j], h[j + 1]);
            cs[j] = den > 0.0 ? h[j] / den : 1.0;
            sn[j] = den > 0.0 ? h[j + 1] / den : 0.0;
            h[j] = den;
            h[j + 1] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            s_jd = j + 1;
            const double res = fabs(gv[j + 1]);
            s_flag = (res <= a.eta * beta0 || !(hn > 0.0) || res != res) ? 1 : 0;
          }
          __syncthreads();
          ++gm_total;
          if (s_flag) break;
        }
        // y = H^-1 g (upper triangular), x += V y
        const int jd = s_jd;
        if (t == 0) {
          for (int i = jd - 1; i >= 0; --i) {
            double s = gv[i];
            for (int c = i + 1; c < jd; ++c) s -= H[c * (m + 1) + i] * hh[c];
            hh[i] = s / H[i * (m + 1) + i];
            hT[i] = (T)hh[i];
          }
        }
        __syncthreads();
        for (int e = t; e < dim; e += NR_THREADS) {
          T s = x[e];
          for (int i = 0; i < jd; ++i) s += hT[i] * Vk[(int64_t)i * dim + e];
          x[e] = s;
        }
        __syncthreads();
        if (s_flag) done = true;
      }
      // Newton update (FP64 state)
      for (int p = t; p < nt; p += NR_THREADS)
        if (ZB_IN(d.t_bus[p], N, 0x40cu)) va[d.t_bus[p]] += (double)x[p];
      for (int p = t; p < d.nq; p += NR_THREADS)
        if (ZB_IN(d.q_bus[p], N, 0x40du)) vm[d.q_bus[p]] += (double)x[nt + p];
      __syncthreads();
    }
    double2* Vo = a.V + (int64_t)b * N;
    for (int i = t; i < N; i += NR_THREADS) Vo[i] = make_double2(Vr[i], Vi[i]);
    if (t == 0) {
      a.iters[b] = it;
      a.conv[b] = (uint8_t)ok;
      if (a.gmres) a.gmres[b] = gm_total;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side: ordering, factorisation, level lists.
// ---------------------------------------------------------------------------

// Minimum-degree order of the symmetrised pattern of A (n x n, rows of
// (col, value) pairs), eliminating one node at a time and joining its
// neighbours; ties go to the lowest index.
std::vector<int> min_degree(int n, const std::vector<std::map<int, double>>& A) {
  std::vector<std::set<int>> adj(n);
  for (int i = 0; i < n; ++i)
    for (auto& kv : A[i])
      if (kv.first != i) {
        adj[i].insert(kv.first);
        adj[kv.first].insert(i);
      }
  std::vector<char> gone(n, 0);
  std::vector<int> order;
  order.reserve(n);
  for (int step = 0; step < n; ++step) {
    int best = -1;
    size_t bd = SIZE_MAX;
    for (int i = 0; i < n; ++i)
      if (!gone[i] && adj[i].size() < bd) {
        bd = adj[i].size();
        best = i;
      }
    gone[best] = 1;
    order.push_back(best);
    std::vector<int> nb(adj[best].begin(), adj[best].end());
    for (int u : nb) adj[u].erase(best);
    for (size_t p = 0; p < nb.size(); ++p)
      for (size_t q = p + 1; q < nb.size(); ++q) {
        adj[nb[p]].insert(nb[q]);
        adj[nb[q]].insert(nb[p]);
      }
    adj[best].clear();
  }
  return order;
}

struct HostFactor {
  int n = 0;
  std::vector<int32_t> perm, l_ptr, l_col, u_ptr, u_col, fl_ptr, fl_row, bl_ptr, bl_row;
  std::vector<double> l_val, u_val, dinv;
};

// LU of P A P^T without pivoting (right-looking, sparse rows), the level
// lists of both triangular solves.  False if a pivot is not usable.
bool factorise(int n, const std::vector<std::map<int, double>>& A, HostFactor& hf,
               std::string& why) {
  hf = HostFactor();
  hf.n = n;
  hf.perm = min_degree(n, A);
  std::vector<int> inv(n);
  for (int i = 0; i < n; ++i) inv[hf.perm[i]] = i;
  std::vector<std::map<int, double>> R(n);            // rows of P A P^T
  std::vector<std::set<int>> below(n);                // rows i > k with an entry in column k
  double amax = 0.0;
  for (int i = 0; i < n; ++i)
    for (auto& kv : A[i]) {
      const int r = inv[i], c = inv[kv.first];
      R[r][c] += kv.second;
      if (r > c) below[c].insert(r);
      amax = std::max(amax, std::fabs(kv.second));
    }
  std::vector<std::vector<std::pair<int, double>>> Lrows(n);
  hf.dinv.assign(n, 0.0);
  std::vector<std::vector<std::pair<int, double>>> Urows(n);
  for (int k = 0; k < n; ++k) {
    auto itp = R[k].find(k);
    const double piv = itp == R[k].end() ? 0.0 : itp->second;
    if (!(std::fabs(piv) > 1e-13 * std::max(amax, 1e-300)) || !std::isfinite(piv)) {
      why = "zero or tiny pivot in the preconditioner factor at row " + std::to_string(k);
      return false;
    }
    hf.dinv[k] = 1.0 / piv;
    for (auto& kv : R[k])
      if (kv.first > k) Urows[k].push_back(kv);
    for (int i : below[k]) {
      auto e = R[i].find(k);
      if (e == R[i].end()) continue;
      const double lik = e->second / piv;
      R[i].erase(e);
      Lrows[i].push_back({k, lik});
      for (auto& kv : Urows[k]) {
        const int j = kv.first;
        auto f = R[i].find(j);
        if (f == R[i].end()) {
          R[i][j] = -lik * kv.second;
          if (i > j) below[j].insert(i);
        } else {
          f->second -= lik * kv.second;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) std::sort(Lrows[i].begin(), Lrows[i].end());
  // level lists: forward (row i after its lower columns), backward (after
  // its upper columns); rows stored slot by slot in level order
  std::vector<int> lev(n, 0);
  int nl = 0;
  for (int i = 0; i < n; ++i) {
    int v = 0;
    for (auto& kv : Lrows[i]) v = std::max(v, lev[kv.first] + 1);
    lev[i] = v;
    nl = std::max(nl, v + 1);
  }
  std::vector<std::vector<int>> byl(nl);
  for (int i = 0; i < n; ++i) byl[lev[i]].push_back(i);
  hf.fl_ptr.push_back(0);
  hf.l_ptr.push_back(0);
  for (auto& v : byl) {
    for (int i : v) {
      hf.fl_row.push_back(i);
      for (auto& kv : Lrows[i]) {
        hf.l_col.push_back(kv.first);
        hf.l_val.push_back(kv.second);
      }
      hf.l_ptr.push_back((int32_t)hf.l_col.size());
    }
    hf.fl_ptr.push_back((int32_t)hf.fl_row.size());
  }
  std::fill(lev.begin(), lev.end(), 0);
  nl = 0;
  for (int i = n - 1; i >= 0; --i) {
    int v = 0;
    for (auto& kv : Urows[i]) v = std::max(v, lev[kv.first] + 1);
    lev[i] = v;
    nl = std::max(nl, v + 1);
  }
  std::vector<std::vector<int>> byb(nl);
  for (int i = 0; i < n; ++i) byb[lev[i]].push_back(i);
  std::vector<double> dinv_row = hf.dinv;
  hf.dinv.clear();
  hf.bl_ptr.push_back(0);
  hf.u_ptr.push_back(0);
  for (auto& v : byb) {
    for (int i : v) {
      hf.bl_row.push_back(i);
      hf.dinv.push_back(dinv_row[i]);
      for (auto& kv : Urows[i]) {
        hf.u_col.push_back(kv.first);
        hf.u_val.push_back(kv.second);
      }
      hf.u_ptr.push_back((int32_t)hf.u_col.size());
    }
    hf.bl_ptr.push_back((int32_t)hf.bl_row.size());
  }
  return true;
}

template <class T>
zbus_status upload(zbus_nr_network net, T** dst, const std::vector<T>& src, cudaStream_t st) {
  const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  ZB_CUDA(cudaMalloc((void**)dst, bytes));
  net->allocs.push_back(*dst);
  if (!src.empty())
    ZB_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return ZBUS_OK;
}

std::vector<float> to_float(const std::vector<double>& v) {
  return std::vector<float>(v.begin(), v.end());
}

zbus_status upload_factor(zbus_nr_network net, const HostFactor& hf, Factor& f, cudaStream_t st) {
  f.n = hf.n;
  ZB_CHECK(upload(net, &f.perm, hf.perm, st));
  ZB_CHECK(upload(net, &f.l_ptr, hf.l_ptr, st));
  ZB_CHECK(upload(net, &f.l_col, hf.l_col, st));
  ZB_CHECK(upload(net, &f.l_val, hf.l_val, st));
  ZB_CHECK(upload(net, &f.u_ptr, hf.u_ptr, st));
  ZB_CHECK(upload(net, &f.u_col, hf.u_col, st));
  ZB_CHECK(upload(net, &f.u_val, hf.u_val, st));
  ZB_CHECK(upload(net, &f.dinv, hf.dinv, st));
  ZB_CHECK(upload(net, &f.l_val_f, to_float(hf.l_val), st));
  ZB_CHECK(upload(net, &f.u_val_f, to_float(hf.u_val), st));
  ZB_CHECK(upload(net, &f.dinv_f, to_float(hf.dinv), st));
  ZB_CHECK(upload(net, &f.fl_ptr, hf.fl_ptr, st));
  ZB_CHECK(upload(net, &f.fl_row, hf.fl_row, st));
  ZB_CHECK(upload(net, &f.bl_ptr, hf.bl_ptr, st));
  ZB_CHECK(upload(net, &f.bl_row, hf.bl_row, st));
  f.n_fl = (int)hf.fl_ptr.size() - 1;
  f.n_bl = (int)hf.bl_ptr.size() - 1;
  f.nnz = (int64_t)hf.l_val.size() + (int64_t)hf.u_val.size() + hf.n;
  return ZBUS_OK;
}

size_t smem_bytes(int m, int N, bool mixed) {
  return sizeof(double) * ((size_t)(m + 1) * m + 2 * m + 2 * (m + 1) + (size_t)(m + 1) * NR_WARPS) +
         (mixed ? sizeof(float) : sizeof(double)) * ((size_t)N + m + 2);
}

int64_t scratch_doubles(const zbus_nr_network net, int m, bool mixed) {
  const int64_t N = net->N, dim = net->nt + net->nq;
  const int64_t kv = mixed ? (krylov_values<float>(N, dim, m) + 1) / 2
                           : krylov_values<double>(N, dim, m);
  const int64_t s = state_doubles(N, dim) + kv;
  return (s + 31) / 32 * 32;
}

}  // namespace
}  // namespace nr

ZB_CHECK_WORD_ACCESSOR(check_word_nr)

}  // namespace zbus

using namespace zbus;
using namespace zbus::nr;

extern "C" {

void zbus_nr_opts_default(zbus_nr_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->gmres_restart = 30;
  o->gmres_max_restarts = 4;
  o->gmres_tol = 1e-6;
  o->precision = ZBUS_NR_FP64;
}

zbus_status zbus_nr_network_create(int32_t N, int64_t nnz, const int32_t* row,
                                   const int32_t* col, const double* val_reim,
                                   const int32_t* bus_type, const double* v_set, double eps,
                                   void* cuda_stream, zbus_nr_network* out) {
  NvtxRange nvtx_range("zbus_nr_network_create");
  set_error("");
  if (!out) return fail(ZBUS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (N < 2) return fail(ZBUS_ERR_ARG, "N must be >= 2");
  if (nnz < 1) return fail(ZBUS_ERR_ARG, "nnz must be >= 1");
  if (!row || !col || !val_reim || !bus_type || !v_set)
    return fail(ZBUS_ERR_ARG, "a required host array is NULL");
  if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(ZBUS_ERR_ARG, "eps must be finite, >= 0");
  int slack = -1;
  for (int i = 0; i < N; ++i) {
    if (bus_type[i] < 0 || bus_type[i] > 2) return fail(ZBUS_ERR_ARG, "bus_type must be 0, 1 or 2");
    if (bus_type[i] == 2) {
      if (slack >= 0) return fail(ZBUS_ERR_ARG, "exactly one slack bus (type 2) is required");
      slack = i;
    }
    if (bus_type[i] != 0 && !(v_set[i] > 0.0 && std::isfinite(v_set[i])))
      return fail(ZBUS_ERR_ARG, "v_set of a PV or slack bus must be finite and > 0");
  }
  if (slack < 0) return fail(ZBUS_ERR_ARG, "exactly one slack bus (type 2) is required");
  std::vector<std::map<int, std::pair<double, double>>> Yrows(N);
  for (int64_t t = 0; t < nnz; ++t) {
    if (row[t] < 0 || row[t] >= N || col[t] < 0 || col[t] >= N)
      return fail(ZBUS_ERR_ARG, "COO index out of range at entry " + std::to_string(t));
    if (!std::isfinite(val_reim[2 * t]) || !std::isfinite(val_reim[2 * t + 1]))
      return fail(ZBUS_ERR_ARG, "COO value not finite at entry " + std::to_string(t));
    auto& e = Yrows[row[t]][col[t]];
    e.first += val_reim[2 * t];
    e.second += val_reim[2 * t + 1];
  }
  auto* net = new zbus_nr_network_s();
  cudaError_t ce = cudaGetDevice(&net->device);
  if (ce != cudaSuccess) {
    delete net;
    return cuda_fail(ce, "cudaGetDevice", __FILE__, __LINE__);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  auto bail = [&](zbus_status s) {
    std::string msg = zbus_last_error();
    cudaStreamSynchronize(st);
    zbus_nr_network_destroy(net);
    set_error(msg);
    return s;
  };
  net->N = N;
  net->slack = slack;
  std::vector<int32_t> pos_t(N, -1), pos_q(N, -1), t_bus, q_bus;
  for (int i = 0; i < N; ++i) {
    if (bus_type[i] != 2) {
      pos_t[i] = (int32_t)t_bus.size();
      t_bus.push_back(i);
    }
    if (bus_type[i] == 0) {
      pos_q[i] = (int32_t)q_bus.size();
      q_bus.push_back(i);
    }
  }
  net->nt = (int)t_bus.size();
  net->nq = (int)q_bus.size();
  // Y in CSR; B' and B'' (+ eps I); G_Q,Theta
  std::vector<int32_t> yp(N + 1, 0), yc, gp(net->nq + 1, 0), gc;
  std::vector<double2> yv;
  std::vector<double> gval;
  std::vector<std::map<int, double>> Bp(net->nt), Bpp(net->nq);
  for (int i = 0; i < N; ++i) {
    for (auto& kv : Yrows[i]) {
      yc.push_back(kv.first);
      yv.push_back(make_double2(kv.second.first, kv.second.second));
      const int j = kv.first;
      if (pos_t[i] >= 0 && pos_t[j] >= 0) Bp[pos_t[i]][pos_t[j]] += -kv.second.second;
      if (pos_q[i] >= 0 && pos_q[j] >= 0) Bpp[pos_q[i]][pos_q[j]] += -kv.second.second;
    }
    yp[i + 1] = (int32_t)yc.size();
  }
  for (int p = 0; p < net->nq; ++p) {
    const int i = q_bus[p];
    for (auto& kv : Yrows[i])
      if (pos_t[kv.first] >= 0) {
        gc.push_back(pos_t[kv.first]);
        gval.push_back(-kv.second.first);
      }
    gp[p + 1] = (int32_t)gc.size();
  }
  for (int p = 0; p < net->nt; ++p) Bp[p][p] += eps;
  for (int p = 0; p < net->nq; ++p) Bpp[p][p] += eps;
  HostFactor fp, fpp;
  std::string why;
  if (!factorise(net->nt, Bp, fp, why)) return bail(fail(ZBUS_ERR_SINGULAR, "B': " + why));
  if (net->nq > 0 && !factorise(net->nq, Bpp, fpp, why))
    return bail(fail(ZBUS_ERR_SINGULAR, "B'': " + why));
  NrDev& d = net->dev;
  d.N = N;
  d.nt = net->nt;
  d.nq = net->nq;
  d.dim = net->nt + net->nq;
  std::vector<int32_t> bt(bus_type, bus_type + N);
  std::vector<double> vs(v_set, v_set + N);
  zbus_status s = ZBUS_OK;
  int32_t *y_ptr, *y_col, *bt_d, *pt_d, *pq_d, *tb_d, *qb_d, *g_ptr, *g_col;
  double2* y_val;
  double *vs_d, *g_val;
  float2* y_val_f;
  float* g_val_f;
  std::vector<float2> yvf(yv.size());
  for (size_t e = 0; e < yv.size(); ++e) yvf[e] = make_float2((float)yv[e].x, (float)yv[e].y);
  if ((s = upload(net, &y_ptr, yp, st)) || (s = upload(net, &y_col, yc, st)) ||
      (s = upload(net, &y_val, yv, st)) || (s = upload(net, &bt_d, bt, st)) ||
      (s = upload(net, &vs_d, vs, st)) || (s = upload(net, &pt_d, pos_t, st)) ||
      (s = upload(net, &pq_d, pos_q, st)) || (s = upload(net, &tb_d, t_bus, st)) ||
      (s = upload(net, &qb_d, q_bus, st)) || (s = upload(net, &g_ptr, gp, st)) ||
      (s = upload(net, &g_col, gc, st)) || (s = upload(net, &g_val, gval, st)) ||
      (s = upload(net, &y_val_f, yvf, st)) || (s = upload(net, &g_val_f, to_float(gval), st)) ||
      (s = upload_factor(net, fp, d.Bp, st)) ||
      (net->nq > 0 && (s = upload_factor(net, fpp, d.Bpp, st))))
    return bail(s);
  d.y_ptr = y_ptr;
  d.y_col = y_col;
  d.y_val = y_val;
  d.bus_type = bt_d;
  d.v_set = vs_d;
  d.pos_t = pt_d;
  d.pos_q = pq_d;
  d.t_bus = tb_d;
  d.q_bus = qb_d;
  d.g_ptr = g_ptr;
  d.g_col = g_col;
  d.g_val = g_val;
  d.y_val_f = y_val_f;
  d.g_val_f = g_val_f;
  ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "setup copies", __FILE__, __LINE__));
  int dev = net->device;
  cudaDeviceGetAttribute(&net->sms, cudaDevAttrMultiProcessorCount, dev);
  *out = net;
  return ZBUS_OK;
}

void zbus_nr_network_destroy(zbus_nr_network net) {
  if (!net) return;
  for (void* p : net->allocs) cudaFree(p);
  cudaFree(net->scratch);
  delete net;
}

zbus_status zbus_nr_network_info(zbus_nr_network net, int32_t* n_theta, int32_t* n_q,
                                 int64_t* factor_nnz, int32_t* factor_levels) {
  set_error("");
  if (!net) return fail(ZBUS_ERR_ARG, "network is NULL");
  if (n_theta) *n_theta = net->nt;
  if (n_q) *n_q = net->nq;
  if (factor_nnz) *factor_nnz = net->dev.Bp.nnz + net->dev.Bpp.nnz;
  if (factor_levels)
    *factor_levels = net->dev.Bp.n_fl + net->dev.Bp.n_bl + net->dev.Bpp.n_fl + net->dev.Bpp.n_bl;
  return ZBUS_OK;
}

zbus_status zbus_nr_solve(zbus_nr_network net, int64_t B, const double* P, const double* Q,
                          double tol, int32_t max_iter, const zbus_nr_opts* opts, double* V_out,
                          int32_t* iters, uint8_t* converged, int32_t* gmres_iters,
                          void* cuda_stream) {
  NvtxRange nvtx_range("zbus_nr_solve");
  set_error("");
  if (!net) return fail(ZBUS_ERR_ARG, "network is NULL");
  if (B < 0 || B > INT32_MAX) return fail(ZBUS_ERR_ARG, "B out of range");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(ZBUS_ERR_ARG, "tol must be finite, >= 0");
  if (max_iter < 0) return fail(ZBUS_ERR_ARG, "max_iter must be >= 0");
  zbus_nr_opts o;
  zbus_nr_opts_default(&o);
  if (opts) o = *opts;
  if (o.gmres_restart < 1 || o.gmres_restart > NR_MAX_RESTART_LEN)
    return fail(ZBUS_ERR_ARG, "gmres_restart must be in 1 .. 60");
  if (o.gmres_max_restarts < 1) return fail(ZBUS_ERR_ARG, "gmres_max_restarts must be >= 1");
  if (!(o.gmres_tol > 0.0) || !(o.gmres_tol < 1.0))
    return fail(ZBUS_ERR_ARG, "gmres_tol must be in (0, 1)");
  if (o.precision != ZBUS_NR_FP64 && o.precision != ZBUS_NR_MIXED)
    return fail(ZBUS_ERR_ARG, "unknown NR precision");
  if (B == 0) return ZBUS_OK;
  if (!P || !Q || !V_out || !iters || !converged)
    return fail(ZBUS_ERR_ARG, "P, Q, V_out, iters and converged are required");
  int dev = -1;
  ZB_CUDA(cudaGetDevice(&dev));
  if (dev != net->device) return fail(ZBUS_ERR_ARG, "current CUDA device differs from the network's");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int m = o.gmres_restart;
  const bool mixed = o.precision == ZBUS_NR_MIXED;
  const size_t smem = smem_bytes(m, net->N, mixed);
  if (smem > 227 * 1024)
    return fail(ZBUS_ERR_ARG, "grid too large for the per-CTA shared work space");
  const void* kern = mixed ? (const void*)k_nr_solve<float> : (const void*)k_nr_solve<double>;
  if (net->smem_set[mixed] < smem) {
    ZB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    net->smem_set[mixed] = smem;
  }
  int per = 0;
  ZB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NR_THREADS, smem));
  const int64_t ctas = std::min<int64_t>(B, (int64_t)net->sms * std::max(1, per));
  const int64_t stride = scratch_doubles(net, m, mixed);
  if (net->scratch_ctas < ctas || net->scratch_stride < stride) {
    ZB_CUDA(cudaStreamSynchronize(st));
    cudaFree(net->scratch);
    net->scratch = nullptr;
    net->scratch_ctas = 0;
    ZB_CUDA(cudaMalloc((void**)&net->scratch, (size_t)ctas * stride * sizeof(double)));
    net->scratch_ctas = ctas;
    net->scratch_stride = stride;
  }
  NrDev d = net->dev;
  d.m = m;
  d.scratch = net->scratch;
  d.stride = stride;
  SolveArgs a;
  a.B = (int)B;
  a.P = P;
  a.Q = Q;
  a.tol = tol;
  a.max_iter = max_iter;
  a.eta = o.gmres_tol;
  a.max_restart = o.gmres_max_restarts;
  a.V = (double2*)V_out;
  a.iters = iters;
  a.conv = converged;
  a.gmres = gmres_iters;
  if (mixed)
    k_nr_solve<float><<<(int)ctas, NR_THREADS, smem, st>>>(d, a);
  else
    k_nr_solve<double><<<(int)ctas, NR_THREADS, smem, st>>>(d, a);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

}  // extern "C"
