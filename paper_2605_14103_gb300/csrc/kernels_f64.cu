// Plain FP64 Z-bus sweep (Sec. II-B):
//   K1  load currents i(v) of wye and delta constant-power loads,
//   K2  D = Z i with the three-real-product (3M) complex scheme, epilogue
//       v <- w + D and per-tile step partials,
//   K3  per-scenario stop test, freeze and stable compaction of the active
//       list; sets the graph's loop condition.
// Plus the run start (v^0), the whole solve of a small feeder in one launch
// (K1-K3 of every sweep in one block per scenario, the latency case) and the
// FP64 power-mismatch check.
#include <cmath>

#include "loads.cuh"
#include "zbus_internal.cuh"

namespace zbus {
namespace {

// ---------------------------------------------------------------------------
// Run start: v^0 = w (or the warm start), flags cleared, every scenario active.
// ---------------------------------------------------------------------------
// The solve's context arrives by value and is stored for the later kernels;
// this kernel itself only uses the by-value copy.
__global__ void k_init(SolveCtx* ctx, SolveCtx h, const double2* __restrict__ w, int n, int B) {
  const double2* Vi = h.V_init;
  double2* V = h.V;
  const int64_t tot = (int64_t)B * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % n);
    V[t] = Vi ? Vi[t] : w[j];
  }
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
       b += (int64_t)gridDim.x * blockDim.x) {
    h.iters[b] = 0;
    h.conv[b] = 0;
    h.list[b] = (int32_t)b;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    h.count = B;
    h.iter = 0;
    h.err = 0;
    *ctx = h;
  }
}

// ---------------------------------------------------------------------------
// K1: i(v) for the active scenarios into the 3M operands Ir, Ii, Ir + Ii,
// [slot][n_pad] each, zero in the padding.  One thread per (slot, bus).
// ---------------------------------------------------------------------------
__global__ void k_currents_f64(const SolveCtx* __restrict__ ctx, int n, int n_pad) {
  const int count = ctx->count;
  const int nbp = n_pad / 3;
  const int64_t tot = (int64_t)count * nbp;
  const int64_t plane = (int64_t)ctx->B * n_pad;
  double* Ir = ctx->Iop;
  double* Ii = Ir + plane;
  double* Is = Ii + plane;
  const double2* __restrict__ V = ctx->V;
  const double2* __restrict__ Sw = ctx->S_wye;
  const double2* __restrict__ Sd = ctx->S_del;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int slot = (int)(t / nbp);
    const int k = (int)(t % nbp);
    const int j0 = 3 * k;
    const int64_t o = (int64_t)slot * n_pad + j0;
    double2 inj[3] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    if (j0 < n && ZB_IN(ctx->list[slot], ctx->B, 0x101u)) {
      const int b = ctx->list[slot];
      const int m = min(3, n - j0);
      const int64_t e = (int64_t)b * n + j0;
      double2 v[3], sw[3], sd[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        v[p] = p < m ? V[e + p] : make_double2(1.0, 0.0);
        sw[p] = (Sw && p < m) ? Sw[e + p] : make_double2(0.0, 0.0);
        sd[p] = (Sd && p < m) ? Sd[e + p] : make_double2(0.0, 0.0);
      }
      bus_injection(v, Sw ? sw : nullptr, Sd ? sd : nullptr, m, inj);
      for (int p = m; p < 3; ++p) inj[p] = make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      Ir[o + p] = inj[p].x;
      Ii[o + p] = inj[p].y;
      Is[o + p] = inj[p].x + inj[p].y;
    }
  }
}

// ---------------------------------------------------------------------------
// K2: FP64 3M contraction over active scenarios.
//   T1 = Zr Ir, T2 = Zi Ii, T3 = (Zr + Zi)(Ir + Ii);  D = (T1 - T2, T3 - T1 - T2)
// Tile: BM scenarios x BN outputs, k in steps of BK, each thread TM x TN.
// Epilogue: v <- w + D in place (w null: v <- v + D, the defect update of
// the FP64 correction sweeps), partials (max |dv|, sum |v_new| - |v_old|) per
// (slot, N-tile), summed in a fixed order.
// ---------------------------------------------------------------------------
constexpr int TM = 2, TN = 4;
constexpr int THR_M = F64_BM / TM;   // 16
constexpr int THR_N = F64_BN / TN;   // 12
constexpr int GEMM_THREADS = THR_M * THR_N;  // 192

__global__ void __launch_bounds__(GEMM_THREADS)
k_gemm3m_f64(const SolveCtx* __restrict__ ctx, const double* __restrict__ Zr,
             const double* __restrict__ Zi, const double* __restrict__ Zs,
             const double2* __restrict__ w, int n, int n_pad) {
  __shared__ double sZ[3][F64_BK][F64_BN];
  __shared__ double sI[3][F64_BK][F64_BM];
  __shared__ double sred[2][F64_BM][THR_N];

  const int count = ctx->count;
  const int ntn = n_pad / F64_BN;
  const int mtiles = (count + F64_BM - 1) / F64_BM;
  const int total = mtiles * ntn;
  const int64_t plane = (int64_t)ctx->B * n_pad;
  const double* Ir = ctx->Iop;
  const double* Ii = Ir + plane;
  const double* Is = Ii + plane;
  double2* V = ctx->V;
  const int32_t* list = ctx->list;
  double* part = ctx->part;

  const int tid = threadIdx.x;
  const int tm = tid / THR_N;   // 0..15
  const int tn = tid % THR_N;   // 0..11

  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const int mt = tile / ntn;
    const int nt = tile % ntn;
    const int row0 = nt * F64_BN;
    const int slot0 = mt * F64_BM;
    double a1[TM][TN], a2[TM][TN], a3[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int c = 0; c < TN; ++c) a1[a][c] = a2[a][c] = a3[a][c] = 0.0;

    for (int k0 = 0; k0 < n_pad; k0 += F64_BK) {
      // Z tile: BN rows x BK, stored k-major in shared memory
      for (int e = tid; e < F64_BN * F64_BK; e += GEMM_THREADS) {
        const int r = e / F64_BK, c = e % F64_BK;
        const int64_t g = (int64_t)(row0 + r) * n_pad + k0 + c;
        sZ[0][c][r] = Zr[g];
        sZ[1][c][r] = Zi[g];
        sZ[2][c][r] = Zs[g];
      }
      for (int e = tid; e < F64_BM * F64_BK; e += GEMM_THREADS) {
        const int r = e / F64_BK, c = e % F64_BK;
        const int slot = slot0 + r;
        double x = 0.0, y = 0.0, s = 0.0;
        if (slot < count) {
          const int64_t g = (int64_t)slot * n_pad + k0 + c;
          x = Ir[g];
          y = Ii[g];
          s = Is[g];
        }
        sI[0][c][r] = x;
        sI[1][c][r] = y;
        sI[2][c][r] = s;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < F64_BK; ++kk) {
        double i1[TM], i2[TM], i3[TM], z1[TN], z2[TN], z3[TN];
#pragma unroll
        for (int a = 0; a < TM; ++a) {
          i1[a] = sI[0][kk][tm * TM + a];
          i2[a] = sI[1][kk][tm * TM + a];
          i3[a] = sI[2][kk][tm * TM + a];
        }
#pragma unroll
        for (int c = 0; c < TN; ++c) {
          z1[c] = sZ[0][kk][tn + THR_N * c];
          z2[c] = sZ[1][kk][tn + THR_N * c];
          z3[c] = sZ[2][kk][tn + THR_N * c];
        }
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int c = 0; c < TN; ++c) {
            a1[a][c] = fma(z1[c], i1[a], a1[a][c]);
            a2[a][c] = fma(z2[c], i2[a], a2[a][c]);
            a3[a][c] = fma(z3[c], i3[a], a3[a][c]);
          }
      }
      __syncthreads();
    }

    // epilogue
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      const int r = tm * TM + a;
      const int slot = slot0 + r;
      double dmax = 0.0, dsum = 0.0;
      if (slot < count && ZB_IN(list[slot], ctx->B, 0x102u)) {
        const int b = list[slot];
#pragma unroll
        for (int c = 0; c < TN; ++c) {
          const int i = row0 + tn + THR_N * c;
          if (i < n) {
            const double dr = a1[a][c] - a2[a][c];
            const double di = a3[a][c] - a1[a][c] - a2[a][c];
            const int64_t g = (int64_t)b * n + i;
            const double2 vo = V[g];
            const double2 wi = w ? w[i] : vo;
            const double2 vn = make_double2(wi.x + dr, wi.y + di);
            V[g] = vn;
            double step = hypot(vn.x - vo.x, vn.y - vo.y);
            if (step != step) step = INFINITY;
            dmax = fmax(dmax, step);
            dsum += hypot(vn.x, vn.y) - hypot(vo.x, vo.y);
          }
        }
      }
      sred[0][r][tn] = dmax;
      sred[1][r][tn] = dsum;
    }
    __syncthreads();
    if (tid < F64_BM) {
      const int slot = slot0 + tid;
      if (slot < count) {
        double dmax = 0.0, dsum = 0.0;
        for (int c = 0; c < THR_N; ++c) {
          dmax = fmax(dmax, sred[0][tid][c]);
          dsum += sred[1][tid][c];
        }
        part[((int64_t)slot * ntn + nt) * 2 + 0] = dmax;
        part[((int64_t)slot * ntn + nt) * 2 + 1] = dsum;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// K2 for small batches (at most one 32-scenario tile): one block per (slot,
// N-tile), one thread per output, so the work spreads over slots x N-tiles
// SMs instead of the single block the tiled kernel would run (the FP64 pipe
// does 2 DFMA per clock per SM, so one block of the tiled kernel takes tens
// of microseconds even at 36 unknowns).  Every output's three products are
// summed over k in the tiled kernel's order (one sequential FMA chain each)
// and the tile partials are grouped like its block reduction (per thread
// column tn the outputs tn, tn + 12, tn + 24, tn + 36, then tn = 0..11), so
// the results are bitwise those of k_gemm3m_f64.
// ---------------------------------------------------------------------------
constexpr int SMALL_THREADS = 64;

__global__ void __launch_bounds__(SMALL_THREADS)
k_gemm3m_f64_small(const SolveCtx* __restrict__ ctx, const double* __restrict__ Zr,
                   const double* __restrict__ Zi, const double* __restrict__ Zs,
                   const double2* __restrict__ w, int n, int n_pad) {
  __shared__ double sdm[F64_BN], sds[F64_BN];
  __shared__ int sok[F64_BN];
  const int count = ctx->count;
  const int slot = blockIdx.x, nt = blockIdx.y;
  if (slot >= count) return;   // whole block
  const int ntn = n_pad / F64_BN;
  const int64_t plane = (int64_t)ctx->B * n_pad;
  const double* __restrict__ Ir = ctx->Iop + (int64_t)slot * n_pad;
  const double* __restrict__ Ii = Ir + plane;
  const double* __restrict__ Is = Ii + plane;
  const int t = threadIdx.x;
  if (t < F64_BN) {
    const int i = nt * F64_BN + t;
    const double* zr = Zr + (int64_t)i * n_pad;
    const double* zi = Zi + (int64_t)i * n_pad;
    const double* zs = Zs + (int64_t)i * n_pad;
    double a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int k = 0; k < n_pad; ++k) {
      a1 = fma(zr[k], Ir[k], a1);
      a2 = fma(zi[k], Ii[k], a2);
      a3 = fma(zs[k], Is[k], a3);
    }
    int ok = 0;
    double dm = 0.0, ds = 0.0;
    if (i < n && ZB_IN(ctx->list[slot], ctx->B, 0x105u)) {
      const int b = ctx->list[slot];
      const double dr = a1 - a2;
      const double di = a3 - a1 - a2;
      const int64_t g = (int64_t)b * n + i;
      double2* V = ctx->V;
      const double2 vo = V[g];
      const double2 wi = w ? w[i] : vo;
      const double2 vn = make_double2(wi.x + dr, wi.y + di);
      V[g] = vn;
      double step = hypot(vn.x - vo.x, vn.y - vo.y);
      if (step != step) step = INFINITY;
      dm = step;
      ds = hypot(vn.x, vn.y) - hypot(vo.x, vo.y);
      ok = 1;
    }
    sdm[t] = dm;
    sds[t] = ds;
    sok[t] = ok;
  }
  __syncthreads();
  if (t == 0) {
    double dmax = 0.0, dsum = 0.0;
    for (int tn = 0; tn < F64_BN / 4; ++tn) {
      double m = 0.0, u = 0.0;
      for (int c = 0; c < 4; ++c) {
        const int o = tn + (F64_BN / 4) * c;
        if (sok[o]) {
          m = fmax(m, sdm[o]);
          u += sds[o];
        }
      }
      dmax = fmax(dmax, m);
      dsum += u;
    }
    ctx->part[((int64_t)slot * ntn + nt) * 2 + 0] = dmax;
    ctx->part[((int64_t)slot * ntn + nt) * 2 + 1] = dsum;
  }
}

// ---------------------------------------------------------------------------
// The whole solve of one small feeder in one launch, for the latency case
// (n_pad <= FUSED_MAX_NPAD unknowns, at most one 32-scenario tile): one block
// per scenario keeps v and the 3M operands in shared memory and runs every
// sweep (K1, K2, K3) itself, so a solve costs one launch instead of four
// kernel nodes per sweep.  Every value is formed with the arithmetic of the
// sweep kernels: the load currents of bus_injection (a thread per unknown
// draws its wye current and its bus's delta branch, then adds the branches
// into its phase as bus_injection does), each output's three products summed
// over k in sequence, the step partials grouped as in k_gemm3m_f64_small and
// reduced over the tiles as in k_decide (maxima in any order, which is exact;
// the sums of the sum-of-magnitudes rule in the same order), so the results
// are bitwise those of the sweep-per-launch path.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(FUSED_THREADS)
k_solve_fused_f64(const double* __restrict__ Zr, const double* __restrict__ Zi,
                  const double* __restrict__ Zs, const double2* __restrict__ w,
                  const double2* __restrict__ V_init, const double2* __restrict__ Sw,
                  const double2* __restrict__ Sd, int n, int n_pad, double tol, int max_iter,
                  int rule, double2* __restrict__ V, int32_t* __restrict__ iters,
                  uint8_t* __restrict__ conv) {
  static_assert(FUSED_THREADS >= FUSED_MAX_NPAD && FUSED_THREADS == 128,
                "one thread per padded unknown; four warps share the outputs");
  __shared__ double2 sv[FUSED_MAX_NPAD];
  __shared__ double2 sdw[FUSED_MAX_NPAD], sib[FUSED_MAX_NPAD];   // wye draws, delta branches
  __shared__ double sIr[FUSED_MAX_NPAD], sIi[FUSED_MAX_NPAD], sIs[FUSED_MAX_NPAD];
  __shared__ double sds[FUSED_MAX_NPAD], su[FUSED_MAX_NPAD / 4];
  __shared__ double swm[FUSED_THREADS / 32];
  __shared__ int sok[FUSED_MAX_NPAD];
  __shared__ int sdone;
  const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int64_t row = (int64_t)b * n;
  const int ntn = n_pad / F64_BN;
  const bool summag = rule == ZBUS_CONV_SUMMAG;
  if (t < n) sv[t] = V_init ? V_init[row + t] : w[t];
  // this thread's unknown: bus j0 / 3, phase p, m valid phases in the bus
  const int j0 = 3 * (t / 3), p = t % 3, m = min(3, n - j0);
  const bool own = t < n;
  const bool delta = Sd != nullptr && m == 3 && own;
  const double2 swj = (Sw && own) ? Sw[row + t] : make_double2(0.0, 0.0);
  const double2 sdj = delta ? Sd[row + t] : make_double2(0.0, 0.0);
  __syncthreads();
  for (int it = 1;; ++it) {
    // K1a: the wye current of this unknown and the delta branch p of its bus
    // (branch p joins phases p and p + 1), as load_draw inside bus_injection
    if (t < n_pad) {
      double2 dw = make_double2(0.0, 0.0), ib = make_double2(0.0, 0.0);
      if (own) {
        if (Sw) dw = load_draw(swj, sv[t]);
        if (delta) {
          const double2 va = sv[t], vb = sv[j0 + (p == 2 ? 0 : p + 1)];
          ib = load_draw(sdj, make_double2(va.x - vb.x, va.y - vb.y));
        }
      }
      sdw[t] = dw;
      sib[t] = ib;
    }
    __syncthreads();
    // K1b: phase p draws branch p and returns branch p - 1; injection = -drawn
    if (t < n_pad) {
      double2 inj = make_double2(0.0, 0.0);
      if (own) {
        double2 d = sdw[t];
        if (delta) {
          const double2 ib = sib[t], iw = sib[j0 + (p == 0 ? 2 : p - 1)];
          d.x += ib.x - iw.x;
          d.y += ib.y - iw.y;
        }
        inj = make_double2(-d.x, -d.y);
      }
      sIr[t] = inj.x;
      sIi[t] = inj.y;
      sIs[t] = inj.x + inj.y;
    }
    __syncthreads();
    // K2: one output per thread, v <- w + D in place (the currents are read
    // from shared memory only).  The outputs are dealt to the four warps in
    // equal parts (n_pad / 4 lanes each), so each SM sub-partition's FP64
    // pipe carries a quarter of the products.
    double dm = 0.0;
    const int per = n_pad / 4;
    const int o = lane < per ? wid * per + lane : -1;
    if (o >= 0) {
      const bool out_own = o < n;
      const double* zr = Zr + (int64_t)o * n_pad;
      const double* zi = Zi + (int64_t)o * n_pad;
      const double* zs = Zs + (int64_t)o * n_pad;
      double a1 = 0.0, a2 = 0.0, a3 = 0.0;
      for (int k = 0; k < n_pad; ++k) {
        a1 = fma(zr[k], sIr[k], a1);
        a2 = fma(zi[k], sIi[k], a2);
        a3 = fma(zs[k], sIs[k], a3);
      }
      int ok = 0;
      double ds = 0.0;
      if (out_own) {
        const double dr = a1 - a2;
        const double di = a3 - a1 - a2;
        const double2 vo = sv[o];
        const double2 wi = w[o];
        const double2 vn = make_double2(wi.x + dr, wi.y + di);
        sv[o] = vn;
        double step = hypot(vn.x - vo.x, vn.y - vo.y);
        if (step != step) step = INFINITY;
        dm = step;
        ds = hypot(vn.x, vn.y) - hypot(vo.x, vo.y);
        ok = 1;
      }
      sds[o] = ds;
      sok[o] = ok;
    }
    // K3: the largest step (maxima are exact in any order; every step is >= 0)
    for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (lane == 0) swm[wid] = dm;
    __syncthreads();
    // the sum-of-magnitudes rule: per tile and thread column tn the outputs
    // tn, tn + 12, tn + 24, tn + 36 in order, then tn = 0..11, then the tiles
    if (summag && t < ntn * (F64_BN / 4)) {
      const int nt = t / (F64_BN / 4), tn = t % (F64_BN / 4);
      double u = 0.0;
      for (int c = 0; c < 4; ++c) {
        const int o = nt * F64_BN + tn + (F64_BN / 4) * c;
        if (sok[o]) u += sds[o];
      }
      su[t] = u;
    }
    __syncthreads();
    if (t == 0) {
      double dmax = 0.0;
      for (int x = 0; x < FUSED_THREADS / 32; ++x) dmax = fmax(dmax, swm[x]);
      double dsum = 0.0;
      if (summag)
        for (int nt = 0; nt < ntn; ++nt) {
          double tu = 0.0;
          for (int tn = 0; tn < F64_BN / 4; ++tn) tu += su[nt * (F64_BN / 4) + tn];
          dsum += tu;
        }
      const double delta_v = summag ? fabs(dsum) : dmax;
      int done = 1;
      if (!isfinite(delta_v)) {
        conv[b] = 0;
      } else if (delta_v <= tol) {
        conv[b] = 1;
      } else if (it < max_iter) {
        done = 0;
      } else {
        conv[b] = 0;
      }
      if (done) iters[b] = it;
      sdone = done;
    }
    __syncthreads();
    if (sdone) break;
    __syncthreads();
  }
  if (t < n) V[row + t] = sv[t];
}

// ---------------------------------------------------------------------------
// K3a: stop test per active scenario (many blocks): reduce the per-tile
// partials in a fixed order, record iters / flags, mark the slots to keep.
// ---------------------------------------------------------------------------
__global__ void k_decide(SolveCtx* __restrict__ ctx) {
  const int count = ctx->count;
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= count) return;
  const int it = ctx->iter + 1;
  const int ntn = ctx->ntn;
  const int b = ctx->list[slot];
  if (!ZB_IN(b, ctx->B, 0x103u)) return;
  const double* part = ctx->part + (int64_t)slot * ntn * 2;
  double dmax = 0.0, dsum = 0.0;
  for (int t = 0; t < ntn; ++t) {
    dmax = fmax(dmax, part[2 * t]);
    dsum += part[2 * t + 1];
  }
  const double delta = ctx->rule == ZBUS_CONV_SUMMAG ? fabs(dsum) : dmax;
  ctx->iters[b] = it;
  int keep = 0;
  if (!isfinite(delta)) {
    ctx->conv[b] = 0;
  } else if (delta <= ctx->tol) {
    ctx->conv[b] = 1;
  } else if (it < ctx->max_iter) {
    keep = 1;
  }
  ctx->keep[slot] = (uint8_t)keep;
}

// ---------------------------------------------------------------------------
// K3b: stable in-place compaction of the active list by the keep marks, one
// block of 1024 threads; advances the sweep counter and sets the loop
// condition of the graph.
// ---------------------------------------------------------------------------
constexpr int CONV_THREADS = 1024;

__global__ void __launch_bounds__(CONV_THREADS)
k_compact(SolveCtx* ctx, cudaGraphConditionalHandle h, int use_handle) {
  __shared__ int swarp[CONV_THREADS / 32];
  __shared__ int sbase, stotal;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int count = ctx->count;
  const int it = ctx->iter + 1;
  int32_t* list = ctx->list;
  const uint8_t* keepv = ctx->keep;
  if (tid == 0) {
    sbase = 0;
    if (ctx->hist && it - 1 < ctx->hist_n) ctx->hist[it - 1] = count;
  }
  __syncthreads();
  for (int base = 0; base < count; base += CONV_THREADS) {
    const int slot = base + tid;
    int keep = 0, b = -1;
    if (slot < count) {
      keep = keepv[slot];
      b = list[slot];
    }
    // block-wide exclusive scan of keep, then an in-place stable write: every
    // read of this chunk happened before the first barrier and every write
    // lands at or before its writer's own slot.
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
    if (keep) list[sbase + swarp[wid] + wpre] = b;
    __syncthreads();
    if (tid == 0) sbase += stotal;
    __syncthreads();
  }
  if (tid == 0) {
    ctx->count = sbase;
    ctx->iter = it;
    if (use_handle) cudaGraphSetConditional(h, sbase > 0 ? 1u : 0u);
  }
}

// ---------------------------------------------------------------------------
// FP64 power mismatch with the sparse admittance matrix:
//   max_j | v_j conj( sum_c Y_LL[j][c] v_c + ys_j - i_j(v) ) |
// One block per scenario, one thread per bus.
// ---------------------------------------------------------------------------
__global__ void k_mismatch(const double2* __restrict__ V, const double2* __restrict__ Sw,
                           const double2* __restrict__ Sd, const int32_t* __restrict__ ptr,
                           const int32_t* __restrict__ col, const double2* __restrict__ val,
                           const double2* __restrict__ ys, int n, double* out) {
  __shared__ double sm[32];
  const int b = blockIdx.x;
  const double2* v = V + (int64_t)b * n;
  double worst = 0.0;
  const int nb = (n + 2) / 3;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    const int j0 = 3 * k;
    const int m = min(3, n - j0);
    double2 vv[3], sw[3], sd[3], inj[3];
    for (int p = 0; p < 3; ++p) {
      vv[p] = p < m ? v[j0 + p] : make_double2(1.0, 0.0);
      sw[p] = (Sw && p < m) ? Sw[(int64_t)b * n + j0 + p] : make_double2(0.0, 0.0);
      sd[p] = (Sd && p < m) ? Sd[(int64_t)b * n + j0 + p] : make_double2(0.0, 0.0);
    }
    bus_injection(vv, Sw ? sw : nullptr, Sd ? sd : nullptr, m, inj);
    for (int p = 0; p < m; ++p) {
      const int j = j0 + p;
      double2 acc = ys[j];
      for (int t = ptr[j]; t < ptr[j + 1]; ++t) {
        if (!ZB_IN(col[t], n, 0x104u)) continue;
        const double2 y = val[t], x = v[col[t]];
        acc.x += y.x * x.x - y.y * x.y;
        acc.y += y.x * x.y + y.y * x.x;
      }
      const double rx = acc.x - inj[p].x, ry = acc.y - inj[p].y;
      // |v conj(r)| = |v| |r|
      double e = hypot(vv[p].x, vv[p].y) * hypot(rx, ry);
      if (e != e) e = INFINITY;
      worst = fmax(worst, e);
    }
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (threadIdx.x == 0) out[b] = x;
  }
}

// ---------------------------------------------------------------------------
// FP64 rate probe: eight independent DFMA chains per thread (no memory
// traffic in the loop), the roofline denominator of the FP64 kernels.  The
// values stay bounded (x <- x a + c with a < 1) and are summed into out only
// when the sum is negative, which it never is, so the chains are kept.
// ---------------------------------------------------------------------------
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(256) k_probe_dfma(double* out, int iters, double a, double c) {
  double x[PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = fma(x[i], a, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) s += x[i];
  if (s < 0.0) out[blockIdx.x] = s;
}

}  // namespace

zbus_status probe_fp64_rate(double* tflops, float* ms_out, cudaStream_t st) {
  int dev = 0, sms = 0;
  ZB_CUDA(cudaGetDevice(&dev));
  ZB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 8 * sms, threads = 256;
  double* out = nullptr;   // written only on a negative sum (never)
  ZB_CUDA(cudaMallocAsync((void**)&out, (size_t)blocks * sizeof(double), st));
  cudaEvent_t e0, e1;
  ZB_CUDA(cudaEventCreate(&e0));
  ZB_CUDA(cudaEventCreate(&e1));
  k_probe_dfma<<<blocks, threads, 0, st>>>(out, 256, 0.999999, 1e-7);   // warm-up
  const int iters = 16384;
  ZB_CUDA(cudaEventRecord(e0, st));
  k_probe_dfma<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);
  ZB_CUDA(cudaEventRecord(e1, st));
  cudaError_t ce = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "FP64 probe", __FILE__, __LINE__);
  ZB_CUDA(cudaStreamSynchronize(st));
  const double flops = 2.0 * PROBE_CHAINS * (double)iters * blocks * threads;
  if (tflops) *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
  if (ms_out) *ms_out = ms;
  return ZBUS_OK;
}

void launch_init(SolveCtx* ctx, const SolveCtx& h, const double2* w, int n, int B,
                 cudaStream_t st) {
  int64_t tot = (int64_t)B * n;
  int grid = (int)std::min<int64_t>(4096, std::max<int64_t>(1, (tot + 255) / 256));
  k_init<<<grid, 256, 0, st>>>(ctx, h, w, n, B);
}

void launch_currents_f64(SolveCtx* ctx, int n, int n_pad, int B, cudaStream_t st) {
  int64_t tot = (int64_t)B * (n_pad / 3);
  int grid = (int)std::min<int64_t>(152 * 16, std::max<int64_t>(1, (tot + 255) / 256));
  k_currents_f64<<<grid, 256, 0, st>>>(ctx, n, n_pad);
}

// Grid of the FP64 contraction for batches of up to B scenarios: the number
// of blocks of the tiled kernel, or -B for batches of one tile at most (the
// per-(slot, N-tile) kernel).
int gemm_f64_grid(int B, int n_pad) {
  if (B <= F64_BM) return -std::max(1, B);
  const int tiles = ((B + F64_BM - 1) / F64_BM) * (n_pad / F64_BN);
  return std::max(1, std::min(tiles, 152 * 4));
}

void launch_gemm_f64(SolveCtx* ctx, const double* Zr, const double* Zi, const double* Zs,
                     const double2* w, int n, int n_pad, int grid, cudaStream_t st) {
  if (grid < 0)
    k_gemm3m_f64_small<<<dim3(-grid, n_pad / F64_BN), SMALL_THREADS, 0, st>>>(ctx, Zr, Zi, Zs, w,
                                                                             n, n_pad);
  else
    k_gemm3m_f64<<<grid, GEMM_THREADS, 0, st>>>(ctx, Zr, Zi, Zs, w, n, n_pad);
}

void launch_solve_fused_f64(const double* Zr, const double* Zi, const double* Zs,
                            const double2* w, const double2* V_init, const double2* S_wye,
                            const double2* S_del, int n, int n_pad, int B, double tol,
                            int max_iter, int rule, double2* V, int32_t* iters, uint8_t* conv,
                            cudaStream_t st) {
  k_solve_fused_f64<<<B, FUSED_THREADS, 0, st>>>(Zr, Zi, Zs, w, V_init, S_wye, S_del, n, n_pad,
                                                  tol, max_iter, rule, V, iters, conv);
}

void launch_converge(SolveCtx* ctx, int B, cudaGraphConditionalHandle h, bool use_handle,
                     cudaStream_t st) {
  k_decide<<<(B + 255) / 256, 256, 0, st>>>(ctx);
  k_compact<<<1, CONV_THREADS, 0, st>>>(ctx, h, use_handle ? 1 : 0);
}

void launch_mismatch(const double2* V, const double2* S_wye, const double2* S_del,
                     const int32_t* ptr, const int32_t* col, const double2* val,
                     const double2* ys, int n, int B, double* out, cudaStream_t st) {
  if (B <= 0) return;
  k_mismatch<<<B, 256, 0, st>>>(V, S_wye, S_del, ptr, col, val, ys, n, out);
}

}  // namespace zbus

namespace zbus {
ZB_CHECK_WORD_ACCESSOR(check_word_f64)
}  // namespace zbus
