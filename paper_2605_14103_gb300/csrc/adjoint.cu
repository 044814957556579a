// Load gradient of the converged Z-bus fixed point (the differentiable solve).
//
// The paper motivates the solver as a component of GPU learning pipelines
// (Sec. I, conclusion).  A loss L(v*) of the solution v* = Z i(v*, S) + w
// (Sec. II-B) is differentiated with respect to the loads through the
// fixed-point condition instead of through the iterations.  The load current
// depends on conj(v) and conj(S) only,
//     di = A conj(dv) + D conj(dS),
// (wye slot j: A_jj = conj(S_j / v_j^2), D_jj = -1 / conj(v_j); delta branch
// x -> y: c = conj(S / u^2), u = v_x - v_y, adds c (x,x), c (y,y), -c (x,y),
// -c (y,x) to A and -1 / conj(u), +1 / conj(u) at rows x, y of its column of
// D).  With G = dL/dRe v + j dL/dIm v, the adjoint of the real-linear map
// dv -> Z A conj(dv) gives
//     lambda = G + A^T mu,   mu = Z^T conj(lambda),
//     dL/dS  = D^T mu        (same complex convention),
// and lambda is reached by iterating those two lines from mu = 0: the
// iteration contracts at the rate of the forward map's linearisation.  Each
// adjoint sweep is the forward FP64 sweep with the roles of its kernels
// changed: the per-bus load kernel forms conj(lambda) from mu (K1'), the 3M
// contraction applies Z^T (its epilogue adds a zero no-load term), and the
// stop test and compaction are the forward ones.  G is scaled per scenario to
// max |G_b| = 1 so that tol is relative to the size of each scenario's loss
// gradient.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "zbus_internal.cuh"

namespace zbus {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// acc + a b with four FMAs
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}

// conj(S / u^2) = conj(S) u^2 / |u|^4; zero for an absent load.
__device__ __forceinline__ double2 load_slope(double2 S, double2 u) {
  if (S.x == 0.0 && S.y == 0.0) return make_double2(0.0, 0.0);
  const double q = u.x * u.x + u.y * u.y;
  const double2 u2 = cmul(u, u);
  const double2 r = cmul(cconj(S), u2);
  const double inv = 1.0 / (q * q);
  return make_double2(r.x * inv, r.y * inv);
}

// x / conj(u) = x u / |u|^2; zero where u = 0 (an absent phase of a padded
// partial-phase bus).
__device__ __forceinline__ double2 div_conj(double2 x, double2 u) {
  const double q = u.x * u.x + u.y * u.y;
  if (q == 0.0) return make_double2(0.0, 0.0);
  const double2 r = cmul(x, u);
  return make_double2(r.x / q, r.y / q);
}

// Transpose of the three n_pad x n_pad 3M arrays of Z (blockIdx.z selects one).
__global__ void k_transpose_3m(const double* __restrict__ Zr, const double* __restrict__ Zi,
                               const double* __restrict__ Zs, double* __restrict__ ZrT,
                               double* __restrict__ ZiT, double* __restrict__ ZsT, int n_pad) {
  __shared__ double tile[32][33];
  const double* src = blockIdx.z == 0 ? Zr : (blockIdx.z == 1 ? Zi : Zs);
  double* dst = blockIdx.z == 0 ? ZrT : (blockIdx.z == 1 ? ZiT : ZsT);
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int row = y0 + r, col = x0 + threadIdx.x;
    if (row < n_pad && col < n_pad) tile[r][threadIdx.x] = src[(int64_t)row * n_pad + col];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int row = x0 + r, col = y0 + threadIdx.x;
    if (row < n_pad && col < n_pad) dst[(int64_t)row * n_pad + col] = tile[threadIdx.x][r];
  }
}

// Per-scenario scale s_b = max_j |G_bj| (1 where G_b is zero).  One warp per
// scenario.
__global__ void k_adj_scale(const double2* __restrict__ G, int n, int B, double* __restrict__ s) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < B; b += warps) {
    const double2* g = G + (int64_t)b * n;
    double m = 0.0;
    for (int j = lane; j < n; j += 32) {
      const double a = hypot(g[j].x, g[j].y);
      m = (a > m || a != a) ? a : m;   // a NaN entry propagates
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, m, o);
      m = (y > m || y != y) ? y : m;
    }
    if (lane == 0) s[b] = m == 0.0 ? 1.0 : m;
  }
}

// Run start of the adjoint sweeps: mu = 0, counters cleared, every scenario
// active; stores the context for the later kernels.
__global__ void k_adj_init(SolveCtx* ctx, SolveCtx h, int n, int B) {
  const int64_t tot = (int64_t)B * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x)
    h.V[t] = make_double2(0.0, 0.0);
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

// K1': conj(lambda), lambda = G / s + A^T mu, for the active scenarios into the
// 3M operands [slot][n_pad] (zero in the padding).  One thread per (slot, bus).
__global__ void k_adj_rhs(const SolveCtx* __restrict__ ctx, int n, int n_pad) {
  const int count = ctx->count;
  const int nbp = n_pad / 3;
  const int64_t tot = (int64_t)count * nbp;
  const int64_t plane = (int64_t)ctx->B * n_pad;
  double* Ir = ctx->Iop;
  double* Ii = Ir + plane;
  double* Is = Ii + plane;
  const double2* __restrict__ mu = ctx->V;
  const double2* __restrict__ V = ctx->Vf;
  const double2* __restrict__ G = ctx->G;
  const double2* __restrict__ Sw = ctx->S_wye;
  const double2* __restrict__ Sd = ctx->S_del;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int slot = (int)(t / nbp);
    const int k = (int)(t % nbp);
    const int j0 = 3 * k;
    const int64_t o = (int64_t)slot * n_pad + j0;
    double2 lam[3] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    if (j0 < n && ZB_IN(ctx->list[slot], ctx->B, 0x301u)) {
      const int b = ctx->list[slot];
      const int m = min(3, n - j0);
      const int64_t e = (int64_t)b * n + j0;
      const double inv_s = 1.0 / ctx->gscale[b];
      double2 v[3], u[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        v[p] = p < m ? V[e + p] : make_double2(1.0, 0.0);
        u[p] = p < m ? mu[e + p] : make_double2(0.0, 0.0);
        const double2 g = p < m ? G[e + p] : make_double2(0.0, 0.0);
        lam[p] = make_double2(g.x * inv_s, g.y * inv_s);
        if (Sw && p < m) {
          const double2 a = load_slope(Sw[e + p], v[p]);
          const double2 d = cmul(a, u[p]);
          lam[p].x += d.x;
          lam[p].y += d.y;
        }
      }
      if (Sd && m == 3) {
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const int y = x == 2 ? 0 : x + 1;
          const double2 c = load_slope(Sd[e + x], csub(v[x], v[y]));
          const double2 d = cmul(c, csub(u[x], u[y]));
          lam[x].x += d.x;
          lam[x].y += d.y;
          lam[y].x -= d.x;
          lam[y].y -= d.y;
        }
      }
#pragma unroll
      for (int p = 0; p < 3; ++p)
        if (p >= m) lam[p] = make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {   // the operand is conj(lambda)
      Ir[o + p] = lam[p].x;
      Ii[o + p] = -lam[p].y;
      Is[o + p] = lam[p].x - lam[p].y;
    }
  }
}

// dL/dS = s D^T mu for every scenario: wye slot j -s mu_j / conj(v_j); delta
// slot x (branch x -> y) s (mu_y - mu_x) / conj(v_x - v_y), zero on a bus the
// network ends inside.  One thread per (scenario, bus).
__global__ void k_adj_out(const double2* __restrict__ mu, const double2* __restrict__ V,
                          const double* __restrict__ gscale, int n, int B,
                          double2* __restrict__ Hw, double2* __restrict__ Hd) {
  const int nb = (n + 2) / 3;
  const int64_t tot = (int64_t)B * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / nb);
    const int j0 = 3 * (int)(t % nb);
    const int m = min(3, n - j0);
    const int64_t e = (int64_t)b * n + j0;
    const double s = gscale[b];
    double2 v[3], u[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      v[p] = p < m ? V[e + p] : make_double2(1.0, 0.0);
      u[p] = p < m ? mu[e + p] : make_double2(0.0, 0.0);
    }
    if (Hw) {
#pragma unroll
      for (int p = 0; p < 3; ++p)
        if (p < m) {
          const double2 h = div_conj(u[p], v[p]);
          Hw[e + p] = make_double2(-s * h.x, -s * h.y);
        }
    }
    if (Hd) {
      if (m == 3) {
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const int y = x == 2 ? 0 : x + 1;
          const double2 h = div_conj(csub(u[y], u[x]), csub(v[x], v[y]));
          Hd[e + x] = make_double2(s * h.x, s * h.y);
        }
      } else {
#pragma unroll
        for (int p = 0; p < 3; ++p)
          if (p < m) Hd[e + p] = make_double2(0.0, 0.0);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Tree form of the adjoint (radial networks): the defect iteration
//     rho = conj(G / s + A^T mu) - Y_LL^T mu,     mu <- mu + T^T rho,
// T^T the backward / forward sweep of the transposed series network (subtree
// sums of rho, then path sums of z_c^T times them), FP64 throughout.  Its
// fixed point is that of the dense adjoint (rho = 0 <=> Y^T mu =
// conj(lambda)); without shunts T^T = Z^T and each sweep equals a dense
// adjoint sweep.  Y_LL^T mu in branch form: with reciprocal branches
// (Y_ba = Y_ab, which the radial detection checks),
//     (Y_LL^T mu)_a = sum_b Y_ab^T (mu_b - mu_a) - Y_as^T mu_a + Sh_a^T mu_a.
// One CTA per scenario runs every sweep (block barriers per tree level).
// Each tree branch's product is formed once: with J_c = Y_cp^T (mu_p - mu_c)
// for bus c and its parent p (mu = 0 at the slack), the branch contributes
// J_c at c and -J_c at p, so the backward sweep forms the subtree sums as
//     S_c = P_c + sum over children k of (S_k + J_k),
//     P_c = conj(lambda_c) - J_c - (shunt terms of c).
// ---------------------------------------------------------------------------
constexpr int AT_THREADS = 128;
constexpr int AT_WARPS = AT_THREADS / 32;

struct AdjTree {
  int n, nb, depth, B, max_iter;
  int64_t nblk;           // branch-form blocks (checked build)
  int onchip;             // mu and r in shared memory (else in the scratch slice)
  double tol;
  const int4* node;       // per breadth-first position: bus, parent position, children range
  const int32_t* lvl;     // [depth + 1]
  const uint8_t* mask;    // phases of each position's parent line
  const double2* z;       // [nb][9] z_c of each position's parent line (FP64)
  const int32_t* pblk;    // [nb] branch-form block of each position's parent line
  const int32_t* bptr;    // branch-form blocks per bus
  const int32_t* bcol;
  const double2* bval;
  const double2* Sw;
  const double2* Sd;
  const double2* V;
  const double2* G;
  double2* Hw;
  double2* Hd;
  int32_t* iters;
  uint8_t* conv;
  double2* scratch;       // per CTA: mu, r, wye slopes, delta slopes, J (5 n)
  int64_t stride;
};

__device__ double at_block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(0xffffffffu, v, o);
    v = (y > v || y != y) ? y : v;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
#pragma unroll
  for (int k = 0; k < AT_WARPS; ++k) m = (red[k] > m || red[k] != red[k]) ? red[k] : m;
  return m;
}

__global__ void __launch_bounds__(AT_THREADS) k_adj_tree(AdjTree a) {
  __shared__ double red[AT_WARPS];
  extern __shared__ double2 at_smem[];   // mu and r when they fit (a.onchip)
  const int t = threadIdx.x;
  const int n = a.n, nb = a.nb;
  double2* g = a.scratch + (int64_t)blockIdx.x * a.stride;
  double2* mu = a.onchip ? at_smem : g;
  double2* r = a.onchip ? at_smem + n : g + n;
  double2* aw = g + 2 * n;
  double2* cd = g + 3 * n;
  double2* jb = g + 4 * n;   // J of each bus's parent branch
  for (int b = blockIdx.x; b < a.B; b += gridDim.x) {
    const int64_t off = (int64_t)b * n;
    const double2* V = a.V + off;
    const double2* G = a.G + off;
    // scale of G, load slopes at V, mu = 0
    double gm = 0.0;
    for (int j = t; j < n; j += AT_THREADS) {
      const double x = hypot(G[j].x, G[j].y);
      gm = (x > gm || x != x) ? x : gm;
    }
    gm = at_block_max(gm, red);
    const double s = gm == 0.0 ? 1.0 : gm;
    const double inv_s = 1.0 / s;
    for (int c = t; c < nb; c += AT_THREADS) {
      const int j0 = 3 * c;
      double2 v[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        v[p] = V[j0 + p];
        aw[j0 + p] = a.Sw ? load_slope(a.Sw[off + j0 + p], v[p]) : make_double2(0.0, 0.0);
        mu[j0 + p] = make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const int y = x == 2 ? 0 : x + 1;
        cd[j0 + x] = a.Sd ? load_slope(a.Sd[off + j0 + x], csub(v[x], v[y]))
                          : make_double2(0.0, 0.0);
      }
    }
    __syncthreads();
    int it = 0, ok = 0;
    for (int k = 1; k <= a.max_iter; ++k) {
      // P_c = conj(G / s + A^T mu)_c - J_c - (shunt terms), per breadth-first
      // position (bus c, parent p)
      for (int i = t; i < nb; i += AT_THREADS) {
        const int4 nd = a.node[i];
        if (!ZB_IN(nd.x, nb, 0x302u) || !ZB_IN(nd.y + 1, nb + 1, 0x303u) ||
            !ZB_IN(a.pblk[i], a.nblk, 0x304u))
          continue;
        const int c = nd.x;
        const int j0 = 3 * c;
        double2 u[3], lam[3], yt[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          u[q] = mu[j0 + q];
          const double2 gq = G[j0 + q];
          lam[q] = cfma(aw[j0 + q], u[q], make_double2(gq.x * inv_s, gq.y * inv_s));
          yt[q] = make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const int y = x == 2 ? 0 : x + 1;
          const double2 d = cmul(cd[j0 + x], csub(u[x], u[y]));
          lam[x].x += d.x;
          lam[x].y += d.y;
          lam[y].x -= d.x;
          lam[y].y -= d.y;
        }
        {   // J_c = Y_cp^T (mu_p - mu_c)
          const double2* Yb = a.bval + (int64_t)a.pblk[i] * 9;
          double2 w[3];
#pragma unroll
          for (int q = 0; q < 3; ++q)
            w[q] = nd.y >= 0 ? csub(mu[3 * a.node[nd.y].x + q], u[q])
                             : make_double2(-u[q].x, -u[q].y);
#pragma unroll
          for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) yt[p] = cfma(Yb[3 * q + p], w[q], yt[p]);
#pragma unroll
          for (int p = 0; p < 3; ++p) jb[j0 + p] = yt[p];
        }
        for (int e = a.bptr[c]; e < a.bptr[c + 1]; ++e) {   // shunts: Sh_c^T mu_c
          if (a.bcol[e] != -2) continue;
          const double2* Yb = a.bval + (int64_t)e * 9;
#pragma unroll
          for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) yt[p] = cfma(Yb[3 * q + p], u[q], yt[p]);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) r[j0 + p] = make_double2(lam[p].x - yt[p].x, -lam[p].y - yt[p].y);
      }
      __syncthreads();
      // backward: S_c = P_c + sum over children of (S_k + J_k), deepest first
      for (int L = a.depth - 2; L >= 0; --L) {
        for (int i = a.lvl[L] + t; i < a.lvl[L + 1]; i += AT_THREADS) {
          const int4 nd = a.node[i];
          if (nd.z == nd.w || !ZB_IN(nd.x, nb, 0x307u)) continue;
          double2* own = r + 3 * nd.x;
          double2 acc[3] = {own[0], own[1], own[2]};
          for (int ch = nd.z; ch < nd.w; ++ch) {
            if (!ZB_IN(ch, nb, 0x305u) || !ZB_IN(a.node[ch].x, nb, 0x306u)) continue;
            const int kb = 3 * a.node[ch].x;
            const int cm = a.mask[ch];   // a phase the child's line lacks stays below
#pragma unroll
            for (int p = 0; p < 3; ++p)
              if ((cm >> p) & 1) {
                acc[p].x += r[kb + p].x + jb[kb + p].x;
                acc[p].y += r[kb + p].y + jb[kb + p].y;
              }
          }
#pragma unroll
          for (int p = 0; p < 3; ++p) own[p] = acc[p];
        }
        __syncthreads();
      }
      // forward: X_c = X_parent + z_c^T S_c on the phases of c's line, in place
      for (int L = 0; L < a.depth; ++L) {
        for (int i = a.lvl[L] + t; i < a.lvl[L + 1]; i += AT_THREADS) {
          const int4 nd = a.node[i];
          if (!ZB_IN(nd.x, nb, 0x308u) || !ZB_IN(nd.y + 1, nb + 1, 0x309u)) continue;
          double2* own = r + 3 * nd.x;
          const double2 sv[3] = {own[0], own[1], own[2]};
          double2 xp[3] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
          const int cm = a.mask[i];
          if (nd.y >= 0) {
            const double2* pa = r + 3 * a.node[nd.y].x;
#pragma unroll
            for (int p = 0; p < 3; ++p)
              if ((cm >> p) & 1) xp[p] = pa[p];
          }
          const double2* z = a.z + (int64_t)i * 9;
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            double2 x = xp[p];
#pragma unroll
            for (int q = 0; q < 3; ++q) x = cfma(z[3 * q + p], sv[q], x);
            own[p] = (cm >> p) & 1 ? x : make_double2(0.0, 0.0);
          }
        }
        __syncthreads();
      }
      // mu += X, squared step size
      double dmax = 0.0;
      for (int j = t; j < n; j += AT_THREADS) {
        const double2 x = r[j];
        mu[j].x += x.x;
        mu[j].y += x.y;
        double st = fma(x.x, x.x, x.y * x.y);
        if (st != st) st = INFINITY;
        dmax = fmax(dmax, st);
      }
      dmax = at_block_max(dmax, red);
      it = k;
      if (dmax <= a.tol * a.tol) {
        ok = 1;
        break;
      }
      if (isinf(dmax)) break;
    }
    // dL/dS = s D^T mu
    for (int c = t; c < nb; c += AT_THREADS) {
      const int j0 = 3 * c;
      double2 v[3], u[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        v[p] = V[j0 + p];
        u[p] = mu[j0 + p];
      }
      if (a.Hw) {
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const double2 h = div_conj(u[p], v[p]);
          a.Hw[off + j0 + p] = make_double2(-s * h.x, -s * h.y);
        }
      }
      if (a.Hd) {
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const int y = x == 2 ? 0 : x + 1;
          const double2 h = div_conj(csub(u[y], u[x]), csub(v[x], v[y]));
          a.Hd[off + j0 + x] = make_double2(s * h.x, s * h.y);
        }
      }
    }
    if (t == 0) {
      a.iters[b] = it;
      a.conv[b] = (uint8_t)ok;
    }
    __syncthreads();
  }
}

int grid_1d(int64_t tot, int cap) {
  return (int)std::min<int64_t>(cap, std::max<int64_t>(1, (tot + 255) / 256));
}

// Z^T operands, the zero no-load term, and per-scenario scratch for B.
zbus_status ensure_adjoint(zbus_network net, int64_t B, cudaStream_t st) {
  const int np = net->n_pad;
  ZB_CHECK(ensure_3m(net, st));
  if (!net->ZrT) {
    const size_t bytes = (size_t)np * np * sizeof(double);
    ZB_CUDA(cudaMalloc((void**)&net->ZrT, bytes));
    ZB_CUDA(cudaMalloc((void**)&net->ZiT, bytes));
    ZB_CUDA(cudaMalloc((void**)&net->ZsT, bytes));
    ZB_CUDA(cudaMalloc((void**)&net->adj_zero, (size_t)np * sizeof(double2)));
    ZB_CUDA(cudaMemsetAsync(net->adj_zero, 0, (size_t)np * sizeof(double2), st));
    const dim3 grid((np + 31) / 32, (np + 31) / 32, 3);
    k_transpose_3m<<<grid, dim3(32, 8), 0, st>>>(net->Zr, net->Zi, net->Zs, net->ZrT, net->ZiT,
                                                  net->ZsT, np);
    ZB_CUDA(cudaGetLastError());
  }
  if (net->adj_cap < B) {
    ZB_CUDA(cudaStreamSynchronize(st));
    cudaFree(net->adj_mu);
    cudaFree(net->adj_scale);
    net->adj_mu = nullptr;
    net->adj_scale = nullptr;
    net->adj_cap = 0;
    ZB_CUDA(cudaMalloc((void**)&net->adj_mu, (size_t)B * net->n * sizeof(double2)));
    ZB_CUDA(cudaMalloc((void**)&net->adj_scale, (size_t)B * sizeof(double)));
    net->adj_cap = B;
  }
  return ZBUS_OK;
}

// One adjoint sweep: K1', the contraction with Z^T, the forward stop test.
zbus_status enqueue_sweep_adjoint(zbus_network net, int64_t B, int grid,
                                  cudaGraphConditionalHandle h, bool use_handle, cudaStream_t st,
                                  cudaEvent_t* ev) {
  (void)ev;
  const int64_t tot = B * (int64_t)(net->n_pad / 3);
  k_adj_rhs<<<grid_1d(tot, 152 * 16), 256, 0, st>>>(net->ws.ctx, net->n, net->n_pad);
  launch_gemm_f64(net->ws.ctx, net->ZrT, net->ZiT, net->ZsT, net->adj_zero, net->n, net->n_pad,
                  grid, st);
  launch_converge(net->ws.ctx, (int)B, h, use_handle, st);
  return ZBUS_OK;
}

// The adjoint on padded device arrays.
zbus_status adjoint_device(zbus_network net, int64_t B, const double* S_wye,
                           const double* S_delta, const double* V, const double* G, double tol,
                           int32_t max_iter, double* dS_wye, double* dS_delta, int32_t* iters,
                           uint8_t* converged, cudaStream_t st) {
  ZB_CHECK(ensure_workspace(net, B));
  ZB_CHECK(ensure_adjoint(net, B, st));
  net->last_group = nullptr;
  SolveCtx h;
  std::memset(&h, 0, sizeof(h));
  h.S_wye = (const double2*)S_wye;
  h.S_del = (const double2*)S_delta;
  h.V = net->adj_mu;
  h.iters = iters;
  h.conv = converged;
  h.list = net->ws.list;
  h.keep = net->ws.keep;
  h.part = net->ws.part;
  h.Iop = net->ws.Iop;
  h.tol = tol;
  h.B = (int32_t)B;
  h.max_iter = max_iter;
  h.rule = ZBUS_CONV_MAXABS;
  h.ntn = net->n_pad / F64_BN;
  h.Vf = (const double2*)V;
  h.G = (const double2*)G;
  h.gscale = net->adj_scale;
  const int n = net->n;
  k_adj_scale<<<grid_1d(B * 32, 4096), 256, 0, st>>>((const double2*)G, n, (int)B,
                                                     net->adj_scale);
  k_adj_init<<<grid_1d(B * (int64_t)n, 4096), 256, 0, st>>>(net->ws.ctx, h, n, (int)B);
  ZB_CUDA(cudaGetLastError());
  const int grid = gemm_f64_grid((int)B, net->n_pad);
  if (use_graphs()) {
    GraphEntry* g = nullptr;
    ZB_CHECK(get_while_graph(net, B, GRAPH_KEY_ADJOINT, grid, enqueue_sweep_adjoint, &g));
    ZB_CUDA(cudaGraphLaunch(g->exec, st));
  } else {
    for (int k = 0; k < max_iter; ++k)
      ZB_CHECK(enqueue_sweep_adjoint(net, B, grid, 0, false, st, nullptr));
  }
  const int nb = (n + 2) / 3;
  k_adj_out<<<grid_1d(B * (int64_t)nb, 4096), 256, 0, st>>>(
      net->adj_mu, (const double2*)V, net->adj_scale, n, (int)B, (double2*)dS_wye,
      (double2*)dS_delta);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

// The tree form on padded device arrays (radial networks).
zbus_status adjoint_tree_device(zbus_network net, int64_t B, const double* S_wye,
                                const double* S_delta, const double* V, const double* G,
                                double tol, int32_t max_iter, double* dS_wye, double* dS_delta,
                                int32_t* iters, uint8_t* converged, cudaStream_t st) {
  net->last_group = nullptr;
  // the iterate and the residual on chip up to 96 KB (two CTAs per SM at the
  // largest such feeder, ~1000 buses), else in the scratch slice
  const size_t onchip = 2 * (size_t)net->n * sizeof(double2);
  const size_t smem = onchip <= 96 * 1024 ? onchip : 0;
  if (smem > 48 * 1024)
    ZB_CUDA(cudaFuncSetAttribute(k_adj_tree, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  int per = 0, sms = 0;
  ZB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_adj_tree, AT_THREADS, smem));
  ZB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, net->device));
  const int64_t ctas = std::min<int64_t>(B, (int64_t)sms * std::max(1, per));
  const int64_t stride = 5 * (int64_t)net->n;
  if (net->adj_tree_ctas < ctas) {
    ZB_CUDA(cudaStreamSynchronize(st));
    cudaFree(net->adj_tree_scratch);
    net->adj_tree_scratch = nullptr;
    net->adj_tree_ctas = 0;
    ZB_CUDA(cudaMalloc((void**)&net->adj_tree_scratch,
                       (size_t)ctas * stride * sizeof(double2)));
    net->adj_tree_ctas = ctas;
  }
  AdjTree a;
  a.n = net->n;
  a.nb = net->nbus;
  a.depth = net->depth;
  a.B = (int)B;
  a.max_iter = max_iter;
  a.tol = tol;
  a.node = net->t_node;
  a.lvl = net->t_lvl;
  a.mask = net->t_mask;
  a.z = net->t_z64;
  a.pblk = net->t_pblk;
  a.nblk = net->nblk;
  a.bptr = net->bsr_ptr;
  a.bcol = net->bsr_col;
  a.bval = net->bsr_val;
  a.Sw = (const double2*)S_wye;
  a.Sd = (const double2*)S_delta;
  a.V = (const double2*)V;
  a.G = (const double2*)G;
  a.Hw = (double2*)dS_wye;
  a.Hd = (double2*)dS_delta;
  a.iters = iters;
  a.conv = converged;
  a.scratch = net->adj_tree_scratch;
  a.stride = stride;
  a.onchip = smem > 0 ? 1 : 0;
  k_adj_tree<<<(int)ctas, AT_THREADS, smem, st>>>(a);
  ZB_CUDA(cudaGetLastError());
  return ZBUS_OK;
}

zbus_status adjoint_any(zbus_network net, bool tree, int64_t B, const double* S_wye,
                        const double* S_delta, const double* V, const double* G, double tol,
                        int32_t max_iter, double* dS_wye, double* dS_delta, int32_t* iters,
                        uint8_t* converged, cudaStream_t st) {
  if (tree)
    return adjoint_tree_device(net, B, S_wye, S_delta, V, G, tol, max_iter, dS_wye, dS_delta,
                               iters, converged, st);
  return adjoint_device(net, B, S_wye, S_delta, V, G, tol, max_iter, dS_wye, dS_delta, iters,
                        converged, st);
}

bool on_device(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

void free_adjoint(zbus_network net) {
  cudaFree(net->ZrT);
  cudaFree(net->ZiT);
  cudaFree(net->ZsT);
  cudaFree(net->adj_zero);
  cudaFree(net->adj_mu);
  cudaFree(net->adj_scale);
  net->ZrT = net->ZiT = net->ZsT = nullptr;
  net->adj_zero = nullptr;
  net->adj_mu = nullptr;
  net->adj_scale = nullptr;
  net->adj_cap = 0;
  cudaFree(net->adj_tree_scratch);
  net->adj_tree_scratch = nullptr;
  net->adj_tree_ctas = 0;
}

ZB_CHECK_WORD_ACCESSOR(check_word_adjoint)

}  // namespace zbus

using namespace zbus;

extern "C" zbus_status zbus_solve_adjoint(zbus_network net, int64_t B, const double* S_wye,
                                          const double* S_delta, const double* V,
                                          const double* G, double tol, int32_t max_iter,
                                          const zbus_solve_opts* opts, double* dS_wye,
                                          double* dS_delta, int32_t* iters, uint8_t* converged,
                                          void* cuda_stream) {
  NvtxRange nvtx_range("zbus_solve_adjoint");
  set_error("");
  if (!net) return fail(ZBUS_ERR_ARG, "network is NULL");
  if (B < 0 || B > INT32_MAX / 4) return fail(ZBUS_ERR_ARG, "B out of range");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(ZBUS_ERR_ARG, "tol must be finite, >= 0");
  if (max_iter < 1) return fail(ZBUS_ERR_ARG, "max_iter must be >= 1");
  const int32_t prec = opts ? opts->precision : ZBUS_FP64;
  if (prec != ZBUS_FP64 && prec != ZBUS_TREE_SWEEP)
    return fail(ZBUS_ERR_UNSUPPORTED, "the adjoint runs in FP64 (dense) or as a tree sweep");
  const bool tree = prec == ZBUS_TREE_SWEEP;
  if (tree && !net->radial)
    return fail(ZBUS_ERR_UNSUPPORTED, "the tree form needs a radial network with reciprocal "
                                      "branches");
  if (B == 0) return ZBUS_OK;
  if (!V || !G || !iters || !converged)
    return fail(ZBUS_ERR_ARG, "V, G, iters and converged are required");
  if ((S_delta || dS_delta) && !net->bus_aligned)
    return fail(ZBUS_ERR_ARG, "delta loads need three unknowns per bus (n % 3 == 0)");
  const void* ptrs[] = {S_wye, S_delta, V, G, dS_wye, dS_delta, iters, converged};
  for (const void* p : ptrs)
    if (!on_device(p)) return fail(ZBUS_ERR_ARG, "the adjoint takes device buffers only");
  int dev = -1;
  ZB_CUDA(cudaGetDevice(&dev));
  if (dev != net->device) return fail(ZBUS_ERR_ARG, "current CUDA device differs from the network's");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!net->phased)
    return adjoint_any(net, tree, B, S_wye, S_delta, V, G, tol, max_iter, dS_wye, dS_delta, iters,
                       converged, st);
  // partial-phase network: into the padded layout; the gradients come back
  // through the buffers of the loads, which the last kernel no longer reads
  double* buf[4];
  ZB_CHECK(phased_stage(net, B, buf));
  if (S_wye) ZB_CHECK(phased_in(net, B, S_wye, buf[0], false, st));
  if (S_delta) ZB_CHECK(phased_in(net, B, S_delta, buf[1], true, st));
  ZB_CHECK(phased_in(net, B, V, buf[2], false, st));
  ZB_CHECK(phased_in(net, B, G, buf[3], false, st));
  ZB_CHECK(adjoint_any(net, tree, B, S_wye ? buf[0] : nullptr, S_delta ? buf[1] : nullptr,
                       buf[2], buf[3], tol, max_iter, dS_wye ? buf[0] : nullptr,
                       dS_delta ? buf[1] : nullptr, iters, converged, st));
  if (dS_wye) ZB_CHECK(phased_out(net, B, buf[0], dS_wye, st));
  if (dS_delta) ZB_CHECK(phased_out_delta(net, B, buf[1], dS_delta, st));
  return ZBUS_OK;
}
