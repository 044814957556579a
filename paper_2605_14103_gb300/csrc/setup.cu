// Network setup (Sec. II-B: slack / non-slack separation and the precomputed
// reduced bus impedance), all arithmetic in FP64 on the device:
//   dense Y_LL, Y_Ls v_s from the coalesced COO entries,
//   Z = Y_LL^{-1} by Gauss-Jordan elimination with partial pivoting,
//   w = -Z (Y_Ls v_s),
//   FP64 contraction operands Zr, Zi, Zr + Zi (zero-padded, row-major).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <numeric>

#include "zbus_internal.cuh"

namespace zbus {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Scatter coalesced Y_LL entries (no duplicates) into a zeroed dense matrix.
__global__ void k_scatter(double2* A, int n, const int32_t* r, const int32_t* c,
                          const double2* v, int64_t m) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x)
    A[(int64_t)r[t] * n + c[t]] = v[t];
}

// The same from the device CSR of Y_LL (one thread per row).
__global__ void k_scatter_csr(double2* A, int n, const int32_t* ptr, const int32_t* col,
                              const double2* v) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    for (int t = ptr[r]; t < ptr[r + 1]; ++t) A[(int64_t)r * n + col[t]] = v[t];
}

// ys[j] = sum_p Y_Ls[j][p] v_s[p] from the slack-column entries (row-sorted,
// so each row's terms are summed in a fixed order by one thread).
__global__ void k_slack_injection(double2* ys, int n, const int32_t* ptr, const int32_t* sp,
                                  const double2* sv, double2 v0, double2 v1, double2 v2) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int t = ptr[j]; t < ptr[j + 1]; ++t) {
    double2 vs = sp[t] == 0 ? v0 : (sp[t] == 1 ? v1 : v2);
    double2 p = cmul(sv[t], vs);
    acc.x += p.x;
    acc.y += p.y;
  }
  ys[j] = acc;
}

// Gauss-Jordan step k, part 1 (one block): choose the pivot row, swap it into
// row k, save column k, scale the pivot row.  info records the first bad pivot.
__global__ void k_gj_pivot(double2* A, int n, int k, int32_t* perm, double2* colk, int32_t* info) {
  __shared__ double sbest[1024];
  __shared__ int sidx[1024];
  const int tid = threadIdx.x;
  double best = -1.0;
  int bi = k;
  for (int i = k + tid; i < n; i += blockDim.x) {
    double2 a = A[(int64_t)i * n + k];
    double m = a.x * a.x + a.y * a.y;
    if (m > best) { best = m; bi = i; }
  }
  sbest[tid] = best;
  sidx[tid] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) {
      double o = sbest[tid + s];
      int oi = sidx[tid + s];
      if (o > sbest[tid] || (o == sbest[tid] && oi < sidx[tid])) { sbest[tid] = o; sidx[tid] = oi; }
    }
    __syncthreads();
  }
  const int p = sidx[0];
  const double pm = sbest[0];
  if (tid == 0) {
    perm[k] = p;
    if (!(pm > 0.0) || !isfinite(pm)) {
      if (*info == 0) *info = k + 1;
    }
  }
  if (p != k) {
    for (int j = tid; j < n; j += blockDim.x) {
      double2 a = A[(int64_t)k * n + j];
      A[(int64_t)k * n + j] = A[(int64_t)p * n + j];
      A[(int64_t)p * n + j] = a;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) colk[i] = A[(int64_t)i * n + k];
  __syncthreads();
  double2 piv = colk[k];
  double d = piv.x * piv.x + piv.y * piv.y;
  double2 inv = (d > 0.0) ? make_double2(piv.x / d, -piv.y / d) : make_double2(0.0, 0.0);
  for (int j = tid; j < n; j += blockDim.x) {
    if (j == k) A[(int64_t)k * n + j] = inv;
    else A[(int64_t)k * n + j] = cmul(A[(int64_t)k * n + j], inv);
  }
}

// Gauss-Jordan step k, part 2: eliminate column k from every other row.
// A[i][j] <- (j == k ? 0 : A[i][j]) - colk[i] * A[k][j]
__global__ void k_gj_update(double2* A, int n, int k, const double2* colk) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double2 akj = A[(int64_t)k * n + j];
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    if (i == k) continue;
    const double2 f = colk[i];
    if (f.x == 0.0 && f.y == 0.0) continue;
    double2 a = (j == k) ? make_double2(0.0, 0.0) : A[(int64_t)i * n + j];
    a.x -= f.x * akj.x - f.y * akj.y;
    a.y -= f.x * akj.y + f.y * akj.x;
    A[(int64_t)i * n + j] = a;
  }
}

// Undo the row interchanges of the elimination as column interchanges of the
// inverse, last step first.  One thread per row.
__global__ void k_gj_unpermute(double2* A, int n, const int32_t* perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2* row = A + (int64_t)i * n;
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      double2 t = row[k];
      row[k] = row[p];
      row[p] = t;
    }
  }
}

// w[i] = -sum_j Z[i][j] ys[j], one warp per row, fixed summation order.
__global__ void k_noload(const double2* Z, const double2* ys, double2* w, int n) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int j = lane; j < n; j += 32) {
    double2 p = cmul(Z[(int64_t)warp * n + j], ys[j]);
    acc.x += p.x;
    acc.y += p.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) w[warp] = make_double2(-acc.x, -acc.y);
}

// Real operand layouts of the FP64 contraction: Zr, Zi, Zr + Zi, zero padded
// to n_pad x n_pad.
__global__ void k_pack_f64(const double2* Z, int n, int n_pad, double* Zr, double* Zi, double* Zs) {
  const int64_t tot = (int64_t)n_pad * n_pad;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n_pad), j = (int)(t % n_pad);
    double2 z = (i < n && j < n) ? Z[(int64_t)i * n + j] : make_double2(0.0, 0.0);
    Zr[t] = z.x;
    Zi[t] = z.y;
    Zs[t] = z.x + z.y;
  }
}

__global__ void k_check_finite(const double2* w, int n, int32_t* info) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(isfinite(w[i].x) && isfinite(w[i].y))) atomicCAS(info, 0, -1);
}

struct Entry {
  int32_t r, c;
  double re, im;
};

template <class T>
zbus_status upload(T** dst, const std::vector<T>& src, cudaStream_t st) {
  size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  ZB_CUDA(cudaMalloc((void**)dst, bytes));
  if (!src.empty()) ZB_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T),
                                            cudaMemcpyHostToDevice, st));
  return ZBUS_OK;
}

// Inverse of a 3x3 complex matrix (row-major) on the phases its entries
// touch (a line of fewer phases has zero rows and columns for the others,
// which stay zero in the result), by Gauss-Jordan elimination with partial
// pivoting; false when a pivot vanishes or no phase is touched.
bool inv3(const double2* a, double2* out) {
  int ph[3], m = 0;
  for (int p = 0; p < 3; ++p) {
    bool any = false;
    for (int q = 0; q < 3; ++q)
      any = any || a[3 * p + q].x != 0.0 || a[3 * p + q].y != 0.0 || a[3 * q + p].x != 0.0 ||
            a[3 * q + p].y != 0.0;
    if (any) ph[m++] = p;
  }
  if (m == 0) return false;
  std::complex<double> g[3][6];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      const double2 x = a[3 * ph[i] + ph[j]];
      g[i][j] = {x.x, x.y};
      g[i][m + j] = i == j ? 1.0 : 0.0;
    }
  double scale = 0.0;
  for (int e = 0; e < 9; ++e) scale = std::max(scale, std::hypot(a[e].x, a[e].y));
  for (int k = 0; k < m; ++k) {
    int piv = k;
    for (int i = k + 1; i < m; ++i)
      if (std::abs(g[i][k]) > std::abs(g[piv][k])) piv = i;
    if (!(std::abs(g[piv][k]) > 1e-13 * scale)) return false;
    if (piv != k)
      for (int j = 0; j < 2 * m; ++j) std::swap(g[k][j], g[piv][j]);
    const std::complex<double> d = 1.0 / g[k][k];
    for (int j = 0; j < 2 * m; ++j) g[k][j] *= d;
    for (int i = 0; i < m; ++i) {
      if (i == k) continue;
      const std::complex<double> f = g[i][k];
      for (int j = 0; j < 2 * m; ++j) g[i][j] -= f * g[k][j];
    }
  }
  for (int e = 0; e < 9; ++e) out[e] = make_double2(0.0, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      out[3 * ph[i] + ph[j]] = make_double2(g[i][m + j].real(), g[i][m + j].imag());
  return true;
}

// Branches of the branch form, for the FP64 mismatch test that forms each
// line's term once: where every neighbour block has an identical mirror
// (Y_ab == Y_ba, bit for bit: lines with symmetric series matrices), the term
// of bus b in row a is the negative of that of bus a in row b,
//   Y_ba (v_a - v_b) = -Y_ab (v_b - v_a).
// Branch k = (a, b, block of Y_ab) with a < b; br_of[t] = k for the block
// (a, b) and -(k + 1) for its mirror (b, a); 0 for slack and shunt blocks.
// Leaves net->nbr = 0 when a block has no identical mirror.
zbus_status build_branches(zbus_network net, const std::vector<int32_t>& bp,
                           const std::vector<int32_t>& bc, const std::vector<double2>& bv,
                           cudaStream_t st) {
  const int nb = net->nbus;
  std::vector<int32_t> br_of(bc.size(), 0);
  std::vector<int4> tab;
  for (int a = 0; a < nb; ++a)
    for (int t = bp[a]; t < bp[a + 1]; ++t) {
      const int b = bc[t];
      if (b < 0) continue;
      int u = -1;
      for (int x = bp[b]; x < bp[b + 1]; ++x)
        if (bc[x] == a) u = x;
      if (u < 0) return ZBUS_OK;
      if (std::memcmp(&bv[(size_t)t * 9], &bv[(size_t)u * 9], 9 * sizeof(double2)) != 0)
        return ZBUS_OK;
      if (b > a) {
        br_of[t] = (int32_t)tab.size();
        tab.push_back(make_int4(a, b, t, 0));
      }
    }
  // mirrors: the block (b, a) with b > a refers to branch (a, b)
  for (int b = 0; b < nb; ++b)
    for (int t = bp[b]; t < bp[b + 1]; ++t) {
      const int a = bc[t];
      if (a < 0 || a > b) continue;
      for (int x = bp[a]; x < bp[a + 1]; ++x)
        if (bc[x] == b) br_of[t] = -(br_of[x] + 1);
    }
  if (tab.empty()) return ZBUS_OK;
  ZB_CHECK(upload(&net->br_tab, tab, st));
  ZB_CHECK(upload(&net->bsr_br, br_of, st));
  net->nbr = (int)tab.size();
  return ZBUS_OK;
}

// Radial structure of the branch form, when the buses form a tree hanging off
// the slack with reciprocal branches (Y_cp = Y_pc): breadth-first positions
// (so every level and every bus's children are contiguous ranges), each
// position's bus, parent and children, the level ranges, and z_c =
// (-Y_c,parent)^{-1}, the series impedance of each bus's parent branch
// (-Y_c,slack for buses on the slack).  For such a network without shunts,
// Y_LL^{-1} r is, at every bus, the sum over its path to the slack of z times
// the subtree sums of r.  Leaves net->radial false otherwise.
zbus_status build_tree(zbus_network net, const std::vector<int32_t>& bp,
                       const std::vector<int32_t>& bc, const std::vector<double2>& bv,
                       cudaStream_t st) {
  const int nb = net->nbus;
  auto block_of = [&](int a, int col) -> int {
    for (int t = bp[a]; t < bp[a + 1]; ++t)
      if (bc[t] == col) return t;
    return -1;
  };
  // parents by a breadth-first search from the slack-connected buses; a bus
  // reached twice means a loop
  std::vector<int32_t> par(nb, -2), roots, queue;
  for (int a = 0; a < nb; ++a)
    if (block_of(a, -1) >= 0) {
      par[a] = -1;
      roots.push_back(a);
    }
  queue = roots;
  for (size_t h = 0; h < queue.size(); ++h) {
    const int a = queue[h];
    for (int t = bp[a]; t < bp[a + 1]; ++t) {
      const int c = bc[t];
      if (c < 0 || c == par[a]) continue;
      if (par[c] != -2) return ZBUS_OK;
      par[c] = a;
      queue.push_back(c);
    }
  }
  if ((int)queue.size() != nb) return ZBUS_OK;
  // levels in breadth-first order (the queue), children of each bus as a
  // contiguous range of that order
  std::vector<int32_t> depth(nb, 0), qpos(nb);
  for (int i = 0; i < nb; ++i) {
    const int c = queue[i];
    qpos[c] = i;
    if (par[c] >= 0) depth[c] = depth[par[c]] + 1;
  }
  const int levels = 1 + *std::max_element(depth.begin(), depth.end());
  std::vector<int32_t> lvl(levels + 1, 0);
  for (int i = 0; i < nb; ++i) lvl[depth[queue[i]] + 1] = i + 1;
  for (int L = 1; L <= levels; ++L) lvl[L] = std::max(lvl[L], lvl[L - 1]);
  std::vector<int4> node(nb);        // per breadth-first position
  std::vector<float2> z((size_t)nb * 9);
  std::vector<double2> z64((size_t)nb * 9);   // the same impedances in FP64, unscaled
  std::vector<int32_t> pblk(nb);              // branch-form block of each position's parent line
  std::vector<float> zs(nb);
  std::vector<uint8_t> mask(nb);     // phases the parent line carries
  int next = (int)roots.size();
  for (int i = 0; i < nb; ++i) {
    const int c = queue[i], p = par[c];
    int cnt = 0;
    for (int t = bp[c]; t < bp[c + 1]; ++t)
      if (bc[t] >= 0 && bc[t] != p) ++cnt;
    node[i] = make_int4(c, p >= 0 ? qpos[p] : -1, next, next + cnt);
    for (int q = next; q < next + cnt; ++q)
      if (par[queue[q]] != c) return ZBUS_OK;   // children not contiguous: not expected
    next += cnt;
    const int t = block_of(c, p >= 0 ? p : -1);
    pblk[i] = t;
    if (p >= 0) {
      const int u = block_of(p, c);
      if (t < 0 || u < 0) return ZBUS_OK;
      double ymax = 0.0, dmax = 0.0;
      for (int e = 0; e < 9; ++e) {
        const double2 x = bv[(size_t)t * 9 + e], y = bv[(size_t)u * 9 + e];
        ymax = std::max(ymax, std::hypot(x.x, x.y));
        dmax = std::max(dmax, std::hypot(x.x - y.x, x.y - y.y));
      }
      if (dmax > 1e-12 * ymax) return ZBUS_OK;   // not reciprocal
    }
    double2 y[9], zi[9];
    for (int e = 0; e < 9; ++e)
      y[e] = make_double2(-bv[(size_t)t * 9 + e].x, -bv[(size_t)t * 9 + e].y);
    if (!inv3(y, zi)) return ZBUS_OK;
    uint8_t mk = 0;
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q)
        if (y[3 * p + q].x != 0.0 || y[3 * p + q].y != 0.0) mk |= (uint8_t)((1 << p) | (1 << q));
    mask[i] = mk;
    double m = 0.0;
    for (int e = 0; e < 9; ++e) m = std::max(m, std::max(std::fabs(zi[e].x), std::fabs(zi[e].y)));
    if (!(m > 0.0) || !std::isfinite(m)) return ZBUS_OK;
    const int ex = std::ilogb(m);
    zs[i] = std::ldexp(1.0f, ex);
    for (int e = 0; e < 9; ++e) z64[(size_t)i * 9 + e] = zi[e];
    for (int e = 0; e < 9; ++e)
      z[(size_t)i * 9 + e] =
          make_float2((float)std::ldexp(zi[e].x, -ex), (float)std::ldexp(zi[e].y, -ex));
  }
  ZB_CHECK(upload(&net->t_lvl, lvl, st));
  ZB_CHECK(upload(&net->t_mask, mask, st));
  ZB_CHECK(upload(&net->t_node, node, st));
  ZB_CHECK(upload(&net->t_z, z, st));
  ZB_CHECK(upload(&net->t_zs, zs, st));
  ZB_CHECK(upload(&net->t_z64, z64, st));
  ZB_CHECK(upload(&net->t_pblk, pblk, st));
  net->depth = levels;
  net->radial = true;
  return ZBUS_OK;
}

}  // namespace

zbus_status build_network(zbus_network net, int32_t n_total, int64_t nnz, const int32_t* row,
                          const int32_t* col, const double* val, const int32_t* slack,
                          const double* vs, cudaStream_t st) {
  const int n = n_total - 3;
  net->n_total = n_total;
  net->n = n;
  net->n_pad = round_up(n, F64_PAD);
  net->bus_aligned = (n % 3) == 0;
  for (int p = 0; p < 3; ++p) net->v_slack[p] = make_double2(vs[2 * p], vs[2 * p + 1]);

  // global index -> unknown index (>= 0) or slack phase (-1 - p)
  std::vector<int32_t> pos(n_total, 0);
  for (int p = 0; p < 3; ++p) pos[slack[p]] = -1 - p;
  int j = 0;
  for (int g = 0; g < n_total; ++g)
    if (pos[g] >= 0) pos[g] = j++;

  // coalesce the COO entries of the non-slack rows (sorted, duplicates summed
  // in input order)
  std::vector<Entry> e;
  e.reserve((size_t)nnz);
  for (int64_t t = 0; t < nnz; ++t) {
    if (pos[row[t]] < 0) continue;
    e.push_back({pos[row[t]], pos[col[t]], val[2 * t], val[2 * t + 1]});
  }
  std::stable_sort(e.begin(), e.end(), [](const Entry& a, const Entry& b) {
    return a.r != b.r ? a.r < b.r : a.c < b.c;  // slack columns (< 0) first, then ascending
  });
  std::vector<Entry> u;
  for (const Entry& x : e) {
    if (!u.empty() && u.back().r == x.r && u.back().c == x.c) {
      u.back().re += x.re;
      u.back().im += x.im;
    } else {
      u.push_back(x);
    }
  }
  // split: Y_LL (c >= 0) as CSR with ascending columns, Y_Ls (c < 0) per row
  std::vector<int32_t> lp(n + 1, 0), sp(n + 1, 0);
  for (const Entry& x : u) {
    if (x.c >= 0) lp[x.r + 1]++;
    else sp[x.r + 1]++;
  }
  for (int i = 0; i < n; ++i) {
    lp[i + 1] += lp[i];
    sp[i + 1] += sp[i];
  }
  std::vector<int32_t> lc(lp[n]), sc(sp[n]);
  std::vector<double2> lv(lp[n]), sv(sp[n]);
  std::vector<int32_t> fl(lp.begin(), lp.end() - 1), fs(sp.begin(), sp.end() - 1);
  for (const Entry& x : u) {
    if (x.c >= 0) {
      int t = fl[x.r]++;
      lc[t] = x.c;
      lv[t] = make_double2(x.re, x.im);
    } else {
      int t = fs[x.r]++;
      sc[t] = -1 - x.c;
      sv[t] = make_double2(x.re, x.im);
    }
  }
  net->nnz_ll = lp[n];
  int mr = 0;
  for (int i = 0; i < n; ++i) mr = std::max(mr, lp[i + 1] - lp[i]);
  net->max_row_nnz = mr;

  // Branch form of the admittance rows, per bus a (rows 3a..3a+2), used by
  // the mixed sweeps and the FP64 mismatch test:
  //   (Y_LL v + Y_Ls v_s)_a = sum_{b != a} Y_ab (v_b - v_a) + Y_as (v_s - v_a) + Sh_a v_a
  // with Sh_a = Y_aa + sum_{b != a} Y_ab + Y_as the block row sum (the shunt;
  // zero up to rounding for series-only lines, and then left out).  Entries:
  // column >= 0 a neighbour bus, -1 the slack, -2 the shunt; 3x3 complex
  // blocks, row-major.  Differences of neighbouring voltages are small, so
  // the products stay well conditioned.
  if (net->bus_aligned) {
    const int nb = n / 3;
    std::vector<int32_t> bp(nb + 1, 0), bc;
    std::vector<double2> bv;
    for (int a = 0; a < nb; ++a) {
      std::vector<int32_t> cols;
      for (int r = 3 * a; r < 3 * a + 3; ++r)
        for (int t = lp[r]; t < lp[r + 1]; ++t)
          if (lc[t] / 3 != a) cols.push_back(lc[t] / 3);
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      double2 diag[9], slk[9], sh[9];
      for (int e = 0; e < 9; ++e) diag[e] = slk[e] = sh[e] = make_double2(0.0, 0.0);
      bool has_slack = false;
      const size_t base = bc.size();
      for (int c : cols) bc.push_back(c);
      bv.resize(bc.size() * 9, make_double2(0.0, 0.0));
      for (int r = 3 * a; r < 3 * a + 3; ++r) {
        for (int t = lp[r]; t < lp[r + 1]; ++t) {
          const int cb = lc[t] / 3;
          const int e = (r - 3 * a) * 3 + (lc[t] - 3 * cb);
          if (cb == a) {
            diag[e] = lv[t];
          } else {
            const size_t k = base + (std::lower_bound(cols.begin(), cols.end(), cb) - cols.begin());
            bv[k * 9 + e] = lv[t];
          }
        }
        for (int t = sp[r]; t < sp[r + 1]; ++t) {
          slk[(r - 3 * a) * 3 + sc[t]] = sv[t];
          has_slack = true;
        }
      }
      // shunt = block row sum, summed in a fixed order
      double ymax = 0.0, smax = 0.0;
      for (int e = 0; e < 9; ++e) {
        double2 acc = diag[e];
        for (size_t k = base; k < bc.size(); ++k) {
          acc.x += bv[k * 9 + e].x;
          acc.y += bv[k * 9 + e].y;
        }
        acc.x += slk[e].x;
        acc.y += slk[e].y;
        sh[e] = acc;
        ymax = std::max(ymax, std::hypot(diag[e].x, diag[e].y));
        smax = std::max(smax, std::hypot(acc.x, acc.y));
      }
      if (has_slack) {
        bc.push_back(-1);
        bv.insert(bv.end(), slk, slk + 9);
      }
      if (smax > 1e-12 * ymax) {
        bc.push_back(-2);
        bv.insert(bv.end(), sh, sh + 9);
      }
      bp[a + 1] = (int32_t)bc.size();
    }
    net->nbus = nb;
    net->nblk = (int64_t)bc.size();
    ZB_CHECK(upload(&net->bsr_ptr, bp, st));
    ZB_CHECK(upload(&net->bsr_col, bc, st));
    ZB_CHECK(upload(&net->bsr_val, bv, st));
    ZB_CHECK(build_branches(net, bp, bc, bv, st));
    ZB_CHECK(build_tree(net, bp, bc, bv, st));
  }

  ZB_CUDA(cudaMalloc((void**)&net->w, n * sizeof(double2)));
  ZB_CUDA(cudaMalloc((void**)&net->ys, n * sizeof(double2)));
  ZB_CHECK(upload(&net->csr_ptr, lp, st));
  ZB_CHECK(upload(&net->csr_col, lc, st));
  ZB_CHECK(upload(&net->csr_val, lv, st));
  int32_t *d_sp = nullptr, *d_sc = nullptr;
  double2* d_sv = nullptr;
  zbus_status s = ZBUS_OK;
  do {
    if ((s = upload(&d_sp, sp, st)) != ZBUS_OK) break;
    if ((s = upload(&d_sc, sc, st)) != ZBUS_OK) break;
    if ((s = upload(&d_sv, sv, st)) != ZBUS_OK) break;
    k_slack_injection<<<(n + 255) / 256, 256, 0, st>>>(net->ys, n, d_sp, d_sc, d_sv,
                                                        net->v_slack[0], net->v_slack[1],
                                                        net->v_slack[2]);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
      s = cuda_fail(ce, "setup kernel launch", __FILE__, __LINE__);
      break;
    }
    s = ensure_3m(net, st);
  } while (0);
  cudaStreamSynchronize(st);
  cudaFree(d_sp);
  cudaFree(d_sc);
  cudaFree(d_sv);
  return s;
}

zbus_status ensure_z(zbus_network net, cudaStream_t st) {
  if (net->Z) return ZBUS_OK;
  const int n = net->n;
  const size_t zb = (size_t)n * n * sizeof(double2);
  ZB_CUDA(cudaMalloc((void**)&net->Z, zb));
  int32_t *d_perm = nullptr, *d_info = nullptr;
  double2* d_colk = nullptr;
  zbus_status s = ZBUS_OK;
  do {
    cudaError_t ce;
    if ((ce = cudaMalloc((void**)&d_perm, n * sizeof(int32_t))) != cudaSuccess ||
        (ce = cudaMalloc((void**)&d_info, sizeof(int32_t))) != cudaSuccess ||
        (ce = cudaMalloc((void**)&d_colk, n * sizeof(double2))) != cudaSuccess) {
      s = cuda_fail(ce, "cudaMalloc(setup scratch)", __FILE__, __LINE__);
      break;
    }
    cudaMemsetAsync(d_info, 0, sizeof(int32_t), st);
    cudaMemsetAsync(net->Z, 0, zb, st);
    k_scatter_csr<<<(n + 255) / 256, 256, 0, st>>>(net->Z, n, net->csr_ptr, net->csr_col,
                                                    net->csr_val);
    const int gy = std::min(n, 256);
    for (int k = 0; k < n; ++k) {
      k_gj_pivot<<<1, 1024, 0, st>>>(net->Z, n, k, d_perm, d_colk, d_info);
      k_gj_update<<<dim3((n + 127) / 128, gy), 128, 0, st>>>(net->Z, n, k, d_colk);
    }
    k_gj_unpermute<<<(n + 127) / 128, 128, 0, st>>>(net->Z, n, d_perm);
    // w = -Z Y_Ls v_s (the same value at every formation: the elimination is
    // deterministic)
    k_noload<<<(n * 32 + 255) / 256, 256, 0, st>>>(net->Z, net->ys, net->w, n);
    k_check_finite<<<(n + 255) / 256, 256, 0, st>>>(net->w, n, d_info);
    if ((ce = cudaGetLastError()) != cudaSuccess) {
      s = cuda_fail(ce, "setup kernel launch", __FILE__, __LINE__);
      break;
    }
    int32_t info = 0;
    if ((ce = cudaMemcpyAsync(&info, d_info, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (ce = cudaStreamSynchronize(st)) != cudaSuccess) {
      s = cuda_fail(ce, "setup synchronize", __FILE__, __LINE__);
      break;
    }
    if (info > 0) {
      s = fail(ZBUS_ERR_SINGULAR, "Y_LL is singular: zero pivot at elimination step " +
                                      std::to_string(info - 1));
    } else if (info < 0) {
      s = fail(ZBUS_ERR_SINGULAR, "no-load voltage is not finite (Y_LL numerically singular)");
    }
  } while (0);
  cudaFree(d_perm);
  cudaFree(d_info);
  cudaFree(d_colk);
  if (s != ZBUS_OK) {
    cudaFree(net->Z);
    net->Z = nullptr;
  }
  return s;
}

zbus_status ensure_3m(zbus_network net, cudaStream_t st) {
  if (net->Zr) return ZBUS_OK;
  ZB_CHECK(ensure_z(net, st));
  const size_t pb = (size_t)net->n_pad * net->n_pad * sizeof(double);
  zbus_status s = ZBUS_OK;
  cudaError_t ce;
  if ((ce = cudaMalloc((void**)&net->Zr, pb)) != cudaSuccess ||
      (ce = cudaMalloc((void**)&net->Zi, pb)) != cudaSuccess ||
      (ce = cudaMalloc((void**)&net->Zs, pb)) != cudaSuccess) {
    s = cuda_fail(ce, "cudaMalloc(3M operands)", __FILE__, __LINE__);
  } else {
    k_pack_f64<<<2048, 256, 0, st>>>(net->Z, net->n, net->n_pad, net->Zr, net->Zi, net->Zs);
    if ((ce = cudaGetLastError()) != cudaSuccess ||
        (ce = cudaStreamSynchronize(st)) != cudaSuccess)
      s = cuda_fail(ce, "3M operands", __FILE__, __LINE__);
  }
  if (s != ZBUS_OK) release_3m(net);
  return s;
}

void release_z(zbus_network net) {
  cudaFree(net->Z);
  net->Z = nullptr;
}

void release_3m(zbus_network net) {
  drop_graphs(net);   // their kernels hold the operand addresses
  free_adjoint(net);
  cudaFree(net->Zr);
  cudaFree(net->Zi);
  cudaFree(net->Zs);
  net->Zr = net->Zi = net->Zs = nullptr;
}

}  // namespace zbus
