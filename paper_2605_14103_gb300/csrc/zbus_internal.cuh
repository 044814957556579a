// Internal declarations of libzbus (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "zbus.h"

namespace zbus {

// ---------------------------------------------------------------------------
// Error plumbing: a thread-local message plus status codes.
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
zbus_status fail(zbus_status s, const std::string& msg);
zbus_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define ZB_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t _e = (call);                                                 \
    if (_e != cudaSuccess) return ::zbus::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define ZB_CHECK(call)                        \
  do {                                        \
    zbus_status _s = (call);                  \
    if (_s != ZBUS_OK) return _s;             \
  } while (0)

// ---------------------------------------------------------------------------
// Tiling constants of the FP64 path.
// ---------------------------------------------------------------------------
constexpr int F64_BM = 32;   // scenarios per tile
constexpr int F64_BN = 48;   // outputs (16 buses) per tile
// whole-solve kernel of the latency case: up to 96 padded unknowns, one
// block of four warps per scenario, batches of one tile at most
constexpr int FUSED_MAX_NPAD = 96;
constexpr int FUSED_THREADS = 128;
constexpr int F64_BK = 16;   // k step
constexpr int F64_PAD = 48;  // n is padded to a multiple of this

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// A named range on the host timeline of profilers (NVTX; no cost without a
// tool attached) around each entry point and each serving sweep.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// Checked build (-DZBUS_CHECKED): every index read from a table (columns,
// active lists, tree nodes, maps, permutations, level lists) is tested
// against the size of the buffer it addresses before the access; a bad one
// records its code in this translation unit's check word and the access is
// skipped.  Nothing traps; zbus_checked_status reports the words.  The normal
// build compiles every test away.
// ---------------------------------------------------------------------------
#ifdef ZBUS_CHECKED
static __device__ unsigned int g_zb_check_word;
__device__ __forceinline__ bool zb_in(long long i, long long n, unsigned int code) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_zb_check_word, 0u, code);
  return false;
}
#define ZB_IN(i, n, code) ::zbus::zb_in((long long)(i), (long long)(n), (code))
#define ZB_CHECK_WORD_ACCESSOR(fn)                                        \
  uint32_t fn(bool clear) {                                              \
    uint32_t v = 0;                                                      \
    cudaMemcpyFromSymbol(&v, g_zb_check_word, sizeof(v));                \
    if (clear) {                                                         \
      const uint32_t z = 0;                                              \
      cudaMemcpyToSymbol(g_zb_check_word, &z, sizeof(z));                \
    }                                                                    \
    return v;                                                            \
  }
#else
#define ZB_IN(i, n, code) true
#define ZB_CHECK_WORD_ACCESSOR(fn) \
  uint32_t fn(bool) { return 0; }
#endif
// the check words of the translation units (0 in the normal build)
uint32_t check_word_f64(bool clear);
uint32_t check_word_group(bool clear);
uint32_t check_word_adjoint(bool clear);
uint32_t check_word_nr(bool clear);
uint32_t check_word_phased(bool clear);

// ---------------------------------------------------------------------------
// Per-solve device context.  Kernels read pointers and sizes from it, so a
// captured graph does not depend on the caller's buffers.
// ---------------------------------------------------------------------------
struct SolveCtx {
  const double2* S_wye;   // [B][n] or nullptr
  const double2* S_del;   // [B][n] or nullptr
  const double2* V_init;  // [B][n] or nullptr
  double2* V;             // [B][n]
  int32_t* iters;         // [B]
  uint8_t* conv;          // [B]
  int32_t* list;          // [B] active slot -> scenario
  double* part;           // [B][ntn][2] per-tile partials (max step, sum-magnitude change)
  double* Iop;            // FP64: 3 x [B][n_pad] (Ir, Ii, Ir+Ii)
  double tol;
  double mismatch_tol;
  int32_t B;
  int32_t count;          // active scenarios
  int32_t iter;           // maps performed so far
  int32_t max_iter;
  int32_t rule;
  int32_t ntn;            // N-tiles of the contraction
  int32_t err;            // device error word (0 = fine)
  // FP64 correction of the mixed forms: max |dS|^2 per scenario (bit
  // patterns of non-negative doubles) and the reported mismatch (or null)
  unsigned long long* mmax;
  double* mm_out;
  int32_t* hist;          // profile mode: active count of sweep k (else nullptr)
  int32_t hist_n;
  uint8_t* keep;          // [B] stop decision of the current sweep, by slot
  // load gradient (adjoint sweeps): V holds the adjoint iterate mu, these the
  // converged voltages, the loss gradient and its per-scenario scale
  const double2* Vf;      // [B][n]
  const double2* G;       // [B][n]
  const double* gscale;   // [B]
};

struct Workspace {
  int64_t cap_B = 0;
  size_t bytes = 0;
  void* base = nullptr;
  SolveCtx* ctx = nullptr;   // device
  int32_t* list = nullptr;
  double* part = nullptr;    // [cap_B][max N-tiles][2]
  double* Iop = nullptr;     // FP64: 3 x [cap_B][n_pad]
  size_t iop_bytes = 0;      // bytes of that region
  void* R = nullptr;         // mixed: [cap_B][K_pad] fp16 / bf16 residual rows
  float* rinv = nullptr;     // mixed: [cap_B] inverse residual scales
  double* mm = nullptr;      // mixed: [cap_B] final FP64 mismatch (-1 if not checked)
  uint8_t* keep = nullptr;   // [cap_B]
  float2* Vh = nullptr;      // mixed: [n][cap_Bp] double-float state, hi
  float2* Vl = nullptr;      // mixed: [n][cap_Bp] lo
  float2* Swf = nullptr;     // mixed: [n][cap_Bp] FP32 wye loads
  float2* Sdf = nullptr;     // mixed: [n][cap_Bp] FP32 delta loads
  uint8_t* st = nullptr;     // mixed: [cap_Bp]
  float* amax = nullptr;     // mixed: [2][cap_Bp]
  int32_t* mt = nullptr;     // mixed: [2][cap_Bp / 128] tile list and flags
  int64_t cap_Bp = 0;        // cap_B rounded up to 128
  uint64_t gen = 0;          // bumped at every reallocation
  int32_t* slot_it = nullptr;   // mixed: [cap_Bp] sweeps since admission
  uint8_t* slot_conv = nullptr; // mixed: [cap_Bp] stop rule met
};

// Low-precision operands of Z for the tensor-core contraction.
struct MixedOperands {
  bool ready = false;
  bool bf16 = false;
  int zparts = 1;            // 1: FP16 row-scaled; 2: BF16 hi + lo
  int K_pad = 0;             // 2n rounded up to 64
  int N_pad = 0;             // 2n rounded up to 256
  void* Z0 = nullptr;        // [N_pad][K_pad] (hi part)
  void* Z1 = nullptr;        // [N_pad][K_pad] (lo part, BF16 only)
  float* zinv = nullptr;     // [N_pad / 2] inverse row scales per complex output
};

// Host-driven profiling run: 4 events per sweep around the three kernels.
struct Profile {
  std::vector<cudaEvent_t> ev;
  int32_t* d_hist = nullptr;
  int32_t cap = 0;
  int32_t sweeps = 0;
};

// Device staging of solves on host buffers: two sets of [cap] scenarios
// (wye loads, delta loads, warm start, V, then iters and flags), a copy stream
// each way, and events ordering copies and sweeps.
struct HostStage {
  int64_t cap = 0;
  double* buf[2] = {nullptr, nullptr};
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t start = nullptr, end = nullptr;
  cudaEvent_t in[2] = {nullptr, nullptr};     // a set's inputs are on the device
  cudaEvent_t done[2] = {nullptr, nullptr};   // a set's chunk is solved
  cudaEvent_t out[2] = {nullptr, nullptr};    // a set's outputs are back in host memory
};

struct GraphEntry {
  int64_t B = 0;
  int32_t precision = -1;
  int32_t grid_gemm = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

}  // namespace zbus

namespace zbus {
struct Group;
}

struct zbus_network_s {
  int device = 0;
  int n = 0;         // unknowns
  int n_total = 0;
  int n_pad = 0;     // FP64 operand padding
  bool bus_aligned = false;  // n % 3 == 0: delta loads allowed
  double2 v_slack[3];
  // device data
  double2* Z = nullptr;      // [n][n]
  double2* w = nullptr;      // [n]
  double2* ys = nullptr;     // [n]  Y_Ls v_s
  double* Zr = nullptr;      // [n_pad][n_pad] row-major, zero padded
  double* Zi = nullptr;
  double* Zs = nullptr;      // Zr + Zi
  int32_t* csr_ptr = nullptr;   // Y_LL rows (n + 1)
  int32_t* csr_col = nullptr;
  double2* csr_val = nullptr;
  int64_t nnz_ll = 0;
  int max_row_nnz = 0;
  float4* csr_df = nullptr;  // Y_LL values as double-float (re hi, re lo, im hi, im lo)
  float4* ys_df = nullptr;   // Y_Ls v_s as double-float
  float4* w_df = nullptr;    // no-load voltage w as double-float (re hi, re lo, im hi, im lo)
  // branch form of the admittance rows per bus (networks with n % 3 == 0):
  // entries with column >= 0 (neighbour bus: Y_ab (v_b - v_a)), -1 (slack:
  // Y_as (v_s - v_a)) or -2 (shunt: Sh_a v_a); 3x3 complex blocks
  int nbus = 0;
  int32_t* bsr_ptr = nullptr;   // [nbus + 1]
  int32_t* bsr_col = nullptr;   // [nblk]
  double2* bsr_val = nullptr;   // [nblk][3][3] row-major complex
  int64_t nblk = 0;
  float4* bsr_df = nullptr;     // [nblk][9] double-float copy (mixed sweeps)
  // branches (pairs of identical mirror blocks), for the FP64 test that forms
  // each line's term once: (a, b, block of Y_ab) with a < b, and per block
  // its branch (k, or -(k + 1) for the mirror); nbr = 0 where not available
  int nbr = 0;
  int4* br_tab = nullptr;       // [nbr]
  int32_t* bsr_br = nullptr;    // [nblk]
  // radial structure (buses form a tree hanging off the slack, reciprocal
  // branches), for the tree-sweep application of Z: breadth-first positions,
  // levels, children ranges, and the inverse series block of each bus's
  // parent branch
  bool radial = false;
  int depth = 0;                // levels of the tree
  int4* t_node = nullptr;       // [nbus] per position: bus, parent position (-1: slack),
                                //        first child position, end of the children
  int32_t* t_lvl = nullptr;     // [depth + 1] first position of each level
  uint8_t* t_mask = nullptr;    // [nbus] phases (bits 0..2) of each position's parent line
  float2* t_z = nullptr;        // [nbus][9] z = y^{-1} of the parent branch, scaled by 2^-e
  float* t_zs = nullptr;        // [nbus] 2^e
  double2* t_z64 = nullptr;     // [nbus][9] the same z in FP64 (the load-gradient sweep)
  int32_t* t_pblk = nullptr;    // [nbus] branch-form block of each position's parent line
  zbus::Workspace ws;
  zbus::MixedOperands mixed[2];   // [0] FP16 row-scaled, [1] BF16 hi + lo
  uint64_t op_gen = 0;            // bumped when the tensor-core operands are freed
  struct zbus::Group* group1 = nullptr;   // single-network mixed solves
  struct zbus::Group* last_group = nullptr;   // group of the last mixed solve (error word)
  std::vector<zbus::GraphEntry> graphs;
  // FP64 correction loop of the mixed forms (group.cu), built for the
  // workspace generation corr_gen
  cudaGraph_t corr_graph = nullptr;
  cudaGraphExec_t corr_exec = nullptr;
  uint64_t corr_gen = 0;
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  zbus::Profile prof;
  zbus::HostStage stage;
  // partial-phase networks: the caller's unknowns (present phases, ascending
  // global index) inside the padded three-phase network solved on the device
  bool phased = false;
  int n_user = 0;                 // the caller's unknowns
  int32_t* ph_map = nullptr;      // [n_user] padded unknown of each caller unknown
  uint8_t* ph_dvalid = nullptr;   // [n_user] 1 where its delta branch has both phases
  double* ph_buf = nullptr;       // four padded [ph_cap][n] complex staging arrays
  int64_t ph_cap = 0;
  // load gradient (zbus_solve_adjoint): Z^T in the 3M layout, a zero no-load
  // term for the contraction epilogue, the adjoint iterate and the
  // per-scenario gradient scales
  double* ZrT = nullptr;
  double* ZiT = nullptr;
  double* ZsT = nullptr;
  double2* adj_zero = nullptr;    // [n_pad]
  double2* adj_mu = nullptr;      // [adj_cap][n]
  double* adj_scale = nullptr;    // [adj_cap]
  int64_t adj_cap = 0;
  double2* adj_tree_scratch = nullptr;   // tree form: [adj_tree_ctas][5 n]
  int64_t adj_tree_ctas = 0;
};

namespace zbus {

// api.cu: where a caller buffer lives (1 device or managed memory, 0 host
// memory, pinned or pageable; -1 null)
int buffer_kind(const void* p);

// noalloc.cu: loads the allocation-free solve's static scratch array on the
// current device and caches its address (called once per network creation)
zbus_status noalloc_prepare(int dev);

// setup.cu: dense operands.  Z = Y_LL^-1 (complex FP64, by Gauss-Jordan from
// the device CSR; also recomputes w) and its 3M copies (Zr, Zi, Zr + Zi) are
// formed on demand and can be released (the serving loop's operand cache);
// a release waits for nothing: the caller makes sure no work uses them.
zbus_status ensure_z(zbus_network net, cudaStream_t st);
zbus_status ensure_3m(zbus_network net, cudaStream_t st);
void release_z(zbus_network net);
void release_3m(zbus_network net);
// mixed.cu: frees the tensor-core operands of both precisions
void release_mixed_ops(zbus_network net);
// api.cu: drops the cached sweep graphs of a network (they hold operand and
// workspace addresses)
void drop_graphs(zbus_network net);

// setup.cu
zbus_status build_network(zbus_network net, int32_t n_total, int64_t nnz, const int32_t* row,
                          const int32_t* col, const double* val, const int32_t* slack,
                          const double* vs, cudaStream_t st);

// kernels_f64.cu
zbus_status probe_fp64_rate(double* tflops, float* ms, cudaStream_t st);
void launch_init(SolveCtx* ctx, const SolveCtx& h, const double2* w, int n, int B,
                 cudaStream_t st);
void launch_currents_f64(SolveCtx* ctx, int n, int n_pad, int B, cudaStream_t st);
void launch_gemm_f64(SolveCtx* ctx, const double* Zr, const double* Zi, const double* Zs,
                     const double2* w, int n, int n_pad, int grid, cudaStream_t st);
int gemm_f64_grid(int B, int n_pad);
void launch_converge(SolveCtx* ctx, int B, cudaGraphConditionalHandle h, bool use_handle,
                     cudaStream_t st);
void launch_solve_fused_f64(const double* Zr, const double* Zi, const double* Zs,
                            const double2* w, const double2* V_init, const double2* S_wye,
                            const double2* S_del, int n, int n_pad, int B, double tol,
                            int max_iter, int rule, double2* V, int32_t* iters, uint8_t* conv,
                            cudaStream_t st);
void launch_mismatch(const double2* V, const double2* S_wye, const double2* S_del,
                     const int32_t* ptr, const int32_t* col, const double2* val,
                     const double2* ys, int n, int B, double* out, cudaStream_t st);


// api.cu
zbus_status ensure_workspace(zbus_network net, int64_t B);
bool use_graphs();   // false when ZBUS_NO_GRAPH=1 (sweeps launched from the host)
// One sweep enqueued on a stream: the last kernel sets the WHILE condition
// through h when use_handle; ev (or nullptr) brackets the kernels.
typedef zbus_status (*SweepFn)(zbus_network net, int64_t B, int grid,
                               cudaGraphConditionalHandle h, bool use_handle, cudaStream_t st,
                               cudaEvent_t* ev);
// Graph keys besides the precisions of the solve.
constexpr int32_t GRAPH_KEY_ADJOINT = -2;
zbus_status get_while_graph(zbus_network net, int64_t B, int32_t key, int grid, SweepFn sweep,
                            GraphEntry** out);

// adjoint.cu
void free_adjoint(zbus_network net);

// phased.cu
zbus_status phased_validate(int32_t n_total, const int32_t* slack_idx, const int32_t* bus_phase,
                            int32_t* n_bus);
void phased_pad_coo(int32_t n_total, int64_t nnz, const int32_t* row, const int32_t* col,
                    const double* val, const int32_t* bus_phase, int32_t n_bus,
                    std::vector<int32_t>& r2, std::vector<int32_t>& c2, std::vector<double>& v2);
zbus_status phased_attach(zbus_network net, int32_t n_total, const int32_t* slack_idx,
                          const int32_t* bus_phase, cudaStream_t st);
// staging: bufs[0..3] = padded [B][n] arrays (wye, delta, warm start, voltages)
zbus_status phased_stage(zbus_network net, int64_t B, double** bufs);
zbus_status phased_in(zbus_network net, int64_t B, const double* src, double* dst, bool delta,
                      cudaStream_t st);
zbus_status phased_out(zbus_network net, int64_t B, const double* src, double* dst,
                       cudaStream_t st);
// phased_out for delta-slot arrays: entries whose branch lacks its second
// phase come out zero
zbus_status phased_out_delta(zbus_network net, int64_t B, const double* src, double* dst,
                             cudaStream_t st);
zbus_status phased_z(zbus_network net, double* Z_out, cudaStream_t st);
void phased_free(zbus_network net);

// group.cu

// mixed.cu
zbus_status make_tmap_2d(CUtensorMap* map, const void* base, bool bf16, uint64_t cols,
                         uint64_t rows, uint32_t box_cols, uint32_t box_rows);
zbus_status prepare_mixed(zbus_network net, int32_t precision, cudaStream_t st);
zbus_status prepare_df(zbus_network net, cudaStream_t st);
// double-float operands of the tree sweep (radial networks only)
zbus_status prepare_tree(zbus_network net, cudaStream_t st);
void free_mixed(zbus_network net);


}  // namespace zbus
