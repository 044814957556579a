// Grouped mixed-precision sweep: several feeders ("items"), each with its own
// scenario slots, advanced together by one set of kernels per sweep.  A
// single-feeder solve is a group of one; the batched solve and the serving
// loop use the same kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "zbus_internal.cuh"

namespace zbus {

// Slot states.
constexpr uint8_t SLOT_ACTIVE = 0;
constexpr uint8_t SLOT_DONE = 1;   // stopped, result not yet collected
constexpr uint8_t SLOT_FREE = 2;

// One feeder of a group (device-visible).
struct ItemDesc {
  // network operands
  const int32_t* bsr_ptr;
  const int32_t* bsr_col;
  const float4* bsr_df;     // [nblk][9] double-float branch-form blocks
  float4 vs_df[3];          // slack phase voltages, double-float (re hi, re lo, im hi, im lo)
  const float* zinv;        // [N_pad / 2] inverse row scales of Z
  int32_t n, nbus, K_pad, N_pad, ntn;
  int32_t Bp;               // slot capacity, multiple of 128
  // slot state, scenario-minor [n][Bp]
  float2* Vh;
  float2* Vl;
  float2* Swf;              // FP32 wye loads (zeros where absent)
  float2* Sdf;              // FP32 delta loads (zeros where absent)
  uint8_t* st;              // [Bp] SLOT_*
  int32_t* it;              // [Bp] sweeps since admission
  uint8_t* conv;            // [Bp] stop rule met
  float* amax;              // [4][Bp] max |r| of the previous / current sweep, the
                            // current sweep's largest line or load current (FP32
                            // sweeps), the FP32-sweep flag (nonzero: on)
  void* R;                  // [Bp][K_pad] fp16 / bf16 residual rows
  float* rinv;              // [Bp] inverse residual scales
  double* part;             // [Bp][ntn][2] per-tile step partials
  // tree sweep (ZBUS_TREE_SWEEP): radial structure and FP32 residual
  const int4* t_node;       // [nbus] per breadth-first position: bus, parent, children range
  const int32_t* t_lvl;     // [tlevels + 1] level ranges of positions
  const uint8_t* t_mask;    // [nbus] phases of each position's parent line
  const float2* t_z;        // [nbus][9] scaled parent-branch impedances
  const float* t_zs;        // [nbus] their scales
  float2* Rt;               // [n][Bp] FP32 residual, scenario-minor
  int32_t tlevels;          // depth of the tree + 1
  int32_t tree_begin;       // first tree block of this item
  // launch decomposition
  int32_t res_begin;        // first residual block
  int32_t res_split;        // residual blocks per 32 slots
  int32_t dec_begin;        // first stop-test block (256 slots each)
  int32_t mt_begin;         // global index of this item's first 128-slot tile
};

// Sweep-loop state of a group (device).
struct GroupState {
  int32_t n_items;
  int32_t active;           // active slots at the start of the sweep
  int32_t sweep;
  int32_t max_iter;
  int32_t rule;
  double tol;
  int32_t err;
  int32_t n_tiles;          // entries of tiles
  int32_t raster;           // one-item groups: 128-slot tiles per group of the tile order
                            // (0: tile by tile, N-tiles fastest)
  int32_t mt_total;         // 128-slot tiles over all items
  int32_t res_blocks;       // residual grid size
  int32_t dec_blocks;       // stop-test grid size
  int32_t tree_groups;      // tree-sweep blocks over all items
  int32_t tree_done;        // tree-sweep blocks finished in this sweep
  int32_t tree_active;      // slots still active after this sweep (tree blocks' sum)
  int32_t stream_state;     // 1: the slot state exceeds what L2 keeps between kernels, so
                            // the contraction epilogue streams it (evict-first)
  int32_t* hist;            // profile mode: active slots of sweep k
  int32_t hist_n;
  uint64_t* tiles;          // (item << 32) | (mt << 16) | nt of every active tile
};

// Host object of a group: device descriptor arrays, tensor maps, loop graph.
struct Group {
  std::vector<zbus_network> nets;
  std::vector<int64_t> Bs;
  int32_t precision = -1;
  int BN = 0;
  int stages = 0;
  int n_items = 0;
  int mt_total = 0;
  int64_t total_Bp = 0;         // slots over all items
  int max_tiles = 0;
  int res_blocks = 0;
  int dec_blocks = 0;
  int tree_groups = 0;          // blocks of the tree sweep
  bool tree_wide = true;        // 16 warps per tree-sweep block (else 8)
  bool tree_onchip = false;     // the block's residual rows in shared memory
  size_t tree_smem = 0;         // their dynamic shared memory (tables)
  int num_sms = 148;
  int max_n = 0;               // largest feeder's unknowns
  void* dmem = nullptr;        // one allocation: items | state | tiles | maps
  ItemDesc* d_items = nullptr;
  GroupState* d_state = nullptr;
  uint64_t* d_tiles = nullptr;
  CUtensorMap* d_tmR = nullptr;
  CUtensorMap* d_tmZ0 = nullptr;
  CUtensorMap* d_tmZ1 = nullptr;
  std::vector<ItemDesc> h_items;
  std::vector<uint64_t> ws_gen;  // workspace generation of each item when built
  std::vector<uint64_t> op_gen;  // operand generation of each item when built
  uint64_t tune_gen = 0;         // tile table generation when built
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // profile mode
  std::vector<cudaEvent_t> ev;
  int32_t* d_hist = nullptr;
  int prof_cap = 0;
  int prof_sweeps = 0;
};

// lazy_ops: items whose tensor-core operands are not formed are built without
// them (the serving cache forms them before the item's first admission and
// then calls group_refresh_item).
zbus_status group_build(Group* g, const std::vector<zbus_network>& nets,
                        const std::vector<int64_t>& Bs, int32_t precision, cudaStream_t st,
                        bool lazy_ops = false);
// Item k's operand addresses (tensor maps, row scales) after its operands
// were formed again.
zbus_status group_refresh_item(Group* g, int k, cudaStream_t st);
void group_free(Group* g);
// Run start for item k: slots [s0, s0 + B) from v^0 (V0 or w) and the loads
// (FP64 [B][n]); admitted slots become active.  fp32_start: a cold start
// (no V0) begins with FP32 residual sweeps.
zbus_status group_admit(Group* g, int k, int64_t s0, int64_t B, const double* V0,
                        const double* S_wye, const double* S_delta, cudaStream_t st,
                        bool v0_broadcast = false, bool fp32_start = false);
// Rebuild the tile list and the active count from the slot states (after
// admissions between sweeps).
zbus_status group_rebuild(Group* g, cudaStream_t st);
// Mark every slot of every item free.
zbus_status group_reset(Group* g, cudaStream_t st);
// Loop parameters and the initial tile list (after the admissions).
zbus_status group_start(Group* g, double tol, int32_t max_iter, int32_t rule, int32_t* hist,
                        int32_t hist_n, cudaStream_t st);
// One sweep (residual, contraction, stop test, tile list); h / use_handle set
// the loop condition when captured in a graph.  ev: 4 events for profiling.
zbus_status group_sweep(Group* g, cudaGraphConditionalHandle h, bool use_handle, cudaStream_t st,
                        cudaEvent_t* ev = nullptr);
// Device-resident loop: sweeps until no slot is active (CUDA graph WHILE).
zbus_status group_run(Group* g, cudaStream_t st);
// Results of item k, slots [s0, s0 + B): merged FP64 voltages, iteration
// counts and flags into caller arrays, then the FP64 mismatch test; a
// converged scenario above mtol gets up to max_corr FP64 correction sweeps
// and loses its flag if it stays above (mm_out, may be null: the final
// mismatch, -1 where not checked).
zbus_status group_collect(Group* g, int k, int64_t s0, int64_t B, double* V_out, int32_t* iters,
                          uint8_t* converged, const double* S_wye, const double* S_delta,
                          double mtol, double* mm_out, int32_t max_corr, cudaStream_t st);
// Shared memory of the position tables of a tree-sweep block for a feeder of
// nbus buses: per bus its node record (16 B), FP16 z block (36 B), scale
// (4 B) and parent-line phase mask (1 B), padded to 16 B.
__host__ __device__ inline size_t tree_table_bytes(int nbus) {
  return ((size_t)57 * nbus + 15) & ~(size_t)15;
}
// Device error word of the group's last run (0: none; 101-104: a bounded
// wait of the tensor-core pipeline gave up), read after synchronising st.
zbus_status group_device_status(Group* g, cudaStream_t st);
// Where the error word lives on the device.
const int32_t* group_error_word(const Group* g);
// Tile configurations the contraction is compiled for (BN, stages).
bool tc_config_ok(int32_t precision, int BN, int stages);
int tc_variants(int32_t precision, int* BN, int* stages, int max);

// tune.cu: tile choice of a workload, table generation (bumped on change).
zbus_status tune_lookup(int32_t precision, int max_n, int64_t total_B, int* BN, int* stages);
uint64_t tune_generation();

}  // namespace zbus
