// exec.h -- the persistent plan executor of libtn: data shared by the host
// exec planner (exec_plan.cpp) and the executor kernel (exec.cu).
//
// A contraction runs as ONE kernel launch.  The host turns the plan's
// pairwise steps (Sec. 4.1 of arXiv:2501.00227) into a flat list of tasks in
// a topological order (by dependency level): a task is a chunk of output
// entries of a general step, one output tile (and split-K slice) of a wide
// step, or the final copy of the scalar.  Persistent CTAs claim tasks with an
// atomic counter; a task first waits until the steps it depends on have
// completed (per-step done counters, acquire loads), runs, then publishes its
// completion (release).  Because a task only waits on tasks earlier in the
// list, and those were claimed by CTAs that are already running, the
// schedule cannot deadlock; every wait is still bounded by a timeout that
// aborts the whole launch with TN_ETIMEOUT.
#pragma once

#include <climits>
#include <cstdint>
#include <mutex>
#include <vector>

#include "tn_internal.h"

namespace tn {

struct ExecStep {
  StepGeom g;
  int64_t a_off, b_off, c_off;   // arena entry offsets (intermediates)
  int64_t scratch_off;           // byte offset of the split-K partial tiles
  int64_t chunk;                 // naive: output entries per task
  int32_t kernel;                // kKernNaive / kKernTiled
  int32_t tile, split, tiles_m, tiles_n;
  int32_t R;                     // naive: threads per output entry
  int32_t ntasks;                // tasks per prime
  int32_t dep_begin, dep_count;  // into the dependency array (exec-step indices)
  int32_t arrive_off;            // first split-K arrival counter of this step
  int32_t ks;                    // naive: k splits per output chunk
  int32_t nchunks;               // naive: output chunks
  int32_t done_target;           // tasks of this step (its done counter's final value)
  int32_t c_shared;              // 1: the output lives in the group task's shared memory at byte c_off
  int32_t vec;                   // tiles: operands staged in 16-byte runs (kVecA | kVecB of tile_device.cuh)
  int32_t final_slot;            // >= 0: the task that completes this step writes raw result slot final_slot
};

// Shared memory of a group task reserved for its internal tensors (bytes),
// and the most members a group may have (their step records are copied to
// shared memory together when the group starts).
constexpr int64_t kGroupSmem = 32 * 1024;
constexpr int kGroupMaxMembers = 16;

// Bytes of an intermediate of rank r in shared memory: values (4 bytes),
// then counts (8 bytes, 8-aligned) for counting, one residue array per prime
// for mod p (prime-major); 16-byte aligned.
inline int64_t shared_tensor_bytes(tn_semiring_t s, int32_t nprimes, int r) {
  const int64_t e = int64_t(1) << r;
  int64_t b = 4 * e;
  if (s == TN_COUNTING_TROPICAL) b = (4 * e + 7) / 8 * 8 + 8 * e;
  if (s == TN_COUNT_MODP) b = 4 * e * (nprimes < 1 ? 1 : nprimes);
  return (b + 15) / 16 * 16;
}

enum ExecTaskKind : int32_t { kTaskNaive = 0, kTaskTile = 1, kTaskFinal = 2, kTaskGroup = 3 };

struct ExecTask {
  int32_t step;   // exec-step index
  int32_t local;  // naive: chunk index; tile: tile * split + rank; group: group index
  int32_t prime;  // prime index (mod p), else 0; -1: every prime in turn
  int32_t kind;
};

// Host-side executor plan for one (plan, semiring, nprimes).
struct ExecPlan {
  tn_semiring_t semiring;
  int32_t nprimes;
  std::vector<ExecStep> steps;     // execution (level) order
  std::vector<int32_t> deps;
  std::vector<ExecTask> tasks;
  std::vector<int32_t> step_level;   // dependency level of each exec step
  std::vector<int32_t> exec_to_plan; // plan step index of each exec step
  int32_t tune_gen = 0;              // launch-table generation the plan was built under
  std::vector<int32_t> group_begin;  // group g's members: group_members[begin[g] .. begin[g+1])
  std::vector<int32_t> group_members;  // exec-step indices, in execution order
  int32_t ngroups = 0;
  int32_t group_h = 1;               // group height limit the plan was built with
  bool batched = false;              // built for a batch / served group
  bool keep = false;                 // every intermediate keeps its own arena block (no reuse)
  bool stored_leaves = false;        // leaf operands are arena tensors at leaf_base (weighted networks)
  // largest |finite value| any tropical tensor of the plan can hold: the
  // vertex count for unit-weight networks (an independent set's size), else
  // unbounded (stored leaves carry arbitrary weights)
  int64_t value_bound = INT64_MAX;
  int64_t leaf_base = 0;             // arena entry offset of the leaf tensors (plan leaf_off within)
  std::vector<int64_t> net_arena_base;  // merged plans: arena entry offset of each network
  int64_t arena_entries = 0;
  int64_t root_off = 0;
  int32_t root_step = -1;
  int32_t n_arrive = 0;
  int32_t nlevels = 0;
  int32_t nraw = 1;   // raw result slots (networks) of one launch
  size_t scratch_bytes = 0;
  // workspace layout (bytes from the start of the workspace)
  size_t ctr_off = 0, ctr_bytes = 0, scratch_base = 0, arena_base = 0, total_bytes = 0;
  // host image of the step / dependency / task tables and its device copy
  // (library-owned, uploaded once per device)
  std::vector<unsigned char> table_image;
  void* d_tables = nullptr;
  int device = -1;
  size_t off_steps = 0, off_deps = 0, off_tasks = 0, off_groups = 0, off_members = 0, table_bytes = 0;
  // executor launch shape
  int grid = 0;
  size_t smem = 0;
};

// Lays out and fills the device table image of X from its steps, deps,
// tasks and groups: steps | dependencies | tasks | group begins | group
// members.  A dependency is written as the pair (exec-step index, that
// step's done_target), so a waiting CTA reads the count it waits for with
// the index.
void exec_write_table_image(ExecPlan* X);

// Builds (or returns the cached) executor plan; thread-safe.
ExecPlan* exec_plan_get(tn_plan_s* p, tn_semiring_t s, int32_t nprimes, int* rc);
// The same with an explicit group height (largest tree of tiny steps one
// CTA runs back to back; 1 disables grouping).
// height: group height limit; batched: the plan runs inside a batch or a
// served group (launch shapes assume parallelism across networks).
ExecPlan* exec_plan_get_h(tn_plan_s* p, tn_semiring_t s, int32_t nprimes, int height, bool batched, int* rc,
                          bool keep = false, bool stored_leaves = false);
// TN_GROUP_HEIGHT, else 1.
int group_height();

// Measured launch shapes (tune.cu): the table's generation, and the entry
// for a step geometry if one is installed.
int32_t tune_generation();
bool tune_lookup(tn_semiring_t s, const StepGeom& g, int* tile, int* split);
void exec_plans_free(tn_plan_s* p);

// Enqueues one contraction through the executor (exec.cu).  keep: use the
// plan whose intermediates all stay in the arena after the launch (no block
// reuse, no groups), for a backward pass over them.  stored_leaves: use the
// plan whose edge / vertex leaves are arena tensors at leaf_base (written by
// the caller before the launch) instead of being generated in the kernels.
int exec_enqueue(tn_plan_s* p, tn_semiring_t s, const void* mods, int32_t nprimes, void* ws,
                 size_t ws_bytes, void* stream, void* d_raw, void* d_trace, bool keep = false,
                 bool stored_leaves = false);

// Launches the executor with the tables already on the device at d_tables.
int exec_launch_core(ExecPlan* X, tn_semiring_t s, const void* mods, void* ws, void* stream, void* d_raw,
                     void* d_trace, const void* d_tables);

// Merges the executor plans of several networks into one launch (batch.cu).
// stored_leaves: the networks' stored-leaf plans (their leaves are arena
// tensors at each network's net_arena_base + leaf_base).
int build_batch_plan(tn_plan_s* const* plans, int32_t count, tn_semiring_t semiring, int32_t nprimes,
                     int group_h, ExecPlan* out, bool stored_leaves = false);

// One-time kernel set-up of the executor instantiation a launch would use
// (attributes, occupancy), so that a later launch can be graph-captured.
int exec_prepare_launch(tn_semiring_t s, const void* mods);

// Bytes per accumulator / per staged value of the tiled tasks, and the
// dynamic shared memory the executor needs (exec.cu).  kw: the width K of a
// k-best element type.
size_t exec_acc_bytes(tn_semiring_t s, int32_t kw = 1);

// The k-best element types (TN_SIZE_MAX_K, TN_COUNTING_MAX_K): contracted
// by the general step body only, one task set (no per-prime tasks), with
// the element width K (2 or 4) in ExecPlan::nprimes.
inline bool is_kbest(tn_semiring_t s) { return s == TN_SIZE_MAX_K || s == TN_COUNTING_MAX_K; }
// Launches a k-best instantiation of the executor (kbest.cu); args is the
// filled dev::ExecArgs of exec_launch_core.
int kbest_launch(ExecPlan* X, tn_semiring_t s, const void* args, void* stream);
size_t exec_smem_bytes(tn_semiring_t s);

}  // namespace tn
