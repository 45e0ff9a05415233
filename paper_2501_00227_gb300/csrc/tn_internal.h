// tn_internal.h -- types shared by the host planner, the kernels and the C ABI
// of libtn.  Not installed; the public interface is include/tn.h.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "tn.h"

namespace tn {

// Largest rank of any tensor the kernels accept (2^30 entries).
constexpr int kMaxRank = 30;
// Largest number of labels one step touches (|LA u LB|).
constexpr int kMaxStepBits = 60;
// Alignment of every tensor inside the workspace arena, in entries.
constexpr int64_t kArenaAlign = 64;
// Bytes reserved at the head of the workspace (status words, raw result).
constexpr size_t kHeaderBytes = 256;

// Where an operand of a step comes from.
enum OperandKind : int32_t {
  kOpArena = 0,   // an intermediate stored in the workspace arena
  kOpEdge = 1,    // an edge leaf B(n_u, n_v): generated in the kernel
  kOpVertex = 2,  // a vertex leaf W(n_v): generated in the kernel
  kOpOne = 3,     // the rank-0 multiplicative identity (single-leaf networks)
  kOpShared = 4,  // an intermediate inside a group task, in the CTA's shared memory
};

// Geometry of one pairwise step, as seen by the kernels.
//
// The step computes C[b, m, n] = (+)_k A[b, m, k] (x) B[b, k, n] where
//   b runs over the batch labels  (in A, in B, kept),
//   m over the labels only in A that are kept,
//   n over the labels only in B that are kept,
//   k over the summed labels (shared ones, and any label of one side alone
//     that no other live tensor uses; the other side broadcasts over it).
// The output is stored contiguously as c = n | m << nn | b << (nn + nm), so
// the output tensor's labels, least significant first, are N, M, batch.
// a_pos[i] is the bit position in A of GEMM coordinate bit i, where the
// coordinate bits are listed as (b bits, m bits, k bits); b_pos likewise for
// B with (b bits, k bits, n bits).  -1 means the operand does not carry that
// label (it broadcasts).
struct StepGeom {
  int32_t nb, nm, nn, nk;
  int32_t ra, rb, rc;
  int32_t a_kind, b_kind;
  int32_t c_identity;  // 1: output entry index = c; 0: scatter c through c_pos
  int8_t a_pos[64];
  int8_t b_pos[64];
  int8_t c_pos[32];    // bit position in the stored output of coordinate bit i of c
};

struct TensorInfo {
  std::vector<int32_t> labels;  // least significant first
  int64_t offset = -1;          // arena offset in entries (intermediates only)
  int32_t producer = -1;        // step that creates it (-1 for leaves)
  int32_t consumer = -1;        // step that consumes it (-1 for the root)
  int32_t kind = kOpArena;
};

// How a step is executed.
enum StepKernel : int32_t {
  kKernNaive = 0,  // one thread per output entry, gathers through bit maps
  kKernTiled = 1,  // register-blocked semiring GEMM with cluster split-K
};

struct Step {
  int32_t a_id, b_id, c_id;
  StepGeom g;
  uint64_t ops;          // 2^{|LA u LB|}
  int32_t kernel = kKernNaive;
  int32_t split_k = 1;   // CTAs of a cluster sharing one output tile
  int32_t tile = 0;      // tile-shape index for kKernTiled
};

}  // namespace tn

struct tn_plan_s {
  int32_t n = 0, m = 0, T = 0;
  std::vector<int32_t> edges;
  std::vector<int32_t> order;
  std::vector<tn::TensorInfo> tensors;   // T leaves then nsteps intermediates
  std::vector<tn::Step> steps;
  int64_t arena_entries = 0;             // arena length in entries (aligned)
  uint64_t tc = 0, rwc = 0, sc = 0;
  int32_t root = -1;                     // id of the scalar result
  void* exec_cache = nullptr;            // executor plans (exec_plan.cu)
  // Slicing (Sec. 4.2.2): sliced vertex labels are fixed per slice and
  // dropped from every leaf; such a plan runs with stored leaves only.
  std::vector<int32_t> sliced;           // sliced labels, in slice-bit order
  std::vector<int64_t> leaf_off;         // entry offset of each leaf in a stored-leaf block
  int64_t leaf_entries = 0;              // entries of all leaves (sum of 2^rank)
  void* slice_cache = nullptr;           // merged plans of slice batches (slice.cu)
};

namespace tn {

// Host planner (plan.cpp).
int build_plan(int32_t n, const int32_t* edges, int32_t m, const int32_t* order, int32_t nsteps,
               tn_plan_s* p, const int32_t* sliced = nullptr, int32_t nsliced = 0);
int greedy_order(int32_t n, const int32_t* edges, int32_t m, double alpha, int32_t nrepeat,
                 uint64_t seed, int32_t* order_out);
// Label classification of one pairwise step (shared by build_plan and
// tn_contract_pair): fills geometry and the output label order (N, M,
// batch).  Labels of each class are numbered in their operand's storage
// order, except that N labels listed in n_first (if given) come first.
int classify_step(const std::vector<int32_t>& la, const std::vector<int32_t>& lb,
                  const std::vector<int32_t>& lc_set, StepGeom* g, std::vector<int32_t>* lc_order,
                  const std::vector<int32_t>* n_first = nullptr);

// Bytes per entry summed over the per-entry regions of a semiring.
size_t bytes_per_entry(tn_semiring_t s, int32_t nprimes);
size_t workspace_bytes(const tn_plan_s* p, tn_semiring_t s, int32_t nprimes);

// CRT (Garner) on the host: x in [0, prod p) from residues; little-endian
// 32-bit limbs.  Returns the number of limbs.
int crt_garner(const uint32_t* residues, const uint32_t* primes, int nprimes, uint32_t* limbs,
               int max_limbs);

}  // namespace tn
