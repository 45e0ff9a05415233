// exec_device.cuh -- device side of the persistent plan executor (see
// exec.h): the kernel k_exec<SR, FOLD> and its task bodies, instantiated by
// exec.cu (the tropical, counting and mod-p element types) and kbest.cu (the
// k-best element types).
//
// One launch contracts a whole network.  Each CTA loops: claim the next task
// (atomic counter), copy its step record to shared memory, wait (warp 0,
// acquire loads, bounded by a timeout) until every step it depends on has
// published all of its tasks, run the task, publish (release).  Wide steps
// run as register-blocked GEMM tiles; their split-K partial tiles go to a
// scratch area and the last CTA of a tile to arrive merges them.  Tensors
// written during the launch are read through L2 only (ld.global.cg).
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "exec.h"
#include "kbest.cuh"
#include "kernels.h"
#include "semiring.cuh"
#include "step_device.cuh"
#include "tile_device.cuh"

namespace tn {
namespace dev {

struct ExecArgs {
  const ExecStep* steps;
  const int2* deps;              // (exec-step index, its done_target) pairs
  const ExecTask* tasks;
  const int32_t* group_begin;    // group g: group_members[group_begin[g] .. group_begin[g+1])
  const int32_t* group_members;  // exec-step indices
  int32_t ntasks_total;
  int32_t nprimes;
  int32_t* done;        // per exec step: finished tasks
  int32_t* arrive;      // split-K arrival counters
  int32_t* task_ctr;    // next task to claim
  uint32_t* status;     // bit 0: a wait timed out
  char* r0;             // arena: values / residues
  char* r1;             // arena: counts
  int64_t prime_stride; // entries between prime blocks
  char* scratch;
  unsigned char* raw;   // result block (TN_RAW_BYTES)
  ModTable mods;
  int32_t semiring;
  int32_t pad_;
  unsigned long long timeout_ns;
  unsigned long long* trace;  // optional: 8 words per task (see tn_contract_trace)
  int32_t nraw;               // raw result slots (networks in the launch)
  int32_t ctr_words;          // launch gate: 4-byte counter words at byte kHeaderBytes of the workspace
  uint32_t* ws;               // launch gate: the workspace (header, then counters)
  unsigned long long epoch;   // launch gate: nonzero = CTA 0 clears the header and counters itself
};

// Launch gate.  Instead of a host memset before the launch, CTA 0 clears the
// workspace header (status word, result block) and the task counters, then
// publishes the launch's epoch (unique per launch in the process) in the
// header's gate word; every CTA waits for that epoch (acquire, bounded by 2 s)
// before it claims a task.  A stale gate word can never match: it holds an
// earlier launch's epoch.
constexpr int kGateByte = 248;  // after the result block at 64..191, before the counters at kHeaderBytes

constexpr uint32_t kStatusTimeout = 1u;

// Phase marks of the running task (global timer, ns), written only while
// tracing: [0] end of the main computation, [1] start of the merge / store.
__shared__ unsigned long long g_trace_mark[2];

__device__ __forceinline__ int32_t ld_acquire(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ Operand exec_operand(const ExecArgs& a, int32_t kind, int64_t off) {
  Operand o;
  o.kind = kind;
  o.vx = 1;
  o.p0 = a.r0 + 4 * off;
  o.p1 = a.r1 ? a.r1 + 8 * off : nullptr;
  o.prime_stride = a.prime_stride;
  return o;
}

// Operand / output of a group member: an arena tensor, a leaf, or a tensor
// of rank `rank` in the group's shared memory at byte offset off (layout of
// shared_tensor_bytes: values, then counts or further primes).
__device__ __forceinline__ Operand exec_operand_g(const ExecArgs& a, int32_t kind, int64_t off, int rank,
                                                  unsigned char* gsm) {
  if (kind != kOpShared) return exec_operand(a, kind, off);
  const int64_t e = int64_t(1) << rank;
  Operand o;
  o.kind = kOpShared;
  o.vx = 1;
  o.p0 = gsm + off;
  o.p1 = gsm + off + (4 * e + 7) / 8 * 8;
  o.prime_stride = e;
  return o;
}
__device__ __forceinline__ Output exec_output_g(const ExecArgs& a, const ExecStep& st, unsigned char* gsm) {
  if (!st.c_shared) return Output{a.r0 + 4 * st.c_off, a.r1 ? a.r1 + 8 * st.c_off : nullptr, a.prime_stride};
  const int64_t e = int64_t(1) << st.g.rc;
  return Output{gsm + st.c_off, gsm + st.c_off + (4 * e + 7) / 8 * 8, e};
}

template <class SR>
struct ExecTile {
  // tropical steps may use 8 x 8 micro-tiles; counting and mod p use 4 x 4
  static constexpr bool kBig = std::is_same<SR, SrI32>::value || std::is_same<SR, SrF32>::value;
};

template <class T>
__device__ __forceinline__ T ldcg_acc(const T* p) {
  return __ldcg(p);
}
template <int K>
__device__ __forceinline__ KMaxVal<K> ldcg_acc(const KMaxVal<K>* p) {
  KMaxVal<K> r;
#pragma unroll
  for (int t = 0; t < K; ++t) r.v[t] = __ldcg(&p->v[t]);
  return r;
}
template <int K>
__device__ __forceinline__ KPolyVal<K> ldcg_acc(const KPolyVal<K>* p) {
  KPolyVal<K> r;
  r.d = __ldcg(&p->d);
#pragma unroll
  for (int t = 0; t < K; ++t) r.c[t] = __ldcg(&p->c[t]);
  return r;
}
__device__ __forceinline__ CntVal ldcg_acc(const CntVal* p) {
  CntVal v;
  v.v = __ldcg(&p->v);
  v.c = __ldcg(&p->c);
  return v;
}

// Arrival on a split counter: returns (to every thread) whether this CTA is
// the last of `split` to arrive; its writes before the call are visible to
// that last CTA.
__device__ __forceinline__ bool arrive_last(int32_t* ctr, int split, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    // acquire-release: publishes this CTA's partial (ordered by the barrier
    // above) and, for the last arriver, makes the other partials visible
    int32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
    *s_flag = old == split - 1;
  }
  __syncthreads();
  return *s_flag != 0;
}

// Task bodies are separate (not inlined) functions so that each gets its own
// register allocation under the kernel's 128-register bound.
template <class SR, class Cfg, int FOLD>
__device__ __noinline__ void exec_tile_task(const ExecArgs& a, const ExecStep& st, const ExecTask& task,
                                               unsigned char* smem, int* s_last, bool prepared) {
  constexpr int BM = Cfg::BM, BN = Cfg::BN, TM = Cfg::TM, TN = Cfg::TN;
  using Acc = typename SR::Acc;
  auto& sm = *reinterpret_cast<TileSmem<SR, Cfg>*>(smem);
  const TileIdx<Cfg>& ix = *reinterpret_cast<const TileIdx<Cfg>*>(smem);
  const StepGeom& g = st.g;
  const int tid = threadIdx.x;
  const int grp = tid / Cfg::GT, gt = tid % Cfg::GT;
  const int tx = gt % Cfg::WN, ty = gt / Cfg::WN;
  const int split = st.split;
  const int rank = task.local % split;
  const int64_t tile = task.local / split;
  const int64_t per_b = int64_t(st.tiles_m) * st.tiles_n;
  const int64_t ntiles = per_b << g.nb;
  const int64_t b = tile / per_b;
  const int64_t tm = (tile % per_b) / st.tiles_n, tn_ = tile % st.tiles_n;
  const int q = task.prime;
  const ModParams mp = a.mods.q[q];
  const int64_t M = int64_t(1) << g.nm, N = int64_t(1) << g.nn, K = int64_t(1) << g.nk;
  // rank r of `split` takes the k chunks [nch r / split, nch (r+1) / split)
  const int64_t nch = K > Cfg::BK ? K / Cfg::BK : 1;
  const int64_t kbeg = nch * rank / split * Cfg::BK;
  const int64_t kend_ = nch * (rank + 1) / split * Cfg::BK;
  const int64_t kstop = kend_ < K ? kend_ : K;
  const Operand A = at_prime(exec_operand(a, g.a_kind, st.a_off), q, mp);
  const Operand B = at_prime(exec_operand(a, g.b_kind, st.b_off), q, mp);
  const Output C = at_prime(Output{a.r0 + 4 * st.c_off, a.r1 ? a.r1 + 8 * st.c_off : nullptr, a.prime_stride}, q);

  Acc acc[TM][TN];
  if constexpr (std::is_same<SR, SrCnt>::value)
    tile_mainloop_counting<Cfg, true, FOLD == kPackedI16>(g, A, B, mp, b, tm, tn_, kbeg, kstop, smem, acc, prepared,
                                                          st.vec);
  else if constexpr (std::is_same<SR, SrI32>::value && FOLD == kPackedI16)
    tile_mainloop_packed<Cfg, true>(g, A, B, b, tm, tn_, kbeg, kstop, *reinterpret_cast<TileSmemP<Cfg>*>(smem), acc,
                                    prepared, st.vec);
  else
    tile_mainloop<SR, Cfg, FOLD, true>(g, A, B, mp, b, tm, tn_, kbeg, kstop, sm, acc, prepared, st.vec);
  tile_merge_groups<SR, Cfg>(acc, reinterpret_cast<Acc*>(smem + tile_merge_off<Cfg>()), mp);

  const uint32_t m0 = static_cast<uint32_t>(tm) * BM, n0 = static_cast<uint32_t>(tn_) * BN;
  const uint32_t cbase = static_cast<uint32_t>(b) << (g.nn + g.nm);
  const uint32_t M32 = 1u << g.nm, N32 = 1u << g.nn;
  static_assert(TN % 4 == 0, "vector epilogue");
  if (a.trace && tid == 0) g_trace_mark[0] = global_ns();
  if (split > 1) {
    // publish this partial tile ([BM][BN], 16-byte stores), then the last
    // CTA of the tile to arrive merges all `split` partial tiles with every
    // thread, four entries at a time
    Acc* part = reinterpret_cast<Acc*>(a.scratch + st.scratch_off) + ((int64_t(q) * ntiles + tile) * split) * (BM * BN);
    if (grp == 0) {
      Acc* mine = part + int64_t(rank) * BM * BN;
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; j += 4) {
          const Acc v[4] = {acc[i][j], acc[i][j + 1], acc[i][j + 2], acc[i][j + 3]};
          SR::st4(mine + (ty * TM + i) * BN + tx * TN + j, v);
        }
    }
    if (!arrive_last(a.arrive + st.arrive_off + int64_t(q) * ntiles + tile, split, s_last)) return;
    if (a.trace && tid == 0) g_trace_mark[1] = global_ns();
    for (int e = 4 * tid; e < BM * BN; e += 4 * kBlock) {
      const uint32_t m = m0 + e / BN, n = n0 + e % BN;
      if (m >= M32 || n >= N32) continue;
      Acc v[4];
      SR::ldcg4(part + e, v);
#pragma unroll 4
      for (int r = 1; r < split; ++r) {
        Acc o[4];
        SR::ldcg4(part + int64_t(r) * BM * BN + e, o);
#pragma unroll
        for (int u = 0; u < 4; ++u) SR::merge(v[u], o[u], mp);
      }
      if (!g.c_identity) {
        // output stored in its consumer's order: 16-byte stores while the two
        // lowest n bits stay the two lowest stored bits, else scattered
        const uint32_t om = ix.offCm[m - m0];
        if (g.nn >= 2 && g.c_pos[0] == 0 && g.c_pos[1] == 1) {
          SR::store4(C, om + ix.offCn[n - n0], v, mp);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (n + u < N32) SR::store(C, om + ix.offCn[n + u - n0], v[u], mp);
        }
      } else if (g.nn >= 2) {
        SR::store4(C, cbase + (m << g.nn) + n, v, mp);  // N >= 4: the 4 entries are in range, 16-byte aligned
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (n + u < N32) SR::store(C, cbase + (m << g.nn) + n + u, v[u], mp);
      }
    }
    return;
  }
  if (a.trace && tid == 0) g_trace_mark[1] = global_ns();
  if (grp != 0) return;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const uint32_t m = m0 + ty * TM + i;
    if (m >= M32) continue;
#pragma unroll
    for (int j = 0; j < TN; j += 4) {
      const uint32_t n = n0 + tx * TN + j;
      const Acc v[4] = {acc[i][j], acc[i][j + 1], acc[i][j + 2], acc[i][j + 3]};
      if (!g.c_identity) {
        const uint32_t om = ix.offCm[m - m0];
        if (g.nn >= 2 && g.c_pos[0] == 0 && g.c_pos[1] == 1) {
          if (n < N32) SR::store4(C, om + ix.offCn[n - n0], v, mp);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (n + u < N32) SR::store(C, om + ix.offCn[n + u - n0], v[u], mp);
        }
      } else if (g.nn >= 2) {
        if (n < N32) SR::store4(C, cbase + (m << g.nn) + n, v, mp);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (n + u < N32) SR::store(C, cbase + (m << g.nn) + n + u, v[u], mp);
      }
    }
  }
}

template <class SR>
__device__ __forceinline__ void exec_naive_task_q(const ExecArgs& a, const ExecStep& st, const ExecTask& task,
                                                  int q, unsigned char* smem, int* s_last);

// High-k block range [kh0, kh1) of a general-step task (k split `ks`).
__device__ __forceinline__ void naive_task_kh(const ExecStep& st, const ExecTask& task, int32_t* kh0,
                                              int32_t* kh1) {
  const int kl = st.g.nk < kNaiveKLoBits ? st.g.nk : kNaiveKLoBits;
  const int32_t nkhi = 1 << (st.g.nk - kl);
  const int r = task.local % st.ks;
  *kh0 = nkhi / st.ks * r;
  *kh1 = *kh0 + nkhi / st.ks;
}

// Outputs [c0, c1) of a mod-p general step for primes q0 .. q0+NP-1 in one
// pass: every term's residues of all NP primes are loaded together.  The
// step's tables must be in shared memory (they do not depend on the prime).
template <int NP>
__device__ __forceinline__ void exec_naive_mp(const ExecArgs& a, const ExecStep& st, int32_t c0, int32_t c1,
                                              int32_t kh0, int32_t kh1, bool whole, int q0, unsigned char* smem,
                                              unsigned char* gsm) {
  using SRN = SrModN<NP>;
  auto& sm = *reinterpret_cast<NaiveSmem<SRN>*>(smem);
  const StepGeom& g = st.g;
  ModParamsN<NP> mp;
  const uint32_t* pa[NP];
  const uint32_t* pb[NP];
  uint32_t* pc[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    mp.q[q] = a.mods.q[q0 + q];
    const int64_t off = int64_t(q0 + q) * a.prime_stride;
    pa[q] = g.a_kind == kOpShared ? reinterpret_cast<const uint32_t*>(gsm + st.a_off) + (int64_t(q0 + q) << g.ra)
                                  : reinterpret_cast<const uint32_t*>(a.r0 + 4 * st.a_off) + off;
    pb[q] = g.b_kind == kOpShared ? reinterpret_cast<const uint32_t*>(gsm + st.b_off) + (int64_t(q0 + q) << g.rb)
                                  : reinterpret_cast<const uint32_t*>(a.r0 + 4 * st.b_off) + off;
    pc[q] = st.c_shared ? reinterpret_cast<uint32_t*>(gsm + st.c_off) + (int64_t(q0 + q) << g.rc)
                        : reinterpret_cast<uint32_t*>(a.r0 + 4 * st.c_off) + off;
  }
  auto la = [&](uint32_t e) {
    ModValN<NP> v;
    if (g.a_kind == kOpShared) {
#pragma unroll
      for (int q = 0; q < NP; ++q) v.v[q] = pa[q][e];
      return v;
    }
    if (g.a_kind != kOpArena) return SRN::leaf(g.a_kind, e, mp);
#pragma unroll
    for (int q = 0; q < NP; ++q) v.v[q] = __ldcg(pa[q] + e);
    return v;
  };
  auto lb = [&](uint32_t e) {
    ModValN<NP> v;
    if (g.b_kind == kOpShared) {
#pragma unroll
      for (int q = 0; q < NP; ++q) v.v[q] = pb[q][e];
      return v;
    }
    if (g.b_kind != kOpArena) return SRN::leaf(g.b_kind, e, mp);
#pragma unroll
    for (int q = 0; q < NP; ++q) v.v[q] = __ldcg(pb[q] + e);
    return v;
  };
  auto sink = [&](uint32_t c, const ModAccN<NP>& v) {
    const uint32_t o = out_offset(g, sm.gt, c);
#pragma unroll
    for (int q = 0; q < NP; ++q) pc[q][o] = barrett64(v.a[q], mp.q[q]);
  };
  if (!whole && st.R == 1 && (c1 - c0) % (kNaiveWideU * kBlock) == 0 && st.chunk % (kNaiveWideU * kBlock) == 0)
    naive_chunk_wide<SRN, kNaiveWideU>(g, la, lb, sink, mp, c0, c1, sm);
  else
    naive_chunk<SRN>(g, la, lb, sink, mp, c0, c1, kh0, kh1, st.R, sm);
}

// Every prime of a mod-p general step (k not split), in groups of up to 4.
__device__ __forceinline__ void exec_naive_all_primes(const ExecArgs& a, const ExecStep& st, int32_t c0,
                                                      int32_t c1, int32_t kh0, int32_t kh1, bool whole,
                                                      unsigned char* smem, unsigned char* gsm) {
  for (int q0 = 0; q0 < a.nprimes; q0 += 4) {
    switch (a.nprimes - q0 < 4 ? a.nprimes - q0 : 4) {
      case 1: exec_naive_mp<1>(a, st, c0, c1, kh0, kh1, whole, q0, smem, gsm); break;
      case 2: exec_naive_mp<2>(a, st, c0, c1, kh0, kh1, whole, q0, smem, gsm); break;
      case 3: exec_naive_mp<3>(a, st, c0, c1, kh0, kh1, whole, q0, smem, gsm); break;
      default: exec_naive_mp<4>(a, st, c0, c1, kh0, kh1, whole, q0, smem, gsm); break;
    }
  }
}

template <class SR>
__device__ __noinline__ void exec_naive_task(const ExecArgs& a, const ExecStep& st, const ExecTask& task,
                                             unsigned char* smem, int* s_last, bool prepared) {
  auto& sm = *reinterpret_cast<NaiveSmem<SR>*>(smem);
  int32_t kh0, kh1;
  naive_task_kh(st, task, &kh0, &kh1);
  if (!prepared) naive_tables<SR>(st.g, sm, kh0, kh1);
  if constexpr (std::is_same<SR, SrMod>::value) {
    if (task.prime < 0) {  // k is not split: all primes in one pass
      const int32_t E = 1 << st.g.rc, chunk = static_cast<int32_t>(st.chunk);
      const int32_t c0 = task.local * chunk, c1 = c0 + chunk < E ? c0 + chunk : E;
      exec_naive_all_primes(a, st, c0, c1, kh0, kh1, false, smem, nullptr);
      return;
    }
  }
  // one prime, or every prime in turn (one inlined copy of the body)
  const int q0 = task.prime >= 0 ? task.prime : 0, q1 = task.prime >= 0 ? task.prime + 1 : a.nprimes;
  for (int q = q0; q < q1; ++q) exec_naive_task_q<SR>(a, st, task, q, smem, s_last);
}

template <class SR>
__device__ __forceinline__ void exec_naive_task_q(const ExecArgs& a, const ExecStep& st, const ExecTask& task,
                                                  int q, unsigned char* smem, int* s_last) {
  using Acc = typename SR::Acc;
  auto& sm = *reinterpret_cast<NaiveSmem<SR>*>(smem);
  const StepGeom& g = st.g;
  const ModParams mp = a.mods.q[q];
  const Operand A = at_prime(exec_operand(a, g.a_kind, st.a_off), q, mp);
  const Operand B = at_prime(exec_operand(a, g.b_kind, st.b_off), q, mp);
  const Output C = at_prime(Output{a.r0 + 4 * st.c_off, a.r1 ? a.r1 + 8 * st.c_off : nullptr, a.prime_stride}, q);
  const int32_t E = 1 << g.rc;
  const int ks = st.ks;
  const int32_t chunk = static_cast<int32_t>(st.chunk);
  const int32_t chunk_id = task.local / ks;
  const int r = task.local % ks;
  const int32_t c0 = chunk_id * chunk;
  const int32_t c1 = c0 + chunk < E ? c0 + chunk : E;
  int32_t kh0, kh1;
  naive_task_kh(st, task, &kh0, &kh1);
  auto la = [&](uint32_t e) { return SR::template load<true>(A, e); };
  auto lb = [&](uint32_t e) { return SR::template load<true>(B, e); };
  if (a.trace && threadIdx.x == 0) g_trace_mark[0] = global_ns();
  // k split: partial results to scratch, and the last CTA of the chunk
  // merges them; else the results go to the output
  Acc* part = reinterpret_cast<Acc*>(a.scratch + st.scratch_off) +
              (int64_t(q) * st.nchunks + chunk_id) * ks * st.chunk;
  auto sink = [&](uint32_t c, const Acc& v) {
    if (ks == 1) SR::store(C, out_offset(g, sm.gt, c), v, mp);
    else part[r * chunk + (static_cast<int32_t>(c) - c0)] = v;
  };
  if (ks == 1 && st.R == 1 && chunk % (kNaiveWideU * kBlock) == 0)
    naive_chunk_wide<SR, kNaiveWideU>(g, la, lb, sink, mp, c0, c1, sm);
  else
    naive_chunk<SR>(g, la, lb, sink, mp, c0, c1, kh0, kh1, st.R, sm);
  if (ks == 1) {
    if (a.trace && threadIdx.x == 0) g_trace_mark[1] = global_ns();
    return;
  }
  if constexpr (IsKBest<SR>::value) return;  // planned without k splits
  if (!arrive_last(a.arrive + st.arrive_off + int64_t(q) * st.nchunks + chunk_id, ks, s_last)) return;
  if (a.trace && threadIdx.x == 0) g_trace_mark[1] = global_ns();
  if (chunk * ks <= kBlock && ks <= 32) {
    // one partial per thread, merged across the ks lanes of each entry
    const int cl = threadIdx.x / ks, rr = threadIdx.x % ks;
    const int32_t c = c0 + cl;
    Acc v = SR::zero(mp);
    if (cl < chunk && c < c1) v = ldcg_acc(part + rr * chunk + cl);
    for (int off = ks / 2; off >= 1; off >>= 1) {
      Acc o = shfl_xor_val(v, off);
      SR::merge(v, o, mp);
    }
    if (rr == 0 && cl < chunk && c < c1) SR::store(C, out_offset(g, sm.gt, static_cast<uint32_t>(c)), v, mp);
    return;
  }
  if (chunk == 1) {
    // one entry (a step summing every label, e.g. the last one) from many
    // partials: every thread merges a strided share, then warps and the CTA
    Acc v = SR::zero(mp);
    for (int rr = threadIdx.x; rr < ks; rr += kBlock) SR::merge(v, ldcg_acc(part + rr), mp);
    for (int off = 16; off >= 1; off >>= 1) {
      Acc o = shfl_xor_val(v, off);
      SR::merge(v, o, mp);
    }
    if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kBlock / 32; ++w) SR::merge(v, sm.red[w], mp);
      SR::store(C, out_offset(g, sm.gt, static_cast<uint32_t>(c0)), v, mp);
    }
    return;
  }
  for (int32_t c = c0 + threadIdx.x; c < c1; c += kBlock) {
    Acc v = ldcg_acc(part + (c - c0));
#pragma unroll 4
    for (int rr = 1; rr < ks; ++rr) SR::merge(v, ldcg_acc(part + rr * chunk + (c - c0)), mp);
    SR::store(C, out_offset(g, sm.gt, static_cast<uint32_t>(c)), v, mp);
  }
}

// Copies the scalar of a network (the output of its last step) into raw
// result slot `slot` (a single contraction uses slot 0; a batch one per
// network).
// All outputs of one general step over its whole k range (a member of a
// group of tiny steps).
template <class SR>
__device__ __forceinline__ void exec_naive_whole(const ExecArgs& a, const ExecStep& st, int q, unsigned char* smem,
                                                 unsigned char* gsm) {
  auto& sm = *reinterpret_cast<NaiveSmem<SR>*>(smem);
  const StepGeom& g = st.g;
  const int kl = g.nk < kNaiveKLoBits ? g.nk : kNaiveKLoBits;
  const int32_t nkhi = 1 << (g.nk - kl);
  naive_tables<SR>(g, sm, 0, nkhi);
  const ModParams mp = a.mods.q[q];
  const Operand A = at_prime(exec_operand_g(a, g.a_kind, st.a_off, g.ra, gsm), q, mp);
  const Operand B = at_prime(exec_operand_g(a, g.b_kind, st.b_off, g.rb, gsm), q, mp);
  const Output C = at_prime(exec_output_g(a, st, gsm), q);
  auto la = [&](uint32_t e) { return SR::template load<true>(A, e); };
  auto lb = [&](uint32_t e) { return SR::template load<true>(B, e); };
  auto sink = [&](uint32_t c, const typename SR::Acc& v) { SR::store(C, out_offset(g, sm.gt, c), v, mp); };
  naive_chunk<SR>(g, la, lb, sink, mp, 0, 1 << g.rc, 0, nkhi, st.R, sm);
}

// Byte offset of a group task's tensors in dynamic shared memory (after the
// general-step tables).
template <class SR>
constexpr size_t group_smem_off() {
  size_t t = sizeof(NaiveSmem<SR>);
  if (std::is_same<SR, SrMod>::value && sizeof(NaiveSmem<SrModN<4>>) > t) t = sizeof(NaiveSmem<SrModN<4>>);
  return (t + 127) / 128 * 128;
}

// A group of tiny steps, run back to back by this CTA: barriers between the
// steps make each step's outputs visible to the next; internal tensors that
// fit live in shared memory after the tables.
template <class SR>
__device__ __noinline__ void exec_group_task(const ExecArgs& a, const ExecTask& task, ExecStep*,
                                             unsigned char* smem) {
  const int b0 = a.group_begin[task.local], b1 = a.group_begin[task.local + 1];
  unsigned char* gsm = smem + group_smem_off<SR>();
  // every member's step record, copied together (one round of loads)
  ExecStep* recs = reinterpret_cast<ExecStep*>(gsm + kGroupSmem);
  constexpr int kWords = static_cast<int>(sizeof(ExecStep) / 4);
  for (int w = threadIdx.x; w < (b1 - b0) * kWords; w += kBlock) {
    const int i = w / kWords;
    reinterpret_cast<int32_t*>(recs + i)[w % kWords] =
        __ldg(reinterpret_cast<const int32_t*>(a.steps + a.group_members[b0 + i]) + w % kWords);
  }
  for (int i = b0; i < b1; ++i) {
    __syncthreads();
    ExecStep* s_step = recs + (i - b0);
    if (task.prime >= 0) {
      exec_naive_whole<SR>(a, *s_step, task.prime, smem, gsm);
    } else if constexpr (std::is_same<SR, SrMod>::value) {
      const StepGeom& g = s_step->g;
      const int kl = g.nk < kNaiveKLoBits ? g.nk : kNaiveKLoBits;
      const int32_t nkhi = 1 << (g.nk - kl);
      naive_tables<SR>(g, *reinterpret_cast<NaiveSmem<SR>*>(smem), 0, nkhi);
      exec_naive_all_primes(a, *s_step, 0, 1 << g.rc, 0, nkhi, true, smem, gsm);
    } else {
      for (int q = 0; q < a.nprimes; ++q) {
        __syncthreads();
        exec_naive_whole<SR>(a, *s_step, q, smem, gsm);
      }
    }
  }
}

template <class SR>
__device__ __forceinline__ void exec_final(const ExecArgs& a, const ExecStep& st, int slot) {
  if (threadIdx.x != 0) return;
  unsigned char* raw = a.raw + static_cast<int64_t>(slot) * TN_RAW_BYTES;
  const char* r0 = a.r0 + 4 * st.c_off;
  if constexpr (IsKBest<SR>::value) {
    // k-best: int32 words at raw[0 ..] (the K values, or d), then the K
    // uint64 coefficients at raw + 32
    const typename SR::Acc v = SR::template load<true>(exec_operand(a, kOpArena, st.c_off), 0u);
    if constexpr (std::is_same<SR, SrKMax<SR::kK>>::value) {
#pragma unroll
      for (int t = 0; t < SR::kK; ++t) reinterpret_cast<int32_t*>(raw)[t] = v.v[t];
    } else {
      *reinterpret_cast<int32_t*>(raw) = v.d;
#pragma unroll
      for (int t = 0; t < SR::kK; ++t) reinterpret_cast<uint64_t*>(raw + 32)[t] = v.c[t];
    }
  } else if (a.semiring == TN_TROPICAL_F32 || a.semiring == TN_TROPICAL_I32) {
    *reinterpret_cast<int32_t*>(raw) = __ldcg(reinterpret_cast<const int32_t*>(r0));
  } else if (a.semiring == TN_COUNTING_TROPICAL) {
    *reinterpret_cast<int32_t*>(raw) = __ldcg(reinterpret_cast<const int32_t*>(r0));
    *reinterpret_cast<uint64_t*>(raw + 8) =
        __ldcg(reinterpret_cast<const uint64_t*>(a.r1 + 8 * st.c_off));
  } else {
    for (int q = 0; q < a.nprimes; ++q)
      reinterpret_cast<uint32_t*>(raw + 16)[q] =
          __ldcg(reinterpret_cast<const uint32_t*>(r0) + q * a.prime_stride);
  }
  *reinterpret_cast<uint32_t*>(raw + 96) = ld_relaxed_u32(a.status);
}

// Warps 1..7 build the index tables of the claimed task while warp 0 waits
// for its dependencies (the tables depend on the step's geometry only), so
// that work leaves the critical path.  Barrier 1 spans exactly these 224
// threads; the tables are complete after the CTA-wide barrier that ends the
// wait.
__device__ __forceinline__ void bar_warps_1_7() { asm volatile("bar.sync 1, 224;" ::: "memory"); }

template <class Cfg>
__device__ __forceinline__ void exec_prepare_tile(const ExecStep& st, const ExecTask& task, unsigned char* smem,
                                                  bool same_step) {
  const int64_t tile = task.local / st.split;
  const int64_t per_b = int64_t(st.tiles_m) * st.tiles_n;
  tile_tables<Cfg>(st.g, *reinterpret_cast<TileIdx<Cfg>*>(smem), tile / per_b, (tile % per_b) / st.tiles_n,
                   tile % st.tiles_n, threadIdx.x - 32, kBlock - 32, bar_warps_1_7, same_step);
}

// Index tables of a task (warps 1-7).  same_step: the previous task of this
// CTA belonged to the same step, so its gather tables (and the general
// step's low-k table) are still in shared memory.
template <class SR>
__device__ __noinline__ void exec_prepare(const ExecStep& st, const ExecTask& task, unsigned char* smem,
                                          bool same_step) {
  if (task.kind == kTaskNaive) {
    int32_t kh0, kh1;
    naive_task_kh(st, task, &kh0, &kh1);
    naive_prepare<SR>(st.g, *reinterpret_cast<NaiveSmem<SR>*>(smem), kh0, kh1, threadIdx.x - 32, kBlock - 32,
                      bar_warps_1_7, same_step);
    return;
  }
  if constexpr (IsKBest<SR>::value) return;
  switch (st.tile) {
    case 0: exec_prepare_tile<TileC0>(st, task, smem, same_step); break;
    case 1: exec_prepare_tile<TileC1>(st, task, smem, same_step); break;
    case 2: exec_prepare_tile<TileC2>(st, task, smem, same_step); break;
    case 3: exec_prepare_tile<TileC3>(st, task, smem, same_step); break;
    case 4: exec_prepare_tile<TileC4>(st, task, smem, same_step); break;
    default: exec_prepare_tile<TileC5>(st, task, smem, same_step); break;
  }
}

template <class SR, int FOLD>
__global__ void __launch_bounds__(kBlock, 2) k_exec(const __grid_constant__ ExecArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ExecStep s_step;
  __shared__ ExecTask s_task;
  __shared__ int s_t, s_abort, s_last;
  __shared__ unsigned long long s_tr[3];  // trace: claimed, records loaded, ready (thread 0)
  const int tid = threadIdx.x;
  // exec step whose record is in s_step and whose index tables are in
  // shared memory (-1: none, e.g. after a group task)
  int cur_step = -1;
  if (tid == 0) s_abort = 0;
  if (a.epoch) {
    unsigned long long* gate = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(a.ws) + kGateByte);
    if (blockIdx.x == 0) {
      for (int i = tid; i < kGateByte / 4; i += kBlock) a.ws[i] = 0u;
      for (int i = tid; i < a.ctr_words; i += kBlock) a.ws[kHeaderBytes / 4 + i] = 0u;
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(gate), "l"(a.epoch) : "memory");
      }
    }
    if (tid == 0) {
      const unsigned long long t0 = global_ns();
      for (;;) {
        unsigned long long e;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(e) : "l"(gate) : "memory");
        if (e == a.epoch) break;
        // CTA 0 is resident and opens the gate within microseconds; after 2 s
        // (whatever the dependency wait limit) this CTA claims nothing, and
        // the others still complete the contraction
        if (global_ns() - t0 > 2000000000ull) {
          s_abort = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __syncthreads();
    if (s_abort) return;
  }
  for (;;) {
    if (tid == 0) {
      if (a.trace) s_tr[0] = global_ns();
      const int t = atomicAdd(a.task_ctr, 1);
      s_t = t;
      if (t < a.ntasks_total) s_task = a.tasks[t];
    }
    __syncthreads();
    const int t = s_t;
    if (t >= a.ntasks_total) break;
    // consecutive tasks of the same step share the step record and the
    // gather tables, and the step's dependencies were met for the first one
    const bool same_step = s_task.step == cur_step && (s_task.kind == kTaskTile || s_task.kind == kTaskNaive);
    if (!same_step) {
      const int32_t* src = reinterpret_cast<const int32_t*>(a.steps + s_task.step);
      int32_t* dst = reinterpret_cast<int32_t*>(&s_step);
      for (int i = tid; i < static_cast<int>(sizeof(ExecStep) / 4); i += kBlock) dst[i] = __ldg(src + i);
      __syncthreads();
    }
    cur_step = s_task.kind == kTaskGroup ? -1 : s_task.step;
    if (a.trace && tid == 0) s_tr[1] = global_ns();
    const bool prepared = s_task.kind == kTaskNaive || s_task.kind == kTaskTile;
    if (tid >= 32 && prepared) exec_prepare<SR>(s_step, s_task, smem, same_step);
    // wait for the steps this one depends on (warp 0, one dependency per lane)
    if (tid < 32 && !same_step) {
      const bool final_task = s_task.kind == kTaskFinal;
      const int nd = final_task ? 1 : s_step.dep_count;
      bool timed_out = false;
      for (int d0 = 0; d0 < nd; d0 += 32) {
        const int d = d0 + tid;
        if (d < nd) {
          const int2 dp =
              final_task ? make_int2(s_task.step, s_step.done_target) : __ldg(a.deps + s_step.dep_begin + d);
          const unsigned long long t0 = global_ns();
          unsigned ns = 32;
          while (ld_acquire(a.done + dp.x) < dp.y) {
            if (global_ns() - t0 > a.timeout_ns || ld_relaxed_u32(a.status) != 0) {
              timed_out = true;
              break;
            }
            __nanosleep(ns);
            if (ns < 128) ns *= 2;
          }
        }
      }
      timed_out = __any_sync(0xffffffffu, timed_out);
      if (tid == 0 && timed_out) {
        atomicOr(a.status, kStatusTimeout);
        for (int r = 0; r < a.nraw; ++r)
          atomicOr(reinterpret_cast<unsigned int*>(a.raw + static_cast<int64_t>(r) * TN_RAW_BYTES + 96),
                   kStatusTimeout);
        s_abort = 1;
      }
    }
    __syncthreads();
    if (s_abort) break;
    if (a.trace && tid == 0) {
      s_tr[2] = global_ns();
      g_trace_mark[0] = g_trace_mark[1] = 0;
    }
    if (s_task.kind == kTaskFinal) {
      exec_final<SR>(a, s_step, s_task.local);
    } else if (s_task.kind == kTaskNaive) {
      exec_naive_task<SR>(a, s_step, s_task, smem, &s_last, prepared);
    } else if constexpr (IsKBest<SR>::value) {
      // the k-best element types have general steps only
    } else if (s_task.kind == kTaskGroup) {
      exec_group_task<SR>(a, s_task, &s_step, smem);
    } else {
      switch (s_step.tile) {
        case 0:
          if constexpr (ExecTile<SR>::kBig) exec_tile_task<SR, TileC0, FOLD>(a, s_step, s_task, smem, &s_last, prepared);
          break;
        case 1: exec_tile_task<SR, TileC1, FOLD>(a, s_step, s_task, smem, &s_last, prepared); break;
        case 2: exec_tile_task<SR, TileC2, FOLD>(a, s_step, s_task, smem, &s_last, prepared); break;
        case 3: exec_tile_task<SR, TileC3, FOLD>(a, s_step, s_task, smem, &s_last, prepared); break;
        case 4: exec_tile_task<SR, TileC4, FOLD>(a, s_step, s_task, smem, &s_last, prepared); break;
        default: exec_tile_task<SR, TileC5, FOLD>(a, s_step, s_task, smem, &s_last, prepared); break;
      }
    }
    __syncthreads();
    if (tid == 0) {
      const unsigned long long t_body = a.trace ? global_ns() : 0;
      if (s_task.kind != kTaskGroup && s_step.final_slot >= 0) {
        // the network's last step: the CTA that completes it (acquiring the
        // other CTAs' writes) also writes the result block
        int32_t old;
        asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;"
                     : "=r"(old)
                     : "l"(a.done + s_task.step)
                     : "memory");
        if (old + 1 == s_step.done_target) exec_final<SR>(a, s_step, s_step.final_slot);
      } else {
        // release: the CTA's writes (ordered by the barrier above) become
        // visible to any CTA that acquires the counter
        asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(a.done + s_task.step) : "memory");
      }
      if (a.trace) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        unsigned long long* tr = a.trace + 8 * static_cast<int64_t>(t);
        tr[0] = s_tr[0];
        tr[1] = s_tr[1];
        tr[2] = s_tr[2];
        tr[3] = t_body;
        tr[4] = global_ns();
        tr[5] = (static_cast<unsigned long long>(smid) << 32) | blockIdx.x;
        tr[6] = g_trace_mark[0];
        tr[7] = g_trace_mark[1];
      }
    }
  }
}

template <class SR, int FOLD>
static size_t smem_for() {
  if constexpr (IsKBest<SR>::value) return sizeof(NaiveSmem<SR>);
  size_t t = tile_smem_bytes<SR, TileC1>();
  if constexpr (std::is_same<SR, SrCnt>::value && FOLD == kPackedI16) {
    const size_t packed[] = {tile_smem_bytes_cnt_packed<TileC1>(), tile_smem_bytes_cnt_packed<TileC2>(),
                             tile_smem_bytes_cnt_packed<TileC3>(), tile_smem_bytes_cnt_packed<TileC4>(),
                             tile_smem_bytes_cnt_packed<TileC5>()};
    for (size_t c : packed) t = c > t ? c : t;
  }
  if constexpr (std::is_same<SR, SrI32>::value && FOLD == kPackedI16) {
    const size_t packed[] = {tile_smem_bytes_packed<TileC0>(), tile_smem_bytes_packed<TileC1>(),
                             tile_smem_bytes_packed<TileC2>(), tile_smem_bytes_packed<TileC3>(),
                             tile_smem_bytes_packed<TileC4>(), tile_smem_bytes_packed<TileC5>()};
    for (size_t c : packed) t = c > t ? c : t;
  }
  const size_t cands[] = {ExecTile<SR>::kBig ? tile_smem_bytes<SR, TileC0>() : 0, tile_smem_bytes<SR, TileC2>(),
                          tile_smem_bytes<SR, TileC3>(), tile_smem_bytes<SR, TileC4>(),
                          tile_smem_bytes<SR, TileC5>(), sizeof(NaiveSmem<SR>),
                          std::is_same<SR, SrMod>::value ? sizeof(NaiveSmem<SrModN<4>>) : 0,
                          group_smem_off<SR>() + static_cast<size_t>(kGroupSmem) +
                              sizeof(ExecStep) * kGroupMaxMembers};
  for (size_t c : cands) t = c > t ? c : t;
  return t;
}

// Resident CTAs of one executor instantiation on the current device
// (computed once per instantiation; one GPU per process).
template <class SR, int FOLD>
static int exec_resident(size_t* smem_out) {
  static int resident = 0;
  static size_t smem = 0;
  if (resident == 0) {
    auto kern = k_exec<SR, FOLD>;
    smem = smem_for<SR, FOLD>();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
        cudaSuccess)
      return -1;
    // prefer the largest shared-memory carveout so that two CTAs fit per SM
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int dev, sms, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem) != cudaSuccess)
      return -1;
    resident = sms * (per_sm < 1 ? 1 : per_sm);
  }
  *smem_out = smem;
  return resident;
}

template <class SR, int FOLD>
static int exec_launch_t(ExecPlan* X, const ExecArgs& args, cudaStream_t st) {
  size_t smem;
  const int resident = exec_resident<SR, FOLD>(&smem);
  if (resident < 0) return TN_ECUDA;
  const int grid = resident < args.ntasks_total ? resident : args.ntasks_total;
  X->grid = grid;
  X->smem = smem;
  k_exec<SR, FOLD><<<grid, kBlock, smem, st>>>(args);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ECUDA;
}

}  // namespace dev

}  // namespace tn
