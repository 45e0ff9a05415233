// api.cu -- the extern "C" entry points of libtn (declared in include/tn.h).
//
// A contraction (Sec. 4.1 of arXiv:2501.00227) is the planned list of
// pairwise steps; each is one kernel launch on the caller's stream, all
// intermediates live in the caller's workspace, and the scalar result is
// copied into a small raw block and decoded on the host (Garner CRT for the
// mod-p count).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "exec.h"
#include "kernels.h"
#include "tn_internal.h"

using tn::dev::ModParams;
using tn::dev::ModTable;
using tn::dev::Operand;
using tn::dev::Output;

namespace tn {

void slice_cache_free(tn_plan_s* p);

namespace {

bool semiring_ok(tn_semiring_t s) {
  return s == TN_TROPICAL_F32 || s == TN_TROPICAL_I32 || s == TN_COUNTING_TROPICAL ||
         s == TN_COUNT_MODP;
}

uint64_t gcd64(uint64_t a, uint64_t b) {
  while (b) {
    uint64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

int make_mods(tn_semiring_t s, const uint32_t* primes, int32_t nprimes, ModTable* mt) {
  std::memset(mt, 0, sizeof(*mt));
  mt->q[0].p = 2;  // unused for the non-modular semirings, but well defined
  if (s != TN_COUNT_MODP) return TN_OK;
  if (primes == nullptr || nprimes < 1 || nprimes > TN_MAX_PRIMES) return TN_EINVAL;
  for (int i = 0; i < nprimes; ++i) {
    uint32_t p = primes[i];
    if (p < 2 || p >= (1u << 31)) return TN_EINVAL;
    for (int j = 0; j < i; ++j)
      if (gcd64(p, primes[j]) != 1) return TN_EINVAL;
    mt->q[i].p = p;
    mt->q[i].r32 = static_cast<uint32_t>((uint64_t(1) << 32) % p);
    mt->q[i].mu = ~0ull / p;
    mt->q[i].x = 1;
  }
  return TN_OK;
}

// Prime slots (primes[q], xs[q]) of a weighted mod-p contraction: the moduli
// need not be distinct (several points per prime), only each in [2, 2^31).
int make_mods_slots(const uint32_t* primes, const uint32_t* xs, int32_t nslots, ModTable* mt) {
  std::memset(mt, 0, sizeof(*mt));
  if (primes == nullptr || xs == nullptr || nslots < 1 || nslots > TN_MAX_PRIMES) return TN_EINVAL;
  for (int i = 0; i < nslots; ++i) {
    const uint32_t p = primes[i];
    if (p < 2 || p >= (1u << 31)) return TN_EINVAL;
    mt->q[i].p = p;
    mt->q[i].r32 = static_cast<uint32_t>((uint64_t(1) << 32) % p);
    mt->q[i].mu = ~0ull / p;
    mt->q[i].x = xs[i] % p;
  }
  return TN_OK;
}

struct Regions {
  char* r0;                 // values / residues
  char* r1;                 // counts
  int64_t prime_stride;     // entries between prime blocks
};

Regions regions(const tn_plan_s* p, tn_semiring_t s, void* ws) {
  Regions r;
  size_t e = static_cast<size_t>(p->arena_entries);
  size_t b4 = (4 * e + 255) / 256 * 256;
  r.r0 = static_cast<char*>(ws) + kHeaderBytes;
  r.r1 = (s == TN_COUNTING_TROPICAL) ? r.r0 + b4 : nullptr;
  r.prime_stride = static_cast<int64_t>(b4 / 4);
  return r;
}

Operand operand_of(const tn_plan_s* p, const Regions& rg, int32_t id) {
  const TensorInfo& t = p->tensors[id];
  Operand o;
  std::memset(&o, 0, sizeof(o));
  o.kind = t.kind;
  o.vx = 1;
  if (t.kind == kOpArena) {
    o.p0 = rg.r0 + 4 * t.offset;
    o.p1 = rg.r1 ? rg.r1 + 8 * t.offset : nullptr;
    o.prime_stride = rg.prime_stride;
  }
  return o;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? TN_OK : TN_ECUDA; }

}  // namespace

// Checked modulus table and raw-result decoding for entry points that live
// in other translation units (tn_contract_static).
int make_mod_table_checked(tn_semiring_t s, const uint32_t* primes, int32_t nprimes, void* mods) {
  if (!semiring_ok(s)) return TN_EINVAL;
  return make_mods(s, primes, nprimes, static_cast<ModTable*>(mods));
}
int decode_raw(tn_semiring_t s, const ModTable& mods, int32_t nprimes, const unsigned char* raw,
               tn_result_t* out);
int make_mod_table_slots(const uint32_t* primes, const uint32_t* xs, int32_t nslots, void* mods) {
  return make_mods_slots(primes, xs, nslots, static_cast<ModTable*>(mods));
}
int decode_raw_any(tn_semiring_t s, const void* mods, int32_t nprimes, const unsigned char* raw,
                   tn_result_t* out) {
  return decode_raw(s, *static_cast<const ModTable*>(mods), nprimes, raw, out);
}

// Workspace a contraction needs: the larger of the per-step layout and the
// executor layout (so one buffer serves both paths).
size_t required_bytes(tn_plan_s* p, tn_semiring_t s, int32_t nprimes) {
  int rc;
  ExecPlan* X = exec_plan_get(p, s, nprimes < 1 ? 1 : nprimes, &rc);
  size_t a = workspace_bytes(p, s, nprimes);
  return X ? std::max(a, X->total_bytes) : ~size_t(0);
}

bool executor_enabled() {
  const char* e = getenv("TN_EXEC");
  return !(e && e[0] == '0');
}

int contract_enqueue(const tn_plan_s* p, tn_semiring_t s, const ModTable& mods, int32_t nprimes,
                     void* ws, cudaStream_t st, void* d_raw, cudaEvent_t* step_events) {
  if (!step_events && executor_enabled())
    return exec_enqueue(const_cast<tn_plan_s*>(p), s, &mods, nprimes, ws, ~size_t(0), st, d_raw, nullptr);
  Regions rg = regions(p, s, ws);
  uint32_t* d_status = static_cast<uint32_t*>(ws);
  int rc = cuda_rc(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st));
  if (rc) return rc;
  const int np = s == TN_COUNT_MODP ? nprimes : 1;
  for (size_t i = 0; i < p->steps.size(); ++i) {
    const Step& step = p->steps[i];
    if (step_events) {
      rc = cuda_rc(cudaEventRecord(step_events[2 * i], st));
      if (rc) return rc;
    }
    Operand A = operand_of(p, rg, step.a_id);
    Operand B = operand_of(p, rg, step.b_id);
    Operand Cin = operand_of(p, rg, step.c_id);
    Output C{const_cast<void*>(Cin.p0), const_cast<void*>(Cin.p1), Cin.prime_stride};
    if (s == TN_COUNT_MODP && dev::umma_route_enabled() && dev::umma_step_fits(step.g, A, B))
      rc = dev::umma_step(step.g, A, B, C, mods, np, st);
    else
      rc = dev::launch_step(s, step.g, A, B, C, mods, np, st, nullptr);
    if (rc) return rc;
    if (step_events) {
      rc = cuda_rc(cudaEventRecord(step_events[2 * i + 1], st));
      if (rc) return rc;
    }
  }
  return dev::launch_finalize(s, operand_of(p, rg, p->root), np, d_status, d_raw, st);
}

int decode_raw(tn_semiring_t s, const ModTable& mods, int32_t nprimes, const unsigned char* raw,
               tn_result_t* out) {
  std::memset(out, 0, sizeof(*out));
  out->status = TN_OK;
  uint32_t flags;
  std::memcpy(&flags, raw + 96, 4);
  if (flags) out->status = TN_ETIMEOUT;
  if (s == TN_TROPICAL_F32) {
    float f;
    std::memcpy(&f, raw, 4);
    out->max_f32 = f;
    out->max_i32 = std::isinf(f) ? INT32_MIN : static_cast<int32_t>(f);
  } else if (s == TN_TROPICAL_I32 || s == TN_COUNTING_TROPICAL) {
    int32_t v;
    std::memcpy(&v, raw, 4);
    bool neg_inf = v < TN_I32_NEG_INF / 2;
    out->max_i32 = neg_inf ? INT32_MIN : v;
    out->max_f32 = neg_inf ? -INFINITY : static_cast<float>(v);
    if (s == TN_COUNTING_TROPICAL) {
      std::memcpy(&out->count, raw + 8, 8);
      if (neg_inf) out->count = 0;
      if (out->count == ~0ull && out->status == TN_OK) out->status = TN_EOVERFLOW;
    }
  } else {
    out->nprimes = nprimes;
    for (int q = 0; q < nprimes; ++q) {
      out->primes[q] = mods.q[q].p;
      std::memcpy(&out->residues[q], raw + 16 + 4 * q, 4);
    }
    int nl = crt_garner(out->residues, out->primes, nprimes, out->crt_limbs, 32);
    if (nl < 0) return TN_EINVAL;
    out->crt_nlimbs = nl;
  }
  return TN_OK;
}

}  // namespace tn

using namespace tn;

extern "C" {

int tn_plan(int32_t n_vertices, const int32_t* edges, int32_t m, const int32_t* order,
            int32_t order_len, tn_plan_t* out) {
  if (out == nullptr) return TN_EINVAL;
  *out = nullptr;
  tn_plan_s* p = new (std::nothrow) tn_plan_s();
  if (!p) return TN_ENOMEM;
  int rc;
  try {
    rc = build_plan(n_vertices, edges, m, order, order_len, p);
  } catch (const std::bad_alloc&) {
    rc = TN_ENOMEM;
  }
  if (rc != TN_OK) {
    delete p;
    return rc;
  }
  *out = p;
  return TN_OK;
}

int tn_order_greedy(int32_t n, const int32_t* edges, int32_t m, double alpha, int32_t nrepeat,
                    uint64_t seed, int32_t* order_out) {
  try {
    return greedy_order(n, edges, m, alpha, nrepeat, seed, order_out);
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
}

int tn_plan_info(tn_plan_t plan, tn_semiring_t semiring, int32_t nprimes, tn_plan_info_t* out) {
  if (!plan || !out || !semiring_ok(semiring)) return TN_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->tc = plan->tc;
  out->sc_elems = plan->sc;
  out->rwc = plan->rwc;
  out->log2_tc = plan->tc ? std::log2(static_cast<double>(plan->tc)) : 0.0;
  out->log2_sc = std::log2(static_cast<double>(plan->sc));
  out->log2_rwc = std::log2(static_cast<double>(plan->rwc));
  out->nsteps = static_cast<int32_t>(plan->steps.size());
  // a sliced plan runs only with stored leaves (tn_contract_sliced)
  const bool stored = !plan->sliced.empty();
  auto xplan = [&](tn_semiring_t sk, int* rc) {
    const int np = nprimes < 1 ? 1 : nprimes;
    return stored ? exec_plan_get_h(plan, sk, np, 1, false, rc, false, true) : exec_plan_get(plan, sk, np, rc);
  };
  for (int k = 0; k < 4; ++k) {
    int rc;
    tn_semiring_t sk = static_cast<tn_semiring_t>(k + 1);
    ExecPlan* X = xplan(sk, &rc);
    if (!X) return rc;
    out->peak_bytes[k] = std::max(workspace_bytes(plan, sk, nprimes), X->total_bytes);
  }
  int wide = 0;
  for (const auto& s : plan->steps) {
    int k, t, sp;
    dev::pick_launch(s.g, semiring, nprimes, &k, &t, &sp);
    wide += k != kKernNaive;
  }
  out->nlaunch_steps = wide;
  int rc;
  ExecPlan* X = xplan(semiring, &rc);
  if (!X) return rc;
  out->exec_table_bytes = X->table_bytes;
  out->exec_tasks = static_cast<int32_t>(X->tasks.size());
  out->exec_levels = X->nlevels;
  out->exec_grid = X->grid;
  out->exec_smem = static_cast<int32_t>(X->smem);
  return TN_OK;
}

int tn_contract_async(tn_plan_t plan, tn_semiring_t semiring, const uint32_t* primes,
                      int32_t nprimes, void* d_workspace, size_t ws_bytes, void* cuda_stream,
                      void* d_raw) {
  if (!plan || !semiring_ok(semiring) || !d_workspace || !d_raw || !plan->sliced.empty()) return TN_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return TN_EINVAL;
  ModTable mods;
  int rc = make_mods(semiring, primes, nprimes, &mods);
  if (rc) return rc;
  if (ws_bytes < required_bytes(plan, semiring, nprimes)) return TN_ENOMEM;
  return contract_enqueue(plan, semiring, mods, nprimes, d_workspace,
                          static_cast<cudaStream_t>(cuda_stream), d_raw, nullptr);
}

int tn_result_decode(tn_semiring_t semiring, const uint32_t* primes, int32_t nprimes,
                     const void* h_raw, tn_result_t* out) {
  if (!semiring_ok(semiring) || !h_raw || !out) return TN_EINVAL;
  ModTable mods;
  int rc = make_mods(semiring, primes, nprimes, &mods);
  if (rc) return rc;
  return decode_raw(semiring, mods, nprimes, static_cast<const unsigned char*>(h_raw), out);
}

int tn_contract(tn_plan_t plan, tn_semiring_t semiring, const uint32_t* primes, int32_t nprimes,
                void* d_workspace, size_t ws_bytes, void* cuda_stream, tn_result_t* out) {
  if (!out) return TN_EINVAL;
  void* d_raw = static_cast<char*>(d_workspace) + 64;
  int rc = tn_contract_async(plan, semiring, primes, nprimes, d_workspace, ws_bytes, cuda_stream,
                             d_raw);
  if (rc) return rc;
  unsigned char raw[TN_RAW_BYTES];
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  rc = cuda_rc(cudaMemcpyAsync(raw, d_raw, TN_RAW_BYTES, cudaMemcpyDeviceToHost, st));
  if (rc) return rc;
  rc = cuda_rc(cudaStreamSynchronize(st));
  if (rc) return rc;
  rc = tn_result_decode(semiring, primes, nprimes, raw, out);
  return rc ? rc : out->status == TN_ETIMEOUT ? TN_ETIMEOUT : TN_OK;
}

int tn_contract_timed(tn_plan_t plan, tn_semiring_t semiring, const uint32_t* primes,
                      int32_t nprimes, void* d_workspace, size_t ws_bytes, void* cuda_stream,
                      tn_result_t* out, float* step_ms, int32_t* step_kernel, uint64_t* step_ops) {
  if (!plan || !out || !semiring_ok(semiring) || !d_workspace) return TN_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return TN_EINVAL;
  ModTable mods;
  int rc = make_mods(semiring, primes, nprimes, &mods);
  if (rc) return rc;
  if (ws_bytes < required_bytes(plan, semiring, nprimes)) return TN_ENOMEM;
  const size_t ns = plan->steps.size();
  std::vector<cudaEvent_t> ev(2 * ns, nullptr);
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) { rc = TN_ECUDA; break; }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void* d_raw = static_cast<char*>(d_workspace) + 64;
  unsigned char raw[TN_RAW_BYTES];
  if (!rc) rc = contract_enqueue(plan, semiring, mods, nprimes, d_workspace, st, d_raw, ev.data());
  if (!rc) rc = cuda_rc(cudaMemcpyAsync(raw, d_raw, TN_RAW_BYTES, cudaMemcpyDeviceToHost, st));
  if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
  for (size_t i = 0; i < ns && !rc; ++i) {
    float ms = 0.f;
    if (step_ms) rc = cuda_rc(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
    if (step_ms) step_ms[i] = ms;
    if (step_kernel) {
      int k, t, sp;
      dev::pick_launch(plan->steps[i].g, semiring, nprimes, &k, &t, &sp);
      step_kernel[i] = k;
    }
    if (step_ops) step_ops[i] = plan->steps[i].ops;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (rc) return rc;
  return decode_raw(semiring, mods, nprimes, raw, out);
}

int tn_contract_trace(tn_plan_t plan, tn_semiring_t semiring, const uint32_t* primes,
                      int32_t nprimes, void* d_workspace, size_t ws_bytes, void* cuda_stream,
                      void* d_trace, int32_t* task_step, int32_t* task_kind, int32_t* step_level,
                      tn_result_t* out) {
  if (!plan || !out || !semiring_ok(semiring) || !d_workspace || !d_trace) return TN_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return TN_EINVAL;
  ModTable mods;
  int rc = make_mods(semiring, primes, nprimes, &mods);
  if (rc) return rc;
  if (ws_bytes < required_bytes(plan, semiring, nprimes)) return TN_ENOMEM;
  ExecPlan* X = exec_plan_get(plan, semiring, nprimes, &rc);
  if (!X) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void* d_raw = static_cast<char*>(d_workspace) + 64;
  rc = exec_enqueue(plan, semiring, &mods, nprimes, d_workspace, ws_bytes, st, d_raw, d_trace);
  if (rc) return rc;
  unsigned char raw[TN_RAW_BYTES];
  rc = cuda_rc(cudaMemcpyAsync(raw, d_raw, TN_RAW_BYTES, cudaMemcpyDeviceToHost, st));
  if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
  if (rc) return rc;
  for (size_t t = 0; t < X->tasks.size(); ++t) {
    if (task_step) task_step[t] = X->tasks[t].step;
    if (task_kind) task_kind[t] = X->tasks[t].kind;
  }
  if (step_level)
    for (size_t i = 0; i < X->steps.size(); ++i) step_level[i] = X->step_level[i];
  return decode_raw(semiring, mods, nprimes, raw, out);
}

int tn_contract_pair(tn_semiring_t semiring, const uint32_t* primes, int32_t nprimes,
                     const void* d_a, const int32_t* la, int32_t ra, const void* d_b,
                     const int32_t* lb, int32_t rb, const int32_t* lc, int32_t rc,
                     void* d_c, void* cuda_stream) {
  if (!semiring_ok(semiring) || !d_a || !d_b || !d_c) return TN_EINVAL;
  if (ra < 0 || rb < 0 || rc < 0 || ra > kMaxRank || rb > kMaxRank || rc > kMaxRank) return TN_EINVAL;
  if ((ra && !la) || (rb && !lb) || (rc && !lc)) return TN_EINVAL;
  std::vector<int32_t> LA(la, la + ra), LB(lb, lb + rb), LC(lc, lc + rc);
  for (auto* v : {&LA, &LB, &LC}) {
    std::vector<int32_t> s = *v;
    std::sort(s.begin(), s.end());
    if (std::adjacent_find(s.begin(), s.end()) != s.end()) return TN_EINVAL;
  }
  ModTable mods;
  int r = make_mods(semiring, primes, nprimes, &mods);
  if (r) return r;
  StepGeom g;
  std::vector<int32_t> order_c;
  r = classify_step(LA, LB, LC, &g, &order_c);
  if (r) return r;
  // the caller fixes the stored label order of C: scatter through c_pos
  g.c_identity = 1;
  for (int j = 0; j < g.rc; ++j) {
    int pos = static_cast<int>(std::find(LC.begin(), LC.end(), order_c[j]) - LC.begin());
    g.c_pos[j] = static_cast<int8_t>(pos);
    if (pos != j) g.c_identity = 0;
  }
  g.a_kind = g.b_kind = kOpArena;
  auto counts_at = [semiring](const void* base, int32_t r_) -> const void* {
    if (semiring != TN_COUNTING_TROPICAL) return nullptr;
    int64_t E = int64_t(1) << r_;
    return static_cast<const char*>(base) + 8 * ((E + 1) / 2);
  };
  Operand A{kOpArena, 0, d_a, counts_at(d_a, ra), int64_t(1) << ra};
  Operand B{kOpArena, 0, d_b, counts_at(d_b, rb), int64_t(1) << rb};
  Output C{d_c, const_cast<void*>(counts_at(d_c, rc)), int64_t(1) << rc};
  const int np = semiring == TN_COUNT_MODP ? nprimes : 1;
  return dev::launch_step(semiring, g, A, B, C, mods, np, static_cast<cudaStream_t>(cuda_stream),
                         nullptr);
}

void tn_plan_destroy(tn_plan_t plan) {
  if (!plan) return;
  slice_cache_free(plan);
  exec_plans_free(plan);
  delete plan;
}

const char* tn_strerror(int code) {
  switch (code) {
    case TN_OK: return "ok";
    case TN_EINVAL: return "invalid argument, graph or order";
    case TN_ENOMEM: return "out of memory or workspace too small";
    case TN_EOVERFLOW: return "uint64 count overflow (saturated)";
    case TN_ETIMEOUT: return "a bounded device wait gave up";
    case TN_EAGAIN: return "not finished yet";
    case TN_ECUDA: return "CUDA runtime error";
  }
  return "unknown error";
}

}  // extern "C"
