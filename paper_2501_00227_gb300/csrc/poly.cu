// poly.cu -- the independence polynomial I(G, x) = sum_k c_k x^k (Eq. 13,
// Sec. 6.2; the GraphPolynomial property of Sec. 5.3) on the mod-p path.
//
// A prime slot is a pair (p, x): its vertex tensors are W = [1, x mod p]
// (Eq. 7 with e^{beta w} = x) and its edge tensors the 0/1 matrix B of Eq. 6,
// so the contraction of the slot is I(G, x) mod p.  One contraction serves
// up to TN_MAX_PRIMES slots (the executor's multi-prime steps read every
// slot of a term together).
//
// tn_independence_polynomial is the finite-field method that Sec. 6.2 names
// for GraphPolynomial: I is evaluated at the d + 1 points x = 1 .. d + 1
// modulo every prime, c_0 .. c_d mod p follow by Newton interpolation
// (divided differences, then the Newton form expanded into monomials), and
// Garner's CRT recovers each coefficient from its residues.  Every
// evaluation runs in the contraction kernels; only the O(d^2) interpolation
// and the CRT run on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "exec.h"
#include "kernels.h"
#include "tn_internal.h"

using tn::dev::ModTable;

namespace tn {
int make_mod_table_slots(const uint32_t* primes, const uint32_t* xs, int32_t nslots, void* mods);
size_t required_bytes(tn_plan_s* p, tn_semiring_t s, int32_t nprimes);
int contract_enqueue(const tn_plan_s* p, tn_semiring_t s, const ModTable& mods, int32_t nprimes, void* ws,
                     cudaStream_t st, void* d_raw, cudaEvent_t* step_events);
int contract_weighted_raw(tn_plan_s* p, tn_semiring_t s, int32_t problem, const int32_t* ew, const int32_t* vw,
                          const uint32_t* primes, const uint32_t* xs, int32_t nslots, void* d_ws, size_t ws_bytes,
                          cudaStream_t st, unsigned char* raw_out, bool keep, ExecPlan** Xout, uint64_t slice);
int weighted_checks(tn_plan_s* p, tn_semiring_t s, int32_t problem, const int32_t* ew, const int32_t* vw);
}  // namespace tn

namespace {

using namespace tn;

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? TN_OK : TN_ECUDA; }

uint32_t mul_mod(uint32_t a, uint32_t b, uint32_t p) {
  return static_cast<uint32_t>(static_cast<uint64_t>(a) * b % p);
}

// a^(p-2) mod p: the inverse of a != 0 modulo the prime p (Fermat)
uint32_t inv_mod_prime(uint32_t a, uint32_t p) {
  uint32_t r = 1 % p, b = a % p;
  for (uint32_t e = p - 2; e; e >>= 1) {
    if (e & 1) r = mul_mod(r, b, p);
    b = mul_mod(b, b, p);
  }
  return r;
}

// Coefficients (lowest first) of the polynomial of degree <= d through
// (xs[i], ys[i]), i = 0..d, modulo the prime p; the xs distinct mod p.
void newton_interpolate(const std::vector<uint32_t>& xs, const std::vector<uint32_t>& ys, uint32_t p,
                        uint32_t* coeffs) {
  const int n = static_cast<int>(xs.size());
  // consecutive points (x_i = x_0 + i, as used here): every difference
  // x_i - x_{i-j} is j, so one inverse per round
  bool consecutive = true;
  for (int i = 1; i < n && consecutive; ++i) consecutive = xs[i] == xs[0] + static_cast<uint32_t>(i);
  std::vector<uint32_t> dd(ys);  // divided differences f[x_0 .. x_i] after the loop
  for (int j = 1; j < n; ++j) {
    const uint32_t inv_j = consecutive ? inv_mod_prime(static_cast<uint32_t>(j) % p, p) : 0u;
    for (int i = n - 1; i >= j; --i) {
      const uint32_t num = (dd[i] + p - dd[i - 1]) % p;
      const uint32_t inv = consecutive ? inv_j : inv_mod_prime((xs[i] + p - xs[i - j]) % p, p);
      dd[i] = mul_mod(num, inv, p);
    }
  }
  // P(x) = dd[0] + (x - x_0)(dd[1] + (x - x_1)(dd[2] + ...)), expanded from
  // the innermost factor outwards
  std::vector<uint32_t> c(n, 0);
  c[0] = dd[n - 1];
  int deg = 0;
  for (int i = n - 2; i >= 0; --i) {
    // c <- c * (x - x_i) + dd[i]
    const uint32_t neg = (p - xs[i] % p) % p;
    for (int k = deg + 1; k >= 1; --k) c[k] = (c[k - 1] + mul_mod(c[k], neg, p)) % p;
    c[0] = (mul_mod(c[0], neg, p) + dd[i]) % p;
    ++deg;
  }
  std::copy(c.begin(), c.end(), coeffs);
}

// Contract the slots on the stream and read their residues (synchronous).
int contract_slots(tn_plan_s* plan, const uint32_t* primes, const uint32_t* xs, int32_t nslots, void* d_ws,
                   size_t ws_bytes, cudaStream_t st, uint32_t* residues) {
  ModTable mods;
  int rc = make_mod_table_slots(primes, xs, nslots, &mods);
  if (rc) return rc;
  if (ws_bytes < required_bytes(plan, TN_COUNT_MODP, nslots)) return TN_ENOMEM;
  void* d_raw = static_cast<char*>(d_ws) + 64;
  rc = contract_enqueue(plan, TN_COUNT_MODP, mods, nslots, d_ws, st, d_raw, nullptr);
  if (rc) return rc;
  unsigned char raw[TN_RAW_BYTES];
  rc = cuda_rc(cudaMemcpyAsync(raw, d_raw, TN_RAW_BYTES, cudaMemcpyDeviceToHost, st));
  if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
  if (rc) return rc;
  uint32_t flags;
  std::memcpy(&flags, raw + 96, 4);
  if (flags) return TN_ETIMEOUT;
  std::memcpy(residues, raw + 16, 4 * static_cast<size_t>(nslots));
  return TN_OK;
}

// Coefficients c_0 .. c_degree of a polynomial given by an evaluator of
// (prime, point) slots: x = 1 .. degree + 1 per prime, TN_MAX_PRIMES slots
// per call, Newton interpolation per prime, Garner CRT per coefficient.
template <class Eval>
int polynomial_from_slots(Eval eval, const uint32_t* primes, int32_t nprimes, int32_t degree,
                          uint32_t* coeff_residues, uint32_t* coeff_limbs, int32_t* coeff_nlimbs) {
  const int npts = degree + 1;
  const int total = npts * nprimes;
  // slot s = q * npts + i evaluates at x = i + 1 modulo primes[q]
  std::vector<uint32_t> sp(total), sx(total), sy(total);
  for (int q = 0; q < nprimes; ++q)
    for (int i = 0; i < npts; ++i) {
      sp[q * npts + i] = primes[q];
      sx[q * npts + i] = static_cast<uint32_t>(i + 1);
    }
  for (int s0 = 0; s0 < total; s0 += TN_MAX_PRIMES) {
    const int ns = std::min(TN_MAX_PRIMES, total - s0);
    const int rc = eval(sp.data() + s0, sx.data() + s0, ns, sy.data() + s0);
    if (rc) return rc;
  }
  std::vector<uint32_t> res(static_cast<size_t>(npts) * nprimes);  // [coefficient][prime]
  std::vector<uint32_t> c(npts);
  for (int q = 0; q < nprimes; ++q) {
    std::vector<uint32_t> xq(sx.begin() + q * npts, sx.begin() + (q + 1) * npts);
    std::vector<uint32_t> yq(sy.begin() + q * npts, sy.begin() + (q + 1) * npts);
    newton_interpolate(xq, yq, primes[q], c.data());
    for (int k = 0; k < npts; ++k) res[static_cast<size_t>(k) * nprimes + q] = c[k];
  }
  if (coeff_residues) std::copy(res.begin(), res.end(), coeff_residues);
  if (coeff_limbs || coeff_nlimbs) {
    for (int k = 0; k < npts; ++k) {
      uint32_t limbs[TN_POLY_LIMBS];
      const int nl = crt_garner(res.data() + static_cast<size_t>(k) * nprimes, primes, nprimes, limbs, TN_POLY_LIMBS);
      if (nl < 0) return TN_EINVAL;
      if (coeff_limbs) {
        std::memset(coeff_limbs + static_cast<size_t>(k) * TN_POLY_LIMBS, 0, 4 * TN_POLY_LIMBS);
        std::memcpy(coeff_limbs + static_cast<size_t>(k) * TN_POLY_LIMBS, limbs, 4 * static_cast<size_t>(nl));
      }
      if (coeff_nlimbs) coeff_nlimbs[k] = nl;
    }
  }
  return TN_OK;
}

bool prime_ok(uint32_t p) {
  if (p < 3 || p >= (1u << 31)) return false;
  for (uint32_t d = 2; d <= p / d; ++d)
    if (p % d == 0) return false;
  return true;
}

}  // namespace

extern "C" {

int tn_contract_modp_x(tn_plan_t plan, const uint32_t* primes, const uint32_t* xs, int32_t nslots,
                       void* d_workspace, size_t ws_bytes, void* cuda_stream, uint32_t* residues) {
  if (!plan || !d_workspace || !residues || !primes || !xs) return TN_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return TN_EINVAL;
  if (nslots < 1 || nslots > TN_MAX_PRIMES) return TN_EINVAL;
  try {
    return contract_slots(plan, primes, xs, nslots, d_workspace, ws_bytes, static_cast<cudaStream_t>(cuda_stream),
                          residues);
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
}

// Argument checks shared by the polynomial entry points.
static int poly_args_ok(tn_plan_t plan, void* d_workspace, const uint32_t* primes, int32_t nprimes, int32_t degree,
                        int32_t max_degree) {
  if (!plan || !d_workspace || !primes || nprimes < 1 || nprimes > TN_POLY_MAX_PRIMES) return TN_EINVAL;
  if (degree < 0 || degree > max_degree) return TN_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return TN_EINVAL;
  for (int q = 0; q < nprimes; ++q) {
    // degree + 1 distinct points 1 .. degree + 1 modulo every prime
    if (!prime_ok(primes[q]) || static_cast<uint64_t>(degree) + 1 >= primes[q]) return TN_EINVAL;
    for (int r = 0; r < q; ++r)
      if (primes[r] == primes[q]) return TN_EINVAL;
  }
  return TN_OK;
}

int tn_independence_polynomial(tn_plan_t plan, const uint32_t* primes, int32_t nprimes, int32_t degree,
                               void* d_workspace, size_t ws_bytes, void* cuda_stream, uint32_t* coeff_residues,
                               uint32_t* coeff_limbs, int32_t* coeff_nlimbs) {
  int rc = poly_args_ok(plan, d_workspace, primes, nprimes, degree, plan ? plan->n : 0);
  if (rc) return rc;
  try {
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    auto eval = [&](const uint32_t* sp, const uint32_t* sx, int ns, uint32_t* sy) {
      return contract_slots(plan, sp, sx, ns, d_workspace, ws_bytes, st, sy);
    };
    return polynomial_from_slots(eval, primes, nprimes, degree, coeff_residues, coeff_limbs, coeff_nlimbs);
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
}

int tn_weighted_polynomial(tn_plan_t plan, int32_t problem, const int32_t* edge_w, const int32_t* vertex_w,
                           const uint32_t* primes, int32_t nprimes, int32_t degree, void* d_workspace,
                           size_t ws_bytes, void* cuda_stream, uint32_t* coeff_residues, uint32_t* coeff_limbs,
                           int32_t* coeff_nlimbs) {
  int rc = poly_args_ok(plan, d_workspace, primes, nprimes, degree, 1 << 15);
  if (rc) return rc;
  rc = weighted_checks(plan, TN_COUNT_MODP, problem, edge_w, vertex_w);
  if (rc) return rc;
  try {
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    auto eval = [&](const uint32_t* sp, const uint32_t* sx, int ns, uint32_t* sy) {
      unsigned char raw[TN_RAW_BYTES];
      int r = contract_weighted_raw(plan, TN_COUNT_MODP, problem, edge_w, vertex_w, sp, sx, ns, d_workspace,
                                    ws_bytes, st, raw, false, nullptr, 0);
      if (r) return r;
      uint32_t flags;
      std::memcpy(&flags, raw + 96, 4);
      if (flags) return static_cast<int>(TN_ETIMEOUT);
      std::memcpy(sy, raw + 16, 4 * static_cast<size_t>(ns));
      return static_cast<int>(TN_OK);
    };
    return polynomial_from_slots(eval, primes, nprimes, degree, coeff_residues, coeff_limbs, coeff_nlimbs);
  } catch (const std::bad_alloc&) {
    return TN_ENOMEM;
  }
}

}  // extern "C"
