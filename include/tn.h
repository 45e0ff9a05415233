/*
 * tn.h -- C ABI of libtn, a GB300 (sm_103a) library that contracts the
 * independent-set (IS) tensor network of arXiv:2501.00227 along a pairwise
 * contraction order, in one of several semirings.
 *
 * The method (paper references are to arXiv:2501.00227):
 *   - Sec. 3.2, Eqs. (4)-(8): a graph G = (V, E) becomes a tensor network with
 *     one rank-2 tensor B per edge, B(n_u, n_v) = [[1, 1], [1, 0]] (semiring
 *     one and zero), and one rank-1 tensor W per vertex, W(n_v) = [1, x];
 *     contracting all of them to a scalar gives the partition function.
 *     Leaves are numbered edges first (in the caller's edge order), then
 *     vertices, as in the flattened einsum printed in Sec. 3.2.
 *   - Sec. 4.1: the contraction is a binary tree; each pairwise step
 *     contracts two tensors (a matricised, GEMM-like product).  tc, sc and
 *     rwc measure an order.
 *   - Sec. 4.2.1, Eq. (9): the greedy order.
 *   - Sec. 5.1 (Table 1), Sec. 5.2, Sec. 5.3: the element type selects the
 *     property: tropical (max,+) -> MIS size (SizeMax); counting tropical ->
 *     number of maximum independent sets (CountingMax); ordinary (+,*) at
 *     x = 1 -> number of all independent sets (CountingAll, PartitionFunction
 *     at beta = 0), computed here exactly as residues modulo 31-bit primes
 *     recombined by the Chinese remainder theorem (the finite-field approach
 *     named in Sec. 6.2).
 *
 * Conventions shared by every call:
 *   - All functions return TN_OK (0) or a negative TN_E* code and never abort.
 *   - Graphs are simple and undirected: edges[2*e], edges[2*e+1] are 0-based
 *     vertex ids, u != v, no repeated edge.  Weights are unit weights.
 *   - A contraction order is an SSA list: with T = m + n leaves, step s
 *     (0 <= s < T-1) contracts ids order[2s] and order[2s+1] (both < T+s, each
 *     id consumed once) into the new id T+s.  The labels kept by a step are
 *     the labels of the pair still used by some other live tensor; the last
 *     step yields the scalar.
 *   - A tensor of rank r over labels L[0..r-1] is a dense array of 2^r
 *     entries; entry x is the value at the assignment where label L[j] takes
 *     bit j of x (L[0] is the least significant bit).
 *   - Device buffers and streams belong to the caller.  Plans and servers are
 *     library-owned; a plan is immutable after tn_plan and may be shared by
 *     threads.
 */
#ifndef TN_H
#define TN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define TN_OK         0
#define TN_EINVAL    (-1)   /* malformed graph, order, semiring or argument      */
#define TN_ENOMEM    (-2)   /* host allocation failed or workspace too small      */
#define TN_EOVERFLOW (-3)   /* a uint64 count reached 2^64-1 (saturated)          */
#define TN_ETIMEOUT  (-4)   /* a bounded device wait gave up                      */
#define TN_EAGAIN    (-5)   /* tn_poll: the ticket has not finished yet           */
#define TN_ECUDA     (-6)   /* a CUDA runtime call failed                         */

/* Element types (Table 1 of the paper).  Device layouts of a tensor with E
 * entries:
 *   TN_TROPICAL_F32       float[E]; -inf is IEEE -inf.  Exact for integer
 *                         values below 2^24.
 *   TN_TROPICAL_I32       int32[E]; "-inf" is any value < TN_I32_NEG_INF / 2
 *                         (kernels start every (max,+) accumulation at
 *                         TN_I32_NEG_INF, so values never go below it).
 *   TN_COUNTING_TROPICAL  int32 max[E] (as TN_TROPICAL_I32), then, starting
 *                         at byte offset 8 * ceil(E / 2), uint64 count[E].
 *                         Counts saturate at UINT64_MAX (= overflow).
 *   TN_COUNT_MODP         uint32 residue[nprimes][E] (prime-major); each
 *                         residue is in [0, p). */
typedef enum {
    TN_TROPICAL_F32 = 1,
    TN_TROPICAL_I32 = 2,
    TN_COUNTING_TROPICAL = 3,
    TN_COUNT_MODP = 4,
    /* k-best element types (tn_contract_kbest only; see there) */
    TN_SIZE_MAX_K = 5,
    TN_COUNTING_MAX_K = 6
} tn_semiring_t;

#define TN_I32_NEG_INF (-(1 << 30))
#define TN_MAX_PRIMES 16

typedef struct tn_plan_s *tn_plan_t;
typedef struct tn_server_s *tn_server_t;

/* Complexity of a plan (Sec. 4.1) and the workspace it needs.
 *   tc       = sum over steps of 2^{|LA u LB|}  (semiring multiply-adds)
 *   sc_elems = largest intermediate tensor, in entries
 *   rwc      = sum over steps of 2^|LA| + 2^|LB| + 2^|LC|  (entries)
 *   peak_bytes[k] = device workspace tn_contract needs for semiring k+1
 *                   (for TN_COUNT_MODP: with the nprimes given to
 *                   tn_plan_info). */
typedef struct {
    double log2_tc, log2_sc, log2_rwc;
    uint64_t tc, sc_elems, rwc;
    uint64_t peak_bytes[4];
    int32_t nsteps;
    int32_t nlaunch_steps;   /* steps executed by the tiled (GEMM) kernels */
    uint64_t exec_table_bytes;  /* step/task tables uploaded once per plan and device */
    int32_t exec_tasks;         /* tasks of one executor launch (this semiring) */
    int32_t exec_levels;        /* dependency levels of the steps */
    int32_t exec_grid;          /* CTAs of the last executor launch (0 before the first) */
    int32_t exec_smem;          /* dynamic shared memory per CTA of that launch, bytes */
} tn_plan_info_t;

/* Result of one contraction.
 *   status   TN_OK, or TN_EOVERFLOW when the count saturated.
 *   max_i32  MIS size (tropical and counting); INT32_MIN for -inf.
 *   max_f32  MIS size as float (TN_TROPICAL_F32).
 *   count    number of maximum independent sets (TN_COUNTING_TROPICAL).
 *   residues number of independent sets modulo primes[i] (TN_COUNT_MODP);
 *   crt_limbs the unique value in [0, prod primes) congruent to every
 *            residue, little-endian 32-bit limbs (crt_nlimbs of them). */
typedef struct {
    int32_t status;
    int32_t max_i32;
    float max_f32;
    uint64_t count;
    int32_t nprimes;
    uint32_t primes[TN_MAX_PRIMES];
    uint32_t residues[TN_MAX_PRIMES];
    int32_t crt_nlimbs;
    uint32_t crt_limbs[32];
} tn_result_t;

/* Build a plan from a graph and a complete SSA order (order_len = number of
 * steps = n + m - 1).  Host only; validates graph and order (TN_EINVAL).
 * The plan holds the per-step label classes, the kernel chosen for each
 * step and the offsets of every intermediate in the workspace.  Every tensor
 * of the order has rank <= 30 (2^30 entries) and every step at most 60
 * labels in all, else TN_EINVAL: an order with a larger intermediate needs
 * slicing (tn_plan_sliced) or a better order. */
int tn_plan(int32_t n_vertices, const int32_t *edges, int32_t m,
            const int32_t *order, int32_t order_len, tn_plan_t *out);

/* Greedy order of Sec. 4.2.1: at every step contract the label-sharing pair
 * with the smallest cost 2^|LC| - alpha * (2^|LA| + 2^|LB|) (Eq. 9), ties
 * broken at random from `seed`; nrepeat runs, keep the one with the smallest
 * (sc, tc).  Disconnected pieces are joined by outer products of the two
 * lowest-rank tensors.  order_out: caller-owned, 2 * (n + m - 1) int32. */
int tn_order_greedy(int32_t n, const int32_t *edges, int32_t m, double alpha,
                    int32_t nrepeat, uint64_t seed, int32_t *order_out);

/* Local-search order of Sec. 4.2.2 (TreeSA): simulated annealing over
 * binary contraction trees with the four rewrites (A*B)*C = (A*C)*B =
 * (C*B)*A and A*(B*C) = B*(A*C) = C*(B*A), cost (Eq. 10, on log2 scales)
 *   L = log2 tc + sc_weight * max(0, log2 sc - sc_target) + rw_weight * log2 rwc,
 * Metropolis acceptance min(1, e^{-beta dL}) (Eq. 11) for beta = beta_start,
 * beta_start + beta_step, ... <= beta_stop, niters sweeps over all internal
 * nodes per beta.  ntrials independent trials (host threads, nthreads = 0:
 * one per core), each started from a greedy order (Sec. 4.2.1, one run,
 * its own seed) or, with random_init, a random tree; the best tree seen is
 * returned.  The paper's defaults: sc_target 20, betas 0.01:0.05:15,
 * ntrials 10, niters 50, sc_weight 1, rw_weight 0.2.  order_out: 2 * (n +
 * m - 1) int32 (an SSA order for tn_plan); log2_out (may be NULL): log2 of
 * tc, sc, rwc of that order.
 *
 * tn_order_treesa_sliced: the same annealing with slicing (Sec. 4.2.2,
 * the paper's nslices and fixed_slices): the nfixed labels fixed_slices
 * are sliced from the start, and nslices more are picked while annealing,
 * one at a time after a beta step (the label whose slicing leaves the
 * smallest largest intermediate, ties by the smallest work, as
 * tn_slice_labels), whenever the tree is above sc_target and in any case
 * from the middle of the schedule on, the rest at its end; costs are those
 * of one slice, so the tree keeps adapting to the labels sliced so far.
 * nfixed + nslices <= min(n, 62); fixed_slices distinct labels in [0, n).
 * order_out as above (an order for tn_plan_sliced with sliced_out);
 * sliced_out: nfixed + nslices int32, the fixed labels then the picked
 * ones; log2_out (may be NULL): log2 of the work of all slices together,
 * of the largest intermediate of one slice, and of the reads and writes
 * of all slices together. */
typedef struct {
    double sc_target;
    double beta_start, beta_step, beta_stop;
    int32_t niters;
    int32_t ntrials;
    double sc_weight, rw_weight;
    int32_t random_init;
    int32_t nthreads;
    uint64_t seed;
} tn_treesa_params_t;
int tn_order_treesa(int32_t n, const int32_t *edges, int32_t m, const tn_treesa_params_t *params,
                    int32_t *order_out, double *log2_out);
int tn_order_treesa_sliced(int32_t n, const int32_t *edges, int32_t m, const tn_treesa_params_t *params,
                           int32_t nslices, const int32_t *fixed_slices, int32_t nfixed, int32_t *order_out,
                           int32_t *sliced_out, double *log2_out);

/* Complexity and workspace sizes of a plan; nprimes sizes the mod-p entry. */
int tn_plan_info(tn_plan_t plan, tn_semiring_t semiring, int32_t nprimes, tn_plan_info_t *out);

/* Contract the whole network on the GPU and return the decoded scalar.
 * primes/nprimes: only for TN_COUNT_MODP (1..TN_MAX_PRIMES pairwise coprime
 * moduli in [2, 2^31)).  d_workspace: caller-owned device memory of at least
 * peak_bytes[semiring-1] bytes, 256-byte aligned.  cuda_stream: a
 * cudaStream_t (NULL = legacy default stream).  Enqueues every kernel on the
 * stream, then waits for that stream to finish (one 64-byte device-to-host
 * copy).  Errors: TN_EINVAL (arguments), TN_ENOMEM (workspace too small),
 * TN_ECUDA (launch failure), TN_ETIMEOUT (a device wait gave up); out->status
 * is TN_EOVERFLOW when a count saturated. */
int tn_contract(tn_plan_t plan, tn_semiring_t semiring, const uint32_t *primes, int32_t nprimes,
                void *d_workspace, size_t ws_bytes, void *cuda_stream, tn_result_t *out);

/* As tn_contract, without waiting: enqueues the contraction and a copy of
 * the raw scalar into d_raw (TN_RAW_BYTES bytes of caller device memory).
 * Decode it later (after the stream is done and the bytes are on the host)
 * with tn_result_decode, which returns TN_OK for any finished launch and
 * puts the launch's outcome in out->status: TN_ETIMEOUT when a device wait
 * gave up (the values are then meaningless), TN_EOVERFLOW when a count
 * saturated. */
#define TN_RAW_BYTES 128
int tn_contract_async(tn_plan_t plan, tn_semiring_t semiring, const uint32_t *primes, int32_t nprimes,
                      void *d_workspace, size_t ws_bytes, void *cuda_stream, void *d_raw);
int tn_result_decode(tn_semiring_t semiring, const uint32_t *primes, int32_t nprimes,
                     const void *h_raw, tn_result_t *out);

/* As tn_contract, and also times every step: a CUDA event pair is recorded
 * on the stream around each step's kernels; after the contraction the call
 * waits and writes, for step i, step_ms[i] (milliseconds) and step_kernel[i]
 * (0 = general kernel, 1 = tiled kernel) and step_ops[i] (= 2^{|LA u LB|},
 * semiring multiply-adds per prime).  Arrays hold tn_plan_info().nsteps
 * entries; any of them may be NULL. */
int tn_contract_timed(tn_plan_t plan, tn_semiring_t semiring, const uint32_t *primes, int32_t nprimes,
                      void *d_workspace, size_t ws_bytes, void *cuda_stream, tn_result_t *out,
                      float *step_ms, int32_t *step_kernel, uint64_t *step_ops);

/* Tracing: as tn_contract through the persistent executor, and records for
 * every executor task t, in d_trace[8t .. 8t+7] (caller device memory of
 * 64 * tn_plan_info().exec_tasks bytes): the global timer (ns) when a CTA
 * claimed it [0], when the task and step records were in shared memory [1],
 * when its dependencies were met [2], when its body ended [3] and when its
 * completion was published [4]; then (SM id << 32 | CTA index) [5]; then two
 * phase marks of the body [6], [7] (general chunk: offset tables built,
 * reduction done; GEMM tile: main loop done, final merge or store started;
 * 0 where the task kind has none).  task_step[t], task_kind[t] (0 general
 * chunk, 1 GEMM tile, 2 final copy -- only when the last step runs inside a
 * group of tiny steps; otherwise the task that completes the last step
 * writes the result -- 3 group of tiny steps) and step_level[i]
 * (dependency level of executor step i) describe the schedule; any of the
 * three may be NULL.  Waits for the stream. */
int tn_contract_trace(tn_plan_t plan, tn_semiring_t semiring, const uint32_t *primes, int32_t nprimes,
                      void *d_workspace, size_t ws_bytes, void *cuda_stream, void *d_trace,
                      int32_t *task_step, int32_t *task_kind, int32_t *step_level, tn_result_t *out);

/* One pairwise contraction (Sec. 4.1) on caller device tensors, with the
 * layout conventions above:
 *   C[c] = (+)_{s} A[a(c, s)] (x) B[b(c, s)]
 * where c runs over assignments of the labels LC (every label of LC must be
 * in LA or LB) and s over assignments of the labels of LA u LB not in LC.
 * Ranks ra, rb, rc <= 30.  For TN_COUNT_MODP every prime is processed (the
 * buffers hold nprimes prime-major blocks).  A, B and C must not overlap.
 * Enqueued on cuda_stream; does not wait.  Uses no workspace. */
int tn_contract_pair(tn_semiring_t semiring, const uint32_t *primes, int32_t nprimes,
                     const void *d_a, const int32_t *la, int32_t ra,
                     const void *d_b, const int32_t *lb, int32_t rb,
                     const int32_t *lc, int32_t rc, void *d_c, void *cuda_stream);

/* Weighted evaluation on the mod-p path.  Slot q is the pair (primes[q],
 * xs[q]): the network's vertex tensors become W = [1, xs[q] mod primes[q]]
 * (Eq. 7 with e^{beta w} = x; the edge tensors stay the 0/1 matrix of Eq. 6),
 * so residues[q] = I(G, xs[q]) mod primes[q], where I(G, x) = sum_k c_k x^k
 * is the independence polynomial (Eq. 13, Sec. 6.2; c_k = number of
 * independent sets of size k).  xs[q] = 1 gives the count of all sets.
 * nslots in 1..TN_MAX_PRIMES; moduli in [2, 2^31), repeats allowed (several
 * points per prime).  d_workspace: at least tn_plan_info(plan,
 * TN_COUNT_MODP, nslots).peak_bytes[TN_COUNT_MODP - 1] bytes, 256-byte
 * aligned, caller-owned.  Synchronous (waits for cuda_stream).  Errors:
 * TN_EINVAL, TN_ENOMEM (workspace too small), TN_ECUDA, TN_ETIMEOUT. */
int tn_contract_modp_x(tn_plan_t plan, const uint32_t *primes, const uint32_t *xs, int32_t nslots,
                       void *d_workspace, size_t ws_bytes, void *cuda_stream, uint32_t *residues);

/* The independence polynomial (the GraphPolynomial property of Sec. 5.3, by
 * the finite-field method of Sec. 6.2): I(G, x) is evaluated on the GPU at
 * x = 1 .. degree + 1 modulo every prime (tn_contract_modp_x, up to
 * TN_MAX_PRIMES evaluations per contraction), the coefficients c_0 ..
 * c_degree are interpolated modulo each prime on the host (Newton divided
 * differences), and combined by Garner's CRT.
 *   primes   nprimes distinct primes in [3, 2^31), each > degree + 1;
 *            nprimes in 1..TN_POLY_MAX_PRIMES.  The result is exact when
 *            prod primes > max_k c_k (2^n always suffices).
 *   degree   at least the independence number alpha(G) (the tropical
 *            contraction's result; n always suffices), at most n.
 *   d_workspace  as for tn_contract_modp_x with nslots =
 *            min(TN_MAX_PRIMES, nprimes * (degree + 1)).
 * Outputs (each may be NULL): coeff_residues[k * nprimes + q] = c_k mod
 * primes[q]; coeff_limbs[k * TN_POLY_LIMBS ..] = c_k mod prod primes as
 * little-endian 32-bit limbs (zero-padded), coeff_nlimbs[k] its significant
 * limbs; k = 0 .. degree.  Synchronous; errors as tn_contract_modp_x.
 * (No counterpart in the paper's API: it returns a polynomial object.) */
#define TN_POLY_MAX_PRIMES 32
#define TN_POLY_LIMBS 32
int tn_independence_polynomial(tn_plan_t plan, const uint32_t *primes, int32_t nprimes, int32_t degree,
                               void *d_workspace, size_t ws_bytes, void *cuda_stream,
                               uint32_t *coeff_residues, uint32_t *coeff_limbs, int32_t *coeff_nlimbs);

/* Weighted networks on the same contraction path (the plan, its order and
 * the executor are those of the unit-weight IS network; only the leaf
 * tensors change).  problem:
 *   TN_PROBLEM_INDEPENDENT_SET  vertex weights w_v (Eqs. 5-7 with energy
 *       -sum w_v n_v): tropical = the largest total weight of an independent
 *       set; counting = (that weight, the number of sets reaching it); mod p
 *       = sum_S x^{w(S)} per slot (p, x) (weights >= 0).  edge_w is ignored;
 *       vertex_w NULL means w_v = 1.
 *   TN_PROBLEM_SPIN_GLASS  the spin glass of Eq. 1 (Sec. 2.1.1, Sec. 6.4),
 *       H = sum_E J_ij s_i s_j + sum_V h_i s_i, s = 2n - 1: tropical =
 *       max_sigma -H = -E_min; counting = (-E_min, ground-state
 *       degeneracy) (the paper's CountingMin with the sign flipped); mod p
 *       = sum_sigma y^{H + sum|J| + sum|h|} per slot (p, y).  edge_w = J
 *       (NULL: 1), vertex_w = h (NULL: 0).
 * edge_w[m], vertex_w[n]: host arrays, copied into the workspace every call.
 * Max-plus semirings need sum of |weights| <= 2^28 (2^24 for
 * TN_TROPICAL_F32), else TN_EINVAL.  The leaf tensors are generated on the
 * GPU into the workspace; d_workspace must hold tn_weighted_workspace_bytes
 * (nslots prime slots for mod p; ignored otherwise), 256-byte aligned.
 * tn_contract_weighted is synchronous; for mod p, out holds the slots'
 * residues (no CRT: slots may repeat a prime).  Errors as tn_contract. */
#define TN_PROBLEM_INDEPENDENT_SET 0
#define TN_PROBLEM_SPIN_GLASS 1
int tn_weighted_workspace_bytes(tn_plan_t plan, tn_semiring_t semiring, int32_t nslots, uint64_t *out);
int tn_contract_weighted(tn_plan_t plan, tn_semiring_t semiring, int32_t problem, const int32_t *edge_w,
                         const int32_t *vertex_w, const uint32_t *primes, const uint32_t *xs, int32_t nslots,
                         void *d_workspace, size_t ws_bytes, void *cuda_stream, tn_result_t *out);

/* The generating polynomial of a weighted network, by the finite-field
 * method of tn_independence_polynomial: c_k = the number of independent sets
 * of weight k (IS, weights >= 0), or the number of spin configurations with
 * H = k - sum|J| - sum|h| (spin glass; the exact energy histogram, from which
 * the partition function of Sec. 6.4 follows for any temperature).  degree
 * at least the polynomial's degree (sum of the weights; 2 (sum|J| + sum|h|)
 * for the spin glass), at most 2^15.  Workspace: tn_weighted_workspace_bytes
 * with nslots = min(TN_MAX_PRIMES, nprimes * (degree + 1)).  Outputs and
 * errors as tn_independence_polynomial. */
int tn_weighted_polynomial(tn_plan_t plan, int32_t problem, const int32_t *edge_w, const int32_t *vertex_w,
                           const uint32_t *primes, int32_t nprimes, int32_t degree, void *d_workspace,
                           size_t ws_bytes, void *cuda_stream, uint32_t *coeff_residues, uint32_t *coeff_limbs,
                           int32_t *coeff_nlimbs);

/* One optimal configuration (the SingleConfigMax property of Sec. 5.3,
 * Table 1): the (max,+) int32 contraction of the network (problem, edge_w,
 * vertex_w as for tn_contract_weighted; unit-weight IS when both weight
 * arrays are NULL) with every intermediate kept, then a backward pass on the
 * GPU that fixes, from the root down, each step's summed labels to the
 * first assignment reaching the step's output entry.  value = the maximum
 * (MIS size / largest weight / -E_min); config[v] in {0, 1} for the n
 * vertices (spin s = 2 config - 1 for the spin glass) is a configuration
 * reaching it.  Where several do, which one is returned depends on the
 * order (the lowest-index maximiser of each step).  d_workspace: at least
 * tn_single_config_workspace_bytes (all intermediates of the plan at once,
 * int32), 256-byte aligned.  Synchronous.  Errors as tn_contract_weighted;
 * TN_EINVAL also when no configuration is allowed. */
int tn_single_config_workspace_bytes(tn_plan_t plan, uint64_t *out);
int tn_single_config_max(tn_plan_t plan, int32_t problem, const int32_t *edge_w, const int32_t *vertex_w,
                         void *d_workspace, size_t ws_bytes, void *cuda_stream, int32_t *value, uint8_t *config);

/* Slicing (Sec. 4.2.2): fix s vertex labels, contract the network once per
 * assignment of them (slice k gives sliced label j the value bit j of k),
 * and add the 2^s results in the element type.  Each slice's tensors lose
 * the sliced labels, so the largest intermediate shrinks by up to 2^s, for
 * up to 2^s times the work; slices are independent units (several GPUs take
 * disjoint slice ranges and combine with tn_result_combine).
 *
 * tn_slice_labels: nslices (0..62) labels for the given order, picked one at
 *   a time as the label whose removal leaves the smallest largest
 *   intermediate, ties by the smallest total work.  sliced_out: nslices
 *   int32; log2_out (may be NULL): log2 of the work of all slices together
 *   and log2 of the largest intermediate of one slice.
 * tn_plan_sliced: as tn_plan, with the leaves' sliced labels dropped
 *   (sliced: nsliced distinct vertex labels, at most 62).  Such a plan runs
 *   with stored leaves only: tn_contract, tn_contract_async and
 *   tn_single_config_max reject it with TN_EINVAL.
 * tn_contract_sliced: slices [slice_begin, slice_end) of a sliced plan (any
 *   plan: 0 sliced labels is one slice), arguments and workspace
 *   (tn_weighted_workspace_bytes) as tn_contract_weighted (problem, weights,
 *   prime slots); out = the element type's sum of those slices (mod p:
 *   residues per slot, no CRT).  Synchronous.
 *   Slices run up to 256 per executor launch (one merged plan of that many
 *   copies, cached with the plan) when the workspace holds
 *   tn_sliced_workspace_bytes(plan, semiring, nslots, batch) for the batch;
 *   with less, fewer per launch, down to one slice per launch.
 * tn_result_combine: out = a (+) b in the element type: max (tropical), max
 *   with counts of ties added and saturated at 2^64 - 1 (counting), residues
 *   added mod their slot's prime (mod p; the slots must agree, else
 *   TN_EINVAL). */
int tn_slice_labels(int32_t n, const int32_t *edges, int32_t m, const int32_t *order, int32_t order_len,
                    int32_t nslices, int32_t *sliced_out, double *log2_out);
int tn_plan_sliced(int32_t n_vertices, const int32_t *edges, int32_t m, const int32_t *order, int32_t order_len,
                   const int32_t *sliced, int32_t nsliced, tn_plan_t *out);
int tn_contract_sliced(tn_plan_t plan, tn_semiring_t semiring, int32_t problem, const int32_t *edge_w,
                       const int32_t *vertex_w, const uint32_t *primes, const uint32_t *xs, int32_t nslots,
                       uint64_t slice_begin, uint64_t slice_end, void *d_workspace, size_t ws_bytes,
                       void *cuda_stream, tn_result_t *out);
int tn_result_combine(tn_semiring_t semiring, const tn_result_t *a, const tn_result_t *b, tn_result_t *out);
int tn_sliced_workspace_bytes(tn_plan_t plan, tn_semiring_t semiring, int32_t nslots, int32_t batch, uint64_t *out);

/* Limit of the executor's dependency waits (no counterpart in the paper).
 * Every task of a contraction waits, bounded, for the steps it reads; a wait
 * that runs past the limit gives up, the launch stops claiming tasks and
 * every CTA returns, and the result's status is TN_ETIMEOUT (the workspace
 * is reset by the next launch, so the context stays usable).  ns: the limit
 * for every launch enqueued after this call, at most 60 s; 0 restores the
 * default of 2 s.  Process-wide; CUDA graphs keep the limit they were
 * captured with.  TN_EINVAL above 60 s.  Tests shorten it to make a wait run
 * out without any fault. */
int tn_set_wait_timeout_ns(uint64_t ns);

/* Register-only throughput of the contraction kernels' inner arithmetic,
 * the denominators of their ALU rooflines (no counterpart in the paper):
 * kind 0 = (max,+) int32 multiply-adds (one __viaddmax_s32 each), kind 1 =
 * mod-p multiply-adds (64-bit accumulate of a 32 x 32-bit product, the high
 * word folded back every fourth term), kind 2 = (max,+) multiply-adds on two
 * int16 lanes (one __viaddmax_s16x2 per two terms).  Runs one warm-up and one timed
 * launch of 8 CTAs per SM, 16 independent chains per thread, `iters` terms
 * each (4 .. 2^24); *tops_out = terms per second / 1e12.  Synchronous;
 * allocates and frees a small device buffer. */
int tn_alu_peak(int32_t kind, int32_t iters, void *cuda_stream, double *tops_out);

/* Measured launch shapes.  The paper leaves the kernel schedule to the
 * contraction backend; this table lets an autotuner (tune.py in the Python
 * package) replace the host's estimate for given step shapes.  entries holds
 * count records of 7 int32: (semiring, nb, nm, nn, nk, tile, split), where
 * nb / nm / nn / nk are the numbers of batch, A-only, B-only and summed
 * labels of a pairwise step (Sec. 4.1), tile is 0..5 (0 = 128 x 128, tropical
 * only; 1 = 64 x 64; 2 = 32 x 32; 3 = 16 x 64; 4 = 64 x 16; 5 = 32 x 128) or -1 (general
 * kernel), and split (1..16) is the number of CTAs sharing one output tile
 * along k.  The record applies to steps the host would run as GEMM tiles.
 * count = 0 removes the table.  The table is process-wide; executor plans
 * built before the call are rebuilt on their next use (the old ones are
 * kept until their plan is destroyed).  Returns TN_EINVAL for a malformed
 * record (nothing is changed then). */
int tn_tune_set(const int32_t *entries, int32_t count);

/* Launch report of a plan: for every pairwise step i (plan order) writes 10
 * int32 at out[10 i]: its index in the executor's task order (the step index
 * of tn_contract_trace), its dependency level, kernel (0 general, 1 GEMM
 * tile), tile shape (-1 for the general kernel), split-K (or k split of the
 * general kernel), number of tasks, then nb, nm, nn, nk.  nsteps must equal
 * tn_plan_info().nsteps. */
int tn_plan_step_info(tn_plan_t plan, tn_semiring_t semiring, int32_t nprimes, int32_t *out, int32_t nsteps);

/* Ablation of the tensor cores for the count modulo p (not used by the
 * contraction).  The batched mod-p GEMM of one pairwise step (Sec. 4.1, the
 * ordinary (+,*) ring of Sec. 5.1 modulo each prime):
 *   C[q][b][i][j] = sum_l A[q][b][i][l] * B[q][b][j][l]  mod primes[q]
 * A: nprimes x batch x m x k, B: nprimes x batch x n x k, C: nprimes x batch
 * x m x n, all uint32 residues < primes[q], row-major, caller-owned device
 * memory.  Residues are cut into four 8-bit limbs whose 16 products run as
 * integer tensor-core MMAs (mma.sync u8 x u8 -> s32; tcgen05.mma kind::i8 is
 * not offered for sm_103a), then recombined mod p.  m must be a multiple of
 * 64, n of 32, k of 32; 1 <= batch <= 65535; primes as for tn_contract.
 * TN_EINVAL otherwise.  Enqueued on cuda_stream; does not wait. */
int tn_modp_gemm_limb(const uint32_t *primes, int32_t nprimes, const void *d_a, const void *d_b, void *d_c,
                      int32_t batch, int32_t m, int32_t n, int32_t k, void *cuda_stream);

/* The same product on the 5th-generation tensor cores: tcgen05.mma kind::f16
 * with bf16 limbs (exact integers 0..255), fp32 accumulators in tensor
 * memory, one accumulator per limb diagonal, folded mod p after every 64
 * terms (each accumulator stays below 2^24, so it is exact).  m must be a
 * multiple of 128, n of 64, k of 64, d_c 16-byte aligned; other arguments as
 * for tn_modp_gemm_limb.  Waits for the stream; TN_ETIMEOUT if the tensor
 * cores did not complete within 2 s (the result is then unspecified). */
int tn_modp_gemm_umma(const uint32_t *primes, int32_t nprimes, const void *d_a, const void *d_b, void *d_c,
                      int32_t batch, int32_t m, int32_t n, int32_t k, void *cuda_stream);

/* SizeMax(k) and CountingMax(k) (Sec. 5.3, Table 1) in one contraction.
 *
 * The network of tn_contract (unit vertex weights) is contracted with a
 * k-best element type (the ExtendedTropical{k} and TruncatedPoly{k} elements
 * of Table 1) along the plan's order, in one executor launch:
 *   TN_SIZE_MAX_K      values[0..k-1] = the k largest independent-set sizes,
 *                      each set counted once (so repeated sizes repeat), in
 *                      decreasing order; INT32_MIN where fewer than k sets
 *                      exist.  counts is not used (may be NULL).
 *   TN_COUNTING_MAX_K  values[0] = alpha (the largest size) and counts[t] =
 *                      the number of independent sets of size alpha - t,
 *                      t < k (the k highest coefficients of the independence
 *                      polynomial, Eq. 13); counts saturate at UINT64_MAX.
 * k in 1..TN_KBEST_MAX.  d_workspace: at least tn_kbest_workspace_bytes()
 * bytes, 256-byte aligned, caller-owned; sliced plans are not accepted.
 * Synchronous (waits for cuda_stream).  *status: TN_OK, TN_EOVERFLOW (a count
 * saturated) or TN_ETIMEOUT.  Returns TN_OK, TN_EINVAL, TN_ENOMEM (workspace
 * too small), TN_ECUDA or TN_ETIMEOUT (a dependency wait ran out; the
 * outputs are then unspecified). */
#define TN_KBEST_MAX 4
int tn_kbest_workspace_bytes(tn_plan_t plan, tn_semiring_t semiring, int32_t k, uint64_t *bytes);
int tn_contract_kbest(tn_plan_t plan, tn_semiring_t semiring, int32_t k, void *d_workspace, size_t ws_bytes,
                      void *cuda_stream, int32_t *values, uint64_t *counts, int32_t *status);

/* Contraction without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (or have nothing to pass as a workspace) -- for
 * example code running where another component owns device memory through
 * its own pool, so a plain cudaMalloc could fail or fragment that pool, or
 * latency-critical host loops that must not risk the implicit device-wide
 * synchronisation that cudaMalloc / cudaFree can cause.
 *
 * It behaves like tn_contract, but its whole workspace (executor counters,
 * split-K scratch, intermediate tensors and the plan's step/task tables) is
 * one file-scope device array of TN_STATIC_WORKSPACE_BYTES (64 MiB) that
 * every GPU loading libtn keeps until the process exits.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.  Plans whose needs
 * (tn_plan_info peak_bytes for the semiring plus exec_table_bytes, each
 * rounded up to 256 bytes) exceed the array are rejected with TN_ENOMEM.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the array, which keeps the
 * previous call's contents; each call clears what must start at zero, and
 * calls that overlap on the GPU (concurrent threads or streams) race on it.
 * Enqueues on cuda_stream and waits for it.  Errors as tn_contract's:
 * TN_EINVAL, TN_ENOMEM (beyond the array), TN_ECUDA and TN_ETIMEOUT (a
 * dependency wait ran out; the result is then unspecified); out->status is
 * TN_EOVERFLOW when a count saturated. */
#define TN_STATIC_WORKSPACE_BYTES (64 * 1024 * 1024)
int tn_contract_static(tn_plan_t plan, tn_semiring_t semiring, const uint32_t *primes, int32_t nprimes,
                       void *cuda_stream, tn_result_t *out);

/* Batching: many independent networks contracted by ONE persistent
 * executor launch (the tasks of all networks merged in dependency-level
 * order, so small networks fill the GPU together), optionally replayed from
 * a CUDA graph.  Paper: each network is an ordinary contraction (Sec. 4.1);
 * grouping is a GB300 execution choice.
 *   tn_batch_create    plans: `count` plans (all must outlive the batch);
 *                      one semiring (and prime list) for all.
 *   tn_batch_info      workspace bytes the batch needs, tasks, levels,
 *                      bytes of its device tables.
 *   tn_batch_contract  enqueues the batch on cuda_stream: d_workspace
 *                      (caller device memory, 256-byte aligned), d_raw
 *                      (count * TN_RAW_BYTES of caller device memory; slot i
 *                      receives network i's raw result, decode each with
 *                      tn_result_decode).  Does not wait.
 *   tn_batch_contract_graph  the same, through a CUDA graph captured on the
 *                      first call for this (workspace, raw, stream) and
 *                      replayed on later calls.
 * The device tables are uploaded on the first contraction (library-owned). */
typedef struct tn_batch_s *tn_batch_t;
int tn_batch_create(const tn_plan_t *plans, int32_t count, tn_semiring_t semiring, const uint32_t *primes,
                    int32_t nprimes, tn_batch_t *out);
int tn_batch_info(tn_batch_t batch, uint64_t *workspace_bytes, int32_t *tasks, int32_t *levels,
                  uint64_t *table_bytes);
int tn_batch_contract(tn_batch_t batch, void *d_workspace, size_t ws_bytes, void *cuda_stream, void *d_raw);
int tn_batch_contract_graph(tn_batch_t batch, void *d_workspace, size_t ws_bytes, void *cuda_stream,
                            void *d_raw);
void tn_batch_destroy(tn_batch_t batch);

/* Serving (continuous batching).  A server owns a worker thread, up to
 * max_inflight (1..64) concurrent grouped launches, each on a stream of its
 * own, and an HBM budget.  tn_submit queues a request and returns a ticket at
 * once (TN_ENOMEM if its plan alone exceeds the budget).  Whenever a launch
 * slot is free, the worker takes the oldest pending request and, in arrival
 * order, the other pending requests with the same semiring and primes whose
 * predicted workspaces (tn_plan_info peak_bytes) still fit in the unused
 * budget (up to 512), and runs them as one persistent executor launch, so
 * requests that arrive while others run overlap with them on the device.
 * tn_poll returns TN_EAGAIN until the ticket's result is ready, then TN_OK
 * (the result is handed out once).  The plan must outlive its request. */
int tn_server_create(size_t hbm_budget_bytes, int32_t max_inflight, tn_server_t *out);
int tn_submit(tn_server_t server, tn_plan_t plan, tn_semiring_t semiring, const uint32_t *primes,
              int32_t nprimes, uint64_t *ticket);
int tn_poll(tn_server_t server, uint64_t ticket, tn_result_t *out);
/* Tickets finished since the last call, oldest first (at most max_tickets;
 * *count of them written to tickets).  Each is reported once; its result is
 * then fetched with tn_poll.  Lets a client wait on many requests without
 * polling every outstanding ticket. */
int tn_server_completed(tn_server_t server, uint64_t *tickets, int32_t max_tickets, int32_t *count);

void tn_plan_destroy(tn_plan_t plan);
void tn_server_destroy(tn_server_t server);
const char *tn_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* TN_H */
