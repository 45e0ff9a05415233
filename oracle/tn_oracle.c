/*
 * tn_oracle.c -- plain, slow, CPU-only oracle for the independent-set (IS)
 * tensor network contraction of arXiv:2501.00227.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this file.  It shares no
 * code, header, table or helper with the GPU library under
 * paper_2501_00227_gb300/csrc, and the GPU library never calls it.
 *
 * What it computes (all exact, all integer valued):
 *   - the tensors of the IS network: one edge tensor B per edge (Eq. 6) and
 *     one vertex tensor W per vertex (Eq. 7); leaves are numbered edges first,
 *     then vertices, as in the flattened einsum of Sec. 3.2;
 *   - a pairwise (binary-tree) contraction along a given SSA order, Sec. 4.1:
 *     each step contracts two live tensors into a new one whose labels are
 *     the labels of the pair still used by some other live tensor (the output
 *     of the whole network is a scalar, Sec. 3.2);
 *   - element types (Table 1, Sec. 5.2, Sec. 5.3):
 *       tropical  (max,+), zero = -inf, one = 0                   -> MIS size
 *       counting  (max,+) paired with a count                      -> #MIS
 *       mod-p     ordinary (+,*) reduced modulo a prime p          -> #IS mod p
 *       k-max     the k largest configuration weights (ExtendedTropical{k})
 *                                                                  -> SizeMax(k)
 *       k-poly    the k highest-order terms of the polynomial of
 *                 configuration counts by weight (TruncatedPoly{k}) -> CountingMax(k)
 *   - the complexity measures tc / sc / rwc of a binary order (Sec. 4.1);
 *   - the greedy order of Sec. 4.2.1 (cost Eq. 9 with alpha = 0);
 *   - brute force over all 2^n vertex subsets (definition of an independent
 *     set, Sec. 2.1.1) as an independent second check;
 *   - weighted networks on the same pairwise contraction: vertex-weighted
 *     independent sets and the spin glass of Eq. 1 (Sec. 2.1.1, Sec. 6.4),
 *     with brute-force energy / weight histograms to check them.
 *
 * Representation: a tensor of rank r over labels L[0..r-1] (vertex ids) is a
 * dense array of 2^r entries; entry x holds the value for the assignment in
 * which label L[j] takes the value of bit j of x (L[0] is the least
 * significant bit).
 *
 * Tropical values are int64 with OR_NEG_INF = INT64_MIN standing for -inf.
 * Counting values are (int64 max, unsigned __int128 count); counts saturate
 * at 2^128-1 (never reached by the tests).  Mod-p values are uint64 < p and
 * every operation is a plain `%`.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_NEG_INF INT64_MIN
#define OR_MAX_RANK 128

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2, OR_ETOOBIG = -3 };
enum { OR_TROPICAL = 1, OR_COUNTING = 2, OR_MODP = 3, OR_KMAX = 4, OR_KPOLY = 5 };
#define OR_MAX_K 16

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* element types                                                       */
/* ------------------------------------------------------------------ */

/* tropical (Sec. 5.2): a (+) b = max(a, b); a (x) b = a + b; -inf absorbs */
static int64_t trop_mul(int64_t a, int64_t b) {
    if (a == OR_NEG_INF || b == OR_NEG_INF) return OR_NEG_INF;
    return a + b;
}
static int64_t trop_add(int64_t a, int64_t b) { return a > b ? a : b; }

/* counting tropical (Sec. 5.3, CountingMax): (n, c).
 * (a, c) (x) (b, d) = (a + b, c * d)
 * (a, c) (+) (b, d) = the pair with the larger first component; on a tie the
 *                      counts add.  zero = (-inf, 0), one = (0, 1).          */
typedef struct { int64_t n; u128 c; } cnt_t;

static const u128 U128_MAX = ~(u128)0;

static u128 sat_mul128(u128 a, u128 b) {
    if (a == 0 || b == 0) return 0;
    if (a > U128_MAX / b) return U128_MAX;
    return a * b;
}
static u128 sat_add128(u128 a, u128 b) {
    u128 s = a + b;
    return s < a ? U128_MAX : s;
}
static cnt_t cnt_mul(cnt_t x, cnt_t y) {
    cnt_t r;
    if (x.n == OR_NEG_INF || y.n == OR_NEG_INF) { r.n = OR_NEG_INF; r.c = 0; return r; }
    r.n = x.n + y.n;
    r.c = sat_mul128(x.c, y.c);
    return r;
}
static cnt_t cnt_add(cnt_t x, cnt_t y) {
    if (x.n > y.n) return x;
    if (y.n > x.n) return y;
    cnt_t r; r.n = x.n; r.c = sat_add128(x.c, y.c);
    return r;
}

/* The k-best element types of Table 1 (Sec. 5.3).  k (1..OR_MAX_K) is the
 * `nprimes` argument of the contraction routines; an element is a run of
 * int64 words:
 *   k-max (SizeMax(k), ExtendedTropical{k}): the k largest values of the
 *     multiset of configuration weights, in decreasing order, padded with
 *     -inf.  a (x) b = the k largest of all pairwise sums a_i + b_j;
 *     a (+) b = the k largest of the union of the two multisets.
 *     zero = all -inf, one = [0, -inf, ...].
 *   k-poly (CountingMax(k), TruncatedPoly{k}): word 0 is the highest order d
 *     (-inf: the zero polynomial), then k coefficients (u128, two words each)
 *     of x^d, x^(d-1), ..., x^(d-k+1).  a (x) b = the product polynomial
 *     truncated to its k highest orders; a (+) b = the sum, truncated to the
 *     k highest orders of the larger leading order.  zero = (-inf, 0...),
 *     one = (0, [1, 0, ...]).
 * Counts saturate at 2^128 - 1 (never reached by the tests). */

/* inserts x into the decreasing list v[0..k-1], dropping the smallest */
static void kmax_insert(int64_t *v, int k, int64_t x) {
    if (x == OR_NEG_INF || x <= v[k - 1]) return;
    int j = k - 1;
    while (j > 0 && v[j - 1] < x) { v[j] = v[j - 1]; j--; }
    v[j] = x;
}
static void kmax_mul(const int64_t *a, const int64_t *b, int k, int64_t *r) {
    for (int t = 0; t < k; t++) r[t] = OR_NEG_INF;
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++) kmax_insert(r, k, trop_mul(a[i], b[j]));
}
static void kmax_add_into(int64_t *acc, const int64_t *b, int k) {
    for (int j = 0; j < k; j++) kmax_insert(acc, k, b[j]);
}

/* a k-poly element is k + 1 u128 words: word 0 holds d (as int64), words
 * 1..k the coefficients */
static int64_t kpoly_d(const u128 *p) { return (int64_t)(uint64_t)p[0]; }
static void kpoly_set_zero(u128 *p, int k) {
    memset(p, 0, sizeof(u128) * (size_t)(k + 1));
    p[0] = (u128)(uint64_t)OR_NEG_INF;
}
/* coefficient of x^e in p */
static u128 kpoly_coef(const u128 *p, int k, int64_t e) {
    int64_t d = kpoly_d(p);
    if (d == OR_NEG_INF || e > d || d - e >= k) return 0;
    return p[1 + (d - e)];
}
static void kpoly_mul(const u128 *a, const u128 *b, int k, u128 *r) {
    kpoly_set_zero(r, k);
    if (kpoly_d(a) == OR_NEG_INF || kpoly_d(b) == OR_NEG_INF) return;
    r[0] = (u128)(uint64_t)(kpoly_d(a) + kpoly_d(b));
    for (int t = 0; t < k; t++)
        for (int i = 0; i <= t; i++) r[1 + t] = sat_add128(r[1 + t], sat_mul128(a[1 + i], b[1 + t - i]));
}
static void kpoly_add_into(u128 *acc, const u128 *b, int k) {
    if (kpoly_d(b) == OR_NEG_INF) return;
    u128 r[OR_MAX_K + 1];
    int64_t da = kpoly_d(acc), db = kpoly_d(b), d = da > db ? da : db;
    r[0] = (u128)(uint64_t)d;
    for (int t = 0; t < k; t++) r[1 + t] = sat_add128(kpoly_coef(acc, k, d - t), kpoly_coef(b, k, d - t));
    memcpy(acc, r, sizeof(u128) * (size_t)(k + 1));
}

/* ------------------------------------------------------------------ */
/* the network: leaves and SSA order                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    int rank;
    int32_t labels[OR_MAX_RANK];
    void *data;      /* 2^rank entries of the element type */
} tensor_t;

static size_t elem_size(int kind, int nprimes) {
    if (kind == OR_TROPICAL) return sizeof(int64_t);
    if (kind == OR_COUNTING) return sizeof(cnt_t);
    if (kind == OR_KMAX) return sizeof(int64_t) * (size_t)nprimes;   /* k values */
    if (kind == OR_KPOLY) return sizeof(u128) * (size_t)(nprimes + 1);  /* d, k coefficients */
    return sizeof(uint64_t) * (size_t)nprimes;   /* one residue per prime */
}

/* Checks that the graph is simple (0 <= u,v < n, u != v, no repeated edge). */
static int check_graph(int n, const int32_t *edges, int m) {
    if (n < 1 || m < 0) return OR_EINVAL;
    for (int e = 0; e < m; e++) {
        int u = edges[2 * e], v = edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return OR_EINVAL;
        for (int f = 0; f < e; f++) {
            int a = edges[2 * f], b = edges[2 * f + 1];
            if ((a == u && b == v) || (a == v && b == u)) return OR_EINVAL;
        }
    }
    return OR_OK;
}

/* Checks an SSA order: T = m + n leaves; step s consumes two distinct ids that
 * exist (< T + s) and were not consumed before; it creates id T + s.  A
 * complete order has T - 1 steps. */
static int check_order(int T, const int32_t *order, int nsteps) {
    if (nsteps != T - 1) return OR_EINVAL;
    char *used = calloc((size_t)(2 * T), 1);
    if (!used) return OR_ENOMEM;
    int rc = OR_OK;
    for (int s = 0; s < nsteps && rc == OR_OK; s++) {
        int i = order[2 * s], j = order[2 * s + 1];
        if (i < 0 || j < 0 || i >= T + s || j >= T + s || i == j || used[i] || used[j]) rc = OR_EINVAL;
        else used[i] = used[j] = 1;
    }
    free(used);
    return rc;
}

/* The network being contracted.
 *   IS (Eqs. (5)-(7)): edge tensor B(n_u, n_v) = [[one, one], [one, zero]];
 *     vertex tensor W(n_v) = [one, e^{beta w_v}]: tropical (max,+) w_v,
 *     counting (w_v, 1), mod p x^{w_v} for the prime slot's x (the
 *     independence polynomial of Eq. 13 at x when w = 1).  Integer weights
 *     g_vertex_w (NULL: w_v = 1); g_vertex_x NULL means x = 1 (count of all
 *     sets).
 *   Spin glass (Eq. 1): H(sigma) = sum_E J_ij s_i s_j + sum_V h_i s_i with
 *     s = 2n - 1 in {-1, +1}.  Tropical / counting maximise -H:
 *     B(n_u, n_v) = -J s_u s_v, W(n_v) = -h s_v (counts 1).  Mod p with the
 *     slot's y: B = y^{J s_u s_v + |J|}, W = y^{h s_v + |h|}, so the network
 *     is sum_sigma y^{H(sigma) + sum|J| + sum|h|} (an energy histogram).
 *     g_edge_w = J (NULL: 1), g_vertex_w = h (NULL: 0).
 * Leaves are numbered edges first (index e), then vertices (index v). */
enum { OR_PROBLEM_IS = 0, OR_PROBLEM_SPIN = 1 };
/* set for the duration of one weighted contraction (not reentrant: the
 * oracle is called from one thread at a time) */
static int g_problem = OR_PROBLEM_IS;
static const int32_t *g_edge_w = NULL;
static const int32_t *g_vertex_w = NULL;
static const uint32_t *g_vertex_x = NULL;

/* b^e mod p by repeated multiplication (e >= 0 is small) */
static uint64_t pow_mod_plain(uint64_t b, int64_t e, uint64_t p) {
    uint64_t r = 1 % p;
    b %= p;
    for (int64_t i = 0; i < e; i++) r = r * b % p;
    return r;
}

static int64_t iabs64(int64_t a) { return a < 0 ? -a : a; }

static int make_leaf(tensor_t *t, int kind, const uint32_t *primes, int nprimes, int is_edge,
                     int32_t u, int32_t v, int32_t idx) {
    t->rank = is_edge ? 2 : 1;
    t->labels[0] = u;
    if (is_edge) t->labels[1] = v;
    size_t ne = (size_t)1 << t->rank;
    t->data = malloc(ne * elem_size(kind, nprimes));
    if (!t->data) return OR_ENOMEM;
    for (size_t x = 0; x < ne; x++) {
        /* value as an exponent: -inf marks a forbidden configuration (IS edge
         * n_u = n_v = 1); mod p raises the slot's point to `mexp` */
        int64_t val, mexp;
        if (g_problem == OR_PROBLEM_IS) {
            if (is_edge) {
                val = x == 3 ? OR_NEG_INF : 0;
                mexp = 0;
            } else {
                int64_t w = g_vertex_w ? g_vertex_w[idx] : 1;
                val = x == 1 ? w : 0;
                mexp = val;
                if (kind == OR_MODP && mexp < 0) return OR_EINVAL;
            }
        } else {
            if (is_edge) {
                int64_t J = g_edge_w ? g_edge_w[idx] : 1;
                int64_t su = 2 * (int64_t)(x & 1) - 1, sv = 2 * (int64_t)((x >> 1) & 1) - 1;
                val = -J * su * sv;
                mexp = J * su * sv + iabs64(J);
            } else {
                int64_t h = g_vertex_w ? g_vertex_w[idx] : 0;
                int64_t sv = 2 * (int64_t)x - 1;
                val = -h * sv;
                mexp = h * sv + iabs64(h);
            }
        }
        if (kind == OR_TROPICAL) {
            ((int64_t *)t->data)[x] = val;
        } else if (kind == OR_COUNTING) {
            cnt_t *d = t->data;
            d[x].n = val;
            d[x].c = val == OR_NEG_INF ? 0 : 1;
        } else if (kind == OR_KMAX) {
            int64_t *d = (int64_t *)t->data + x * (size_t)nprimes;
            for (int q = 0; q < nprimes; q++) d[q] = OR_NEG_INF;
            d[0] = val;
        } else if (kind == OR_KPOLY) {
            u128 *d = (u128 *)t->data + x * (size_t)(nprimes + 1);
            kpoly_set_zero(d, nprimes);
            d[0] = (u128)(uint64_t)val;
            d[1] = val == OR_NEG_INF ? 0 : 1;
        } else {
            uint64_t *d = t->data;
            for (int q = 0; q < nprimes; q++) {
                uint64_t pt = g_vertex_x ? g_vertex_x[q] : 1;
                d[x * nprimes + q] = val == OR_NEG_INF ? 0 : pow_mod_plain(pt, mexp, primes[q]);
            }
        }
    }
    return OR_OK;
}

/* position of label l in L[0..r-1], or -1 */
static int find_label(const int32_t *L, int r, int32_t l) {
    for (int j = 0; j < r; j++) if (L[j] == l) return j;
    return -1;
}

/* ------------------------------------------------------------------ */
/* one pairwise contraction (Sec. 4.1):                                */
/*   C[c] = (+)_{s} A[a(c, s)] (x) B[b(c, s)]                          */
/* where c ranges over assignments of the output labels LC and s over  */
/* assignments of the summed labels S = (LA u LB) \ LC.                */
/* ------------------------------------------------------------------ */
static int contract_pair(int kind, const uint32_t *primes, int nprimes,
                         const tensor_t *A, const tensor_t *B, tensor_t *C) {
    int32_t S[2 * OR_MAX_RANK];
    int ns = 0;
    for (int j = 0; j < A->rank; j++)
        if (find_label(C->labels, C->rank, A->labels[j]) < 0) S[ns++] = A->labels[j];
    for (int j = 0; j < B->rank; j++)
        if (find_label(C->labels, C->rank, B->labels[j]) < 0 &&
            find_label(A->labels, A->rank, B->labels[j]) < 0) S[ns++] = B->labels[j];
    if (ns > 40 || C->rank > 34 || A->rank > 34 || B->rank > 34) return OR_ETOOBIG;

    /* offset of each summed-label assignment s into A and into B */
    size_t nsum = (size_t)1 << ns;
    uint64_t *sa = malloc(nsum * sizeof(uint64_t)), *sb = malloc(nsum * sizeof(uint64_t));
    if (!sa || !sb) { free(sa); free(sb); return OR_ENOMEM; }
    for (size_t s = 0; s < nsum; s++) {
        uint64_t oa = 0, ob = 0;
        for (int j = 0; j < ns; j++) {
            if (!((s >> j) & 1)) continue;
            int pa = find_label(A->labels, A->rank, S[j]);
            int pb = find_label(B->labels, B->rank, S[j]);
            if (pa >= 0) oa |= (uint64_t)1 << pa;
            if (pb >= 0) ob |= (uint64_t)1 << pb;
        }
        sa[s] = oa; sb[s] = ob;
    }
    /* position of each output label in A and in B (-1 if absent) */
    int ca[OR_MAX_RANK], cb[OR_MAX_RANK];
    for (int j = 0; j < C->rank; j++) {
        ca[j] = find_label(A->labels, A->rank, C->labels[j]);
        cb[j] = find_label(B->labels, B->rank, C->labels[j]);
    }

    size_t nc = (size_t)1 << C->rank;
    C->data = malloc(nc * elem_size(kind, nprimes));
    if (!C->data) { free(sa); free(sb); return OR_ENOMEM; }

#pragma omp parallel for schedule(static)
    for (long long ci = 0; ci < (long long)nc; ci++) {
        uint64_t c = (uint64_t)ci, ba = 0, bb = 0;
        for (int j = 0; j < C->rank; j++) {
            if (!((c >> j) & 1)) continue;
            if (ca[j] >= 0) ba |= (uint64_t)1 << ca[j];
            if (cb[j] >= 0) bb |= (uint64_t)1 << cb[j];
        }
        if (kind == OR_TROPICAL) {
            const int64_t *a = A->data, *b = B->data;
            int64_t acc = OR_NEG_INF;                      /* zero */
            for (size_t s = 0; s < nsum; s++)
                acc = trop_add(acc, trop_mul(a[ba | sa[s]], b[bb | sb[s]]));
            ((int64_t *)C->data)[c] = acc;
        } else if (kind == OR_COUNTING) {
            const cnt_t *a = A->data, *b = B->data;
            cnt_t acc; acc.n = OR_NEG_INF; acc.c = 0;     /* zero */
            for (size_t s = 0; s < nsum; s++)
                acc = cnt_add(acc, cnt_mul(a[ba | sa[s]], b[bb | sb[s]]));
            ((cnt_t *)C->data)[c] = acc;
        } else if (kind == OR_KMAX) {
            const int64_t *a = A->data, *b = B->data;
            int64_t *acc = (int64_t *)C->data + c * (size_t)nprimes, prod[OR_MAX_K];
            for (int q = 0; q < nprimes; q++) acc[q] = OR_NEG_INF;          /* zero */
            for (size_t s = 0; s < nsum; s++) {
                kmax_mul(a + (ba | sa[s]) * (size_t)nprimes, b + (bb | sb[s]) * (size_t)nprimes, nprimes, prod);
                kmax_add_into(acc, prod, nprimes);
            }
        } else if (kind == OR_KPOLY) {
            const u128 *a = A->data, *b = B->data;
            const size_t w = (size_t)(nprimes + 1);
            u128 *acc = (u128 *)C->data + c * w, prod[OR_MAX_K + 1];
            kpoly_set_zero(acc, nprimes);                                  /* zero */
            for (size_t s = 0; s < nsum; s++) {
                kpoly_mul(a + (ba | sa[s]) * w, b + (bb | sb[s]) * w, nprimes, prod);
                kpoly_add_into(acc, prod, nprimes);
            }
        } else {
            const uint64_t *a = A->data, *b = B->data;
            uint64_t *out = (uint64_t *)C->data + c * nprimes;
            for (int q = 0; q < nprimes; q++) {
                uint64_t p = primes[q], acc = 0;
                for (size_t s = 0; s < nsum; s++) {
                    uint64_t prod = (a[(ba | sa[s]) * nprimes + q] * b[(bb | sb[s]) * nprimes + q]) % p;
                    acc = (acc + prod) % p;
                }
                out[q] = acc;
            }
        }
    }
    free(sa); free(sb);
    return OR_OK;
}

/* Output labels of contracting live tensors i and j: the labels of the pair
 * still used by some other live tensor (the network output is a scalar). */
static void output_labels(const tensor_t *ti, const tensor_t *tj, const int *users, tensor_t *out) {
    out->rank = 0;
    for (int k = 0; k < ti->rank; k++) {
        int32_t l = ti->labels[k];
        int others = users[l] - 1 - (find_label(tj->labels, tj->rank, l) >= 0);
        if (others > 0) out->labels[out->rank++] = l;
    }
    for (int k = 0; k < tj->rank; k++) {
        int32_t l = tj->labels[k];
        if (find_label(ti->labels, ti->rank, l) >= 0) continue;
        if (users[l] - 1 > 0) out->labels[out->rank++] = l;
    }
}

/* Contract the whole network along an SSA order and write the scalar into
 * *result (element type `kind`).  With a single leaf (n = 1, m = 0) the scalar
 * is the (+)-sum of that leaf's entries. */
static int contract_network(int kind, const uint32_t *primes, int nprimes, int n, const int32_t *edges,
                            int m, const int32_t *order, int nsteps, void *result) {
    int rc = check_graph(n, edges, m);
    if (rc) return rc;
    int T = m + n;
    rc = check_order(T, order, nsteps);
    if (rc) return rc;
    if (kind == OR_MODP) {
        if (nprimes < 1) return OR_EINVAL;
        for (int q = 0; q < nprimes; q++) if (primes[q] < 2 || primes[q] >= (1u << 31)) return OR_EINVAL;
    }
    if ((kind == OR_KMAX || kind == OR_KPOLY) && (nprimes < 1 || nprimes > OR_MAX_K)) return OR_EINVAL;
    tensor_t *t = calloc((size_t)(2 * T), sizeof(tensor_t));
    int *users = calloc((size_t)n, sizeof(int));
    if (!t || !users) { free(t); free(users); return OR_ENOMEM; }
    for (int e = 0; e < m && !rc; e++) rc = make_leaf(&t[e], kind, primes, nprimes, 1, edges[2 * e], edges[2 * e + 1], e);
    for (int v = 0; v < n && !rc; v++) rc = make_leaf(&t[m + v], kind, primes, nprimes, 0, v, 0, v);
    for (int i = 0; i < T && !rc; i++) for (int k = 0; k < t[i].rank; k++) users[t[i].labels[k]]++;

    int root = 0;
    for (int s = 0; s < nsteps && !rc; s++) {
        int i = order[2 * s], j = order[2 * s + 1], c = T + s;
        output_labels(&t[i], &t[j], users, &t[c]);
        rc = contract_pair(kind, primes, nprimes, &t[i], &t[j], &t[c]);
        if (rc) break;
        for (int k = 0; k < t[i].rank; k++) users[t[i].labels[k]]--;
        for (int k = 0; k < t[j].rank; k++) users[t[j].labels[k]]--;
        for (int k = 0; k < t[c].rank; k++) users[t[c].labels[k]]++;
        free(t[i].data); t[i].data = NULL;
        free(t[j].data); t[j].data = NULL;
        root = c;
    }
    if (!rc) {
        tensor_t *r = &t[root];
        size_t ne = (size_t)1 << r->rank;          /* rank 0 unless T == 1 */
        if (kind == OR_TROPICAL) {
            int64_t acc = OR_NEG_INF;
            for (size_t x = 0; x < ne; x++) acc = trop_add(acc, ((int64_t *)r->data)[x]);
            *(int64_t *)result = acc;
        } else if (kind == OR_COUNTING) {
            cnt_t acc; acc.n = OR_NEG_INF; acc.c = 0;
            for (size_t x = 0; x < ne; x++) acc = cnt_add(acc, ((cnt_t *)r->data)[x]);
            *(cnt_t *)result = acc;
        } else if (kind == OR_KMAX) {
            int64_t *acc = result;
            for (int q = 0; q < nprimes; q++) acc[q] = OR_NEG_INF;
            for (size_t x = 0; x < ne; x++) kmax_add_into(acc, (int64_t *)r->data + x * (size_t)nprimes, nprimes);
        } else if (kind == OR_KPOLY) {
            u128 *acc = result;
            kpoly_set_zero(acc, nprimes);
            for (size_t x = 0; x < ne; x++) kpoly_add_into(acc, (u128 *)r->data + x * (size_t)(nprimes + 1), nprimes);
        } else {
            for (int q = 0; q < nprimes; q++) {
                uint64_t acc = 0;
                for (size_t x = 0; x < ne; x++) acc = (acc + ((uint64_t *)r->data)[x * nprimes + q]) % primes[q];
                ((uint64_t *)result)[q] = acc;
            }
        }
    }
    for (int i = 0; i < 2 * T; i++) free(t[i].data);
    free(t); free(users);
    return rc;
}

/* ------------------------------------------------------------------ */
/* exported entry points (ctypes)                                      */
/* ------------------------------------------------------------------ */

int or_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int or_check_order(int n, const int32_t *edges, int m, const int32_t *order, int nsteps) {
    int rc = check_graph(n, edges, m);
    return rc ? rc : check_order(m + n, order, nsteps);
}

/* MIS size: *max_out = tropical scalar (INT64_MIN if -inf). */
int or_contract_tropical(int n, const int32_t *edges, int m, const int32_t *order, int nsteps,
                         int64_t *max_out) {
    return contract_network(OR_TROPICAL, NULL, 0, n, edges, m, order, nsteps, max_out);
}

/* (MIS size, number of maximum independent sets); the count is returned as
 * two 64-bit halves of the 128-bit value. */
int or_contract_counting(int n, const int32_t *edges, int m, const int32_t *order, int nsteps,
                         int64_t *max_out, uint64_t *count_lo, uint64_t *count_hi) {
    cnt_t r;
    int rc = contract_network(OR_COUNTING, NULL, 0, n, edges, m, order, nsteps, &r);
    if (!rc) { *max_out = r.n; *count_lo = (uint64_t)r.c; *count_hi = (uint64_t)(r.c >> 64); }
    return rc;
}

/* Number of independent sets modulo each prime (Z at beta = 0, Sec. 5.1). */
int or_contract_modp(int n, const int32_t *edges, int m, const int32_t *order, int nsteps,
                     const uint32_t *primes, int nprimes, uint64_t *residues) {
    return contract_network(OR_MODP, primes, nprimes, n, edges, m, order, nsteps, residues);
}

/* As or_contract_modp with vertex tensors W = [1, xs[q]] in prime slot q:
 * residues[q] = sum over independent sets S of xs[q]^|S|  mod primes[q]. */
int or_contract_modp_x(int n, const int32_t *edges, int m, const int32_t *order, int nsteps,
                       const uint32_t *primes, const uint32_t *xs, int nprimes, uint64_t *residues) {
    g_vertex_x = xs;
    int rc = contract_network(OR_MODP, primes, nprimes, n, edges, m, order, nsteps, residues);
    g_vertex_x = NULL;
    return rc;
}

/* Weighted networks (see make_leaf): problem OR_PROBLEM_IS with vertex
 * weights vertex_w (NULL: 1), or OR_PROBLEM_SPIN with couplings edge_w
 * (NULL: 1) and fields vertex_w (NULL: 0).  kind OR_TROPICAL -> *trop;
 * OR_COUNTING -> (*cnt_n, count as lo/hi 64-bit halves); OR_MODP -> one
 * residue per slot (primes[q], xs[q]) (xs NULL: x = 1). */
int or_contract_weighted(int kind, int problem, int n, const int32_t *edges, int m, const int32_t *edge_w,
                         const int32_t *vertex_w, const int32_t *order, int nsteps, const uint32_t *primes,
                         const uint32_t *xs, int nprimes, int64_t *trop, int64_t *cnt_n, uint64_t *cnt_lo,
                         uint64_t *cnt_hi, uint64_t *residues) {
    if (problem != OR_PROBLEM_IS && problem != OR_PROBLEM_SPIN) return OR_EINVAL;
    g_problem = problem;
    g_edge_w = edge_w;
    g_vertex_w = vertex_w;
    g_vertex_x = xs;
    int rc;
    if (kind == OR_TROPICAL) {
        rc = contract_network(OR_TROPICAL, NULL, 0, n, edges, m, order, nsteps, trop);
    } else if (kind == OR_COUNTING) {
        cnt_t r;
        rc = contract_network(OR_COUNTING, NULL, 0, n, edges, m, order, nsteps, &r);
        if (!rc) { *cnt_n = r.n; *cnt_lo = (uint64_t)r.c; *cnt_hi = (uint64_t)(r.c >> 64); }
    } else {
        rc = contract_network(OR_MODP, primes, nprimes, n, edges, m, order, nsteps, residues);
    }
    g_problem = OR_PROBLEM_IS;
    g_edge_w = g_vertex_w = NULL;
    g_vertex_x = NULL;
    return rc;
}

/* The k-best properties of Sec. 5.3 (Table 1) on the networks of
 * or_contract_weighted (problem, edge_w, vertex_w as there; NULL weights give
 * the unit-weight IS network), along an SSA order, 1 <= k <= OR_MAX_K:
 *   kind OR_KMAX  -> vals[0..k-1]: the k largest total weights over all
 *                    configurations, with multiplicity, decreasing
 *                    (SizeMax(k); INT64_MIN for -inf);
 *   kind OR_KPOLY -> *d: the largest weight, and (c_lo, c_hi)[t]: the number
 *                    of configurations of weight d - t, t < k (CountingMax(k)). */
int or_contract_kbest(int kind, int problem, int n, const int32_t *edges, int m, const int32_t *edge_w,
                      const int32_t *vertex_w, const int32_t *order, int nsteps, int k, int64_t *vals,
                      int64_t *d, uint64_t *c_lo, uint64_t *c_hi) {
    if ((kind != OR_KMAX && kind != OR_KPOLY) || (problem != OR_PROBLEM_IS && problem != OR_PROBLEM_SPIN))
        return OR_EINVAL;
    g_problem = problem;
    g_edge_w = edge_w;
    g_vertex_w = vertex_w;
    int rc;
    if (kind == OR_KMAX) {
        rc = contract_network(OR_KMAX, NULL, k, n, edges, m, order, nsteps, vals);
    } else {
        u128 r[OR_MAX_K + 1];
        rc = k < 1 || k > OR_MAX_K ? OR_EINVAL : contract_network(OR_KPOLY, NULL, k, n, edges, m, order, nsteps, r);
        if (!rc) {
            *d = kpoly_d(r);
            for (int t = 0; t < k; t++) { c_lo[t] = (uint64_t)r[1 + t]; c_hi[t] = (uint64_t)(r[1 + t] >> 64); }
        }
    }
    g_problem = OR_PROBLEM_IS;
    g_edge_w = g_vertex_w = NULL;
    return rc;
}

/* Eq. (1): H(sigma) = sum_E J_ij s_i s_j + sum_V h_i s_i for one spin
 * configuration s in {-1, +1}^n (J NULL: 1, h NULL: 0). */
int64_t or_spin_energy(int n, const int32_t *edges, int m, const int32_t *J, const int32_t *h,
                       const int8_t *spins) {
    int64_t e = 0;
    for (int k = 0; k < m; k++) e += (int64_t)(J ? J[k] : 1) * spins[edges[2 * k]] * spins[edges[2 * k + 1]];
    for (int v = 0; v < n; v++) e += (int64_t)(h ? h[v] : 0) * spins[v];
    return e;
}

/* Brute force over all 2^n spin configurations (n <= 30): hist[H + shift]
 * counts the configurations of each energy, shift = sum |J| + sum |h|,
 * hist has 2 * shift + 1 entries. */
int or_bruteforce_spin(int n, const int32_t *edges, int m, const int32_t *J, const int32_t *h, int64_t shift,
                       uint64_t *hist) {
    if (n < 0 || n > 30) return OR_EINVAL;
    int8_t s[32];
    for (uint64_t c = 0; c < ((uint64_t)1 << n); c++) {
        for (int v = 0; v < n; v++) s[v] = ((c >> v) & 1) ? 1 : -1;
        int64_t e = or_spin_energy(n, edges, m, J, h, s) + shift;
        if (e < 0 || e > 2 * shift) return OR_EINVAL;
        hist[e]++;
    }
    return OR_OK;
}

/* Brute force over all 2^n vertex subsets (n <= 30): hist[w(S)] counts the
 * independent sets S of each total weight w(S) = sum_{v in S} w_v (w_v >= 0;
 * hist has sum w_v + 1 entries). */
int or_bruteforce_weighted_is(int n, const int32_t *edges, int m, const int32_t *w, uint64_t *hist) {
    if (n < 0 || n > 30) return OR_EINVAL;
    for (uint64_t c = 0; c < ((uint64_t)1 << n); c++) {
        int ok = 1;
        for (int k = 0; k < m && ok; k++) ok = !(((c >> edges[2 * k]) & 1) && ((c >> edges[2 * k + 1]) & 1));
        if (!ok) continue;
        int64_t tot = 0;
        for (int v = 0; v < n; v++) if ((c >> v) & 1) tot += w[v];
        hist[tot]++;
    }
    return OR_OK;
}

/* One pairwise contraction on caller tensors (labels as above, LC given). */
static int pair_common(int kind, const uint32_t *primes, int nprimes,
                       const void *a, const int32_t *la, int ra,
                       const void *b, const int32_t *lb, int rb,
                       const int32_t *lc, int rc_, void *c) {
    if (ra < 0 || rb < 0 || rc_ < 0 || ra > 30 || rb > 30 || rc_ > 30) return OR_EINVAL;
    tensor_t A = {0}, B = {0}, C = {0};
    A.rank = ra; B.rank = rb; C.rank = rc_;
    memcpy(A.labels, la, sizeof(int32_t) * (size_t)ra);
    memcpy(B.labels, lb, sizeof(int32_t) * (size_t)rb);
    memcpy(C.labels, lc, sizeof(int32_t) * (size_t)rc_);
    for (int j = 0; j < rc_; j++)
        if (find_label(la, ra, lc[j]) < 0 && find_label(lb, rb, lc[j]) < 0) return OR_EINVAL;
    A.data = (void *)a; B.data = (void *)b;
    int rc = contract_pair(kind, primes, nprimes, &A, &B, &C);
    if (rc) return rc;
    memcpy(c, C.data, ((size_t)1 << rc_) * elem_size(kind, nprimes));
    free(C.data);
    return OR_OK;
}

int or_pair_tropical(const int64_t *a, const int32_t *la, int ra, const int64_t *b, const int32_t *lb, int rb,
                     const int32_t *lc, int rc, int64_t *c) {
    return pair_common(OR_TROPICAL, NULL, 0, a, la, ra, b, lb, rb, lc, rc, c);
}

/* counting pair: values n[], counts as 64-bit inputs; output counts as 128-bit (lo, hi) */
int or_pair_counting(const int64_t *an, const uint64_t *ac, const int32_t *la, int ra,
                     const int64_t *bn, const uint64_t *bc, const int32_t *lb, int rb,
                     const int32_t *lc, int rc, int64_t *cn, uint64_t *c_lo, uint64_t *c_hi) {
    size_t na = (size_t)1 << ra, nb = (size_t)1 << rb, ncc = (size_t)1 << rc;
    cnt_t *A = malloc(na * sizeof(cnt_t)), *B = malloc(nb * sizeof(cnt_t)), *C = malloc(ncc * sizeof(cnt_t));
    int r = OR_ENOMEM;
    if (A && B && C) {
        for (size_t x = 0; x < na; x++) { A[x].n = an[x]; A[x].c = ac[x]; }
        for (size_t x = 0; x < nb; x++) { B[x].n = bn[x]; B[x].c = bc[x]; }
        r = pair_common(OR_COUNTING, NULL, 0, A, la, ra, B, lb, rb, lc, rc, C);
        if (!r) for (size_t x = 0; x < ncc; x++) { cn[x] = C[x].n; c_lo[x] = (uint64_t)C[x].c; c_hi[x] = (uint64_t)(C[x].c >> 64); }
    }
    free(A); free(B); free(C);
    return r;
}

/* mod-p pair, one prime, residues as uint64 */
int or_pair_modp(const uint64_t *a, const int32_t *la, int ra, const uint64_t *b, const int32_t *lb, int rb,
                 const int32_t *lc, int rc, uint32_t p, uint64_t *c) {
    if (p < 2 || p >= (1u << 31)) return OR_EINVAL;
    return pair_common(OR_MODP, &p, 1, a, la, ra, b, lb, rb, lc, rc, c);
}

/* ------------------------------------------------------------------ */
/* complexity of an order (Sec. 4.1)                                   */
/*   tc  = sum over steps of 2^{|LA u LB|}   (operations)              */
/*   sc  = max over steps of 2^{|LC|}        (largest intermediate)    */
/*   rwc = sum over steps of 2^|LA| + 2^|LB| + 2^|LC|                  */
/* returned as doubles (exact below 2^53).                             */
/* ------------------------------------------------------------------ */
int or_complexity(int n, const int32_t *edges, int m, const int32_t *order, int nsteps,
                  double *tc, double *sc, double *rwc) {
    int rc = or_check_order(n, edges, m, order, nsteps);
    if (rc) return rc;
    int T = m + n;
    tensor_t *t = calloc((size_t)(2 * T), sizeof(tensor_t));
    int *users = calloc((size_t)n, sizeof(int));
    if (!t || !users) { free(t); free(users); return OR_ENOMEM; }
    for (int e = 0; e < m; e++) { t[e].rank = 2; t[e].labels[0] = edges[2 * e]; t[e].labels[1] = edges[2 * e + 1]; }
    for (int v = 0; v < n; v++) { t[m + v].rank = 1; t[m + v].labels[0] = v; }
    for (int i = 0; i < T; i++) for (int k = 0; k < t[i].rank; k++) users[t[i].labels[k]]++;
    double TC = 0, SC = 0, RW = 0;
    for (int s = 0; s < nsteps; s++) {
        int i = order[2 * s], j = order[2 * s + 1], c = T + s;
        output_labels(&t[i], &t[j], users, &t[c]);
        int uni = t[i].rank;
        for (int k = 0; k < t[j].rank; k++) if (find_label(t[i].labels, t[i].rank, t[j].labels[k]) < 0) uni++;
        TC += (double)((uint64_t)1 << uni);
        double sz = (double)((uint64_t)1 << t[c].rank);
        if (sz > SC) SC = sz;
        RW += (double)((uint64_t)1 << t[i].rank) + (double)((uint64_t)1 << t[j].rank) + sz;
        for (int k = 0; k < t[i].rank; k++) users[t[i].labels[k]]--;
        for (int k = 0; k < t[j].rank; k++) users[t[j].labels[k]]--;
        for (int k = 0; k < t[c].rank; k++) users[t[c].labels[k]]++;
    }
    if (nsteps == 0) SC = (double)((uint64_t)1 << t[0].rank);
    *tc = TC; *sc = SC; *rwc = RW;
    free(t); free(users);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* greedy order (Sec. 4.2.1, Eq. 9 with alpha = 0, temperature 0)      */
/* At each step every pair of live tensors that shares a label is a    */
/* candidate; its cost is the size 2^{|LC|} of the tensor it would     */
/* produce.  The cheapest pair is contracted (ties broken uniformly at */
/* random).  If no pair shares a label, the two lowest-rank tensors    */
/* are contracted (an outer product).  The whole run is repeated       */
/* nrepeat times and the order with the smallest (sc, tc) is kept.     */
/* ------------------------------------------------------------------ */
static uint64_t sm64(uint64_t *s) {           /* splitmix64 (Steele et al. 2014) */
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int greedy_once(int n, const int32_t *edges, int m, uint64_t *rng, int32_t *order,
                       double *tc_out, int *sc_out) {
    int T = m + n;
    tensor_t *t = calloc((size_t)(2 * T), sizeof(tensor_t));
    int *users = calloc((size_t)n, sizeof(int));
    char *live = calloc((size_t)(2 * T), 1);
    int cap = 1 << 16;
    int32_t *cand = malloc(sizeof(int32_t) * 2 * (size_t)cap);
    if (!t || !users || !live || !cand) { free(t); free(users); free(live); free(cand); return OR_ENOMEM; }
    for (int e = 0; e < m; e++) { t[e].rank = 2; t[e].labels[0] = edges[2 * e]; t[e].labels[1] = edges[2 * e + 1]; }
    for (int v = 0; v < n; v++) { t[m + v].rank = 1; t[m + v].labels[0] = v; }
    for (int i = 0; i < T; i++) { live[i] = 1; for (int k = 0; k < t[i].rank; k++) users[t[i].labels[k]]++; }
    double TC = 0; int SC = 0;
    int rc = OR_OK;
    /* per-step lists of the live tensors that hold each label */
    int *ucount = calloc((size_t)n, sizeof(int));
    int *ustart = calloc((size_t)n + 1, sizeof(int));
    int *ulist = malloc(sizeof(int) * (size_t)(2 * T) * OR_MAX_RANK);
    if (!ucount || !ustart || !ulist) { free(ucount); free(ustart); free(ulist); rc = OR_ENOMEM; goto done; }
    for (int s = 0; s < T - 1; s++) {
        int best = 1 << 30, ncand = 0;
        int ntot = T + s;
        memset(ucount, 0, sizeof(int) * (size_t)n);
        for (int i = 0; i < ntot; i++)
            if (live[i]) for (int k = 0; k < t[i].rank; k++) ucount[t[i].labels[k]]++;
        ustart[0] = 0;
        for (int l = 0; l < n; l++) ustart[l + 1] = ustart[l] + ucount[l];
        memset(ucount, 0, sizeof(int) * (size_t)n);
        for (int i = 0; i < ntot; i++)
            if (live[i]) for (int k = 0; k < t[i].rank; k++) {
                int l = t[i].labels[k];
                ulist[ustart[l] + ucount[l]++] = i;
            }
        /* every pair sharing a label, visited once: at its smallest shared label */
        for (int l = 0; l < n; l++) {
            for (int x = ustart[l]; x < ustart[l + 1]; x++) {
                for (int y = x + 1; y < ustart[l + 1]; y++) {
                    int i = ulist[x], j = ulist[y];
                    if (i > j) { int tmp = i; i = j; j = tmp; }
                    int smaller_shared = 0;
                    for (int k = 0; k < t[i].rank && !smaller_shared; k++)
                        smaller_shared = t[i].labels[k] < l && find_label(t[j].labels, t[j].rank, t[i].labels[k]) >= 0;
                    if (smaller_shared) continue;
                    tensor_t o;
                    output_labels(&t[i], &t[j], users, &o);
                    if (o.rank < best) { best = o.rank; ncand = 0; }
                    if (o.rank == best) {
                        if (ncand == cap) {
                            cap *= 2;
                            int32_t *nc = realloc(cand, sizeof(int32_t) * 2 * (size_t)cap);
                            if (!nc) { free(ucount); free(ustart); free(ulist); rc = OR_ENOMEM; goto done; }
                            cand = nc;
                        }
                        cand[2 * ncand] = i; cand[2 * ncand + 1] = j; ncand++;
                    }
                }
            }
        }
        int pi, pj;
        if (ncand > 0) {
            uint64_t r = sm64(rng) % (uint64_t)ncand;
            pi = cand[2 * r]; pj = cand[2 * r + 1];
        } else {
            /* disconnected: outer product of the two lowest-rank live tensors */
            pi = pj = -1;
            for (int i = 0; i < ntot; i++) {
                if (!live[i]) continue;
                if (pi < 0 || t[i].rank < t[pi].rank) { pj = pi; pi = i; }
                else if (pj < 0 || t[i].rank < t[pj].rank) pj = i;
            }
        }
        int c = T + s;
        output_labels(&t[pi], &t[pj], users, &t[c]);
        if (t[c].rank > 62) { rc = OR_ETOOBIG; goto done; }
        int uni = t[pi].rank;
        for (int k = 0; k < t[pj].rank; k++) if (find_label(t[pi].labels, t[pi].rank, t[pj].labels[k]) < 0) uni++;
        TC += (double)((uint64_t)1 << (uni > 62 ? 62 : uni));
        if (t[c].rank > SC) SC = t[c].rank;
        for (int k = 0; k < t[pi].rank; k++) users[t[pi].labels[k]]--;
        for (int k = 0; k < t[pj].rank; k++) users[t[pj].labels[k]]--;
        for (int k = 0; k < t[c].rank; k++) users[t[c].labels[k]]++;
        live[pi] = live[pj] = 0; live[c] = 1;
        order[2 * s] = pi; order[2 * s + 1] = pj;
    }
    free(ucount); free(ustart); free(ulist);
    *tc_out = TC; *sc_out = SC;
done:
    free(t); free(users); free(live); free(cand);
    return rc;
}

int or_greedy_order(int n, const int32_t *edges, int m, int nrepeat, uint64_t seed, int32_t *order_out) {
    int rc = check_graph(n, edges, m);
    if (rc) return rc;
    int T = m + n;
    if (T < 2) return OR_OK;                   /* nothing to contract */
    if (nrepeat < 1) nrepeat = 1;
    int32_t *tmp = malloc(sizeof(int32_t) * 2 * (size_t)(T - 1));
    if (!tmp) return OR_ENOMEM;
    uint64_t rng = seed;
    double best_tc = 0; int best_sc = -1;
    for (int r = 0; r < nrepeat; r++) {
        double tc; int sc;
        rc = greedy_once(n, edges, m, &rng, tmp, &tc, &sc);
        if (rc) break;
        if (best_sc < 0 || sc < best_sc || (sc == best_sc && tc < best_tc)) {
            best_sc = sc; best_tc = tc;
            memcpy(order_out, tmp, sizeof(int32_t) * 2 * (size_t)(T - 1));
        }
    }
    free(tmp);
    return rc;
}

/* ------------------------------------------------------------------ */
/* brute force (definition of an independent set, Sec. 2.1.1):        */
/* poly[k] = number of vertex subsets of size k with no edge inside.   */
/* ------------------------------------------------------------------ */
int or_bruteforce_poly(int n, const int32_t *edges, int m, uint64_t *poly) {
    int rc = check_graph(n, edges, m);
    if (rc) return rc;
    if (n > 30) return OR_ETOOBIG;
    uint32_t adj[32] = {0};
    for (int e = 0; e < m; e++) {
        adj[edges[2 * e]] |= 1u << edges[2 * e + 1];
        adj[edges[2 * e + 1]] |= 1u << edges[2 * e];
    }
    for (int k = 0; k <= n; k++) poly[k] = 0;
    uint64_t total = (uint64_t)1 << n;
    for (uint64_t S = 0; S < total; S++) {
        int ok = 1;
        for (int v = 0; v < n && ok; v++)
            if (((S >> v) & 1) && (adj[v] & (uint32_t)S)) ok = 0;
        if (ok) poly[__builtin_popcountll(S)]++;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* flat contraction (Eq. 8 for any graph): the network's scalar as one */
/* (+)-sum over all 2^n assignments of the (x)-product of every edge   */
/* tensor and every vertex tensor entry, built from make_leaf's        */
/* tensors.  No contraction order is involved.  n <= 26.               */
/* ------------------------------------------------------------------ */
int or_flat_contract(int kind, int n, const int32_t *edges, int m, const uint32_t *primes, int nprimes,
                     int64_t *val_out, uint64_t *count_lo, uint64_t *count_hi, uint64_t *residues) {
    int rc = check_graph(n, edges, m);
    if (rc) return rc;
    if (n > 26) return OR_ETOOBIG;
    if (kind == OR_MODP) {
        if (nprimes < 1) return OR_EINVAL;
        for (int q = 0; q < nprimes; q++) if (primes[q] < 2 || primes[q] >= (1u << 31)) return OR_EINVAL;
    }
    if ((kind == OR_KMAX || kind == OR_KPOLY) && (nprimes < 1 || nprimes > OR_MAX_K)) return OR_EINVAL;
    int np_ = kind == OR_MODP ? nprimes : 0;
    int T = m + n;
    tensor_t *t = calloc((size_t)T, sizeof(tensor_t));
    if (!t) return OR_ENOMEM;
    for (int e = 0; e < m && !rc; e++) rc = make_leaf(&t[e], kind, primes, np_, 1, edges[2 * e], edges[2 * e + 1], e);
    for (int v = 0; v < n && !rc; v++) rc = make_leaf(&t[m + v], kind, primes, np_, 0, v, 0, v);
    if (!rc) {
        int64_t tacc = OR_NEG_INF;
        cnt_t cacc; cacc.n = OR_NEG_INF; cacc.c = 0;
        uint64_t macc[64] = {0};
        if (np_ > 64) rc = OR_EINVAL;
        for (uint64_t x = 0; !rc && x < ((uint64_t)1 << n); x++) {
            int64_t tp = 0;                            /* one */
            cnt_t cp; cp.n = 0; cp.c = 1;
            uint64_t mp[64];
            for (int q = 0; q < np_; q++) mp[q] = 1 % primes[q];
            for (int i = 0; i < T; i++) {
                size_t idx = 0;                        /* entry of tensor i at assignment x */
                for (int j = 0; j < t[i].rank; j++) idx |= (size_t)((x >> t[i].labels[j]) & 1) << j;
                if (kind == OR_TROPICAL) tp = trop_mul(tp, ((int64_t *)t[i].data)[idx]);
                else if (kind == OR_COUNTING) cp = cnt_mul(cp, ((cnt_t *)t[i].data)[idx]);
                else for (int q = 0; q < np_; q++) mp[q] = (mp[q] * ((uint64_t *)t[i].data)[idx * np_ + q]) % primes[q];
            }
            if (kind == OR_TROPICAL) tacc = trop_add(tacc, tp);
            else if (kind == OR_COUNTING) cacc = cnt_add(cacc, cp);
            else for (int q = 0; q < np_; q++) macc[q] = (macc[q] + mp[q]) % primes[q];
        }
        if (!rc) {
            if (kind == OR_TROPICAL) *val_out = tacc;
            else if (kind == OR_COUNTING) { *val_out = cacc.n; *count_lo = (uint64_t)cacc.c; *count_hi = (uint64_t)(cacc.c >> 64); }
            else for (int q = 0; q < np_; q++) residues[q] = macc[q];
        }
    }
    for (int i = 0; i < T; i++) free(t[i].data);
    free(t);
    return rc;
}
