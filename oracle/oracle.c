/*
 * oracle.c -- plain, slow, obviously-correct CPU reference for the constrained
 * multilinear sieve of "Restless reachability problems in temporal graphs"
 * (arXiv 2010.08423).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, import or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do. It shares no code, header, table or constant generator
 * with the CUDA implementation.
 *
 * Every routine follows the paper's definitions directly:
 *   - restless walk / path:            Sec. "Preliminaries" (restless walk),
 *   - walk generating function:        Eq. (1), Sec. "Generating restless walks",
 *   - multilinear sieve:               Eq. (2), Lemma "Multilinear sieving",
 *   - constrained (colored) sieve:     Eq. (3), Lemma "Constrained multilinear sieving",
 *   - fine-grained decision oracle:    Algorithm 1,
 *   - k-RestlessReach / MotifReach:    Theorems "algo:krestlessreach" and
 *                                      "algo:restlessmotifreach",
 *   - exhaustive temporal DFS:         Sec. "Baselines" (exhaustive search).
 * No blocking, prefix sums, chunking or factoring: windows are scanned
 * linearly (each vertex's in-edges in time order, from the first one inside
 * the window to the last), sieve points one at a time, layers one at a time.
 *
 * Readings of the paper that this file fixes (the paper is silent or garbled):
 *   - field: GF(2)[x]/(x^64+x^4+x^3+x+1) (the paper uses b = 64 but names no
 *     modulus);
 *   - random values: splitmix64 in counter form (the paper names no PRNG);
 *   - the wait bound is delta of the vertex being left (restless-walk definition),
 *     both window ends inclusive;
 *   - y is keyed by (input edge index, position), so parallel edges are distinct
 *     variables (symbol table: y_{uv,l,j} encodes edge (u,v,j) at position l);
 *   - the source is enforced by seeding layer 1 only at s; every walk that comes
 *     back to s repeats x_s and vanishes, which is what the 2-colour reduction
 *     of the k-RestlessReach theorem achieves;
 *   - shades of M are enumerated colour by colour in ascending colour order.
 *
 * Parity pins: every function here is pinned by tests under tests/ that do
 * not re-type its formula (field axioms, irreducibility via Fermat, published
 * splitmix64 outputs, the figure examples, brute-force DFS and the
 * determinant identity). No function is "parity unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* GF(2^64): elements are uint64, bit i is the coefficient of x^i.            */
/* ------------------------------------------------------------------------- */

/* Low part of the modulus x^64 + x^4 + x^3 + x + 1, i.e. what x^64 reduces to. */
#define ORC_POLY_LOW 0x1BULL

/* Shift-and-add multiplication: for each set bit i of b add a * x^i, reducing
 * a * x after every step (x^64 -> x^4+x^3+x+1). Textbook "Russian peasant"
 * multiplication in GF(2)[x]/(p). */
uint64_t orc_gf_mul(uint64_t a, uint64_t b)
{
    uint64_t r = 0;
    for (int i = 0; i < 64; ++i) {
        if ((b >> i) & 1ULL)
            r ^= a;
        uint64_t carry = a >> 63;
        a <<= 1;
        if (carry)
            a ^= ORC_POLY_LOW;
    }
    return r;
}

/* out[i] = a[i] * b[i] for i < count (bulk form of orc_gf_mul for tests). */
void orc_gf_mul_many(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t count)
{
    for (uint64_t i = 0; i < count; ++i)
        out[i] = orc_gf_mul(a[i], b[i]);
}

/* a^e by square-and-multiply. */
uint64_t orc_gf_pow(uint64_t a, uint64_t e)
{
    uint64_t r = 1;
    while (e) {
        if (e & 1ULL)
            r = orc_gf_mul(r, a);
        a = orc_gf_mul(a, a);
        e >>= 1;
    }
    return r;
}

/* Inverse by Fermat: a^(2^64 - 2). Returns 0 for a == 0. */
uint64_t orc_gf_inv(uint64_t a)
{
    return orc_gf_pow(a, 0xFFFFFFFFFFFFFFFEULL);
}

/* ------------------------------------------------------------------------- */
/* splitmix64 (Steele, Lea, Flood, OOPSLA 2014), counter form.                */
/* ------------------------------------------------------------------------- */

#define ORC_GOLDEN 0x9E3779B97F4A7C15ULL

uint64_t orc_sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number i (0-based) of the sequential generator whose state starts
 * at `key`: the state is advanced by the golden gamma before each output. */
uint64_t orc_sm_draw(uint64_t key, uint64_t i)
{
    return orc_sm_mix(key + (i + 1) * ORC_GOLDEN);
}

/* Family tags: one independent stream per variable family. */
enum { ORC_TAG_Y = 1, ORC_TAG_Z = 2, ORC_TAG_GAMMA = 3, ORC_TAG_OMEGA = 4 };

uint64_t orc_family_key(uint64_t seed, uint64_t tag)
{
    return orc_sm_mix(seed ^ tag);
}

/* y_{e,l}: edge variable of input edge e at walk position l (1-based). */
uint64_t orc_y(uint64_t seed, uint64_t e, uint32_t l)
{
    return orc_sm_draw(orc_family_key(seed, ORC_TAG_Y), e * 32 + (l - 1));
}

/* ------------------------------------------------------------------------- */
/* z-assignment, Eq. (3) (colored) or iid (plain, Eq. (2)).                   */
/* ------------------------------------------------------------------------- */

/*
 * Fills z[u*k + (j-1)] = z_{u,j} for u < n, j = 1..k.
 *
 * Plain (motif == NULL): z_{u,j} = draw(key_Z, u*32 + j-1), independent
 * uniform values as in the uncolored sieve (Lemma "Multilinear sieving").
 *
 * Colored (motif != NULL, k colours): the multiset M is turned into shades,
 * mu(c) shades per colour c, numbered 0..k-1 colour by colour in ascending
 * colour order (S_c is that colour's index range). Then, Eq. (3),
 *     z_{u,j} = sum_{d in S_{c(u)}} gamma_{u,d} * omega_{d,j},
 * with gamma_{u,d} = draw(key_GAMMA, u*32 + d) and
 * omega_{d,j} = draw(key_OMEGA, d*32 + j-1); z_{u,j} = 0 when c(u) is not in M.
 *
 * Returns 0 on success, 1 on invalid arguments.
 */
int orc_ztable(uint32_t n, uint32_t k, uint64_t seed, const uint8_t *color,
               const uint8_t *motif, uint64_t *z)
{
    if (k < 1 || k > 31)
        return 1;
    if (motif == NULL) {
        uint64_t kz = orc_family_key(seed, ORC_TAG_Z);
        for (uint64_t u = 0; u < n; ++u)
            for (uint32_t j = 1; j <= k; ++j)
                z[u * k + (j - 1)] = orc_sm_draw(kz, u * 32 + (j - 1));
        return 0;
    }
    if (color == NULL)
        return 1;
    /* mu(c) and the first shade of each colour (ascending colour order). */
    uint32_t mu[256];
    uint32_t first[256];
    memset(mu, 0, sizeof mu);
    for (uint32_t i = 0; i < k; ++i)
        mu[motif[i]]++;
    uint32_t next = 0;
    for (uint32_t c = 0; c < 256; ++c) {
        first[c] = next;
        next += mu[c];
    }
    uint64_t kg = orc_family_key(seed, ORC_TAG_GAMMA);
    uint64_t ko = orc_family_key(seed, ORC_TAG_OMEGA);
    for (uint64_t u = 0; u < n; ++u) {
        uint32_t c = color[u];
        for (uint32_t j = 1; j <= k; ++j) {
            uint64_t acc = 0;
            for (uint32_t d = first[c]; d < first[c] + mu[c]; ++d) {
                uint64_t gamma = orc_sm_draw(kg, u * 32 + d);
                uint64_t omega = orc_sm_draw(ko, (uint64_t)d * 32 + (j - 1));
                acc ^= orc_gf_mul(gamma, omega);
            }
            z[u * k + (j - 1)] = acc;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The sieve, edge-layer form of Eq. (1) + Eq. (2)/(3), Algorithm 1.          */
/* ------------------------------------------------------------------------- */

/* Restless continuation test: after arriving at u by an edge at time tf, the
 * walk may leave u by an edge at time te iff 0 <= te - tf <= delta(u)
 * (restless-walk definition; both window ends inclusive). Done in 64 bits so
 * that uint32 times and waits cannot overflow. */
static int orc_continues(uint32_t tf, uint32_t te, uint32_t delta_u)
{
    int64_t d = (int64_t)te - (int64_t)tf;
    return d >= 0 && d <= (int64_t)delta_u;
}

/* in-edge lists: for each vertex, the input indices of edges ending there,
 * ordered by (time, input index), so that the edges a walk may have arrived
 * by before leaving u at time te (Eq. (1)'s j in {0..delta(u)}: arrival times
 * te - delta(u) .. te) are one run of u's list. */
typedef struct {
    uint64_t *start; /* n+1 */
    uint64_t *edge;  /* m   */
    uint32_t *time;  /* m: time[q] = t[edge[q]] */
} orc_inlists;

static int orc_cmp_u64(const void *a, const void *b)
{
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int orc_build_inlists(uint32_t n, uint64_t m, const uint32_t *dst, const uint32_t *t,
                             orc_inlists *L)
{
    L->start = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    L->edge = (uint64_t *)malloc((size_t)(m ? m : 1) * sizeof(uint64_t));
    L->time = (uint32_t *)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
    uint64_t *fill = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!L->start || !L->edge || !L->time || !fill) {
        free(fill);
        return 1;
    }
    for (uint64_t e = 0; e < m; ++e)
        L->start[dst[e] + 1]++;
    for (uint32_t v = 0; v < n; ++v)
        L->start[v + 1] += L->start[v];
    memcpy(fill, L->start, ((size_t)n + 1) * sizeof(uint64_t));
    /* key (time, input index) per edge, then each list sorted by key */
    for (uint64_t e = 0; e < m; ++e)
        L->edge[fill[dst[e]]++] = ((uint64_t)t[e] << 32) | e;
    free(fill);
    for (uint32_t v = 0; v < n; ++v)
        qsort(L->edge + L->start[v], (size_t)(L->start[v + 1] - L->start[v]), sizeof(uint64_t),
              orc_cmp_u64);
    for (uint64_t q = 0; q < m; ++q) {
        L->time[q] = (uint32_t)(L->edge[q] >> 32);
        L->edge[q] &= 0xFFFFFFFFULL;
    }
    return 0;
}

/* Position of the first edge of u's list that arrives at time >= tmin. */
static uint64_t orc_first_at_or_after(const orc_inlists *IN, uint32_t u, int64_t tmin)
{
    uint64_t lo = IN->start[u], hi = IN->start[u + 1];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if ((int64_t)IN->time[mid] < tmin)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

/* Eq. (1)'s window sum for an edge leaving u at time te: the XOR of prev[f]
 * over u's in-edges f with t_f <= te <= t_f + delta(u). In u's time-ordered
 * list these follow the first edge arriving at te - delta(u) or later, and end
 * at the first edge the walk cannot continue from (one arriving after te). */
static uint64_t orc_window_sum(const orc_inlists *IN, uint32_t u, uint32_t te, uint32_t delta_u,
                               const uint64_t *prev)
{
    uint64_t w = 0;
    for (uint64_t q = orc_first_at_or_after(IN, u, (int64_t)te - (int64_t)delta_u);
         q < IN->start[u + 1]; ++q) {
        if (!orc_continues(IN->time[q], te, delta_u))
            break;
        w ^= prev[IN->edge[q]];
    }
    return w;
}

static void orc_free_inlists(orc_inlists *L)
{
    free(L->start);
    free(L->edge);
    free(L->time);
}

/*
 * Evaluates, for one sieve point L (bit j-1 of `mask` set <=> label j in L),
 * the per-vertex sum over the k-1 edge layers:
 *   x_u^L      = sum_{j in L} z_{u,j}                              (Eq. (2)/(3))
 *   P_1^L[e]   = [u_e = s] * y_{e,1} * x_s^L * x_{v_e}^L           (layer 1, Alg. 1 init at s)
 *   P_l^L[e]   = y_{e,l} * x_{v_e}^L * sum_{f : v_f = u_e, t_f <= t_e <= t_f + delta(u_e)} P_{l-1}^L[f]
 *                                                                  (Eq. (1), l = 2..k-1)
 *   out[v]    ^= sum_{e : v_e = v} P_{k-1}^L[e]
 *   eout[e]   ^= P_{k-1}^L[e]            (if eout is not NULL)
 * P_l^L[e] is the evaluation of all restless walks with l edges whose last
 * edge is e, i.e. Eq. (1)'s chi_{v_e, l+1, t_e} restricted to edge e.
 */
static void orc_one_point(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                          const uint32_t *t, const uint32_t *delta, const orc_inlists *IN,
                          uint32_t s, uint32_t k, uint64_t seed, const uint64_t *z,
                          uint32_t mask, uint64_t *x, uint64_t *prev, uint64_t *cur,
                          uint64_t *out, uint64_t *eout, const uint8_t *sources, int par)
{
    /* par != 0: the loops over vertices and edges are shared by the threads
     * (each iteration writes only its own element) */
#pragma omp parallel for if (par) schedule(static)
    for (int64_t u = 0; u < (int64_t)n; ++u) {
        uint64_t acc = 0;
        for (uint32_t j = 1; j <= k; ++j)
            if ((mask >> (j - 1)) & 1U)
                acc ^= z[u * k + (j - 1)];
        x[u] = acc;
    }
    /* layer 1 */
#pragma omp parallel for if (par) schedule(static)
    for (int64_t e = 0; e < (int64_t)m; ++e) {
        if (sources) {
            /* a set of sources: every edge leaving one of them starts a walk */
            prev[e] = sources[src[e]]
                          ? orc_gf_mul(orc_gf_mul(orc_y(seed, e, 1), x[src[e]]), x[dst[e]])
                          : 0;
            continue;
        }
        if (src[e] == s)
            prev[e] = orc_gf_mul(orc_gf_mul(orc_y(seed, e, 1), x[s]), x[dst[e]]);
        else
            prev[e] = 0;
    }
    /* layers 2..k-1 */
    for (uint32_t l = 2; l <= k - 1; ++l) {
#pragma omp parallel for if (par) schedule(dynamic, 4096)
        for (int64_t e = 0; e < (int64_t)m; ++e) {
            uint32_t u = src[e];
            uint64_t w = orc_window_sum(IN, u, t[e], delta[u], prev);
            /* a zero window sum makes the product zero */
            cur[e] = w ? orc_gf_mul(orc_gf_mul(orc_y(seed, e, l), x[dst[e]]), w) : 0;
        }
        uint64_t *tmp = prev;
        prev = cur;
        cur = tmp;
    }
    for (uint64_t e = 0; e < m; ++e)
        out[dst[e]] ^= prev[e];
    if (eout)
        for (uint64_t e = 0; e < m; ++e)
            eout[e] ^= prev[e];
}

/*
 * orc_sieve: the fine-grained decision oracle's per-vertex sums (Algorithm 1,
 * ell = k), summed over the requested sieve points.
 *
 *   n, m, src, dst, t, delta   temporal multigraph, edge e = (src[e], dst[e], t[e])
 *   color, motif               NULL/NULL for a plain query; otherwise colours
 *                              (n) and the motif multiset (k entries)
 *   s, k, seed                 source, number of path vertices, random seed
 *   masks, nmasks              sieve points to evaluate; masks == NULL means all
 *                              2^k points 0..2^k-1
 *   S                          out, n values: XOR over the evaluated points
 *   per_mask                   optional out, nmasks*n values (row p = point masks[p])
 *   sources                    optional, n flags: a set of sources (Sec. "Discussion":
 *                              the multi-source variant); layer 1 then starts at
 *                              every edge leaving a flagged vertex u, with x_u in
 *                              place of x_s, and s is ignored
 *   deleted                    optional, n flags: vertices removed from the graph
 *                              (the extraction's G^{l-1} = G^l minus u_l, Sec.
 *                              "Extracting an optimal solution using k queries"),
 *                              realised as z_u = 0, which makes every walk through
 *                              u vanish and leaves all other terms unchanged
 *   E                          optional out, m values: for every edge e the XOR over
 *                              the evaluated points of P_{k-1}^L[e] (the walks of k
 *                              vertices whose last edge is e; Algorithm 1's
 *                              per-time polynomials are the sums of E over the
 *                              edges into u at time i)
 *   nthreads                   OpenMP threads over sieve points (0 = default)
 *
 * Returns 0 on success, 1 on invalid input, 2 on allocation failure.
 */
int orc_sieve(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
              const uint32_t *t, const uint32_t *delta, const uint8_t *color,
              const uint8_t *motif, uint32_t s, uint32_t k, uint64_t seed,
              const uint32_t *masks, uint32_t nmasks, uint64_t *S, uint64_t *per_mask,
              uint64_t *E, const uint8_t *deleted, const uint8_t *sources, int nthreads)
{
    if (k < 2 || k > 20 || s >= n || m >= (1ULL << 32))
        return 1;
    for (uint64_t e = 0; e < m; ++e)
        if (src[e] >= n || dst[e] >= n || src[e] == dst[e])
            return 1;
    uint64_t npts = masks ? nmasks : (1ULL << k);
    uint64_t *z = (uint64_t *)malloc((size_t)n * k * sizeof(uint64_t) + 8);
    if (!z)
        return 2;
    if (orc_ztable(n, k, seed, color, motif, z)) {
        free(z);
        return 1;
    }
    if (deleted)
        for (uint64_t u = 0; u < n; ++u)
            if (deleted[u])
                for (uint32_t j = 0; j < k; ++j)
                    z[u * k + j] = 0;
    orc_inlists IN;
    if (orc_build_inlists(n, m, dst, t, &IN)) {
        free(z);
        return 2;
    }
    memset(S, 0, (size_t)n * sizeof(uint64_t));
    if (E)
        memset(E, 0, (size_t)m * sizeof(uint64_t));
    int fail = 0;
    int threads = 1;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
    threads = omp_get_max_threads();
#else
    (void)nthreads;
#endif
    if ((int64_t)npts < threads) {
        /* fewer points than threads: one point at a time, the threads sharing
         * each layer's edges */
        uint64_t *x = (uint64_t *)malloc((size_t)n * sizeof(uint64_t) + 8);
        uint64_t *prev = (uint64_t *)malloc((size_t)m * sizeof(uint64_t) + 8);
        uint64_t *cur = (uint64_t *)malloc((size_t)m * sizeof(uint64_t) + 8);
        uint64_t *one = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
        if (!x || !prev || !cur || !one) {
            fail = 1;
        } else {
            for (uint64_t p = 0; p < npts; ++p) {
                uint32_t mask = masks ? masks[p] : (uint32_t)p;
                memset(one, 0, (size_t)n * sizeof(uint64_t));
                orc_one_point(n, m, src, dst, t, delta, &IN, s, k, seed, z, mask, x, prev, cur,
                              one, E, sources, 1);
                for (uint32_t v = 0; v < n; ++v)
                    S[v] ^= one[v];
                if (per_mask)
                    memcpy(per_mask + (size_t)p * n, one, (size_t)n * sizeof(uint64_t));
            }
        }
        free(x);
        free(prev);
        free(cur);
        free(one);
        orc_free_inlists(&IN);
        free(z);
        return fail ? 2 : 0;
    }
#pragma omp parallel
    {
        uint64_t *x = (uint64_t *)malloc((size_t)n * sizeof(uint64_t) + 8);
        uint64_t *prev = (uint64_t *)malloc((size_t)m * sizeof(uint64_t) + 8);
        uint64_t *cur = (uint64_t *)malloc((size_t)m * sizeof(uint64_t) + 8);
        uint64_t *acc = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
        uint64_t *one = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
        uint64_t *eacc = E ? (uint64_t *)calloc((size_t)m + 1, sizeof(uint64_t)) : NULL;
        if (!x || !prev || !cur || !acc || !one || (E && !eacc)) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t p = 0; p < (int64_t)npts; ++p) {
                uint32_t mask = masks ? masks[p] : (uint32_t)p;
                memset(one, 0, (size_t)n * sizeof(uint64_t));
                orc_one_point(n, m, src, dst, t, delta, &IN, s, k, seed, z, mask, x, prev,
                              cur, one, eacc, sources, 0);
                for (uint32_t v = 0; v < n; ++v)
                    acc[v] ^= one[v];
                if (per_mask)
                    memcpy(per_mask + (size_t)p * n, one, (size_t)n * sizeof(uint64_t));
            }
#pragma omp critical
            {
                for (uint32_t v = 0; v < n; ++v)
                    S[v] ^= acc[v];
                if (E)
                    for (uint64_t e = 0; e < m; ++e)
                        E[e] ^= eacc[e];
            }
        }
        free(x);
        free(prev);
        free(cur);
        free(acc);
        free(one);
        free(eacc);
    }
    orc_free_inlists(&IN);
    free(z);
    return fail ? 2 : 0;
}

/* Number of OpenMP threads a parallel region gets by default. */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Brute force: exhaustive temporal DFS (Sec. "Baselines") and the            */
/* determinant identity that the sieve must satisfy exactly.                  */
/* ------------------------------------------------------------------------- */

/* Determinant of a k x k matrix over GF(2^64) by Gaussian elimination. In
 * characteristic 2 the row-swap sign is +1, and the determinant equals the
 * permanent. The matrix is destroyed. */
uint64_t orc_gf_det(uint32_t k, uint64_t *a)
{
    uint64_t det = 1;
    for (uint32_t c = 0; c < k; ++c) {
        uint32_t piv = k;
        for (uint32_t r = c; r < k; ++r)
            if (a[r * k + c]) {
                piv = r;
                break;
            }
        if (piv == k)
            return 0;
        if (piv != c)
            for (uint32_t j = 0; j < k; ++j) {
                uint64_t tmp = a[c * k + j];
                a[c * k + j] = a[piv * k + j];
                a[piv * k + j] = tmp;
            }
        uint64_t p = a[c * k + c];
        det = orc_gf_mul(det, p);
        uint64_t pinv = orc_gf_inv(p);
        for (uint32_t r = c + 1; r < k; ++r) {
            uint64_t f = orc_gf_mul(a[r * k + c], pinv);
            if (!f)
                continue;
            for (uint32_t j = c; j < k; ++j)
                a[r * k + j] ^= orc_gf_mul(f, a[c * k + j]);
        }
    }
    return det;
}

typedef struct {
    uint32_t n;
    const uint32_t *src, *dst, *t, *delta;
    const uint8_t *color;
    const uint8_t *motif;
    uint32_t k;
    uint64_t seed;
    const uint64_t *z; /* may be NULL when only decisions are needed */
    /* out-edge lists */
    const uint64_t *ostart, *oedge;
    /* DFS state */
    uint32_t *pathv;   /* k vertices */
    uint64_t *pathe;   /* k-1 edges */
    uint8_t *onpath;   /* n */
    uint32_t need[256];/* remaining colour counts (motif) */
    uint8_t *reach;    /* out: n */
    uint64_t *Sdet;    /* out: n (may be NULL) */
    uint64_t *Edet;    /* out: m, by last edge (may be NULL) */
    uint32_t *arrive;  /* out: n, earliest last-edge time (may be NULL) */
    const uint8_t *deleted; /* n flags: vertices no path may use (may be NULL) */
    uint64_t *mat;     /* k*k scratch */
    uint64_t npaths;
} orc_dfs;

/* Called with a complete restless path u_1..u_k (edges e_1..e_{k-1}). */
static void orc_dfs_emit(orc_dfs *D)
{
    uint32_t k = D->k;
    uint32_t end = D->pathv[k - 1];
    uint64_t last = D->pathe[k - 2];
    D->reach[end] = 1;
    D->npaths++;
    if (D->arrive && D->t[last] < D->arrive[end])
        D->arrive[end] = D->t[last];
    if (!D->Sdet && !D->Edet)
        return;
    /* weight = prod_l y_{e_l, l} * det(Z_P), Z_P[i][j] = z_{u_i, j} */
    uint64_t w = 1;
    for (uint32_t l = 1; l <= k - 1; ++l)
        w = orc_gf_mul(w, orc_y(D->seed, D->pathe[l - 1], l));
    for (uint32_t i = 0; i < k; ++i)
        for (uint32_t j = 0; j < k; ++j)
            D->mat[i * k + j] = D->z[(uint64_t)D->pathv[i] * k + j];
    w = orc_gf_mul(w, orc_gf_det(k, D->mat));
    if (D->Sdet)
        D->Sdet[end] ^= w;
    if (D->Edet)
        D->Edet[last] ^= w;
}

static void orc_dfs_rec(orc_dfs *D, uint32_t depth /* vertices so far */)
{
    if (depth == D->k) {
        orc_dfs_emit(D);
        return;
    }
    uint32_t u = D->pathv[depth - 1];
    for (uint64_t q = D->ostart[u]; q < D->ostart[u + 1]; ++q) {
        uint64_t e = D->oedge[q];
        uint32_t v = D->dst[e];
        if (D->onpath[v] || (D->deleted && D->deleted[v]))
            continue;
        if (depth >= 2 && !orc_continues(D->t[D->pathe[depth - 2]], D->t[e], D->delta[u]))
            continue;
        if (D->motif) {
            uint8_t c = D->color[v];
            if (D->need[c] == 0)
                continue;
            D->need[c]--;
        }
        D->onpath[v] = 1;
        D->pathv[depth] = v;
        D->pathe[depth - 1] = e;
        orc_dfs_rec(D, depth + 1);
        D->onpath[v] = 0;
        if (D->motif)
            D->need[D->color[v]]++;
    }
}

/*
 * orc_dfs_paths: exhaustive temporal DFS from s over restless paths with
 * exactly k vertices (the paper's exhaustive-search baseline, restricted to
 * exact length and, for motif queries, to paths whose colour multiset is M).
 *
 *   reach[v] = 1 iff such a path ends at v (always filled).
 *   Sdet (optional) = for each v, XOR over such paths P ending at v of
 *       prod_{l=1}^{k-1} y_{e_l, l} * det(Z_P),   Z_P[i][j] = z_{u_i, j},
 *   with z the same assignment the sieve uses. The sieve's sum over L of
 *   prod_i x_{u_i}^L equals the permanent of Z_P in characteristic 2
 *   (non-surjective label maps are counted an even number of times), which
 *   equals det(Z_P); walks that repeat a vertex give equal rows and vanish.
 *   So Sdet must equal orc_sieve's S bit for bit.
 *   Edet (optional, m) = the same sum split by the path's last edge, which
 *   must equal orc_sieve's E bit for bit.
 *   arrive (optional, n) = the earliest time of a path's last edge among the
 *   paths ending at v (UINT32_MAX if none): the minimum reachability time R_v
 *   of Algorithm 1, found without any sieve.
 *   deleted (optional, n flags) = vertices that no path may visit (the graph
 *   without them).
 *
 * Returns the number of paths found (saturating), or (uint64)-1 on bad input.
 */
uint64_t orc_dfs_paths(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                       const uint32_t *t, const uint32_t *delta, const uint8_t *color,
                       const uint8_t *motif, uint32_t s, uint32_t k, uint64_t seed,
                       uint8_t *reach, uint64_t *Sdet, uint64_t *Edet, uint32_t *arrive,
                       const uint8_t *deleted)
{
    if (k < 2 || k > 31 || s >= n)
        return (uint64_t)-1;
    orc_dfs D;
    memset(&D, 0, sizeof D);
    D.n = n;
    D.src = src;
    D.dst = dst;
    D.t = t;
    D.delta = delta;
    D.color = color;
    D.motif = motif;
    D.k = k;
    D.seed = seed;
    uint64_t *ostart = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint64_t *oedge = (uint64_t *)malloc((size_t)(m ? m : 1) * sizeof(uint64_t));
    uint64_t *fill = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t e = 0; e < m; ++e)
        ostart[src[e] + 1]++;
    for (uint32_t v = 0; v < n; ++v)
        ostart[v + 1] += ostart[v];
    memcpy(fill, ostart, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t e = 0; e < m; ++e)
        oedge[fill[src[e]]++] = e;
    free(fill);
    D.ostart = ostart;
    D.oedge = oedge;
    uint64_t *z = NULL;
    if (Sdet || Edet) {
        z = (uint64_t *)malloc((size_t)n * k * sizeof(uint64_t) + 8);
        orc_ztable(n, k, seed, color, motif, z);
    }
    if (Sdet)
        memset(Sdet, 0, (size_t)n * sizeof(uint64_t));
    if (Edet)
        memset(Edet, 0, (size_t)m * sizeof(uint64_t));
    if (arrive)
        for (uint32_t v = 0; v < n; ++v)
            arrive[v] = UINT32_MAX;
    D.z = z;
    D.Sdet = Sdet;
    D.Edet = Edet;
    D.arrive = arrive;
    D.deleted = deleted;
    D.pathv = (uint32_t *)malloc(k * sizeof(uint32_t));
    D.pathe = (uint64_t *)malloc(k * sizeof(uint64_t));
    D.onpath = (uint8_t *)calloc(n, 1);
    D.mat = (uint64_t *)malloc((size_t)k * k * sizeof(uint64_t));
    D.reach = reach;
    memset(reach, 0, n);
    int ok = 1;
    if (motif) {
        for (uint32_t i = 0; i < k; ++i)
            D.need[motif[i]]++;
        if (D.need[color[s]] == 0)
            ok = 0; /* the source itself must take one of M's colours */
        else
            D.need[color[s]]--;
    }
    if (ok) {
        D.pathv[0] = s;
        D.onpath[s] = 1;
        orc_dfs_rec(&D, 1);
    }
    free(D.pathv);
    free(D.pathe);
    free(D.onpath);
    free(D.mat);
    free(z);
    free(ostart);
    free(oedge);
    return D.npaths;
}
