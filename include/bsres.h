/*
 * bsres.h -- C ABI of the GB300 multi-modular resultant / gcd library (libbsres.so).
 *
 * The library computes, exactly and on one GPU, the symbolic operations that the
 * Bisolve / GeoTop curve analysis needs (Sec. 5.1 of the paper, "GPU-accelerated
 * symbolic computations"):
 *
 *   - the bivariate resultant res(f, g; y) in Z[x] (or res(f, g; x) in Z[y]) by the
 *     modular route of Sec. 5.1 steps (a)-(e): reduce modulo many 31-bit primes,
 *     evaluate at many points, take univariate resultants mod p, interpolate, and
 *     reconstruct the integer coefficients by mixed-radix Chinese remaindering;
 *   - the monic gcd of two polynomials in Z_p[x] (Sec. 5.1, "Computing gcds in Z[x]",
 *     step (b));
 *   - the square-free part of a polynomial in Z[x] and its full square-free
 *     factorisation by Yun's algorithm (Sec. 2.1, BiProject), and the gcd in Z[x], all
 *     by the modular route of Sec. 5.1 ("Computing gcds in Z[x]");
 *   - the principal subresultant coefficients of two bivariate polynomials, exact or
 *     modulo one prime, and on them the fiber counts of Sec. 3.3 (the number N of curve
 *     points over the critical values, its bounds N^- and N^+), Teissier's Q and the split
 *     of R* by the multiplicity of Q at its roots;
 *   - the content of a bivariate polynomial with respect to one variable and its
 *     primitive part (Sec. 4: vertical lines).
 *
 * Integer encoding.  Every integer coefficient is a fixed number of little-endian
 * uint32 limbs in two's complement (limb 0 is the least significant; the sign is the
 * top bit of the last limb).  All coefficients of one polynomial use the same limb count.
 *
 * Bivariate layout (Sec. 2, "Notation": f = sum f_ij x^i y^j).  A bs_bipoly is a dense
 * (deg_y + 1) x (deg_x + 1) grid: the coefficient of x^i y^j starts at
 * c[(j * (deg_x + 1) + i) * limbs].  deg_x and deg_y are grid extents; trailing zero rows
 * or columns are allowed (the library finds the actual degrees itself).
 *
 * Univariate layout.  A bs_upoly holds deg + 1 coefficients in ascending order, the
 * coefficient of x^i at c[i * limbs]; deg = -1 denotes the zero polynomial.
 *
 * Ownership.  Inputs are borrowed for the duration of a call (or, for the *_device
 * entry points, until the work enqueued on the context's stream has finished).
 * Outputs are caller-allocated.  The context owns its device memory and stream.
 *
 * Errors.  Every entry point returns a status code (BS_OK = 0 on success).  A call that
 * fails leaves its outputs unspecified and the context usable.  bs_error_string()
 * turns a code into text; bs_last_error_detail() returns a message about the most
 * recent failure on a context.
 *
 * Threads.  A context may be used by one host thread at a time.
 */
#ifndef BSRES_H
#define BSRES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BS_OK            0
#define BS_ERR_ARG       1  /* invalid argument (null pointer, negative size, bad var)  */
#define BS_ERR_NOMEM     2  /* device memory budget exceeded (admission refused)        */
#define BS_ERR_UNLUCKY   3  /* more unlucky primes than spare primes were provided for  */
#define BS_ERR_TIMEOUT   4  /* a bounded device-side wait expired                       */
#define BS_ERR_CUDA      5  /* a CUDA runtime call failed                               */
#define BS_ERR_ZERO      6  /* square-free part of the zero polynomial                  */
#define BS_ERR_RANGE     7  /* problem exceeds the prime table or the transform size    */
#define BS_ERR_INTERNAL  8  /* a device-side consistency check failed                   */
#define BS_ERR_CAPACITY  9  /* caller-provided output capacity is too small             */
#define BS_PENDING      10  /* bs_poll: the job has not finished yet (not an error)      */

typedef struct bs_ctx bs_ctx;

typedef struct {
    int32_t deg_x;        /* grid extent in x (>= 0)                                   */
    int32_t deg_y;        /* grid extent in y (>= 0)                                   */
    int32_t limbs;        /* uint32 limbs per coefficient (1..64)                      */
    const uint32_t *c;    /* (deg_y+1)*(deg_x+1)*limbs limbs, layout above             */
} bs_bipoly;

typedef struct {
    int32_t deg;          /* degree, or -1 for the zero polynomial (capacity on input) */
    int32_t limbs;        /* limbs per coefficient (capacity on input)                 */
    uint32_t *c;          /* (deg+1)*limbs limbs                                       */
} bs_upoly;

/* Work statistics of the most recent resultant call on a context. */
typedef struct {
    int32_t jobs;             /* resultants in the call                                 */
    int64_t primes_needed;    /* sum over jobs of the primes the coefficient bound asks */
    int64_t primes_evaluated; /* sum over jobs of the primes evaluated (with spares)    */
    int64_t primes_rejected;  /* primes dropped as unlucky (lc vanishing mod p or at a  */
                              /* point of the prime's evaluation set)                   */
    int64_t instances;        /* univariate resultants mod p computed                   */
    int64_t mulmods_alg;      /* algorithmic count m_y*n_y summed over instances        */
    int32_t max_points;       /* largest transform size N used                          */
    int32_t max_primes;       /* largest prime count of one job                         */
} bs_stats;

/* ---------------------------------------------------------------------------------
 * Context
 * ------------------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `mem_budget` caps the device memory the
 * context may hold for work buffers (0 = 90% of the free memory).  The context creates
 * its own non-blocking stream.  On success *out receives the context. */
int bs_init(int device, size_t mem_budget, bs_ctx **out);

/* Destroy a context and release its device memory (waits for its stream). */
void bs_free(bs_ctx *ctx);

/* Make the context enqueue its work on `stream` (a cudaStream_t; NULL restores the
 * context's own stream).  The caller keeps ownership of the stream. */
int bs_set_stream(bs_ctx *ctx, void *stream);

const char *bs_error_string(int status);
const char *bs_last_error_detail(const bs_ctx *ctx);
int bs_last_stats(const bs_ctx *ctx, bs_stats *out);

/* ---------------------------------------------------------------------------------
 * Resultants (Sec. 2 "Resultants"; modular route Sec. 5.1 steps (a)-(e))
 * ------------------------------------------------------------------------------ */

/* The plan of res(f, g; var) (host only, no context or GPU needed).  Degrees are the
 * actual degrees found in the data; e is the eliminated variable, o the other one.
 * Errors: BS_ERR_ARG for a null pointer, var other than 0 or 1, a negative grid extent,
 * limbs outside 1..64 or a null coefficient array. */
typedef struct {
    int32_t trivial;      /* 0 general; 1 the result is 0; 2 the result is 1            */
    int32_t m_e, n_e;     /* degrees of f and g in the eliminated variable              */
    int32_t D;            /* degree bound of the result: min(tdeg f * tdeg g,           */
                          /*   n_e deg_o f + m_e deg_o g) (Sec. 2); -1 if the result is 0 */
    int32_t N;            /* points per prime: the smallest power of two > D            */
    int32_t k_need;       /* primes with prod p > 4 B (B the coefficient bound)         */
    int32_t k_total;      /* primes evaluated: k_need plus spares for unlucky primes    */
    int32_t out_limbs;    /* limbs that hold every coefficient of the result            */
    int64_t log2B_q16;    /* upper bound of log2 B in units of 2^-16                    */
} bs_plan_info;

int bs_plan(const bs_bipoly *f, const bs_bipoly *g, int var, bs_plan_info *out);

/* Size query.  Upper bounds, computed from the grid extents and limb counts only, on
 * the degree and on the limbs per coefficient of res(f, g; var).  var = 1 eliminates y
 * (result in Z[x]), var = 0 eliminates x (result in Z[y]). */
int bs_resultant_bounds(const bs_bipoly *f, const bs_bipoly *g, int var,
                        int32_t *deg_cap, int32_t *limbs_cap);

/* res(f, g; var) with host-resident inputs and output.  The result is exact.
 * If out->c is NULL the call only stores the degree and limb capacities the result
 * needs into out->deg and out->limbs and returns BS_OK (nothing is computed on the GPU
 * beyond planning); the degree stored is the bound D of the plan and the limb count
 * is an upper bound.  Otherwise out->deg and out->limbs give the capacity; on success
 * out->deg is set to the true degree (-1 for the zero polynomial) and coefficients
 * deg+1..capacity are zero-filled; each coefficient is sign-extended to out->limbs.
 * Limits (BS_ERR_RANGE beyond them): degree at most 64 in the eliminated variable (the
 * univariate stage keeps both polynomials in registers), at most 2^14 points per prime
 * (degree bound D < 16384), at most 64 limbs per input coefficient, and a bound that the
 * 6213 table primes cover (about 190,000 bits). */
int bs_resultant(bs_ctx *ctx, const bs_bipoly *f, const bs_bipoly *g, int var,
                 bs_upoly *out);

/* res(f, g; var) with device-resident inputs and output, enqueued on the context's
 * stream without host synchronisation.  f->c, g->c, out->c are device pointers;
 * out->deg and out->limbs must be at least the capacities that bs_resultant_bounds()
 * returns.  The plan (degrees, coefficient bound, prime count) is computed on the
 * device.  The output receives coefficients 0..out->deg (zero above the true degree),
 * sign-extended to out->limbs.  Device-side failures (unlucky-prime cap, consistency
 * checks) are recorded in a status word that bs_device_status() returns. */
int bs_resultant_device(bs_ctx *ctx, const bs_bipoly *f, const bs_bipoly *g, int var,
                        bs_upoly *out);

/* res(f, g; var) with device-resident buffers, for callers that cannot allocate device
 * memory while they run: programs whose device memory is owned by another allocator or
 * framework (a caching allocator, a fixed memory budget handed out by the host
 * application), and latency-critical loops that must not pay for an allocation and the
 * synchronisation cudaMalloc implies.  The paper has no counterpart; this is a service
 * of the library.
 *
 * Arguments, layout, capacities and the asynchronous behaviour are those of
 * bs_resultant_device.  The call performs no cudaMalloc or cudaFree: all of its scratch
 * is carved out of one static device array of 32 MiB (33554432 bytes) compiled into the
 * library, which every GPU that loads the library holds until the process exits.  A
 * problem whose scratch (sized from the grid extents and limb counts, like
 * bs_resultant_bounds) exceeds 32 MiB is rejected with BS_ERR_RANGE; for example the
 * degree-32 discriminant with 32-bit coefficients does not fit, a degree-12 one does.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress and keeps it for the life of the process (resetting the device
 * afterwards is not supported); make that first call before any stream capture.  Every call
 * shares the one array and leaves its contents behind (the call clears what must start
 * at zero), so calls whose GPU work overlaps -- on different streams or contexts of the
 * same device -- race and corrupt each other's results.  The call does not grow the
 * context's prime and transform tables: a problem larger than every earlier allocating
 * resultant call on the context returns BS_ERR_RANGE until one such call has been made. */
int bs_resultant_device_noalloc(bs_ctx *ctx, const bs_bipoly *f, const bs_bipoly *g,
                                int var, bs_upoly *out);

/* Wait for the context's stream and return the first device-side status recorded since
 * the previous call of this function (BS_OK if none), then clear it. */
int bs_device_status(bs_ctx *ctx);

/* n resultants res(f[i], g[i]; var) with host-resident inputs and outputs, computed
 * as one batch: all pairs share each kernel launch, the univariate-resultant stage is
 * one persistent launch per degree class, and the device stages are replayed from a
 * CUDA graph.  out[i] follows the rules of bs_resultant (a NULL out[i].c makes the
 * whole call a size query). */
int bs_resultant_batch(bs_ctx *ctx, int n, const bs_bipoly *f, const bs_bipoly *g,
                       int var, bs_upoly *out);

/* Univariate resultants mod p with formal degrees (step (c) of Sec. 5.1 on given
 * images).  For each of n instances: a has da+1 coefficients and b has db+1
 * coefficients (ascending, reduced into [0, p)), read from a + i*lda and b + i*ldb;
 * the instance's prime is p[i] and must be one of the library's table primes
 * (2^30 < p < 2^31, p = 1 mod 2^14).  res[i] = det of the Sylvester matrix of (a, b)
 * mod p[i], leading coefficients allowed to vanish.  Host buffers; 0 <= da, db < 128. */
int bs_uni_resultant_modp(bs_ctx *ctx, int n, const uint32_t *p,
                          const uint32_t *a, int da, int lda,
                          const uint32_t *b, int db, int ldb, uint32_t *res);

/* The first `count` table primes (2^30 < p < 2^31, p = 1 mod 2^14, decreasing). */
int bs_prime_table(int count, uint32_t *primes);

/* ---------------------------------------------------------------------------------
 * gcd and square-free part (Sec. 5.1 "Computing gcds in Z[x]"; Sec. 2.1 BiProject)
 *
 * The univariate inputs of bs_squarefree_part, bs_gcd_z, bs_modgcd_batch and the
 * square-free factorisation take up to 256 limbs per coefficient (8192 bits), so a
 * resultant's output can be passed back as input.
 * ------------------------------------------------------------------------------ */

/* Monic gcd of a (degree da) and b (degree db) in Z_p[x], p prime (2 < p < 2^31),
 * coefficients in [0, p), ascending, host buffers.  g must hold max(da, db) + 1 entries;
 * *dg receives the gcd's degree (-1 when a = b = 0).  da or db may be -1 (zero poly). */
int bs_gcd_modp(bs_ctx *ctx, const uint32_t *a, int da, const uint32_t *b, int db,
                uint32_t p, uint32_t *g, int *dg);

/* Square-free part R* = pp(R / gcd(R, R')) of a non-zero R in Z[x], primitive with a
 * positive leading coefficient (Sec. 2.1: the projection's square-free factorisation
 * starts from gcd(R, R'); Sec. 5.1: gcds in Z[x] by the modular route).
 *
 * r: host buffer, r->c[i * r->limbs + l] is limb l of the coefficient of x^i (two's
 * complement, little-endian limbs); leading zero coefficients are ignored.
 * out: host buffer owned by the caller.  With out->c == NULL the call only writes upper
 * bounds to out->deg and out->limbs and returns BS_OK.  Otherwise out->deg and
 * out->limbs give the capacity (out->deg must be at least the trimmed degree of r); on
 * success out->deg is set to deg R* and the coefficients are written with out->limbs
 * limbs each (sign-extended; positions above deg R* up to the capacity are zeroed).
 *
 * The work runs on the context's stream; the call waits for it.  Errors: BS_ERR_ARG,
 * BS_ERR_ZERO for R = 0, BS_ERR_RANGE when 3 (deg r + 1) words exceed one block's shared
 * memory or the coefficient bound exceeds the prime table, BS_ERR_CAPACITY when the
 * output capacity is too small, BS_ERR_UNLUCKY when fewer than the needed primes agree on
 * the minimal gcd degree. */
int bs_squarefree_part(bs_ctx *ctx, const bs_upoly *r, bs_upoly *out);

/* gcd of a and b in Z[x] (Sec. 5.1 "Computing gcds in Z[x]"): the primitive gcd times
 * the gcd of the contents, with a positive leading coefficient; gcd(0, 0) is the zero
 * polynomial (out->deg = -1) and gcd(0, u) is u with a positive leading coefficient.
 * Primes dividing lc(a) lc(b) are skipped and only primes with the minimal gcd degree are
 * used (Brown's rule); the images are lifted by Chinese remaindering up to Mignotte's
 * bound 2^deg ||a||_2 for the input a of smaller norm.
 *
 * a, b, out: host buffers in the layout of bs_squarefree_part; out->c == NULL is a size
 * query (upper bounds).  The call waits for the device.  Errors: BS_ERR_ARG,
 * BS_ERR_RANGE (deg a + deg b + 3 words above one block's shared memory, or a bound above
 * the prime table), BS_ERR_CAPACITY, BS_ERR_UNLUCKY. */
int bs_gcd_z(bs_ctx *ctx, const bs_upoly *a, const bs_upoly *b, bs_upoly *out);

/* n modular gcd jobs in one pass of launches: kind[j] = 0 computes gcd(a[j], b[j]) as
 * bs_gcd_z, kind[j] = 1 the square-free part of a[j] as bs_squarefree_part, kind[j] = 2
 * the exact quotient a[j] / b[j] (b[j] must divide a[j] in Z[x]: a remainder modulo a
 * prime is reported as BS_ERR_ARG, a quotient that is not integral is not detected; the
 * images a mod p / b mod p for primes not dividing lc(b) are lifted under Mignotte's bound
 * 2^deg(q) ||a||_2).  b may be NULL when every kind is 1.  If any out[j].c is NULL, every
 * out[j] receives its upper bounds and nothing runs.  Returns the first failing job's
 * status. */
int bs_modgcd_batch(bs_ctx *ctx, int n, const int *kind, const bs_upoly *a, const bs_upoly *b,
                    bs_upoly *out);

/* Square-free factorisation of a non-zero R in Z[x] by Yun's algorithm (Sec. 2.1,
 * BiProject): the primitive, square-free, pairwise coprime r_1, ..., r_s with positive
 * leading coefficients and R = c r_1 r_2^2 ... r_s^s for an integer c; r_s is not
 * constant, and a multiplicity below s that R does not have gives r_i = 1.  A constant R
 * has no factors (s = 0).  Yun's algorithm runs modulo many primes; primes dividing lc(R)
 * are skipped and only those with the minimal deg gcd(R, R') mod p are used (they agree
 * on the factor degrees); the images lc(R) monic(r_i) are lifted by Chinese remaindering
 * up to Mignotte's bound 2^deg(r_i) ||R||_2, and their contents removed (Sec. 5.1).
 *
 * r: host buffer in the layout of bs_squarefree_part.
 * out: host buffer owned by the caller receiving the factors packed one after the other:
 * the deg r_1 + 1 coefficients of r_1 (ascending), then those of r_2, and so on, out->limbs
 * limbs each (sign-extended); on success out->deg = (total coefficients) - 1, or -1 for s = 0.
 * fdeg: host array of cap_factors entries receiving deg r_1, ..., deg r_s; *nfac = s.
 * With out->c == NULL the call only writes upper bounds (out->deg = 2 deg R - 1, out->limbs,
 * *nfac = deg R as the factor capacity) and returns BS_OK.
 *
 * The call waits for the device.  Errors: BS_ERR_ARG, BS_ERR_ZERO for R = 0, BS_ERR_RANGE
 * when 4 (deg r + 1) words exceed one block's shared memory or the bound exceeds the prime
 * table, BS_ERR_CAPACITY when out or cap_factors is too small, BS_ERR_UNLUCKY when fewer
 * than the needed primes agree on the minimal gcd degree and the factor degrees. */
int bs_squarefree_factorization(bs_ctx *ctx, const bs_upoly *r, int cap_factors, int32_t *fdeg,
                                int32_t *nfac, bs_upoly *out);

/* n factorisations in one pass of launches: job j reads r[j] and writes out[j], nfac[j]
 * and fdeg[j * cap_factors ...].  If any out[j].c is NULL, every job receives its upper
 * bounds and nothing runs.  Returns the first failing job's status. */
int bs_squarefree_factorization_batch(bs_ctx *ctx, int n, const bs_upoly *r, int cap_factors,
                                      int32_t *fdeg, int32_t *nfac, bs_upoly *out);

/* ---------------------------------------------------------------------------------
 * Principal subresultant coefficients (Sec. 3.3, "(Exact) Computation of N")
 * ------------------------------------------------------------------------------ */

/* sr_0, ..., sr_(q-1) of f and g with respect to the eliminated variable (var as in
 * bs_resultant), q = min(m_e, n_e) for the actual degrees m_e, n_e (q = 0 when either
 * polynomial is zero or constant in that variable).  sr_i is the coefficient of the i-th
 * power in the i-th subresultant: the determinant of the Sylvester-like matrix with
 * n_e - i shifted rows of f and m_e - i shifted rows of g whose columns run from the
 * highest power down to the i-th; sr_0 is the resultant.  Computed exactly, by the modular
 * route of the resultant (same primes, points, rejection rule and bounds: each sr_i is a
 * minor of the Sylvester matrix).
 *
 * out: caller-owned array of cap_q host polynomials; out[i] receives sr_i in the layout
 * of bs_resultant (out[i].deg = -1 for the zero polynomial).  *q receives q.  With out ==
 * NULL or out[0].c == NULL the call is a size query: *q and, for i < min(q, cap_q), upper
 * bounds in out[i].deg and out[i].limbs.  The call waits for the device.
 * Errors: BS_ERR_ARG, BS_ERR_RANGE (degree in the eliminated variable above 64, transform
 * or prime table too small), BS_ERR_CAPACITY (cap_q < q or an output too small),
 * BS_ERR_UNLUCKY. */
int bs_psc(bs_ctx *ctx, const bs_bipoly *f, const bs_bipoly *g, int var, int cap_q, int32_t *q,
           bs_upoly *out);

/* The psc sequence modulo one prime (Sec. 3.3, "Computation of N^-"): sr_i mod p for the
 * first table prime p that the rejection rule of the resultant accepts (p divides no
 * leading coefficient of f and g; *p receives it).  *q as for bs_psc.  With coef == NULL
 * a size query: *q and *dmax (the degree bound; residues need dmax + 1 words per index).
 * Otherwise *dmax is the caller's capacity (at least the bound): coef[i * (dmax + 1) + j]
 * receives coefficient j of sr_i mod p in [0, p), deg[i] its degree (-1 for zero).
 * Errors as for bs_psc. */
int bs_psc_modp(bs_ctx *ctx, const bs_bipoly *f, const bs_bipoly *g, int var, int32_t *q,
                int32_t *dmax, int32_t *deg, uint32_t *coef, uint32_t *p);

/* The number N of distinct points of the curve f = 0 over its critical values with
 * respect to the eliminated variable (var = 1: over the roots of R = res(f, f_y; y)), and
 * the square-free decomposition R* = R_1 R_2 ... by fibers (Sec. 3.3): R_i(alpha) = 0
 * exactly when f(alpha, y) has n_y - i distinct roots, N = sum_i (n_y - i) deg R_i.
 * mode 0: exact (psc's in Z[x], gcds in Z[x]); mode 1: the lower bound N^- from the same
 * chain over Z_p for one prime (*p receives it; 0 in mode 0); mode 2: the upper bound
 * N^+ = deg R* n_y - deg R + deg gcd(R^inf mod p, Q mod p) with Teissier's Q (see
 * bs_teissier_q) for one prime p (*p receives it; *s = 0).  f must have a constant
 * leading coefficient in the eliminated variable (no vertical asymptote) and at most 63
 * limbs per coefficient.  degs[i - 1] = deg R_i for i = 1..*s (cap entries available).
 * Errors: BS_ERR_ARG (non-constant leading coefficient, bad arguments), BS_ERR_ZERO (f = 0,
 * or R = 0: f is not square-free), BS_ERR_CAPACITY (cap < s), BS_ERR_RANGE, BS_ERR_UNLUCKY. */
int bs_fiber_count(bs_ctx *ctx, const bs_bipoly *f, int var, int mode, int cap, int32_t *degs,
                   int32_t *s, int64_t *N, uint32_t *p);

/* Content of f with respect to the eliminated variable (var as in bs_resultant): h = the
 * gcd in Z[x] of f's coefficients f_0, ..., f_n (polynomials in the other variable), with
 * a positive leading coefficient, and optionally the primitive part f / h as its rows
 * (Sec. 4: a non-constant content defines vertical lines, which the curve analysis
 * divides out first).  The gcds (a pairwise tree, batched) and the quotients run on the
 * device by the modular route.
 * h: caller-owned output in the layout of bs_squarefree_part.  rows: NULL, or an array of
 * cap_rows outputs receiving (f / h)_0, ..., (f / h)_n; *nrows = n + 1 (n the degree in the
 * eliminated variable).  With h->c == NULL, or rows[0].c == NULL when rows are asked for,
 * a size query: *nrows and upper bounds in h and rows[e].
 * Errors: BS_ERR_ARG, BS_ERR_ZERO (f = 0), BS_ERR_CAPACITY, BS_ERR_RANGE, BS_ERR_UNLUCKY. */
int bs_content(bs_ctx *ctx, const bs_bipoly *f, int var, bs_upoly *h, int cap_rows, bs_upoly *rows,
               int32_t *nrows);

/* The d-th subresultant polynomial S_d(f, g) = sum_j s_j y^j with respect to the eliminated
 * variable (var as in bs_resultant), 0 <= d < min(m, n) for the actual degrees m, n of f
 * and g in that variable (Sec. 3.3: the Sres_i matrix with n - d shifted rows of f, m - d
 * rows of g and the polynomials in its last column; s_d = sr_d).  The coefficients s_j are
 * minors of the Sylvester matrix, so the resultant's plan, primes, points, rejection rule
 * and bounds serve them; each (prime, point) image stops the division-free elimination of
 * the psc stage when the shorter polynomial first reaches degree d.
 * out: caller-owned array of cap host polynomials; out[j] receives s_j in the layout of
 * bs_resultant (deg -1 for zero), *n = d + 1.  With out == NULL or out[0].c == NULL a size
 * query (*n and upper bounds in out[j]).  The call waits for the device.
 * Errors: BS_ERR_ARG (d out of range, bad arguments), BS_ERR_CAPACITY (cap < d + 1 or an
 * output too small), BS_ERR_RANGE, BS_ERR_UNLUCKY as for bs_psc. */
int bs_subresultant(bs_ctx *ctx, const bs_bipoly *f, const bs_bipoly *g, int var, int d, int cap,
                    int32_t *n, bs_upoly *out);

/* gcd(f, g) in Z[x, y] (Sec. 3.3 takes h = gcd(f_x, f_y)), by the eliminated variable var:
 * gcd(cont f, cont g) * pp(S_d(f, g)), where cont is the gcd in Z[x] of the coefficients
 * with respect to the eliminated variable, d the index of the first principal subresultant
 * coefficient that is not identically zero (d = the degree of the gcd in that variable),
 * and pp divides by the content; when every sr_i vanishes the polynomial of smaller degree
 * replaces S_d.  The result has a positive leading coefficient (the highest power of the
 * other variable in its top row).  gcd(0, g) = +-g with that sign; gcd(0, 0) has no rows.
 * The psc sequence, S_d, the contents, the exact quotients and the product by the
 * content's gcd all run on the device.
 * rows: caller-owned array of cap_rows host polynomials receiving the coefficients h_j of
 * the powers of the eliminated variable (layout of bs_squarefree_part), *nrows = deg + 1.
 * With rows == NULL or rows[0].c == NULL a size query (it runs the computation and writes
 * the exact sizes).  Errors: BS_ERR_ARG, BS_ERR_CAPACITY, BS_ERR_RANGE, BS_ERR_UNLUCKY. */
int bs_gcd_bivariate(bs_ctx *ctx, const bs_bipoly *f, const bs_bipoly *g, int var, int cap_rows,
                     bs_upoly *rows, int32_t *nrows);

/* Teissier's Q = res(f_x*, f_y*; y) of Sec. 3.3 exactly, where f_x* = f_x / h, f_y* = f_y / h
 * and h = gcd(f_x, f_y) as bs_gcd_bivariate returns it (for var = 0 the roles of x and y are
 * exchanged), and *d = deg_y h.  With m, n the y-degrees of f_x and f_y, the cofactor
 * property of subresultants gives sr_d(f_x, f_y) = lc_y(h)^(m + n - 2d) Q, so Q is one exact
 * quotient in Z[x] of the psc sr_d by a power of lc_y(h); when every sr_i vanishes (or one
 * derivative is free of y) one cofactor is free of y and Q is its power.  No condition on
 * lc_y(f); f_x = 0 gives Q = 0 (deg -1).
 * Q: caller-owned output in the layout of bs_squarefree_part; Q->c == NULL is a size query
 * (it runs the computation).  Errors as for bs_gcd_bivariate, BS_ERR_ZERO for f = 0,
 * BS_ERR_RANGE for coefficients of f of 64 limbs (the derivatives need one more). */
int bs_teissier_q(bs_ctx *ctx, const bs_bipoly *f, int var, bs_upoly *Q, int32_t *d);

/* The square-free part R* of a non-zero R in Z[x] split by the multiplicity of a non-zero
 * Q at its roots (Sec. 3.3: Teissier's test weighs mult(R, alpha) against mult(Q, alpha) at
 * the critical values alpha, Q as returned by bs_teissier_q): the primitive, pairwise
 * coprime c_0, c_1, ..., c_t with positive leading coefficients and R* = c_0 c_1 ... c_t,
 * where c_k(alpha) = 0 exactly for the roots alpha of R with mult(Q, alpha) = k; c_t is
 * not constant unless t = 0, and a multiplicity below t that no root has gives c_k = 1.
 * With Yun's factorisation Q = c q_1 q_2^2 ... q_s^s (bs_squarefree_factorization),
 * c_k = gcd(R*, q_k) for k >= 1 and c_0 = R* / gcd(R*, Q*), Q* the square-free part of Q;
 * the square-free parts, the factorisation, the gcds and the quotient run on the device by
 * the modular route (four passes of launches).
 * r, q: host buffers in the layout of bs_squarefree_part.
 * out, fdeg, nfac: as for bs_squarefree_factorization, with c_0, ..., c_t packed one after
 * the other, fdeg[k] = deg c_k (cap_factors entries available) and *nfac = t + 1.  With
 * out->c == NULL the call only writes upper bounds (out->deg = deg R + deg Q, out->limbs,
 * *nfac = deg Q + 1 as the factor capacity) and returns BS_OK.
 * Errors: BS_ERR_ARG, BS_ERR_ZERO (R = 0 or Q = 0), BS_ERR_CAPACITY, BS_ERR_RANGE and
 * BS_ERR_UNLUCKY as for bs_squarefree_factorization and bs_gcd_z. */
int bs_root_multiplicity(bs_ctx *ctx, const bs_upoly *r, const bs_upoly *q, int cap_factors,
                         int32_t *fdeg, int32_t *nfac, bs_upoly *out);

/* Launch shapes of the batched stages (bs_autotune_batch). */
typedef struct {
  int32_t eval_warps;          /* rows (one warp each) per evaluation block, 1..8 */
  int32_t eval_blocks_per_sm;  /* cap of the persistent evaluation grid */
  int32_t uni_threads[6];      /* threads per univariate-resultant block by degree class
                                  (eliminated-variable length <= 8, 16, 24, 33, 48, 65): 64, 128 or 256 */
  int32_t crt_tile;            /* coefficients (one warp each) per reconstruction block: 1, 2, 4, 8 */
  int32_t crt_blocks_per_sm;   /* cap of the persistent reconstruction grid */
  float ms_default;            /* device time of the batch's stages with the default shapes */
  float ms_tuned;              /* ... with the chosen shapes (CUDA events, best of two runs) */
  int32_t trials;              /* shape combinations measured */
  int32_t eval_independent;    /* 1: evaluation by independent warps (one row each, the prime's
                                  tables read through L1; eval_warps unused), 0: blocks of
                                  eval_warps rows of one prime with the tables staged */
} bs_tune_info;

/* Autotune the launch shapes for batches like this one: plans and uploads the batch, then
 * runs its stages on the context's stream once per candidate shape (coordinate descent:
 * evaluation warps per block and grid, the evaluation variant, univariate threads per
 * block for each degree class present, reconstruction tile and grid), keeping for each
 * stage the shape with the least device time.  The chosen shapes stay on the context and
 * apply to its later bs_resultant_batch and bs_resultant calls; of them only the
 * evaluation variant also applies to the device-planned entry points.  *info (may be
 * NULL) receives them.  Results are not returned; the call waits for the device.  Errors
 * as bs_resultant_batch. */
int bs_autotune_batch(bs_ctx *ctx, int n, const bs_bipoly *f, const bs_bipoly *g, int var,
                      bs_tune_info *info);

/* Set the batched launch shapes explicitly (t == NULL restores the defaults: evaluation
 * by independent warps with 5 blocks of 7 warps per SM, 128 threads per univariate block, 8
 * coefficients and 4 blocks per SM for reconstruction).  The timing fields of *t are
 * ignored.  BS_ERR_ARG for a shape outside the ranges of bs_tune_info. */
int bs_set_tune(bs_ctx *ctx, const bs_tune_info *t);

/* ---------------------------------------------------------------------------------
 * Serving: continuous batching of resultant and gcd jobs
 *
 * bs_serve_start() starts `slots` worker threads on the context, each with its own CUDA
 * stream, and one device arena of `arena_bytes` (0: half the free device memory, capped
 * by the context's budget).  bs_submit() copies a job's operands and queues it.  A free
 * worker forms a batch from the queued jobs of the head job's type (resultants in y,
 * resultants in x, or gcd / square-free jobs) and work class (a resultant whose plan
 * counts more than 2e9 multiply-reduce operations in its univariate stage, about a
 * millisecond of the GPU, is large, one of at most 2e8 tiny, any other job small), first
 * come first served and at most `max_batch` jobs; with two or more slots the last half of
 * the workers (at least one) take no large jobs.  Tiny and small
 * batches run on a stream of the highest priority, large ones on a stream of the lowest
 * with grids of short blocks sized by their work, so small jobs neither queue behind
 * large ones nor wait for a large kernel to free the SMs (their blocks start as the large
 * kernel's blocks end), and a large batch alone still has the whole GPU.  The batch is
 * admitted once the arena can hold it; the worker then runs the batch
 * (one graph launch for resultants, one pass of launches for gcds), posts the results
 * and frees the arena space.  Workers run concurrently, so batches admitted while
 * others are on the GPU overlap with them.  Every intermediate (residues, images,
 * reconstructions) stays in the arena; only operands and results cross PCIe.
 *
 * While a serving loop runs, the context accepts only bs_submit, bs_poll, bs_wait,
 * bs_serve_stats and bs_serve_stop; its other compute entry points return BS_ERR_ARG.
 * These five may be called from any host thread.
 * ------------------------------------------------------------------------------ */

#define BS_JOB_RESULTANT 0  /* res(f, g; var) */
#define BS_JOB_GCD       1  /* gcd(a, b) in Z[x], as bs_gcd_z */
#define BS_JOB_SQFREE    2  /* square-free part of a, as bs_squarefree_part */

typedef struct {
  int32_t kind;      /* BS_JOB_* */
  int32_t var;       /* resultants: 0 eliminates x, 1 eliminates y */
  bs_bipoly f, g;    /* resultant operands (copied by bs_submit) */
  bs_upoly a, b;     /* gcd operands; b unused for BS_JOB_SQFREE (copied by bs_submit) */
} bs_job;

typedef struct {
  int32_t status;    /* the job's status (BS_OK or an error code) */
  int32_t deg;       /* degree of the result (-1: zero polynomial) */
  int32_t limbs;     /* limbs per coefficient of the result */
  uint32_t *c;       /* caller buffer for the coefficients, or NULL (shape only) */
  int64_t cap_words; /* capacity of c in uint32 words */
  double queue_ms;   /* submit -> admitted into a batch */
  double latency_ms; /* submit -> result ready */
} bs_result;

typedef struct {
  int64_t submitted, completed, batches, jobs_in_batches, queued;
  int32_t inflight, max_inflight;   /* batches on the GPU now / at most at once */
  int64_t arena_bytes, arena_used, arena_peak;
  /* wall time summed over the batches run so far, per phase of a batch: host planning,
   * device work (upload, kernels and download, until the slot's stream is idle; batches
   * of several slots overlap) and the formatting of the results */
  double host_plan_ms, device_ms, host_finish_ms;
} bs_serve_info;

/* Start the serving loop (1 <= slots <= 16, max_batch >= 1).  BS_ERR_NOMEM if the arena
 * cannot be allocated or exceeds the context's budget. */
int bs_serve_start(bs_ctx *ctx, int slots, int max_batch, size_t arena_bytes);

/* Finish every queued and running job, then stop the workers and free the arena.
 * Tickets not yet collected are dropped. */
int bs_serve_stop(bs_ctx *ctx);

/* Queue a job; *ticket identifies it.  The operands are validated and planned here:
 * BS_ERR_ARG / BS_ERR_RANGE for a bad job, BS_ERR_NOMEM when the job alone needs more
 * device memory than the arena holds. */
int bs_submit(bs_ctx *ctx, const bs_job *job, uint64_t *ticket);

/* BS_PENDING while the job runs or waits.  Once it has finished: fills r (status, deg,
 * limbs, timings) and returns BS_OK; if r->c is not NULL and holds (deg + 1) * limbs
 * words, the coefficients are copied there and the ticket is released (a later poll of
 * it returns BS_ERR_ARG).  BS_ERR_CAPACITY if r->c is too small. */
int bs_poll(bs_ctx *ctx, uint64_t ticket, bs_result *r);

/* Block until the job has finished or timeout_ms elapsed (negative: no limit);
 * BS_OK or BS_ERR_TIMEOUT. */
int bs_wait(bs_ctx *ctx, uint64_t ticket, int timeout_ms);

/* Counters of the serving loop. */
int bs_serve_stats(bs_ctx *ctx, bs_serve_info *out);

/* ---------------------------------------------------------------------------------
 * Measurement
 *
 * Every stage's kernel launches lie in an NVTX range named "bs.plan", "bs.eval",
 * "bs.unires", "bs.interp" or "bs.crt", and bs_resultant, bs_resultant_batch,
 * bs_resultant_device and each served batch ("bs.serve.batch", "bs.serve.large_batch")
 * in one of their own, so that a profiler can select them (ncu --nvtx --nvtx-include
 * "bs.unires/"); without a tool attached the ranges cost nothing.
 * ------------------------------------------------------------------------------ */

/* Throughput of one integer-multiply instruction kind on every SM of the context's
 * device, in operations per second: kind 0 mad.lo.u32, 1 mad.hi.u32, 2 mad.wide.u32,
 * 3 one Montgomery multiplication mod a 31-bit prime as the kernels perform it.  Runs a
 * few short kernels on the context's stream and waits for them. */
int bs_alu_probe(bs_ctx *ctx, int kind, double *ops_per_s);

/* Turn per-stage timing on or off.  When on, resultant calls record CUDA events on the
 * context's stream around the stages (and do not use CUDA graphs). */
int bs_profile(bs_ctx *ctx, int enable);

/* Milliseconds of the stages of the most recent resultant call, measured with CUDA
 * events on the context's stream: ms[0] plan, ms[1] reduce + evaluate, ms[2] univariate
 * resultants, ms[3] interpolation, ms[4] reconstruction (n entries are written, n <= 5).
 * Waits for the call to finish.  BS_ERR_ARG if profiling is off. */
int bs_stage_times(bs_ctx *ctx, float *ms, int n);

#ifdef __cplusplus
}
#endif

#endif /* BSRES_H */
