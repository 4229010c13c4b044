/* polymul.h -- C-ABI of the GB300 sparse multivariate polynomial product.
 *
 * The library computes the exact schoolbook product h = f * g of two sparse
 * multivariate polynomials held in distributed format: a list of terms, each
 * a coefficient with an exponent vector (Gastineau & Laskar, "Highly Scalable
 * Multiplication for Distributed Sparse Multivariate Polynomials on Many-core
 * Systems", Sec. 1 and Sec. 2).  Every pairwise term product
 * a_i b_j x^(alpha_i + beta_j) is formed and equal monomials are combined
 * into a result sorted in ascending monomial order (Sec. 2, Alg. 1).
 *
 * All compute runs in the library's CUDA kernels for sm_103a.  Every pointer
 * named "device" below must be device memory of the current CUDA device (for
 * example a PyTorch CUDA tensor's data pointer); the library never frees
 * caller memory.  `stream` is a cudaStream_t passed as void* (NULL = the
 * legacy default stream); all work is ordered on it.  Calls return only after
 * the result is complete and its size is known on the host.
 *
 * Monomial order: lexicographic with x_1 most significant.  Exponents are
 * packed into one 64-bit key (Sec. 7: "packed on a 64-bit unsigned
 * integer"): x_1 occupies the most significant field.  Each field's width
 * counts one guard bit (the field's top bit): every exponent must be
 * < 2^(w_v - 1), so adding two packed keys never carries between fields and
 * multiplying two monomials is one integer add.
 *
 * Coefficient rings:
 *   PM_COEF_M61        uint64 inputs (any value, reduced mod p on load),
 *                      results in [0, p), p = 2^61 - 1.
 *   PM_COEF_I64_ACC128 int64 inputs, exact results as int128 stored as two
 *                      uint64 words per term (low word first, two's
 *                      complement); products whose int128 bound rule fails
 *                      are refused (PM_ECOEF_BOUND).
 *   PM_COEF_I64_ACC192 int64 inputs, exact results as 192-bit integers,
 *                      three uint64 words per term (low word first, two's
 *                      complement): a sum of at most 2^31 products of
 *                      magnitude <= 2^126 always fits, so no bound rule
 *                      applies (the batched and no-allocation entry points
 *                      do not take this kind).
 *
 * Input conventions: terms in any order; a repeated monomial's coefficients
 * are summed; zero coefficients are dropped.  The result never holds a zero
 * coefficient or a repeated monomial (the canonical form of Sec. 2).
 */
#ifndef POLYMUL_H
#define POLYMUL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PM_MAX_VARS 16

/* ---- error codes (negative) ---------------------------------------------- */
#define PM_OK             0
#define PM_EINVAL        -1  /* bad packing, kind, pointer or size              */
#define PM_EEXP_OVERFLOW -2  /* an input or product exponent reaches its guard  */
#define PM_ECOEF_BOUND   -3  /* int64 kind: the int128 bound rule fails         */
#define PM_ECAPACITY     -4  /* h->cap too small; h->n holds the needed size    */
#define PM_ENOMEM        -5  /* device scratch allocation failed                */
#define PM_ETIMEOUT      -6  /* a bounded device wait gave up                   */
#define PM_ECUDA         -7  /* a CUDA runtime call failed                      */
#define PM_EPLAN         -8  /* a plan's inputs no longer match it (pm_plan_*)  */
#define PM_ECANCELED     -9  /* a serving request was cancelled before admission */

/* ---- types ---------------------------------------------------------------- */

/* Exponent packing: nvars in [1, 16]; field_bits[v] in [1, 32] is the width
 * of x_{v+1}'s field including its guard bit; the widths sum to <= 64. */
typedef struct pm_packing {
    uint32_t nvars;
    uint8_t field_bits[PM_MAX_VARS];
} pm_packing;

typedef enum pm_coef_kind {
    PM_COEF_M61 = 0,
    PM_COEF_I64_ACC128 = 1,
    PM_COEF_I64_ACC192 = 2
} pm_coef_kind;

/* Input terms (device): exps is n x nvars uint32, row-major; coefs is n
 * uint64 (M61) or n int64 (I64 kinds).  n < 2^31. */
typedef struct pm_terms_in {
    const uint32_t *exps;
    const void *coefs;
    uint64_t n;
} pm_terms_in;

/* Output terms (device): keys is cap packed uint64 keys; coefs is cap uint64
 * (M61) or 2*cap uint64 words (I64_ACC128).  On success n = number of terms
 * written.  On PM_ECAPACITY n = the number of terms the result has. */
typedef struct pm_terms_out {
    uint64_t *keys;
    void *coefs;
    uint64_t n;
    uint64_t cap;
} pm_terms_out;

/* Strategies for the per-range accumulate step. */
#define PM_STRATEGY_AUTO   0  /* autotuner's choice (default)                      */
#define PM_STRATEGY_DIRECT 1  /* direct-addressed shared-memory accumulation       */
#define PM_STRATEGY_SORT   2  /* shared-memory radix sort + segmented reduce       */
#define PM_STRATEGY_HASH   3  /* hashed windows: a shared-memory hash table per
                                 window of up to 2^31 ranks (sparse results in
                                 large boxes)                                      */
#define PM_STRATEGY_BUCKET 4  /* every term product written to a bucket of the
                                 output key space (two passes over the
                                 pp-matrix), each bucket sorted and reduced in
                                 shared memory: results about as large as the
                                 term products (mod p and int128 kinds; takes
                                 32 or 56 bytes of scratch per term product)    */

/* Tuning knobs; pass NULL (or zeros) for the autotuned defaults. */
/* Direct strategy accumulators (mod p kind). */
#define PM_ACC_AUTO   0  /* direct: three limbs; hash: limbs when
                            min(n_f, n_g) <= 65537, else wide, with the limbs
                            in windows of at most 65537 rows with products   */
#define PM_ACC_WIDE   1  /* 64-bit sum + 32-bit wrap count per slot             */
#define PM_ACC_LIMBS  2  /* four 16-bit limbs in 32-bit counters per slot       */
#define PM_ACC_LIMBS3 3  /* direct: three limbs (22, 21, 21 bits) in 32-bit
                            counters per slot, normalised between the passes
                            of at most 1023 rows (any operand sizes)           */

typedef struct pm_options {
    int32_t strategy;          /* PM_STRATEGY_*                                     */
    uint32_t slots;            /* direct: output slots per window (0 = the most
                                  shared memory allows)                            */
    uint32_t chunk;            /* sort: term products per range (<= 4096)            */
    uint32_t ranges_per_sm;    /* direct: groups per SM; sort: unused                 */
    int32_t accumulator;       /* PM_ACC_*; PM_ACC_LIMBS needs min(n_f, n_g) <= 65537;
                                  PM_ACC_LIMBS3 applies to the direct strategy  */
    uint32_t cost_row;         /* direct: group cost model, cost of one row of f
                                  reaching a window, in term products (0 = 3)       */
    uint32_t cost_window;      /* direct: cost of one window in term products
                                  (0 = 23000); the groups balance
                                  products + cost_row rows + cost_window windows    */
    uint32_t grid_l;           /* the parameter l of the Sec. 5 almost regular grid
                                  ((l+1)^2 points of the pp-matrix, 1..4096; 0 =
                                  chosen from the sizes): sort, the first
                                  splitters before counting and refinement;
                                  direct, the cost sample of the groups.  64 is
                                  the paper's setting.  The result does not
                                  depend on it                                      */
} pm_options;

/* Per-call counters (all optional; pass NULL). */
typedef struct pm_stats {
    uint64_t n_f, n_g;         /* canonical operand sizes                         */
    uint64_t term_products;    /* n_f * n_g                                       */
    uint64_t n_out;            /* result terms                                    */
    uint64_t n_ranges;         /* output key ranges (one CTA each; hash: windows
                                  run over all rounds)                            */
    uint64_t box;              /* output-exponent box size used for ranks          */
    int32_t strategy;          /* PM_STRATEGY_DIRECT, _SORT, _HASH or _BUCKET     */
    uint32_t refine_rounds;    /* partition refinement rounds (sort); window
                                  rounds (hash); buckets sorted outside shared
                                  memory (bucket)                                 */
    uint32_t kernel_launches;  /* kernels launched by the call                     */
    uint32_t host_syncs;       /* stream synchronisations by the call              */
    float ms_range_kernel;     /* device time of the accumulate kernel alone: one
                                  launch of k_direct or k_range_sort (ms)         */
    float ms_range_step;       /* device time of the range step: windows,
                                  FindEdge and the accumulate kernel (ms)         */
} pm_stats;

/* ---- entry points ---------------------------------------------------------- */

/* h = f * g (Sec. 2, Alg. 1).  Steps, all on the device:
 *   (a) pack exponents into guard-bit keys, reduce coefficients, sort each
 *       operand and combine repeated monomials (Sec. 7 packing);
 *   (b) split the output key space into disjoint left-closed, right-open
 *       ranges [S_k, S_{k+1}) whose term-product counts O_k are balanced
 *       (Sec. 2 first step, Sec. 3 operation counts);
 *   (c)+(d) one CTA per range forms its term products from per-row column
 *       bounds (FindEdge, Sec. 2) and accumulates them in shared memory,
 *       with no atomics or locks on the result (Alg. 1 second step);
 *   (e) drops zero coefficients and concatenates the ranges in ascending
 *       order (Alg. 1, last line).
 * Errors: PM_EINVAL, PM_EEXP_OVERFLOW, PM_ECOEF_BOUND (int64 kind: a
 * repeated input monomial's sum leaves int64, or
 * max|a| * max|b| * min(n_f, n_g) >= 2^127 over the canonical operands),
 * PM_ECAPACITY (h->n set to the needed size), PM_ENOMEM, PM_ECUDA.  On any
 * error h's buffers hold unspecified data and h->n = 0 except for
 * PM_ECAPACITY.  Scratch memory comes from the device's stream-ordered
 * allocator and is released before return. */
int pm_polymul(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
               pm_terms_out *h, const pm_options *opt, pm_stats *stats, void *stream);

/* ---- the product on a caller-owned workspace ----------------------------------
 *
 * Alg. 1 (Sec. 2) takes the operands A, B and gives C; its working storage
 * -- the canonical operands, the splitters S_k, the per-row edges of
 * FindEdge, the per-interval results D_k before their concatenation -- is
 * the implementation's.  pm_polymul takes it from the device's stream-
 * ordered allocator.  For callers that own all device memory (an engine
 * with its own arena, a framework allocator), the same product runs on a
 * workspace the caller allocates, and the call itself allocates no device
 * memory:
 *
 *   pm_workspace_size  runs the product once on the given inputs (its own
 *                      scratch from the stream-ordered allocator, no output
 *                      written) and reports the workspace bytes a
 *                      pm_polymul_ws call on the same inputs, options and
 *                      autotuner state takes, and the result size (so h can
 *                      be sized too).  The bytes are exact for the direct
 *                      and sort strategies; for the hashed-window strategy,
 *                      whose window splits can differ between runs (a window
 *                      is split when a bounded hash-table probe runs out,
 *                      which depends on the order of concurrent inserts),
 *                      they include a margin of one quarter.
 *   pm_polymul_ws      pm_polymul with every scratch block carved from
 *                      `workspace` (device memory of workspace_bytes,
 *                      256-byte aligned).  Running out of workspace returns
 *                      PM_ENOMEM (h->n = 0) before any kernel touches memory
 *                      past its end.  The workspace must not be used by
 *                      anything else until the call's work on `stream` is
 *                      done (the call synchronises `stream` before a
 *                      successful return).
 * Errors are those of pm_polymul, plus PM_EINVAL for a misaligned or null
 * workspace with nonzero size. */
int pm_workspace_size(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                      const pm_options *opt, uint64_t *workspace_bytes, uint64_t *n_out, void *stream);
int pm_polymul_ws(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                  pm_terms_out *h, const pm_options *opt, pm_stats *stats, void *workspace,
                  uint64_t workspace_bytes, void *stream);

/* ---- slices of the output key space (Alg. 2: one product over several GPUs) --
 *
 * Alg. 2 (Sec. 3) spreads one product over N nodes: every node holds A and
 * B, the intervals [S_k, S_{k+1}) of the first step are split into N
 * groups of consecutive intervals by their cumulative operation counts
 * O_k, each node computes the terms of its group, and the slices are
 * gathered in ascending order.  The groups own disjoint key ranges, so the
 * gather is a concatenation: no reduction.
 *
 *   pm_shard_bounds      the split: bounds[0..nshards] (host) with
 *                        bounds[0] = 0, bounds[nshards] = 2^64 - 1, and
 *                        bounds[m] for 0 < m < nshards the first splitter
 *                        S_k (the Sec. 5 grid over the canonical operands,
 *                        about 64 intervals per shard) whose count of term
 *                        products below it reaches m / nshards of all of
 *                        them.  products[m] (host, optional) receives shard
 *                        m's term products.  Deterministic: every rank that
 *                        calls it on the same inputs gets the same bounds.
 *   pm_polymul_range     pm_polymul restricted to the result terms whose
 *                        packed key k has key_lo <= k < key_hi; the
 *                        concatenation of the slices of consecutive bounds
 *                        is the whole product, bit for bit.  An empty slice
 *                        gives h->n = 0.  Statistics count the whole
 *                        product's operands.
 *   pm_split_cumulative  the host-side rule of the split alone: cum[0..n)
 *                        ascending cumulative counts at n interval
 *                        boundaries; cut[0..nshards] receives, for each
 *                        shard m, the boundary index it starts at: cut[0] =
 *                        0, cut[nshards] = n - 1, and cut[m] the first index
 *                        whose count is at least m / nshards of cum[n-1]
 *                        (never before cut[m-1]).  Host memory only; needs
 *                        no GPU.
 * Errors: those of pm_polymul; PM_EINVAL for nshards outside 1..65536, null
 * arrays, or counts that are not ascending. */
int pm_shard_bounds(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                    uint32_t nshards, uint64_t *bounds, uint64_t *products, void *stream);
int pm_polymul_range(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                     uint64_t key_lo, uint64_t key_hi, pm_terms_out *h, const pm_options *opt, pm_stats *stats,
                     void *stream);
int pm_split_cumulative(const uint64_t *cum, uint32_t n, uint32_t nshards, uint32_t *cut);

/* Upper bound on the number of result terms: min(n_f * n_g, box) with box =
 * prod_v (max_f e_v + max_g e_v + 1) over the input terms.  Sizes h->cap. */
int pm_out_bound(const pm_packing *pk, const pm_terms_in *f, const pm_terms_in *g,
                 uint64_t *bound, void *stream);

/* The first step of Alg. 1 (Sec. 2) with the almost regular grid of Sec. 5:
 * for sorted packed keys alpha[0..na) and beta[0..nb) (device, ascending;
 * the canonical operands), the splitters S -- the grid's points
 * alpha_i + beta_j and gamma_end = alpha[na-1] + beta[nb-1] + 1 (the
 * exclusive end of the last interval), sorted and deduplicated -- into
 * splitters[0..cap) (device).  Grid: rows i = 0, s_i, 2 s_i, ... with
 * s_i = max(floor(na / l), 1); on them columns j = j0 + m s_j with
 * s_j = max(floor(nb / l), 1) and j0 = floor(nb / 2l) on every second grid
 * row, else 0; then the last row and the last column at the same steps
 * (0-based indexes; columns past the matrix clamped to its last).
 * *n_out = |S|.  Errors: PM_EINVAL (l outside 1..4096, null pointers, an
 * operand of 2^31 terms or more), PM_ECAPACITY (*n_out > cap: nothing
 * written).  na = 0 or nb = 0 gives *n_out = 0.  The interval boundaries of
 * the sort strategy start from these splitters; the direct strategy samples
 * its group costs at the same grid points. */
int pm_grid(const uint64_t *alpha, uint64_t na, const uint64_t *beta, uint64_t nb, uint32_t l, uint64_t *splitters,
            uint64_t cap, uint64_t *n_out, void *stream);

/* Unpack n packed keys (device) into an n x nvars uint32 exponent matrix
 * (device, row-major).  Inverse of the packing of Sec. 7. */
int pm_unpack(const pm_packing *pk, const uint64_t *keys, uint64_t n, uint32_t *exps, void *stream);

/* Pack n exponent vectors (device, n x nvars uint32) into keys (device).
 * Fails with PM_EEXP_OVERFLOW if an exponent reaches its guard bit. */
int pm_pack(const pm_packing *pk, const uint32_t *exps, uint64_t n, uint64_t *keys, void *stream);

/* ---- plans: one product, repeated, as a CUDA graph ---------------------------
 *
 * pm_polymul reads a small status block on the host twice per call (input
 * maxima; canonical operand sizes, maxima and extreme keys) and once for
 * the result size, and launches about thirty kernels, so for products of a
 * few hundred microseconds the host's launches and waits are a large part
 * of the call.  A plan runs the product once (filling h, exactly like
 * pm_polymul), records the two status blocks, and captures the whole device
 * path -- packing, canonical operands, groups, windows, FindEdge,
 * accumulation, compaction -- into one CUDA graph.  pm_plan_run replays it:
 * every kernel runs again on the current contents of f's and g's buffers
 * (only the host decisions are reused), with no host synchronisation.
 *
 * Every host decision of the call is a function of the two status blocks,
 * so a replay is exact whenever the blocks it computes equal the recorded
 * ones; on the device, check kernels compare them and on any difference the
 * kernels that index by data return at entry and pm_plan_finish reports
 * PM_EPLAN (the inputs' exponent maxima, canonical sizes or extreme
 * monomials changed: re-create the plan, or call pm_polymul).  Coefficients
 * may change freely (int64 kind: up to the recorded largest magnitudes),
 * and so may monomials that keep those statistics.
 * Products that take the sort strategy (whose partition refinement reads
 * counts on the host) are not captured: their plan runs plain pm_polymul
 * calls (pm_plan_captured returns 0).
 *
 * The pointers in f, g and h are kept by the plan: their buffers must stay
 * allocated and unmoved until pm_plan_destroy.  Scratch memory lives in the
 * graph's allocation nodes.  A plan may be run on any stream; runs of one
 * plan must not overlap. */
typedef struct pm_plan pm_plan;

/* Runs h = f * g once (all pm_polymul errors apply, and fail the plan) and
 * captures the graph.  *plan receives the handle. */
int pm_plan_create(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                   pm_terms_out *h, const pm_options *opt, pm_plan **plan, void *stream);
/* Enqueue one replay on `stream` (asynchronous; h's buffers are rewritten). */
int pm_plan_run(pm_plan *plan, void *stream);
/* Wait for the last replay on `stream`; *n_out = its result size.  Returns
 * PM_OK, PM_EPLAN (inputs no longer match: h holds no result),
 * PM_ECAPACITY (*n_out > h->cap: nothing was written) or PM_ECUDA. */
int pm_plan_finish(pm_plan *plan, uint64_t *n_out, void *stream);
/* Like pm_plan_finish, and the result also lands in host memory: after the
 * last replay on `stream`, one kernel reads the result size on the device
 * and copies that many keys (host_keys[n]) and coefficients (host_coefs,
 * the kind's words per term) from h into page-locked host buffers of
 * host_cap terms (cudaMallocHost / cudaHostAlloc: device-accessible), then
 * one synchronisation.  Returns what pm_plan_finish returns, PM_ECAPACITY
 * also when *n_out > host_cap (nothing copied), PM_EINVAL for null or not
 * page-locked buffers.  For plans that are not captured the copy follows
 * the plain call's result.  The point is one host synchronisation per
 * product instead of one for the size and one for the copies. */
int pm_plan_finish_to_host(pm_plan *plan, uint64_t *host_keys, void *host_coefs, uint64_t host_cap,
                           uint64_t *n_out, void *stream);
/* 1 if the plan replays a captured graph, 0 if it runs plain calls. */
int pm_plan_captured(const pm_plan *plan);
void pm_plan_destroy(pm_plan *plan);

/* ---- autotuning ---------------------------------------------------------------
 *
 * Like the paper's one-time tuning of l (Sec. 5, Sec. 7), but over this
 * library's knobs: pm_autotune runs every candidate configuration (direct
 * strategy x groups per SM x window slots x accumulator, sort strategy x
 * chunk) on the given product, times each with CUDA events on `stream`,
 * returns the fastest in *best and keeps it for the product's shape class
 * (kind, nvars, floor(log2) of n_f, n_g and of pm_out_bound's value);
 * pm_polymul called with NULL or all-zero options uses the kept choice for
 * products of that class.  h receives the product.  pm_batch_autotune does
 * the same for a batch's range size and ranges per work item, timing plans
 * on an evenly spaced sample of at most 256 items. */
#define PM_TUNE_MAX_CANDIDATES 24

typedef struct pm_tune_report {
    uint32_t count;            /* candidates timed                                */
    uint32_t best;             /* index of the fastest                            */
    pm_options candidates[PM_TUNE_MAX_CANDIDATES];
    float ms[PM_TUNE_MAX_CANDIDATES];  /* best of 2 runs; -1 when refused         */
} pm_tune_report;

int pm_autotune(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g, pm_terms_out *h,
                pm_options *best, pm_tune_report *report, void *stream);

/* ---- batches of independent products (one device pass, a CUDA graph) ------
 *
 * Alg. 1 applied to every product of a batch in one pass: per operand,
 * canonical form; per product, the grid splitters of Sec. 5 (first step);
 * one persistent kernel whose CTAs take runs of consecutive output ranges
 * from a device work counter (the dynamic scheduling of Sec. 2) and sort and
 * reduce each range in shared memory; then per product the concatenation of
 * its ranges.  No host synchronisation happens inside the pass, so it is
 * captured once into a CUDA graph when the plan is created and each run
 * replays that graph.  Every product uses the sort strategy.
 *
 * Output placement: an item whose h.cap >= n_f * n_g has its ranges written
 * straight into h, each at the count of its product's term products below
 * the range, and moved left in place when some term products shared a
 * monomial; h[h.n, h.cap) then holds unspecified words.  An item with a
 * smaller h.cap has its ranges written to the plan's workspace and copied
 * into h once their sizes are known (PM_ECAPACITY when they do not fit).
 *
 * Limits: n_f, n_g <= PM_BATCH_MAX_TERMS per product (larger products belong
 * to pm_polymul).  A plan keeps device pointers to the items' inputs and
 * outputs: they must stay valid and unmoved while the plan is used; a run
 * recomputes every product from the current contents of the inputs. */
#define PM_BATCH_MAX_TERMS 8192u

typedef struct pm_batch_item {
    pm_packing pk;
    int32_t coef_kind;         /* pm_coef_kind                                     */
    pm_terms_in f, g;          /* device inputs, as for pm_polymul                 */
    pm_terms_out h;            /* device outputs; h.n is written by finish          */
    int32_t status;            /* written by finish: PM_OK or this item's error    */
} pm_batch_item;

typedef struct pm_batch_options {
    uint32_t range_target;     /* term products per output range: 64..4096 when
                                  every item is PM_COEF_M61 (default 3072),
                                  64..3072 otherwise (default 2048); a larger
                                  value is PM_EINVAL                              */
    uint32_t ranges_per_item;  /* consecutive ranges per work item (default 16)   */
} pm_batch_options;

typedef struct pm_batch_stats {
    uint64_t term_products;    /* sum of n_f * n_g over the items                 */
    uint64_t n_out;            /* result terms of the items that succeeded        */
    uint64_t n_ranges;         /* output ranges over all items                    */
    uint64_t work_items;       /* work-queue entries of the persistent kernel     */
    uint32_t kernel_launches;  /* kernels per run                                 */
    int32_t graph;             /* 1 when runs replay a CUDA graph                 */
} pm_batch_stats;

typedef struct pm_batch_plan pm_batch_plan;  /* opaque */

/* Validate the items, allocate the plan's device memory (cudaMalloc; freed
 * by pm_batch_plan_destroy) and capture the pass into a CUDA graph. */
int pm_batch_plan_create(const pm_batch_item *items, uint32_t count, const pm_batch_options *opt,
                         pm_batch_plan **plan, void *stream);
/* Launch the pass on `stream` (one graph launch; no host synchronisation). */
int pm_batch_plan_run(pm_batch_plan *plan, void *stream);
/* Synchronise `stream`, write each item's status and h.n, fill stats.
 * Returns PM_OK or the first failing item's error code. */
int pm_batch_plan_finish(pm_batch_plan *plan, pm_batch_item *items, pm_batch_stats *stats, void *stream);
void pm_batch_plan_destroy(pm_batch_plan *plan);
/* create + run + finish + destroy */
int pm_batch_polymul(pm_batch_item *items, uint32_t count, const pm_batch_options *opt, pm_batch_stats *stats,
                     void *stream);

typedef struct pm_batch_tune_report {
    uint32_t count, best, sample;
    pm_batch_options candidates[PM_TUNE_MAX_CANDIDATES];
    float ms[PM_TUNE_MAX_CANDIDATES];
} pm_batch_tune_report;

int pm_batch_autotune(const pm_batch_item *items, uint32_t count, pm_batch_options *best,
                      pm_batch_tune_report *report, void *stream);

/* Workspace mode of the same pass, for engines that own their memory and
 * streams: nothing is allocated and nothing synchronises, so it can also be
 * captured into a graph by the caller.  pm_batch_workspace reports the
 * device bytes (256-byte aligned workspace) and pinned host bytes the items
 * need; pm_batch_enqueue puts the pass on `stream`, copying the items'
 * descriptors from host_ws and their results back into host_ws at the end;
 * once the stream has passed that point, pm_batch_collect writes each item's
 * status and h.n from host_ws.  The workspaces must not be reused before
 * then. */
int pm_batch_workspace(const pm_batch_item *items, uint32_t count, const pm_batch_options *opt,
                       uint64_t *device_bytes, uint64_t *host_bytes);
int pm_batch_enqueue(const pm_batch_item *items, uint32_t count, const pm_batch_options *opt, void *device_ws,
                     uint64_t device_bytes, void *host_ws, uint64_t host_bytes, void *stream);
int pm_batch_collect(pm_batch_item *items, uint32_t count, const void *host_ws);

/* ---- serving: a continuous-batching request loop ----------------------------
 *
 * The paper has no serving layer; this is the request loop the library adds
 * around the batched pass.  Requests (one product each, with device-resident
 * inputs and outputs owned by the caller) are admitted in arrival order
 * whenever one of `streams` stream slots and enough of the engine's device
 * arena (`device_budget` bytes, the HBM budget, allocated once at create)
 * and pinned staging are free; the admitted products that fit the batch
 * kernels form one batch (at most `max_batch`), enqueued in workspace mode,
 * so batches admitted while others run overlap on the device.  Products
 * above PM_BATCH_MAX_TERMS go to a worker thread running pm_polymul on its
 * own stream.  A request whose workspace can never fit the budget completes
 * with PM_ENOMEM.  All calls on one server must come from one host thread. */
typedef struct pm_server pm_server;

typedef struct pm_server_config {
    uint64_t device_budget;    /* device arena bytes (default 8 GiB)              */
    uint64_t host_budget;      /* pinned staging bytes (default 64 MiB)           */
    uint32_t streams;          /* batches in flight at most (default 4)           */
    uint32_t max_batch;        /* products per batch at most (default 256)        */
    pm_batch_options batch;
} pm_server_config;

typedef struct pm_server_done {
    uint64_t tag;              /* the caller's tag from pm_server_submit          */
    int32_t status;            /* PM_OK or the product's error code               */
    uint32_t pad;
    uint64_t n;                /* result terms written to the request's h          */
    double t_submit, t_admit, t_done;  /* server clock, seconds                   */
} pm_server_done;

typedef struct pm_server_state_t {
    uint32_t queued, in_flight, big_queued, big_active, max_in_flight, pad;
    uint64_t batches;          /* batches launched so far                         */
    uint64_t device_used;      /* arena bytes held by batches in flight           */
    double clock;              /* server clock, seconds                           */
} pm_server_state_t;

int pm_server_create(const pm_server_config *cfg, pm_server **srv);
/* Queue one product (the descriptor is copied; the device buffers it points
 * to must stay valid until the request completes). */
int pm_server_submit(pm_server *srv, const pm_batch_item *item, uint64_t tag);
/* Withdraw a request that has not been admitted yet: it completes at once
 * (reported by the next pm_server_progress) with status PM_ECANCELED, and
 * nothing is written to its output.  A request already admitted to the GPU
 * runs to completion; for it, and for an unknown tag, the call returns
 * PM_EINVAL.  Only the first queued request with the tag is withdrawn. */
int pm_server_cancel(pm_server *srv, uint64_t tag);
/* Reap finished batches, admit and launch queued requests, and return up to
 * `cap` completions.  Never blocks on the device. */
int pm_server_progress(pm_server *srv, pm_server_done *done, uint32_t cap, uint32_t *n_done);
int pm_server_state(pm_server *srv, pm_server_state_t *state);
/* Waits for work in flight, then frees the server's memory and streams. */
void pm_server_destroy(pm_server *srv);

/* ---- the product without device allocation --------------------------------
 *
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot allocate device memory: code running where cudaMalloc (or any
 * allocator) is forbidden or would synchronise the device, such as a
 * real-time thread, an allocator callback, or a plugin whose host
 * application owns every device allocation.  pm_polymul takes its scratch
 * from the stream-ordered allocator; this entry point takes all of its
 * scratch from a file-scope static device array of PM_NOALLOC_SCRATCH_BYTES
 * that every GPU which loads the library holds until the process exits, and
 * it calls no cudaMalloc, cudaFree or other allocating routine.  It runs one
 * kernel (one CTA) that forms, sorts and reduces all term products, so it is
 * meant for small products only.
 *
 * Arguments, results and error codes are those of pm_polymul (without
 * options or statistics), with these limits: n_f, n_g <= PM_NOALLOC_MAX_TERMS
 * and n_f * n_g <= PM_NOALLOC_MAX_PRODUCTS (raw input sizes); larger inputs
 * fail with PM_EINVAL before any work.  The caller allocates the inputs and
 * the outputs.
 *
 * The first call on a device looks up the device address of the static
 * array (cudaGetSymbolAddress) with that device current and keeps it for the
 * life of the process; make that first call before any stream capture.  A
 * device reset (cudaDeviceReset) or a switch to another context on the same
 * device after that first call is not supported: the kept address would no
 * longer be valid.  Every call shares the array, which keeps the
 * last call's contents (the kernel clears what must start at zero), so calls
 * whose executions overlap on the GPU race: serialise them.  The call
 * synchronises `stream` before it returns.
 *
 * When several errors apply they are reported in pm_polymul's order: an
 * input exponent at its guard bit, then a repeated input monomial whose
 * int64 sum overflows, then a product exponent at its guard bit, then the
 * int128 bound rule, then the capacity. */
#define PM_NOALLOC_MAX_TERMS     4096u
#define PM_NOALLOC_MAX_PRODUCTS  65536u
#define PM_NOALLOC_SCRATCH_BYTES (4u << 20)

int pm_polymul_noalloc(const pm_packing *pk, int coef_kind, const pm_terms_in *f, const pm_terms_in *g,
                       pm_terms_out *h, void *stream);

/* Human-readable message for an error code (static storage). */
const char *pm_strerror(int code);

/* Library version: major * 10000 + minor * 100 + patch. */
int pm_version(void);

#ifdef __cplusplus
}
#endif
#endif
