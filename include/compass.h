/*
 * compass.h -- C ABI of libcompass: GB300 (sm_103a) Fast-AGMS sketch build with
 * push-down selection, and the sketch-merging join-size estimate of COMPASS
 * (Izenov, Datta, Rusu, Shin, "COMPASS: Online Sketch-based Query Optimization for
 * In-Memory Databases", arXiv 2102.02440).
 *
 * Conventions shared by every entry point:
 *  - Pointers named *_dev are CUDA device memory owned by the caller; *_host are host
 *    memory owned by the caller.  The library never allocates device memory and never
 *    frees caller memory.  Workspaces are passed in by the caller, sized by the
 *    matching *_bytes query.
 *  - `stream` is a cudaStream_t (0 = legacy default stream).  Every device call is
 *    asynchronous on it; nothing synchronises unless stated.
 *  - Argument errors are detected on the host, before any launch, and returned as
 *    CMP_EINVAL (nothing is enqueued).  Conditions only the device can see (an int128
 *    estimate that overflows, a bounded wait that ran out) are written to *status_dev
 *    (first error wins; the caller zeroes it).  A failed launch returns CMP_ECUDA.
 *  - No call aborts the process or throws across the ABI.
 */
#ifndef COMPASS_H
#define COMPASS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t cmp_status;
#define CMP_OK 0
#define CMP_EINVAL (-1)       /* bad argument (host-detected, nothing enqueued)       */
#define CMP_EUNSUPPORTED (-2) /* valid input this version does not handle             */
#define CMP_EOVERFLOW (-3)    /* an exact integer result left its representation      */
#define CMP_ECUDA (-4)        /* a CUDA call or kernel launch failed                  */
#define CMP_EWORKSPACE (-5)   /* workspace or plan buffer smaller than required       */
#define CMP_ETIMEOUT (-6)     /* a bounded device-side wait ran out                   */

#define CMP_MAX_COLS 32       /* columns per table descriptor     */
#define CMP_MAX_PREDS 8       /* conjuncts per table              */
#define CMP_MAX_SKETCHES 16   /* sketches (join edges) per table  */
#define CMP_MAX_D 64          /* sketch rows                      */
#define CMP_MAX_W (1 << 20)   /* buckets per sketch row           */
#define CMP_MAX_TABLES 64     /* tables per join graph (sub-plan masks are uint64) */

enum { CMP_I32 = 0, CMP_I64 = 1 };                       /* column element types */
enum { CMP_RANGE = 0, CMP_EQ = 1, CMP_IN_BITMAP = 2 };  /* predicate operators  */

/* One column: `data` is a device pointer to n_rows elements of `dtype`.  `flags`
 * declares what the caller knows about a key column, as a catalog would; both are
 * performance hints, and the sketches are the same whether they hold or not:
 *   CMP_COL_UNIQUE  the values are distinct (a primary key).  The batched build hashes
 *                   the column once per surviving row with the counters in shared memory
 *                   (no per-key counting, which cannot merge anything here).
 *   CMP_COL_DOMAIN  the values lie in [dom_lo, dom_hi) (e.g. a foreign key's referenced
 *                   key range).  Key aggregation sizes its count array to that range.  If
 *                   a surviving value lies outside it, the column is hashed per row in
 *                   the same build. */
#define CMP_COL_UNIQUE 1
#define CMP_COL_DOMAIN 2
typedef struct {
  const void* data;
  int32_t dtype;
  int32_t flags;   /* CMP_COL_UNIQUE | CMP_COL_DOMAIN, or 0 */
  int64_t dom_lo;  /* CMP_COL_DOMAIN: first value of the declared range */
  int64_t dom_hi;  /* CMP_COL_DOMAIN: one past its last value */
} cmp_col;

/* One conjunct of a table's selection (Sec. 2, "Partitioned query execution": the
 * selection is pushed down and only satisfying tuples update the sketches; Sec. 1 names
 * point, subset and range predicates).  Values are compared as int64 (int32 columns are
 * sign-extended):  CMP_RANGE keeps lo <= v < hi;  CMP_EQ keeps v == lo;  CMP_IN_BITMAP
 * keeps 0 <= v < bitmap_nbits with bit v set in `bitmap` (device, uint32 words, bit v is
 * bit (v & 31) of word v >> 5) -- subset and LIKE predicates resolved to codes. */
typedef struct {
  int32_t col;
  int32_t op;
  int64_t lo;
  int64_t hi;
  const uint32_t* bitmap;
  int64_t bitmap_nbits;
} cmp_pred;

/* Hash parameters of one (edge, sketch row): Carter-Wegman polynomials over the prime
 * p = 2^61 - 1 (the paper asks for a per-row bucket hash h and a 4-wise independent
 * +-1 family xi, Sec. 3.1-3.2, without naming one).  With x = key mod p in [0, p):
 *   h(x)  = ((a x + b) mod p) mod w,
 *   xi(x) = +1 if (c3 x^3 + c2 x^2 + c1 x + c0) mod p is even, else -1.
 * All fields are < p and a != 0. */
typedef struct {
  uint64_t a, b, c0, c1, c2, c3;
} cmp_hash;

/* A base table with its pushed-down selection and its attribute-level sketches: one
 * sketch per join edge the table takes part in, each on the key column of that join
 * (Sec. 2 "Workflow": two joins on the same attribute get two independent sketches).
 * All arrays here are HOST arrays; the pointers inside cmp_col / cmp_pred are device
 * pointers. */
typedef struct {
  int64_t n_rows;           /* 0 .. 2^31 - 1 (int32 counters, Sec. 6.1)          */
  int32_t n_cols;           /* 0 .. CMP_MAX_COLS                                   */
  int32_t n_preds;          /* 0 .. CMP_MAX_PREDS (conjunction; 0 = keep all)      */
  int32_t n_sketches;       /* 0 .. CMP_MAX_SKETCHES                               */
  int32_t reserved;
  const cmp_col* cols;      /* [n_cols]                                            */
  const cmp_pred* preds;    /* [n_preds]                                           */
  const int32_t* key_col;   /* [n_sketches] column index holding the join key      */
  const int32_t* edge_id;   /* [n_sketches] join-graph edge of the sketch          */
  uint64_t sample_seed;     /* row sample, see below                               */
  double sample_rate;       /* 0 or 1: every row; in (0, 1): a Bernoulli sample    */
} cmp_table;

/* Row sample (Sec. 2 "Workflow": sketches may be built over a sample only, trading
 * accuracy for time).  With sample_rate p in (0, 1), row r (0-based, of the whole table)
 * takes part in the selection only if output r of SplitMix64 (Steele, Lea & Flood 2014)
 * seeded with sample_seed, z = sample_seed + (r + 1) * 0x9E3779B97F4A7C15 mixed by the
 * generator's finaliser, is below floor(p * 2^64) (at least 1): one independent trial per
 * row, computed from r alone, so every launch shape and both builds sample the same rows.
 * The survivor count is then the number of sampled rows that satisfy the predicates.
 * Sample tables with different seeds; the estimates scale back with cmp_graph.sample_rate
 * and cmp_part_join.sample_rate. */

/* Build launch shape.  Zero / negative fields mean "choose automatically" (the
 * autotuned table when one is loaded, else a size heuristic). */
typedef struct {
  int32_t mode;           /* 0 auto, 1 shared-memory private counters, 2 L2-resident global counters */
  int32_t pairs_per_slab; /* (sketch, row) pairs a CTA privatises in mode 1                          */
  int32_t threads;        /* threads per CTA (multiple of 32, <= 1024)                              */
  int32_t tile_rows;      /* rows per tile (multiple of 128, <= 16384)                              */
  int32_t dedupe;         /* -1 auto, 0 off, 1 aggregate equal keys of a tile before hashing        */
  int32_t ctas_per_sm;    /* CTAs per SM the grid is sized for                                      */
  int32_t aggregate;      /* batched build only: -1 auto (tables of >= 2^18 rows), 0 off, 1 every
                             table: aggregate each key column's survivors per distinct key before
                             hashing (needs dedupe; same counters)                                  */
  int32_t unique;         /* batched build only: 0 or 1 on, -1 off: key columns declared
                             CMP_COL_UNIQUE are hashed once per row with shared-memory counters  */
} cmp_build_cfg;

/* ---------------------------------------------------------------------- general */

/* Version of this interface (CMP_ABI_VERSION); bindings refuse a library that differs. */
#define CMP_ABI_VERSION 7
int32_t cmp_abi_version(void);
const char* cmp_status_str(cmp_status s);

/* Draws the hash parameters of every (edge, row), host only.  SplitMix64 (Steele, Lea &
 * Flood 2014) seeded with `seed`, consumed in the order edge ascending, row ascending,
 * fields a, b, c0, c1, c2, c3; each field is the output's top 61 bits, p itself maps to
 * 0, and a = 0 becomes 1.  out_host: [n_edges * d], entry e*d + i.  Both endpoint
 * tables of an edge use that edge's parameters (Sec. 3.1: the two sketches of a join
 * share their random functions). */
cmp_status cmp_hash_params(uint64_t seed, int32_t n_edges, int32_t d, cmp_hash* out_host);

/* ----------------------------------------------------------------- sketch build */

/* Push-down selection fused with the Fast-AGMS update (Sec. 2 "Partitioned query
 * execution"; Sec. 3.2 "Fast-AGMS Sketches": for every tuple satisfying the selection
 * and every row i of every sketch of the table, C[s][i][h_i(key)] += xi_i(key)).
 *   hash_dev      [n_edges * d] parameters (from cmp_hash_params, copied to the device)
 *   counters_dev  [n_sketches][d][w] int32, overwritten (zeroed, then built)
 *   survivors_dev one int64, overwritten with the exact number of selected tuples
 *   status_dev    one int32 device status word (0 = OK)
 *   cfg           NULL or a launch shape
 * d in 1..CMP_MAX_D, w in 1..CMP_MAX_W.  Counters are int32 and wrap-exact; tables with
 * more than 2^31 - 1 rows are rejected (CMP_EINVAL).  Results are identical for every
 * launch shape.  Enqueues a memset and one kernel on `stream`. */
cmp_status cmp_sketch_build(const cmp_table* table, int32_t d, int32_t w, const cmp_hash* hash_dev,
                            int32_t n_edges, int32_t* counters_dev, int64_t* survivors_dev,
                            int32_t* status_dev, const cmp_build_cfg* cfg, void* stream);

/* Batched build (all attribute-level sketches of every table of a query, or of many
 * queries, in ONE persistent build launch; Sec. 2: every table's selection and sketches
 * are built in the same push-down pass, and per-worker partial sketches merge by addition,
 * Sec. 2 "Sketches").  Two host steps encode a plan, the caller copies it to the
 * device (any H2D copy), then cmp_sketch_build_batched enqueues a zeroing kernel and the
 * build kernel reading it.  The plan holds device pointers, so it stays valid as long as
 * the columns and outputs do; it can be replayed and captured in a CUDA graph.
 *   counters_dev_host  host array [n_tables] of device pointers, each [n_sketches][d][w]
 *   survivors_dev      device [n_tables] int64
 *   ws_dev, ws_bytes   device workspace of at least the *ws_bytes cmp_build_plan_bytes
 *                      reports (0 when no key column is aggregated; NULL allowed then),
 *                      caller-owned, contents irrelevant between calls
 * Key aggregation (cfg->aggregate): the survivors of each key column of a large table
 * that is not declared unique are first counted per distinct key, then each distinct key
 * is hashed once per (sketch, row) with its count as the multiplier.  The count array
 * covers the column's declared domain (CMP_COL_DOMAIN, at most 2^27 values), else the
 * power of two at or above min(rows, 2^27), indexed by the key modulo its size; the
 * counting pass also finds the surviving keys' range.  The update is linear and the
 * counters wrap exactly, so the result is bit-identical to one update per tuple; a column
 * whose surviving keys span more values than its array (or leave its declared domain)
 * falls back to the per-row path in the same build.  Key columns declared unique
 * (CMP_COL_UNIQUE, cfg->unique) are hashed once per surviving row by a kernel that keeps
 * one or more (sketch, row) pairs' counters in shared memory: int32, or two 16-bit halves
 * per word with every carry and borrow added to the global counter, so the counters stay
 * exact.  A unique column with a declared domain of at most 2^32 keys, at most four
 * times the table's rows, in a table without predicates or sample, is instead marked in a
 * presence bitmap over its domain by the counting pass and hashed in key order: every
 * (sketch, row) pair walks runs of consecutive keys, advancing h's and xi's residues by
 * finite differences (additions mod p, the same integers as evaluating the polynomials);
 * a key outside the domain, or one seen twice, sends the column to the per-row path.
 * Launches: zeroing, then (when present) clearing + counting, the unique-key kernel, the
 * row kernel, the hashing of the counted keys and the presence-bitmap kernel.
 * cmp_build_plan_encode returns CMP_EWORKSPACE if plan_bytes is too small;
 * cmp_sketch_build_batched returns CMP_EWORKSPACE if ws_bytes is. */
cmp_status cmp_build_plan_bytes(const cmp_table* tables, int32_t n_tables, int32_t d, int32_t w,
                                const cmp_build_cfg* cfg, size_t* plan_bytes, size_t* ws_bytes);
cmp_status cmp_build_plan_encode(const cmp_table* tables, int32_t n_tables, int32_t d, int32_t w,
                                 int32_t n_edges, int32_t* const* counters_dev_host, int64_t* survivors_dev,
                                 const cmp_build_cfg* cfg, void* plan_host, size_t plan_bytes);
cmp_status cmp_sketch_build_batched(const void* plan_host, const void* plan_dev, const cmp_hash* hash_dev,
                                    void* ws_dev, size_t ws_bytes, int32_t* status_dev, void* stream);

/* Counts of an encoded batched-build plan (host only, no GPU): tables, aggregated key
 * columns (presence bitmaps included), unique-key slabs and items and that kernel's grid,
 * the row kernel's grid, the workspace, the number of kernels one cmp_sketch_build_batched
 * call enqueues, and the presence-bitmap columns among the aggregated ones.
 * CMP_EINVAL for a NULL argument or a blob that is not a build plan. */
typedef struct {
  int32_t n_tables, n_agg, n_unique_slabs, unique_grid;
  int64_t n_unique_items, row_grid, ws_bytes;
  int32_t launches, n_presence;
} cmp_build_plan_info;
cmp_status cmp_build_plan_stats(const void* plan_host, cmp_build_plan_info* info);

/* ------------------------------------------------------------------- estimation */

/* Presort of sketch rows by magnitude (prepares the merged contraction of Sec. 4.2: the
 * merged value of a bucket tuple is the operand of minimum |.|, so every sum over a
 * merged sketch splits into sums over buckets above / below a magnitude threshold).
 * For each of the n_rows rows of length w in counters_dev (row-major), writes the
 * bucket permutation that sorts the row by (|C|, bucket index) ascending into perm_dev
 * and the sorted magnitudes into abs_sorted_dev (both [n_rows][w]).  Rows with
 * w <= 16384 are sorted in shared memory and need no workspace; longer rows are sorted
 * in chunks and merged in global memory, 64 rows at a time, in ws_dev of
 * cmp_presort_ws_bytes(n_rows, w) bytes (CMP_EWORKSPACE if smaller). */
size_t cmp_presort_ws_bytes(int64_t n_rows, int32_t w);
cmp_status cmp_presort(const int32_t* counters_dev, int64_t n_rows, int32_t w, uint32_t* abs_sorted_dev,
                       int32_t* perm_dev, void* ws_dev, size_t ws_bytes, void* stream);

/* Cross ranks between the sorted rows of one table's sketches (prepares the merged
 * contraction, like cmp_presort; independent of any sub-plan, so every sub-plan that
 * contains the table reuses them -- the paper caches merged sketches and products for
 * the same reason, Sec. 5).  For a table with k sketches on edges edge_id_host[0..k),
 * with abs_sorted_dev / perm_dev its [k][d][w] presort outputs, writes ranks_dev
 * [k][k][d][w] int32:  for x != y, ranks[x][y][i][r] = the number of buckets j of row i
 * of sketch y whose |C_y[i][j]| is < abs_x[i][r], or <= it when edge_id[y] < edge_id[x];
 * on the diagonal, ranks[x][x][i][j] = the sorted position of bucket j (the inverse of
 * perm).  d counts rows only (k * k * d < 2^31): with k = 1, the rows of many one-sketch
 * tables stored back to back can be processed in one call. */
cmp_status cmp_cross_ranks(const uint32_t* abs_sorted_dev, const int32_t* perm_dev, int32_t k, int32_t d, int32_t w,
                           const int32_t* edge_id_host, int32_t* ranks_dev, void* stream);

/* cmp_cross_ranks of n_tables tables in one launch.  Table t has k_host[t] sketches (0 to
 * CMP_MAX_SKETCHES) and owns, in order, the next k_t * d presorted rows of abs_sorted_dev /
 * perm_dev and the next k_t * k_t * d * w int32 of ranks_dev; edge_ids_host holds the
 * tables' edge ids back to back (sum of k_t entries).  Results equal one cmp_cross_ranks
 * call per table.  CMP_EINVAL for bad sizes or a total of CTAs (sum k_t^2 d) >= 2^31. */
cmp_status cmp_cross_ranks_multi(const uint32_t* abs_sorted_dev, const int32_t* perm_dev, int32_t n_tables,
                                 const int32_t* k_host, const int32_t* edge_ids_host, int32_t d, int32_t w,
                                 int32_t* ranks_dev, void* stream);

/* A join graph whose sketches have been built and presorted.  Edge e joins tables
 * edge_u[e] and edge_v[e]; endpoint 0 is the edge_u side, 1 the edge_v side.  All
 * arrays are HOST arrays; entries of sketch/abs_sorted/perm are DEVICE pointers to the
 * endpoint's [d][w] sketch (int32), sorted magnitudes (uint32) and permutation (int32),
 * and ranks points into its table's cross-rank array. */
typedef struct {
  int32_t n_tables;                  /* 1 .. CMP_MAX_TABLES */
  int32_t n_edges;
  const int32_t* edge_u;             /* [n_edges] */
  const int32_t* edge_v;             /* [n_edges] */
  const int32_t* const* sketch;      /* [2 * n_edges] */
  const uint32_t* const* abs_sorted; /* [2 * n_edges] */
  const int32_t* const* perm;        /* [2 * n_edges] */
  const int32_t* const* ranks;       /* [2 * n_edges]: the endpoint table's cmp_cross_ranks block of this sketch,
                                        ranks_dev + x * k * d * w for the endpoint's sketch index x of its
                                        table's k sketches */
  const int32_t* slot;               /* [2 * n_edges]: the endpoint's sketch index x within its table (host) */
  const int64_t* survivors_dev;      /* device [n_tables]: exact selected counts */
  const double* sample_rate;         /* NULL, or [n_tables] the rate each table's sketches were built at
                                        (cmp_table.sample_rate: 0 or 1 = unsampled, else in (0, 1)) */
} cmp_graph;

/* Estimates of many sub-plans, possibly of many graphs, in one launch sequence
 * (Sec. 5, Alg. 1 calls the estimate for every enumerated sub-plan; Sec. 4.2 composes the
 * attribute-level sketches of the sub-plan's joins by merging).  Sub-plan q is table set
 * sub_mask[q] (bit t = table t) of graph sub_graph[q]; it must be connected in the graph
 * induced by its tables (cross products are excluded, Sec. 2 "Plan enumeration"), else
 * CMP_EINVAL.  Its edges are every edge with both ends in the set.
 *   |S| = 1: the estimate is the exact selected count (push-down, Sec. 2).
 *   |S| >= 2: for every sketch row i, the exact integer
 *       E_i = sum over all bucket assignments j of the sub-plan's edges of
 *             prod over tables t of M_t(j restricted to t's edges),
 *     where M_t is t's merged sketch: the value of the sketch (among t's sketches of
 *     the sub-plan's edges, in ascending edge id) whose bucket has the minimum |value|,
 *     the first such on ties (the merge equation of Sec. 4.2, iterated).  For one edge
 *     this is the Fast-AGMS inner product of Sec. 3.2.  The estimate is the median of
 *     E_0..E_{d-1} (Sec. 3.2), exact, rounded once to double (even d: mean of the two
 *     middle values).  A sub-plan with rho independent cycles (edges - tables + 1) is
 *     evaluated by conditioning on the buckets of rho non-tree edges, w^rho tree
 *     contractions per row; rho > 3, or w^rho > 2^31 - 1, returns CMP_EUNSUPPORTED from
 *     the plan step.
 *   Sampled tables (sample_rate): the estimate (the median, or the selected count of a
 *     single table) is multiplied by the sub-plan's scale, the product over its tables in
 *     ascending order of 1 / rate (double, left to right), which makes the two-way
 *     estimate unbiased over the independent samples; row_est stays the exact integers of
 *     the sampled sketches.
 * Host steps: cmp_estimate_plan_bytes sizes the plan and the device workspace, and
 * cmp_estimate_plan_encode writes the plan; the caller copies it to the device.  Then
 * cmp_estimate enqueues the launches.
 *   est_dev      [n_sub] double
 *   row_est_dev  NULL or [n_sub][d][2] int64: each exact row estimate as a little-endian
 *                two's-complement int128 (low word first); unspecified for the rows of a
 *                sub-plan that has a row beyond int128 (see below)
 * Exact range.  Rows are evaluated in int128 (int64 storage where it suffices).  A row whose
 * value, or an intermediate value of its evaluation, leaves int128 is evaluated again,
 * exactly, by a second tier (the sub-plan's other rows keep their int128 values): on the
 * generic path, one unit per conditioning chunk, modulo 16 primes p_j = 2^62 - c_j, and in
 * double on magnitudes rounded upwards (a bound B on |E|); when B < 2^990 (below half the
 * primes' product) the row is the unique integer with those residues (Garner's algorithm),
 * and est is the exact median of the rows rounded once.  est is NaN and the status gets
 * CMP_EOVERFLOW only when B >= 2^990, or when more than min(n_sub d, 2^19) rows, or more
 * than min(d x the plan's conditioning chunks, 2^20) units, of one call need the tier.
 * Flag CMP_EST_NO_WIDE turns the tier off (rows beyond int128 are then NaN with
 * CMP_EOVERFLOW). */
/* Estimate launch shape; zero fields choose automatically.
 * Sub-plans whose only cycle is a triangle, with every other table a leaf of one of its
 * three tables, are evaluated by the triangle path: the conditioned sum regrouped as
 * batched dominance sums, O(w G log w) per sketch row for G distinct clamp ranks, instead
 * of one tree contraction per conditioning value (O(w^2)).  Both give the same exact
 * integers.  It needs w <= 16384; flag CMP_EST_GENERIC_ONLY turns it off.
 * Flag CMP_EST_CACHE_MESSAGES: incremental evaluation of tree sub-plans (Sec. 4.2: an
 * (n+1)-D merged sketch extends an n-D one; Sec. 5: merged sketches cached across the
 * enumerated sub-plans).  Each tree sub-plan is rooted at its lowest table id; a child
 * subtree T joined to the rest by edge e sends one message over e, the contraction of T's
 * merged sketches with its sketch on e, which depends on (graph, e, T) alone.  Messages
 * referenced by two or more sub-plans or larger subtrees are computed once per sketch row,
 * level by level (smaller subtrees first), into the workspace (16 bytes per bucket and
 * row), and every user reads them there.  The estimates and row estimates are the same
 * exact integers as without the flag. */
#define CMP_EST_GENERIC_ONLY 1
#define CMP_EST_CACHE_MESSAGES 2
/* Flag CMP_EST_STAR_LATTICE: sub-plans made of one root table joined to leaves only, grouped
 * by (graph, root) with K >= 3 leaf edges U over the family, are evaluated for all leaf
 * subsets at once (Sec. 5: products of sketches cached across the enumeration's
 * sub-plans).  In sketch row i a star over leaf set S has the exact row estimate
 * sum_{a in S} T_a(S minus a), where T_a(V) = sum_r w_a(r) prod_{b in V} f_ab(r) over a's
 * sorted order, w_a the root-times-leaf products and f_ab the leaf suffix sums at the cross
 * ranks: the same sum as the merged contraction, regrouped.  T_a is computed for every V as
 * an exact int128 product of two tables over r (2^(K-1) entries per edge and row, 17 bytes
 * each, in the workspace), then each star gathers |S| entries.  A family is planned this way
 * when K 2^(K-1) <= 2 sum_S |S|^2 over its requested stars (it is dense enough); other
 * sub-plans are planned as without the flag.  Rows that stay in int128 are the same exact
 * integers; a row where an intermediate value left int128 is passed to the exact tier
 * (cmp_estimate, "Exact range").  When enough rows of one (family, sketch row) reach it
 * (count x 3K >= 2^(K+1)), the tier evaluates the family's lattice again modulo each prime
 * they need and as a magnitude bound, and sums each row's entries; otherwise it evaluates
 * the rows on the generic path.  Either way the rows are the same exact integers. */
#define CMP_EST_STAR_LATTICE 4
#define CMP_EST_NO_WIDE 8
typedef struct {
  int32_t threads;     /* threads per CTA (multiple of 32, <= 1024)                */
  int32_t ctas_per_sm; /* resident CTAs per SM the persistent grid is sized for    */
  int32_t cond_chunk;  /* conditioning values per work item of a cyclic sub-plan   */
  int32_t flags;       /* CMP_EST_GENERIC_ONLY | CMP_EST_CACHE_MESSAGES | CMP_EST_STAR_LATTICE |
                          CMP_EST_NO_WIDE; other bits: CMP_EINVAL */
} cmp_estimate_cfg;

cmp_status cmp_estimate_plan_bytes(const cmp_graph* graphs, int32_t n_graphs, int32_t d, int32_t w, int32_t n_sub,
                                   const int32_t* sub_graph, const uint64_t* sub_mask, const cmp_estimate_cfg* cfg,
                                   size_t* plan_bytes, size_t* ws_bytes);
cmp_status cmp_estimate_plan_encode(const cmp_graph* graphs, int32_t n_graphs, int32_t d, int32_t w, int32_t n_sub,
                                    const int32_t* sub_graph, const uint64_t* sub_mask, const cmp_estimate_cfg* cfg,
                                    void* plan_host, size_t plan_bytes);
cmp_status cmp_estimate(const void* plan_host, const void* plan_dev, void* ws_dev, size_t ws_bytes, double* est_dev,
                        int64_t* row_est_dev, int32_t* status_dev, void* stream);
/* cmp_estimate with every exact row as a wide integer: wide_rows_dev NULL or
 * [n_sub][d][16] int64, each row a little-endian two's-complement 1024-bit integer (16
 * limbs), including the rows the exact tier computed (unspecified for a sub-plan whose
 * estimate is NaN). */
cmp_status cmp_estimate_ex(const void* plan_host, const void* plan_dev, void* ws_dev, size_t ws_bytes, double* est_dev,
                           int64_t* row_est_dev, int64_t* wide_rows_dev, int32_t* status_dev, void* stream);

/* Counts of an encoded estimate plan (host only, no GPU): sub-plans, work items (one per
 * sketch row and conditioning chunk), table operations over all sub-plans and cached
 * messages (each evaluated once per item of its owner), cached subtree messages
 * (CMP_EST_CACHE_MESSAGES) with their items and launch levels, triangle sub-plans, and the
 * persistent grid.  CMP_EINVAL for a NULL argument or a blob that is not an estimate plan. */
typedef struct {
  int64_t n_sub, n_items, n_ops, n_jobs, n_job_items, n_tri;
  int32_t n_levels, grid;
  int64_t n_star, n_star_sub, n_star_entries; /* star families, their sub-plans, lattice entries */
} cmp_estimate_plan_info;
cmp_status cmp_estimate_plan_stats(const void* plan_host, cmp_estimate_plan_info* info);

/* ------------------------------------------------------- partitioned sketches */
/* Sketch partitioning (Sec. 4.1): the unbiased estimator of a fixed multi-way join.  A
 * table that joins through edges e_1..e_k gets, per sketch row i, a k-dimensional tensor
 * of width[e_1] x ... x width[e_k] int32 counters (axis l for edge e_l, row-major: the last
 * axis is contiguous; layout [d][prod of its widths]).  Every tuple that satisfies the
 * table's selection adds xi_{e_1,i}(key_1) * ... * xi_{e_k,i}(key_k) to the counter at
 * (h_{e_1,i}(key_1), ..., h_{e_k,i}(key_k)), where h and xi are the (edge, row) functions of
 * cmp_hash with the edge's own width, which both endpoint tables of an edge use.  A one-axis
 * tensor is the 1-D sketch of cmp_sketch_build; a zero-axis tensor holds the selected count.
 * Unlike merged 1-D sketches, the tensors serve only the join they were built for. */
#define CMP_PART_MAX_AXES 4
#define CMP_PART_MAX_SIZE 2147483647LL /* counters per tensor row */

/* Build launch shape; zero fields choose automatically. */
typedef struct {
  int32_t mode;         /* 0 auto, 1 shared-memory private tensors, 2 L2-resident global counters */
  int32_t rows_per_cta; /* sketch rows a CTA updates (mode 1: rows whose tensors it privatises)   */
  int32_t threads;      /* threads per CTA (multiple of 32, <= 1024)                              */
  int32_t tile_rows;    /* rows per tile (multiple of 128, <= 16384)                              */
  int32_t ctas_per_sm;  /* CTAs per SM the grid is sized for                                      */
  int32_t reserved;
} cmp_part_build_cfg;

/* Builds the partitioned sketch of one table.  Its axes are the table's sketches in order:
 * axis l joins on edge table->edge_id[l] with key column table->key_col[l] (distinct edges,
 * 0 .. CMP_PART_MAX_AXES of them).
 *   width_host    [n_sketches] buckets per axis, 1 .. CMP_MAX_W, product <= CMP_PART_MAX_SIZE
 *   hash_dev      [n_edges * d] parameters (cmp_hash_params)
 *   counters_dev  [d][prod width_host] int32, overwritten
 *   survivors_dev one int64, overwritten with the exact selected count
 * Counters are int32 and wrap-exact; results are identical for every launch shape.  Enqueues
 * two memsets and one kernel on `stream`. */
cmp_status cmp_part_build(const cmp_table* table, int32_t d, const int32_t* width_host, const cmp_hash* hash_dev,
                          int32_t n_edges, int32_t* counters_dev, int64_t* survivors_dev,
                          const cmp_part_build_cfg* cfg, void* stream);

/* A tree-shaped join over partitioned sketches (host arrays; tensor entries are device
 * pointers).  The edges form a spanning tree of the tables, and table t's axes are exactly
 * its incident edges, in the order of its tensor. */
typedef struct {
  int32_t n_tables;               /* 1 .. CMP_MAX_TABLES                                   */
  int32_t n_edges;                /* n_tables - 1                                          */
  const int32_t* edge_u;          /* [n_edges]                                             */
  const int32_t* edge_v;          /* [n_edges]                                             */
  const int32_t* width;           /* [n_edges] buckets of each edge                        */
  const int32_t* n_axes;          /* [n_tables]                                            */
  const int32_t* axis_edge;       /* table 0's axes, then table 1's, ... (sum n_axes)      */
  const int32_t* const* tensor;   /* [n_tables] device [d][prod of the table's widths]     */
  const double* sample_rate;      /* NULL, or [n_tables] build sample rates (as cmp_graph)  */
} cmp_part_join;

/* Estimate of the join (Sec. 4.1): per sketch row i the exact integer
 *   E_i = sum over all bucket assignments j of the edges of prod over tables t of T_t[i][j|t],
 * the full contraction of the tables' tensors (for the chain k - mk - t, the sum over i, j
 * of sk_k[i] sk_part(mk)[i, j] sk_t[j]); the estimate is the median of E_0..E_{d-1}
 * (Sec. 3.2), rounded once to double (even d: the mean of the two middle values).
 * Evaluation order (it fixes which rows are out of range): the tree is rooted at table 0; a
 * table's message to its parent is its tensor with every child axis contracted, the root's
 * value is its tensor with every axis contracted; a table contracts its child axes one at a
 * time, last axis first, each contraction multiplying every entry by the child's message
 * entry at its index on that axis and summing over the axis; a leaf's message is its own
 * tensor.  Values are int128 and sums are exact; a row where a single product or a value
 * after a contraction leaves int128 has est NaN and CMP_EOVERFLOW in the status.  With
 * sample rates, est is multiplied by the product over the tables, ascending, of 1 / rate
 * (the contraction is linear in every tensor, so this keeps it unbiased).
 *   ws_dev       *ws_bytes from cmp_part_estimate_ws_bytes (intermediate messages), caller-owned
 *   est_dev      one double
 *   row_est_dev  NULL or [d][2] int64: each row value as a little-endian two's-complement
 *                int128 (low word first; unspecified for out-of-range rows)
 * One launch per contracted edge plus one finalize launch (no host synchronisation; can be
 * captured in a CUDA graph).  CMP_EINVAL for a join that is not a tree or whose axes do not
 * match its edges; CMP_EWORKSPACE if ws_bytes is too small. */
cmp_status cmp_part_estimate_ws_bytes(const cmp_part_join* join, int32_t d, size_t* ws_bytes);
cmp_status cmp_part_estimate(const cmp_part_join* join, int32_t d, void* ws_dev, size_t ws_bytes, double* est_dev,
                             int64_t* row_est_dev, int32_t* status_dev, void* stream);

/* cmp_part_estimate with options.  The contraction of long int32 rows streams them through
 * shared memory with bulk copies, each waited for on an mbarrier; a wait that does not see
 * its copy complete within wait_polls polls gives up: the warp writes CMP_ETIMEOUT to the
 * status word, waits (with the default bound) for its copies still in flight, and returns,
 * leaving that launch's outputs incomplete.  wait_polls: -1 the default (2^22 polls, which
 * no healthy copy comes near), 0 .. 2^31-1 a smaller budget (0 gives up at the first wait,
 * to exercise the timeout path).  cfg NULL: as cmp_part_estimate. */
typedef struct {
  int32_t wait_polls;
  int32_t reserved;
} cmp_part_estimate_cfg;
cmp_status cmp_part_estimate_ex(const cmp_part_join* join, int32_t d, void* ws_dev, size_t ws_bytes, double* est_dev,
                                int64_t* row_est_dev, int32_t* status_dev, const cmp_part_estimate_cfg* cfg,
                                void* stream);

/* ------------------------------------------------------ join-order enumeration */
/* Algorithm 1 of Sec. 5 on the estimates of a cmp_estimate run, for every join graph of a
 * batch at once (one thread per graph; the estimates stay on the device).  From every source
 * table in increasing f(v) = alpha card(v) / max card + beta deg(v) / max deg (card = the
 * graph's survivors_dev, deg = join edges at v), a depth-first search extends a left-deep
 * prefix by its neighbours in increasing estimate of the extended sub-plan, prunes a prefix
 * whose cost exceeds the best complete plan's, and ends the source's search after max_plans
 * complete plans.  A plan's cost is the sum of the estimates of its join prefixes of two or
 * more tables (the first table adds nothing).  Ties go to the lower table id; a NaN estimate
 * counts as +inf, a negative one as 0; of equal-cost plans the first found is kept.
 *   sub_graph / sub_mask  the sub-plan list of the cmp_estimate plan whose est_dev is passed:
 *                         est_dev[q] is the estimate of sub_mask[q] in graph sub_graph[q].
 *                         Every connected sub-plan of two or more tables that the search
 *                         reaches must be in it (else +inf and CMP_EUNSUPPORTED in the status).
 *   order_dev   [n_graphs][64] int32: the best plan's tables in join order, -1 after the last
 *               (or everywhere when no plan was found)
 *   cost_dev    [n_graphs] double: its cost (+inf if none)
 *   stats_dev   [n_graphs][3] int64: complete plans reached, prefix extensions, pruned prefixes
 *   ws_dev      the search stacks, *ws_bytes from cmp_enum_plan_bytes (one per graph)
 * A search that exceeds max_nodes prefix extensions stops with CMP_ETIMEOUT in the status
 * (its best plan so far is reported). */
typedef struct {
  double alpha, beta; /* f(v) weights; both 0: 0.5 and 0.5                                */
  int64_t max_plans;  /* complete plans per source: 0 = 10 (the paper's default), -1 = no limit */
  int64_t max_nodes;  /* prefix extensions per graph before the search stops; 0 = 2^26      */
} cmp_enum_cfg;

cmp_status cmp_enum_plan_bytes(const cmp_graph* graphs, int32_t n_graphs, int32_t n_sub, const int32_t* sub_graph,
                               const uint64_t* sub_mask, size_t* plan_bytes, size_t* ws_bytes);
cmp_status cmp_enum_plan_encode(const cmp_graph* graphs, int32_t n_graphs, int32_t n_sub, const int32_t* sub_graph,
                                const uint64_t* sub_mask, void* plan_host, size_t plan_bytes);
cmp_status cmp_enumerate(const void* plan_host, const void* plan_dev, const double* est_dev, const cmp_enum_cfg* cfg,
                         void* ws_dev, size_t ws_bytes, int32_t* order_dev, double* cost_dev, int64_t* stats_dev,
                         int32_t* status_dev, void* stream);

/* ------------------------------------------------------------- learned combiner */
/* Not in the paper, which combines the d row estimates of a sketch by their median
 * (Sec. 3.2).  A 2-layer perceptron over features of the row estimates replaces the
 * median:  y = base + W2 relu(W1 x + b1) + b2,  nin -> nh -> 1, predicting ln(1 + J) / 32
 * for join size J, where base = max(x[skip], 0) if skip >= 0 (a skip connection: with
 * skip = the median row feature, d / 2, the network learns a correction to the median)
 * and 0 if skip = -1.  Parameters are fp32 (the master copy the optimiser updates), laid out
 * W1[nh][nin], b1[nh], W2[nh], b2; every forward and backward pass uses their bfloat16
 * roundings (nearest even) and accumulates in fp32.  nin <= 66, nh <= 64. */

/* Number of parameters, or -1 for unsupported sizes. */
int64_t cmp_mlp_param_count(int32_t nin, int32_t nh);

/* Self-join size estimate of each sketch: f2_dev[s] = median over rows i of
 * sum_j C[s][i][j]^2 (the Fast-AGMS estimator of Sec. 3.2 applied to a sketch with
 * itself), exact per row and rounded once.  counters_dev: [n_sketches][d][w]. */
cmp_status cmp_sketch_f2(const int32_t* counters_dev, int64_t n_sketches, int32_t d, int32_t w, double* f2_dev,
                         void* stream);

/* Features of n estimates: with v the d values sign(E_i) ln(1 + |E_i|) / 32 sorted
 * ascending and m = d / 2, feat_dev[q] (fp32, d + 2 values) = v_i - v_m for i != m, v_m at
 * i = m (the median order statistic itself), then ln(1 + f2a[q]) / 32 and
 * ln(1 + f2b[q]) / 32.  row_est_dev: [n][d][2] int128 row estimates as from cmp_estimate. */
cmp_status cmp_mlp_features(const int64_t* row_est_dev, int64_t n, int32_t d, const double* f2a_dev,
                            const double* f2b_dev, float* feat_dev, void* stream);

/* cmp_mlp_features with the self-join sizes of all sketches in one array: f2a[q] =
 * f2_dev[f2_index_dev[2q]] and f2b[q] = f2_dev[f2_index_dev[2q + 1]], an index of -1 giving
 * 0 (e.g. f2_dev from one cmp_sketch_f2 call over every sketch, f2_index_dev [n][2] int32 the
 * two sketches of each two-table sub-plan, -1 elsewhere).  The indices must be below the
 * length of f2_dev. */
cmp_status cmp_mlp_features_indexed(const int64_t* row_est_dev, int64_t n, int32_t d, const double* f2_dev,
                                    const int32_t* f2_index_dev, float* feat_dev, void* stream);

/* Forward pass: y_dev[s] for the n rows of x_dev ([n][nin] fp32). */
cmp_status cmp_mlp_infer(const float* params_dev, int32_t nin, int32_t nh, int32_t skip, const float* x_dev, int64_t n,
                         float* y_dev, void* stream);

/* Combined estimate of n sub-plans: est_dev[q] = median_dev[q] (the plain median of
 * cmp_estimate) where it is at least one tuple, else max(exp(32 y_dev[q]) - 1, 0) (the
 * network's prediction).  The median stays the estimate wherever it gives a usable join
 * size; the network replaces it where the median row estimate is zero or negative. */
cmp_status cmp_mlp_combine(const double* median_dev, const float* y_dev, int64_t n, double* est_dev, void* stream);

/* The combination with its rule spelled out: est_dev[q] = the network's prediction
 * max(exp(32 y_dev[q]) - 1, 0) where sub-plan q is eligible (eligible_dev NULL: all, else
 * [n] uint8, nonzero = eligible) and its median is below use_median_at, else median_dev[q].
 * use_median_at = 1 is cmp_mlp_combine; +infinity lets the network replace the median on
 * every eligible sub-plan (a NaN median then gives the network's value too); NaN: CMP_EINVAL.
 * Sub-plans the network was not trained on (e.g. of three or more tables) stay on the
 * median by leaving them ineligible. */
cmp_status cmp_mlp_combine_ex(const double* median_dev, const float* y_dev, const uint8_t* eligible_dev, int64_t n,
                              double use_median_at, double* est_dev, void* stream);

/* One full-batch training step on n samples: loss = (1/n) sum (y - t)^2 when
 * huber_delta == 0, else the mean Huber loss (0.5 e^2 for |e| <= delta, delta (|e| -
 * delta / 2) beyond; its linear tails make the fit follow the conditional median), its
 * gradient with respect to the bf16-rounded parameters (summed in a fixed order, so runs
 * are reproducible), then Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with
 * `step` >= 1) on params/adam_m/adam_v (fp32, zero-initialised moments).  loss_dev and
 * grad_dev (the gradient before the update) are optional outputs.  Workspace:
 * cmp_mlp_train_ws_bytes(nin, nh, n) bytes. */
size_t cmp_mlp_train_ws_bytes(int32_t nin, int32_t nh, int64_t n);
cmp_status cmp_mlp_train_step(float* params_dev, float* adam_m_dev, float* adam_v_dev, int32_t nin, int32_t nh,
                              int32_t skip, const float* x_dev, const float* y_dev, int64_t n, float huber_delta,
                              float lr, int32_t step, float* loss_dev, float* grad_dev, void* ws_dev, size_t ws_bytes,
                              void* stream);

/* ------------------------------------------------------------ microbenchmark */
/* The integer roofline of the build's hashing on the GPU at hand: the Carter-Wegman
 * bucket and sign (cmp_hash; Sec. 3.1-3.2 ask for a per-row bucket hash and a 4-wise sign
 * family) of keys 0 .. n_keys-1 for each of the n_pairs parameter sets hash_dev[0..n_pairs)
 * (1..64), with no memory traffic and no counter updates, in the two forms the build uses:
 * form 0 shares the key's powers x^2, x^3 among the pairs (aggregated and int32-slab
 * paths), form 1 evaluates each pair by Horner's rule (packed-slab path).  w: a power of
 * two (the bucket mask).  XORs a checksum of every evaluation into *out_dev (one uint64,
 * device) so that none can be skipped.  n_keys <= 2^31.  Asynchronous on `stream`. */
cmp_status cmp_microbench_cw(const cmp_hash* hash_dev, int32_t n_pairs, int64_t n_keys, int32_t w, int32_t form,
                             uint64_t* out_dev, void* stream);

/* Size of the device workspace built into the library for cmp_estimate_noalloc. */
#define CMP_NOALLOC_WS_BYTES (32u << 20)

/* cmp_estimate without a caller-provided workspace.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory themselves, such as
 * an operator running inside a host engine that owns every device allocation (a
 * database's GPU executor, a serving process with a fixed memory pool), or a latency-
 * critical path that must not call cudaMalloc because it can synchronise the device.
 * Arguments and results are those of cmp_estimate for the same plan.
 *   Workspace: a fixed array of CMP_NOALLOC_WS_BYTES bytes inside the library's device
 *   image, held by every GPU that loads the library until the process exits.  The
 *   library allocates and frees nothing at call time.  The array holds, in this order,
 *   the plan's fixed part (per-item partial sums, and the cached messages and star
 *   lattices of CMP_EST_CACHE_MESSAGES / CMP_EST_STAR_LATTICE), the generic kernel's
 *   per-CTA scratch areas (always at least one), and the scratch of triangle rows (one
 *   row = one triangle sub-plan on one sketch row).  A plan is rejected with
 *   CMP_EWORKSPACE unless fixed part + one CTA scratch area + one triangle row (when the
 *   plan has triangle sub-plans) fit.  Beyond that, the persistent grid shrinks to the
 *   number of CTA scratch areas that fit next to one triangle row, so a large plan runs
 *   with fewer CTAs than cmp_estimate would use, and the triangle rows that do not fit
 *   in the rest run in successive waves of launches on the same stream.
 *   Set-up: the first call on each device looks up the array's device address (with
 *   that device current) and caches it; make that first call before any stream capture.
 *   Sharing: every call, on any stream, uses the same array.  Nothing in it needs to
 *   start at zero (each launch writes what it reads), and it keeps the last call's
 *   contents; calls whose executions overlap on the GPU race on it, so serialise them
 *   (one stream, or events between streams). */
cmp_status cmp_estimate_noalloc(const void* plan_host, const void* plan_dev, double* est_dev, int64_t* row_est_dev,
                                int32_t* status_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* COMPASS_H */
